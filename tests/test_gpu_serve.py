"""The serving loop (pgdto_submit / pgdto_poll): continuous batching over device-resident
design sessions.  Each session's results equal the same steps run alone through a handle
(bit for bit: the same kernels and the same reduction order), the first step also matches
the oracle, admission respects the HBM budget, and a session runs one step at a time."""

import time

import numpy as np
import pytest

from oracle import oracle_step
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _wait(srv, ticket, timeout=60.0):
    from paper_2511_13905_gb300 import binding
    t0 = time.time()
    while True:
        st, done, info = srv.poll(ticket)
        assert st == binding.PGDTO_OK
        if done != binding.PGDTO_ERR_BUSY:
            return done, info
        assert time.time() - t0 < timeout, "request did not complete"
        time.sleep(0.0005)


def _sessions():
    reqs = [{"id": 0, "n": 5000, "m": 1, "mode": "single", "seed": 11},
            {"id": 1, "n": 40000, "m": 2, "mode": "independent", "seed": 12},
            {"id": 2, "n": 12000, "m": 4, "mode": "independent", "seed": 13},
            {"id": 3, "n": 30000, "m": 2, "mode": "coupled", "seed": 14},
            {"id": 4, "n": 70001, "m": 1, "mode": "single", "seed": 15}]
    return [(r, inputs.request_problem(r)) for r in reqs]


def _grads(p, x, k):
    """Sensitivities of step k at design x (synthetic, as the workload recipes)."""
    rng = np.random.default_rng(1000 + k)
    s = rng.lognormal(0.0, 1.0, x.size)
    g = (-3.0 * x.astype(np.float64) ** 2 * s).astype(np.float32)
    if p["mode"] == "independent":
        seg = p["seg"]
        gval = [float(np.sum(x[seg[j]:seg[j + 1]], dtype=np.float64)) for j in range(p["m"])]
    else:
        gval = list(np.atleast_2d(p["A"]).astype(np.float64) @ x.astype(np.float64))
    return g, gval


def test_served_sessions_equal_steps_alone(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    steps = 3
    sess = _sessions()
    srv = binding.Server(budget_bytes=8 << 30, max_sessions=64, engine=2)
    xs = {r["id"]: p["x"].copy() for r, p in sess}
    served = {}
    first_step_inputs = {}
    for k in range(steps):
        tickets = {}
        for r, p in sess:
            g, gval = _grads(p, xs[r["id"]], k)
            if k == 0:
                first_step_inputs[r["id"]] = (g, gval)
            out = np.empty(p["n"], np.float32)
            st, t = srv.submit(r["id"], p["n"], p["m"], g, np.ascontiguousarray(p["A"]), gval, p["G"], out,
                               x0=p["x"] if k == 0 else None, seg=p.get("seg"), close=(k == steps - 1))
            assert st == binding.PGDTO_OK
            tickets[r["id"]] = (t, out)
        for rid, (t, out) in tickets.items():
            done, info = _wait(srv, t)
            assert done == binding.PGDTO_OK, (rid, done)
            xs[rid] = out
            served[(rid, k)] = (out.copy(), list(info.lambda_))
    stats = srv.stats()
    assert stats["steps"] == steps * len(sess) and stats["sessions"] == 0 and stats["bytes_in_use"] == 0
    srv.close()

    # the same steps alone through one handle per session
    for r, p in sess:
        eng = 1 if p["mode"] == "coupled" else 2
        h = binding.Handle(p["n"], p["m"], seg=p.get("seg"), engine=eng)
        h.set_state(None, None, None, 0)
        x = torch.from_numpy(p["x"].copy()).to(dev)
        A = torch.from_numpy(np.ascontiguousarray(p["A"])).to(dev)
        xh = p["x"].copy()
        for k in range(steps):
            g, gval = _grads(p, xh, k)
            st, info = h.step(x, torch.from_numpy(g).to(dev), A, gval, p["G"])
            assert st == 0
            xh = x.cpu().numpy()
            out, lam = served[(r["id"], k)]
            assert np.array_equal(xh, out), (r["id"], k)
            assert lam == list(info.lambda_)
        h.close()

    # and the first step of each session against the oracle
    for r, p in sess:
        g, gval = first_step_inputs[r["id"]]
        ref = oracle_step(p["x"], p["x"], g, np.zeros(p["n"]), np.zeros(p["n"]), p["A"], gval, p["G"], 0,
                          mode=p["mode"], seg=p.get("seg"))
        out, lam = served[(r["id"], 0)]
        if p["mode"] == "independent":
            seg = p["seg"]
            a = p["A"].astype(np.float64)

            def f(x):
                return (np.array([a[seg[j]:seg[j + 1]] @ x[seg[j]:seg[j + 1]] for j in range(p["m"])]),
                        np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(x[seg[j]:seg[j + 1]]) for j in range(p["m"])]))
            err = parity_errors(out, lam[:p["m"]], ref["x_new"], ref["lam"], f, ref["b"], C, 0.0, 1.0,
                                amax=np.ones(p["m"]))
        else:
            err = parity_errors(out, lam[:p["m"]], ref["x_new"], ref["lam"], p["A"], ref["b"], C, 0.0, 1.0)
        assert err["lam_rel"] <= 1e-6 and err["x_abs"] <= 1e-6 and err["viol_rel"] <= 1e-6, (r["id"], err)


def test_admission_budget_and_one_step_per_session(dev):
    from paper_2511_13905_gb300 import binding
    r, p = _sessions()[4]
    g, gval = _grads(p, p["x"], 0)
    out = np.empty(p["n"], np.float32)
    tiny = binding.Server(budget_bytes=1 << 20, max_sessions=4)
    st, _ = tiny.submit(7, p["n"], 1, g, p["A"], gval, p["G"], out, x0=p["x"])
    assert st == binding.PGDTO_ERR_BUSY  # the session would not fit the budget
    tiny.close()
    srv = binding.Server(budget_bytes=1 << 30, max_sessions=1)
    st, t1 = srv.submit(7, p["n"], 1, g, p["A"], gval, p["G"], out, x0=p["x"])
    assert st == binding.PGDTO_OK
    st, _ = srv.submit(7, p["n"], 1, g, p["A"], gval, p["G"], out)
    assert st in (binding.PGDTO_ERR_BUSY, binding.PGDTO_OK)  # busy unless the first step already finished
    out2 = np.empty(p["n"], np.float32)
    st2, _ = srv.submit(8, p["n"], 1, g, p["A"], gval, p["G"], out2, x0=p["x"])
    assert st2 == binding.PGDTO_ERR_BUSY  # session limit
    done, _ = _wait(srv, t1)
    assert done == binding.PGDTO_OK
    srv.close()


def test_wait_blocks_and_stamps_completion(dev):
    """pgdto_wait: blocks until the step is published, returns the same report as a poll
    would, and stamps the completion on the server's clock; a reported or unknown ticket
    is an argument error."""
    from paper_2511_13905_gb300 import binding
    sess = _sessions()
    srv = binding.Server(budget_bytes=8 << 30, max_sessions=64)
    t0 = srv.clock_us()
    tickets = []
    for r, p in sess:
        g, gval = _grads(p, p["x"], 0)
        out = np.empty(p["n"], np.float32)
        st, t = srv.submit(r["id"], p["n"], p["m"], g, np.ascontiguousarray(p["A"]), gval, p["G"], out,
                           x0=p["x"], seg=p.get("seg"))
        assert st == binding.PGDTO_OK
        tickets.append((t, out))
    stamps = []
    for t, out in reversed(tickets):
        st, done, info, t_done = srv.wait(t, timeout_ms=60000)
        assert st == binding.PGDTO_OK and done == binding.PGDTO_OK
        assert np.all(np.isfinite(out)) and info.passes >= 0
        assert t0 <= t_done <= srv.clock_us()
        stamps.append(t_done)
        st, _, _, _ = srv.wait(t, timeout_ms=0)
        assert st == binding.PGDTO_ERR_ARG  # reported once
    st, _, _, _ = srv.wait(123456789, timeout_ms=0)
    assert st == binding.PGDTO_ERR_ARG
    srv.close()


def test_served_equality_session_equals_a_handle(dev):
    """A session whose row is an equality (eq_mask on its first request) gives the same
    step as a handle created with that mask."""
    import torch
    from paper_2511_13905_gb300 import binding
    p = inputs.request_problem({"id": 0, "n": 20000, "m": 1, "mode": "single", "seed": 77})
    g, gval = _grads(p, p["x"], 0)
    G = np.array(gval) + 0.02 * p["n"]  # more volume than now: binds from below as an equality
    srv = binding.Server(budget_bytes=1 << 30, max_sessions=4)
    out = np.empty(p["n"], np.float32)
    st, t = srv.submit(5, p["n"], 1, g, np.ascontiguousarray(p["A"]), gval, G, out, x0=p["x"], eq_mask=1)
    assert st == binding.PGDTO_OK
    st, done, info, _ = srv.wait(t)
    assert st == binding.PGDTO_OK and done == binding.PGDTO_OK
    srv.close()
    h = binding.Handle(p["n"], 1, eq_mask=1)
    h.set_state(None, None, None, 0)
    x = torch.from_numpy(p["x"].copy()).to(dev)
    st, info1 = h.step(x, torch.from_numpy(g).to(dev), torch.from_numpy(np.ascontiguousarray(p["A"])).to(dev), gval, G)
    torch.cuda.synchronize()
    h.close()
    assert st == 0 and info1.lambda_[0] < 0.0
    assert np.array_equal(x.cpu().numpy(), out)
    assert info.lambda_[0] == info1.lambda_[0]


def test_large_coupled_session_in_the_mix_equals_its_run_alone(dev):
    """A coupled session of more than 2^20 variables (four rows) served together with the
    small sessions: its steps equal the same steps run alone through a handle (the same
    grid-engine kernel, bit for bit), and its first step matches the oracle."""
    import torch
    from paper_2511_13905_gb300 import binding
    steps = 2
    big = {"id": 9, "n": (1 << 20) + 3, "m": 4, "mode": "coupled", "seed": 19}
    sess = _sessions() + [(big, inputs.request_problem(big))]
    srv = binding.Server(budget_bytes=16 << 30, max_sessions=64)
    xs = {r["id"]: p["x"].copy() for r, p in sess}
    served = {}
    first = None
    for k in range(steps):
        tickets = {}
        for r, p in sess:
            g, gval = _grads(p, xs[r["id"]], k)
            if k == 0 and r["id"] == big["id"]:
                first = (g, gval)
            out = np.empty(p["n"], np.float32)
            st, t = srv.submit(r["id"], p["n"], p["m"], g, np.ascontiguousarray(p["A"]), gval, p["G"], out,
                               x0=p["x"] if k == 0 else None, seg=p.get("seg"), close=(k == steps - 1))
            assert st == binding.PGDTO_OK
            tickets[r["id"]] = (t, out)
        for rid, (t, out) in tickets.items():
            done, info = _wait(srv, t)
            assert done == binding.PGDTO_OK, (rid, done)
            xs[rid] = out
            served[(rid, k)] = (out.copy(), list(info.lambda_))
    srv.close()
    p = sess[-1][1]
    h = binding.Handle(p["n"], p["m"], engine=1)
    h.set_state(None, None, None, 0)
    x = torch.from_numpy(p["x"].copy()).to(dev)
    A = torch.from_numpy(np.ascontiguousarray(p["A"])).to(dev)
    xh = p["x"].copy()
    for k in range(steps):
        g, gval = _grads(p, xh, k)
        st, info = h.step(x, torch.from_numpy(g).to(dev), A, gval, p["G"])
        assert st == 0
        xh = x.cpu().numpy()
        out, lam = served[(big["id"], k)]
        assert np.array_equal(xh, out), k
        assert lam == list(info.lambda_)
    h.close()
    g, gval = first
    ref = oracle_step(p["x"], p["x"], g, np.zeros(p["n"]), np.zeros(p["n"]), p["A"], gval, p["G"], 0,
                      mode="coupled")
    out, lam = served[(big["id"], 0)]
    err = parity_errors(out, lam[:4], ref["x_new"], ref["lam"], p["A"], ref["b"], C, 0.0, 1.0)
    print("large coupled session, first step vs oracle:", {k: err[k] for k in ("lam_rel", "x_abs", "viol_rel")})
    assert err["lam_rel"] <= 1e-6 and err["x_abs"] <= 1e-6 and err["viol_rel"] <= 1e-6, err


def test_open_then_submit_equals_a_first_submit(dev):
    """pgdto_server_open admits a session and uploads its design without a step; the first
    submit then needs no x0 and gives the same step as a session opened by its first submit.
    Opening twice is an argument error, and the budget applies at open."""
    from paper_2511_13905_gb300 import binding
    r, p = _sessions()[1]
    g, gval = _grads(p, p["x"], 0)
    A = np.ascontiguousarray(p["A"])
    srv = binding.Server(budget_bytes=4 << 30, max_sessions=8)
    assert srv.open(1, p["n"], p["m"], p["x"], seg=p.get("seg")) == binding.PGDTO_OK
    assert srv.open(1, p["n"], p["m"], p["x"], seg=p.get("seg")) == binding.PGDTO_ERR_ARG
    out1 = np.empty(p["n"], np.float32)
    st, t1 = srv.submit(1, p["n"], p["m"], g, A, gval, p["G"], out1, seg=p.get("seg"))
    assert st == binding.PGDTO_OK
    out2 = np.empty(p["n"], np.float32)
    st, t2 = srv.submit(2, p["n"], p["m"], g, A, gval, p["G"], out2, x0=p["x"], seg=p.get("seg"))
    assert st == binding.PGDTO_OK
    for t in (t1, t2):
        st, done, _, _ = srv.wait(t)
        assert st == binding.PGDTO_OK and done == binding.PGDTO_OK
    assert np.array_equal(out1, out2)
    srv.close()
    tiny = binding.Server(budget_bytes=1 << 20, max_sessions=4)
    assert tiny.open(3, p["n"], p["m"], p["x"], seg=p.get("seg")) == binding.PGDTO_ERR_BUSY
    tiny.close()
