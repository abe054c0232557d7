"""Parity of the CUDA path (single row / independent rows) with the FP64 oracle, element by
element, through the C ABI.  Tolerances: lambda relative 1e-6 (floor for inactive rows),
x absolute 1e-6, |a^T x - b| / |b| 1e-6 (oracle.checks.parity_errors)."""

import numpy as np
import pytest

from oracle import oracle_step
from oracle import projection as P
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = {"lam_rel": 1e-6, "x_abs": 1e-6, "viol_rel": 1e-6}


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def T(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def check(err, what=""):
    bad = {k: err[k] for k in TOL if not err[k] <= TOL[k]}
    assert not bad, "%s parity: %s (all: %s)" % (what, bad, {k: err[k] for k in TOL})


def seg_matvec(a, seg):
    a = np.asarray(a, dtype=np.float64)

    def f(x):
        ax = np.array([a[seg[j]:seg[j + 1]] @ x[seg[j]:seg[j + 1]] for j in range(len(seg) - 1)])
        aa = np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(x[seg[j]:seg[j + 1]]) for j in range(len(seg) - 1)])
        return ax, aa
    return f


def seg_amax(a, seg):
    return np.array([max(np.max(np.abs(a[seg[j]:seg[j + 1]])), 1e-30) for j in range(len(seg) - 1)])


# --------------------------------------------------------------------------- projection

def run_project(dev, z, a, b, lo=0.0, hi=1.0, seg=None, offset=0):
    """Project through the C ABI; ``offset`` shifts the arrays inside a larger buffer so the
    pointers are not 16-byte aligned (scalar path)."""
    import torch
    from paper_2511_13905_gb300 import binding
    n = z.size
    m = 1 if seg is None else len(seg) - 1
    h = binding.Handle(n, m, seg=seg, lo=lo, hi=hi)
    if offset:
        zb = torch.zeros(n + offset, dtype=torch.float32, device=dev)
        ab = torch.zeros(n + offset, dtype=torch.float32, device=dev)
        zb[offset:] = T(z, dev)
        ab[offset:] = T(a, dev)
        zt, at = zb[offset:], ab[offset:]
        xb = torch.zeros(n + offset, dtype=torch.float32, device=dev)
        xt = xb[offset:]
    else:
        zt, at = T(z, dev), T(a, dev)
        xt = torch.empty_like(zt)
    st, lam, info = h.project(zt, at, b, xt)
    torch.cuda.synchronize()
    out = xt.cpu().numpy().astype(np.float64)
    h.close()
    return st, np.array(lam), out, info


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 64, 1000, 4097, 100003, 1 << 20])
def test_project_single_sizes(dev, n):
    rng = np.random.default_rng(n)
    z = rng.uniform(-0.3, 1.3, n).astype(np.float32)
    a = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    b = float(a.astype(np.float64) @ np.clip(z, 0, 1).astype(np.float64)) * 0.7
    st, lam, x, info = run_project(dev, z, a, [b])
    assert st == 0, info.status
    lam_ref = P.solve_single_exact(z.astype(np.float64), a.astype(np.float64), b, 0.0, 1.0, C)
    x_ref = np.clip(z.astype(np.float64) - lam_ref * a.astype(np.float64), 0, 1)
    check(parity_errors(x, lam, x_ref, [lam_ref], a[None, :], [b], C, 0.0, 1.0), "n=%d" % n)


@pytest.mark.parametrize("case", ["negative_a", "mixed_sign", "zeros_in_a", "inactive", "infeasible",
                                  "all_zero_a", "wide_box", "unaligned"])
def test_project_single_edge_cases(dev, case):
    rng = np.random.default_rng(hash(case) % 1000)
    n = 3001
    lo, hi = 0.0, 1.0
    z = rng.uniform(-0.5, 1.5, n)
    a = rng.uniform(0.2, 2.0, n)
    frac = 0.6
    offset = 0
    if case == "negative_a":
        a = -a
        frac = 1.4
    elif case == "mixed_sign":
        a = rng.standard_normal(n)
    elif case == "zeros_in_a":
        a[::3] = 0.0
    elif case == "inactive":
        frac = 2.0
    elif case == "infeasible":
        frac = -1.0
    elif case == "all_zero_a":
        a[:] = 0.0
    elif case == "wide_box":
        lo, hi = -2.0, 3.0
        z = rng.uniform(-4, 5, n)
    elif case == "unaligned":
        offset = 1
    z = z.astype(np.float32)
    a = a.astype(np.float32)
    z64, a64 = z.astype(np.float64), a.astype(np.float64)
    base = float(a64 @ np.clip(z64, lo, hi))
    b = base * frac if case != "infeasible" else -10.0
    if case == "all_zero_a":
        b = 1.0
    st, lam, x, info = run_project(dev, z, a, [b], lo, hi, offset=offset)
    assert st == 0, info.status
    lam_ref = P.solve_single_exact(z64, a64, b, lo, hi, C)
    x_ref = np.clip(z64 - lam_ref * a64, lo, hi)
    check(parity_errors(x, lam, x_ref, [lam_ref], a[None, :], [b], C, lo, hi), case)
    if case in ("inactive", "all_zero_a"):
        assert lam[0] == 0.0
        assert np.array_equal(x, np.clip(z64, lo, hi).astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("m,ragged", [(2, False), (3, True), (4, True), (4, False)])
def test_project_independent(dev, m, ragged):
    rng = np.random.default_rng(10 * m + ragged)
    n = 50021 if ragged else 4 * 16384
    if ragged:
        cuts = np.sort(rng.choice(np.arange(1, n), m - 1, replace=False))
        seg = [0] + [int(c) for c in cuts] + [n]
    else:
        seg = [int(v) for v in np.linspace(0, n, m + 1)]
    z = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    a = rng.uniform(0.5, 1.5, n).astype(np.float32)
    z64, a64 = z.astype(np.float64), a.astype(np.float64)
    b = [0.5 * float(a64[seg[j]:seg[j + 1]] @ np.clip(z64[seg[j]:seg[j + 1]], 0, 1)) for j in range(m)]
    if m >= 3:
        b[1] = 1e9  # one inactive row
    st, lam, x, info = run_project(dev, z, a, b, seg=seg)
    assert st == 0, info.status
    lam_ref = P.solve_independent_exact(z64, a64, seg, b, 0.0, 1.0, C)
    x_ref = P.independent_primal(z64, a64, seg, lam_ref, 0.0, 1.0)
    err = parity_errors(x, lam, x_ref, lam_ref, seg_matvec(a, seg), b, C, 0.0, 1.0, amax=seg_amax(a, seg))
    check(err, "m=%d" % m)


def test_project_is_deterministic(dev):
    rng = np.random.default_rng(3)
    n = 300007
    z = rng.uniform(-0.3, 1.3, n).astype(np.float32)
    a = rng.lognormal(0, 1, n).astype(np.float32)
    b = 0.5 * float(a.astype(np.float64) @ np.clip(z, 0, 1))
    outs = [run_project(dev, z, a, [b]) for _ in range(5)]
    for st, lam, x, _ in outs[1:]:
        assert lam[0] == outs[0][1][0]
        assert np.array_equal(x, outs[0][2])


# --------------------------------------------------------------------------- full steps

def run_step(dev, cfg, handle=None, seg=None):
    import torch
    from paper_2511_13905_gb300 import binding
    n, m = cfg["n"], cfg["m"]
    h = handle or binding.Handle(n, m, seg=seg)
    x = T(cfg["x"], dev)
    if cfg["t"] > 0:
        h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    else:
        h.set_state(None, None, None, 0)
    st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], cfg["G"])
    torch.cuda.synchronize()
    out = x.cpu().numpy().astype(np.float64)
    if handle is None:
        h.close()
    return st, info, out


def compare_step(cfg, info, x_dev, mode):
    ref = oracle_step(cfg["x"], cfg.get("x_prev", cfg["x"]), cfg["g"], cfg.get("g_prev", cfg["g"]),
                      cfg.get("d_prev", np.zeros(cfg["n"])), cfg["A"], cfg["gval"], cfg["G"], cfg["t"],
                      mode=mode, seg=cfg.get("seg"))
    m = cfg["m"]
    lam = np.array(list(info.lambda_)[:m])
    assert info.alpha == pytest.approx(ref["alpha"], rel=1e-6)
    assert info.beta == pytest.approx(ref["beta"], rel=1e-6, abs=1e-12)
    if mode == "independent":
        seg = cfg["seg"]
        err = parity_errors(x_dev, lam, ref["x_new"], ref["lam"], seg_matvec(cfg["A"], seg), ref["b"], C,
                            0.0, 1.0, amax=seg_amax(cfg["A"], seg))
    else:
        err = parity_errors(x_dev, lam, ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0)
    check(err, cfg["name"])
    # the stopping ratio of Alg. 3; its error is bounded by ||x_dev - x_ref|| / ||x_ref|| plus
    # the rounding of the two norms, which the device forms from FP32 partial sums
    nrm = float(np.linalg.norm(ref["x_new"]))
    slack = max(1e-5 * ref["rel_change"],
                float(np.linalg.norm(x_dev - ref["x_new"])) / max(nrm, 1e-30) + 1e-6 * ref["rel_change"] + 1e-12)
    assert abs(info.rel_change - ref["rel_change"]) <= slack
    assert np.allclose(np.array(list(info.b)[:m]), ref["b"], rtol=1e-7)
    return ref, err


def test_step_config1_full(dev):
    cfg = inputs.config1()
    st, info, x = run_step(dev, cfg)
    assert st == 0, info.status
    compare_step(cfg, info, x, "single")


@pytest.mark.parametrize("dims", [(8, 4, 4, ), (48, 24, 24), None])
def test_step_config3(dev, dims):
    cfg = inputs.config3(dims=dims)
    st, info, x = run_step(dev, cfg, seg=cfg["seg"])
    assert st == 0, info.status
    compare_step(cfg, info, x, "independent")


def _config2_state_sequence(cfg, steps):
    """The oracle's own trajectory for workload 2 (FP64 steps, FP32 state as a caller would hold it)."""
    n = cfg["n"]
    x = cfg["x"].astype(np.float32)
    x_prev = np.zeros(n, np.float32)
    g_prev = np.zeros(n, np.float32)
    d_prev = np.zeros(n, np.float32)
    seq = []
    for t in range(steps):
        A, gval = inputs.config2_inputs(cfg, x)
        seq.append({"x": x.copy(), "x_prev": x_prev.copy(), "g_prev": g_prev.copy(), "d_prev": d_prev.copy(),
                    "A": A, "gval": gval, "t": t})
        ref = oracle_step(x, x_prev, cfg["g"], g_prev, d_prev, A, gval, cfg["G"], t, mode="single")
        x_prev, g_prev, d_prev = x.copy(), cfg["g"].copy(), ref["d"].astype(np.float32)
        x = ref["x_new"].astype(np.float32)
    return seq


@pytest.mark.parametrize("dims,steps", [((32, 16, 16), 50), (None, 50)])
def test_step_config2_trajectory(dev, dims, steps):
    """Every step of the workload-2 run, fed the oracle's state, against the oracle's step."""
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config2(dims=dims)
    n = cfg["n"]
    h = binding.Handle(n, 1)
    for s in _config2_state_sequence(cfg, steps):
        c = {"name": "%s t=%d" % (cfg["name"], s["t"]), "n": n, "m": 1, "x": s["x"], "x_prev": s["x_prev"],
             "g": cfg["g"], "g_prev": s["g_prev"], "d_prev": s["d_prev"], "A": s["A"], "gval": s["gval"],
             "G": cfg["G"], "t": s["t"]}
        st, info, x = run_step(dev, c, handle=h)
        assert st == 0, (s["t"], info.status)
        compare_step(c, info, x, "single")
    h.close()


def test_step_chain_matches_state_rotation(dev):
    """Two consecutive steps through one handle equal two oracle steps (state kept on device)."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(128, 64))
    n = cfg["n"]
    h = binding.Handle(n, 1)
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), 1)
    x = T(cfg["x"], dev)
    g1 = cfg["g"]
    st, info1 = h.step(x, T(g1, dev), T(cfg["A"], dev), cfg["gval"], cfg["G"])
    assert st == 0
    x1 = x.cpu().numpy()
    ref1 = oracle_step(cfg["x"], cfg["x_prev"], g1, cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], cfg["G"], 1)
    # second step: a new gradient drawn from the same recipe at x1
    s = np.random.default_rng(77).lognormal(0, 1, n)
    g2 = (-3.0 * x1.astype(np.float64) ** 2 * s).astype(np.float32)
    gval2 = np.array([float(np.sum(x1, dtype=np.float64))])
    st, info2 = h.step(x, T(g2, dev), T(cfg["A"], dev), gval2, cfg["G"])
    assert st == 0
    torch.cuda.synchronize()
    ref2 = oracle_step(x1, cfg["x"], g2, g1, ref1["d"].astype(np.float32), cfg["A"], gval2, cfg["G"], 2)
    assert info2.alpha == pytest.approx(ref2["alpha"], rel=1e-6)
    assert info2.beta == pytest.approx(ref2["beta"], rel=1e-5, abs=1e-12)
    err = parity_errors(x.cpu().numpy(), [info2.lambda_[0]], ref2["x_new"], ref2["lam"], cfg["A"], ref2["b"],
                        C, 0.0, 1.0)
    check(err, "second step")
    xp = torch.empty(n, device=dev)
    gp = torch.empty(n, device=dev)
    dp = torch.empty(n, device=dev)
    assert h.get_state(xp, gp, dp) == 3
    torch.cuda.synchronize()
    assert np.array_equal(xp.cpu().numpy(), x1)
    assert np.array_equal(gp.cpu().numpy(), g2)
    assert np.allclose(dp.cpu().numpy(), ref2["d"], rtol=1e-6, atol=1e-6)
    h.close()


def test_step_host_buffers_match_device_step(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(64, 64))
    st, info, x_dev = run_step(dev, cfg)
    h = binding.Handle(cfg["n"], 1)
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    xh = torch.from_numpy(cfg["x"].copy()).pin_memory()
    st2, info2 = h.step_host(xh, torch.from_numpy(cfg["g"]).pin_memory(), torch.from_numpy(cfg["A"]).pin_memory(),
                             cfg["gval"], cfg["G"])
    assert st2 == 0
    assert np.array_equal(xh.numpy().astype(np.float64), x_dev)
    assert info2.lambda_[0] == info.lambda_[0]
    h.close()


def test_nonfinite_input_is_reported(dev):
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(32, 32))
    g = cfg["g"].copy()
    g[17] = np.nan
    c = dict(cfg, g=g)
    h = binding.Handle(cfg["n"], 1)
    st, info, _ = run_step(dev, c, handle=h)
    assert st == binding.PGDTO_ERR_NONFINITE
    # the error is reported once; the same handle then takes a clean step
    st, info, x = run_step(dev, cfg, handle=h)
    assert st == 0
    compare_step(cfg, info, x, "single")
    h.close()
