"""The optimizer loop around the step (Alg. 3): the fallback rule after the warm-up, the
global relaxation omega, and the relative-change stop, against the oracle."""

import numpy as np
import pytest

from oracle import oracle_step
from oracle.checks import parity_errors
from oracle.step import StepParams
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = {"lam_rel": 1e-6, "x_abs": 1e-6, "viol_rel": 1e-6}
BRANCH = {"fallback": 0, "bb1": 1, "lipschitz": 2}


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
    assert not bad, "%s parity: %s" % (what, bad)


def gpu_step(dev, h, s, g, G):
    import torch
    x = T(s["x"], dev)
    if s["t"] > 0:
        h.set_state(T(s["x_prev"], dev), T(s["g_prev"], dev), T(s["d_prev"], dev), s["t"])
    else:
        h.set_state(None, None, None, 0)
    st, info = h.step(x, T(g, dev), T(s["A"], dev), s["gval"], G)
    torch.cuda.synchronize()
    return st, info, x.cpu().numpy().astype(np.float64)


def test_fallback_after_warmup(dev):
    """Workload 2 driven past t_warmup = 50 by an objective gradient that keeps changing
    (g_t = g (1 + 0.1 cos 0.7 t)): from t = 50 on the nonlinear row's violation decides
    between the fallback step and the spectral step (Alg. 3).  Every step from t = 44
    to 61 is compared with the oracle's step from the oracle's own state."""
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config2(dims=(32, 16, 16))
    n = cfg["n"]
    x = cfg["x"].astype(np.float32)
    x_prev = np.zeros(n, np.float32)
    g_prev = np.zeros(n, np.float32)
    d_prev = np.zeros(n, np.float32)
    h = binding.Handle(n, 1)
    seen = []
    for t in range(62):
        A, gval = inputs.config2_inputs(cfg, x)
        g = (cfg["g"] * np.float32(1.0 + 0.1 * np.cos(0.7 * t))).astype(np.float32)
        ref = oracle_step(x, x_prev, g, g_prev, d_prev, A, gval, cfg["G"], t)
        if t >= 44:
            s = {"x": x, "x_prev": x_prev, "g_prev": g_prev, "d_prev": d_prev, "A": A, "gval": gval, "t": t}
            st, info, xg = gpu_step(dev, h, s, g, cfg["G"])
            assert st in (0, binding.PGDTO_NOT_CONVERGED), (t, st)
            assert info.branch == BRANCH[ref["branch"]], (t, info.branch, ref["branch"])
            assert info.alpha == pytest.approx(ref["alpha"], rel=1e-6)
            check(parity_errors(xg, [info.lambda_[0]], ref["x_new"], ref["lam"], A, ref["b"], C, 0.0, 1.0),
                  "t=%d" % t)
            seen.append((t, ref["branch"], float(np.max(gval - cfg["G"]))))
        x_prev, g_prev, d_prev = x.copy(), g.copy(), ref["d"].astype(np.float32)
        x = ref["x_new"].astype(np.float32)
    h.close()
    # the window holds spectral steps and a fallback that only the warm-up rule explains
    assert any(b != "fallback" for _, b, _ in seen)
    assert any(t >= 50 and b == "fallback" and v > 1e-6 for t, b, v in seen), seen


def test_fallback_rule_switches_at_warmup(dev):
    """At t = t_warmup - 1 a violated row still takes the spectral step; at t = t_warmup
    it takes the fallback step (the host decides the rule from g_val and G)."""
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(64, 32))
    n = cfg["n"]
    G = cfg["gval"] - 5.0  # the nonlinear row is violated by 5
    for t, want in ((49, "spectral"), (50, "fallback")):
        h = binding.Handle(n, 1)
        s = dict(cfg, t=t)
        st, info, xg = gpu_step(dev, h, s, cfg["g"], G)
        h.close()
        ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], G, t)
        assert st == 0
        assert (ref["branch"] == "fallback") == (want == "fallback")
        assert info.branch == BRANCH[ref["branch"]]
        assert info.alpha == pytest.approx(ref["alpha"], rel=1e-6)
        check(parity_errors(xg, [info.lambda_[0]], ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0),
              "t=%d" % t)


@pytest.mark.parametrize("omega", [0.5, 1.3])
def test_relaxation_omega(dev, omega):
    """z = x + omega alpha d (Sec. 3.4, global relaxation)."""
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(128, 64))
    h = binding.Handle(cfg["n"], 1, omega=omega)
    st, info, xg = gpu_step(dev, h, cfg, cfg["g"], cfg["G"])
    h.close()
    assert st == 0
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], cfg["G"],
                      cfg["t"], p=StepParams(omega=omega))
    check(parity_errors(xg, [info.lambda_[0]], ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0),
          "omega=%g" % omega)
    assert info.rel_change == pytest.approx(ref["rel_change"], rel=1e-4)


def test_loop_until_relative_change_stop(dev):
    """Alg. 3 run to its stopping rule ||x_{t+1} - x_t|| / ||x_{t+1}|| < tol with the state
    on the device (the caller's loop), beside the oracle's loop on the host: both stop at
    the same iteration and end on the same design."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(96, 48))
    n = cfg["n"]
    s_rng = np.random.default_rng(5).lognormal(0.0, 1.0, n)

    def sens(x):
        x = x.astype(np.float64)
        return (-3.0 * x * x * s_rng).astype(np.float32), np.array([float(np.sum(x.astype(np.float32),
                                                                                 dtype=np.float64))])

    tol = 1e-3
    # oracle loop
    x = cfg["x"].astype(np.float32)
    xp, gp, dp = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32)
    stop_ref = None
    for t in range(200):
        g, gval = sens(x)
        ref = oracle_step(x, xp, g, gp, dp, cfg["A"], gval, cfg["G"], t)
        xp, gp, dp = x, g, ref["d"].astype(np.float32)
        x = ref["x_new"].astype(np.float32)
        if ref["rel_change"] < tol:
            stop_ref = t
            break
    assert stop_ref is not None and stop_ref > 3
    # device loop
    h = binding.Handle(n, 1)
    h.set_state(None, None, None, 0)
    xd = T(cfg["x"], dev)
    Ad = T(cfg["A"], dev)
    stop_gpu = None
    for t in range(200):
        g, gval = sens(xd.cpu().numpy())
        st, info = h.step(xd, T(g, dev), Ad, gval, cfg["G"])
        assert st == 0
        if info.rel_change < tol:
            stop_gpu = t
            break
    torch.cuda.synchronize()
    h.close()
    assert stop_gpu == stop_ref
    assert float(np.max(np.abs(xd.cpu().numpy().astype(np.float64) - x.astype(np.float64)))) < 1e-4


def test_warm_started_steps_match_the_oracle(dev):
    """Consecutive steps of one handle seed each search with the previous step's lam (warm
    start); each step still equals the oracle's step from the same state (read back with
    pgdto_get_state)."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config2(dims=(48, 24, 24))
    n = cfg["n"]
    h = binding.Handle(n, 1)
    h.set_state(None, None, None, 0)
    x = T(cfg["x"], dev)
    xp, gp, dp = (torch.empty(n, device=dev) for _ in range(3))
    passes = []
    for t in range(14):
        x_now = x.cpu().numpy()
        t_now = h.get_state(xp, gp, dp)
        assert t_now == t
        A, gval = inputs.config2_inputs(cfg, x_now)
        st, info = h.step(x, T(cfg["g"], dev), T(A, dev), gval, cfg["G"])
        torch.cuda.synchronize()
        assert st == 0, (t, st)
        ref = oracle_step(x_now, xp.cpu().numpy(), cfg["g"], gp.cpu().numpy(), dp.cpu().numpy(), A, gval, cfg["G"], t)
        check(parity_errors(x.cpu().numpy(), [info.lambda_[0]], ref["x_new"], ref["lam"], A, ref["b"], C, 0.0, 1.0),
              "warm t=%d" % t)
        passes.append(info.passes)
    h.close()
    assert max(passes) <= 20


def test_warm_started_coupled_steps_match_the_oracle(dev):
    """Consecutive coupled-row steps of one handle start Newton at the previous step's
    multipliers (warm start); each step equals the oracle's step from the same state."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config4(dims=(40, 20, 20))
    n, m = cfg["n"], cfg["m"]
    h = binding.Handle(n, m, mode="coupled")
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    x = T(cfg["x"], dev)
    A = T(cfg["A"], dev)
    xp, gp, dp = (torch.empty(n, device=dev) for _ in range(3))
    rng = np.random.default_rng(3)
    s = rng.lognormal(0.0, 1.0, n)
    passes = []
    for k in range(8):
        x_now = x.cpu().numpy()
        t_now = h.get_state(xp, gp, dp)
        g = (-3.0 * x_now.astype(np.float64) ** 2 * s).astype(np.float32)
        gval = cfg["A"].astype(np.float64) @ x_now.astype(np.float64)
        st, info = h.step(x, T(g, dev), A, gval, cfg["G"])
        torch.cuda.synchronize()
        assert st == 0, (k, info.as_dict(m))
        ref = oracle_step(x_now, xp.cpu().numpy(), g, gp.cpu().numpy(), dp.cpu().numpy(), cfg["A"], gval, cfg["G"],
                          t_now, mode="coupled")
        lam = np.array(list(info.lambda_)[:m])
        check(parity_errors(x.cpu().numpy(), lam, ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0),
              "coupled warm k=%d" % k)
        passes.append(info.passes)
    h.close()
    assert passes[-1] <= passes[0] + 2  # the warm start does not make the later steps longer
