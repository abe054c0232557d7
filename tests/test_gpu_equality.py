"""Equality rows (Sec. 3.2.4) on the GPU against the oracle: always active, multiplier of
either sign, residual a^T x - b - 2 lam / C equal to zero.  Single rows from both sides
and past saturation (both engines), independent rows with a mixed mask, coupled rows, full
steps, and the fallback rule's |g - G| for an equality."""

import numpy as np
import pytest

from oracle import oracle_step
from oracle import projection as P
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = {"lam_rel": 1e-6, "x_abs": 1e-6, "viol_rel": 1e-6}
GRID, CLUSTER = 1, 2


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


def project(dev, z, A, b, eq_mask, seg=None, engine=0):
    import torch
    from paper_2511_13905_gb300 import binding
    m = len(b)
    n = z.size
    h = binding.Handle(n, m, seg=seg, eq_mask=eq_mask, engine=engine)
    xt = torch.empty(n, device=dev)
    st, lam, info = h.project(T(z, dev), T(A, dev), b, xt)
    torch.cuda.synchronize()
    h.close()
    return st, np.array(lam), xt.cpu().numpy().astype(np.float64), info


def single_case(n, seed, side):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.3, 1.3, n).astype(np.float32)
    a = (rng.lognormal(0.0, 0.7, n) * rng.choice([-1.0, 1.0], n, p=[0.15, 0.85])).astype(np.float32)
    a64, z64 = a.astype(np.float64), z.astype(np.float64)
    base = float(a64 @ np.clip(z64, 0, 1))
    spread = float(np.abs(a64).sum())
    b = {"above": base + 0.05 * spread, "below": base - 0.05 * spread,
         "unreachable": float(np.where(a64 > 0, a64, 0.0).sum()) + 0.01 * spread + 1.0}[side]
    return z, a, b


@pytest.mark.parametrize("engine", [GRID, CLUSTER])
@pytest.mark.parametrize("n,seed,side", [(1000, 1, "above"), (4097, 2, "below"), (65537, 3, "above"),
                                         (300001, 4, "above"), (777, 5, "unreachable"), (1 << 20, 6, "above")])
def test_single_equality_row(dev, engine, n, seed, side):
    z, a, b = single_case(n, seed, side)
    st, lam, x, info = project(dev, z, a, [b], 1, engine=engine)
    assert st == 0, info.as_dict(1)
    z64, a64 = z.astype(np.float64), a.astype(np.float64)
    lr = P.solve_single_exact(z64, a64, b, 0.0, 1.0, C, equality=True)
    if side in ("above", "unreachable"):
        assert lr < 0.0  # binds from below: the inequality reading would give 0
    xr = np.clip(z64 - lr * a64, 0.0, 1.0)
    check(parity_errors(x, lam, xr, [lr], a[None, :], [b], C, 0.0, 1.0, eq=[True]),
          "n=%d %s engine %d" % (n, side, engine))


@pytest.mark.parametrize("engine", [GRID, CLUSTER])
def test_independent_rows_mixed_mask(dev, engine):
    """Workload-3 layout, four material rows, rows 0 and 2 equalities (one binding from
    each side), against the oracle's full step."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config3(dims=(24, 16, 12))
    eq = [True, False, True, False]
    G = cfg["G"].copy()
    # row 2 asks for more material than the clipped trial point holds, so as an equality it
    # binds from below (lam_2 < 0)
    ref0 = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], G,
                       cfg["t"], mode="independent", seg=cfg["seg"])
    s2, e2 = cfg["seg"][2], cfg["seg"][3]
    G[2] = cfg["gval"][2] + float(np.clip(ref0["z"][s2:e2], 0, 1).sum() - cfg["x"][s2:e2].astype(np.float64).sum()) \
        + 0.05 * (e2 - s2)
    h = binding.Handle(cfg["n"], 4, seg=cfg["seg"], eq_mask=0b0101, engine=engine)
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], G)
    torch.cuda.synchronize()
    h.close()
    assert st == 0, info.as_dict(4)
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], G,
                      cfg["t"], mode="independent", seg=cfg["seg"], eq=eq)
    assert ref["lam"][2] < 0.0 < ref["lam"][0]
    seg = cfg["seg"]
    a = cfg["A"].astype(np.float64)

    def f(xv):
        ax = np.array([a[seg[j]:seg[j + 1]] @ xv[seg[j]:seg[j + 1]] for j in range(4)])
        aa = np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(xv[seg[j]:seg[j + 1]]) for j in range(4)])
        return ax, aa
    lam = np.array(list(info.lambda_)[:4])
    check(parity_errors(x.cpu().numpy(), lam, ref["x_new"], ref["lam"], f, ref["b"], C, 0.0, 1.0,
                        amax=np.ones(4), eq=eq), "independent engine %d" % engine)


@pytest.mark.parametrize("n,m,mask,seed", [(5000, 2, 0b01, 1), (40000, 3, 0b010, 2), (100003, 4, 0b1001, 3),
                                           (65536, 2, 0b11, 4)])
def test_coupled_with_equality_rows(dev, n, m, mask, seed):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.2, 1.2, n)
    A = np.vstack([np.ones(n)] + [rng.uniform(-1, 1, n) for _ in range(m - 1)])
    xin = rng.uniform(0.2, 0.6, n)
    b = A @ xin
    b[0] = 0.4 * n
    eq = [(mask >> j) & 1 == 1 for j in range(m)]
    z32, A32 = z.astype(np.float32), A.astype(np.float32)
    st, lam, x, info = project(dev, z32, A32, b, mask)
    assert st == 0, info.as_dict(m)
    lam_ref, rinfo = P.solve_coupled_exact(z32.astype(np.float64), A32.astype(np.float64), b, 0.0, 1.0, C, eq=eq)
    assert rinfo["kkt"]["worst"] < 1e-9
    x_ref = P.primal_from_dual(z32.astype(np.float64), A32.astype(np.float64), lam_ref, 0.0, 1.0)
    check(parity_errors(x, lam, x_ref, lam_ref, A32, b, C, 0.0, 1.0, eq=eq),
          "n=%d m=%d mask=%s ref=%s" % (n, m, bin(mask), lam_ref))


def test_coupled_step_volume_equality(dev):
    """Workload 4 (small mesh) with the volume row as an equality at 0.33 n, a full step:
    as an inequality that row is inactive, as an equality it binds from below (lam_0 < 0)
    while the centre-of-mass rows stay feasible."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config4(dims=(32, 16, 16))
    G = cfg["G"].copy()
    G[0] = 0.33 * cfg["n"]
    h = binding.Handle(cfg["n"], 4, mode="coupled", eq_mask=0b0001)
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], G)
    torch.cuda.synchronize()
    h.close()
    assert st == 0, info.as_dict(4)
    eq = [True, False, False, False]
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], G,
                      cfg["t"], mode="coupled", eq=eq)
    assert ref["lam"][0] < 0.0
    lam = np.array(list(info.lambda_)[:4])
    check(parity_errors(x.cpu().numpy(), lam, ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0, eq=eq),
          "coupled step")


def test_fallback_rule_counts_an_equality_from_both_sides(dev):
    """After the warm-up an equality row with g < G - tol_N triggers the fallback step
    (|g - G| > tol_N); the same row as an inequality does not."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(64, 32))
    G = cfg["gval"] + 5.0  # satisfied as an inequality, violated as an equality
    for mask, want in ((1, "fallback"), (0, "spectral")):
        h = binding.Handle(cfg["n"], 1, eq_mask=mask)
        h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), 60)
        x = T(cfg["x"], dev)
        st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], G)
        torch.cuda.synchronize()
        h.close()
        assert st == 0
        ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"], G,
                          60, eq=[mask == 1])
        assert (ref["branch"] == "fallback") == (want == "fallback")
        assert info.branch == {"fallback": 0, "bb1": 1, "lipschitz": 2}[ref["branch"]]
        check(parity_errors(x.cpu().numpy(), [info.lambda_[0]], ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0,
                            1.0, eq=[mask == 1]), "mask %d" % mask)


def test_eq_mask_validation(dev):
    from paper_2511_13905_gb300 import binding
    with pytest.raises(binding.PgdtoError):
        binding.Handle(100, 2, eq_mask=0b100)  # a flag for a row that does not exist
