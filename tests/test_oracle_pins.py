"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* hand-derived fixtures (tests/golden, each with its derivation);
* brute-force KKT enumeration of the QP (oracle/bruteforce.py uses no dual machinery);
* SciPy's SLSQP on the primal QP with explicit slack variables (a library routine);
* closed forms, invariants (KKT, projection variational inequality, idempotence,
  monotonicity of the dual residual), and finite differences of eq. h for eq. reg_jacobian.
"""

import json
import os

import numpy as np
import pytest

import oracle
from oracle import projection as P
from oracle.bruteforce import project_bruteforce
from oracle.checks import kkt_report
from oracle.step import StepParams, oracle_step, step_scalars
from paper_2511_13905_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C = 1e12


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------- golden fixtures

@pytest.mark.parametrize("case", _load("step_scalars.json")["cases"], ids=lambda c: c["name"])
def test_step_scalars_golden(case):
    sc = step_scalars(case["x"], case["x_prev"], case["g"], case["g_prev"], case["t"],
                      case["gval"], case["G"], StepParams(), eq=case.get("eq"))
    assert sc["branch"] == case["branch"]
    assert sc["alpha"] == pytest.approx(case["alpha"], rel=1e-12)
    assert sc["beta"] == pytest.approx(case["beta"], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("case", _load("projections.json")["cases"], ids=lambda c: c["name"])
def test_projection_golden(case):
    z = np.array(case["z"])
    A = np.array(case["A"])
    b = np.array(case["b"])
    Cc = case.get("C", C)
    lam_ref = np.array(case["lam"])
    x_ref = np.array(case["x"])
    lam, _ = P.solve_coupled_exact(z, A, b, case["lo"], case["hi"], Cc)
    assert np.allclose(lam, lam_ref, rtol=1e-10, atol=1e-12)
    assert np.allclose(P.primal_from_dual(z, A, lam, case["lo"], case["hi"]), x_ref, atol=1e-10)
    if A.shape[0] == 1:
        l1 = P.solve_single_exact(z, A[0], b[0], case["lo"], case["hi"], Cc)
        assert l1 == pytest.approx(lam_ref[0], rel=1e-10, abs=1e-12)
        lb, _ = P.solve_single_bisect(z, A[0], b[0], case["lo"], case["hi"], Cc, tol_B=1e-13)
        assert lb == pytest.approx(lam_ref[0], rel=1e-9, abs=1e-12)
    la, info = P.alg2_general_projection(z, A, b, case["lo"], case["hi"], Cc, tol_B=1e-13, tol_N=1e-12)
    assert np.allclose(la, lam_ref, rtol=1e-8, atol=1e-10)


def test_full_step_golden():
    c = _load("full_step.json")
    n = len(c["x"])
    out = oracle_step(c["x"], c["x"], c["g"], np.zeros(n), np.zeros(n), c["A"], c["gval"], c["G"],
                      c["t"], StepParams(), mode="single", lo=c["lo"], hi=c["hi"])
    assert out["alpha"] == pytest.approx(c["alpha"], rel=1e-14)
    assert np.allclose(out["d"], c["d"], atol=0)
    assert np.allclose(out["z"], c["z"], atol=1e-15)
    assert np.allclose(out["b"], c["b"], atol=1e-15)
    assert np.allclose(out["lam"], c["lam"], rtol=1e-10)
    assert np.allclose(out["x_new"], c["x_new"], atol=1e-12)
    assert out["rel_change"] == pytest.approx(c["rel_change"], rel=1e-10)


def test_full_step_t1_golden():
    """t = 1: the PR+ direction d = -g + beta d_prev (eq. CG) with beta > 0 and the
    relaxed trial point z = x + omega alpha d (Sec. 3.4) with omega = 0.5."""
    c = _load("full_step_t1.json")
    out = oracle_step(c["x"], c["x_prev"], c["g"], c["g_prev"], c["d_prev"], c["A"], c["gval"], c["G"],
                      c["t"], StepParams(omega=c["omega"]), mode="single", lo=c["lo"], hi=c["hi"])
    assert out["branch"] == c["branch"]
    assert out["alpha"] == pytest.approx(c["alpha"], rel=1e-14)
    assert out["beta"] == pytest.approx(c["beta"], rel=1e-14)
    assert np.allclose(out["d"], c["d"], rtol=0, atol=1e-15)
    assert np.allclose(out["z"], c["z"], rtol=0, atol=1e-15)
    assert np.allclose(out["b"], c["b"], atol=1e-15)
    assert np.allclose(out["lam"], c["lam"], rtol=1e-12)
    assert np.allclose(out["x_new"], c["x_new"], atol=1e-14)
    assert out["rel_change"] == pytest.approx(c["rel_change"], rel=1e-12)


# ----------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(24))
def test_exact_solvers_match_bruteforce(seed):
    m = 1 + seed % 4
    n = 4 + seed % 3
    z, A, b = inputs.random_projection(n, m, 100 + seed, feasible=(seed % 5 != 0))
    z = z.astype(np.float64)
    A = A.astype(np.float64)
    x_bf, lam_bf, _ = oracle.project_bruteforce(z, A, b, 0.0, 1.0, C)
    lam, info = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C)
    assert np.allclose(lam, lam_bf, rtol=1e-9, atol=1e-12)
    assert np.allclose(P.primal_from_dual(z, A, lam, 0.0, 1.0), x_bf, atol=1e-10)
    if m == 1:
        assert P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, C) == pytest.approx(lam_bf[0], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_moderate_C(seed):
    """With C = 3 the slack is a visible part of the optimum: pins the 2 lam / C term of eq. h."""
    z, A, b = inputs.random_projection(5, 2, 300 + seed, feasible=False)
    z = z.astype(np.float64)
    A = A.astype(np.float64)
    x_bf, lam_bf, _ = oracle.project_bruteforce(z, A, b, 0.0, 1.0, 3.0)
    lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, 3.0)
    assert np.allclose(lam, lam_bf, rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------------- SLSQP on the primal QP

def _slsqp_primal(z, A, b, lo, hi, Cc):
    """min ||x - z||^2 + (C/2)||s||^2 s.t. lo <= x <= hi, A x - s <= b, s >= 0 with SciPy."""
    opt = pytest.importorskip("scipy.optimize")
    m, n = A.shape

    def f(v):
        x, s = v[:n], v[n:]
        return float((x - z) @ (x - z) + 0.5 * Cc * (s @ s))

    def grad(v):
        x, s = v[:n], v[n:]
        return np.concatenate([2 * (x - z), Cc * s])

    cons = [{"type": "ineq", "fun": lambda v: b - A @ v[:n] + v[n:],
             "jac": lambda v: np.hstack([-A, np.eye(m)])}]
    bounds = [(lo, hi)] * n + [(0.0, None)] * m
    v0 = np.concatenate([np.clip(z, lo, hi), np.zeros(m)])
    res = opt.minimize(f, v0, jac=grad, bounds=bounds, constraints=cons, method="SLSQP",
                       options={"ftol": 1e-15, "maxiter": 2000})
    return res.x[:n], res.x[n:]


@pytest.mark.parametrize("seed,feasible,Cc", [(0, True, C), (1, True, C), (2, False, 20.0),
                                             (3, False, 50.0), (4, True, 20.0)])
def test_primal_qp_matches_slsqp(seed, feasible, Cc):
    z, A, b = inputs.random_projection(30, 3, 500 + seed, feasible=feasible)
    z = z.astype(np.float64)
    A = A.astype(np.float64)
    x_s, s_s = _slsqp_primal(z, A, b, 0.0, 1.0, Cc)
    lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, Cc)
    x = P.primal_from_dual(z, A, lam, 0.0, 1.0)
    assert np.max(np.abs(x - x_s)) < 1e-5
    # slack of the QP is s_j = 2 lam_j / C (KKT of the QP above)
    assert np.allclose(2.0 * lam / Cc, s_s, atol=1e-5)


# ----------------------------------------------------------------- closed forms

def test_closed_form_all_free():
    rng = np.random.default_rng(7)
    n = 1000
    z = rng.uniform(0.3, 0.7, n)
    a = rng.uniform(0.5, 1.5, n)
    b = float(a @ z) - 0.5
    lam_cf = (a @ z - b) / (a @ a + 2.0 / C)
    assert np.all((z - lam_cf * a >= 0) & (z - lam_cf * a <= 1))
    assert P.solve_single_exact(z, a, b, 0.0, 1.0, C) == pytest.approx(lam_cf, rel=1e-13)


def test_closed_form_trivially_feasible():
    rng = np.random.default_rng(8)
    z = rng.uniform(-0.5, 1.5, 500)
    A = rng.uniform(0.1, 1.0, (3, 500))
    b = A @ np.clip(z, 0, 1) + 1.0
    lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C)
    assert np.all(lam == 0)
    assert np.array_equal(P.primal_from_dual(z, A, lam, 0, 1), np.clip(z, 0, 1))


def test_closed_form_infeasible_all_clipped():
    rng = np.random.default_rng(9)
    z = rng.uniform(0.0, 1.0, 400)
    a = rng.uniform(0.2, 1.0, 400)
    b = -3.0
    lam = P.solve_single_exact(z, a, b, 0.0, 1.0, C)
    assert lam == pytest.approx(0.5 * C * (0.0 - b), rel=1e-12)
    lb, _ = P.solve_single_bisect(z, a, b, 0.0, 1.0, C)
    assert lb == pytest.approx(0.5 * C * (0.0 - b), rel=1e-12)


def test_independent_rows_are_separate_solves():
    cfg = inputs.config3(dims=(8, 6, 5))
    x = cfg["x"].astype(np.float64)
    a = cfg["A"].astype(np.float64)
    z = x + 0.3 * np.random.default_rng(1).standard_normal(cfg["n"])
    seg = cfg["seg"]
    b = cfg["G"]
    lam_seg = P.solve_independent_exact(z, a, seg, b, 0.0, 1.0, C)
    Ad = P.segmented_to_dense(a, seg, cfg["n"])
    lam_dense, _ = P.solve_coupled_exact(z, Ad, b, 0.0, 1.0, C)
    assert np.allclose(lam_seg, lam_dense, rtol=1e-10)


# ----------------------------------------------------------------- invariants

@pytest.mark.parametrize("cfgfun", ["config1", "config4"])
def test_kkt_and_variational_inequality(cfgfun):
    if cfgfun == "config1":
        cfg = inputs.config1(dims=(64, 32))
    else:
        cfg = inputs.config4(dims=(16, 8, 8))
    out = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"],
                      cfg["gval"], cfg["G"], cfg["t"], mode=cfg["mode"])
    A = np.atleast_2d(cfg["A"]).astype(np.float64)
    rep = kkt_report(out["z"], A, out["b"], out["lam"], out["x_new"], 0.0, 1.0, C)
    assert rep["worst"] < 1e-11
    # (z - x*)^T (w - x*) <= 0 for feasible w (exact projection up to the O(1/C) slack)
    rng = np.random.default_rng(3)
    xs = out["x_new"]
    for _ in range(20):
        w = rng.uniform(0, 1, xs.size) * xs  # shrinks toward 0
        if np.all(A @ w <= out["b"]):
            assert (out["z"] - xs) @ (w - xs) <= 1e-6 * max(1.0, np.abs(out["z"] - xs).sum())


def test_idempotence():
    rng = np.random.default_rng(11)
    z = rng.uniform(-0.5, 1.5, 300)
    A = np.abs(rng.standard_normal((2, 300))) + 0.1
    b = A @ np.full(300, 0.4)
    lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C)
    x = P.primal_from_dual(z, A, lam, 0.0, 1.0)
    lam2, _ = P.solve_coupled_exact(x, A, b, 0.0, 1.0, C)
    x2 = P.primal_from_dual(x, A, lam2, 0.0, 1.0)
    assert np.max(np.abs(x2 - x)) < 1e-9


def test_single_row_residual_monotone():
    cfg = inputs.config1(dims=(32, 16))
    z = cfg["x"].astype(np.float64) + 0.2
    a = cfg["A"][0].astype(np.float64)
    grid = np.linspace(0.0, 2.0, 401)
    r = [P.residual(z, a[None, :], [0.4 * a.size], [lam], 0.0, 1.0, C)[0] for lam in grid]
    # nonincreasing everywhere (App. A.2); strictly while some variable is free
    assert np.all(np.diff(r) <= 1e-12)
    assert np.all(np.diff(r)[: 100] < 0)


def test_jacobian_matches_finite_differences():
    rng = np.random.default_rng(5)
    z = rng.uniform(-0.3, 1.3, 200)
    A = rng.standard_normal((3, 200))
    b = rng.standard_normal(3)
    lam = np.array([0.05, 0.02, 0.03])
    Cc = 10.0
    J = P.jacobian_h(z, A, lam, 0.0, 1.0, Cc)
    eps = 1e-7
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        # h(y) with y = -lam: dh/dy_k = -(r(lam + e) - r(lam - e)) / (2 eps)
        fd = -(P.residual(z, A, b, lam + e, 0, 1, Cc) - P.residual(z, A, b, lam - e, 0, 1, Cc)) / (2 * eps)
        assert np.allclose(J[:, k], fd, rtol=1e-6, atol=1e-6)


def test_newton_descent_identity():
    """grad M^T Delta = ||Phi||^2 (App. A.3.3) for the Newton direction."""
    rng = np.random.default_rng(6)
    z = rng.uniform(-0.3, 1.3, 100)
    A = rng.standard_normal((3, 100))
    b = rng.standard_normal(3)
    y = np.array([-0.1, 0.0, -0.05])
    h = P.residual(z, A, b, -y, 0, 1, C)
    Ph = P.phi(h, y)
    Jh = P.jacobian_h(z, A, -y, 0, 1, C)
    D = np.diag((h > 0).astype(float))
    Jp = D @ Jh + np.eye(3) - D
    Delta = np.linalg.solve(Jp, Ph)
    assert (Jp.T @ Ph) @ Delta == pytest.approx(Ph @ Ph, rel=1e-10)


# ----------------------------------------------------------------- paper algorithms vs exact

def test_bisection_agrees_with_exact_single():
    cfg = inputs.config1()
    out = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"],
                      cfg["gval"], cfg["G"], cfg["t"], mode="single")
    lb, its = P.solve_single_bisect(out["z"], cfg["A"][0].astype(np.float64), out["b"][0], 0.0, 1.0, C,
                                    tol_B=1e-8)
    assert abs(lb - out["lam"][0]) <= 1e-8
    assert 10 < its < 200


def test_alg2_agrees_with_exact_on_coupled_workload():
    cfg = inputs.config4(dims=(32, 16, 16))
    out = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"],
                      cfg["gval"], cfg["G"], cfg["t"], mode="coupled")
    A = cfg["A"].astype(np.float64)
    lam2, info = P.alg2_general_projection(out["z"], A, out["b"], 0.0, 1.0, C, tol_B=1e-12, tol_N=1e-12)
    assert info["converged"]
    assert np.allclose(lam2, out["lam"], rtol=1e-6, atol=1e-9)


def test_config4_infeasible_seed_is_regularised():
    cfg = inputs.config4(dims=(16, 8, 8), infeasible=True)
    out = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"],
                      cfg["gval"], cfg["G"], cfg["t"], mode="coupled")
    A = cfg["A"].astype(np.float64)
    # row 2 (first moment along y, all coefficients > 0, b < 0) cannot hold for x >= 0
    assert np.all(A[2] > 0) and out["b"][2] < 0
    assert out["lam"][2] > 1e9
    rep = kkt_report(out["z"], A, out["b"], out["lam"], out["x_new"], 0.0, 1.0, C)
    assert rep["worst"] < 1e-11


# --------------------------------------------------------------------------- equality rows
# Sec. 3.2.4: an equality row is always active; its multiplier has either sign and the
# regularised residual a^T x - b - 2 lam / C is zero.  Pinned by the brute-force KKT
# enumeration (equality rows in every active set, no sign condition), SciPy on the primal
# QP with a free slack, closed forms, and the C -> infinity limit.

def _eq_problem(n, m, seed, side):
    """Tiny problem whose equality rows bind from `side` ('above': the inequality reading
    would leave them inactive, so lam < 0; 'below': lam > 0)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.3, 1.3, n)
    A = rng.uniform(0.2, 1.5, (m, n)) * rng.choice([-1.0, 1.0], (m, n), p=[0.2, 0.8])
    xc = np.clip(z, 0.0, 1.0)
    target = A @ xc
    b = target + (0.3 if side == "above" else -0.3) * np.abs(A).sum(axis=1) / n
    return z, A, b


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("side", ["above", "below"])
def test_equality_single_row_matches_bruteforce(seed, side):
    z, A, b = _eq_problem(6, 1, 900 + seed, side)
    for Cc in (C, 4.0):
        _, lam_bf, _ = project_bruteforce(z, A, b, 0.0, 1.0, Cc, eq=[True])
        lam = P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, Cc, equality=True)
        assert lam == pytest.approx(lam_bf[0], rel=1e-10, abs=1e-12)
        lb, _ = P.solve_single_bisect(z, A[0], b[0], 0.0, 1.0, Cc, tol_B=1e-14, equality=True)
        assert lb == pytest.approx(lam, rel=1e-9, abs=1e-12)
        if side == "above" and Cc == C:
            assert lam < 0.0  # the inequality reading would have lam = 0
            assert P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, Cc) == 0.0


@pytest.mark.parametrize("seed", range(10))
def test_equality_coupled_matches_bruteforce(seed):
    rng = np.random.default_rng(950 + seed)
    m = 2 + seed % 2
    z, A, b = _eq_problem(5, m, 950 + seed, "above" if seed % 3 else "below")
    eq = rng.uniform(size=m) < 0.5
    eq[seed % m] = True
    for Cc in (C, 3.0):
        _, lam_bf, _ = project_bruteforce(z, A, b, 0.0, 1.0, Cc, eq=eq)
        lam, info = P.solve_coupled_exact(z, A, b, 0.0, 1.0, Cc, eq=eq)
        assert np.allclose(lam, lam_bf, rtol=1e-9, atol=1e-12), (lam, lam_bf, eq)
        assert info["kkt"]["worst"] < 1e-10
        lam2, inf2 = P.alg2_general_projection(z, A, b, 0.0, 1.0, Cc, tol_N=1e-12, single="exact", eq=eq)
        assert np.allclose(lam2, lam_bf, rtol=1e-7, atol=1e-10), (lam2, lam_bf, inf2)
        assert inf2["newton_iters"] <= 20  # semismooth Newton: a few steps on 5 variables


@pytest.mark.parametrize("seed", range(4))
def test_equality_primal_qp_matches_slsqp(seed):
    """min ||x - z||^2 + (C/2)||s||^2 s.t. lo <= x <= hi, a_j^T x - s_j <= b_j (s_j >= 0) for
    inequality rows and a_j^T x - s_j = b_j (s_j free) for equality rows."""
    opt = pytest.importorskip("scipy.optimize")
    Cc = 20.0
    z, A, b = _eq_problem(7, 2, 980 + seed, "above")
    eq = np.array([True, False])
    m, n = A.shape

    def f(v):
        x, s = v[:n], v[n:]
        return float((x - z) @ (x - z) + 0.5 * Cc * s @ s)

    cons = [{"type": "eq", "fun": lambda v: A[0] @ v[:n] - v[n] - b[0]},
            {"type": "ineq", "fun": lambda v: b[1] + v[n + 1] - A[1] @ v[:n]}]
    bounds = [(0.0, 1.0)] * n + [(None, None), (0.0, None)]
    res = opt.minimize(f, np.concatenate([np.clip(z, 0, 1), np.zeros(m)]), method="SLSQP", bounds=bounds,
                       constraints=cons, options={"ftol": 1e-15, "maxiter": 500})
    lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, Cc, eq=eq)
    x = P.primal_from_dual(z, A, lam, 0.0, 1.0)
    assert np.allclose(x, res.x[:n], atol=2e-6)
    assert 2.0 * lam[0] / Cc == pytest.approx(res.x[n], abs=2e-6)  # slack s = 2 lam / C, either sign


def test_equality_closed_forms():
    rng = np.random.default_rng(11)
    n = 50
    a = rng.uniform(0.5, 1.5, n)
    z = rng.uniform(0.4, 0.6, n)
    # all free: lam = (a^T z - b) / (|a|^2 + 2/C), here negative
    b = float(a @ z) + 0.01
    lam = P.solve_single_exact(z, a, b, 0.0, 1.0, C, equality=True)
    assert lam == pytest.approx((a @ z - b) / (a @ a + 2.0 / C), rel=1e-12)
    assert lam < 0.0
    # unreachable from above (b beyond a^T hi): every x at the row-maximising bound and
    # lam = (C/2)(S_max - b)
    b2 = float(a.sum()) + 3.0
    lam2 = P.solve_single_exact(z, a, b2, 0.0, 1.0, C, equality=True)
    assert lam2 == pytest.approx(0.5 * C * (a.sum() - b2), rel=1e-10)
    # exactly met at lam = 0
    b3 = float(a @ np.clip(z, 0, 1))
    assert P.solve_single_exact(z, a, b3, 0.0, 1.0, C, equality=True) == 0.0


def test_equality_met_exactly_in_the_limit():
    """C -> infinity (Sec. 3.2.3): a feasible equality row holds to rounding, and the
    result is the Euclidean projection onto box and hyperplane (the same at 1e12 and 1e15)."""
    z, A, b = _eq_problem(400, 1, 990, "above")
    l1 = P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, 1e12, equality=True)
    l2 = P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, 1e15, equality=True)
    x1 = P.primal_from_dual(z, A, [l1], 0.0, 1.0)
    x2 = P.primal_from_dual(z, A, [l2], 0.0, 1.0)
    assert abs(float(A[0] @ x1) - b[0]) < 1e-9 * abs(b[0])
    assert np.allclose(x1, x2, atol=1e-9)


def test_equality_with_nonnegative_multiplier_equals_the_inequality():
    """When the equality row's multiplier comes out >= 0 the inequality reading has the
    same optimum (an active inequality)."""
    for seed in range(6):
        z, A, b = _eq_problem(30, 2, 1000 + seed, "below")
        lam_e, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C, eq=[True, True])
        if np.all(lam_e >= 0):
            lam_i, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C)
            assert np.allclose(lam_e, lam_i, rtol=1e-9, atol=1e-12)


def test_equality_rows_in_a_full_step():
    """oracle_step with equality rows: independent rows (one of them an equality) and a
    coupled pair, against the same projections written out directly."""
    cfg = inputs.config3(dims=(10, 8, 6), materials=2)
    eq = [True, False]
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"],
                      cfg["gval"], cfg["G"], cfg["t"], mode="independent", seg=cfg["seg"], eq=eq)
    lam = P.solve_independent_exact(ref["z"], cfg["A"].astype(np.float64), cfg["seg"], ref["b"], 0.0, 1.0, C, eq=eq)
    assert np.allclose(ref["lam"], lam)
    seg = cfg["seg"]
    ax = float(cfg["A"][seg[0]:seg[1]].astype(np.float64) @ ref["x_new"][seg[0]:seg[1]])
    assert abs(ax - ref["b"][0] - 2.0 * ref["lam"][0] / C) < 1e-9 * abs(ref["b"][0])
