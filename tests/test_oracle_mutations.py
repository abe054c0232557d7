"""Planted mistakes: each one is written into a copy of the oracle (CPU only) and at least
one pin must catch it.  This shows that the pins of test_oracle_pins.py would notice the
plausible slips (a dropped term, a wrong sign or factor, a wrong branch boundary)."""

import importlib.util
import json
import os
import shutil
import sys
import uuid

import numpy as np
import pytest

from paper_2511_13905_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
C = 1e12


def _load_copy(tmp_path, fname=None, old=None, new=None):
    name = "oracle_copy_" + uuid.uuid4().hex[:8]
    dst = tmp_path / name
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("__pycache__"))
    if fname is not None:
        src = (dst / fname).read_text()
        assert old in src, (fname, old)
        (dst / fname).write_text(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py",
                                                  submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return mod


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _pins(mod):
    """Run a fixed set of pins against an oracle copy; return the names of those that fail."""
    failed = []
    P = mod.projection
    S = mod.step
    try:
        for c in _golden("step_scalars.json")["cases"]:
            sc = S.step_scalars(c["x"], c["x_prev"], c["g"], c["g_prev"], c["t"], c["gval"], c["G"],
                                S.StepParams(), eq=c.get("eq"))
            ok = (sc["branch"] == c["branch"] and np.isclose(sc["alpha"], c["alpha"], rtol=1e-12)
                  and np.isclose(sc["beta"], c["beta"], rtol=1e-12, atol=1e-15))
            if not ok:
                failed.append("golden_scalars:" + c["name"])
                break
    except Exception as e:  # a mutant may also crash
        failed.append("golden_scalars:exception:%s" % e)
    try:
        for c in _golden("projections.json")["cases"]:
            z, A, b = np.array(c["z"]), np.array(c["A"]), np.array(c["b"])
            lam, _ = P.solve_coupled_exact(z, A, b, c["lo"], c["hi"], c.get("C", C))
            x = P.primal_from_dual(z, A, lam, c["lo"], c["hi"])
            if not (np.allclose(lam, c["lam"], rtol=1e-10, atol=1e-12) and np.allclose(x, c["x"], atol=1e-10)):
                failed.append("golden_projection:" + c["name"])
                break
            if A.shape[0] == 1:
                l1 = P.solve_single_exact(z, A[0], b[0], c["lo"], c["hi"], c.get("C", C))
                if not np.isclose(l1, c["lam"][0], rtol=1e-10, atol=1e-12):
                    failed.append("golden_single:" + c["name"])
                    break
                lb, _ = P.solve_single_bisect(z, A[0], b[0], c["lo"], c["hi"], c.get("C", C), tol_B=1e-13)
                if not np.isclose(lb, c["lam"][0], rtol=1e-9, atol=1e-12):
                    failed.append("golden_bisect:" + c["name"])
                    break
    except Exception as e:
        failed.append("golden_projection:exception:%s" % e)
    try:
        c = _golden("full_step.json")
        n = len(c["x"])
        out = S.oracle_step(c["x"], c["x"], c["g"], np.zeros(n), np.zeros(n), c["A"], c["gval"], c["G"],
                            c["t"], S.StepParams(), mode="single")
        if not (np.allclose(out["x_new"], c["x_new"], atol=1e-12) and np.allclose(out["b"], c["b"])):
            failed.append("golden_full_step")
    except Exception as e:
        failed.append("golden_full_step:exception:%s" % e)
    try:
        c = _golden("full_step_t1.json")
        out = S.oracle_step(c["x"], c["x_prev"], c["g"], c["g_prev"], c["d_prev"], c["A"], c["gval"], c["G"],
                            c["t"], S.StepParams(omega=c["omega"]), mode="single")
        if not (np.allclose(out["d"], c["d"], atol=1e-15) and np.allclose(out["z"], c["z"], atol=1e-15)
                and np.allclose(out["x_new"], c["x_new"], atol=1e-14)):
            failed.append("golden_full_step_t1")
    except Exception as e:
        failed.append("golden_full_step_t1:exception:%s" % e)
    try:
        for seed, Cc in [(301, 3.0), (302, 3.0), (103, C), (107, C)]:
            z, A, b = inputs.random_projection(5, 2, seed, feasible=(Cc != 3.0))
            z, A = z.astype(np.float64), A.astype(np.float64)
            _, lam_bf, _ = mod.project_bruteforce(z, A, b, 0.0, 1.0, Cc)
            lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, Cc)
            if not np.allclose(lam, lam_bf, rtol=1e-9, atol=1e-12):
                failed.append("bruteforce:%d" % seed)
                break
    except Exception as e:
        failed.append("bruteforce:exception:%s" % e)
    try:
        # equality rows (Sec. 3.2.4): single row from both sides, and coupled with one
        # equality row, against the brute-force enumeration; Alg. 2 on the coupled case
        for seed, m, side, eq in [(901, 1, 1.0, [True]), (902, 1, -1.0, [True]), (951, 2, 1.0, [True, False]),
                                  (953, 3, 1.0, [False, True, False]), (957, 3, -1.0, [True, False, True])]:
            r = np.random.default_rng(seed)
            z = r.uniform(-0.3, 1.3, 5)
            A = r.uniform(0.2, 1.5, (m, 5))
            b = A @ np.clip(z, 0, 1) + side * 0.3 * A.sum(axis=1) / 5
            _, lam_bf, _ = mod.project_bruteforce(z, A, b, 0.0, 1.0, C, eq=eq)
            lam, _ = P.solve_coupled_exact(z, A, b, 0.0, 1.0, C, eq=eq)
            ok = np.allclose(lam, lam_bf, rtol=1e-9, atol=1e-12)
            if m == 1:
                l1 = P.solve_single_exact(z, A[0], b[0], 0.0, 1.0, C, equality=True)
                lb, _ = P.solve_single_bisect(z, A[0], b[0], 0.0, 1.0, C, tol_B=1e-14, equality=True)
                ok = ok and np.isclose(l1, lam_bf[0], rtol=1e-10, atol=1e-12) and np.isclose(lb, lam_bf[0], rtol=1e-8)
            else:
                l2, inf2 = P.alg2_general_projection(z, A, b, 0.0, 1.0, C, tol_N=1e-12, single="exact", eq=eq)
                # semismooth Newton settles a 5-variable problem in a few steps
                ok = ok and np.allclose(l2, lam_bf, rtol=1e-7, atol=1e-10) and inf2["newton_iters"] <= 20
            if not ok:
                failed.append("equality:%d" % seed)
                break
    except Exception as e:
        failed.append("equality:exception:%s" % e)
    try:
        rng = np.random.default_rng(5)
        z = rng.uniform(-0.3, 1.3, 200)
        A = rng.standard_normal((3, 200))
        b = rng.standard_normal(3)
        lam = np.array([0.05, 0.02, 0.03])
        J = P.jacobian_h(z, A, lam, 0.0, 1.0, 10.0)
        eps = 1e-7
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            fd = -(P.residual(z, A, b, lam + e, 0, 1, 10.0) - P.residual(z, A, b, lam - e, 0, 1, 10.0)) / (2 * eps)
            if not np.allclose(J[:, k], fd, rtol=1e-6, atol=1e-6):
                failed.append("jacobian_fd")
                break
    except Exception as e:
        failed.append("jacobian_fd:exception:%s" % e)
    return failed


MUTANTS = [
    ("step.py", "float(s @ s) / sty", "sty / float(s @ s)"),                      # inverted BB1 ratio
    ("step.py", "2.0 * lip", "lip"),                                               # dropped 2 in 2/L
    ("step.py", "max(float(g @ (g - gp)) / den, 0.0)", "float(g @ (g - gp)) / den"),  # PR instead of PR+
    ("step.py", "t >= p.t_warmup", "t > p.t_warmup"),                              # warm-up boundary
    ("step.py", "sty > p.eps_alpha", "sty > 0.0"),                                 # eps_alpha threshold ignored
    ("step.py", "b = G - gval + A2 @ x", "b = G - gval"),                          # linearisation point dropped
    ("step.py", "z = x + p.omega * alpha * d", "z = x - p.omega * alpha * d"),     # wrong sign of the step
    ("step.py", "-g + beta * np.asarray(d_prev", "-g - beta * np.asarray(d_prev"),  # sign of the CG term
    ("step.py", "z = x + p.omega * alpha * d", "z = x + alpha * d"),              # relaxation omega dropped
    ("step.py", "np.where(E, np.abs(dg), np.maximum(dg, 0.0))", "np.maximum(dg, 0.0)"),  # equality trigger one-sided
    ("projection.py", "np.clip(z - lam * a, lo, hi) - b", "np.clip(z + lam * a, lo, hi) - b"),  # sign in r(lam)
    ("projection.py", "_piecewise_root(z, a, b, lo, hi, 2.0 / C)", "_piecewise_root(z, a, b, lo, hi, 1.0 / C)"),  # 2/C -> 1/C
    ("projection.py", "/ (float(u[free] @ u[free]) + reg)", "/ (float(u[free] @ u[free]) + 0.5 * reg)"),  # regulariser in the piece root
    ("projection.py", "return np.clip(np.asarray(z, dtype=np.float64) - A.T @",
     "return np.clip(np.asarray(z, dtype=np.float64) + A.T @"),                   # sign in x(lam)
    ("projection.py", "Af = A[:, chi]", "Af = A"),                                 # Jacobian ignores the free set
    ("projection.py", "return A @ x - np.asarray(b, dtype=np.float64) - 2.0 * lam / C",
     "return A @ x - np.asarray(b, dtype=np.float64)"),                            # dropped slack term of eq. h
    ("projection.py", "    return -_piecewise_root(z, -a, -b, lo, hi, 2.0 / C)",
     "    return _piecewise_root(z, -a, -b, lo, hi, 2.0 / C)"),                    # equality: mirrored root's sign
    ("projection.py", "    if not equality or r0 == 0.0:\n        return 0.0\n    return -_piecewise_root",
     "    if True:\n        return 0.0\n    return -_piecewise_root"),            # equality read as an inequality
    ("projection.py", "lam = np.where(E, lam, np.maximum(lam, 0.0))", "lam = np.maximum(lam, 0.0)"),  # equality clamped
    ("projection.py", "Dphi = np.diag(((h > 0) | E).astype(np.float64))",
     "Dphi = np.diag((h > 0).astype(np.float64))"),                               # Alg. 2: Phi = h dropped
    ("bruteforce.py", "if np.any(lam[Sineq] < -tol", "if np.any(lam[S] < -tol"),  # pin itself: sign test on equality rows
]


def test_unmutated_oracle_passes_the_pins(tmp_path):
    assert _pins(_load_copy(tmp_path)) == []


@pytest.mark.parametrize("fname,old,new", MUTANTS,
                         ids=lambda v: v if len(v) < 30 else v[:30])
def test_planted_mistake_is_caught(tmp_path, fname, old, new):
    mod = _load_copy(tmp_path, fname, old, new)
    assert _pins(mod), "no pin caught the mistake %r -> %r in %s" % (old, new, fname)
