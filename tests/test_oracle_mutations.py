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
                                S.StepParams())
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
    ("projection.py", "np.clip(z - lam * a, lo, hi) - b", "np.clip(z + lam * a, lo, hi) - b"),  # sign in r(lam)
    ("projection.py", "_piecewise_root(z, a, b, lo, hi, 2.0 / C)", "_piecewise_root(z, a, b, lo, hi, 1.0 / C)"),  # 2/C -> 1/C
    ("projection.py", "/ (float(u[free] @ u[free]) + reg)", "/ (float(u[free] @ u[free]) + 0.5 * reg)"),  # regulariser in the piece root
    ("projection.py", "return np.clip(np.asarray(z, dtype=np.float64) - A.T @",
     "return np.clip(np.asarray(z, dtype=np.float64) + A.T @"),                   # sign in x(lam)
    ("projection.py", "Af = A[:, chi]", "Af = A"),                                 # Jacobian ignores the free set
    ("projection.py", "return A @ x - np.asarray(b, dtype=np.float64) - 2.0 * lam / C",
     "return A @ x - np.asarray(b, dtype=np.float64)"),                            # dropped slack term of eq. h
]


def test_unmutated_oracle_passes_the_pins(tmp_path):
    assert _pins(_load_copy(tmp_path)) == []


@pytest.mark.parametrize("fname,old,new", MUTANTS,
                         ids=lambda v: v if len(v) < 30 else v[:30])
def test_planted_mistake_is_caught(tmp_path, fname, old, new):
    mod = _load_copy(tmp_path, fname, old, new)
    assert _pins(mod), "no pin caught the mistake %r -> %r in %s" % (old, new, fname)
