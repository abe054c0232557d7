"""Seeded synthetic workloads for the PGD-TO step (shared by the tests, the bench and smoke).

This module holds no arithmetic of the optimizer: it only draws the arrays a
finite-element code would hand to the step (design x, objective gradient, constraint
rows and values) with the shapes and value distributions of the paper's four
benchmark problems (Sec. 4.1), in FP64, and casts them to FP32.  Both the CUDA path
and the oracle read the same FP32 arrays.

Workloads (seed = 20251113 + index):
  1  volume-constrained compliance, 2D 256x128 quads, n = 32768, one linear row
  2  compliance-constrained volume, 3D 128x64x64 hexes, n = 524288, one nonlinear row
     (synthetic compliance g(x) = sum_e s_e (1 - x_e^3), regenerated each step)
  3  four materials on 3D 192x96x96, n = 4 x 1769472, four independent volume rows
  4  volume + three first-moment (centre of mass) rows on 3D 256x128x128, n = 4194304
  5  serving stream of step requests with log-uniform n and m in {1, 2, 4}
Smaller meshes of the same kind are produced by passing ``dims``.
"""

from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20251113

FULL_DIMS = {
    1: (256, 128),
    2: (128, 64, 64),
    3: (192, 96, 96),
    4: (256, 128, 128),
}


def _rng(config, seed_offset=0):
    return np.random.default_rng(SEED_BASE + config + seed_offset)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _prior_state(rng, x, g_of_x, lo, hi):
    """A seeded 'previous iterate': x_prev = clip(x + 0.01 N(0,1)), its gradient, d_prev = -g_prev."""
    x_prev = np.clip(x + 0.01 * rng.standard_normal(x.shape), lo, hi)
    g_prev = g_of_x(x_prev)
    return x_prev, g_prev, -g_prev


def config1(dims=None, seed_offset=0):
    """Single linear volume row, 2D mesh: x ~ U(0.2, 0.8), g = -3 x^2 s, s ~ lognormal(0, 1),
    a = 1, G = 0.4 n, one prior step (t = 1)."""
    dims = dims or FULL_DIMS[1]
    n = int(np.prod(dims))
    rng = _rng(1, seed_offset)
    x = rng.uniform(0.2, 0.8, n)
    s = rng.lognormal(0.0, 1.0, n)

    def grad(xx):
        return -3.0 * xx * xx * s

    x_prev, g_prev, d_prev = _prior_state(rng, x, grad, 0.0, 1.0)
    x32 = _f32(x)
    a = np.ones((1, n), dtype=np.float32)
    # a linear row passes g_j(x_t) = a_j^T x_t
    gval = np.array([float(np.sum(x32, dtype=np.float64))])
    return {
        "name": "volume_2d_%dx%d" % dims, "config": 1, "n": n, "m": 1, "mode": "single",
        "lo": 0.0, "hi": 1.0, "t": 1,
        "x": x32, "x_prev": _f32(x_prev), "g": _f32(grad(x)), "g_prev": _f32(g_prev),
        "d_prev": _f32(d_prev), "A": a, "gval": gval, "G": np.array([0.4 * n]),
    }


class ComplianceSurrogate:
    """Synthetic stand-in for the FEA of workload 2: g(x) = sum_e s_e (1 - x_e^3).

    Its gradient -3 x^2 s is the constraint row; its value is the row's g_j(x_t).
    The objective (total volume) has gradient 1 everywhere.
    """

    def __init__(self, s):
        self.s = np.asarray(s, dtype=np.float64)

    def value(self, x):
        x = np.asarray(x, dtype=np.float64)
        return float(np.sum(self.s * (1.0 - x * x * x)))

    def row(self, x):
        x = np.asarray(x, dtype=np.float64)
        return -3.0 * x * x * self.s


def config2(dims=None, seed_offset=0):
    """Min volume under the synthetic compliance row; x0 ~ U(0.2, 0.8), s ~ lognormal(0, 1.5),
    G = g(x0) / 1.05 (x0 is 5% infeasible).  Runs from t = 0 for 50 steps."""
    dims = dims or FULL_DIMS[2]
    n = int(np.prod(dims))
    rng = _rng(2, seed_offset)
    x0 = _f32(rng.uniform(0.2, 0.8, n))
    s = _f32(rng.lognormal(0.0, 1.5, n))
    sur = ComplianceSurrogate(s)
    G = sur.value(x0) / 1.05
    return {
        "name": "min_volume_3d_%dx%dx%d" % dims, "config": 2, "n": n, "m": 1, "mode": "single",
        "lo": 0.0, "hi": 1.0, "t": 0, "steps": 50,
        "x": x0, "s": s, "g": np.ones(n, dtype=np.float32), "surrogate": sur,
        "G": np.array([G]),
    }


def config2_inputs(cfg, x):
    """The step inputs workload 2's FEA stand-in hands over at design x: (A, gval)."""
    sur = cfg["surrogate"]
    x32 = np.asarray(x, dtype=np.float32)
    return _f32(sur.row(x32))[None, :], np.array([sur.value(x32)])


def config3(dims=None, seed_offset=0, materials=4):
    """Four materials, independent volume rows: x ~ U(0, 0.5), g = -lognormal(0, 1), a = 1,
    G_j = f_j * n_seg with f = 0.10/0.08/0.06/0.04, material-major segments, t = 1."""
    dims = dims or FULL_DIMS[3]
    n_seg = int(np.prod(dims))
    n = n_seg * materials
    rng = _rng(3, seed_offset)
    x = rng.uniform(0.0, 0.5, n)
    gmag = rng.lognormal(0.0, 1.0, n)
    g = -gmag
    x_prev = np.clip(x + 0.01 * rng.standard_normal(n), 0.0, 1.0)
    g_prev = -gmag * np.exp(0.05 * rng.standard_normal(n))
    x32 = _f32(x)
    seg = np.arange(materials + 1, dtype=np.int64) * n_seg
    fr = np.array([0.10, 0.08, 0.06, 0.04])[:materials]
    gval = np.array([float(np.sum(x32[seg[j]:seg[j + 1]], dtype=np.float64)) for j in range(materials)])
    return {
        "name": "multimaterial_3d_%dx%dx%d_x%d" % (dims + (materials,)), "config": 3, "n": n,
        "m": materials, "mode": "independent", "lo": 0.0, "hi": 1.0, "t": 1,
        "x": x32, "x_prev": _f32(x_prev), "g": _f32(g), "g_prev": _f32(g_prev),
        "d_prev": _f32(-g_prev), "A": np.ones(n, dtype=np.float32), "seg": seg,
        "gval": gval, "G": fr * n_seg,
    }


def config4(dims=None, seed_offset=0, infeasible=False):
    """Volume + first-moment rows on a 3D box mesh: rows a_0 = v, a_k = v (c_k - t_k);
    G_0 = 0.3 sum v, G_k = r sum v with r = 0.01 (longest side 1, element size 1/nx).
    The feasible seed draws the target t inside the domain; the infeasible seed puts
    t_1 below the domain (all a_1 > 0) with G_1 = -r sum v, so no x >= 0 satisfies row 1.
    Design x ~ U(0.2, 0.8), g = -3 x^2 s with s ~ lognormal(0, 1), one prior step."""
    dims = dims or FULL_DIMS[4]
    nx, ny, nz = dims
    n = nx * ny * nz
    rng = _rng(4, seed_offset + (100 if infeasible else 0))
    h = 1.0 / nx
    cx = (np.arange(nx) + 0.5) * h
    cy = (np.arange(ny) + 0.5) * h
    cz = (np.arange(nz) + 0.5) * h
    CX, CY, CZ = np.meshgrid(cx, cy, cz, indexing="ij")
    cent = [CX.ravel(), CY.ravel(), CZ.ravel()]
    ext = [nx * h, ny * h, nz * h]
    t = np.array([rng.uniform(0.2, 0.4) * ext[0], rng.uniform(0.2, 0.4) * ext[1],
                  rng.uniform(0.6, 0.8) * ext[2]])
    v = np.ones(n)
    r = 0.01
    G = np.array([0.3 * n, r * n, r * n, r * n])
    if infeasible:
        t[1] = -0.1 * ext[1]
        G[2] = -r * n
    A = np.stack([v] + [v * (cent[k] - t[k]) for k in range(3)])
    x = rng.uniform(0.2, 0.8, n)
    s = rng.lognormal(0.0, 1.0, n)

    def grad(xx):
        return -3.0 * xx * xx * s

    x_prev, g_prev, d_prev = _prior_state(rng, x, grad, 0.0, 1.0)
    x32 = _f32(x)
    A32 = _f32(A)
    gval = A32.astype(np.float64) @ x32.astype(np.float64)
    return {
        "name": "volume_com_3d_%dx%dx%d%s" % (nx, ny, nz, "_infeasible" if infeasible else ""),
        "config": 4, "n": n, "m": 4, "mode": "coupled", "lo": 0.0, "hi": 1.0, "t": 1,
        "x": x32, "x_prev": _f32(x_prev), "g": _f32(grad(x)), "g_prev": _f32(g_prev),
        "d_prev": _f32(d_prev), "A": A32, "gval": gval, "G": G, "target": t,
    }


def random_projection(n, m, seed, coupled=True, feasible=True, zspread=0.3, lo=0.0, hi=1.0):
    """A generic projection problem (z, A, b) for edge-case and small parity tests.

    z ~ U(lo - zspread, hi + zspread); coupled rows are dense with entries ~ N(0, 1) plus
    an offset so rows are not orthogonal; b is set from a random box point so that the
    problem is feasible, or pushed below the row minimum when ``feasible`` is False.
    """
    rng = np.random.default_rng(seed)
    z = rng.uniform(lo - zspread, hi + zspread, n)
    if coupled:
        A = rng.standard_normal((m, n)) + 0.5
    else:
        A = np.abs(rng.standard_normal((m, n))) + 0.1
    xin = rng.uniform(lo, hi, n)
    b = A @ xin - 0.2 * np.abs(A) @ np.full(n, 0.5 * (hi - lo)) * rng.uniform(0.0, 1.0, m)
    if not feasible:
        rowmin = np.minimum(A * lo, A * hi).sum(axis=1)
        b[0] = rowmin[0] - 0.1 * abs(rowmin[0]) - 1.0
    return _f32(z), _f32(A), b


def serving_requests(count=2048, seed_offset=0, n_min=4096, n_max=4 * 1024 * 1024):
    """Workload 5: request descriptors with log-uniform n, m in {1, 2, 4} and a per-request seed.

    Half of the m > 1 requests have independent rows (equal segments), half coupled.
    Arrival times are drawn later from a Poisson process at the chosen rate.
    """
    rng = _rng(5, seed_offset)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        m = int(rng.choice([1, 2, 4]))
        mode = "single" if m == 1 else ("independent" if rng.uniform() < 0.5 else "coupled")
        if mode == "independent":
            n = max(m, (n // m) * m)
        out.append({"id": i, "n": n, "m": m, "mode": mode, "seed": SEED_BASE + 1000 + i})
    return out


def request_problem(req):
    """Inputs of one serving request (same recipes as workloads 1, 3 and 4, size req['n'])."""
    rng = np.random.default_rng(req["seed"])
    n, m, mode = req["n"], req["m"], req["mode"]
    x = rng.uniform(0.2, 0.8, n)
    s = rng.lognormal(0.0, 1.0, n)
    g = -3.0 * x * x * s
    x_prev = np.clip(x + 0.01 * rng.standard_normal(n), 0.0, 1.0)
    g_prev = -3.0 * x_prev * x_prev * s
    x32 = _f32(x)
    out = {"n": n, "m": m, "mode": mode, "lo": 0.0, "hi": 1.0, "t": 1, "x": x32,
           "x_prev": _f32(x_prev), "g": _f32(g), "g_prev": _f32(g_prev), "d_prev": _f32(-g_prev)}
    if mode == "single":
        out["A"] = np.ones((1, n), dtype=np.float32)
        out["gval"] = np.array([float(np.sum(x32, dtype=np.float64))])
        out["G"] = np.array([0.4 * n])
    elif mode == "independent":
        n_seg = n // m
        seg = np.arange(m + 1, dtype=np.int64) * n_seg
        out["A"] = np.ones(n, dtype=np.float32)
        out["seg"] = seg
        out["gval"] = np.array([float(np.sum(x32[seg[j]:seg[j + 1]], dtype=np.float64)) for j in range(m)])
        out["G"] = np.linspace(0.45, 0.35, m) * n_seg
    else:
        pos = rng.uniform(0.0, 1.0, (m - 1, n))
        tgt = rng.uniform(0.2, 0.4, m - 1)
        A = np.vstack([np.ones((1, n)), pos - tgt[:, None]])
        A32 = _f32(A)
        out["A"] = A32
        out["gval"] = A32.astype(np.float64) @ x32.astype(np.float64)
        out["G"] = np.concatenate([[0.35 * n], np.full(m - 1, 0.01 * n)])
    return out
