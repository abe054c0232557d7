"""KKT residuals and parity metrics (test infrastructure; see package docstring).

KKT system of the regularised projection: App. A.3.2 (rkkt1-rkkt11), restated for
lam = -y and x = z + delta:
  stationarity   x = clip(z - A^T lam, lo, hi)             (rkkt5, rkkt7, rkkt8)
  primal         r_j = a_j^T x - b_j - 2 lam_j / C <= 0     (rkkt1 with s_j = 2 lam_j / C)
  dual           lam_j >= 0                                  (rkkt11)
  complementary  lam_j r_j = 0                               (rkkt9)
"""

from __future__ import annotations

import numpy as np

from .projection import eq_mask, primal_from_dual, row_scale


def kkt_report(z, A, b, lam, x, lo, hi, C, eq=None):
    """Scaled KKT residuals of (x, lam); 'worst' is their maximum.

    Row quantities are divided by max(1, |b_j|, sum_i |a_ji x_i|); the complementarity
    residual is |lam_j r_j| divided by that scale times max(1, lam_j).  An equality row
    (``eq``, Sec. 3.2.4) must have r_j = 0 and may have either sign of lam_j.
    """
    z = np.asarray(z, dtype=np.float64)
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    b = np.asarray(b, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    scale = row_scale(A, b, x)
    r = A @ x - b - 2.0 * lam / C
    E = eq_mask(eq, A.shape[0])
    rep = {
        "stationarity": float(np.max(np.abs(x - primal_from_dual(z, A, lam, lo, hi)), initial=0.0)),
        "box": float(max(np.max(lo - x, initial=0.0), np.max(x - hi, initial=0.0), 0.0)),
        "primal": float(np.max(np.where(E, np.abs(r), np.maximum(r, 0.0)) / scale)),
        "dual": float(np.max(np.where(E, 0.0, np.maximum(-lam, 0.0)))),
        "complementarity": float(np.max(np.where(E, 0.0, np.abs(lam * r) / (scale * np.maximum(1.0, lam))))),
    }
    rep["worst"] = max(rep.values())
    return rep


def lambda_floor(A, lo, hi):
    """lam_floor_j = 1e-3 (hi - lo) / max_i |a_ji|: the scale below which lam_j counts as zero."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    amax = np.max(np.abs(A), axis=1)
    amax[amax == 0] = 1.0
    return 1e-3 * (hi - lo) / amax


def parity_errors(x_dev, lam_dev, x_ref, lam_ref, A, b, C, lo, hi, amax=None, eq=None):
    """Error of a device result against the oracle, per result.

    lam_rel   max_j |lam_dev - lam_ref| / max(|lam_ref|, lam_floor_j)
    x_abs     max_i |x_dev - x_ref|
    viol_rel  active rows (lam_ref > 0, and every equality row of ``eq``):
              |a_j^T x_dev - b_j - 2 lam_dev_j / C| / den_j;
              inactive rows: max(a_j^T x_dev - b_j, 0) / den_j;
              den_j = max(|b_j|, sum_i |a_ji x_dev_i|)
    ``A`` may be an (m, n) array, or a callable returning (A x, |A| |x|) for a vector x
    (used for the segmented layout without forming the dense matrix).
    ``amax`` overrides max_i |a_ji| for lam_floor when A is a callable.
    """
    x_dev = np.asarray(x_dev, dtype=np.float64)
    x_ref = np.asarray(x_ref, dtype=np.float64)
    lam_dev = np.atleast_1d(np.asarray(lam_dev, dtype=np.float64))
    lam_ref = np.atleast_1d(np.asarray(lam_ref, dtype=np.float64))
    b = np.atleast_1d(np.asarray(b, dtype=np.float64))
    if callable(A):
        ax, absax = A(x_dev)
        floor = 1e-3 * (hi - lo) / np.asarray(amax, dtype=np.float64)
    else:
        A2 = np.atleast_2d(np.asarray(A, dtype=np.float64))
        ax = A2 @ x_dev
        absax = np.abs(A2) @ np.abs(x_dev)
        floor = lambda_floor(A2, lo, hi)
    den = np.maximum(np.abs(b), absax)
    den[den == 0] = 1.0
    active = (lam_ref > 0) | eq_mask(eq, lam_ref.size)
    viol = np.where(active, np.abs(ax - b - 2.0 * lam_dev / C), np.maximum(ax - b, 0.0)) / den
    return {
        "lam_rel": float(np.max(np.abs(lam_dev - lam_ref) / np.maximum(np.abs(lam_ref), floor))),
        "x_abs": float(np.max(np.abs(x_dev - x_ref), initial=0.0)),
        "viol_rel": float(np.max(viol)),
        "lam_rel_per_row": (np.abs(lam_dev - lam_ref) / np.maximum(np.abs(lam_ref), floor)).tolist(),
        "viol_rel_per_row": viol.tolist(),
    }
