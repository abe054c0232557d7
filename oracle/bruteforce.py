"""Brute-force active-pattern enumeration for tiny projections (test infrastructure).

A pin, not a solver: it uses only the textbook KKT conditions of the convex QP

    min_x ||x - z||^2 + (C/2)||s||^2  s.t.  lo <= x <= hi,  A x - s <= b,  s >= 0

and none of the paper's dual machinery.  For every box pattern (each x_i at lo, free
or at hi) and every set S of rows taken as active, the stationarity conditions
x_F = z_F - A_SF^T lam_S and the active rows a_j^T x - b_j - 2 lam_j / C = 0 form a
linear system in lam_S.  A pattern whose solution satisfies every sign and
consistency condition is a KKT point; the QP is strictly convex, so there is exactly
one and it is the optimum.  Cost 3^n 2^m small solves: n <= 8 only.

Equality rows (Sec. 3.2.4) are rows a_j^T x - s_j = b_j with a free slack: they are in
every active set and their multiplier has no sign condition.
"""

from __future__ import annotations

import itertools

import numpy as np


def project_bruteforce(z, A, b, lo, hi, C, tol=1e-10, eq=None):
    """Return (x, lam, n_kkt_points) for the regularised projection of z; n <= 8.
    ``eq``: boolean mask of equality rows (None: every row is an inequality)."""
    z = np.asarray(z, dtype=np.float64)
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    if n > 8:
        raise ValueError("brute force is limited to n <= 8")
    E = np.zeros(m, dtype=bool) if eq is None else np.asarray(eq, dtype=bool)
    ineq = [j for j in range(m) if not E[j]]
    found = []
    for k in range(len(ineq) + 1):
        for Si in itertools.combinations(ineq, k):
            S = sorted(set(Si) | set(np.flatnonzero(E).tolist()))
            Sineq = list(Si)
            for pattern in itertools.product((0, 1, 2), repeat=n):
                pat = np.array(pattern)
                F = pat == 1
                xfix = np.where(pat == 0, lo, hi).astype(np.float64)
                lam = np.zeros(m)
                if S:
                    As = A[S]
                    M = As[:, F] @ As[:, F].T + (2.0 / C) * np.eye(len(S))
                    rhs = As[:, F] @ z[F] + As[:, ~F] @ xfix[~F] - b[S]
                    try:
                        lam[S] = np.linalg.solve(M, rhs)
                    except np.linalg.LinAlgError:
                        continue
                w = z - A.T @ lam
                x = np.where(F, w, xfix)
                # slack for rounding: w carries the error of A^T lam, rows that of |A||x|
                tw = tol + 1e-14 * float(np.max(np.abs(A.T @ lam), initial=0.0))
                if np.any(lam[Sineq] < -tol * max(1.0, float(np.max(np.abs(lam))))):
                    continue
                if np.any(w[F] < lo - tw) or np.any(w[F] > hi + tw):
                    continue
                if np.any(w[pat == 0] > lo + tw) or np.any(w[pat == 2] < hi - tw):
                    continue
                r = A @ x - b - 2.0 * lam / C
                inactive = ~E
                inactive[S] = False
                rs = np.maximum(1.0, np.maximum(np.abs(b), np.abs(A) @ np.abs(x)))
                if np.any(r[inactive] > tol * rs[inactive]):
                    continue
                found.append((x, lam))
    if not found:
        raise RuntimeError("no KKT point found")
    x0, l0 = found[0]
    for x, lam in found[1:]:
        if np.max(np.abs(x - x0)) > 1e-8 or np.max(np.abs(lam - l0)) > 1e-8 * max(1.0, np.max(np.abs(l0))):
            raise RuntimeError("two different KKT points: the QP should be strictly convex")
    return x0, l0, len(found)
