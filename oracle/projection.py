"""Regularised dual projection in FP64 (test infrastructure; see package docstring).

Paper sections followed here:
  * Thm 1 / Thm 2 and eq. delta_y_robust -- the solution form x(lam) = clip(z - A^T lam, lo, hi);
  * eq. h -- the row residual, written r_j(lam) = a_j^T x(lam) - b_j - 2 lam_j / C (lam = -y);
  * eq. reg_jacobian -- J_h = A D(y) A^T + (2/C) I, D = indicator of the free set;
  * eq. phi -- the semismooth residual Phi and its generalised Jacobian (App. A.3.3);
  * Alg. 1 -- bisection on one constraint; Sec. 3.2.2 -- independent rows;
  * Alg. 2 -- stage 1 single-row candidates, stage 2 semismooth Newton with line search.

The "exact" solvers compute the unique optimum that the paper's iterations converge
to (Thm 2 states it is unique); the parity tests compare the CUDA path with them.
The "paper" solvers (Alg. 1 bisection, Alg. 2) follow the printed algorithms step by
step and are what the CPU baseline times.
"""

from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------- basics

def primal_from_dual(z, A, lam, lo, hi):
    """x(lam) = clip(z - A^T lam, lo, hi): Thm 2 / eq. delta_y_robust with x = z + delta, lam = -y."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    return np.clip(np.asarray(z, dtype=np.float64) - A.T @ np.asarray(lam, dtype=np.float64), lo, hi)


def residual(z, A, b, lam, lo, hi, C):
    """r_j(lam) = a_j^T x(lam) - b_j - 2 lam_j / C  (eq. h with y = -lam).

    r_j <= 0 is the regularised row j; r is strictly decreasing in lam because its
    Jacobian is -(A D A^T + (2/C) I) (eq. reg_jacobian).
    """
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    lam = np.asarray(lam, dtype=np.float64)
    x = primal_from_dual(z, A, lam, lo, hi)
    return A @ x - np.asarray(b, dtype=np.float64) - 2.0 * lam / C


def free_set(z, A, lam, lo, hi):
    """chi_i(y): 1 where lo <= z_i - (A^T lam)_i <= hi, inclusive as in eq. delta_y_robust."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    w = np.asarray(z, dtype=np.float64) - A.T @ np.asarray(lam, dtype=np.float64)
    return (w >= lo) & (w <= hi)


def jacobian_h(z, A, lam, lo, hi, C):
    """J_h(y) = A D(y) A^T + (2/C) I  (eq. reg_jacobian); dh/dy, so dr/dlam = -J_h."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    chi = free_set(z, A, lam, lo, hi)
    Af = A[:, chi]
    return Af @ Af.T + (2.0 / C) * np.eye(A.shape[0])


def eq_mask(eq, m):
    """Boolean mask of the equality rows among m rows (Sec. 3.2.4); None: all inequalities."""
    out = np.zeros(m, dtype=bool)
    if eq is not None:
        out[:] = np.asarray(eq, dtype=bool)
    return out


def phi(h, y, eq=None):
    """Phi_j(y) = max(h_j, 0) + sign(max(-h_j, 0)) * y_j  (eq. phi); for an equality row
    Phi_j = h_j, the row being always active (Sec. 3.2.4)."""
    h = np.asarray(h, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.maximum(h, 0.0) + np.sign(np.maximum(-h, 0.0)) * y
    E = eq_mask(eq, h.size)
    out[E] = h[E]
    return out


def row_scale(A, b, x):
    """Per-row magnitude max(1, |b_j|, sum_i |a_ji x_i|) used to make tolerances relative."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    return np.maximum.reduce([np.ones(A.shape[0]), np.abs(np.asarray(b, dtype=np.float64)),
                              np.abs(A) @ np.abs(np.asarray(x, dtype=np.float64))])


# --------------------------------------------------------------------------- one row

def _r1(z, a, b, lo, hi, C, lam):
    """Single-row residual r(lam) = a^T clip(z - lam a) - b - 2 lam / C (App. A.2 with eq. h)."""
    return float(a @ np.clip(z - lam * a, lo, hi) - b - 2.0 * lam / C)


def _saturation_bound(z, a, lo, hi):
    """lam_hi = max(0, max_i max((z_i - lo)/a_i, (z_i - hi)/a_i)) over a_i != 0.

    Alg. 1's lower bracket y_l written for lam = -y.  Rows with a_i = 0 never move and
    are skipped.  For lam >= lam_hi every element sits at the bound that minimises
    a_i x_i, so r(lam) is linear there (only the -2 lam / C term changes).
    """
    nz = a != 0
    if not np.any(nz):
        return 0.0
    t1 = (z[nz] - lo) / a[nz]
    t2 = (z[nz] - hi) / a[nz]
    return max(0.0, float(np.max(np.maximum(t1, t2))))


def _piecewise_root(w, u, c, lo, hi, reg):
    """Unique root gamma > 0 of psi(gamma) = u^T clip(w - gamma u, lo, hi) - c - reg gamma, psi(0) > 0.

    psi is piecewise linear and strictly decreasing (reg > 0), with breakpoints
    (w_i - hi)/u_i and (w_i - lo)/u_i.  The breakpoints above 0 are sorted, the piece
    holding the sign change is found by binary search over them, and on that piece,
    where the free set F is fixed, psi is linear and its root is
        gamma = (sum_{clipped} u_i x_i + sum_F u_i w_i - c) / (sum_F u_i^2 + reg).
    """
    def psi(gam):
        return float(u @ np.clip(w - gam * u, lo, hi) - c - reg * gam)

    nz = u != 0
    bps = np.concatenate([(w[nz] - lo) / u[nz], (w[nz] - hi) / u[nz]])
    bps = np.unique(bps[bps > 0.0])
    # invariant: psi(bps[i]) > 0 for i < left_i, psi(bps[i]) <= 0 for i >= right_i
    left_i, right_i = 0, len(bps)
    while left_i < right_i:
        mid = (left_i + right_i) // 2
        if psi(float(bps[mid])) > 0.0:
            left_i = mid + 1
        else:
            right_i = mid
    left = 0.0 if left_i == 0 else float(bps[left_i - 1])
    right = float(bps[left_i]) if left_i < len(bps) else None
    probe = left + 1.0 if right is None else 0.5 * (left + right)
    v = w - probe * u
    free = (v >= lo) & (v <= hi) & nz
    clipped = ~free
    const = float(u[clipped] @ np.clip(v[clipped], lo, hi))
    gam = (const + float(u[free] @ w[free]) - c) / (float(u[free] @ u[free]) + reg)
    # the root lies on [left, right]; rounding may put it a hair outside
    if right is not None:
        return min(max(gam, left), right)
    return max(gam, left)


def solve_single_exact(z, a, b, lo, hi, C, equality=False):
    """Exact root of the regularised single-row dual equation (App. A.2 + eq. h).

    r(lam) = a^T clip(z - lam a) - b - 2 lam / C is piecewise linear and strictly
    decreasing with breakpoints (z_i - hi)/a_i and (z_i - lo)/a_i (the continuous
    quadratic knapsack the paper credits to Pardalos & Kovoor).  If r(0) <= 0 the row
    is inactive and lam = 0 (Alg. 1's feasibility test); otherwise the root is found
    exactly on its linear piece (_piecewise_root).  Past the last breakpoint the free
    set is empty and the root is lam = (C/2)(S_min - b).

    An equality row (Sec. 3.2.4) is always active: lam ranges over R and r(lam) = 0.
    When r(0) < 0 the root is negative.  With mu = -lam, r(-mu) = -psi(mu) where psi is
    the residual of the mirrored row (-a, -b), which is positive at 0, so the root is
    minus the mirrored row's (positive) root.
    """
    z = np.asarray(z, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = float(b)
    r0 = _r1(z, a, b, lo, hi, C, 0.0)
    if r0 > 0.0:
        return _piecewise_root(z, a, b, lo, hi, 2.0 / C)
    if not equality or r0 == 0.0:
        return 0.0
    return -_piecewise_root(z, -a, -b, lo, hi, 2.0 / C)


def solve_single_bisect(z, a, b, lo, hi, C, tol_B=1e-8, rel_tol=0.0, max_iter=100000, equality=False):
    """Alg. 1 (single-constraint bisection) written for lam = -y, regularised as eq. h.

    Steps, in the paper's order: test lam = 0 (delta(0) feasible -> return 0); bracket
    [0, lam_hi] with lam_hi from Alg. 1's y_l; halve until the bracket is at most
    max(tol_B, rel_tol * lam_hi_current) wide; return the midpoint.  When even the
    saturated point violates the row, r is linear beyond lam_hi and its root
    (C/2)(S_min - b) is returned directly (the regularised reading of the bracket).
    An equality row (Sec. 3.2.4) with r(0) < 0 runs the same steps on the mirrored row
    (-a, -b) and returns minus its root (see solve_single_exact).
    Returns (lam, number_of_halvings).
    """
    z = np.asarray(z, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = float(b)
    r0 = _r1(z, a, b, lo, hi, C, 0.0)
    if r0 <= 0.0:
        if not equality or r0 == 0.0:
            return 0.0, 0
        lam, it = solve_single_bisect(z, -a, -b, lo, hi, C, tol_B, rel_tol, max_iter)
        return -lam, it
    lam_lo = 0.0
    lam_hi = _saturation_bound(z, a, lo, hi)
    if _r1(z, a, b, lo, hi, C, lam_hi) > 0.0:
        s_min = float(a @ np.clip(z - lam_hi * a, lo, hi))
        return 0.5 * C * (s_min - b), 0
    it = 0
    while lam_hi - lam_lo > max(tol_B, rel_tol * lam_hi) and it < max_iter:
        mid = 0.5 * (lam_lo + lam_hi)
        if _r1(z, a, b, lo, hi, C, mid) > 0.0:
            lam_lo = mid
        else:
            lam_hi = mid
        it += 1
    return 0.5 * (lam_lo + lam_hi), it


def solve_independent_exact(z, a, seg, b, lo, hi, C, eq=None):
    """Sec. 3.2.2: rows with disjoint supports seg[j]:seg[j+1] are m separate single-row solves.

    ``a`` holds one coefficient per variable (the value of the row that owns it).
    Variables outside every segment (none in the shipped workloads) are only clipped.
    ``eq`` marks equality rows (Sec. 3.2.4).
    """
    seg = [int(s) for s in seg]
    E = eq_mask(eq, len(seg) - 1)
    lam = np.zeros(len(seg) - 1)
    for j in range(len(seg) - 1):
        s, e = seg[j], seg[j + 1]
        lam[j] = solve_single_exact(z[s:e], a[s:e], b[j], lo, hi, C, equality=bool(E[j]))
    return lam


def solve_independent_bisect(z, a, seg, b, lo, hi, C, tol_B=1e-8, rel_tol=0.0, eq=None):
    """Sec. 3.2.2 with Alg. 1 per row; returns (lam, halvings per row)."""
    seg = [int(s) for s in seg]
    E = eq_mask(eq, len(seg) - 1)
    lam = np.zeros(len(seg) - 1)
    its = []
    for j in range(len(seg) - 1):
        s, e = seg[j], seg[j + 1]
        lam[j], it = solve_single_bisect(z[s:e], a[s:e], b[j], lo, hi, C, tol_B, rel_tol, equality=bool(E[j]))
        its.append(it)
    return lam, its


def independent_primal(z, a, seg, lam, lo, hi):
    """x_i = clip(z_i - lam_{row(i)} a_i, lo, hi) for the segmented layout."""
    z = np.asarray(z, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    shift = np.zeros_like(z)
    for j in range(len(seg) - 1):
        s, e = int(seg[j]), int(seg[j + 1])
        shift[s:e] = lam[j] * a[s:e]
    return np.clip(z - shift, lo, hi)


def segmented_to_dense(a, seg, n):
    """Dense m x n row matrix equivalent of the segmented layout (for checks on small n)."""
    m = len(seg) - 1
    A = np.zeros((m, n))
    for j in range(m):
        s, e = int(seg[j]), int(seg[j + 1])
        A[j, s:e] = a[s:e]
    return A


# --------------------------------------------------------------------------- coupled rows

def _newton_stage2(z, A, b, lo, hi, C, y0, tol, maxiter, c1=1e-4, c2=0.9, eq=None):
    """Alg. 2 stage 2: semismooth Newton on Phi(y) with a backtracking line search on M.

    Each iteration: h(y) (eq. h), Phi (eq. phi), J_h (eq. reg_jacobian),
    J_Phi = D_Phi J_h + I - D_Phi (App. A.3.3), solve J_Phi Delta = Phi, then the
    largest gamma in {1, 1/2, ..., 2^-40} with M(y_new) <= M(y) - c1 gamma grad M^T Delta,
    where grad M^T Delta = ||Phi||^2 (App. A.3.3).  y_new = min(y - gamma Delta, 0): the
    clamp keeps the iterate dual feasible (reading of eq. phi, whose roots with y_j > 0
    are not KKT points).  The curvature condition with c2 is evaluated and recorded
    only.  Stops when ||Phi||_inf <= tol * scale_j row by row or after maxiter.
    Equality rows (Sec. 3.2.4): Phi_j = h_j, its row of J_Phi is J_h's, and y_j is not
    clamped.
    Returns (y, iterations, converged, curvature_failures).
    """
    m = A.shape[0]
    E = eq_mask(eq, m)

    def clamp(v):
        return np.where(E, v, np.minimum(v, 0.0))

    y = clamp(np.asarray(y0, dtype=np.float64).copy())
    curv_fail = 0
    for k in range(maxiter + 1):
        lam = -y
        h = residual(z, A, b, lam, lo, hi, C)
        Ph = phi(h, y, E)
        scale = row_scale(A, b, primal_from_dual(z, A, lam, lo, hi))
        if np.all(np.abs(Ph) <= tol * scale):
            return y, k, True, curv_fail
        if k == maxiter:
            break
        Jh = jacobian_h(z, A, lam, lo, hi, C)
        Dphi = np.diag(((h > 0) | E).astype(np.float64))
        Jphi = Dphi @ Jh + np.eye(m) - Dphi
        Delta = np.linalg.solve(Jphi, Ph)
        M0 = 0.5 * float(Ph @ Ph)
        slope = float(Ph @ Ph)
        gamma = 1.0
        accepted = None
        for _ in range(41):
            y_new = clamp(y - gamma * Delta)
            h_new = residual(z, A, b, -y_new, lo, hi, C)
            P_new = phi(h_new, y_new, E)
            if 0.5 * float(P_new @ P_new) <= M0 - c1 * gamma * slope:
                accepted = y_new
                # curvature condition of App. A.3.3, recorded only
                Jh_n = jacobian_h(z, A, -y_new, lo, hi, C)
                D_n = np.diag(((h_new > 0) | E).astype(np.float64))
                J_n = D_n @ Jh_n + np.eye(m) - D_n
                if float((J_n.T @ P_new) @ Delta) > c2 * slope:
                    curv_fail += 1
                break
            gamma *= 0.5
        if accepted is None:
            # no decrease found on the grid: keep the smallest clamped step and go on
            accepted = clamp(y - gamma * Delta)
        y = accepted
    return y, maxiter, False, curv_fail


def _polish_pattern(z, A, b, lo, hi, C, lam):
    """Solve the linear KKT system on the active pattern read off lam (rows lam_j > 0, free set F).

    (A_SF A_SF^T + (2/C) I) lam_S = A_SF z_F + A_S,notF x_fixed - b_S.  Exact on the
    right pattern; the caller keeps it only if the KKT check passes.
    """
    m, n = A.shape
    S = np.flatnonzero(lam > 0)
    if len(S) == 0:
        return lam.copy()
    w = z - A.T @ lam
    F = (w >= lo) & (w <= hi)
    xfix = np.clip(w, lo, hi)
    xfix[F] = 0.0
    As = A[S]
    M = As[:, F] @ As[:, F].T + (2.0 / C) * np.eye(len(S))
    rhs = As[:, F] @ z[F] + As[:, ~F] @ xfix[~F] - b[S]
    out = np.zeros(m)
    out[S] = np.linalg.solve(M, rhs)
    return out


def _states(w, lo, hi):
    """Per-variable piece label: 0 below lo (x = lo), 1 free (inclusive), 2 above hi (x = hi)."""
    return np.where(w < lo, 0, np.where(w > hi, 2, 1))


def _solve_on_rows(z, A, b, lo, hi, C, S, lam_init, max_iter=200):
    """Maximise the concave dual over lam_S in R^|S| with lam_j = 0 off S (no sign bound).

    The dual of the regularised projection is concave with gradient r(lam) and Hessian
    -(A D A^T + (2/C) I) (eq. reg_jacobian), piecewise quadratic.  Newton with an exact
    line search: on the current free set F the quadratic piece is maximised by the
    linear system (A_SF A_SF^T + (2/C) I) lam_S = A_SF z_F + A_S,notF x_notF - b_S; if
    that point keeps the same free set it is the maximiser, otherwise the dual is
    maximised exactly along the segment towards it (a one-dimensional piecewise root,
    _piecewise_root) and the step repeats.  The -2 lam/C term keeps every step finite.
    """
    m = A.shape[0]
    lam = np.zeros(m)
    lam[S] = np.asarray(lam_init, dtype=np.float64)[S]
    As = A[S]
    for _ in range(max_iter):
        w = z - A.T @ lam
        F = (w >= lo) & (w <= hi)
        xc = np.clip(w, lo, hi)
        M = As[:, F] @ As[:, F].T + (2.0 / C) * np.eye(len(S))
        rhs = As[:, F] @ z[F] + As[:, ~F] @ xc[~F] - b[S]
        target = np.zeros(m)
        target[S] = np.linalg.solve(M, rhs)
        w_t = z - A.T @ target
        # same piece = same state (lo / free / hi) for every variable
        if np.array_equal(_states(w_t, lo, hi), _states(w, lo, hi)):
            return target
        d = target - lam
        u = A.T @ d
        # phi'(gamma) = d^T r(lam + gamma d) = u^T clip(w - gamma u) - d^T(b + 2 lam / C) - 2 gamma |d|^2 / C
        c = float(d[S] @ (b[S] + 2.0 * lam[S] / C))
        slope0 = float(u @ xc) - c
        if slope0 <= 0.0:
            return target
        gam = _piecewise_root(w, u, c, lo, hi, 2.0 * float(d @ d) / C)
        lam = lam + gam * d
    return lam


def solve_coupled_exact(z, A, b, lo, hi, C, lam0=None, kkt_tol=1e-11, eq=None):
    """Unique optimum of the regularised projection for coupled rows (Thm 2).

    A KKT point has some set S of rows with lam_j >= 0 free to move and r_j <= 0 on the
    others.  For a candidate S the dual is maximised over lam_S without sign bounds
    (_solve_on_rows); the candidate is the answer when lam_S >= 0 and every other row
    satisfies r_j <= 0.  The first candidate is the set of rows that Alg. 2's stage 1
    single-row candidates mark active (lam0 > 0); after it every subset of the m <= 4
    rows is tried, largest first.  Equality rows (``eq``, Sec. 3.2.4) belong to every
    candidate set and keep their sign.  Returns (lam, info dict with the scaled KKT report).
    """
    from itertools import combinations

    from .checks import kkt_report

    z = np.asarray(z, dtype=np.float64)
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    b = np.asarray(b, dtype=np.float64)
    m = A.shape[0]
    E = eq_mask(eq, m)
    if lam0 is None:
        lam0 = np.array([solve_single_exact(z, A[j], b[j], lo, hi, C, equality=bool(E[j])) for j in range(m)])
    lam0 = np.asarray(lam0, dtype=np.float64)
    ineq = [j for j in range(m) if not E[j]]
    always = set(np.flatnonzero(E).tolist())
    first = tuple(sorted(always | {j for j in ineq if lam0[j] > 0}))
    order = [first]
    for k in range(len(ineq), -1, -1):
        for S in combinations(ineq, k):
            S = tuple(sorted(always | set(S)))
            if S not in order:
                order.append(S)
    best = None
    for tried, S in enumerate(order):
        S = list(S)
        lam = _solve_on_rows(z, A, b, lo, hi, C, S, lam0) if S else np.zeros(m)
        tiny = 1e-13 * max(1.0, float(np.max(np.abs(lam))))
        if np.any((lam < -tiny) & ~E):
            continue
        lam = np.where(E, lam, np.maximum(lam, 0.0))
        rep = kkt_report(z, A, b, lam, primal_from_dual(z, A, lam, lo, hi), lo, hi, C, eq=E)
        if best is None or rep["worst"] < best[1]["worst"]:
            best = (lam, rep, tried + 1)
        if rep["worst"] <= kkt_tol:
            break
    lam, rep, tried = best
    return lam, {"row_sets_tried": tried, "kkt": rep}


def alg2_general_projection(z, A, b, lo, hi, C, tol_B=1e-8, tol_N=1e-6, maxiter=200,
                            single="bisect", rel_tol_B=0.0, eq=None):
    """Alg. 2, general multi-constraint projection, step by step.

    Stage 1: for each row j, Alg. 1 gives a candidate lam_j with the other rows at
    zero; the candidate is accepted when every row k satisfies the linearised
    constraint a_k^T x - b_k <= tol_N * scale_k (the paper's test, made relative to the
    row magnitude; the -alpha grad f term the printed test omits is part of b here).
    The candidates are tested one at a time with the others at zero (the text's
    "if one such solution is feasible"); Stage 2 starts from all candidates together.
    Stage 2: semismooth Newton (see _newton_stage2) until ||Phi||_inf <= tol_N * scale.
    Equality rows (``eq``, Sec. 3.2.4): the stage-1 candidate of such a row is its
    single-row root over all of R; a candidate is accepted only if every equality row
    holds (|h_k| <= tol_N * scale_k); stage 2 uses Phi_k = h_k for them.
    Returns (lam, info dict with 'stage', 'newton_iters', 'converged').
    """
    z = np.asarray(z, dtype=np.float64)
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    b = np.asarray(b, dtype=np.float64)
    m = A.shape[0]
    E = eq_mask(eq, m)
    cand = np.zeros(m)
    for j in range(m):
        if single == "exact":
            lj = solve_single_exact(z, A[j], b[j], lo, hi, C, equality=bool(E[j]))
        else:
            lj, _ = solve_single_bisect(z, A[j], b[j], lo, hi, C, tol_B, rel_tol_B, equality=bool(E[j]))
        cand[j] = lj
        lam = np.zeros(m)
        lam[j] = lj
        x = primal_from_dual(z, A, lam, lo, hi)
        viol = A @ x - b
        h = viol - 2.0 * lam / C
        sc = row_scale(A, b, x)
        if np.all(np.where(E, np.abs(h), viol) <= tol_N * sc):
            return lam, {"stage": 1, "accepted_row": j, "newton_iters": 0, "converged": True}
    y, its, conv, curv = _newton_stage2(z, A, b, lo, hi, C, -cand, tol_N, maxiter, eq=E)
    return -y, {"stage": 2, "newton_iters": its, "converged": conv, "curvature_failures": curv}
