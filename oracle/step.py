"""One iteration of Alg. 3 (full PGD for TO) in FP64 (test infrastructure).

Order of the steps, as in Alg. 3:
  1. step size: the fallback alpha = min(alpha_max, alpha_fb / ||grad f||_inf) at t = 0 or
     when t >= t_warmup and ||max(g(x_t) - G, 0)||_inf > tol_N; otherwise the spectral
     step of eq. final_alpha (BB1 when s^T y > eps_alpha, else the Lipschitz step of
     eq. alpha), all capped by alpha_max;
  2. direction: PR+ conjugate gradient, eq. CG (d_0 = -grad f_0);
  3. trial point z = x_t + omega alpha d;
  4. projection of z onto the linearisation about x_t, with
     b_j = G_j - g_j(x_t) + a_j^T x_t (Sec. 3.2, eq. linearized: the constraint
     g_j + (x_{t+1} - x_t)^T grad g_j <= G_j);
  5. x_{t+1} = x(lam*), the stopping ratio ||x_{t+1} - x_t|| / ||x_{t+1}||.

Readings where the paper is silent: ||y|| = 0 gives the Lipschitz ratio +inf (so
alpha = alpha_max); ||s|| = 0 at t >= 1 takes the fallback step; ||g_prev|| = 0 gives
beta = 0.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import projection as P


@dataclass
class StepParams:
    """Defaults of Sec. 3.5 (C, alpha_max, tol_B, tol_N), Sec. 3.3 (alpha_fb = 0.2),
    Sec. 3.4 (eps_alpha = 1e-6, t_warmup = 50, omega = 1) and App. A.3.3 (c1, c2)."""
    C: float = 1e12
    alpha_max: float = 1e2
    alpha_fallback: float = 0.2
    tol_B: float = 1e-8
    tol_N: float = 1e-6
    omega: float = 1.0
    eps_alpha: float = 1e-6
    t_warmup: int = 50
    c1: float = 1e-4
    c2: float = 0.9
    maxiter_newton: int = 200


def step_scalars(x, x_prev, g, g_prev, t, gval, G, p: StepParams, eq=None):
    """alpha_t and beta_t of Alg. 3 (eq. final_alpha, eq. alpha, eq. CG) and which branch set alpha.

    The fallback trigger measures the violation g_j - G_j of an inequality row and
    |g_j - G_j| of an equality row (Sec. 3.2.4: the row must hold either way)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    gnorm_inf = float(np.max(np.abs(g))) if g.size else 0.0
    fallback_alpha = p.alpha_max if gnorm_inf == 0.0 else min(p.alpha_max, p.alpha_fallback / gnorm_inf)
    dg = np.atleast_1d(np.asarray(gval, dtype=np.float64) - np.asarray(G, dtype=np.float64))
    E = P.eq_mask(eq, dg.size)
    viol = float(np.max(np.where(E, np.abs(dg), np.maximum(dg, 0.0))))
    if t == 0 or (t >= p.t_warmup and viol > p.tol_N):
        alpha, branch = fallback_alpha, "fallback"
    else:
        s = x - np.asarray(x_prev, dtype=np.float64)
        y = g - np.asarray(g_prev, dtype=np.float64)
        ns = float(np.sqrt(s @ s))
        ny = float(np.sqrt(y @ y))
        sty = float(s @ y)
        if ns == 0.0:
            alpha, branch = fallback_alpha, "fallback"
        else:
            lip = np.inf if ny == 0.0 else ns / ny
            if sty > p.eps_alpha:
                alpha = min(float(s @ s) / sty, 2.0 * lip, p.alpha_max)
                branch = "bb1"
            else:
                alpha = min(lip, p.alpha_max)
                branch = "lipschitz"
    if t == 0:
        beta = 0.0
    else:
        gp = np.asarray(g_prev, dtype=np.float64)
        den = float(gp @ gp)
        beta = 0.0 if den == 0.0 else max(float(g @ (g - gp)) / den, 0.0)
    return {"alpha": float(alpha), "beta": float(beta), "branch": branch, "viol": viol}


def oracle_step(x, x_prev, g, g_prev, d_prev, A, gval, G, t, p: StepParams | None = None,
                mode="single", seg=None, projector="exact", lo=0.0, hi=1.0, eq=None, lam_given=None):
    """One Alg. 3 iteration.  Returns a dict with x_new, d, z, lam, b, alpha, beta, ...

    mode: 'single' (A is one row), 'independent' (A holds one coefficient per variable
    and seg the row offsets), 'coupled' (A is m x n).  projector: 'exact' gives the
    unique optimum (what parity is measured against); 'paper' runs Alg. 1 / Alg. 2 with
    the paper's tolerances (what the CPU baseline times).  eq: boolean mask of the
    equality rows g_j(x) = G_j (Sec. 3.2.4), linearised the same way.
    lam_given: multipliers to use instead of solving (a stored result of the exact
    projector for a problem too large to solve again in a test, written by a script under
    tests/golden that calls this function); everything else is computed as above.
    """
    p = p or StepParams()
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    sc = step_scalars(x, x_prev, g, g_prev, t, gval, G, p, eq=eq)
    alpha, beta = sc["alpha"], sc["beta"]
    d = -g if t == 0 else -g + beta * np.asarray(d_prev, dtype=np.float64)
    z = x + p.omega * alpha * d
    gval = np.atleast_1d(np.asarray(gval, dtype=np.float64))
    G = np.atleast_1d(np.asarray(G, dtype=np.float64))
    info = {"stage": 0, "newton_iters": 0}
    if mode == "independent":
        a = np.asarray(A, dtype=np.float64)
        seg = [int(s) for s in seg]
        ax = np.array([a[seg[j]:seg[j + 1]] @ x[seg[j]:seg[j + 1]] for j in range(len(seg) - 1)])
        b = G - gval + ax
        if lam_given is not None:
            lam = np.asarray(lam_given, dtype=np.float64)
        elif projector == "exact":
            lam = P.solve_independent_exact(z, a, seg, b, lo, hi, p.C, eq=eq)
        else:
            lam, _ = P.solve_independent_bisect(z, a, seg, b, lo, hi, p.C, p.tol_B, eq=eq)
        x_new = P.independent_primal(z, a, seg, lam, lo, hi)
        ax_new = np.array([a[seg[j]:seg[j + 1]] @ x_new[seg[j]:seg[j + 1]] for j in range(len(seg) - 1)])
    else:
        A2 = np.atleast_2d(np.asarray(A, dtype=np.float64))
        b = G - gval + A2 @ x
        E = P.eq_mask(eq, A2.shape[0])
        if lam_given is not None:
            lam = np.asarray(lam_given, dtype=np.float64)
        elif A2.shape[0] == 1 or mode == "single":
            if projector == "exact":
                lam = np.array([P.solve_single_exact(z, A2[0], b[0], lo, hi, p.C, equality=bool(E[0]))])
            else:
                lam = np.array([P.solve_single_bisect(z, A2[0], b[0], lo, hi, p.C, p.tol_B,
                                                      equality=bool(E[0]))[0]])
        elif projector == "exact":
            lam, info = P.solve_coupled_exact(z, A2, b, lo, hi, p.C, eq=E)
        else:
            lam, info = P.alg2_general_projection(z, A2, b, lo, hi, p.C, p.tol_B, p.tol_N,
                                                  p.maxiter_newton, eq=E)
        x_new = P.primal_from_dual(z, A2, lam, lo, hi)
        ax_new = A2 @ x_new
    nrm = float(np.linalg.norm(x_new))
    rel = float(np.linalg.norm(x_new - x)) / nrm if nrm > 0 else float("inf")
    return {
        "x_new": x_new, "d": d, "z": z, "lam": np.atleast_1d(lam), "b": b,
        "alpha": alpha, "beta": beta, "branch": sc["branch"], "rel_change": rel,
        "ax_new": ax_new, "info": info,
    }
