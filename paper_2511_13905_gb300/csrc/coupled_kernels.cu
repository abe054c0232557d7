// coupled_kernels.cu -- fused PGD-TO step / projection for m <= 4 coupled rows (Alg. 2).
//
// One cooperative launch; A is m dense rows of n floats.  Phases (each ends in one grid
// reduction, dev_common.cuh):
//   A  step size and PR+ coefficient (as for single rows)
//   B  double-float trial point z, state copies; per row a_j^T x_t, r_j(0), the saturation
//      bound and the free-set curvature at 0 (Alg. 1's inputs for each row)
//   S1 Alg. 2 stage 1: the m single-row searches (row j alone, the others at zero) run
//      side by side, K trial points per row per pass
//   F  feasibility of each single-row candidate against every row (m x m sums); a
//      candidate that satisfies all rows ends the projection (stage 1 accepted)
//   E  evaluation at the dual iterate lam: h = A x(lam) - b - 2 lam / C, J_h = A D A^T + 2/C
//      (eq. h, eq. reg_jacobian) and sum_i |a_ji x_i| for the row scales
//   LS exact line search along the Newton direction d: phi'(g) = d^T h(lam + g d) is the
//      residual of a single virtual row u = A^T d on w0 = z - A^T lam, so it reuses the
//      root search of the single-row path; then back to E
//   D  x = clip(z - A^T lam) in double-float, a_j^T x, ||x - x_t||, ||x||
// Stage 2 solves J_h on the working set {lam_j > 0 or h_j > 0} (the semismooth Newton
// system of App. A.3.3 restricted to the rows that can move) and, instead of backtracking
// on the merit ||Phi||^2 / 2, maximises the concave dual exactly along the direction,
// which keeps lam >= 0 by capping the step.
#include <float.h>
#include <math.h>
#include <string.h>

#include <type_traits>

#include "dev_common.cuh"
#include "kernels.h"
#include "step_common.cuh"

namespace pgdto {

enum CoupledMode : int { kModeDone = 0, kModeStage1 = 1, kModeFeas = 2, kModeEval = 3, kModeLine = 4 };

struct CoupledBcast {
    // step scalars c = omega alpha and beta as float pairs (field names shared with the
    // single-row kernel's templates)
    float c_hi, c_lo, beta_hi, beta_lo;
    int branch, status;
    int any_active;  // root searches still running (stage 1 or line search)
    int mode;        // what the next pass computes (CoupledMode)
    float pts[kMaxRows][K];
    int active[kMaxRows];
    float lam_hi[kMaxRows], lam_lo[kMaxRows];  // stage-1 candidates, then the final lam
    // dual iterate and Newton direction, split into float pairs for the element passes
    float it_hi[kMaxRows], it_lo[kMaxRows];
    float d_hi[kMaxRows], d_lo[kMaxRows];
    int cand_row[kMaxRows];  // rows whose stage-1 candidate is tested in the F pass
    int ncand;
    int pad;
};

struct NewtonState {
    double lam[kMaxRows];   // current dual iterate
    double d[kMaxRows];     // current direction
    double base[kMaxRows];  // iterate the direction was computed at (the full step is a trial)
    double base_phi;        // scaled KKT residual at base
    double base_slope, base_dtb, base_dd;  // line-search data at base along d
    double cap;             // largest step keeping lam >= 0 along d
    double tol;
    double phi;             // largest scaled |h_j| seen at the last evaluation
    int iters;
    int passes;             // passes after the trial-point pass
    int stage;              // 1 stage-1 candidate accepted, 2 Newton
    int how;                // 3 if an iteration limit was hit
    int ls_expand;          // 1: line-search bracket open on the right, 2: closed by the cap
    int stall;              // evaluations in a row without progress at the rounding floor
    int eq_mask;            // equality rows (always in the working set, never clamped or capped)
    int trial;              // lam is the full Newton step from base, not yet accepted
    // Float-pair copies written by the Newton update (phase E), which runs without FP64
    // arithmetic; the doubles above (lam, d, base, base_*, phi) lag them while `stale` is
    // set and are refreshed by nt_sync before the paths that read them.  The iterate and
    // the direction themselves are bc.it_hi/it_lo and bc.d_hi/d_lo.
    float base_h[kMaxRows], base_l[kMaxRows];
    float fphi, fbase_phi;
    float slope_h, slope_l, dtb_h, dtb_l, dd_h, dd_l;
    int stale;
};

// Search state of one problem.  Every CTA keeps its own copy in shared memory and runs the
// scalar updates on it after each grid all-reduce (identical totals, identical code, so
// identical copies); block 0 writes the report to the workspace at the end.
struct CoupledState {
    CoupledBcast bc;
    RowState rows[kMaxRows];  // stage-1 searches
    RowState ls;              // the line search
    NewtonState nt;
    DeviceInfo info;
};

struct CoupledWork {
    GridCtrl ctrl;
    CoupledState st;   // st.info: the report after a launch
    Partials part[2];  // block partials of alternate rounds
};

size_t coupled_work_bytes() { return sizeof(CoupledWork); }
size_t coupled_work_ctrl_bytes() { return sizeof(GridCtrl); }
DeviceInfo* coupled_work_info(CoupledWork* ws) { return &ws->st.info; }

// sc.tot layout of each pass
//   B:   5 per row (a^T x_t, a^T clip(z), free curvature at 0, S_min, S_max), 3 maxima
//        per row (the upper saturation bound, minus the lower one, max |a_j|); all but the
//        first two sums are formed only when stage 1 runs
//   S1:  2K per row
//   F:   m per candidate row (sums of every row at that candidate)
//   E:   [0, m) h sums a_j^T x, [m, 2m) sum |a_j x|, [2m, 2m + 10) J upper triangle
//   LS:  2K
//   D:   [0, m) a_j^T x, m: ||x - x_t||^2, m + 1: ||x||^2
template <int M>
__device__ __forceinline__ int jidx(int j, int k) {  // row-major upper-triangle index of (j, k), j <= k
    return j * M - (j * (j - 1)) / 2 + (k - j);
}

// ----------------------------------------------------------------------- scalar updates

// The Newton iteration's counters and tolerances before the first pass of a step.
__device__ __forceinline__ void cnewton_reset(CoupledState* ws, const CoupledArgs& a) {
    volatile NewtonState* nt = &ws->nt;
    nt->iters = 0;
    nt->how = 0;
    nt->stage = 0;
    nt->passes = 0;
    nt->stall = 0;
    nt->trial = 0;
    nt->phi = INFINITY;
    nt->fphi = INFINITY;
    nt->fbase_phi = 0.0f;
    nt->stale = 0;
    nt->tol = 1e-8;  // relative tolerance of the line search (the next Newton step corrects)
    nt->eq_mask = a.eq_mask;
}

// Phase B: inputs of the single-row searches (Alg. 2 stage 1), as for a single row; an
// equality row (Sec. 3.2.4) with r(0) < 0 searches below 0 (see the single-row kernel).
template <int M>
__device__ void cupd_after_trial(const CoupledArgs& a, const BlockScratch& sc, CoupledState* ws) {
    const int lane = threadIdx.x, j = lane >> 3, k = lane & 7;
    volatile CoupledBcast* bc = &ws->bc;
    volatile RowState* rows = ws->rows;
    const bool row = j < M;
    const int jj = row ? j : 0;
    const double two_c = a.two_c;
    const double ax = a.proj ? 0.0 : df_to_double(sc.tot[5 * jj + 0]);
    const double r0s = df_to_double(sc.tot[5 * jj + 1]);
    const double sf = df_to_double(sc.tot[5 * jj + 2]);
    const double smin = df_to_double(sc.tot[5 * jj + 3]);
    const double smax = df_to_double(sc.tot[5 * jj + 4]);
    const bool eq = (a.eq_mask >> jj) & 1;
    if (!(a.stage1 && !a.lam_prev)) {
        // stage 2 comes next (from lam = 0 or the previous step's lam): b_j, the status, and
        // whether any row is violated at lam = 0 are all it needs from this pass
        const bool finite = isfinite(ax) && isfinite(r0s);
        const double b = a.bconst[jj] + ax;
        const double r0 = r0s - b;
        const bool act = row && finite && (r0 > 0.0 || (eq && r0 < 0.0));
        if (row && k == 0) {
            ws->info.b[j] = b;
            rows[j].reg = two_c;
            store_row(&rows[j], b, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, r0, 0, 0, 0);
            publish_lambda(bc, j, 0.0);
        }
        const unsigned any = __ballot_sync(kFull, act);
        const unsigned bad = __ballot_sync(kFull, row && !finite);
        if (lane == 0) {
            int status = a.proj ? kOk : bc->status;
            if (bad) status = kErrNonfinite;
            bc->status = status;
            bc->any_active = (status == kOk && any) ? 1 : 0;
            cnewton_reset(ws, a);
        }
        return;
    }
    const double lsat = (double)sc.totmax[2 * jj];
    const double lneg = -(double)sc.totmax[2 * jj + 1];
    const bool finite = isfinite(ax) && isfinite(r0s) && isfinite(sf) && isfinite(smin) && isfinite(smax);
    const double b = a.bconst[jj] + ax;
    const double r0 = r0s - b;
    const bool up = r0 > 0.0;
    const bool down = eq && r0 < 0.0;
    double L, rL, SLs, H, rH, SHs;
    if (down) {
        float Lf = (float)(lneg * (1.0 + 1e-5) - 1e-30);
        if (!((double)Lf < 0.0)) Lf = -FLT_MIN;
        L = (double)Lf;
        rL = smax - b - two_c * L;
        SLs = two_c;
        H = 0.0;
        rH = r0;
        SHs = sf + two_c;
    } else {
        float Hf = (float)(lsat * (1.0 + 1e-5) + 1e-30);
        if (!((double)Hf > 0.0)) Hf = FLT_MIN;
        L = 0.0;
        rL = r0;
        SLs = sf + two_c;
        H = (double)Hf;
        rH = smin - b - two_c * H;
        SHs = two_c;
    }
    // the closed form of a row violated even at its saturation bound needs the full pass's
    // sums (stage 1); without them every violated row goes to the Newton iteration, which
    // reaches the same regularised optimum
    const bool full = a.stage1 && !a.lam_prev;
    const bool closed = full && (down ? rL < 0.0 : (up && rH > 0.0));
    const bool search = row && finite && (up || down) && !closed;
    double q = 0.0;
    if (k == 0) q = rL / SLs;
    else if (k == 1) q = rH / SHs;
    const double NL = L + __shfl_sync(kFull, q, lane & ~7);
    const double NH = H + __shfl_sync(kFull, q, (lane & ~7) + 1);
    const float p = next_point(lane, L, rL, H, rH, NL, NH, true);
    if (row && k == 0) {
        ws->info.b[j] = b;
        rows[j].reg = two_c;
        if (search) {
            store_row(&rows[j], b, L, rL, SLs, H, rH, SHs, 0.0, 0.0, 1, 0, 2);
            rows[j].famax = sc.totmax[2 * M + jj];
            bc->active[j] = 1;
        } else if (closed) {
            const double lam = 0.5 * a.C * ((down ? smax : smin) - b);
            store_row(&rows[j], b, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, lam, 0.0, 0, 0, 1);
            publish_lambda(bc, j, lam);
        } else {
            store_row(&rows[j], b, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, r0, 0, 0, 0);
            publish_lambda(bc, j, 0.0);
        }
    }
    if (search) bc->pts[j][k] = p;
    const unsigned any = __ballot_sync(kFull, search);
    const unsigned bad = __ballot_sync(kFull, row && !finite);
    if (lane == 0) {
        int status = a.proj ? kOk : bc->status;
        if (bad) status = kErrNonfinite;
        bc->status = status;
        bc->any_active = (status == kOk && any) ? 1 : 0;
        cnewton_reset(ws, a);
    }
}

// Candidates of stage 1 are known: set up the feasibility pass (or finish at lam = 0).
template <int M>
__device__ void cupd_plan_feasibility(CoupledState* ws) {
    volatile CoupledBcast* bc = &ws->bc;
    volatile RowState* rows = ws->rows;
    if (threadIdx.x != 0) return;
    int nc = 0;
    for (int j = 0; j < M; ++j)
        if (rows[j].lam != 0.0) bc->cand_row[nc++] = j;  // equality rows may be negative
    bc->ncand = nc;
    volatile NewtonState* nt = &ws->nt;
    for (int j = 0; j < M; ++j) {
        nt->lam[j] = 0.0;
        bc->it_hi[j] = 0.0f;
        bc->it_lo[j] = 0.0f;
    }
    if (nc == 0) {
        // every row holds at lam = 0: that is the KKT point
        nt->stage = 1;
        bc->mode = kModeDone;
    } else {
        bc->mode = kModeFeas;
    }
}

// Refresh the FP64 Newton state from the float pairs the phase-E update left (thread 0).
__device__ __forceinline__ void nt_sync(volatile NewtonState* nt, volatile CoupledBcast* bc, int m) {
    if (!nt->stale) return;
    for (int j = 0; j < m; ++j) {
        nt->lam[j] = (double)bc->it_hi[j] + (double)bc->it_lo[j];
        nt->d[j] = (double)bc->d_hi[j] + (double)bc->d_lo[j];
        nt->base[j] = (double)nt->base_h[j] + (double)nt->base_l[j];
    }
    nt->phi = (double)nt->fphi;
    nt->base_phi = (double)nt->fbase_phi;
    nt->base_slope = (double)nt->slope_h + (double)nt->slope_l;
    nt->base_dtb = (double)nt->dtb_h + (double)nt->dtb_l;
    nt->base_dd = (double)nt->dd_h + (double)nt->dd_l;
    nt->stale = 0;
}

__device__ __forceinline__ void set_iterate(volatile CoupledBcast* bc, volatile NewtonState* nt, int m) {
    for (int j = 0; j < m; ++j) {
        float h, l;
        split_double(nt->lam[j], h, l);
        bc->it_hi[j] = h;
        bc->it_lo[j] = l;
    }
}

// Start of stage 2 without stage 1.  Warm: the session's previous step left its
// multipliers; a design's dual moves little from one step to the next, so Newton starts
// there (inequality multipliers clamped at 0, equality ones not).  Cold (zero): Newton
// starts at lam = 0, where h is the rows' violation at the trial point; the globalised
// iteration reaches the same optimum as from stage 1's candidates, and on the 4-row
// volume/centre-of-mass workload it took 6 evaluations against stage 1's 3 search passes,
// its feasibility pass and 7 evaluations.
template <int M>
__device__ void cupd_warm_start(const CoupledArgs& a, CoupledState* ws, bool zero) {
    volatile CoupledBcast* bc = &ws->bc;
    volatile NewtonState* nt = &ws->nt;
    for (int j = 0; j < M; ++j) {
        const double l = zero ? 0.0 : a.lam_prev[j];
        nt->lam[j] = ((a.eq_mask >> j) & 1) ? (isfinite(l) ? l : 0.0) : (l > 0.0 ? l : 0.0);
        bc->active[j] = 0;
    }
    bc->any_active = 0;
    nt->stage = 2;
    nt->trial = 0;
    set_iterate(bc, nt, M);
    bc->mode = kModeEval;
}


// Phase F: accept the first single-row candidate that every row admits (Alg. 2 stage 1);
// otherwise start stage 2 from all candidates together.
template <int M>
__device__ void cupd_after_feasibility(const CoupledArgs& a, const BlockScratch& sc, CoupledState* ws) {
    if (threadIdx.x != 0) return;
    volatile CoupledBcast* bc = &ws->bc;
    volatile RowState* rows = ws->rows;
    volatile NewtonState* nt = &ws->nt;
    const int nc = bc->ncand;
    int accepted = -1;
    for (int c = 0; c < nc && accepted < 0; ++c) {
        const int j = bc->cand_row[c];
        bool ok = true;
        for (int k = 0; k < M; ++k) {
            if (k == j) continue;  // row j holds at its own root by construction
            const double r = df_to_double(sc.tot[c * M + k]) - rows[k].b;
            // admitted when the row holds to 1e-9 of its magnitude (tighter than tol_N so the
            // accepted point is the regularised optimum to the parity tolerance); an
            // equality row must hold from both sides
            const double rr = ((a.eq_mask >> k) & 1) ? fabs(r) : r;
            if (!(rr <= 1e-9 * fmax(1.0, fabs(rows[k].b)))) ok = false;
        }
        if (ok) accepted = j;
    }
    if (accepted >= 0) {
        for (int k = 0; k < M; ++k) nt->lam[k] = (k == accepted) ? rows[accepted].lam : 0.0;
        nt->stage = 1;
        bc->mode = kModeDone;
    } else {
        for (int k = 0; k < M; ++k) nt->lam[k] = rows[k].lam;
        nt->stage = 2;
        bc->mode = kModeEval;
    }
    set_iterate(bc, nt, M);
}

// Line search along nt->d from nt->base (nt->lam is reset to base): first points
// around the Newton step g = 1; phi'(0) = d^T h(base) = d^T J d > 0.
template <int M>
__device__ void cstart_line_search(CoupledState* ws) {
    volatile CoupledBcast* bc = &ws->bc;
    volatile NewtonState* nt = &ws->nt;
    volatile RowState* ls = &ws->ls;
    nt_sync(nt, bc, M);
    for (int j = 0; j < M; ++j) nt->lam[j] = nt->base[j];
    set_iterate(bc, nt, M);
    double cap = INFINITY;  // the step at which an inequality multiplier reaches 0
    for (int j = 0; j < M; ++j)
        if (nt->d[j] < 0.0 && !((nt->eq_mask >> j) & 1)) cap = fmin(cap, nt->base[j] / (-nt->d[j]));
    nt->cap = cap;
    ls->b = nt->base_dtb;
    ls->reg = nt->base_dd;
    ls->L = 0.0;
    ls->rL = nt->base_slope;
    ls->SL = nt->base_slope;
    ls->passes = 0;
    ls->active = 1;
    ls->how = 2;
    const float base[K] = {0.125f, 0.25f, 0.5f, 0.75f, 1.0f, 1.25f, 2.0f, 8.0f};
    if (isfinite(cap)) {
        ls->H = cap;
        ls->rH = 0.0;
        ls->SH = 0.0;
        for (int k = 0; k < K; ++k) {
            double v = fmin((double)base[k], cap * (double)(k + 1) / (double)K);
            if (k == K - 1) v = cap;
            bc->pts[0][k] = (float)v;
        }
        nt->ls_expand = 2;  // bracket closed by the cap
    } else {
        ls->H = INFINITY;
        for (int k = 0; k < K; ++k) bc->pts[0][k] = base[k];
        nt->ls_expand = 1;
    }
    row_refresh_floats(ls);
    nt->trial = 0;
    bc->any_active = 1;
    bc->mode = kModeLine;
}

// Phase E: h and J_h at lam.  A full Newton step under test is accepted when the scaled
// KKT residual fell; otherwise the step is replaced by an exact line search from its base.
// At an accepted point: KKT test, then the Newton direction on the working set and the
// next full step max(lam + d, 0) as the new trial.
// Phase E's update on warp 0, one row per lane, in double-float arithmetic on the FP32
// pipes with no FP64 instruction: lane r < M forms h_r and its scale, holds row r of the
// Jacobian during the elimination (the pivot row is broadcast by shuffles) and stores row
// r's results as float pairs (the FP64 copies are refreshed later, nt_sync).  An FP64
// one-thread version took about 29,000 cycles per call here and an FP64 one-lane-per-row
// one about 9,000: an FP64 warp instruction costs many issue cycles on this part however
// few lanes are active.
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DF shfl_df(DF v, int src) {
    return DF{__shfl_sync(kFull, v.hi, src), __shfl_sync(kFull, v.lo, src)};
}

template <int M>
__device__ void cupd_after_eval(const CoupledArgs& a, const BlockScratch& sc, CoupledState* ws) {
    const int lane = threadIdx.x;
    volatile CoupledBcast* bc = &ws->bc;
    volatile RowState* rows = ws->rows;
    volatile NewtonState* nt = &ws->nt;
    const bool row = lane < M;
    const int r = row ? lane : 0;
    const DF two_c = DF{a.two_c_df[0], a.two_c_df[1]};
    const bool eq = (a.eq_mask >> r) & 1;
    const DF lam = DF{bc->it_hi[r], bc->it_lo[r]};
    const DF b = DF{rows[r].b_hi, rows[r].b_lo};
    const DF h = df_sub(df_sub(sc.tot[r], b), df_mul(two_c, lam));
    const float scale = fmaxf(1.0f, fmaxf(fabsf(b.hi), sc.tot[M + r].hi));
    const bool lpos = df_pos(lam), hpos = df_pos(h);
    const bool act = lpos || eq;
    const float tol = 1e-9f * scale;
    bool conv = __all_sync(kFull, !row || (act ? fabsf(h.hi) <= tol : h.hi <= tol));
    if (!__all_sync(kFull, !row || isfinite(h.hi))) {
        if (lane == 0) {
            bc->status = kErrNonfinite;
            bc->mode = kModeDone;
        }
        return;
    }
    float ph = row ? __fdividef(act ? fabsf(h.hi) : fmaxf(h.hi, 0.0f), scale) : 0.0f;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) ph = fmaxf(ph, __shfl_xor_sync(kFull, ph, o));
    const float phi = __shfl_sync(kFull, ph, 0);
    int iters = nt->iters;
    if (nt->trial) {
        if (!(phi < nt->fbase_phi * (1.0f - 1e-4f) || phi <= 1e-8f)) {
            if (lane == 0) cstart_line_search<M>(ws);  // the full step did not reduce the residual
            return;
        }
        iters += 1;
    }
    // stop at the rounding floor of the FP32 sums: the scaled KKT residual is small and
    // has stopped halving over the last iterations
    const float prev = nt->fphi;
    const int stall = (iters >= 2 && phi <= 1e-7f && phi >= 0.5f * prev) ? nt->stall + 1 : 0;
    if (stall >= 2) conv = true;
    // working set: rows with lam_j > 0, h_j > 0, and equality rows (always)
    const unsigned rmask = (1u << M) - 1u;
    unsigned inS = __ballot_sync(kFull, row && (lpos || hpos || eq)) & rmask;
    __syncwarp();
    if (lane == 0) {
        nt->trial = 0;
        nt->iters = iters;
        nt->stall = stall;
        nt->fphi = phi;
        nt->stale = 1;
    }
    if (conv || inS == 0u) {
        if (lane == 0) bc->mode = kModeDone;
        return;
    }
    if (iters >= a.maxiter_newton) {
        if (lane == 0) {
            nt->how = 3;
            bc->mode = kModeDone;
        }
        return;
    }
    // J_SS d_S = h_S (eq. reg_jacobian restricted to the working set): Gaussian elimination
    // on the full M x M system with the rows and columns outside the set replaced by the
    // identity (d_j = 0 there); a row at lam_j = 0 whose direction would push it below zero
    // leaves the set and the system is solved again (at most M times).  J_SS is symmetric
    // positive definite (A D A^T + (2/C) I), so no pivoting is needed.
    DF dq[M];
#pragma unroll
    for (int round = 0; round < M; ++round) {
        DF Mr[M];
        const bool rin = (inS >> r) & 1u;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            const int lo_ = r < q ? r : q, hi_ = r < q ? q : r;
            DF v = sc.tot[2 * M + jidx<M>(lo_, hi_)];
            if (r == q) v = df_add(v, two_c);
            Mr[q] = (rin && ((inS >> q) & 1u)) ? v : DF{r == q ? 1.0f : 0.0f, 0.0f};
        }
        DF rhs = rin ? h : df_zero();
        DF inv[M];
#pragma unroll
        for (int p = 0; p < M; ++p) {
            DF prow[M];
#pragma unroll
            for (int q = p; q < M; ++q) prow[q] = shfl_df(Mr[q], p);
            const DF prhs = shfl_df(rhs, p);
            inv[p] = df_div(DF{1.0f, 0.0f}, prow[p]);
            if (r > p) {
                const DF f = df_mul(Mr[p], inv[p]);
#pragma unroll
                for (int q = p; q < M; ++q) Mr[q] = df_sub(Mr[q], df_mul(f, prow[q]));
                rhs = df_sub(rhs, df_mul(f, prhs));
            }
        }
#pragma unroll
        for (int p = M - 1; p >= 0; --p) {
            DF v = rhs;
#pragma unroll
            for (int q = p + 1; q < M; ++q) v = df_sub(v, df_mul(Mr[q], dq[q]));
            dq[p] = shfl_df(df_mul(v, inv[p]), p);
        }
        const unsigned drop =
            __ballot_sync(kFull, row && ((inS >> r) & 1u) && !lpos && df_pos(df_neg(dq[r])) && !eq) & rmask;
        if (drop == 0u || drop == inS) break;
        inS &= ~drop;
    }
    const DF dr = row ? dq[r] : df_zero();
    DF s0 = df_mul(dr, h), stb = df_mul(dr, df_add(b, df_mul(two_c, lam))), sdd = df_mul(dr, dr);
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        s0 = df_add(s0, DF{__shfl_xor_sync(kFull, s0.hi, o), __shfl_xor_sync(kFull, s0.lo, o)});
        stb = df_add(stb, DF{__shfl_xor_sync(kFull, stb.hi, o), __shfl_xor_sync(kFull, stb.lo, o)});
        sdd = df_add(sdd, DF{__shfl_xor_sync(kFull, sdd.hi, o), __shfl_xor_sync(kFull, sdd.lo, o)});
    }
    if (!df_pos(s0)) {
        if (lane == 0) bc->mode = kModeDone;  // no ascent along d: the rounding floor is reached
        return;
    }
    if (row) {
        bc->d_hi[r] = dr.hi;
        bc->d_lo[r] = dr.lo;
        nt->base_h[r] = lam.hi;
        nt->base_l[r] = lam.lo;
        // the full Newton step, kept in lam >= 0, is evaluated by the next E pass
        DF ln = df_add(lam, dr);
        if (!eq && !df_pos(ln)) ln = df_zero();
        bc->it_hi[r] = ln.hi;
        bc->it_lo[r] = ln.lo;
    }
    if (lane == 0) {
        const DF dd = df_mul(two_c, sdd);
        nt->fbase_phi = phi;
        nt->slope_h = s0.hi;
        nt->slope_l = s0.lo;
        nt->dtb_h = stb.hi;
        nt->dtb_l = stb.lo;
        nt->dd_h = dd.hi;
        nt->dd_l = dd.lo;
        nt->trial = 1;
        bc->mode = kModeEval;
    }
}

// Phase LS: one pass of the exact line search along d.  The first pass of a direction
// either finds the sign change of phi' among its points or, if phi' > 0 at all of them,
// takes the cap (closed bracket) or moves the bracket right (open bracket).  Later
// passes are the shared root search.  When it ends, lam <- max(lam + g d, 0).
template <int M>
__device__ void cupd_after_line(const CoupledArgs& a, const BlockScratch& sc, CoupledState* ws) {
    const int lane = threadIdx.x;
    volatile CoupledBcast* bc = &ws->bc;
    volatile NewtonState* nt = &ws->nt;
    volatile RowState* ls = &ws->ls;
    const int expand = nt->ls_expand;
    if (expand) {
        const int k = lane & 7;
        const double gk = (double)bc->pts[0][k];
        const double rk = df_to_double(sc.tot[k]) - ls->b - ls->reg * gk;
        const double Sk = df_to_double(sc.tot[K + k]) + ls->reg;
        const unsigned nonpos = __ballot_sync(kFull, lane < K && !(rk > 0.0)) & 0xffu;
        const int kH = nonpos ? __ffs(nonpos) - 1 : -1;
        double L = ls->L, rL = ls->rL, SL = ls->SL;
        const double gL = __shfl_sync(kFull, gk, kH > 0 ? kH - 1 : 0);
        const double rLn = __shfl_sync(kFull, rk, kH > 0 ? kH - 1 : 0);
        const double SLn = __shfl_sync(kFull, Sk, kH > 0 ? kH - 1 : 0);
        const double gH = __shfl_sync(kFull, gk, kH >= 0 ? kH : K - 1);
        const double rHn = __shfl_sync(kFull, rk, kH >= 0 ? kH : K - 1);
        const double SHn = __shfl_sync(kFull, Sk, kH >= 0 ? kH : K - 1);
        if (kH > 0) {
            L = gL;
            rL = rLn;
            SL = SLn;
        }
        if (kH >= 0) {
            // bracket [L, H] closed: next points from the shared rule
            double q = 0.0;
            if (k == 0) q = rL / SL;
            else if (k == 1) q = rHn / SHn;
            const double NL = L + __shfl_sync(kFull, q, 0);
            const double NH = gH + __shfl_sync(kFull, q, 1);
            const float p = next_point(lane, L, rL, gH, rHn, NL, NH);
            if (lane < K) bc->pts[0][lane] = p;
            if (lane == 0) {
                store_row(ls, ls->b, L, rL, SL, gH, rHn, SHn, 0.0, 0.0, 1, ls->passes + 1, 2);
                nt->ls_expand = 0;
                bc->any_active = 1;
            }
        } else if (lane == 0) {
            // phi' > 0 at every point
            if (expand == 2 || ls->passes >= 4) {
                store_row(ls, ls->b, gH, rHn, SHn, gH, rHn, SHn, expand == 2 ? nt->cap : gH, 0.0, 0, ls->passes + 1,
                          2);
                bc->any_active = 0;
            } else {
                store_row(ls, ls->b, gH, rHn, SHn, INFINITY, 0.0, 0.0, 0.0, 0.0, 1, ls->passes + 1, 2);
                const float mult[K] = {2.0f, 3.0f, 4.0f, 6.0f, 8.0f, 16.0f, 64.0f, 1024.0f};
                for (int q = 0; q < K; ++q) bc->pts[0][q] = (float)(gH * (double)mult[q]);
                bc->any_active = 1;
            }
        }
    } else {
        search_pass_update(sc, 0, ls, bc, 1, nt->tol, a.max_passes);
    }
    __syncwarp();
    if (lane != 0) return;
    nt->passes = nt->passes + 1;
    if (bc->any_active) return;
    nt_sync(nt, bc, M);
    // line search finished: take the step
    double g = ls->lam;
    const double cap = nt->cap;
    const bool at_cap = isfinite(cap) && g >= cap * (1.0 - 1e-12);
    if (at_cap) g = cap;
    for (int j = 0; j < M; ++j) {
        const double dj = nt->d[j];
        double v = nt->lam[j] + g * dj;
        if (!((a.eq_mask >> j) & 1)) {  // an equality multiplier keeps its sign
            if (v < 0.0 || (at_cap && dj < 0.0 && nt->lam[j] / (-dj) <= cap * (1.0 + 1e-12))) v = fmax(v, 0.0);
            if (at_cap && dj < 0.0 && nt->lam[j] / (-dj) <= cap * (1.0 + 1e-12)) v = 0.0;
        }
        nt->lam[j] = v;
    }
    nt->iters = nt->iters + 1;
    nt->trial = 0;
    set_iterate(bc, nt, M);
    bc->mode = kModeEval;
}

// When the projection is decided, publish lam for the final pass (thread 0).
template <int M>
__device__ __forceinline__ void cfinish_if_done(CoupledState* ws) {
    volatile CoupledBcast* bc = &ws->bc;
    volatile NewtonState* nt = &ws->nt;
    if (bc->mode != kModeDone) return;
    nt_sync(nt, bc, M);
    for (int j = 0; j < M; ++j) {
        float h, l;
        split_double(nt->lam[j], h, l);
        bc->lam_hi[j] = h;
        bc->lam_lo[j] = l;
    }
}

// After phase D: the report.
template <int M>
__device__ void cupd_final(const CoupledArgs& a, const BlockScratch& sc, CoupledState* ws, int* sticky,
                           unsigned long long* launches) {
    const int lane = threadIdx.x;
    volatile DeviceInfo* inf = &ws->info;
    volatile RowState* rows = ws->rows;
    volatile CoupledBcast* bc = &ws->bc;
    volatile NewtonState* nt = &ws->nt;
    double rc = 0.0;
    if (lane == 1 && !a.proj) {
        const double dd = df_to_double(sc.tot[M]);
        const double nn = df_to_double(sc.tot[M + 1]);
        rc = nn > 0.0 ? sqrt(dd / nn) : INFINITY;
    }
    rc = __shfl_sync(kFull, rc, 1);
    if (lane != 0) return;
    nt_sync(nt, bc, M);
    int status = bc->status;
    for (int j = 0; j < M; ++j) {
        const double ax = df_to_double(sc.tot[j]);
        inf->lambda[j] = nt->lam[j];
        inf->viol[j] = ax - rows[j].b;
        inf->b[j] = rows[j].b;
        if (!isfinite(ax) && status == kOk) status = kErrNonfinite;
    }
    for (int j = M; j < kMaxRows; ++j) {
        inf->lambda[j] = 0.0;
        inf->viol[j] = 0.0;
        inf->b[j] = 0.0;
    }
    if (nt->how == 3 && status == kOk) status = kNotConverged;
    if (!a.proj) {
        inf->rel_change = rc;
    } else {
        inf->rel_change = 0.0;
        inf->alpha = 0.0;
        inf->beta = 0.0;
        inf->branch = -1;
        inf->t = -1;
    }
    inf->phi_inf = nt->phi;
    inf->passes = nt->passes;
    inf->newton_iters = nt->iters;
    inf->stage = nt->stage;
    inf->status = status;
    if (status != kOk && sticky) atomicCAS(sticky, kOk, status);
    if (launches) *launches += 1ull;
}

// ----------------------------------------------------------------------- element passes

template <bool VEC, int M>
__global__ void __launch_bounds__(kThreads, 1) coupled_kernel(CoupledArgs a) {
    __shared__ BlockScratch sc;
    __shared__ CoupledBcast bc;
    __shared__ CoupledState cst;
    CoupledState* const cs = &cst;
    CoupledWork* ws = a.ws;
    if (ld_volatile_i32(&ws->ctrl.abort)) return;
    const int nb = gridDim.x, blk = blockIdx.x;
    const float lo = a.lo, hi = a.hi;
    const int64_t n = a.n;
    if (blk == 0 && threadIdx.x == 0) {
        volatile GridCtrl* vc = &ws->ctrl;
        vc->trace_start = globaltimer_ns();
        vc->ntrace = 0;
    }
    grid_sync_init(&ws->ctrl, sc);
    // test hook: block 0 never arrives, so every other block's first wait runs out its budget
    if (a.fault_inject == 1 && blk == 0) return;
    {
        unsigned* w = reinterpret_cast<unsigned*>(&cs->info);  // every report field starts defined
        for (int i = threadIdx.x; i < (int)(sizeof(DeviceInfo) / 4); i += blockDim.x) w[i] = 0u;
        __syncthreads();
    }
    // the broadcast part of this CTA's state, for the element passes
    auto fetch = [&]() {
        const unsigned* src = reinterpret_cast<const unsigned*>(&cs->bc);
        unsigned* d = reinterpret_cast<unsigned*>(&bc);
        for (int i = threadIdx.x; i < (int)(sizeof(CoupledBcast) / 4); i += blockDim.x) d[i] = src[i];
        __syncthreads();
    };
    int64_t cb, ce;
    block_chunk(0, n, blk, nb, cb, ce);
    const float* zh_src = a.proj ? a.z_in : a.z;
    const bool has_lo = !a.proj;

    if (!a.proj) {
        // ------------------------------------------------------------ phase A
        AccSplit<6, 0> acc;
        acc.init();
        float gmax = 0.0f;
        if (a.t > 0) {
            auto e = [&](float x, float xp, float g, float gp) {
                const float s = x - xp, y = g - gp;
                acc.f[0] = fmaf(s, s, acc.f[0]);
                acc.f[1] = fmaf(s, y, acc.f[1]);
                acc.f[2] = fmaf(y, y, acc.f[2]);
                acc.f[3] = fmaf(g, y, acc.f[3]);
                acc.f[4] = fmaf(gp, gp, acc.f[4]);
                acc.f[5] = fmaf(g, g, acc.f[5]);
                gmax = fmaxf(gmax, fabsf(g));
            };
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 x = LD4L2(a.x, v), xp = LD4(a.x_prev, v), g = LD4L2(a.g, v), gp = LD4(a.g_prev, v);
                    e(x.x, xp.x, g.x, gp.x);
                    e(x.y, xp.y, g.y, gp.y);
                    e(x.z, xp.z, g.z, gp.z);
                    e(x.w, xp.w, g.w, gp.w);
                    acc.tick();
                },
                [&](int64_t i) {
                    e(a.x[i], a.x_prev[i], a.g[i], a.g_prev[i]);
                    acc.tick();
                });
        } else {
            auto e = [&](float g) {
                acc.f[5] = fmaf(g, g, acc.f[5]);
                gmax = fmaxf(gmax, fabsf(g));
            };
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 g = LD4L2(a.g, v);
                    e(g.x);
                    e(g.y);
                    e(g.z);
                    e(g.w);
                    acc.tick();
                },
                [&](int64_t i) {
                    e(a.g[i]);
                    acc.tick();
                });
        }
        acc.fold();
        {
            float mx[1] = {gmax};
            block_reduce<6, 1>(acc.d, mx, sc);
        }
        if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, 6, 1, a.timeout_cycles,
                                [&](BlockScratch& s) { update_step_scalars(a, s, &cs->bc, &cs->info); }))
            return;
        fetch();
        if (bc.status != kOk) {
            if (blk == 0 && threadIdx.x == 0) {
                ws->st.info.status = bc.status;
                atomicCAS(&ws->ctrl.status, kOk, bc.status);
            }
            return;
        }
    }

    // ---------------------------------------------------------------- phase B
    {
        const float ch = a.proj ? 0.0f : bc.c_hi, cl = a.proj ? 0.0f : bc.c_lo;
        const float bh = a.proj ? 0.0f : bc.beta_hi, bl = a.proj ? 0.0f : bc.beta_lo;
        const bool first = a.t == 0;
        AccSplit<5 * M, 0> acc;
        acc.init();
        float mx[3 * M];  // per row: the upper saturation bound, minus the lower one, max |a_j|
        // a_j^T x_t enters b_j: exact products, hi parts summed with TwoSum, the rest in bl
        float bsh[M], bsl[M];
#pragma unroll
        for (int j = 0; j < M; ++j) mx[2 * j] = mx[2 * j + 1] = mx[2 * M + j] = bsh[j] = bsl[j] = 0.0f;
        const int eqm = a.eq_mask;
        // Stage 1 (params.stage1 on a cold start) brackets each row's single-row search with
        // the free-set curvature at 0, the row-minimising and row-maximising bound sums and the
        // saturation bounds (a division per element and row); stage 2 alone needs only b_j and
        // the rows' violation at lam = 0, so the lean variant of the pass sums those two
        const bool full = a.stage1 && !a.lam_prev;
        auto rowsum = [&](auto fullc, float z, const float (&av)[M], float x) {
            constexpr bool F = decltype(fullc)::value;
            const bool fr = z >= lo && z <= hi;
            const float xc = clampf(z, lo, hi);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float aj = av[j];
                const float ph = aj * x;
                const DF t = two_sum(bsh[j], ph);
                bsh[j] = t.hi;
                bsl[j] = __fadd_rn(bsl[j], __fadd_rn(t.lo, fmaf(aj, x, -ph)));
                acc.f[5 * j + 1] = fmaf(aj, xc, acc.f[5 * j + 1]);
                if constexpr (F) {
                    mx[2 * M + j] = fmaxf(mx[2 * M + j], fabsf(aj));
                    acc.f[5 * j + 2] = fr ? fmaf(aj, aj, acc.f[5 * j + 2]) : acc.f[5 * j + 2];
                    acc.f[5 * j + 3] += aj > 0.0f ? aj * lo : (aj < 0.0f ? aj * hi : 0.0f);
                    acc.f[5 * j + 4] += aj > 0.0f ? aj * hi : (aj < 0.0f ? aj * lo : 0.0f);
                    if (aj != 0.0f) {
                        // saturation bounds: only used widened by 1e-5, so a fast division will do
                        const float ra = __fdividef(1.0f, aj);
                        mx[2 * j] = fmaxf(mx[2 * j], (aj > 0.0f ? z - lo : z - hi) * ra);
                        if ((eqm >> j) & 1)
                            mx[2 * j + 1] = fmaxf(mx[2 * j + 1], -(aj > 0.0f ? z - hi : z - lo) * ra);
                    }
                }
            }
        };
        // d_t and z = x + c d_t in double-float (as in the single-row kernel)
        auto trial = [&](float x, float g, float dp, float& dout, float& zh, float& zl) {
            float uh, ul;
            if (first) {
                uh = -g;
                ul = 0.0f;
            } else {
                const float p = bh * dp;
                const float pe = fmaf(bh, dp, -p);
                const DF s = two_sum(p, -g);
                uh = s.hi;
                ul = __fadd_rn(s.lo, fmaf(bl, dp, pe));
            }
            const DF u = fast_two_sum(uh, ul);
            const float vh = ch * u.hi;
            const float ve = fmaf(ch, u.hi, -vh);
            const float vl = __fadd_rn(ve, fmaf(ch, u.lo, cl * u.hi));
            const DF s = two_sum(x, vh);
            const DF z = fast_two_sum(s.hi, __fadd_rn(s.lo, vl));
            dout = u.hi;
            zh = z.hi;
            zl = z.lo;
        };
        auto pass = [&](auto fullc) {
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 A4[M];
    #pragma unroll
                    for (int j = 0; j < M; ++j) A4[j] = LD4L2(a.A + (int64_t)j * n, v);
                    if (a.proj) {
                        float4 z = LD4L2(a.z_in, v);
                        const float zz[4] = {z.x, z.y, z.z, z.w};
    #pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float av[M];
    #pragma unroll
                            for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                            rowsum(fullc, zz[q], av, 0.0f);
                        }
                    } else {
                        float4 x = LD4(a.x, v), g = LD4(a.g, v);
                        float4 dp = first ? make_float4(0.f, 0.f, 0.f, 0.f) : LD4(a.d_prev, v);
                        float4 d, zh, zl;
                        const float xx[4] = {x.x, x.y, x.z, x.w}, gg[4] = {g.x, g.y, g.z, g.w};
                        const float pp[4] = {dp.x, dp.y, dp.z, dp.w};
                        float dd[4], h4[4], l4[4];
    #pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            trial(xx[q], gg[q], pp[q], dd[q], h4[q], l4[q]);
                            float av[M];
    #pragma unroll
                            for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                            rowsum(fullc, h4[q], av, xx[q]);
                        }
                        d = make_float4(dd[0], dd[1], dd[2], dd[3]);
                        zh = make_float4(h4[0], h4[1], h4[2], h4[3]);
                        zl = make_float4(l4[0], l4[1], l4[2], l4[3]);
                        __stcs(reinterpret_cast<float4*>(a.d_new) + v, d);
                        reinterpret_cast<float4*>(a.z)[v] = zh;
                        reinterpret_cast<float4*>(a.zlo)[v] = zl;
                        __stcs(reinterpret_cast<float4*>(a.x_prev) + v, x);
                        __stcs(reinterpret_cast<float4*>(a.g_prev) + v, g);
                    }
                    acc.tick();
                },
                [&](int64_t i) {
                    float av[M];
    #pragma unroll
                    for (int j = 0; j < M; ++j) av[j] = a.A[(int64_t)j * n + i];
                    if (a.proj) {
                        rowsum(fullc, a.z_in[i], av, 0.0f);
                    } else {
                        const float x = a.x[i], g = a.g[i];
                        float d, zh, zl;
                        trial(x, g, first ? 0.0f : a.d_prev[i], d, zh, zl);
                        a.d_new[i] = d;
                        a.z[i] = zh;
                        a.zlo[i] = zl;
                        a.x_prev[i] = x;
                        a.g_prev[i] = g;
                        rowsum(fullc, zh, av, x);
                    }
                    acc.tick();
                });
        };
        if (full) {
            pass(std::true_type{});
        } else {
            pass(std::false_type{});
        }
        acc.fold();
#pragma unroll
        for (int j = 0; j < M; ++j) acc.d[5 * j] = df_add(acc.d[5 * j], fast_two_sum(bsh[j], bsl[j]));
        block_reduce<5 * M, 3 * M>(acc.d, mx, sc);
        if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, 5 * M, 3 * M, a.timeout_cycles, [&](BlockScratch& s) {
                cupd_after_trial<M>(a, s, cs);
                __syncwarp();
                if (threadIdx.x == 0) {
                    volatile CoupledBcast* vb = &cs->bc;
                    if (vb->status != kOk) vb->mode = kModeDone;
                    else if (a.lam_prev) cupd_warm_start<M>(a, cs, false);
                    else if (!vb->any_active) cupd_plan_feasibility<M>(cs);
                    else if (a.stage1) vb->mode = kModeStage1;
                    else cupd_warm_start<M>(a, cs, true);
                    cfinish_if_done<M>(cs);
                }
            }))
            return;
        fetch();
        if (bc.status != kOk) {
            if (blk == 0 && threadIdx.x == 0) {
                ws->st.info.status = bc.status;
                atomicCAS(&ws->ctrl.status, kOk, bc.status);
            }
            return;
        }
    }

    // ---------------------------------------------------------------- S1, F, E, LS
    while (bc.mode != kModeDone) {
        const int mode = bc.mode;
        if (mode == kModeStage1) {
            // Alg. 2 stage 1: row j alone (others at zero), K points per active row
            for (int j = 0; j < M; ++j) {
                if (!bc.active[j]) continue;
                float p[K];
#pragma unroll
                for (int k = 0; k < K; ++k) p[k] = bc.pts[j][k];
                AccSplit<K, K> acc;
                acc.init();
                const float* Aj = a.A + (int64_t)j * n;
                auto e = [&](float z, float zl, float av) {
                    const float aa = av * av;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float w = __fadd_rn(fmaf(-p[k], av, z), zl);
                        const float x = clampf(w, lo, hi);  // free exactly when the clip leaves w
                        acc.f[k] = fmaf(av, x, acc.f[k]);
                        acc.f[K + k] += (x == w) ? aa : 0.0f;
                    }
                };
                for_chunk<VEC>(
                    cb, ce,
                    [&](int64_t v) {
                        float4 z = LD4L2(zh_src, v), av = LD4L2(Aj, v);
                        float4 zl = has_lo ? LD4L2(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f);
                        e(z.x, zl.x, av.x);
                        e(z.y, zl.y, av.y);
                        e(z.z, zl.z, av.z);
                        e(z.w, zl.w, av.w);
                        acc.tick();
                    },
                    [&](int64_t i) {
                        e(zh_src[i], has_lo ? a.zlo[i] : 0.0f, Aj[i]);
                        acc.tick();
                    });
                acc.fold();
                block_reduce<2 * K, 0>(acc.d, nullptr, sc, 2 * K * j, 0);
            }
            if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, 2 * K * M, 0, a.timeout_cycles,
                                    [&](BlockScratch& s) {
                                        search_pass_update(s, 0, cs->rows, &cs->bc, M, a.tol_lambda, a.max_passes);
                                        __syncwarp();
                                        if (threadIdx.x == 0) {
                                            volatile NewtonState* nt = &cs->nt;
                                            nt->passes = nt->passes + 1;
                                            if (!cs->bc.any_active) cupd_plan_feasibility<M>(cs);
                                            cfinish_if_done<M>(cs);
                                        }
                                    }))
                return;
        } else if (mode == kModeFeas) {
            // every row's sum at each single-row candidate lam_j e_j
            const int nc = bc.ncand;
            int crow[M];
            float clh[M], cll[M];
#pragma unroll
            for (int c = 0; c < M; ++c) {
                crow[c] = c < nc ? bc.cand_row[c] : 0;
                clh[c] = bc.lam_hi[crow[c]];
                cll[c] = bc.lam_lo[crow[c]];
            }
            AccSplit<M * M, 0> acc;
            acc.init();
            auto e = [&](float z, float zl, const float (&av)[M]) {
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    if (c >= nc) break;
                    float aj = av[0];
#pragma unroll
                    for (int q = 1; q < M; ++q) aj = crow[c] == q ? av[q] : aj;
                    const float w = __fadd_rn(fmaf(-clh[c], aj, z), fmaf(-cll[c], aj, zl));
                    const float x = clampf(w, lo, hi);
#pragma unroll
                    for (int k = 0; k < M; ++k) acc.f[c * M + k] = fmaf(av[k], x, acc.f[c * M + k]);
                }
            };
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 z = LD4L2(zh_src, v);
                    float4 zl = has_lo ? LD4L2(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 A4[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) A4[j] = LD4L2(a.A + (int64_t)j * n, v);
                    const float zz[4] = {z.x, z.y, z.z, z.w}, ll[4] = {zl.x, zl.y, zl.z, zl.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float av[M];
#pragma unroll
                        for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                        e(zz[q], ll[q], av);
                    }
                    acc.tick();
                },
                [&](int64_t i) {
                    float av[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) av[j] = a.A[(int64_t)j * n + i];
                    e(zh_src[i], has_lo ? a.zlo[i] : 0.0f, av);
                    acc.tick();
                });
            acc.fold();
            block_reduce<M * M, 0>(acc.d, nullptr, sc);
            if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, M * M, 0, a.timeout_cycles, [&](BlockScratch& s) {
                    cupd_after_feasibility<M>(a, s, cs);
                    if (threadIdx.x == 0) {
                        volatile NewtonState* nt = &cs->nt;
                        nt->passes = nt->passes + 1;
                        cfinish_if_done<M>(cs);
                    }
                }))
                return;
        } else if (mode == kModeEval) {
            // h, row magnitudes and J_h at the iterate (eq. h, eq. reg_jacobian)
            float lh[M], ll[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                lh[j] = bc.it_hi[j];
                ll[j] = bc.it_lo[j];
            }
            constexpr int NJ = M * (M + 1) / 2;
            AccSplit<M, M + NJ> acc;
            acc.init();
            auto e = [&](float z, float zl, const float (&av)[M]) {
                float w = z, wl = zl;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    w = fmaf(-lh[j], av[j], w);
                    wl = fmaf(-ll[j], av[j], wl);
                }
                w = __fadd_rn(w, wl);
                const float x = clampf(w, lo, hi);
                const bool fr = w >= lo && w <= hi;
                int t = 0;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const float ax = av[j] * x;
                    acc.f[j] += ax;
                    acc.f[M + j] += fabsf(ax);
#pragma unroll
                    for (int k = j; k < M; ++k) {
                        acc.f[2 * M + t] = fr ? fmaf(av[j], av[k], acc.f[2 * M + t]) : acc.f[2 * M + t];
                        ++t;
                    }
                }
            };
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 z = LD4L2(zh_src, v);
                    float4 zl = has_lo ? LD4L2(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 A4[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) A4[j] = LD4L2(a.A + (int64_t)j * n, v);
                    const float zz[4] = {z.x, z.y, z.z, z.w}, l4[4] = {zl.x, zl.y, zl.z, zl.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float av[M];
#pragma unroll
                        for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                        e(zz[q], l4[q], av);
                    }
                    acc.tick();
                },
                [&](int64_t i) {
                    float av[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) av[j] = a.A[(int64_t)j * n + i];
                    e(zh_src[i], has_lo ? a.zlo[i] : 0.0f, av);
                    acc.tick();
                });
            acc.fold();
            block_reduce<2 * M + NJ, 0>(acc.d, nullptr, sc);
            if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, 2 * M + NJ, 0, a.timeout_cycles,
                                    [&](BlockScratch& s) {
                                        cupd_after_eval<M>(a, s, cs);
                                        __syncwarp();
                                        if (threadIdx.x == 0) {
                                            volatile NewtonState* nt = &cs->nt;
                                            nt->passes = nt->passes + 1;
                                            cfinish_if_done<M>(cs);
                                        }
                                    }))
                return;
        } else {
            // exact line search along d: virtual row u = A^T d on w0 = z - A^T lam
            float lh[M], ll[M], dh[M], p[K];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                lh[j] = bc.it_hi[j];
                ll[j] = bc.it_lo[j];
                dh[j] = bc.d_hi[j];
            }
#pragma unroll
            for (int k = 0; k < K; ++k) p[k] = bc.pts[0][k];
            AccSplit<K, K> acc;
            acc.init();
            auto e = [&](float z, float zl, const float (&av)[M]) {
                float w = z, wl = zl, u = 0.0f;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    w = fmaf(-lh[j], av[j], w);
                    wl = fmaf(-ll[j], av[j], wl);
                    u = fmaf(dh[j], av[j], u);
                }
                w = __fadd_rn(w, wl);
                const float uu = u * u;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float wk = fmaf(-p[k], u, w);
                    const float xk = clampf(wk, lo, hi);
                    acc.f[k] = fmaf(u, xk, acc.f[k]);
                    acc.f[K + k] += (xk == wk) ? uu : 0.0f;
                }
            };
            for_chunk<VEC>(
                cb, ce,
                [&](int64_t v) {
                    float4 z = LD4L2(zh_src, v);
                    float4 zl = has_lo ? LD4L2(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 A4[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) A4[j] = LD4L2(a.A + (int64_t)j * n, v);
                    const float zz[4] = {z.x, z.y, z.z, z.w}, l4[4] = {zl.x, zl.y, zl.z, zl.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float av[M];
#pragma unroll
                        for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                        e(zz[q], l4[q], av);
                    }
                    acc.tick();
                },
                [&](int64_t i) {
                    float av[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) av[j] = a.A[(int64_t)j * n + i];
                    e(zh_src[i], has_lo ? a.zlo[i] : 0.0f, av);
                    acc.tick();
                });
            acc.fold();
            block_reduce<2 * K, 0>(acc.d, nullptr, sc);
            if (!grid_allreduce_update(&ws->ctrl, ws->part, sc, 2 * K, 0, a.timeout_cycles, [&](BlockScratch& s) {
                    cupd_after_line<M>(a, s, cs);
                    if (threadIdx.x == 0) cfinish_if_done<M>(cs);
                }))
                return;
        }
        fetch();
        if (bc.status != kOk) break;
    }

    // ---------------------------------------------------------------- phase D
    {
        float lh[M], ll[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            lh[j] = bc.lam_hi[j];
            ll[j] = bc.lam_lo[j];
        }
        AccSplit<M + 2, 0> acc;
        acc.init();
        // x = clip(z - sum_j lam_j a_j): hi parts with TwoSum, lo parts and product errors
        // gathered separately, so x is exact to FP32 rounding of the result
        auto e = [&](float x, float z, float zl, const float (&av)[M]) -> float {
            float sh = z, comp = zl;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float ph = lh[j] * av[j];
                const float pe = fmaf(lh[j], av[j], -ph);
                const DF t = two_sum(sh, -ph);
                sh = t.hi;
                comp = __fadd_rn(comp, __fsub_rn(t.lo, fmaf(ll[j], av[j], pe)));
            }
            const float xn = clampf(__fadd_rn(sh, comp), lo, hi);
#pragma unroll
            for (int j = 0; j < M; ++j) acc.f[j] = fmaf(av[j], xn, acc.f[j]);
            const float dx = xn - x;
            acc.f[M] = fmaf(dx, dx, acc.f[M]);
            acc.f[M + 1] = fmaf(xn, xn, acc.f[M + 1]);
            return xn;
        };
        float* out = a.proj ? a.x_out : a.x;
        for_chunk<VEC>(
            cb, ce,
            [&](int64_t v) {
                float4 z = LD4(zh_src, v);
                float4 zl = has_lo ? LD4(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 x = a.proj ? make_float4(0.f, 0.f, 0.f, 0.f) : LD4(a.x, v);
                float4 A4[M];
#pragma unroll
                for (int j = 0; j < M; ++j) A4[j] = LD4(a.A + (int64_t)j * n, v);
                const float zz[4] = {z.x, z.y, z.z, z.w}, l4[4] = {zl.x, zl.y, zl.z, zl.w};
                const float xx[4] = {x.x, x.y, x.z, x.w};
                float o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float av[M];
#pragma unroll
                    for (int j = 0; j < M; ++j) av[j] = reinterpret_cast<const float*>(&A4[j])[q];
                    o[q] = e(xx[q], zz[q], l4[q], av);
                }
                __stcs(reinterpret_cast<float4*>(out) + v, make_float4(o[0], o[1], o[2], o[3]));
                acc.tick();
            },
            [&](int64_t i) {
                float av[M];
#pragma unroll
                for (int j = 0; j < M; ++j) av[j] = a.A[(int64_t)j * n + i];
                out[i] = e(a.proj ? 0.0f : a.x[i], zh_src[i], has_lo ? a.zlo[i] : 0.0f, av);
                acc.tick();
            });
        acc.fold();
        block_reduce<M + 2, 0>(acc.d, nullptr, sc);
        const bool fin = grid_allreduce_update(&ws->ctrl, ws->part, sc, M + 2, 0, a.timeout_cycles,
                                               [&](BlockScratch& s) {
                                                   cupd_final<M>(a, s, cs, blk == 0 ? &ws->ctrl.status : nullptr,
                                                                 blk == 0 ? &ws->ctrl.launches : nullptr);
                                               });
        if (fin && blk == 0) {
            const unsigned* src = reinterpret_cast<const unsigned*>(&cs->info);
            unsigned* d = reinterpret_cast<unsigned*>(&ws->st.info);
            for (int i = threadIdx.x; i < (int)(sizeof(DeviceInfo) / 4); i += blockDim.x) d[i] = src[i];
        }
    }
}

template <bool VEC, int M>
static cudaError_t launch_coupled_t(const CoupledArgs& a, int blocks, cudaStream_t stream) {
    void* args[] = {const_cast<CoupledArgs*>(&a)};
    return cudaLaunchCooperativeKernel((void*)coupled_kernel<VEC, M>, dim3(blocks), dim3(kThreads), args, 0, stream);
}

cudaError_t launch_coupled(const CoupledArgs& a, int blocks, cudaStream_t stream) {
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec = al(a.x) && al(a.g) && al(a.A) && al(a.x_prev) && al(a.g_prev) && al(a.d_prev) &&
                     al(a.d_new) && al(a.z) && al(a.zlo) && al(a.z_in) && al(a.x_out) && (a.n % 4 == 0);
    switch (a.m) {
        case 2: return vec ? launch_coupled_t<true, 2>(a, blocks, stream) : launch_coupled_t<false, 2>(a, blocks, stream);
        case 3: return vec ? launch_coupled_t<true, 3>(a, blocks, stream) : launch_coupled_t<false, 3>(a, blocks, stream);
        case 4: return vec ? launch_coupled_t<true, 4>(a, blocks, stream) : launch_coupled_t<false, 4>(a, blocks, stream);
        default: return cudaErrorInvalidValue;
    }
}

int max_blocks_coupled(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per = 1 << 20;
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, coupled_kernel<true, 2>, kThreads, 0);
    per = v < per ? v : per;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, coupled_kernel<true, 4>, kThreads, 0);
    per = v < per ? v : per;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, coupled_kernel<false, 4>, kThreads, 0);
    per = v < per ? v : per;
    if (per < 1) per = 1;
    int nb = sms * per;
    return nb > kMaxBlocks ? kMaxBlocks : nb;
}

}  // namespace pgdto
