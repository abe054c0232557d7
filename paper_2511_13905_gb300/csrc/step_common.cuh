// step_common.cuh -- pieces shared by the single/independent-row and the coupled-row
// kernels: per-thread accumulators, the block-share iterator, the step-size update of
// Alg. 3, and the warp-parallel one-dimensional root search used for Alg. 1 rows and for
// the exact line search of the coupled Newton iteration.
#pragma once

#include <float.h>
#include <math.h>

#include "dev_common.cuh"
#include "kernels.h"

namespace pgdto {

constexpr int K = 8;           // trial points per root-search pass
constexpr int kFoldEvery = 2;  // float4 groups accumulated in FP32 before folding into DF
constexpr unsigned kFull = 0xffffffffu;

// State of one monotone piecewise-linear root search r(t) = S(t) - b - reg t = 0 on [L, H]
// with r(L) > 0 >= r(H); SL, SH are the slopes -dr/dt at the ends.
struct RowState {
    double b, L, rL, SL, H, rH, SH, lam, rlast, reg;
    double cC, cAA;  // free-set compaction: sum over decided elements of a*bound + a z, and of a^2
    double visited;  // element evaluations of this row's passes
    int active, passes, how, nrefine;  // nrefine: extra final passes at a refined root
    // the same bracket in float / double-float form: the per-pass update works on these
    // (FP64 issues at a small fraction of the FP32 rate here and sits on the critical path)
    float b_hi, b_lo, fL, fH, rL_hi, rL_lo, rH_hi, rH_lo, fSL, fSH, freg;
    float lam_hi, lam_lo;  // lam as a float pair
    float famax;           // max |a| over the row (single/independent rows; 0 where not set)
    float fzla;            // sum |a z_lo| over the row: the shift of a row sum without z_lo
};

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// ----------------------------------------------------------------------- scalar updates
//
// The updates run on warp 0 of every block (grid engine) or of the cluster's first block.
// FP64 throughput is a small fraction of FP32 on this part, a division is a long
// dependent sequence, and a warp instruction costs the same whatever its active lanes, so
// the work is spread over lanes: lane 8j + k handles trial point k of search j (4
// searches x 8 points = 32 lanes), per-search quantities are computed redundantly by the 8
// lanes of the group, and each update issues one warp-wide FP64 division.

// Step size and PR+ coefficient (Alg. 3; eq. final_alpha, eq. alpha, eq. CG), in
// double-float arithmetic (FP32 pipes; FP64 issues slowly here): the quotients to about
// 1e-14, far below what the FP32 trial point z = x + omega alpha d resolves.
template <class Args, class Bcast>
__device__ void update_step_scalars(const Args& a, const BlockScratch& sc, volatile Bcast* bc,
                                    volatile DeviceInfo* inf) {
    const int lane = threadIdx.x;
    const DF ss = sc.tot[0], sy = sc.tot[1], yy = sc.tot[2], gy = sc.tot[3], pp = sc.tot[4], gg = sc.tot[5];
    const float gmax = sc.totmax[0];
    const DF amax = DF{a.step_df[0], a.step_df[1]}, afb = DF{a.step_df[2], a.step_df[3]};
    const DF eps = DF{a.step_df[4], a.step_df[5]}, om = DF{a.step_df[6], a.step_df[7]};
    // the four quotients in one warp-wide division (each lane its own operands): lane 0 the
    // BB1 ratio s's / s'y, lane 1 s's / y'y (||s|| / ||y|| after the root), lane 2 the PR
    // coefficient g'y / ||g_prev||^2, lane 3 the fallback alpha_fb / ||g||_inf
    const DF num = lane == 0 ? ss : lane == 1 ? ss : lane == 2 ? gy : afb;
    const DF den = lane == 0 ? sy : lane == 1 ? yy : lane == 2 ? pp : DF{gmax, 0.0f};
    DF q = df_div(num, den);
    const DF rq = df_sqrt(q);
    const DF inf_df = DF{INFINITY, 0.0f};
    if (lane == 1) q = yy.hi > 0.0f ? rq : inf_df;
    else if (lane == 2) q = pp.hi > 0.0f ? q : df_zero();
    else if (lane == 3) q = gmax > 0.0f ? q : inf_df;
    const DF bb = DF{__shfl_sync(kFull, q.hi, 0), __shfl_sync(kFull, q.lo, 0)};
    const DF lip = DF{__shfl_sync(kFull, q.hi, 1), __shfl_sync(kFull, q.lo, 1)};
    const DF pr = DF{__shfl_sync(kFull, q.hi, 2), __shfl_sync(kFull, q.lo, 2)};
    const DF fbq = DF{__shfl_sync(kFull, q.hi, 3), __shfl_sync(kFull, q.lo, 3)};
    if (lane != 0) return;
    int status = kOk;
    if (!(isfinite(ss.hi) && isfinite(sy.hi) && isfinite(yy.hi) && isfinite(gy.hi) && isfinite(pp.hi) &&
          isfinite(gg.hi)))
        status = kErrNonfinite;
    const DF fb = df_min(amax, fbq);
    DF alpha;
    int branch;
    if (a.force_fallback || a.t == 0 || (ss.hi == 0.0f && ss.lo == 0.0f)) {
        alpha = fb;
        branch = 0;
    } else if (df_lt(eps, sy)) {
        alpha = df_min(df_min(bb, DF{2.0f * lip.hi, 2.0f * lip.lo}), amax);
        branch = 1;
    } else {
        alpha = df_min(lip, amax);
        branch = 2;
    }
    const DF beta = (a.t == 0 || !df_lt(df_zero(), pr)) ? df_zero() : pr;
    const DF c = df_mul(om, alpha);
    bc->c_hi = c.hi;
    bc->c_lo = c.lo;
    bc->beta_hi = beta.hi;
    bc->beta_lo = beta.lo;
    bc->branch = branch;
    bc->status = status;
    inf->alpha = df_to_double(alpha);
    inf->beta = df_to_double(beta);
    inf->branch = branch;
    inf->t = a.t;
}


__device__ __forceinline__ double float_ulp(double v) {
    float f = (float)fabs(v);
    return (double)nextafterf(f, INFINITY) - (double)f;
}

// Ascending bitonic sort of one float per lane within aligned groups of 8 lanes.
__device__ __forceinline__ float group8_sort(float v, int lane) {
    const int i = lane & 7;
#pragma unroll
    for (int size = 2; size <= 8; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const float o = __shfl_xor_sync(kFull, v, stride);
            const bool up = (i & size) == 0;
            const bool lower = (i & stride) == 0;
            v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return v;
}

// Trial point k of the next pass inside (L, H): Newton from the lower end (k = 0), from the
// upper end (k = 1), the secant point (k = 2), and a uniform fill (k = 3..7) that
// guarantees the bracket shrinks by at least a factor 6.  Returns the group-sorted value.
// A bracket that contains 0 or spans more than a factor of 4 is searched on a geometric
// ladder base * {1/8, 1/4, 1/2, 2, 4} around the Newton estimate from its zero end (the
// secant otherwise) rather than on uniform points: the saturation bound that closes the
// first bracket is often tens of times the root.
__device__ __forceinline__ bool wide_bracket(double L, double H) {
    const double a = fabs(L), b = fabs(H);
    return L * H <= 0.0 || fmax(a, b) > 4.0 * fmin(a, b);
}

__device__ __forceinline__ float next_point(int lane, double L, double rL, double H, double rH, double NL,
                                            double NH, bool cold = false) {
    const int k = lane & 7;
    const double w = H - L;
    double v;
    if (cold && wide_bracket(L, H)) {
        // a cold start: all eight points on the ladder around the Newton estimate from the
        // zero end, as next_point_warm_f does for single rows
        const double sec = L + rL * w / (rL - rH);
        const double base = (L == 0.0 && NL > L && NL < H) ? NL : (H == 0.0 && NH > L && NH < H) ? NH : sec;
        v = base * (k == 0 ? 0.125 : k == 1 ? 0.5 : k == 2 ? 0.8 : k == 3 ? 1.0 : k == 4 ? 1.2 : k == 5 ? 1.45
                    : k == 6 ? 2.0 : 4.0);
    } else if (k == 0) v = NL;
    else if (k == 1) v = NH;
    else if (k == 2) v = L + rL * w / (rL - rH);
    else if (wide_bracket(L, H)) {
        const double sec = L + rL * w / (rL - rH);
        const double base = (L == 0.0 && NL > L && NL < H) ? NL : (H == 0.0 && NH > L && NH < H) ? NH : sec;
        v = base * (k == 3 ? 0.125 : k == 4 ? 0.25 : k == 5 ? 0.5 : k == 6 ? 2.0 : 4.0);
    } else {
        v = L + w * (double)(k - 2) * (1.0 / 6.0);
    }
    if (!(v > L && v < H)) v = L + w * ((double)k + 0.5) * 0.125;
    float f = (float)v;
    if (!((double)f > L && (double)f < H)) {
        f = (float)(0.5 * (L + H));
        if (!((double)f > L && (double)f < H)) f = (float)H;
    }
    return group8_sort(f, lane);
}

// Warm-start ladder: K points around the previous step's root lp in ascending order,
// lp (1 -+ 0.003), (1 -+ 0.01), (1 -+ 0.03), (1 -+ 0.1).  They need no bracket, so a step
// with a usable lp evaluates them in the same pass that forms the trial point (the search's
// first pass then costs no round of its own).  Computed in FP32 from the rounded lp, the
// same way by every CTA and by the update that reads the sums.
__device__ __forceinline__ bool ladder_usable(float lp) { return lp != 0.0f && isfinite(lp); }

__device__ __forceinline__ float ladder_point(float lp, int k) {
    const int i = lp > 0.0f ? k : K - 1 - k;
    const float f = i == 0 ? 0.9f
                  : i == 1 ? 0.97f
                  : i == 2 ? 0.99f
                  : i == 3 ? 0.997f
                  : i == 4 ? 1.003f
                  : i == 5 ? 1.01f
                  : i == 6 ? 1.03f
                  : 1.1f;
    return lp * f;
}

// First points of a search that has the previous step's root lp (warm start): Newton from
// both ends, the secant, the midpoint, and a ladder lp (1 -+ 0.003), lp (1 -+ 0.03) around
// it, since a design's dual moves little from one step to the next.  Without a usable lp
// (outside (L, H)) the points are next_point's.  Either way any lp only changes where the
// first pass looks.  Every lane reaches the one group8_sort (full-warp shuffles).  The
// caller passes the Newton points NL, NH and the secant point sec = L + rL (H - L) / (rL -
// rH), so that no lane divides here.
__device__ __forceinline__ float next_point_warm(int lane, double L, double H, double NL, double NH, double sec,
                                                 double lp) {
    const int k = lane & 7;
    const bool warm = lp > L && lp < H;
    const double w = H - L;
    double v;
    if (k == 0) v = NL;
    else if (k == 1) v = NH;
    else if (k == 2) v = sec;
    else if (!warm && wide_bracket(L, H)) {
        const double base = (L == 0.0 && NL > L && NL < H) ? NL : (H == 0.0 && NH > L && NH < H) ? NH : sec;
        v = base * (k == 3 ? 0.125 : k == 4 ? 0.25 : k == 5 ? 0.5 : k == 6 ? 2.0 : 4.0);
    } else if (!warm) v = L + w * (double)(k - 2) * (1.0 / 6.0);
    else if (k == 3) v = L + 0.5 * w;
    else v = lp * (k == 4 ? 0.97 : k == 5 ? 0.997 : k == 6 ? 1.003 : 1.03);
    if (!(v > L && v < H)) v = L + w * ((double)k + 0.5) * 0.125;
    float fv = (float)v;
    if (!((double)fv > L && (double)fv < H)) {
        fv = (float)(0.5 * (L + H));
        if (!((double)fv > L && (double)fv < H)) fv = (float)H;
    }
    return group8_sort(fv, lane);
}

// next_point_warm in FP32 (the points are FP32 anyway), from the float bracket [L, H] and
// the Newton points NL, NH and secant point sec already formed.
__device__ __forceinline__ float next_point_warm_f(int lane, float L, float H, float NL, float NH, float sec,
                                                   float lp) {
    const int k = lane & 7;
    const bool warm = lp > L && lp < H;
    const float w = H - L;
    const float am = fabsf(L), bm = fabsf(H);
    float v;
    if (!warm && (L * H <= 0.0f || fmaxf(am, bm) > 4.0f * fminf(am, bm))) {
        // a cold start's bracket runs from 0 to a saturation bound, often tens of times the
        // root, so Newton from its far end and the secant are wasted: all eight points go on a
        // ladder around the Newton estimate from the zero end, dense near it (the estimate
        // is usually within a few tens of percent) with far points in case it is not
        const float base = (L == 0.0f && NL > L && NL < H) ? NL : (H == 0.0f && NH > L && NH < H) ? NH : sec;
        v = base * (k == 0 ? 0.125f : k == 1 ? 0.5f : k == 2 ? 0.8f : k == 3 ? 1.0f : k == 4 ? 1.2f
                    : k == 5 ? 1.45f : k == 6 ? 2.0f : 4.0f);
    } else if (k == 0) v = NL;
    else if (k == 1) v = NH;
    else if (k == 2) v = sec;
    else if (!warm) v = fmaf(w, (float)(k - 2) * (1.0f / 6.0f), L);
    else if (k == 3) v = fmaf(0.5f, w, L);
    else v = lp * (k == 4 ? 0.97f : k == 5 ? 0.997f : k == 6 ? 1.003f : 1.03f);
    if (!(v > L && v < H)) v = fmaf(w, ((float)k + 0.5f) * 0.125f, L);
    if (!(v > L && v < H)) {
        v = L + 0.5f * w;
        if (!(v > L && v < H)) v = H;
    }
    return group8_sort(v, lane);
}

__device__ __forceinline__ void store_row(volatile RowState* r, double b, double L, double rL, double SL, double H,
                                          double rH, double SH, double lam, double rlast, int active, int passes,
                                          int how) {
    r->b = b;  // reg (the slope of the regulariser term) is set once when the search starts
    r->L = L;
    r->rL = rL;
    r->SL = SL;
    r->H = H;
    r->rH = rH;
    r->SH = SH;
    r->lam = lam;
    {
        float lh, ll;
        split_double(lam, lh, ll);
        r->lam_hi = lh;
        r->lam_lo = ll;
    }
    r->rlast = rlast;
    r->active = active;
    r->passes = passes;
    r->how = how;
    r->nrefine = 0;
    r->cC = 0.0;
    r->cAA = 0.0;
    r->visited = 0.0;
    float h, l;
    split_double(b, h, l);
    r->b_hi = h;
    r->b_lo = l;
    split_double(rL, h, l);
    r->rL_hi = h;
    r->rL_lo = l;
    split_double(rH, h, l);
    r->rH_hi = h;
    r->rH_lo = l;
    r->fL = (float)L;  // bracket ends are float trial points (or 0 / the float saturation bound)
    r->fH = (float)H;
    r->fSL = (float)SL;
    r->fSH = (float)SH;
    r->freg = (float)r->reg;
    r->famax = 0.0f;
    r->fzla = 0.0f;
}

// Refresh the float / double-float copy of a bracket whose FP64 fields were set directly.
__device__ __forceinline__ void row_refresh_floats(volatile RowState* r) {
    float h, l;
    split_double(r->b, h, l);
    r->b_hi = h;
    r->b_lo = l;
    split_double(r->rL, h, l);
    r->rL_hi = h;
    r->rL_lo = l;
    split_double(r->rH, h, l);
    r->rH_hi = h;
    r->rH_lo = l;
    r->fL = (float)r->L;
    r->fH = (float)r->H;
    r->fSL = (float)r->SL;
    r->fSH = (float)r->SH;
    r->freg = (float)r->reg;
}

template <class Bcast>
__device__ __forceinline__ void publish_lambda(volatile Bcast* bc, int j, double lam) {
    float h, l;
    split_double(lam, h, l);
    bc->lam_hi[j] = h;
    bc->lam_lo[j] = l;
    bc->active[j] = 0;
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

template <class Bcast>
__device__ __forceinline__ void publish_lambda_df(volatile Bcast* bc, int j, DF lam) {
    bc->lam_hi[j] = lam.hi;
    bc->lam_lo[j] = lam.lo;
    bc->active[j] = 0;
}

// store_row for a search formed in double-float (single and independent rows): the
// bracket is kept in its float / double-float form only (what the passes' update reads);
// b, lam and rlast also in FP64 for the final refinement and the report.
__device__ __forceinline__ void store_row_df(volatile RowState* r, DF b, float L, DF rL, DF SL, float H, DF rH,
                                             DF SH, DF lam, double rlast, float freg, int active, int how) {
    r->b = df_to_double(b);
    r->L = 0.0;
    r->rL = 0.0;
    r->SL = 0.0;
    r->H = 0.0;
    r->rH = 0.0;
    r->SH = 0.0;
    r->lam = df_to_double(lam);
    r->lam_hi = lam.hi;
    r->lam_lo = lam.lo;
    r->rlast = rlast;
    r->active = active;
    r->passes = 0;
    r->how = how;
    r->nrefine = 0;
    r->cC = 0.0;
    r->cAA = 0.0;
    r->visited = 0.0;
    r->b_hi = b.hi;
    r->b_lo = b.lo;
    r->rL_hi = rL.hi;
    r->rL_lo = rL.lo;
    r->rH_hi = rH.hi;
    r->rH_lo = rH.lo;
    r->fL = L;
    r->fH = H;
    r->fSL = SL.hi;
    r->fSH = SH.hi;
    r->freg = freg;
    r->famax = 0.0f;
    r->fzla = 0.0f;
}


// a / b for a double-float a and a float b, to double-float accuracy.
__device__ __forceinline__ DF df_div_f(DF a, float b) {
    const float q1 = __fdiv_rn(a.hi, b);
    const float r = __fadd_rn(fmaf(-q1, b, a.hi), a.lo);
    return fast_two_sum(q1, __fdiv_rn(r, b));
}

__device__ __forceinline__ bool df_pos(DF a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }

__device__ __forceinline__ float float_ulp_f(float v) {
    const float f = fabsf(v);
    return nextafterf(f, INFINITY) - f;
}

// v moved by k float spacings towards +infinity (v finite and non-zero; the caller keeps
// the result inside the bracket).
__device__ __forceinline__ float float_steps(float v, int k) {
    return __int_as_float(__float_as_int(v) + (v > 0.0f ? k : -k));
}

// Root in (L, H) of the cubic Hermite interpolant of r on the bracket: values rL > 0 >= rH
// and slopes -SL, -SH at its ends.  A safeguarded Newton iteration on the cubic in
// t = (lam - L) / (H - L), started at the secant point, keeping the sign bracket in t.
__device__ __forceinline__ float hermite_root(float L, float H, float rL, float rH, float SL, float SH) {
    const float w = H - L;
    const float dL = -SL * w, dH = -SH * w;
    const float c1 = dL;
    const float c2 = 3.0f * (rH - rL) - 2.0f * dL - dH;
    const float c3 = 2.0f * (rL - rH) + dL + dH;
    float tl = 0.0f, th = 1.0f;
    float t = __fdividef(rL, rL - rH);
    if (!(t > 0.0f && t < 1.0f)) t = 0.5f;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const float f = fmaf(fmaf(fmaf(c3, t, c2), t, c1), t, rL);
        if (f > 0.0f) tl = t;
        else th = t;
        const float fp = fmaf(fmaf(3.0f * c3, t, 2.0f * c2), t, c1);
        float tn = t - __fdividef(f, fp);
        if (!(tn > tl && tn < th)) tn = 0.5f * (tl + th);
        t = tn;
    }
    return fmaf(t, w, L);
}

// Trial point k of the next pass inside (L, H), float version of next_point.
//  * Once the Newton predictions from both ends lie inside the bracket and agree to a few
//    float spacings, the root is located as finely as FP32 trial points can express it:
//    the points are the floats around the prediction (-4, -2, -1, 0, +1, +2, +4, +8
//    spacings), so the bracket closes on two neighbouring floats in one pass.
//  * A bracket that contains 0 or spans more than a factor of 4 keeps the geometric
//    ladder around the Newton estimate from its zero end (the secant otherwise).
//  * Otherwise: Newton from both ends, the secant, the root e of the cubic Hermite
//    interpolant of the bracket (values and slopes at both ends: far more accurate than
//    either Newton step on a smooth stretch of r), and e -+ d, e -+ d/4 with d the largest
//    distance from e to the other estimates, so the points cluster where the root is.
__device__ __forceinline__ float next_point_f(int lane, float L, float rL, float H, float rH, float NL, float NH,
                                              float SL, float SH) {
    const int k = lane & 7;
    const float w = H - L;
    const float am = fabsf(L), bm = fabsf(H);
    const float ulp = float_ulp_f(fmaxf(am, bm));
    const bool inL = NL > L && NL < H, inH = NH > L && NH < H;
    const bool tight = inL && inH && fabsf(NL - NH) <= 16.0f * ulp;
    const float sec = L + rL * __fdiv_rn(w, rL - rH);
    float v;
    if (tight) {
        const float e = 0.5f * NL + 0.5f * NH;
        v = e == 0.0f ? e : float_steps(e, k == 0 ? -4 : k == 1 ? -2 : k == 2 ? -1 : k == 3 ? 0 : k == 4 ? 1
                                          : k == 5 ? 2 : k == 6 ? 4 : 8);
    } else if (k == 0) v = NL;
    else if (k == 1) v = NH;
    else if (k == 2) v = sec;
    else if (L * H <= 0.0f || fmaxf(am, bm) > 4.0f * fminf(am, bm)) {
        const float base = (L == 0.0f && inL) ? NL : (H == 0.0f && inH) ? NH : sec;
        v = base * (k == 3 ? 0.125f : k == 4 ? 0.25f : k == 5 ? 0.5f : k == 6 ? 2.0f : 4.0f);
    } else {
        const float e = hermite_root(L, H, rL, rH, SL, SH);
        const bool inS = sec > L && sec < H;
        float d = ulp;
        if (inL) d = fmaxf(d, fabsf(NL - e));
        if (inH) d = fmaxf(d, fabsf(NH - e));
        if (inS) d = fmaxf(d, fabsf(sec - e));
        v = k == 3 ? e : k == 4 ? e - d : k == 5 ? e + d : k == 6 ? fmaf(-0.25f, d, e) : fmaf(0.25f, d, e);
    }
    if (!(v > L && v < H)) v = fmaf(w, ((float)k + 0.5f) * 0.125f, L);
    if (!(v > L && v < H)) {
        v = L + 0.5f * w;
        if (!(v > L && v < H)) v = H;
    }
    return group8_sort(v, lane);
}

// One pass of the root searches: the pass evaluated, for each active search j, the sums
// S(t_k) (tot[base + 2K j + k], double-float) and the free-set curvature (tot[base + 2K j +
// K + k], float) at the points bc->pts[j][k].  Moves each bracket, stops a search when
// Newton from both ends of its bracket agrees (both ends on one linear piece), when the
// bracket is within tol or a few float spacings, or at max_passes (flagged), and writes
// the next points.  Works in float and double-float; FP64 only for a finished root.
// CMP: the pass summed only the elements not yet decided (free-set compaction); each row
// then adds the decided elements' part, C + sum a z - t_k sum a^2, from its row state,
// and the pass's three extra sums (the elements it decided) join that state.
// Searches in `held` (bit j) were not evaluated in this pass: they keep their bracket and
// points and stay active.
// DEC: the pass summed per point only the elements whose clip state changes between the
// lowest and the highest point; the others came as three sums at tot[base + stride j + 2K
// ...]: C (a x bound over the elements clipped at every point), AZ (a w_m over those free
// at every point, w_m their value at the reference point t_m = pts[j][kMidPoint]) and AA
// (a^2 over the same), and each point adds C + AZ - (t_k - t_m) AA and AA back.
// Out of line: a step calls it from more than one place (the warm-start ladder's round and
// the later passes, the coupled rows' stage 1 and line search), and one copy of its code
// is fetched into the instruction cache once per launch instead of once per call site.
constexpr int kMidPoint = 3;

template <class Bcast, bool CMP = false, bool DEC = false>
__device__ __noinline__ void search_pass_update(const BlockScratch& sc, int base, volatile RowState* rows,
                                                volatile Bcast* bc, int nsearch, double tol_lambda, int max_passes,
                                                unsigned held = 0u) {
    static_assert(!(CMP && DEC), "one pass layout at a time");
    constexpr int stride = CMP ? 2 * K + 4 : (DEC ? 2 * K + 3 : 2 * K);
    const int lane = threadIdx.x, j = lane >> 3, k = lane & 7, g0 = lane & ~7;
    const int jj = j < nsearch ? j : 0;
    const bool act = j < nsearch && rows[jj].active;
    const bool hold = act && ((held >> jj) & 1u);
    const bool row = act && !hold;
    const float reg = rows[jj].freg;
    const DF b = DF{rows[jj].b_hi, rows[jj].b_lo};
    float L = rows[jj].fL, H = rows[jj].fH, SL = rows[jj].fSL, SH = rows[jj].fSH;
    DF rL = DF{rows[jj].rL_hi, rows[jj].rL_lo}, rH = DF{rows[jj].rH_hi, rows[jj].rH_lo};
    const int passes = rows[jj].passes + 1;
    const float lk = bc->pts[jj][k];
    // r_k = S_k - b - reg t_k
    const float pr = reg * lk;
    DF rk = df_add(sc.tot[base + stride * jj + k], df_neg(b));
    rk = df_add(rk, DF{-pr, -fmaf(reg, lk, -pr)});
    float Sk = sc.tot[base + stride * jj + K + k].hi + reg;
    if (CMP) {
        float ch, cl;
        split_double(rows[jj].cC - (double)lk * rows[jj].cAA, ch, cl);
        rk = df_add(rk, DF{ch, cl});
        Sk += (float)rows[jj].cAA;
    }
    if (DEC) {
        const int o = base + stride * jj + 2 * K;
        const float tm = __shfl_sync(kFull, lk, g0 + kMidPoint);
        const DF aa = sc.tot[o + 2];
        const DF dec = df_add(df_add(sc.tot[o], sc.tot[o + 1]), df_neg(df_mul(two_sum(lk, -tm), aa)));
        rk = df_add(rk, dec);
        Sk += aa.hi;
    }
    // new lower end: the largest point with r > 0; new upper end: the smallest point above
    // it with r <= 0 (points the rounding noise puts out of order are ignored)
    const unsigned pos = (__ballot_sync(kFull, row && df_pos(rk) && lk > L && lk < H) >> g0) & 0xffu;
    const int kL = pos ? 31 - __clz(pos) : -1;
    const int sL = g0 + (kL < 0 ? 0 : kL);
    const float lL = __shfl_sync(kFull, lk, sL);
    const float rLh = __shfl_sync(kFull, rk.hi, sL), rLl = __shfl_sync(kFull, rk.lo, sL);
    const float SLn = __shfl_sync(kFull, Sk, sL);
    if (kL >= 0) {
        L = lL;
        rL = DF{rLh, rLl};
        SL = SLn;
    }
    const unsigned neg = (__ballot_sync(kFull, row && !df_pos(rk) && lk > L && lk < H) >> g0) & 0xffu;
    const int kH = neg ? __ffs(neg) - 1 : -1;
    const int sH = g0 + (kH < 0 ? 0 : kH);
    const float hH = __shfl_sync(kFull, lk, sH);
    const float rHh = __shfl_sync(kFull, rk.hi, sH), rHl = __shfl_sync(kFull, rk.lo, sH);
    const float SHn = __shfl_sync(kFull, Sk, sH);
    if (kH >= 0) {
        H = hH;
        rH = DF{rHh, rHl};
        SH = SHn;
    }
    // Newton from both ends, NL = L + rL / SL and NH = H + rH / SH, in double-float
    DF q = df_zero();
    if (k == 0) q = df_div_f(rL, SL);
    else if (k == 1) q = df_div_f(rH, SH);
    const DF qL = DF{__shfl_sync(kFull, q.hi, g0), __shfl_sync(kFull, q.lo, g0)};
    const DF qH = DF{__shfl_sync(kFull, q.hi, g0 + 1), __shfl_sync(kFull, q.lo, g0 + 1)};
    const DF NL = df_add_f(qL, L), NH = df_add_f(qH, H);
    const DF gap = df_add(NL, df_neg(NH));
    const DF wd = two_sum(H, -L);
    const float w = wd.hi;
    // tolerances relative to the bracket's magnitude (a negative bracket ends at 0).  Where
    // the row's largest |a| is known the search may also stop once the two Newton
    // predictions agree to 1000 tol_lambda of the root and to 1e-8 / max|a|: the final pass
    // then takes one exact Newton step from their midpoint, which is within half that gap of
    // the root, so (at the default tol_lambda) the step moves x by less than 1e-8 and lam by
    // less than 5e-8 of itself, inside the final pass's acceptance window (1e-7 for both);
    // its own test runs the pass again if it is not
    const float mag = fmaxf(fabsf(L), fabsf(H));
    const float tol = (float)tol_lambda * mag;
    const float am = rows[jj].famax;
    const float tolg = am > 0.0f ? fmaxf(tol, fminf(1000.0f * tol, __fdividef(1e-8f, am))) : tol;
    bool done = false;
    int how = 2;
    if (kH >= 0 && rH.hi == 0.0f && rH.lo == 0.0f) done = true;
    else if (fabsf(gap.hi) <= tolg || w <= tol || w <= 4.0f * float_ulp_f(mag)) done = true;
    if (!done && passes >= max_passes) {
        done = true;
        how = 3;  // not converged
    }
    done = done && row;
    const float p = next_point_f(lane, L, rL.hi, H, rH.hi, NL.hi, NH.hi, SL, SH);
    if (row && k == 0) {
        volatile RowState* r = &rows[j];
        r->fL = L;
        r->fH = H;
        r->fSL = SL;
        r->fSH = SH;
        r->rL_hi = rL.hi;
        r->rL_lo = rL.lo;
        r->rH_hi = rH.hi;
        r->rH_lo = rH.lo;
        r->passes = passes;
        if (CMP) {
            const int o = base + stride * j + 2 * K;
            r->cC = r->cC + df_to_double(sc.tot[o]) + df_to_double(sc.tot[o + 1]);
            r->cAA = r->cAA + df_to_double(sc.tot[o + 2]);
            r->visited = r->visited + df_to_double(sc.tot[o + 3]);
        }
        if (done) {
            // the root: the midpoint of the two Newton predictions (double-float), in [L, H]
            DF root;
            if (kH >= 0 && rH.hi == 0.0f && rH.lo == 0.0f) {
                root = DF{H, 0.0f};
            } else {
                const DF s2 = df_add(NL, NH);
                root = DF{0.5f * s2.hi, 0.5f * s2.lo};
            }
            if (df_lt(root, DF{L, 0.0f})) root = DF{L, 0.0f};
            if (df_lt(DF{H, 0.0f}, root)) root = DF{H, 0.0f};
            r->lam = df_to_double(root);
            r->lam_hi = root.hi;
            r->lam_lo = root.lo;
            r->rlast = (double)fmaxf(fabsf(rL.hi), fabsf(rH.hi));
            r->active = 0;
            r->how = how;
            publish_lambda_df(bc, j, root);
        }
    }
    if (row && !done) bc->pts[j][k] = p;
    const unsigned still = __ballot_sync(kFull, (row && !done) || hold);
    if (lane == 0) bc->any_active = still ? 1 : 0;
}

// ----------------------------------------------------------------------- element passes

template <int N>
struct Acc {
    float f[N];
    DF d[N];
    int cnt;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            f[i] = 0.0f;
            d[i] = df_zero();
        }
        cnt = 0;
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            d[i] = df_add_f(d[i], f[i]);
            f[i] = 0.0f;
        }
        cnt = 0;
    }
    __device__ __forceinline__ void tick() {
        if (++cnt == kFoldEvery) fold();
    }
};

// Accumulators whose first NP entries fold into double-float after every PF float4
// groups and whose other NQ entries after every PS groups.  The defaults (1, 4) serve the
// single passes whose sums enter the result (b, the final residual); the root-search passes
// only steer the search (the final pass recomputes r exactly and refines the root), so
// they fold less often.
constexpr int kFoldSlow = 4;

template <int NP, int NQ, int PF = 1, int PS = kFoldSlow>
struct AccSplit {
    static_assert(PS % PF == 0, "the slow fold period must be a multiple of the fast one");
    static constexpr int N = NP + NQ;
    float f[N];
    DF d[N];
    int cnt;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            f[i] = 0.0f;
            d[i] = df_zero();
        }
        cnt = 0;
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            d[i] = df_add_f(d[i], f[i]);
            f[i] = 0.0f;
        }
        cnt = 0;
    }
    __device__ __forceinline__ void tick() {
        ++cnt;
        if (cnt % PF == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                d[i] = df_add_f(d[i], f[i]);
                f[i] = 0.0f;
            }
        }
        if (cnt == PS) {
#pragma unroll
            for (int i = NP; i < N; ++i) {
                d[i] = df_add_f(d[i], f[i]);
                f[i] = 0.0f;
            }
            cnt = 0;
        }
    }
};

// Iterate the block's share [cb, ce): f4(v) for aligned float4 groups v (elements 4v..4v+3),
// f1(i) for the unaligned head and tail, then tick() per group.
template <bool VEC, class F4, class F1>
__device__ __forceinline__ void for_chunk(int64_t cb, int64_t ce, F4&& f4, F1&& f1) {
    if (VEC) {
        int64_t vb = (cb + 3) & ~int64_t(3);
        if (vb > ce) vb = ce;
        int64_t ve = ce & ~int64_t(3);
        if (ve < vb) ve = vb;
        for (int64_t i = cb + threadIdx.x; i < vb; i += blockDim.x) f1(i);
        for (int64_t v = (vb >> 2) + threadIdx.x; v < (ve >> 2); v += blockDim.x) f4(v);
        for (int64_t i = ve + threadIdx.x; i < ce; i += blockDim.x) f1(i);
    } else {
        for (int64_t i = cb + threadIdx.x; i < ce; i += blockDim.x) f1(i);
    }
}

// for_chunk with two float4 groups per iteration: load4(v) issues a group's loads and
// returns them, use4(data) consumes them (and ticks).  Both groups' loads are in flight
// before either is used, which hides more of the memory latency of a streaming pass.
// The groups are consumed in the same order as for_chunk's, so the sums are the same bits.
template <bool VEC, class L4, class U4, class F1>
__device__ __forceinline__ void for_chunk_x2(int64_t cb, int64_t ce, L4&& load4, U4&& use4, F1&& f1) {
    if (VEC) {
        int64_t vb = (cb + 3) & ~int64_t(3);
        if (vb > ce) vb = ce;
        int64_t ve = ce & ~int64_t(3);
        if (ve < vb) ve = vb;
        for (int64_t i = cb + threadIdx.x; i < vb; i += blockDim.x) f1(i);
        const int64_t st = blockDim.x, v1 = ve >> 2;
        int64_t v = (vb >> 2) + threadIdx.x;
        for (; v + st < v1; v += 2 * st) {
            auto d0 = load4(v);
            auto d1 = load4(v + st);
            use4(d0);
            use4(d1);
        }
        if (v < v1) use4(load4(v));
        for (int64_t i = ve + threadIdx.x; i < ce; i += blockDim.x) f1(i);
    } else {
        for (int64_t i = cb + threadIdx.x; i < ce; i += blockDim.x) f1(i);
    }
}

#define LD4(p, v) (__ldcs(reinterpret_cast<const float4*>(p) + (v)))
#define LD4L2(p, v) (__ldcg(reinterpret_cast<const float4*>(p) + (v)))


}  // namespace pgdto
