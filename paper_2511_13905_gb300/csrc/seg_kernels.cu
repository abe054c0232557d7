// seg_kernels.cu -- fused PGD-TO step / projection for one row or independent rows.
//
// One cooperative launch runs the whole step (Alg. 3) for m = 1 (Alg. 1) and for rows
// with disjoint supports (Sec. 3.2.2), each row owning a contiguous segment of x:
//
//   phase A  one pass over x, x_prev, g, g_prev: s^T s, s^T y, y^T y, g^T y, ||g_prev||^2,
//            ||g||_inf  ->  alpha (eq. final_alpha / eq. alpha / fallback) and beta (eq. CG)
//   phase B  one pass: d = -g + beta d_prev, z = x + omega alpha d; writes d, z and the
//            state copies; per row a^T x_t (for b), r(0) (Alg. 1 feasibility test), the
//            free-set curvature at 0 and the saturation bound of Alg. 1's bracket
//   phase C  root-search passes over z and a: r(lam_k) = a^T clip(z - lam_k a) - b - 2 lam_k/C
//            and its slope at K points per pass; the scalar update moves the bracket, stops
//            when both ends lie on one linear piece, and picks the next points
//   phase D  one pass: x_{t+1} = clip(x + c(beta d_prev - g) - lam a) evaluated in
//            double-float arithmetic, a^T x_{t+1}, ||x_{t+1} - x_t||^2, ||x_{t+1}||^2
//
// The projection-only entry runs B (without the step part), C and D on a given z.
// Each phase ends in one grid-wide reduction (dev_common.cuh); with a warm start the first
// search pass is evaluated right after phase B and shares its reduction.
#include <float.h>
#include <math.h>
#include <string.h>

#include <cooperative_groups.h>

#include "dev_common.cuh"
#include "kernels.h"
#include "step_common.cuh"

namespace cg = cooperative_groups;

namespace pgdto {

// Values per row in the trial-point pass's reduction: a^T x_t, r(0) + b, the free-set
// curvature at 0, the sums of a times the row-minimising and row-maximising bounds, and
// sum |a z_lo| (how far the FP32 trial point z_hi alone moves a row sum).
constexpr int kBVals = 6;

struct SegBcast {
    float c_hi, c_lo, beta_hi, beta_lo;  // step scalars c = omega alpha and beta as float pairs
    int branch, any_active, status, refine;  // refine: phase D runs again at the refined lam
    float pts[kMaxRows][K];
    int active[kMaxRows];
    float lam_hi[kMaxRows], lam_lo[kMaxRows];
    int cmode[kMaxRows];              // free-set compaction: 0 all elements, 1 all + build lists, 2 lists
    float brL[kMaxRows], brH[kMaxRows];  // the bracket the current points lie in
};

// Search state of one problem: in global memory for the grid engine, in the shared memory
// of the cluster's first CTA for the cluster engine.
struct SegState {
    SegBcast bc;
    RowState rows[kMaxRows];
    DeviceInfo info;
};

struct SegWork {
    GridCtrl ctrl;
    SegState st;       // the grid engine's report (info) after a launch
    Partials part[2];  // block partials of alternate rounds
};

size_t seg_work_bytes() { return sizeof(SegWork); }
size_t seg_work_ctrl_bytes() { return sizeof(GridCtrl); }
DeviceInfo* seg_work_info(SegWork* ws) { return &ws->st.info; }

__device__ __forceinline__ bool all_finite(const BlockScratch& sc, int nv) {
    for (int i = 0; i < nv; ++i)
        if (!isfinite(sc.tot[i].hi)) return false;
    return true;
}

// ----------------------------------------------------------------------- scalar updates
//
// The updates run on warp 0 of every block (grid engine) or of the cluster's first block.
// FP64 throughput is a small fraction of FP32 on this part, a division is a long
// dependent sequence, and a warp instruction costs the same whatever its active lanes, so
// the work is spread over lanes: lane 8j + k handles trial point k of row j (4 rows x 8
// points = 32 lanes), per-row quantities are computed redundantly by the 8 lanes of the
// row's group, and each update issues one warp-wide FP64 division.

// After phase B: feasibility at lam = 0, bracket [0, H] (Alg. 1), closed form when the row
// is violated even with every variable at its row-minimising bound (regularised root).
// An equality row (Sec. 3.2.4) with r(0) < 0 binds from below: its root is negative, in
// [L, 0] with L the lowest breakpoint (every variable at its row-maximising bound below
// it), or (C/2)(S_max - b) when even that point leaves r < 0.
// ladder: the pass evaluated with phase B used the warm-start ladder; rows with a usable
// previous root take their points from it, so the first points are computed only when
// some row has none.
__device__ void update_after_trial(const SegArgs& a, const BlockScratch& sc, SegState* ws, bool ladder = false) {
    // double-float throughout (FP32 pipes; FP64 issues slowly here), FP64 only for the
    // values kept for the report and the final refinement
    const int lane = threadIdx.x, j = lane >> 3, k = lane & 7;
    volatile SegBcast* bc = &ws->bc;
    volatile RowState* rows = ws->rows;
    const bool row = j < a.nrows;
    const int jj = row ? j : 0;
    const DF two_c = DF{a.two_c_df[0], a.two_c_df[1]};
    const DF ax = a.proj ? df_zero() : sc.tot[kBVals * jj + 0];
    const DF r0s = sc.tot[kBVals * jj + 1], sf = sc.tot[kBVals * jj + 2];
    const DF smin = sc.tot[kBVals * jj + 3], smax = sc.tot[kBVals * jj + 4];
    const float zla = sc.tot[kBVals * jj + 5].hi;
    const float lsat = sc.totmax[3 * jj];
    const float lneg = -sc.totmax[3 * jj + 1];
    const float amax = sc.totmax[3 * jj + 2];
    const bool eq = (a.eq_mask >> jj) & 1;
    const bool finite = isfinite(ax.hi) && isfinite(r0s.hi) && isfinite(sf.hi) && isfinite(smin.hi) &&
                        isfinite(smax.hi);
    const DF b = df_add(DF{a.bconst_df[2 * jj], a.bconst_df[2 * jj + 1]}, ax);
    const DF r0 = df_add(r0s, df_neg(b));
    const bool up = df_pos(r0);
    const bool down = eq && df_pos(df_neg(r0));
    float L, H;
    DF rL, SLs, rH, SHs;
    if (down) {
        // the saturation bounds are only used widened (by 1e-5 and a tiny absolute margin)
        float Lf = fmaf(lneg, 1.00001f, -1e-30f);
        if (!(Lf < 0.0f)) Lf = -FLT_MIN;
        L = Lf;
        rL = df_add(df_add(smax, df_neg(b)), df_neg(df_mul(two_c, DF{L, 0.0f})));
        SLs = two_c;
        H = 0.0f;
        rH = r0;
        SHs = df_add(sf, two_c);
    } else {
        float Hf = fmaf(lsat, 1.00001f, 1e-30f);
        if (!(Hf > 0.0f)) Hf = FLT_MIN;
        L = 0.0f;
        rL = r0;
        SLs = df_add(sf, two_c);
        H = Hf;
        rH = df_add(df_add(smin, df_neg(b)), df_neg(df_mul(two_c, DF{H, 0.0f})));
        SHs = two_c;
    }
    const bool closed = down ? df_pos(df_neg(rL)) : (up && df_pos(rH));
    const bool search = row && finite && (up || down) && !closed;
    const bool need = !ladder || __ballot_sync(kFull, row && !ladder_usable((float)a.lam_prev[jj])) != 0u;
    float p = 0.0f;
    if (need) {  // warp-uniform
        // the row's first Newton quotients and secant offset in one warp-wide division: lane
        // k = 0 of the group divides for the Newton point from L, k = 1 from H, the others
        // the secant
        const DF num = k == 0 ? rL : k == 1 ? rH : df_mul(rL, DF{H - L, 0.0f});
        const DF den = k == 0 ? SLs : k == 1 ? SHs : df_add(rL, df_neg(rH));
        const DF q = df_div(num, den);
        const int g0 = lane & ~7;
        const float NL = (df_add_f(DF{__shfl_sync(kFull, q.hi, g0), __shfl_sync(kFull, q.lo, g0)}, L)).hi;
        const float NH = (df_add_f(DF{__shfl_sync(kFull, q.hi, g0 + 1), __shfl_sync(kFull, q.lo, g0 + 1)}, H)).hi;
        const float sec = (df_add_f(DF{__shfl_sync(kFull, q.hi, g0 + 2), __shfl_sync(kFull, q.lo, g0 + 2)}, L)).hi;
        const float lp = a.lam_prev ? (float)a.lam_prev[jj] : (down ? 1.0f : -1.0f);
        p = next_point_warm_f(lane, L, H, NL, NH, sec, lp);
    }
    if (row && k == 0) {
        ws->info.b[j] = df_to_double(b);
        rows[j].reg = a.two_c;
        if (search) {
            store_row_df(&rows[j], b, L, rL, SLs, H, rH, SHs, df_zero(), 0.0, two_c.hi, 1, 2);
            rows[j].famax = amax;
            rows[j].fzla = zla;
            bc->active[j] = 1;
            bc->cmode[j] = 0;
            bc->brL[j] = L;
            bc->brH[j] = H;
        } else if (closed) {
            const DF lam = df_mul(DF{a.half_c_df[0], a.half_c_df[1]}, df_add(down ? smax : smin, df_neg(b)));
            store_row_df(&rows[j], b, 0.0f, df_zero(), df_zero(), 0.0f, df_zero(), df_zero(), lam, 0.0, two_c.hi, 0, 1);
            publish_lambda_df(bc, j, lam);
        } else {
            store_row_df(&rows[j], b, 0.0f, df_zero(), df_zero(), 0.0f, df_zero(), df_zero(), df_zero(),
                         df_to_double(r0), two_c.hi, 0, 0);
            publish_lambda_df(bc, j, df_zero());
        }
    }
    if (search && need) bc->pts[j][k] = p;
    const unsigned any = __ballot_sync(kFull, search);
    const unsigned bad = __ballot_sync(kFull, row && !finite);
    if (lane == 0) {
        int status = a.proj ? kOk : bc->status;
        if (bad) status = kErrNonfinite;
        bc->status = status;
        bc->any_active = (status == kOk && any) ? 1 : 0;
    }
}

// After phase D: the report.  Lane j < nrows refines row j; lane kMaxRows computes the
// relative change; both divisions are one warp-wide double-float division (FP32 pipes;
// FP64 issues slowly here).
__device__ void update_final(const SegArgs& a, const BlockScratch& sc, SegState* ws, int* sticky,
                             unsigned long long* launches) {
    const int lane = threadIdx.x;
    const int nr = a.nrows;
    volatile DeviceInfo* inf = &ws->info;
    volatile RowState* rows = ws->rows;
    volatile SegBcast* bc = &ws->bc;
    const bool rl = lane < nr;
    const int j = rl ? lane : 0;
    const DF two_c = DF{a.two_c_df[0], a.two_c_df[1]};
    const DF ax = sc.tot[j];
    const DF bj = DF{rows[j].b_hi, rows[j].b_lo};
    DF lam = DF{rows[j].lam_hi, rows[j].lam_lo};
    const DF S = df_add(sc.tot[nr + j], two_c);
    const DF r = df_add(df_add(ax, df_neg(bj)), df_neg(df_mul(two_c, lam)));
    const DF dd = a.proj ? df_zero() : sc.tot[2 * nr];
    const DF nn = a.proj ? DF{1.0f, 0.0f} : sc.tot[2 * nr + 1];
    const bool rcl = lane == kMaxRows;
    const DF q = df_div(rcl ? dd : r, rcl ? nn : S);
    const DF rq = df_sqrt(q);
    const double rcl_v = a.proj ? 0.0 : (nn.hi > 0.0f ? df_to_double(rq) : INFINITY);
    const double rc = __shfl_sync(kFull, rcl_v, kMaxRows);
    // One Newton step per searched row on the accurate residual of this pass.  The
    // search's FP32 trial sums carry rounding noise (well under 1e-6 (|b| + |a^T x|)),
    // which can leave its root outside its last bracket by up to that noise over the
    // slope, on a neighbouring linear piece.  A correction within four bracket widths or
    // that noise scale is taken.  The pass wrote x at the uncorrected lam, and a change dl
    // of lam moves a free x_i by dl a_i: a correction larger than 1e-7 lam, or one that
    // moves some free x_i by more than 1e-7 (max |a_i| over the free set), runs this pass
    // again at the corrected lam, at most eight times.
    const bool eqj = (a.eq_mask >> j) & 1;
    bool again = false;
    if (rl && rows[j].how == 2 && (df_pos(lam) || eqj)) {
        const bool spos = df_pos(S);
        const DF dl = spos ? q : df_zero();
        const float w = rows[j].fH - rows[j].fL;
        const float adl = fabsf(dl.hi);
        // the search may have run on z_hi alone (shares streaming from global memory), whose
        // root is off by up to sum |a z_lo| over the slope: such a correction is taken too
        const bool near = adl <= 4.0f * w ||
                          (spos && adl * S.hi <= 1e-6f * (fabsf(bj.hi) + fabsf(ax.hi)) + 2.0f * rows[j].fzla);
        const DF ln = df_add(lam, dl);
        if (near && (df_pos(ln) || eqj)) {
            lam = ln;
            if ((adl > 1e-7f * fabsf(lam.hi) || adl * sc.totmax[j] > 1e-7f) && rows[j].nrefine < 8) {
                rows[j].nrefine = rows[j].nrefine + 1;
                rows[j].lam_hi = lam.hi;
                rows[j].lam_lo = lam.lo;
                publish_lambda_df(bc, j, lam);
                again = true;
            }
        }
    }
    const unsigned again_m = __ballot_sync(kFull, again);
    if (lane == 0) bc->refine = again_m ? 1 : 0;
    if (again_m) return;
    if (lane < kMaxRows) {
        inf->lambda[lane] = rl ? df_to_double(lam) : 0.0;
        inf->viol[lane] = rl ? df_to_double(df_add(ax, df_neg(bj))) : 0.0;
        inf->b[lane] = rl ? rows[j].b : 0.0;
    }
    const unsigned nconv = __ballot_sync(kFull, rl && rows[j].how == 3);
    const unsigned nfin = __ballot_sync(kFull, rl && !isfinite(ax.hi));
    if (lane != 0) return;
    int status = bc->status;
    int passes = 0;
    double phi = 0.0, vis = 0.0;
    for (int i = 0; i < nr; ++i) {
        passes = max(passes, rows[i].passes + rows[i].nrefine);
        phi = fmax(phi, fabs(rows[i].rlast));
        vis += rows[i].visited;
    }
    // the first row (in row order) that did not converge or is not finite names the status
    if ((nconv | nfin) && status == kOk) status = (nconv >> (__ffs(nconv | nfin) - 1)) & 1u ? kNotConverged : kErrNonfinite;
    if (!a.proj) {
        inf->rel_change = rc;
    } else {
        inf->rel_change = 0.0;
        inf->alpha = 0.0;
        inf->beta = 0.0;
        inf->branch = -1;
        inf->t = -1;
    }
    inf->phi_inf = phi;
    inf->passes = passes;
    inf->visited = vis;
    inf->newton_iters = 0;
    inf->stage = 0;
    inf->status = status;
    if (status != kOk && sticky) atomicCAS(sticky, kOk, status);
    if (launches) *launches += 1ull;
}

// Early exit after a non-finite reduction: report and stop.
__device__ void report_status_only(SegState* ws, int* sticky, unsigned long long* launches, int status) {
    volatile DeviceInfo* inf = &ws->info;
    inf->status = status;
    inf->passes = 0;
    if (sticky) atomicCAS(sticky, kOk, status);
    if (launches) *launches += 1ull;
}

// ----------------------------------------------------------------------- element passes

// Grid engine: the CTAs of one cooperative launch share one problem; phases end in a
// grid-wide all-reduce through global memory after which every CTA runs the scalar
// update on its own copy of the search state in shared memory (dev_common.cuh).  Block 0
// owns the side effects: the sticky status, the launch count and the report, which it
// copies to global memory when the step ends (publish).
struct GridSyncSeg {
    SegWork* ws;
    long long timeout;
    SegState* st;  // this CTA's copy of the search state
    __device__ int rank() const { return blockIdx.x; }
    __device__ int size() const { return gridDim.x; }
    __device__ SegState* state() const { return st; }
    __device__ int* sticky() const { return blockIdx.x == 0 ? &ws->ctrl.status : nullptr; }
    __device__ unsigned long long* launches() const { return blockIdx.x == 0 ? &ws->ctrl.launches : nullptr; }
    template <class F>
    __device__ bool reduce(BlockScratch& sc, int nv, int nm, F&& f) const {
        SegState* s0 = st;
        return grid_allreduce_update(&ws->ctrl, ws->part, sc, nv, nm, timeout, [&](BlockScratch& s) { f(s, s0); });
    }
    __device__ void fetch(SegBcast& bc) const {
        const unsigned* src = reinterpret_cast<const unsigned*>(&st->bc);
        unsigned* d = reinterpret_cast<unsigned*>(&bc);
        for (int i = threadIdx.x; i < (int)(sizeof(SegBcast) / 4); i += blockDim.x) d[i] = src[i];
        __syncthreads();
    }
    // Every thread of every CTA calls this at the end of the step.
    __device__ void publish() const {
        if (blockIdx.x != 0) return;
        __syncthreads();
        const unsigned* src = reinterpret_cast<const unsigned*>(&st->info);
        unsigned* d = reinterpret_cast<unsigned*>(&ws->st.info);
        for (int i = threadIdx.x; i < (int)(sizeof(DeviceInfo) / 4); i += blockDim.x) d[i] = src[i];
    }
};

// Cluster engine: the CTAs of one thread-block cluster share one problem; phases end in a
// reduction through distributed shared memory and hardware cluster barriers, with the
// search state in the first CTA's shared memory.
struct ClusterSyncSeg {
    SegState* st;  // this CTA's copy; the first CTA's is the live one
    GridCtrl* trace;  // phase timeline of a single-problem launch (the handle's), or null
    __device__ int rank() const { return (int)cg::this_cluster().block_rank(); }
    __device__ int size() const { return (int)cg::this_cluster().num_blocks(); }
    __device__ SegState* state() const { return st; }
    __device__ int* sticky() const { return nullptr; }
    __device__ unsigned long long* launches() const { return nullptr; }
    template <class F>
    __device__ bool reduce(BlockScratch& sc, int nv, int nm, F&& f) const {
        SegState* s0 = st;
        GridCtrl* tr = trace;
        cluster_reduce_update(sc, nv, nm, [&](BlockScratch& s) {
            f(s, s0);
            if (tr && threadIdx.x == 0) {
                __syncwarp(1u);
                volatile GridCtrl* vc = tr;
                const int k = vc->ntrace;
                if (k >= 0 && k < 62) {
                    vc->trace[k] = globaltimer_ns();
                    vc->ntrace = k + 1;
                }
            }
        });
        return true;
    }
    __device__ void publish() const {}  // the kernel copies the first CTA's report
    __device__ void fetch(SegBcast& bc) const {
        const SegBcast* src = cg::this_cluster().map_shared_rank(&st->bc, 0);
        const unsigned* sw = reinterpret_cast<const unsigned*>(src);
        unsigned* d = reinterpret_cast<unsigned*>(&bc);
        for (int i = threadIdx.x; i < (int)(sizeof(SegBcast) / 4); i += blockDim.x) d[i] = sw[i];
        __syncthreads();
    }
};

// One PGD-TO step (or projection) on the problem `a`, executed by the CTAs of `sy`.
// Dynamic shared memory of the residency (three arrays of SegArgs::sm_elems floats).
extern __shared__ float4 seg_dyn_sm[];

template <bool B>
struct BoolC {
    static constexpr bool value = B;
};

template <bool VEC, bool CMP, class Sync>
__device__ void seg_body(const SegArgs& a, const Sync& sy, BlockScratch& sc, SegBcast& bc, float* sm) {
    const int nb = sy.size(), blk = sy.rank();
    const float lo = a.lo, hi = a.hi;
    // A block whose share of a row is empty (seg_row_chunk) contributes zeros to that row's
    // sums; the row loops end with a barrier before the grid reduction reads them.
    auto zero_tot = [&](int voff, int nv, int moff, int nm) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) sc.tot[voff + i] = df_zero();
        for (int i = threadIdx.x; i < nm; i += blockDim.x) sc.totmax[moff + i] = 0.0f;
    };

    if (!a.proj) {
        // ------------------------------------------------------------ phase A
        AccSplit<6, 0> acc;
        acc.init();
        float gmax = 0.0f;
        int64_t cb, ce;
        block_chunk(0, a.n, blk, nb, cb, ce);
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
            struct G4 {
                float4 x, xp, g, gp;
            };
            for_chunk_x2<VEC>(
                cb, ce,
                [&](int64_t v) { return G4{LD4L2(a.x, v), LD4(a.x_prev, v), LD4L2(a.g, v), LD4(a.g_prev, v)}; },
                [&](const G4& q) {
                    e(q.x.x, q.xp.x, q.g.x, q.gp.x);
                    e(q.x.y, q.xp.y, q.g.y, q.gp.y);
                    e(q.x.z, q.xp.z, q.g.z, q.gp.z);
                    e(q.x.w, q.xp.w, q.g.w, q.gp.w);
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
            for_chunk_x2<VEC>(
                cb, ce, [&](int64_t v) { return LD4L2(a.g, v); },
                [&](const float4& g) {
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
        if (!sy.reduce(sc, 6, 1, [&](BlockScratch& s, SegState* st) { update_step_scalars(a, s, &st->bc, &st->info); }))
            return;
        sy.fetch(bc);
        if (bc.status != kOk) {
            if (blk == 0 && threadIdx.x == 0) report_status_only(sy.state(), sy.sticky(), sy.launches(), bc.status);
            sy.publish();
            return;
        }
    }

    // ---------------------------------------------------------------- phase B
    // Cache policy: a stream read or written for the last time in the step is evict-first
    // (LD4, __stcs); the trial point z_hi and the coefficients, which the passes read
    // again, keep normal priority.  On a problem larger than L2 this keeps the kernel's
    // code and the round partials resident while hundreds of MB stream past.
    // Residency: when this CTA's share fits the dynamic shared memory, phase B keeps the
    // trial point (z_hi, z_lo) and the coefficients there and phases C and D read them
    // back from it instead of global memory (z is then not written to global memory).
    const bool res = sm != nullptr && a.sm_elems > 0 && seg_res_need(a.seg, a.nrows, blk, nb) <= a.sm_elems;
    // warm start: the first search pass evaluates the ladder around the previous root and
    // shares phase B's reduction (the lean variant; the compaction variant keeps them apart)
    const bool ladder = !CMP && !a.proj && a.lam_prev != nullptr;
    float* const smz = sm;
    float* const sml = sm + a.sm_elems;
    float* const sma = sm + 2 * a.sm_elems;
    {
        const float ch = a.proj ? 0.0f : bc.c_hi, bh = a.proj ? 0.0f : bc.beta_hi;
        const bool first = a.t == 0;
        int roff = 0;
        for (int j = 0; j < a.nrows; ++j) {
            // acc: free-set curvature at 0, sum a * (row-minimising bound), sum a * (row-
            // maximising bound), sum |a z_lo|; the sums that enter b and r(0) are the TwoSum
            // pairs below
            AccSplit<0, 4, 1, 4> acc;
            acc.init();
            float lsat = 0.0f, lnegm = 0.0f, amx = 0.0f;
            const bool eqj = (a.eq_mask >> j) & 1;
            int64_t cb, ce;
            seg_row_chunk(a.seg, a.nrows, j, blk, nb, cb, ce);
            if (ce <= cb) {
                zero_tot(kBVals * j, kBVals, 3 * j, 3);
                continue;
            }
            const int64_t rb = cb & ~int64_t(3);
            const int off = roff;
            roff += seg_res_span(cb, ce);
            // a^T x_t (it enters b) and r(0) + b = a^T clip(z_hi + z_lo) decide whether the row
            // binds: exact products, hi parts summed with TwoSum, everything else in the lo sum
            float axh = 0.0f, axl = 0.0f, r0h = 0.0f, r0l = 0.0f;
            auto e = [&](float z, float zl, float av, float x) {
                const float ph = av * x;
                const DF t = two_sum(axh, ph);
                axh = t.hi;
                axl = __fadd_rn(axl, __fadd_rn(t.lo, fmaf(av, x, -ph)));
                // free when z_hi + z_lo lies in [lo, hi] (z_hi at a bound decides by z_lo's sign)
                const bool fr = (z > lo || (z == lo && zl >= 0.0f)) && (z < hi || (z == hi && zl <= 0.0f));
                const float xc = fr ? z : (z < lo || (z == lo && zl < 0.0f) ? lo : hi);
                const float q = av * xc;
                const DF u = two_sum(r0h, q);
                r0h = u.hi;
                r0l = __fadd_rn(r0l, __fadd_rn(u.lo, fmaf(av, xc, -q) + (fr ? av * zl : 0.0f)));
                acc.f[0] = fr ? fmaf(av, av, acc.f[0]) : acc.f[0];
                acc.f[1] += av > 0.0f ? av * lo : (av < 0.0f ? av * hi : 0.0f);
                acc.f[2] += av > 0.0f ? av * hi : (av < 0.0f ? av * lo : 0.0f);
                acc.f[3] = fmaf(fabsf(av), fabsf(zl), acc.f[3]);
                amx = fmaxf(amx, fabsf(av));
                if (av != 0.0f) {
                    // saturation bounds: only used widened by 1e-5, so a fast division will do
                    const float ra = __fdividef(1.0f, av);
                    lsat = fmaxf(lsat, (av > 0.0f ? z - lo : z - hi) * ra);
                    if (eqj) lnegm = fmaxf(lnegm, -(av > 0.0f ? z - hi : z - lo) * ra);
                }
            };
            if (a.proj) {
                for_chunk<VEC>(
                    cb, ce,
                    [&](int64_t v) {
                        float4 z = LD4L2(a.z_in, v), av = LD4L2(a.A, v);
                        e(z.x, 0.0f, av.x, 0.0f);
                        e(z.y, 0.0f, av.y, 0.0f);
                        e(z.z, 0.0f, av.z, 0.0f);
                        e(z.w, 0.0f, av.w, 0.0f);
                        if (res) {
                            const int q = (off >> 2) + (int)(v - (rb >> 2));
                            reinterpret_cast<float4*>(smz)[q] = z;
                            reinterpret_cast<float4*>(sma)[q] = av;
                        }
                        acc.tick();
                    },
                    [&](int64_t i) {
                        const float z = a.z_in[i], av = a.A[i];
                        e(z, 0.0f, av, 0.0f);
                        if (res) {
                            smz[off + (int)(i - rb)] = z;
                            sma[off + (int)(i - rb)] = av;
                        }
                        acc.tick();
                    });
            } else {
                const float cl = bc.c_lo, bl = bc.beta_lo;
                // d_t = beta d_prev - g and z = x + c d_t in double-float: the FP32 direction is
                // the stored state, (z_hi, z_lo) the trial point the projection sees
                auto st = [&](float x, float g, float dp, float av, float& dout, float& zh, float& zl) {
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
                    e(z.hi, z.lo, av, x);
                };
                struct B4 {
                    int64_t v;
                    float4 x, g, av, dp;
                };
                for_chunk_x2<VEC>(
                    cb, ce,
                    [&](int64_t v) {
                        return B4{v, LD4(a.x, v), LD4(a.g, v), LD4L2(a.A, v),
                                  first ? make_float4(0.f, 0.f, 0.f, 0.f) : LD4(a.d_prev, v)};
                    },
                    [&](const B4& q) {
                        const int64_t v = q.v;
                        const float4 x = q.x, g = q.g, av = q.av, dp = q.dp;
                        float4 d, zh, zl;
                        st(x.x, g.x, dp.x, av.x, d.x, zh.x, zl.x);
                        st(x.y, g.y, dp.y, av.y, d.y, zh.y, zl.y);
                        st(x.z, g.z, dp.z, av.z, d.z, zh.z, zl.z);
                        st(x.w, g.w, dp.w, av.w, d.w, zh.w, zl.w);
                        __stcs(reinterpret_cast<float4*>(a.d_new) + v, d);
                        if (res) {
                            const int q = (off >> 2) + (int)(v - (rb >> 2));
                            reinterpret_cast<float4*>(smz)[q] = zh;
                            reinterpret_cast<float4*>(sml)[q] = zl;
                            reinterpret_cast<float4*>(sma)[q] = av;
                        } else {
                            reinterpret_cast<float4*>(a.z)[v] = zh;
                            __stcs(reinterpret_cast<float4*>(a.zlo) + v, zl);
                        }
                        __stcs(reinterpret_cast<float4*>(a.x_prev) + v, x);
                        __stcs(reinterpret_cast<float4*>(a.g_prev) + v, g);
                        acc.tick();
                    },
                    [&](int64_t i) {
                        const float x = a.x[i], g = a.g[i], av = a.A[i];
                        float d, zh, zl;
                        st(x, g, first ? 0.0f : a.d_prev[i], av, d, zh, zl);
                        a.d_new[i] = d;
                        if (res) {
                            smz[off + (int)(i - rb)] = zh;
                            sml[off + (int)(i - rb)] = zl;
                            sma[off + (int)(i - rb)] = av;
                        } else {
                            a.z[i] = zh;
                            a.zlo[i] = zl;
                        }
                        a.x_prev[i] = x;
                        a.g_prev[i] = g;
                        acc.tick();
                    });
            }
            acc.fold();
            const DF v[kBVals] = {fast_two_sum(axh, axl), fast_two_sum(r0h, r0l), acc.d[0], acc.d[1], acc.d[2],
                                  acc.d[3]};
            float mx[3] = {lsat, lnegm, amx};
            block_reduce<kBVals, 3>(v, mx, sc, kBVals * j, 3 * j);
        }
        __syncthreads();
        if (!ladder) {
            if (!sy.reduce(sc, kBVals * a.nrows, 3 * a.nrows,
                           [&](BlockScratch& s, SegState* st) { update_after_trial(a, s, st); }))
                return;
            sy.fetch(bc);
            if (bc.status != kOk) {
                if (blk == 0 && threadIdx.x == 0) report_status_only(sy.state(), sy.sticky(), sy.launches(), bc.status);
                sy.publish();
                return;
            }
        }
    }

    // ---------------------------------------------------------------- phase C
    // Root-search passes.  Free-set compaction (Sec. 4.2.1): from the second pass on, an
    // element whose state (below lo / free / above hi) is the same at both ends of the
    // bracket the pass's points lie in keeps that state for every later (narrower)
    // bracket, since w = z - lam a is linear in lam.  Its part of r is then a*bound or
    // a z - lam a^2: such elements go into three per-row sums (exact products), and each
    // thread keeps a list of the undecided rest of its share, which the later passes
    // evaluate alone, filtering the list as they go.  The row update adds the decided part
    // back (search_pass_update with CMP).  A margin of a few ulp keeps elements within
    // rounding of a bound undecided.
    if constexpr (CMP) {
        const float* zsrc = a.proj ? a.z_in : a.z;
        const bool has_lo = !a.proj;
        const bool cmp = a.cidx != nullptr;
        const int nthr = blockDim.x, tid = threadIdx.x;
        const int64_t lstride = cmp ? seg_list_cta(a.seg, a.nrows, nb, nthr) : 0;
        while (bc.any_active) {
            int roff = 0;
            for (int j = 0; j < a.nrows; ++j) {
                int64_t cb, ce;
                seg_row_chunk(a.seg, a.nrows, j, blk, nb, cb, ce);
                const int64_t rb = cb & ~int64_t(3);
                const int off = roff;
                roff += seg_res_span(cb, ce);
                if (!bc.active[j]) continue;
                if (ce <= cb) {
                    if (cmp && bc.cmode[j] != 0) a.ccnt[((int64_t)blk * kMaxRows + j) * nthr + tid] = 0;
                    zero_tot((2 * K + 4) * j, 2 * K + 4, 0, 0);
                    continue;
                }
                float p[K];
    #pragma unroll
                for (int k = 0; k < K; ++k) p[k] = bc.pts[j][k];
                const int mode = cmp ? bc.cmode[j] : 0;
                const float bl = bc.brL[j], bu = bc.brH[j];
                int* lst = cmp ? a.cidx + (int64_t)blk * lstride + seg_list_row_off(a.seg, a.nrows, j, nb, nthr)
                               : nullptr;
                int* cntp = cmp ? a.ccnt + ((int64_t)blk * kMaxRows + j) * nthr + tid : nullptr;
                int nkeep = 0;
                // acc.f[0, K): r sums at the points; [K, K + 3): the elements this pass decides
                // (sum a*bound, sum a z, sum a^2; these steer the search only, the final pass
                // recomputes r exactly); [K + 3, 2K + 3): free-set curvature at the points
                AccSplit<K + 3, K, 2, 8> acc;
                acc.init();
                int nvis = 0;  // elements this thread evaluates in this pass
                auto e = [&](float z, float zl, float av) {
                    const float aa = av * av;
    #pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float w = __fadd_rn(fmaf(-p[k], av, z), zl);
                        const float x = clampf(w, lo, hi);  // free exactly when the clip leaves w
                        acc.f[k] = fmaf(av, x, acc.f[k]);
                        acc.f[K + 3 + k] += (x == w) ? aa : 0.0f;
                    }
                };
                // the K points, then (when classifying) the state at both bracket ends
                auto visit = [&](int i, float z, float zl, float av) {
                    e(z, zl, av);
                    ++nvis;
                    if (mode == 0) return;
                    const float wl = __fadd_rn(fmaf(-bl, av, z), zl);
                    const float wu = __fadd_rn(fmaf(-bu, av, z), zl);
                    const float mg = 4e-7f * (fabsf(z) + fabsf(bl * av) + fabsf(bu * av) + (hi - lo));
                    const int sl = wl < lo - mg ? 0 : (wl > hi + mg ? 2 : (wl > lo + mg && wl < hi - mg ? 1 : 3));
                    const int su = wu < lo - mg ? 0 : (wu > hi + mg ? 2 : (wu > lo + mg && wu < hi - mg ? 1 : 3));
                    if (sl == su && sl != 3) {
                        if (sl == 1) {
                            acc.f[K + 1] = fmaf(av, z, fmaf(av, zl, acc.f[K + 1]));
                            acc.f[K + 2] = fmaf(av, av, acc.f[K + 2]);
                        } else {
                            acc.f[K] = fmaf(av, sl == 0 ? lo : hi, acc.f[K]);
                        }
                    } else {
                        lst[nkeep * nthr + tid] = i;
                        ++nkeep;
                    }
                };
                // one element loop per source (shared or global memory), per trial point form
                // (with or without z_lo) and per kind of pass (with or without classification),
                // fixed at compile time: a pass before the lists exist runs the plain loop
                auto run = [&](auto rc, auto lc, auto cc) {
                    constexpr bool R = decltype(rc)::value;
                    constexpr bool HL = decltype(lc)::value;
                    constexpr bool CL = decltype(cc)::value;
                    auto vis = [&](int i, float z, float zl, float av) {
                        if constexpr (CL) {
                            visit(i, z, zl, av);
                        } else {
                            e(z, zl, av);
                            ++nvis;
                        }
                    };
                    if (CL && mode == 2) {
                        const int cnt = *cntp;
                        int q4 = 0;
                        for (int q = 0; q < cnt; ++q) {
                            const int i = lst[q * nthr + tid];
                            if constexpr (R) {
                                const int li = off + (int)(i - rb);
                                vis(i, smz[li], HL ? sml[li] : 0.0f, sma[li]);
                            } else {
                                vis(i, zsrc[i], HL ? a.zlo[i] : 0.0f, a.A[i]);
                            }
                            if (++q4 == 4) {
                                acc.tick();
                                q4 = 0;
                            }
                        }
                        return;
                    }
                    for_chunk<VEC>(
                        cb, ce,
                        [&](int64_t v) {
                            float4 z, zl = make_float4(0.f, 0.f, 0.f, 0.f), av;
                            if constexpr (R) {
                                const int q = (off >> 2) + (int)(v - (rb >> 2));
                                z = reinterpret_cast<const float4*>(smz)[q];
                                if constexpr (HL) zl = reinterpret_cast<const float4*>(sml)[q];
                                av = reinterpret_cast<const float4*>(sma)[q];
                            } else {
                                z = LD4L2(zsrc, v);
                                if constexpr (HL) zl = LD4L2(a.zlo, v);
                                av = LD4L2(a.A, v);
                            }
                            const int i0 = (int)(4 * v);
                            vis(i0, z.x, zl.x, av.x);
                            vis(i0 + 1, z.y, zl.y, av.y);
                            vis(i0 + 2, z.z, zl.z, av.z);
                            vis(i0 + 3, z.w, zl.w, av.w);
                            acc.tick();
                        },
                        [&](int64_t i) {
                            if constexpr (R) {
                                const int q = off + (int)(i - rb);
                                vis((int)i, smz[q], HL ? sml[q] : 0.0f, sma[q]);
                            } else {
                                vis((int)i, zsrc[i], HL ? a.zlo[i] : 0.0f, a.A[i]);
                            }
                            acc.tick();
                        });
                };
                if (mode == 0) {
                    if (res) {
                        if (has_lo) run(BoolC<true>{}, BoolC<true>{}, BoolC<false>{});
                        else run(BoolC<true>{}, BoolC<false>{}, BoolC<false>{});
                    } else {
                        if (has_lo) run(BoolC<false>{}, BoolC<true>{}, BoolC<false>{});
                        else run(BoolC<false>{}, BoolC<false>{}, BoolC<false>{});
                    }
                } else {
                    if (res) {
                        if (has_lo) run(BoolC<true>{}, BoolC<true>{}, BoolC<true>{});
                        else run(BoolC<true>{}, BoolC<false>{}, BoolC<true>{});
                    } else {
                        if (has_lo) run(BoolC<false>{}, BoolC<true>{}, BoolC<true>{});
                        else run(BoolC<false>{}, BoolC<false>{}, BoolC<true>{});
                    }
                }
                if (mode != 0) *cntp = nkeep;
                acc.fold();
                DF v[2 * K + 4];
    #pragma unroll
                for (int k = 0; k < K; ++k) {
                    v[k] = acc.d[k];
                    v[K + k] = acc.d[K + 3 + k];
                }
                v[2 * K] = acc.d[K];
                v[2 * K + 1] = acc.d[K + 1];
                v[2 * K + 2] = acc.d[K + 2];
                v[2 * K + 3] = DF{(float)nvis, 0.0f};
                block_reduce<2 * K + 4, 0>(v, nullptr, sc, (2 * K + 4) * j, 0);
            }
            __syncthreads();
            if (!sy.reduce(sc, (2 * K + 4) * a.nrows, 0, [&](BlockScratch& s, SegState* st) {
                    search_pass_update<SegBcast, true>(s, 0, st->rows, &st->bc, a.nrows, a.tol_lambda, a.max_passes);
                    __syncwarp();
                    // the next pass classifies against the bracket its points will lie in.  The
                    // lists are built once the bracket is within 50% of the root (the share of
                    // elements it leaves undecided follows its width; the search usually ends
                    // two passes later) and used from then on
                    if (threadIdx.x < a.nrows) {
                        const int r = threadIdx.x;
                        volatile SegBcast* vb = &st->bc;
                        if (vb->active[r]) {
                            const float L = st->rows[r].fL, H = st->rows[r].fH;
                            const int cm = vb->cmode[r];
                            const bool narrow = (H - L) <= 0.5f * fmaxf(fabsf(L), fabsf(H));
                            vb->cmode[r] = !a.cidx ? 0 : (cm >= 1 ? 2 : (narrow ? 1 : 0));
                            vb->brL[r] = L;
                            vb->brH[r] = H;
                        }
                    }
                }))
                return;
            sy.fetch(bc);
        }
    } else {
        // without compaction every pass visits every element (compile-time variant: none of
        // the list bookkeeping in the loop, 2K sums per row)
        const float* zsrc = a.proj ? a.z_in : a.z;
        const bool has_lo = !a.proj;
        const int nr = a.nrows;
        bool lad = ladder;  // this pass evaluates the ladder and completes phase B's round
        while (lad || bc.any_active) {
            int roff = 0;
            for (int j = 0; j < nr; ++j) {
                int64_t cb, ce;
                seg_row_chunk(a.seg, a.nrows, j, blk, nb, cb, ce);
                const int64_t rb = cb & ~int64_t(3);
                const int off = roff;
                roff += seg_res_span(cb, ce);
                float p[K];
                if (lad) {
                    const float lp = (float)a.lam_prev[j];
                    if (!ladder_usable(lp)) continue;
#pragma unroll
                    for (int k = 0; k < K; ++k) p[k] = ladder_point(lp, k);
                } else {
                    if (!bc.active[j]) continue;
#pragma unroll
                    for (int k = 0; k < K; ++k) p[k] = bc.pts[j][k];
                }
                if (ce <= cb) {
                    zero_tot((lad ? kBVals * nr : 0) + (2 * K + 3) * j, 2 * K + 3, 0, 0);
                    continue;
                }
                // acc.f[0, K): r sums at the points of the elements whose clip state changes
                // between the lowest and the highest point; [K, K + 3): the other elements as
                // C = sum a bound (clipped at every point), AZ = sum a w_m and AA = sum a^2
                // (free at every point; w_m the value at the reference point); [K + 3, 2K + 3):
                // free-set curvature at the points.  w = z - t a is monotone in t, so the state
                // at both extreme points decides every point between them; once the bracket is
                // narrow almost every element is decided and costs a few operations, not 8 x 7.
                // The decision costs a few operations per element and pays only when the
                // points are close together (few elements change state between them); the
                // span test is the same in every thread, so a pass takes one loop or the other.
                AccSplit<K + 3, K, 2, 8> acc;
                acc.init();
                const float pm = p[kMidPoint];
                const bool narrow = (p[K - 1] - p[0]) <= 4e-3f * fmaxf(fabsf(p[0]), fabsf(p[K - 1]));
                // w = z - t a at point t: with z_lo added when the pass reads it (hl), else the
                // FP32 value alone (adding a zero z_lo would cost an instruction per point)
                auto wat = [&](auto hl, float t, float z, float zl, float av) {
                    const float w = fmaf(-t, av, z);
                    if constexpr (decltype(hl)::value) {
                        return __fadd_rn(w, zl);
                    } else {
                        return w;
                    }
                };
                auto all_points = [&](auto hl, float z, float zl, float av) {
                    const float aa = av * av;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float w = wat(hl, p[k], z, zl, av);
                        const float x = clampf(w, lo, hi);  // free exactly when the clip leaves w
                        acc.f[k] = fmaf(av, x, acc.f[k]);
                        acc.f[K + 3 + k] += (x == w) ? aa : 0.0f;
                    }
                };
                // In a narrow pass the decided part is branch-free and an element whose state
                // changes between the extreme points takes every point under a warp vote, so
                // the every-point code runs only in warps that hold such an element (with a
                // zero coefficient in the lanes that do not, which adds nothing).
                auto e = [&](auto hl, float z, float zl, float av) {
                    if (narrow) {
                        const float w0 = wat(hl, p[0], z, zl, av);
                        const float w1 = wat(hl, p[K - 1], z, zl, av);
                        const float wmn = fminf(w0, w1), wmx = fmaxf(w0, w1);
                        const bool sat = wmx < lo || wmn > hi;
                        const bool fre = wmn >= lo && wmx <= hi;
                        acc.f[K] = fmaf(sat ? av : 0.0f, wmx < lo ? lo : hi, acc.f[K]);
                        const float af = fre ? av : 0.0f;
                        acc.f[K + 1] = fmaf(af, wat(hl, pm, z, zl, av), acc.f[K + 1]);
                        acc.f[K + 2] = fmaf(af, av, acc.f[K + 2]);
                        const bool und = !sat && !fre;
                        if (__any_sync(__activemask(), und)) all_points(hl, z, zl, und ? av : 0.0f);
                        return;
                    }
                    all_points(hl, z, zl, av);
                };
                auto run = [&](auto rc, auto lc) {
                    constexpr bool R = decltype(rc)::value;
                    constexpr bool HL = decltype(lc)::value;
                    struct P4 {
                        float4 z, zl, av;
                    };
                    const BoolC<HL> hl;
                    auto use4 = [&](const P4& q) {
                        e(hl, q.z.x, q.zl.x, q.av.x);
                        e(hl, q.z.y, q.zl.y, q.av.y);
                        e(hl, q.z.z, q.zl.z, q.av.z);
                        e(hl, q.z.w, q.zl.w, q.av.w);
                        acc.tick();
                    };
                    auto use1 = [&](int64_t i) {
                        if constexpr (R) {
                            const int q = off + (int)(i - rb);
                            e(hl, smz[q], HL ? sml[q] : 0.0f, sma[q]);
                        } else {
                            e(hl, zsrc[i], HL ? a.zlo[i] : 0.0f, a.A[i]);
                        }
                        acc.tick();
                    };
                    if constexpr (R) {
                        // shared memory: short latency, one group per iteration
                        for_chunk<VEC>(
                            cb, ce,
                            [&](int64_t v) {
                                const int q = (off >> 2) + (int)(v - (rb >> 2));
                                P4 d{reinterpret_cast<const float4*>(smz)[q], make_float4(0.f, 0.f, 0.f, 0.f),
                                     reinterpret_cast<const float4*>(sma)[q]};
                                if constexpr (HL) d.zl = reinterpret_cast<const float4*>(sml)[q];
                                use4(d);
                            },
                            use1);
                    } else {
                        for_chunk_x2<VEC>(
                            cb, ce,
                            [&](int64_t v) {
                                return P4{LD4L2(zsrc, v), HL ? LD4L2(a.zlo, v) : make_float4(0.f, 0.f, 0.f, 0.f),
                                          LD4L2(a.A, v)};
                            },
                            use4, use1);
                    }
                };
                // a share streaming from global memory reads z_hi and a only (two thirds of the
                // bytes); the final pass reads z_lo and corrects the root (update_final)
                if (res) {
                    if (has_lo) run(BoolC<true>{}, BoolC<true>{});
                    else run(BoolC<true>{}, BoolC<false>{});
                } else {
                    run(BoolC<false>{}, BoolC<false>{});
                }
                acc.fold();
                // two gathers of 16 and 3 values: one of 19 would round up to 32 per lane
                DF v[2 * K], u[3];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    v[k] = acc.d[k];
                    v[K + k] = acc.d[K + 3 + k];
                }
                u[0] = acc.d[K];
                u[1] = acc.d[K + 1];
                u[2] = acc.d[K + 2];
                const int voff = (lad ? kBVals * nr : 0) + (2 * K + 3) * j;
                block_reduce<2 * K, 0>(v, nullptr, sc, voff, 0);
                block_reduce<3, 0>(u, nullptr, sc, voff + 2 * K, 0);
            }
            __syncthreads();
            if (lad) {
                // phase B's update, then the ladder pass's: rows that search and had no
                // usable previous root keep the first points update_after_trial gave them
                if (!sy.reduce(sc, (kBVals + 2 * K + 3) * nr, 3 * nr, [&](BlockScratch& s, SegState* st) {
                        update_after_trial(a, s, st, true);
                        __syncwarp();
                        volatile SegBcast* vb = &st->bc;
                        volatile RowState* vr = st->rows;
                        if (vb->status != kOk) return;
                        const int lane = threadIdx.x, jr = lane >> 3, k = lane & 7;
                        const int jj = jr < nr ? jr : 0;
                        const float lp = (float)a.lam_prev[jj];
                        const bool ev = jr < nr && ladder_usable(lp);
                        const bool act = jr < nr && vr[jj].active;
                        if (act && ev) vb->pts[jr][k] = ladder_point(lp, k);
                        if (ev && k == 0) vr[jr].visited = vr[jr].visited + (double)(a.seg[jr + 1] - a.seg[jr]);
                        const unsigned hb = __ballot_sync(kFull, k == 0 && act && !ev);
                        unsigned held = 0u;
#pragma unroll
                        for (int r = 0; r < kMaxRows; ++r) held |= ((hb >> (8 * r)) & 1u) << r;
                        __syncwarp();
                        search_pass_update<SegBcast, false, true>(s, kBVals * nr, vr, vb, nr, a.tol_lambda, a.max_passes,
                                                                  held);
                    }))
                    return;
                sy.fetch(bc);
                if (bc.status != kOk) {
                    if (blk == 0 && threadIdx.x == 0)
                        report_status_only(sy.state(), sy.sticky(), sy.launches(), bc.status);
                    sy.publish();
                    return;
                }
                lad = false;
                continue;
            }
            if (!sy.reduce(sc, (2 * K + 3) * a.nrows, 0, [&](BlockScratch& s, SegState* st) {
                    // every element of each active row was visited
                    if (threadIdx.x < a.nrows && st->bc.active[threadIdx.x])
                        st->rows[threadIdx.x].visited =
                            st->rows[threadIdx.x].visited + (double)(a.seg[threadIdx.x + 1] - a.seg[threadIdx.x]);
                    __syncwarp();
                    search_pass_update<SegBcast, false, true>(s, 0, st->rows, &st->bc, a.nrows, a.tol_lambda,
                                                              a.max_passes);
                }))
                return;
            sy.fetch(bc);
        }
    }

    // ---------------------------------------------------------------- phase D
    // x = clip(z - lam a) from the double-float difference w = (z_hi + z_lo) - (lam_hi +
    // lam_lo) a, and the residual sum a^T x with exact products accumulated in
    // double-float per element, with the free-set slope beside it: update_final refines
    // lam by a Newton step on that residual and may ask for this pass again at the
    // refined lam (x_t is read from x_prev, so a repeated pass sees the same input).
    for (;;) {
        // nrm: ||x_{t+1} - x_t||^2 and ||x_{t+1}||^2; the per-row sums are scalars of the row
        // loop, kept per row by register selects (a runtime-indexed array would live in
        // local memory)
        AccSplit<2, 0> nrm;
        nrm.init();
        DF rsum[kMaxRows], rslope[kMaxRows];
        float amax_free[kMaxRows] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < kMaxRows; ++q) rsum[q] = rslope[q] = df_zero();
        int roff = 0;
        for (int j = 0; j < a.nrows; ++j) {
            const float lh = bc.lam_hi[j], ll = bc.lam_lo[j];
            int64_t cb, ce;
            seg_row_chunk(a.seg, a.nrows, j, blk, nb, cb, ce);
            const int64_t rb = cb & ~int64_t(3);
            const int off = roff;
            roff += seg_res_span(cb, ce);
            float sh = 0.0f, sl = 0.0f, sfree = 0.0f;  // a^T x as hi (TwoSum) + lo; slope
            float amf = 0.0f;  // max |a| over the free set: how far a change of lam moves x
            DF ra = df_zero(), rs = df_zero();
            int cnt = 0;
            auto e = [&](float x, float zh, float zl, float av) -> float {
                const float p = lh * av;
                const float pe = fmaf(lh, av, -p);
                const DF s = two_sum(zh, -p);
                const DF w = fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(zl, fmaf(ll, av, pe))));
                // free when w_hi + w_lo lies in [lo, hi] (w_hi at a bound decides by w_lo's sign)
                const bool below = w.hi < lo || (w.hi == lo && w.lo < 0.0f);
                const bool above = w.hi > hi || (w.hi == hi && w.lo > 0.0f);
                const bool fr = !below && !above;
                const float xn = fr ? w.hi : (below ? lo : hi);
                const float xl = fr ? w.lo : 0.0f;
                const float ph = av * xn;
                const DF t = two_sum(sh, ph);
                sh = t.hi;
                sl = __fadd_rn(sl, __fadd_rn(t.lo, fmaf(av, xn, -ph) + av * xl));
                sfree = fr ? fmaf(av, av, sfree) : sfree;
                amf = fr ? fmaxf(amf, fabsf(av)) : amf;
                const float dx = xn - x;
                nrm.f[0] = fmaf(dx, dx, nrm.f[0]);
                nrm.f[1] = fmaf(xn, xn, nrm.f[1]);
                return xn;
            };
            auto fold = [&]() {
                ra = df_add(ra, fast_two_sum(sh, sl));
                rs = df_add_f(rs, sfree);
                sh = sl = sfree = 0.0f;
            };
            if (a.proj) {
                for_chunk<VEC>(
                    cb, ce,
                    [&](int64_t v) {
                        float4 z, av;
                        if (res) {
                            const int q = (off >> 2) + (int)(v - (rb >> 2));
                            z = reinterpret_cast<const float4*>(smz)[q];
                            av = reinterpret_cast<const float4*>(sma)[q];
                        } else {
                            z = LD4(a.z_in, v);
                            av = LD4(a.A, v);
                        }
                        float4 o;
                        o.x = e(0.0f, z.x, 0.0f, av.x);
                        o.y = e(0.0f, z.y, 0.0f, av.y);
                        o.z = e(0.0f, z.z, 0.0f, av.z);
                        o.w = e(0.0f, z.w, 0.0f, av.w);
                        __stcs(reinterpret_cast<float4*>(a.x_out) + v, o);
                        if (++cnt == kFoldEvery) {
                            fold();
                            cnt = 0;
                        }
                    },
                    [&](int64_t i) {
                        const int q = off + (int)(i - rb);
                        a.x_out[i] = res ? e(0.0f, smz[q], 0.0f, sma[q]) : e(0.0f, a.z_in[i], 0.0f, a.A[i]);
                    });
            } else {
                struct D4 {
                    int64_t v;
                    float4 x, zh, zl, av;
                };
                for_chunk_x2<VEC>(
                    cb, ce,
                    [&](int64_t v) {
                        D4 q;
                        q.v = v;
                        q.x = LD4(a.x_prev, v);
                        if (res) {
                            const int k = (off >> 2) + (int)(v - (rb >> 2));
                            q.zh = reinterpret_cast<const float4*>(smz)[k];
                            q.zl = reinterpret_cast<const float4*>(sml)[k];
                            q.av = reinterpret_cast<const float4*>(sma)[k];
                        } else {
                            q.zh = LD4(a.z, v);
                            q.zl = LD4(a.zlo, v);
                            q.av = LD4(a.A, v);
                        }
                        return q;
                    },
                    [&](const D4& q) {
                        float4 o;
                        o.x = e(q.x.x, q.zh.x, q.zl.x, q.av.x);
                        o.y = e(q.x.y, q.zh.y, q.zl.y, q.av.y);
                        o.z = e(q.x.z, q.zh.z, q.zl.z, q.av.z);
                        o.w = e(q.x.w, q.zh.w, q.zl.w, q.av.w);
                        __stcs(reinterpret_cast<float4*>(a.x) + q.v, o);
                        if (++cnt == kFoldEvery) {
                            fold();
                            cnt = 0;
                            nrm.fold();
                        }
                    },
                    [&](int64_t i) {
                        const int q = off + (int)(i - rb);
                        a.x[i] = res ? e(a.x_prev[i], smz[q], sml[q], sma[q])
                                     : e(a.x_prev[i], a.z[i], a.zlo[i], a.A[i]);
                    });
            }
            fold();
#pragma unroll
            for (int q = 0; q < kMaxRows; ++q)
                if (q == j) {  // register selects
                    amax_free[q] = amf;
                    rsum[q] = ra;
                    rslope[q] = rs;
                }
        }
        nrm.fold();
        // pack: rows' a^T x, rows' slopes, then the two norms
        const int nr = a.nrows;
        DF packed[2 * kMaxRows + 2];
#pragma unroll
        for (int k = 0; k < 2 * kMaxRows + 2; ++k) {
            DF v = df_zero();
#pragma unroll
            for (int q = 0; q < kMaxRows; ++q) {
                if (q < nr && k == q) v = rsum[q];
                if (q < nr && k == nr + q) v = rslope[q];
            }
            if (k == 2 * nr) v = nrm.d[0];
            if (k == 2 * nr + 1) v = nrm.d[1];
            packed[k] = v;
        }
        const int nv = 2 * nr + (a.proj ? 0 : 2);
        block_reduce<2 * kMaxRows + 2, kMaxRows>(packed, amax_free, sc);
        if (!sy.reduce(sc, nv, nr, [&](BlockScratch& s, SegState* st) { update_final(a, s, st, sy.sticky(), sy.launches()); }))
            return;
        sy.fetch(bc);
        if (!bc.refine) break;
    }
    sy.publish();
}

template <bool VEC, bool CMP>
__global__ void __launch_bounds__(kThreads, 1) seg_kernel(SegArgs a) {
    __shared__ BlockScratch sc;
    __shared__ SegBcast bc;
    __shared__ SegState st;
    SegWork* ws = a.ws;
    if (ld_volatile_i32(&ws->ctrl.abort)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        volatile GridCtrl* vc = &ws->ctrl;
        vc->trace_start = globaltimer_ns();
        vc->ntrace = 0;
    }
    grid_sync_init(&ws->ctrl, sc);
    // test hook: block 0 never arrives, so every other block's first wait runs out its budget
    if (a.fault_inject == 1 && blockIdx.x == 0) return;
    {
        unsigned* w = reinterpret_cast<unsigned*>(&st.info);  // every report field starts defined
        for (int i = threadIdx.x; i < (int)(sizeof(DeviceInfo) / 4); i += blockDim.x) w[i] = 0u;
        __syncthreads();
    }
    GridSyncSeg sy{ws, a.timeout_cycles, &st};
    seg_body<VEC, CMP>(a, sy, sc, bc, a.sm_elems > 0 ? reinterpret_cast<float*>(seg_dyn_sm) : nullptr);
}

// Cluster engine over a list of problems: cluster c takes problems c, c + nclusters, ...
// Problem 0 travels in the launch parameters (a single problem needs no upload), the rest
// in `items`.  Each problem's report goes to its info_out.
template <bool VEC, bool CMP>
__global__ void __launch_bounds__(kClusterThreads, 2) seg_cluster_kernel(SegArgs first, const SegArgs* __restrict__ items,
                                                                  int nitems) {
    __shared__ BlockScratch sc;
    __shared__ SegBcast bc;
    __shared__ SegState st;
    cg::cluster_group cl = cg::this_cluster();
    const int S = (int)cl.num_blocks();
    const int cid = blockIdx.x / S, ncl = gridDim.x / S;
    for (int it = cid; it < nitems; it += ncl) {
        const SegArgs& a = it == 0 ? first : items[it];
        GridCtrl* tr = (nitems == 1 && a.ws) ? &a.ws->ctrl : nullptr;
        if (tr && cl.block_rank() == 0 && threadIdx.x == 0) {
            volatile GridCtrl* vc = tr;
            vc->trace_start = globaltimer_ns();
            vc->ntrace = 0;
        }
        ClusterSyncSeg sy{&st, tr};
        seg_body<VEC, CMP>(a, sy, sc, bc, a.sm_elems > 0 ? reinterpret_cast<float*>(seg_dyn_sm) : nullptr);
        if (cl.block_rank() == 0 && threadIdx.x == 0 && a.info_out) {
            const unsigned* src = reinterpret_cast<const unsigned*>(&st.info);
            unsigned* dst = reinterpret_cast<unsigned*>(a.info_out);
            for (int i = 0; i < (int)(sizeof(DeviceInfo) / 4); ++i) dst[i] = src[i];
        }
        cl.sync();  // shared state is reused by the next problem
    }
}

static size_t res_bytes(int sm_elems) { return (size_t)3 * (size_t)sm_elems * sizeof(float); }

// Each kernel may take its engine's largest residency; set once per kernel.
template <class K>
static void allow_res_smem(K kernel, int cap = kResMaxElems) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_bytes(cap));
}

template <bool VEC, bool CMP>
static cudaError_t launch_seg_t(const SegArgs& a, int blocks, cudaStream_t stream) {
    static bool attr_set = false;
    if (!attr_set) {
        allow_res_smem(seg_kernel<VEC, CMP>);
        attr_set = true;
    }
    void* args[] = {const_cast<SegArgs*>(&a)};
    return cudaLaunchCooperativeKernel((void*)seg_kernel<VEC, CMP>, dim3(blocks), dim3(kThreads), args,
                                       res_bytes(a.sm_elems), stream);
}

// The compaction variant runs when the problem brings its lists (a.cidx).
cudaError_t launch_seg(const SegArgs& a, int blocks, cudaStream_t stream) {
    bool vec = true;
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    vec = al(a.x) && al(a.g) && al(a.A) && al(a.x_prev) && al(a.g_prev) && al(a.d_prev) && al(a.d_new) &&
          al(a.z) && al(a.zlo) && al(a.z_in) && al(a.x_out);
    if (a.cidx) return vec ? launch_seg_t<true, true>(a, blocks, stream) : launch_seg_t<false, true>(a, blocks, stream);
    return vec ? launch_seg_t<true, false>(a, blocks, stream) : launch_seg_t<false, false>(a, blocks, stream);
}

template <bool VEC, bool CMP>
static cudaError_t launch_clusters_t(const SegArgs& first, const SegArgs* items, int nitems, int ncl, int S,
                                     int sm_elems, cudaStream_t stream) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(seg_cluster_kernel<VEC, CMP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        allow_res_smem(seg_cluster_kernel<VEC, CMP>, kResMaxElemsCluster);
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl * S);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = res_bytes(sm_elems);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, seg_cluster_kernel<VEC, CMP>, first, items, nitems);
}

cudaError_t launch_seg_clusters(const SegArgs& first, const SegArgs* items, int nitems, int nclusters, int cluster,
                                bool vec, cudaStream_t stream, int sm_elems, bool cmp) {
    if (nitems < 1 || nclusters < 1 || cluster < 1 || cluster > 16) return cudaErrorInvalidValue;
    if (sm_elems < 0 || sm_elems > kResMaxElemsCluster || (sm_elems & 3)) return cudaErrorInvalidValue;
    if (cmp)
        return vec ? launch_clusters_t<true, true>(first, items, nitems, nclusters, cluster, sm_elems, stream)
                   : launch_clusters_t<false, true>(first, items, nitems, nclusters, cluster, sm_elems, stream);
    return vec ? launch_clusters_t<true, false>(first, items, nitems, nclusters, cluster, sm_elems, stream)
               : launch_clusters_t<false, false>(first, items, nitems, nclusters, cluster, sm_elems, stream);
}

bool seg_args_aligned(const SegArgs& a) {
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return al(a.x) && al(a.g) && al(a.A) && al(a.x_prev) && al(a.g_prev) && al(a.d_prev) && al(a.d_new) &&
           al(a.z) && al(a.zlo) && al(a.z_in) && al(a.x_out);
}

int seg_cluster_shape(int device, int* cluster, int* max_clusters) {
    static int cached_dev = -1, cached_s = 0, cached_n = 0;
    if (cached_dev == device) {
        *cluster = cached_s;
        *max_clusters = cached_n;
        return 0;
    }
    cudaFuncSetAttribute(seg_cluster_kernel<true, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(seg_cluster_kernel<false, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterThreads);
    int s = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&s, seg_cluster_kernel<true, false>, &cfg) != cudaSuccess || s < 1) s = 8;
    if (s > 16) s = 16;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(s);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, seg_cluster_kernel<true, false>, &cfg) != cudaSuccess || nc < 1) nc = 1;
    cached_dev = device;
    cached_s = s;
    cached_n = nc;
    *cluster = s;
    *max_clusters = nc;
    return 0;
}

int max_blocks_seg(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    // co-resident blocks with the largest residency (a cooperative launch needs them all)
    // every variant must fit the same grid (the cooperative launch needs all blocks resident)
    per = 1 << 30;
    const void* ks[4] = {(const void*)seg_kernel<true, false>, (const void*)seg_kernel<false, false>,
                         (const void*)seg_kernel<true, true>, (const void*)seg_kernel<false, true>};
    for (const void* k : ks) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_bytes(kResMaxElems));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, kThreads, res_bytes(kResMaxElems));
        per = v < per ? v : per;
    }
    if (per < 1) per = 1;
    int nb = sms * per;
    return nb > kMaxBlocks ? kMaxBlocks : nb;
}

}  // namespace pgdto

// ------------------------------------------------------------------ allocation-free projection
//
// pgdto_project_noalloc serves callers that cannot allocate device memory: processes whose
// device memory is handed out by another allocator or fixed at start-up (a cudaMalloc there
// fails or fragments the pool), and loops that must never wait on the driver's allocator.
// It runs the projection kernel
// above with its workspace in the file-scope array below instead of a handle's allocation.
// Every GPU that loads this library holds the array until the process exits.

#include <mutex>

#include "../../include/pgdto.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(pgdto::SegWork)];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices];
// tests only (pgdto_noalloc_set_test_fault): block 0 leaves before the first grid reduction
// and every wait has this budget, so the other blocks' waits run out
int g_noalloc_fault_inject = 0;
int g_noalloc_timeout_ms = 0;

// Device address of the array on `device`, looked up once per device with that device
// current.  Host code only ever sees the array through this address: the symbol name
// itself is a host-side stand-in, not a device pointer.
cudaError_t noalloc_workspace(int device, void** out) {
    if (device < 0 || device >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" pgdto_status pgdto_project_noalloc(int64_t n, int m, const int64_t* seg_offsets, float lo, float hi,
                                              double C, const float* z, const float* A, const double* b,
                                              float* x_out, double* lambda_out, pgdto_info* info,
                                              void* cuda_stream) {
    using namespace pgdto;
    if (n < 1 || m < 1 || m > kMaxRows || !z || !A || !b || !x_out) return PGDTO_ERR_ARG;
    if (m > 1 && !seg_offsets) return PGDTO_ERR_ARG;
    if (!(isfinite(lo) && isfinite(hi) && lo < hi) || !(C > 0.0 && isfinite(C))) return PGDTO_ERR_ARG;
    SegArgs a;
    memset(&a, 0, sizeof(a));
    a.seg[0] = 0;
    a.seg[m] = n;
    if (seg_offsets) {
        if (seg_offsets[0] != 0 || seg_offsets[m] != n) return PGDTO_ERR_ARG;
        for (int j = 0; j < m; ++j) {
            if (seg_offsets[j + 1] <= seg_offsets[j]) return PGDTO_ERR_ARG;
            a.seg[j] = seg_offsets[j];
        }
    }
    for (int j = 0; j < m; ++j) {
        if (!isfinite(b[j])) return PGDTO_ERR_NONFINITE;
        a.bconst[j] = b[j];
        split_to_floats(b[j], a.bconst_df + 2 * j);
    }
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PGDTO_ERR_CUDA;
    void* ws = nullptr;
    if (noalloc_workspace(device, &ws) != cudaSuccess) return PGDTO_ERR_CUDA;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    pgdto_params p;
    pgdto_params_default(&p);
    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
    if (clock_khz <= 0) clock_khz = 2000000;
    a.n = n;
    a.nrows = m;
    a.t = 0;
    a.proj = 1;
    a.lo = lo;
    a.hi = hi;
    a.A = A;
    a.z_in = z;
    a.x_out = x_out;
    a.C = C;
    a.two_c = 2.0 / C;
    split_to_floats(a.two_c, a.two_c_df);
    split_to_floats(0.5 * C, a.half_c_df);
    a.tol_lambda = p.tol_lambda;
    a.max_passes = p.max_passes;
    int timeout_ms = p.barrier_timeout_ms;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        a.fault_inject = g_noalloc_fault_inject;
        if (g_noalloc_timeout_ms > 0) timeout_ms = g_noalloc_timeout_ms;
    }
    a.timeout_cycles = (long long)clock_khz * (long long)timeout_ms;
    a.ws = (SegWork*)ws;
    DeviceInfo* report = seg_work_info((SegWork*)ws);
    // The barrier counters, the sticky status and the abort flag must start at zero.  The
    // report is filled with 0xff bytes (status -1, NaN values): a kernel whose blocks gave
    // up waiting never publishes it, and what the last call left there must not read as
    // this call's result.  The rest of the array is rewritten before it is read.
    if (cudaMemsetAsync(ws, 0, sizeof(GridCtrl), stream) != cudaSuccess) return PGDTO_ERR_CUDA;
    if (cudaMemsetAsync(report, 0xff, sizeof(DeviceInfo), stream) != cudaSuccess) return PGDTO_ERR_CUDA;
    if (launch_seg(a, max_blocks_seg(device), stream) != cudaSuccess) return PGDTO_ERR_CUDA;
    if (!info && !lambda_out) return PGDTO_OK;
    DeviceInfo di;
    int ctrl[4];  // GridCtrl: count, pad, sticky status, abort flag
    if (cudaMemcpyAsync(&di, report, sizeof(di), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaMemcpyAsync(ctrl, ws, sizeof(ctrl), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return PGDTO_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return PGDTO_ERR_CUDA;
    int status = di.status;
    if (ctrl[3]) status = ctrl[2] ? ctrl[2] : PGDTO_ERR_TIMEOUT;  // a wait was abandoned
    else if (ctrl[2] && status == PGDTO_OK) status = ctrl[2];
    else if (status < PGDTO_OK || status > PGDTO_ERR_UNSUPPORTED) status = PGDTO_ERR_TIMEOUT;  // never published
    if (info) {
        memcpy(info, &di, sizeof(di));
        info->status = status;
    }
    if (lambda_out)
        for (int j = 0; j < m; ++j) lambda_out[j] = di.lambda[j];
    return (pgdto_status)status;
}

extern "C" pgdto_status pgdto_noalloc_set_test_fault(int fault_inject, int timeout_ms) {
    if ((fault_inject != 0 && fault_inject != 1) || timeout_ms < 0) return PGDTO_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    g_noalloc_fault_inject = fault_inject;
    g_noalloc_timeout_ms = timeout_ms;
    return PGDTO_OK;
}
