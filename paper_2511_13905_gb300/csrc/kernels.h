// kernels.h -- host-visible kernel argument blocks and launch entry points (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pgdto {

constexpr int kMaxRows = 4;

// Report of a step or projection (written by block 0 at the end); same layout as pgdto_info.
struct DeviceInfo {
    double alpha, beta;
    double lambda[kMaxRows], b[kMaxRows], viol[kMaxRows];
    double rel_change, phi_inf;
    int passes, newton_iters, stage, branch, status, t;
    double visited;
};

struct SegWork;      // single / independent rows workspace (seg_kernels.cu)
struct CoupledWork;  // coupled rows workspace (coupled_kernels.cu)

// Arguments of the fused step / projection kernel for single and independent rows.
struct SegArgs {
    int64_t n;
    int nrows;
    int t;
    int proj;            // 1: projection only (z_in, b given), 0: full step
    int force_fallback;  // Alg. 3 fallback rule decided on the host (t == 0 or late violation)
    int64_t seg[kMaxRows + 1];
    float lo, hi;
    float* x;            // step: rho_t in, rho_{t+1} out
    const float* g;      // grad f(rho_t)
    const float* A;      // one coefficient per variable
    float* x_prev;       // state, overwritten with rho_t
    float* g_prev;       // state, overwritten with grad f(rho_t)
    const float* d_prev; // state d_{t-1}
    float* d_new;        // d_t (the other buffer of the pair)
    float* z;            // trial point scratch, rounded to FP32 (z_hi)
    float* zlo;          // rounding residual of the trial point: z = z_hi + z_lo exactly enough
    const float* z_in;   // projection input
    float* x_out;        // projection output
    double bconst[kMaxRows];  // step: G_j - g_j(x_t); projection: b_j
    double C, alpha_max, alpha_fb, eps_alpha, omega, tol_lambda;
    double two_c;         // 2 / C, the slope of the regulariser term (computed by the host)
    float step_df[8];     // alpha_max, alpha_fb, eps_alpha, omega as (hi, lo) float pairs
    float bconst_df[2 * kMaxRows];  // bconst as (hi, lo) float pairs
    float two_c_df[2], half_c_df[2];  // 2 / C and C / 2 as (hi, lo) float pairs
    int max_passes;
    int fault_inject;
    long long timeout_cycles;
    SegWork* ws;          // grid engine workspace
    DeviceInfo* info_out; // cluster engine: where this problem's report goes
    int sm_elems;         // shared-memory residency: floats per array (z_hi, z_lo, a); 0 = off
    const double* lam_prev;  // warm start: the previous step's lam per row (device), or null
    int eq_mask;          // bit j: row j is an equality (always active, lam_j of either sign)
    int* cidx;            // free-set compaction: per-thread lists of undecided elements, or null
    int* ccnt;            // their lengths, per CTA, row and thread
};

// Work split of a problem over nb blocks.  seg_chunk(s, e, blk, nb) is block blk's
// contiguous share of [s, e), a multiple of four long (the last one shorter or empty).
__host__ __device__ inline void seg_chunk(int64_t s, int64_t e, int blk, int nb, int64_t& cb, int64_t& ce) {
    int64_t len = e - s;
    int64_t per = (len + nb - 1) / nb;
    per = (per + 3) & ~int64_t(3);
    if (per < 4) per = 4;
    cb = s + per * blk;
    ce = cb + per;
    if (cb > e) cb = e;
    if (ce > e) ce = e;
}

// Block blk's share of row j: the block owns the chunk seg_chunk(0, n) of the whole array
// and takes the part of it that lies in the row's segment [seg[j], seg[j + 1]).  With
// several rows most of a block's shares are empty: a block's passes run over one or two
// rows' elements in long loops rather than over a short piece of every row.
__host__ __device__ inline void seg_row_chunk(const int64_t* seg, int nrows, int j, int blk, int nb, int64_t& cb,
                                              int64_t& ce) {
    int64_t gb, ge;
    seg_chunk(seg[0], seg[nrows], blk, nb, gb, ge);
    cb = gb > seg[j] ? gb : seg[j];
    ce = ge < seg[j + 1] ? ge : seg[j + 1];
    if (ce < cb) ce = cb;
}

// Free-set compaction lists.  Every thread keeps the elements of its own share that a
// root search has not yet decided, entry q of thread t of a row at q * nthr + t (coalesced
// when all threads read entry q), so appending needs no scan and the order is fixed.  A
// thread visits at most seg_list_cap elements of a share in one sweep (float4 groups with
// stride nthr, plus one element of the unaligned head and one of the tail).  Every row of
// every block gets room for the longest block chunk.
__host__ __device__ inline int seg_list_cap(int64_t len, int nthr) {
    const int64_t ng = len / 4 + 1;
    return (int)(4 * ((ng + nthr - 1) / nthr) + 2);
}

__host__ __device__ inline int64_t seg_list_row_off(const int64_t* seg, int nrows, int j, int nb, int nthr) {
    int64_t gb, ge;
    seg_chunk(seg[0], seg[nrows], 0, nb, gb, ge);
    const int64_t per = ge - gb;
    return (int64_t)j * nthr * seg_list_cap(per < 4 ? 4 : per, nthr);
}

// Ints of one CTA's lists (every row).
__host__ __device__ inline int64_t seg_list_cta(const int64_t* seg, int nrows, int nb, int nthr) {
    return seg_list_row_off(seg, nrows, nrows, nb, nthr);
}

// Shared-memory residency of a CTA's share of a problem.  The CTA's share of row j is
// [cb_j, ce_j) (seg_row_chunk); a non-empty one is kept from base_j = cb_j rounded down to
// a multiple of four, at a float4-aligned offset, rows one after another.  seg_res_need
// is the number of floats per array the CTA needs; the host sizes the launch's dynamic
// shared memory with the same function the device uses to decide.
__host__ __device__ inline int seg_res_span(int64_t cb, int64_t ce) {
    if (ce <= cb) return 0;
    const int64_t b4 = cb & ~int64_t(3);
    return (int)(((ce - b4) + 3) & ~int64_t(3));
}

__host__ __device__ inline int seg_res_need(const int64_t* seg, int nrows, int blk, int nb) {
    int tot = 0;
    for (int j = 0; j < nrows; ++j) {
        int64_t cb, ce;
        seg_row_chunk(seg, nrows, j, blk, nb, cb, ce);
        tot += seg_res_span(cb, ce);
    }
    return tot;
}

// Largest need over the CTAs of a problem split over nb blocks.
inline int seg_res_need_max(const int64_t* seg, int nrows, int nb) {
    int mx = 0;
    for (int b = 0; b < nb; ++b) {
        const int v = seg_res_need(seg, nrows, b, nb);
        mx = v > mx ? v : mx;
    }
    return mx;
}

// Residency capacity per array (floats): three arrays fit next to the static scratch in
// the 227 KB a CTA may hold.
constexpr int kResMaxElems = 16384 + 32;
// The same for the cluster engine, whose two CTAs per SM share the SM's 228 KB.
constexpr int kResMaxElemsCluster = 8192 + 32;

// Arguments of the coupled-rows (Alg. 2) step / projection kernel.
struct CoupledArgs {
    int64_t n;
    int m;
    int t;
    int proj;
    int force_fallback;
    float lo, hi;
    float* x;
    const float* g;
    const float* A;      // m rows of n floats
    float* x_prev;
    float* g_prev;
    const float* d_prev;
    float* d_new;
    float* z;
    float* zlo;
    const float* z_in;
    float* x_out;
    double bconst[kMaxRows];
    double C, alpha_max, alpha_fb, eps_alpha, omega, tol_lambda, tol_N, c1;
    double two_c;         // 2 / C (computed by the host)
    float two_c_df[2];    // 2 / C as a (hi, lo) float pair
    float step_df[8];     // alpha_max, alpha_fb, eps_alpha, omega as (hi, lo) float pairs
    int max_passes, maxiter_newton;
    int fault_inject;
    long long timeout_cycles;
    CoupledWork* ws;
    int eq_mask;          // bit j: row j is an equality (always active, lam_j of either sign)
    const double* lam_prev;  // warm start: the previous step's lam (device), or null
    int stage1;              // cold start: 1 = Alg. 2's stage 1 first, 0 = Newton from lam = 0
};

// A double as an unevaluated sum hi + lo of two floats (host side).
inline void split_to_floats(double v, float* out) {
    out[0] = (float)v;
    out[1] = (float)(v - (double)out[0]);
}

// Workspace management (sizes in bytes, device-resident, zero-initialised by the host).
size_t seg_work_bytes();
size_t coupled_work_bytes();
DeviceInfo* seg_work_info(SegWork* ws);
DeviceInfo* coupled_work_info(CoupledWork* ws);
size_t seg_work_ctrl_bytes();       // leading GridCtrl block to clear after an error
size_t coupled_work_ctrl_bytes();

// Launch helpers: cooperative launch on `stream` with `blocks` CTAs of kThreads threads
// (dynamic shared memory for a.sm_elems floats per residency array).
cudaError_t launch_seg(const SegArgs& a, int blocks, cudaStream_t stream);
// Cluster engine: `items` (device array of `nitems` problems) on `nclusters` clusters of
// `cluster` CTAs each.  vec: every pointer of every item is 16-byte aligned.  sm_elems:
// residency floats per array, at least every item's sm_elems (a multiple of 4).  cmp: some
// item brings compaction lists (the compaction variant of the kernel runs).
cudaError_t launch_seg_clusters(const SegArgs& first, const SegArgs* items, int nitems, int nclusters, int cluster,
                                bool vec, cudaStream_t stream, int sm_elems, bool cmp);
bool seg_args_aligned(const SegArgs& a);
// Largest cluster size (<= 16) the cluster engine can use, and how many such clusters fit.
int seg_cluster_shape(int device, int* cluster, int* max_clusters);
cudaError_t launch_coupled(const CoupledArgs& a, int blocks, cudaStream_t stream);
// Largest co-resident grid for each kernel on the current device.
int max_blocks_seg(int device);
int max_blocks_coupled(int device);

}  // namespace pgdto
