// api.cu -- the C ABI of include/pgdto.h: argument checks, handle and workspace
// ownership, state rotation, launches on the caller's stream, and the report read-back.
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgdto.h"
#include "dev_common.cuh"
#include "handle_internal.h"
#include "kernels.h"

using namespace pgdto;

struct pgdto_handle {
    int64_t n;
    int m;
    pgdto_mode mode;
    int64_t seg[kMaxRows + 1];
    float lo, hi;
    pgdto_params p;
    cudaStream_t stream;
    int device;
    int blocks;               // cooperative grid size
    long long timeout_cycles;
    int t;                    // iteration index of the next step
    // device buffers owned by the handle
    float* x_prev;
    float* g_prev;
    float* d[2];              // d_{t-1} in d[cur], d_t written to d[1 - cur]
    int cur;
    float* z;
    float* zlo;
    void* work;               // SegWork or CoupledWork
    size_t work_bytes;
    size_t ctrl_bytes;
    DeviceInfo* dev_info;
    // host-buffer entry: device staging for x, grad f and A
    float* hx;
    float* hg;
    float* hA;
    int64_t a_len;            // floats in A for this mode
    int64_t launches;
    int last_was_project;
    int warm;                 // the last report is a step's: its lam seeds the next step's search
    int engine;               // 1 grid, 2 cluster
    int cl_size, cl_max;      // this problem's cluster size; clusters co-resident at the largest size
    int res_grid, res_cluster;  // shared-memory residency floats per array on each engine (0 = off)
    SegArgs* items;           // device list for the batched entries (grown on demand)
    SegArgs* items_host;      // pinned staging of that list
    cudaEvent_t items_ev;     // the last upload of items_host (it is rewritten only after)
    int items_cap;
    cudaStream_t aux[4];      // batched launches: one stream per further cluster size
    int* cidx;                // free-set compaction lists (both engines' layouts fit), or null
    int* ccnt;
    cudaEvent_t fork_ev, join_ev[4];
};

static const int64_t kClusterElemsDefault = 8192;

// Cluster-engine block shares chosen by pgdto_autotune_batch, per device and per
// power-of-two bucket of n (bucket b holds 2^(b-1) < n <= 2^b); 0 = not tuned.  Handles
// created with params.cluster_elems = 0 take the entry of their device and bucket.
static std::mutex g_tune_mu;
static int g_tuned[64][64];

static int n_bucket(int64_t n) {
    int b = 0;
    while (b < 63 && (int64_t(1) << b) < n) ++b;
    return b;
}

int pgdto_tuned_cluster_elems(int device, int64_t n) {
    if (device < 0 || device >= 64 || n < 1) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned[device][n_bucket(n)];
}

void pgdto_set_tuned_cluster_elems(int device, int64_t n, int elems) {
    if (device < 0 || device >= 64 || n < 1 || elems < 0) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[device][n_bucket(n)] = elems;
}

extern "C" void pgdto_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    memset(g_tuned, 0, sizeof(g_tuned));
}

// Residency floats per array for a problem split over nb blocks (0 when a block's share
// does not fit the shared memory).
static int res_elems(const int64_t* seg, int m, int nb, int cap) {
    const int need = seg_res_need_max(seg, m, nb);
    return need <= cap ? ((need + 3) & ~3) : 0;
}

// Blocks of a problem's cluster: ceil(n / per_cta) rounded up to a power of two, at most
// the device's largest cluster.  A function of n alone, so a problem reduces in the same
// order alone and in any batch.
static int cluster_size_for(int64_t n, int64_t per_cta, int s_max) {
    const int64_t want = (n + per_cta - 1) / per_cta;
    int s = 1;
    while (s < want && s * 2 <= s_max) s *= 2;
    return s;
}

// Problems up to this many variables run on one thread-block cluster by default: their
// steps are bound by synchronisation latency, which the cluster barriers cut, while
// larger ones need every SM's share of HBM bandwidth.
static const int64_t kClusterMaxN = int64_t(1) << 17;

static pgdto_status cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return PGDTO_ERR_OOM;
    return PGDTO_ERR_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

extern "C" pgdto_status pgdto_params_default(pgdto_params* p) {
    if (!p) return PGDTO_ERR_ARG;
    p->C = 1e12;
    p->alpha_max = 1e2;
    p->alpha_fallback = 0.2;
    p->tol_B = 1e-8;
    p->tol_N = 1e-6;
    p->omega = 1.0;
    p->eps_alpha = 1e-6;
    p->c1 = 1e-4;
    p->c2 = 0.9;
    p->tol_lambda = 1e-10;
    p->t_warmup = 50;
    p->maxiter_newton = 50;
    p->max_passes = 64;
    p->barrier_timeout_ms = 2000;
    p->mode = PGDTO_AUTO;
    p->fault_inject = 0;
    p->engine = 0;
    p->cluster_elems = 0;
    p->eq_mask = 0;
    p->compaction = 0;
    p->stage1 = 0;
    return PGDTO_OK;
}

extern "C" const char* pgdto_version(void) { return "pgdto-gb300 0.1 sm_103a"; }

static void free_handle(pgdto_handle* h) {
    if (!h) return;
    cudaFree(h->x_prev);
    cudaFree(h->g_prev);
    cudaFree(h->d[0]);
    cudaFree(h->d[1]);
    cudaFree(h->z);
    cudaFree(h->zlo);
    cudaFree(h->work);
    cudaFree(h->hx);
    cudaFree(h->hg);
    cudaFree(h->hA);
    cudaFree(h->items);
    cudaFree(h->cidx);
    cudaFree(h->ccnt);
    cudaFreeHost(h->items_host);
    if (h->items_ev) cudaEventDestroy(h->items_ev);
    for (int g = 0; g < 4; ++g) {
        if (h->aux[g]) cudaStreamDestroy(h->aux[g]);
        if (h->join_ev[g]) cudaEventDestroy(h->join_ev[g]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    delete h;
}

static bool params_ok(const pgdto_params& p) {
    return p.C > 0 && isfinite(p.C) && p.alpha_max > 0 && p.alpha_fallback > 0 && p.tol_N >= 0 && p.omega > 0 &&
           p.eps_alpha >= 0 && p.tol_lambda > 0 && p.tol_lambda < 1e-2 && p.t_warmup >= 0 &&
           p.maxiter_newton >= 1 && p.max_passes >= 1 && p.max_passes <= 100000 && p.barrier_timeout_ms >= 1 &&
           (p.fault_inject == 0 || p.fault_inject == 1) && p.engine >= 0 && p.engine <= 2 && p.cluster_elems >= 0 &&
           p.eq_mask >= 0 && p.eq_mask < 16 && (p.compaction == 0 || p.compaction == 1) &&
           (p.stage1 == 0 || p.stage1 == 1);
}

extern "C" pgdto_status pgdto_create(pgdto_handle** out, int64_t n, int m, const int64_t* seg_offsets, float lo,
                                     float hi, const pgdto_params* params, void* cuda_stream) {
    if (!out) return PGDTO_ERR_ARG;
    *out = nullptr;
    if (n < 1 || m < 1 || m > kMaxRows) return PGDTO_ERR_ARG;
    if (!(isfinite(lo) && isfinite(hi) && lo < hi)) return PGDTO_ERR_ARG;
    pgdto_params p;
    if (params) {
        p = *params;
    } else {
        pgdto_params_default(&p);
    }
    if (!params_ok(p)) return PGDTO_ERR_ARG;
    if (p.eq_mask >> m) return PGDTO_ERR_ARG;  // equality flags only for existing rows
    pgdto_mode mode = p.mode;
    if (mode == PGDTO_AUTO) mode = (m == 1) ? PGDTO_SINGLE : (seg_offsets ? PGDTO_INDEPENDENT : PGDTO_COUPLED);
    if (mode == PGDTO_SINGLE && m != 1) return PGDTO_ERR_ARG;
    if (mode == PGDTO_INDEPENDENT && !seg_offsets) return PGDTO_ERR_ARG;
    if (mode == PGDTO_COUPLED && seg_offsets) return PGDTO_ERR_ARG;
    pgdto_handle* h = new pgdto_handle();
    memset(h, 0, sizeof(*h));
    h->n = n;
    h->m = m;
    h->mode = mode;
    h->lo = lo;
    h->hi = hi;
    h->p = p;
    h->stream = (cudaStream_t)cuda_stream;
    if (mode == PGDTO_INDEPENDENT) {
        if (seg_offsets[0] != 0 || seg_offsets[m] != n) {
            delete h;
            return PGDTO_ERR_ARG;
        }
        for (int j = 0; j < m; ++j)
            if (seg_offsets[j + 1] <= seg_offsets[j]) {
                delete h;
                return PGDTO_ERR_ARG;
            }
        for (int j = 0; j <= m; ++j) h->seg[j] = seg_offsets[j];
        h->a_len = n;
    } else if (mode == PGDTO_SINGLE) {
        h->seg[0] = 0;
        h->seg[1] = n;
        h->a_len = n;
    } else {
        h->a_len = n * (int64_t)m;
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e);
    }
    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, h->device);
    if (clock_khz <= 0) clock_khz = 2000000;
    h->timeout_cycles = (long long)clock_khz * (long long)p.barrier_timeout_ms;
    if (mode == PGDTO_COUPLED) {
        h->blocks = max_blocks_coupled(h->device);
        h->work_bytes = coupled_work_bytes();
        h->ctrl_bytes = coupled_work_ctrl_bytes();
    } else {
        h->blocks = max_blocks_seg(h->device);
        h->work_bytes = seg_work_bytes();
        h->ctrl_bytes = seg_work_ctrl_bytes();
    }
    if (h->blocks < 1) {
        delete h;
        return PGDTO_ERR_UNSUPPORTED;
    }
    h->engine = 1;
    if (mode != PGDTO_COUPLED) {
        int s_max = 0;
        seg_cluster_shape(h->device, &s_max, &h->cl_max);
        int64_t share = p.cluster_elems;
        if (share == 0) share = pgdto_tuned_cluster_elems(h->device, n);
        if (share == 0) share = kClusterElemsDefault;
        h->cl_size = cluster_size_for(n, share, s_max);
        h->res_grid = res_elems(h->seg, m, h->blocks, kResMaxElems);
        h->res_cluster = res_elems(h->seg, m, h->cl_size, kResMaxElemsCluster);
        if (p.engine == 2 || (p.engine == 0 && n <= kClusterMaxN)) h->engine = 2;
    } else if (p.engine == 2) {
        delete h;
        return PGDTO_ERR_UNSUPPORTED;
    }
    const size_t nb = (size_t)n * sizeof(float);
    if ((e = cudaMalloc(&h->x_prev, nb)) != cudaSuccess || (e = cudaMalloc(&h->g_prev, nb)) != cudaSuccess ||
        (e = cudaMalloc(&h->d[0], nb)) != cudaSuccess || (e = cudaMalloc(&h->d[1], nb)) != cudaSuccess ||
        (e = cudaMalloc(&h->z, nb)) != cudaSuccess || (e = cudaMalloc(&h->zlo, nb)) != cudaSuccess ||
        (e = cudaMalloc(&h->work, h->work_bytes)) != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e);
    }
    if (mode != PGDTO_COUPLED && p.compaction && n < (int64_t)0x7fffffff) {
        // compaction lists (32-bit element indices): room for the grid and the cluster layout
        const int64_t lg = (int64_t)h->blocks * seg_list_cta(h->seg, m, h->blocks, kThreads);
        const int64_t lc = (int64_t)h->cl_size * seg_list_cta(h->seg, m, h->cl_size, kClusterThreads);
        const int nbm = h->blocks > h->cl_size ? h->blocks : h->cl_size;
        if ((e = cudaMalloc(&h->cidx, (size_t)(lg > lc ? lg : lc) * sizeof(int))) != cudaSuccess ||
            (e = cudaMalloc(&h->ccnt, (size_t)nbm * kMaxRows * kThreads * sizeof(int))) != cudaSuccess) {
            free_handle(h);
            return cuda_fail(e);
        }
    }
    h->dev_info = mode == PGDTO_COUPLED ? coupled_work_info((CoupledWork*)h->work) : seg_work_info((SegWork*)h->work);
    if ((e = cudaMemsetAsync(h->work, 0, h->work_bytes, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->x_prev, 0, nb, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->g_prev, 0, nb, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->d[0], 0, nb, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->d[1], 0, nb, h->stream)) != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e);
    }
    *out = h;
    return PGDTO_OK;
}

extern "C" void pgdto_destroy(pgdto_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_handle(h);
}

extern "C" pgdto_status pgdto_set_stream(pgdto_handle* h, void* s) {
    if (!h) return PGDTO_ERR_ARG;
    h->stream = (cudaStream_t)s;
    return PGDTO_OK;
}

extern "C" int64_t pgdto_kernel_launches(const pgdto_handle* h) { return h ? h->launches : -1; }

int pgdto_handle_whole_gpu(const pgdto_handle* h) { return h && h->engine == 1 ? 1 : 0; }

extern "C" pgdto_status pgdto_set_state(pgdto_handle* h, const float* x_prev, const float* g_prev,
                                        const float* d_prev, int t) {
    if (!h || t < 0) return PGDTO_ERR_ARG;
    const size_t nb = (size_t)h->n * sizeof(float);
    float* dcur = h->d[h->cur];
    if (x_prev) CK(cudaMemcpyAsync(h->x_prev, x_prev, nb, cudaMemcpyDeviceToDevice, h->stream));
    else CK(cudaMemsetAsync(h->x_prev, 0, nb, h->stream));
    if (g_prev) CK(cudaMemcpyAsync(h->g_prev, g_prev, nb, cudaMemcpyDeviceToDevice, h->stream));
    else CK(cudaMemsetAsync(h->g_prev, 0, nb, h->stream));
    if (d_prev) CK(cudaMemcpyAsync(dcur, d_prev, nb, cudaMemcpyDeviceToDevice, h->stream));
    else CK(cudaMemsetAsync(dcur, 0, nb, h->stream));
    h->t = t;
    h->warm = 0;
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_get_state(pgdto_handle* h, float* x_prev, float* g_prev, float* d_prev, int* t) {
    if (!h) return PGDTO_ERR_ARG;
    const size_t nb = (size_t)h->n * sizeof(float);
    if (x_prev) CK(cudaMemcpyAsync(x_prev, h->x_prev, nb, cudaMemcpyDeviceToDevice, h->stream));
    if (g_prev) CK(cudaMemcpyAsync(g_prev, h->g_prev, nb, cudaMemcpyDeviceToDevice, h->stream));
    if (d_prev) CK(cudaMemcpyAsync(d_prev, h->d[h->cur], nb, cudaMemcpyDeviceToDevice, h->stream));
    if (t) *t = h->t;
    return PGDTO_OK;
}

// Read the device report; clear the sticky device error once it has been reported.
// The step status from a copied report and control block; an error is reported once, after
// which the control block is cleared on the stream so the next launch starts clean.
static pgdto_status interpret_info(pgdto_handle* h, const DeviceInfo& di, const int* ctrl, pgdto_info* info,
                                   bool wait_reset) {
    int status = di.status;
    const int sticky = ctrl[2];
    const int aborted = ctrl[3];
    if (aborted && status == PGDTO_OK) status = sticky ? sticky : PGDTO_ERR_TIMEOUT;
    if (sticky != 0 || aborted) {
        cudaMemsetAsync(h->work, 0, h->ctrl_bytes, h->stream);
        if (wait_reset) cudaStreamSynchronize(h->stream);
        if (status == PGDTO_OK) status = sticky;
    }
    if (info) {
        static_assert(sizeof(DeviceInfo) == sizeof(pgdto_info), "report layouts differ");
        memcpy(info, &di, sizeof(di));
        info->status = status;
    }
    return (pgdto_status)status;
}

static pgdto_status read_info(pgdto_handle* h, pgdto_info* info, double* lambda_out) {
    DeviceInfo di;
    cudaError_t e = cudaMemcpyAsync(&di, h->dev_info, sizeof(di), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int ctrl[4];
    e = cudaMemcpyAsync(ctrl, h->work, sizeof(ctrl), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (lambda_out)
        for (int j = 0; j < h->m; ++j) lambda_out[j] = di.lambda[j];
    return interpret_info(h, di, ctrl, info, true);
}

pgdto_status pgdto_info_enqueue(pgdto_handle* h, pgdto_info_slot* slot) {
    if (!h || !slot) return PGDTO_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(&slot->info, h->dev_info, sizeof(DeviceInfo), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(slot->ctrl, h->work, sizeof(slot->ctrl), cudaMemcpyDeviceToHost, h->stream);
    return e == cudaSuccess ? PGDTO_OK : cuda_fail(e);
}

pgdto_status pgdto_info_collect(pgdto_handle* h, const pgdto_info_slot* slot, pgdto_info* info) {
    if (!h || !slot) return PGDTO_ERR_ARG;
    DeviceInfo di;
    memcpy(&di, &slot->info, sizeof(di));
    return interpret_info(h, di, slot->ctrl, info, false);
}

extern "C" pgdto_status pgdto_last_info(pgdto_handle* h, pgdto_info* info, double* lambda_out) {
    if (!h) return PGDTO_ERR_ARG;
    return read_info(h, info, lambda_out);
}

// The step parameters the device works with in double-float: (hi, lo) float pairs.
static void fill_step_df(const pgdto_params& p, float* out) {
    const double v[4] = {p.alpha_max, p.alpha_fallback, p.eps_alpha, p.omega};
    for (int i = 0; i < 4; ++i) {
        out[2 * i] = (float)v[i];
        out[2 * i + 1] = (float)(v[i] - (double)out[2 * i]);
    }
}

static void fill_seg_args(pgdto_handle* h, bool proj, float* x, const float* g, const float* A,
                          const double* bconst, const float* z_in, float* x_out, bool force_fallback, SegArgs& a) {
    memset(&a, 0, sizeof(a));
    a.n = h->n;
    a.nrows = h->m;
    a.t = h->t;
    a.proj = proj ? 1 : 0;
    a.force_fallback = force_fallback ? 1 : 0;
    for (int j = 0; j <= h->m; ++j) a.seg[j] = h->seg[j];
    a.lo = h->lo;
    a.hi = h->hi;
    a.x = x;
    a.g = g;
    a.A = A;
    a.x_prev = h->x_prev;
    a.g_prev = h->g_prev;
    a.d_prev = h->d[h->cur];
    a.d_new = h->d[1 - h->cur];
    a.z = h->z;
    a.zlo = h->zlo;
    a.z_in = z_in;
    a.x_out = x_out;
    for (int j = 0; j < h->m; ++j) {
        a.bconst[j] = bconst[j];
        split_to_floats(bconst[j], a.bconst_df + 2 * j);
    }
    a.C = h->p.C;
    a.two_c = 2.0 / h->p.C;
    split_to_floats(a.two_c, a.two_c_df);
    split_to_floats(0.5 * h->p.C, a.half_c_df);
    fill_step_df(h->p, a.step_df);
    a.alpha_max = h->p.alpha_max;
    a.alpha_fb = h->p.alpha_fallback;
    a.eps_alpha = h->p.eps_alpha;
    a.omega = h->p.omega;
    a.tol_lambda = h->p.tol_lambda;
    a.max_passes = h->p.max_passes;
    a.fault_inject = h->p.fault_inject;
    a.timeout_cycles = h->timeout_cycles;
    a.ws = (SegWork*)h->work;
    a.info_out = h->dev_info;
    a.eq_mask = h->p.eq_mask;
    a.cidx = h->cidx;
    a.ccnt = h->ccnt;
    // warm start from the previous step's lam, still in the handle's report on the device
    a.lam_prev = (!proj && h->warm)
                     ? reinterpret_cast<const double*>(reinterpret_cast<const char*>(h->dev_info) +
                                                       offsetof(DeviceInfo, lambda))
                     : nullptr;
}

static pgdto_status launch(pgdto_handle* h, bool proj, float* x, const float* g, const float* A, const double* bconst,
                           const float* z_in, float* x_out, bool force_fallback) {
    cudaError_t e;
    if (h->mode == PGDTO_COUPLED) {
        CoupledArgs a;
        memset(&a, 0, sizeof(a));
        a.n = h->n;
        a.m = h->m;
        a.t = h->t;
        a.proj = proj ? 1 : 0;
        a.force_fallback = force_fallback ? 1 : 0;
        a.lo = h->lo;
        a.hi = h->hi;
        a.x = x;
        a.g = g;
        a.A = A;
        a.x_prev = h->x_prev;
        a.g_prev = h->g_prev;
        a.d_prev = h->d[h->cur];
        a.d_new = h->d[1 - h->cur];
        a.z = h->z;
        a.zlo = h->zlo;
        a.z_in = z_in;
        a.x_out = x_out;
        for (int j = 0; j < h->m; ++j) a.bconst[j] = bconst[j];
        a.C = h->p.C;
        a.two_c = 2.0 / h->p.C;
        split_to_floats(a.two_c, a.two_c_df);
        fill_step_df(h->p, a.step_df);
        a.alpha_max = h->p.alpha_max;
        a.alpha_fb = h->p.alpha_fallback;
        a.eps_alpha = h->p.eps_alpha;
        a.omega = h->p.omega;
        a.tol_lambda = h->p.tol_lambda;
        a.tol_N = h->p.tol_N;
        a.c1 = h->p.c1;
        a.max_passes = h->p.max_passes;
        a.maxiter_newton = h->p.maxiter_newton;
        a.fault_inject = h->p.fault_inject;
        a.timeout_cycles = h->timeout_cycles;
        a.ws = (CoupledWork*)h->work;
        a.eq_mask = h->p.eq_mask;
        a.stage1 = h->p.stage1;
        // warm start from the previous step's multipliers, still in the handle's report
        a.lam_prev = (!proj && h->warm)
                         ? reinterpret_cast<const double*>(reinterpret_cast<const char*>(h->dev_info) +
                                                           offsetof(DeviceInfo, lambda))
                         : nullptr;
        e = launch_coupled(a, h->blocks, h->stream);
    } else {
        SegArgs a;
        fill_seg_args(h, proj, x, g, A, bconst, z_in, x_out, force_fallback, a);
        // free-set compaction pays where a CTA's share streams from global memory; a
        // resident share's passes are bound by their reductions, not by element work
        if (h->engine == 2 && !h->p.fault_inject) {
            a.sm_elems = h->res_cluster;
            if (a.sm_elems > 0) a.cidx = nullptr;
            e = launch_seg_clusters(a, nullptr, 1, 1, h->cl_size, seg_args_aligned(a), h->stream, a.sm_elems,
                                    a.cidx != nullptr);
        } else {
            a.sm_elems = h->res_grid;
            if (a.sm_elems > 0) a.cidx = nullptr;
            e = launch_seg(a, h->blocks, h->stream);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e);
    h->launches += 1;
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_step(pgdto_handle* h, float* x, const float* grad_f, const float* A,
                                   const double* g_val, const double* G, pgdto_info* info) {
    if (!h || !x || !grad_f || !A || !g_val || !G) return PGDTO_ERR_ARG;
    double bconst[kMaxRows] = {0, 0, 0, 0};
    double viol = 0.0;
    for (int j = 0; j < h->m; ++j) {
        if (!(isfinite(g_val[j]) && isfinite(G[j]))) return PGDTO_ERR_NONFINITE;
        bconst[j] = G[j] - g_val[j];
        // Alg. 3's fallback trigger: violation g - G of an inequality, |g - G| of an equality
        viol = fmax(viol, ((h->p.eq_mask >> j) & 1) ? fabs(g_val[j] - G[j]) : g_val[j] - G[j]);
    }
    // Alg. 3: fallback step at t = 0, or after the warm-up when a constraint is violated
    const bool fallback = h->t == 0 || (h->t >= h->p.t_warmup && viol > h->p.tol_N);
    pgdto_status s = launch(h, false, x, grad_f, A, bconst, nullptr, nullptr, fallback);
    if (s != PGDTO_OK) return s;
    h->cur = 1 - h->cur;  // d_t becomes d_prev
    h->t += 1;
    h->last_was_project = 0;
    h->warm = 1;
    if (info) return read_info(h, info, nullptr);
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_step_host(pgdto_handle* h, float* x, const float* grad_f, const float* A,
                                        const double* g_val, const double* G, pgdto_info* info) {
    if (!h || !x || !grad_f || !A || !g_val || !G) return PGDTO_ERR_ARG;
    const size_t nb = (size_t)h->n * sizeof(float);
    const size_t ab = (size_t)h->a_len * sizeof(float);
    if (!h->hx) {
        cudaError_t e;
        if ((e = cudaMalloc(&h->hx, nb)) != cudaSuccess || (e = cudaMalloc(&h->hg, nb)) != cudaSuccess ||
            (e = cudaMalloc(&h->hA, ab)) != cudaSuccess) {
            cudaFree(h->hx);
            cudaFree(h->hg);
            cudaFree(h->hA);
            h->hx = h->hg = h->hA = nullptr;
            return cuda_fail(e);
        }
    }
    CK(cudaMemcpyAsync(h->hx, x, nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->hg, grad_f, nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->hA, A, ab, cudaMemcpyHostToDevice, h->stream));
    pgdto_status s = pgdto_step(h, h->hx, h->hg, h->hA, g_val, G, nullptr);
    if (s != PGDTO_OK) return s;
    CK(cudaMemcpyAsync(x, h->hx, nb, cudaMemcpyDeviceToHost, h->stream));
    return read_info(h, info, nullptr);
}

extern "C" pgdto_status pgdto_project(pgdto_handle* h, const float* z, const float* A, const double* b, float* x_out,
                                      double* lambda_out, pgdto_info* info) {
    if (!h || !z || !A || !b || !x_out) return PGDTO_ERR_ARG;
    double bb[kMaxRows] = {0, 0, 0, 0};
    for (int j = 0; j < h->m; ++j) {
        if (!isfinite(b[j])) return PGDTO_ERR_NONFINITE;
        bb[j] = b[j];
    }
    pgdto_status s = launch(h, true, nullptr, nullptr, A, bb, z, x_out, false);
    if (s != PGDTO_OK) return s;
    h->last_was_project = 1;
    h->warm = 0;
    if (info || lambda_out) return read_info(h, info, lambda_out);
    return PGDTO_OK;
}

extern "C" int pgdto_trace(pgdto_handle* h, double* us_out, int max_marks) {
    if (!h || max_marks < 0 || (max_marks > 0 && !us_out)) return -1;
    GridCtrl c;
    if (cudaMemcpyAsync(&c, h->work, sizeof(c), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
    int k = c.ntrace < 0 ? 0 : (c.ntrace > 62 ? 62 : c.ntrace);
    for (int i = 0; i < k && i < max_marks; ++i) us_out[i] = (double)(c.trace[i] - c.trace_start) * 1e-3;
    return k;
}

// ------------------------------------------------------------------ batched entries

static pgdto_status ensure_items(pgdto_handle* h, int count) {
    if (!h->items_ev) {
        cudaError_t e = cudaEventCreateWithFlags(&h->items_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (h->items_cap >= count) return PGDTO_OK;
    cudaEventSynchronize(h->items_ev);  // the old buffers may still be read by a queued copy
    cudaStreamSynchronize(h->stream);
    cudaFree(h->items);
    cudaFreeHost(h->items_host);
    h->items = nullptr;
    h->items_host = nullptr;
    h->items_cap = 0;
    int cap = count < 64 ? 64 : count;
    cudaError_t e = cudaMalloc(&h->items, sizeof(SegArgs) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMallocHost(&h->items_host, sizeof(SegArgs) * (size_t)cap);
    if (e != cudaSuccess) return cuda_fail(e);
    h->items_cap = cap;
    return PGDTO_OK;
}

static pgdto_status ensure_fork(pgdto_handle* h, int groups) {
    if (!h->fork_ev && cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess)
        return PGDTO_ERR_CUDA;
    for (int g = 0; g + 1 < groups; ++g) {
        if (!h->aux[g] && cudaStreamCreateWithFlags(&h->aux[g], cudaStreamNonBlocking) != cudaSuccess)
            return PGDTO_ERR_CUDA;
        if (!h->join_ev[g] && cudaEventCreateWithFlags(&h->join_ev[g], cudaEventDisableTiming) != cudaSuccess)
            return PGDTO_ERR_CUDA;
    }
    return PGDTO_OK;
}

// One cluster per problem.  Problems are grouped by cluster size (one launch per size, the
// launches of different sizes run side by side on forked streams and join the handle's
// stream), and each group lists its problems largest first: the block scheduler starts
// clusters in order, so the longest do not trail at the end.
static pgdto_status launch_many(int count, pgdto_handle* const* hs, SegArgs* args, bool vec) {
    pgdto_handle* h0 = hs[0];
    for (int k = 0; k < count; ++k) {
        args[k].sm_elems = hs[k]->res_cluster;
        if (args[k].sm_elems > 0) args[k].cidx = nullptr;  // resident: no compaction (see launch)
    }
    if (count == 1) {
        cudaError_t e = launch_seg_clusters(args[0], nullptr, 1, 1, h0->cl_size, vec, h0->stream, args[0].sm_elems,
                                            args[0].cidx != nullptr);
        if (e != cudaSuccess) return cuda_fail(e);
        h0->launches += 1;
        return PGDTO_OK;
    }
    pgdto_status s = ensure_items(h0, count);
    if (s != PGDTO_OK) return s;
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (hs[a]->cl_size != hs[b]->cl_size) return hs[a]->cl_size > hs[b]->cl_size;
        return hs[a]->n > hs[b]->n;
    });
    cudaEventSynchronize(h0->items_ev);
    for (int k = 0; k < count; ++k) h0->items_host[k] = args[order[k]];
    cudaError_t e = cudaMemcpyAsync(h0->items, h0->items_host, sizeof(SegArgs) * (size_t)count,
                                    cudaMemcpyHostToDevice, h0->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h0->items_ev, h0->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int starts[6], sizes[6], smem[6], ng = 0;
    for (int k = 0; k < count; ++k) {
        if (k == 0 || hs[order[k]]->cl_size != hs[order[k - 1]]->cl_size) {
            starts[ng] = k;
            sizes[ng] = hs[order[k]]->cl_size;
            smem[ng] = 0;
            ++ng;
        }
        smem[ng - 1] = hs[order[k]]->res_cluster > smem[ng - 1] ? hs[order[k]]->res_cluster : smem[ng - 1];
    }
    starts[ng] = count;
    if (ng > 1) {
        s = ensure_fork(h0, ng);
        if (s != PGDTO_OK) return s;
        e = cudaEventRecord(h0->fork_ev, h0->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (int g = 0; g < ng; ++g) {
        cudaStream_t st = g == 0 ? h0->stream : h0->aux[g - 1];
        if (g > 0 && (e = cudaStreamWaitEvent(st, h0->fork_ev, 0)) != cudaSuccess) return cuda_fail(e);
        const int cnt = starts[g + 1] - starts[g];
        bool cmp = false;
        for (int k = starts[g]; k < starts[g + 1]; ++k) cmp = cmp || h0->items_host[k].cidx != nullptr;
        e = launch_seg_clusters(h0->items_host[starts[g]], h0->items + starts[g], cnt, cnt, sizes[g], vec, st,
                                smem[g], cmp);
        if (e != cudaSuccess) return cuda_fail(e);
        if (g > 0) {
            if ((e = cudaEventRecord(h0->join_ev[g - 1], st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(h0->stream, h0->join_ev[g - 1], 0)) != cudaSuccess)
                return cuda_fail(e);
        }
    }
    h0->launches += ng;
    return PGDTO_OK;
}

static pgdto_status check_many(int count, pgdto_handle* const* hs) {
    if (count < 1 || !hs) return PGDTO_ERR_ARG;
    for (int k = 0; k < count; ++k) {
        if (!hs[k] || hs[k]->mode == PGDTO_COUPLED || hs[k]->p.fault_inject) return PGDTO_ERR_ARG;
        if (hs[k]->stream != hs[0]->stream || hs[k]->device != hs[0]->device) return PGDTO_ERR_ARG;
        for (int q = 0; q < k; ++q)
            if (hs[q] == hs[k]) return PGDTO_ERR_ARG;  // one step per handle per launch
    }
    if (hs[0]->cl_size < 1) return PGDTO_ERR_UNSUPPORTED;
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_step_many(int count, pgdto_handle* const* hs, float* const* x,
                                        const float* const* grad_f, const float* const* A, const double* g_val,
                                        const double* G, pgdto_info* infos) {
    pgdto_status s = check_many(count, hs);
    if (s != PGDTO_OK) return s;
    if (!x || !grad_f || !A || !g_val || !G) return PGDTO_ERR_ARG;
    SegArgs* args = new SegArgs[count];
    bool vec = true;
    for (int k = 0; k < count; ++k) {
        pgdto_handle* h = hs[k];
        if (!x[k] || !grad_f[k] || !A[k]) {
            delete[] args;
            return PGDTO_ERR_ARG;
        }
        double bconst[kMaxRows] = {0, 0, 0, 0};
        double viol = 0.0;
        for (int j = 0; j < h->m; ++j) {
            const double gv = g_val[4 * k + j], gg = G[4 * k + j];
            if (!(isfinite(gv) && isfinite(gg))) {
                delete[] args;
                return PGDTO_ERR_NONFINITE;
            }
            bconst[j] = gg - gv;
            viol = fmax(viol, ((h->p.eq_mask >> j) & 1) ? fabs(gv - gg) : gv - gg);
        }
        const bool fallback = h->t == 0 || (h->t >= h->p.t_warmup && viol > h->p.tol_N);
        fill_seg_args(h, false, x[k], grad_f[k], A[k], bconst, nullptr, nullptr, fallback, args[k]);
        vec = vec && seg_args_aligned(args[k]);
    }
    s = launch_many(count, hs, args, vec);
    delete[] args;
    if (s != PGDTO_OK) return s;
    for (int k = 0; k < count; ++k) {
        hs[k]->cur = 1 - hs[k]->cur;
        hs[k]->t += 1;
        hs[k]->last_was_project = 0;
        hs[k]->warm = 1;
    }
    if (!infos) return PGDTO_OK;
    pgdto_status worst = PGDTO_OK;
    for (int k = 0; k < count; ++k) {
        pgdto_status r = read_info(hs[k], &infos[k], nullptr);
        if (r != PGDTO_OK && worst == PGDTO_OK) worst = r;
    }
    return worst;
}

extern "C" pgdto_status pgdto_project_many(int count, pgdto_handle* const* hs, const float* const* z,
                                           const float* const* A, const double* b, float* const* x_out,
                                           double* lambda_out, pgdto_info* infos) {
    pgdto_status s = check_many(count, hs);
    if (s != PGDTO_OK) return s;
    if (!z || !A || !b || !x_out) return PGDTO_ERR_ARG;
    SegArgs* args = new SegArgs[count];
    bool vec = true;
    for (int k = 0; k < count; ++k) {
        pgdto_handle* h = hs[k];
        if (!z[k] || !A[k] || !x_out[k]) {
            delete[] args;
            return PGDTO_ERR_ARG;
        }
        double bb[kMaxRows] = {0, 0, 0, 0};
        for (int j = 0; j < h->m; ++j) {
            if (!isfinite(b[4 * k + j])) {
                delete[] args;
                return PGDTO_ERR_NONFINITE;
            }
            bb[j] = b[4 * k + j];
        }
        fill_seg_args(h, true, nullptr, nullptr, A[k], bb, z[k], x_out[k], false, args[k]);
        vec = vec && seg_args_aligned(args[k]);
    }
    s = launch_many(count, hs, args, vec);
    delete[] args;
    if (s != PGDTO_OK) return s;
    for (int k = 0; k < count; ++k) {
        hs[k]->last_was_project = 1;
        hs[k]->warm = 0;
    }
    if (!infos && !lambda_out) return PGDTO_OK;
    pgdto_status worst = PGDTO_OK;
    for (int k = 0; k < count; ++k) {
        pgdto_info tmp;
        pgdto_status r = read_info(hs[k], infos ? &infos[k] : &tmp, lambda_out ? lambda_out + 4 * k : nullptr);
        if (r != PGDTO_OK && worst == PGDTO_OK) worst = r;
    }
    return worst;
}
