// tune.cu -- per-device choice of the cluster engine's block share for the batched form.
//
// A batched step (pgdto_step_many) gives each problem a thread-block cluster whose size
// follows from n and the block share params.cluster_elems: fewer, fuller blocks leave more
// of the GPU to the other problems of the batch, more blocks shorten each problem's passes.
// Which wins depends on n, on the batch size and on the part, so pgdto_autotune_batch
// measures it: it builds `count` synthetic single-row problems of n variables on the device,
// times a few batched steps for each candidate share with CUDA events, and records the
// fastest in the per-device table that pgdto_create reads when params.cluster_elems is 0.
// The paper has no counterpart; the step timed is Alg. 3 as in pgdto_step.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgdto.h"
#include "handle_internal.h"

namespace {

constexpr int kFillThreads = 256;
constexpr int kWarm = 3;
constexpr int kTimed = 5;
constexpr int kCandidates[] = {1024, 2048, 4096, 8192};
constexpr int64_t kMaxTuneN = int64_t(1) << 17;  // the cluster engine's range under engine = auto
constexpr int kMaxTuneCount = 4096;

// "lowbias32", an integer hash found by C. Wellons' hash-prospector search; a value in
// [0, 1) from the top 24 bits.
__device__ __forceinline__ float unit_hash(uint32_t v) {
    v ^= v >> 16;
    v *= 0x7feb352du;
    v ^= v >> 15;
    v *= 0x846ca68bu;
    v ^= v >> 16;
    return (float)(v >> 8) * (1.0f / 16777216.0f);
}

// Synthetic problems: design x in [0, 1), sensitivities in [-1, 1), coefficients in
// [0.5, 1.5), a previous iterate 0.01 away and a previous gradient 0.1 away, the previous
// direction its negative.  Element i of the whole batch draws from counters 5i .. 5i + 4
// (below 2^32 for the largest batch accepted).
__global__ void fill_problems(float* __restrict__ x, float* __restrict__ g, float* __restrict__ a,
                              float* __restrict__ xp, float* __restrict__ gp, float* __restrict__ dp,
                              int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(5 * i);
        const float xv = unit_hash(c), gv = 2.0f * unit_hash(c + 1) - 1.0f;
        x[i] = xv;
        g[i] = gv;
        a[i] = 0.5f + unit_hash(c + 2);
        xp[i] = fminf(fmaxf(xv - 0.01f * (2.0f * unit_hash(c + 3) - 1.0f), 0.0f), 1.0f);
        const float gpv = gv + 0.1f * (2.0f * unit_hash(c + 4) - 1.0f);
        gp[i] = gpv;
        dp[i] = -gpv;
    }
}

// A bounded device-side wait of `cycles` clock cycles: it keeps the stream busy while the
// host marshals the batch, so the events that follow bracket device work only.
__global__ void spin_cycles(long long cycles) {
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) {
    }
}

struct Buffers {
    float* p[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    ~Buffers() {
        for (float* q : p)
            if (q) cudaFree(q);
    }
};

struct Handles {
    std::vector<pgdto_handle*> h;
    ~Handles() {
        for (pgdto_handle* q : h) pgdto_destroy(q);
    }
};

pgdto_status fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? PGDTO_ERR_OOM : PGDTO_ERR_CUDA; }

}  // namespace

extern "C" pgdto_status pgdto_autotune_batch(int64_t n, int count, int* best_out, double* ms_out,
                                             void* cuda_stream) {
    if (n < 1 || n > kMaxTuneN || count < 1 || count > kMaxTuneCount) return PGDTO_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return fail(e);
    const int64_t total = n * (int64_t)count;
    const size_t bytes = (size_t)total * sizeof(float);
    // x, its starting copy, g, a, x_prev, g_prev, d_prev
    Buffers buf;
    for (float*& q : buf.p)
        if ((e = cudaMalloc(&q, bytes)) != cudaSuccess) return fail(e);
    float *x = buf.p[0], *x0 = buf.p[1], *g = buf.p[2], *a = buf.p[3];
    float *xp = buf.p[4], *gp = buf.p[5], *dp = buf.p[6];
    const int fill_blocks = (int)std::min<int64_t>((total + kFillThreads - 1) / kFillThreads, 4096);
    fill_problems<<<fill_blocks, kFillThreads, 0, stream>>>(x0, g, a, xp, gp, dp, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);

    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
    if (clock_khz <= 0) clock_khz = 2000000;
    const long long spin = (long long)clock_khz;  // about 1 ms

    std::vector<float*> xs(count), gs(count), as(count);
    std::vector<double> gval(4 * (size_t)count, 0.0), G(4 * (size_t)count, 0.0);
    for (int k = 0; k < count; ++k) {
        xs[k] = x + k * n;
        gs[k] = g + k * n;
        as[k] = a + k * n;
        // E[a x] = 0.5 per variable: the row sits above its bound, so the projection binds
        gval[4 * k] = 0.5 * (double)n;
        G[4 * k] = 0.45 * (double)n;
    }
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(e);
    }
    int best = 0;
    double best_ms = 0.0;
    pgdto_status st = PGDTO_OK;
    for (int c : kCandidates) {
        pgdto_params p;
        pgdto_params_default(&p);
        p.mode = PGDTO_SINGLE;
        p.engine = 2;
        p.cluster_elems = c;
        Handles hs;
        hs.h.assign(count, nullptr);
        bool made = true;
        for (int k = 0; k < count && made; ++k) {
            st = pgdto_create(&hs.h[k], n, 1, nullptr, 0.0f, 1.0f, &p, stream);
            if (st == PGDTO_ERR_UNSUPPORTED) made = false;  // this share does not fit: skip it
            else if (st != PGDTO_OK) break;
        }
        if (!made) {
            st = PGDTO_OK;
            continue;
        }
        if (st != PGDTO_OK) break;
        std::vector<float> ms;
        for (int r = 0; r < kWarm + kTimed && st == PGDTO_OK; ++r) {
            if ((e = cudaMemcpyAsync(x, x0, bytes, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess) {
                st = fail(e);
                break;
            }
            for (int k = 0; k < count && st == PGDTO_OK; ++k)
                st = pgdto_set_state(hs.h[k], xp + k * n, gp + k * n, dp + k * n, 1);
            if (st != PGDTO_OK) break;
            spin_cycles<<<1, 1, 0, stream>>>(spin);
            cudaEventRecord(ev[0], stream);
            st = pgdto_step_many(count, hs.h.data(), xs.data(), gs.data(), as.data(), gval.data(), G.data(),
                                 nullptr);
            cudaEventRecord(ev[1], stream);
            if (st != PGDTO_OK) break;
            if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) {
                st = fail(e);
                break;
            }
            for (int k = 0; k < count && st == PGDTO_OK; ++k) {
                pgdto_info info;
                const pgdto_status r2 = pgdto_last_info(hs.h[k], &info, nullptr);
                if (r2 != PGDTO_OK && r2 != PGDTO_NOT_CONVERGED) st = r2;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[0], ev[1]);
            if (r >= kWarm) ms.push_back(t);
        }
        if (st != PGDTO_OK) break;
        std::sort(ms.begin(), ms.end());
        const double med = ms[ms.size() / 2];
        if (best == 0 || med < best_ms) {
            best = c;
            best_ms = med;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != PGDTO_OK) return st;
    if (best == 0) return PGDTO_ERR_UNSUPPORTED;
    pgdto_set_tuned_cluster_elems(device, n, best);
    if (best_out) *best_out = best;
    if (ms_out) *ms_out = best_ms;
    return PGDTO_OK;
}
