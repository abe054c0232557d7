// dev_common.cuh -- device building blocks shared by the PGD-TO kernels (sm_103a).
//
//  * double-float ("DF") accumulation: a value kept as an unevaluated sum hi + lo of two
//    floats, combined with Knuth's TwoSum and Dekker's FastTwoSum (error-free transforms),
//    so reductions over millions of FP32 terms keep ~44 bits without FP64 arithmetic
//    (FP64 throughput is a small fraction of FP32 on this part);
//  * warp / block reductions of DF values;
//  * a grid-wide all-reduce step: every block writes its partial sums and arrives on a
//    counter; once all have arrived, every block sums all partials in a fixed order and
//    runs the scalar update on its own copy of the search state, so no result is
//    broadcast.  Waits are bounded: a block that has waited longer than its budget
//    records PGDTO_ERR_TIMEOUT, raises an abort flag and returns, so a fault elsewhere
//    never hangs the GPU.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace pgdto {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// The cluster engine runs two 256-thread CTAs per SM: while one CTA's scalar update holds its
// warps at a barrier, the other CTA's element pass keeps the SM busy.
constexpr int kClusterThreads = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxVals = 136;   // DF values per grid reduction (4 rows x 2 x 16 points + spare)
constexpr int kMaxBlockVals = 32;  // DF values one block_reduce call gathers per warp
constexpr int kMaxMax = 12;     // float max values per grid reduction (3 per row of 4)

// status codes shared with include/pgdto.h
enum : int { kOk = 0, kErrNonfinite = 4, kErrTimeout = 5, kNotConverged = 7 };

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_zero() { return DF{0.0f, 0.0f}; }

// Knuth TwoSum: s = fl(a + b), e = (a + b) - s exactly.
__device__ __forceinline__ DF two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// Dekker FastTwoSum, valid when |a| >= |b| (or a == 0).
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return DF{s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
    DF s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Double-float multiply, divide and square root after Dekker's double-length arithmetic
// (T. J. Dekker, "A floating-point technique for extending the available precision",
// 1971), with the exact products taken by FMA.
//
// a * b to double-float accuracy (the product of the hi parts exact via FMA).
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

// a / b to double-float accuracy: q1 = a.hi / b.hi, then one correction from the exact
// remainder a - q1 b.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const float p = q1 * b.hi;
    DF r = df_add(a, DF{-p, -fmaf(q1, b.hi, -p)});
    r = df_add_f(r, -q1 * b.lo);
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// sqrt(a) for a > 0 to double-float accuracy: s = sqrt(a.hi), then one Newton correction
// (a - s^2) / (2 s) from the exact square.
__device__ __forceinline__ DF df_sqrt(DF a) {
    const float s = __fsqrt_rn(a.hi);
    const float p = s * s;
    const DF r = df_add(a, DF{-p, -fmaf(s, s, -p)});
    const DF v = fast_two_sum(s, __fdiv_rn(r.hi, 2.0f * s));
    return (a.hi > 0.0f && a.hi < INFINITY) ? v : DF{s, 0.0f};  // 0, inf and NaN as sqrtf gives them
}

__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ DF df_min(DF a, DF b) { return df_lt(b, a) ? b : a; }

// Split a double into hi + lo floats (hi = nearest float, lo = nearest float of the rest).
__device__ __host__ __forceinline__ void split_double(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ DF warp_reduce_df(DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, u);
    }
    return v;
}

__device__ __forceinline__ float warp_reduce_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------ memory ordering

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned atom_add_relaxed_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// ------------------------------------------------------------------ grid control block

struct GridCtrl {
    unsigned count;    // arrivals in the current round
    int pad0;
    int status;        // sticky pgdto_status of device work
    int abort;         // raised by a block that gave up; every wait then returns
    unsigned long long launches;  // kernels that ran to completion (diagnostics)
    int pad1[26];
    unsigned gen;      // round counter, bumped by the last block to arrive (own 128-byte line: the
    int pad2[31];      // waiting blocks poll it while the others still arrive on `count`)
    unsigned long long trace_start;  // globaltimer at kernel entry (block 0)
    unsigned long long trace[62];    // globaltimer after each grid round's update (block 0)
    int ntrace;
    int pad3[3];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Partial sums of one grid reduction: DF values (SoA over blocks) and float maxima.
struct Partials {
    float2 v[kMaxVals][kMaxBlocks];
    float mx[kMaxMax][kMaxBlocks];
};

// Per-block scratch for reductions (shared memory).
struct BlockScratch {
    DF warp_vals[kMaxBlockVals][kWarps];  // sized for the largest block (512 threads)
    float warp_max[kMaxMax][kWarps];
    DF tot[kMaxVals];
    float totmax[kMaxMax];
    int flag;
    unsigned gen;
};

__host__ __device__ constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }

// Warp sums of P values per lane by recursive halving: at each of the first log2(P)
// butterfly steps a lane keeps one half of its values (the upper one when its lane bit
// for that step is set), sends the other half to its partner and adds the partner's copy
// of the half it keeps; the remaining steps are plain butterfly additions.  Every value is
// summed over all 32 lanes by the same fixed tree, with P - 1 + (5 - log2 P) exchanges
// instead of 5 P.  On return w[0] holds the warp total of value `idx`.
template <int P, int N, int O>
struct WarpHalving {
    __device__ static __forceinline__ void run(DF (&w)[P], int lane, int& idx) {
        if constexpr (O > 0) {
            if constexpr (N > 1) {
                constexpr int H = N / 2;
                const bool up = (lane & O) != 0;
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    const DF send = up ? w[i] : w[H + i];
                    const DF keep = up ? w[H + i] : w[i];
                    DF r;
                    r.hi = __shfl_xor_sync(0xffffffffu, send.hi, O);
                    r.lo = __shfl_xor_sync(0xffffffffu, send.lo, O);
                    w[i] = df_add(keep, r);
                }
                if (up) idx += H;
                WarpHalving<P, H, O / 2>::run(w, lane, idx);
            } else {
                DF r;
                r.hi = __shfl_xor_sync(0xffffffffu, w[0].hi, O);
                r.lo = __shfl_xor_sync(0xffffffffu, w[0].lo, O);
                w[0] = df_add(w[0], r);
                WarpHalving<P, 1, O / 2>::run(w, lane, idx);
            }
        }
    }
};

// Reduce NV per-thread DF values and NM per-thread maxima (mx may be null when NM == 0);
// the block totals land in sc.tot[voff + i] and sc.totmax[moff + i].
template <int NV, int NM>
__device__ __forceinline__ void block_reduce(const DF (&v)[NV], const float* mx, BlockScratch& sc, int voff = 0,
                                             int moff = 0) {
    static_assert(NV <= kMaxBlockVals && NM <= kMaxMax, "block_reduce gathers at most kMaxBlockVals values");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if constexpr (NV > 0) {
        constexpr int P = pow2_ceil(NV);
        static_assert(P <= 32, "one warp sums at most 32 values at once");
        DF w[P];
#pragma unroll
        for (int i = 0; i < P; ++i) w[i] = i < NV ? v[i] : df_zero();
        int idx = 0;
        WarpHalving<P, P, 16>::run(w, lane, idx);
        // lanes that differ only in the bits of the plain steps hold the same total
        if (idx < NV && (lane & (32 / P - 1)) == 0) sc.warp_vals[idx][warp] = w[0];
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        float r = warp_reduce_max(mx[i]);
        if (lane == 0) sc.warp_max[i][warp] = r;
    }
    __syncthreads();
    for (int i = warp; i < NV; i += nw) {
        DF r = lane < nw ? sc.warp_vals[i][lane] : df_zero();
        r = warp_reduce_df(r);
        if (lane == 0) sc.tot[voff + i] = r;
    }
    for (int i = warp; i < NM; i += nw) {
        float r = lane < nw ? sc.warp_max[i][lane] : -INFINITY;
        r = warp_reduce_max(r);
        if (lane == 0) sc.totmax[moff + i] = r;
    }
    __syncthreads();
}

// Grid-wide all-reduce of sc.tot[0..nv) / sc.totmax[0..nm) followed by the scalar update,
// which every block runs on its own copy of the state.  Each block publishes its totals in
// the round's partials buffer and arrives; the last to arrive resets the count and
// releases the round.  Every block then sums all partials in block order and runs
// update(sc) on its warp 0: every block computes the same totals and, with the same code
// on the same inputs, the same state, so no result has to be broadcast.  Rounds alternate
// between two buffers: a block cannot pass the next round before every block has arrived
// there, after reading this round's partials, so it is never more than one round ahead.
// Returns false if the wait was abandoned (timeout or abort); the caller must then return.
// Block 0 appends the round's completion time to ctrl->trace.
//
// The part that is the same in every round (publish, arrive, wait, gather) is one
// out-of-line function: a step runs several rounds, and each inlined copy of this code
// would be fetched into the instruction cache cold (the caller's L2 traffic between steps
// evicts the kernel's code), where one shared copy is fetched once per launch.
static __device__ __noinline__ bool grid_round_gather(GridCtrl* ctrl, Partials* part2, BlockScratch& sc, int nv,
                                                     int nm, long long timeout_cycles) {
    const int tid = threadIdx.x;
    const int nb = gridDim.x;
    Partials* part = part2 + (sc.gen & 1u);
    for (int i = tid; i < nv; i += blockDim.x) part->v[i][blockIdx.x] = make_float2(sc.tot[i].hi, sc.tot[i].lo);
    for (int i = tid; i < nm; i += blockDim.x) part->mx[i][blockIdx.x] = sc.totmax[i];
    __syncthreads();
    if (tid == 0) {
        // release: the block's partials (written before the barrier above) are visible to
        // whoever observes this arrival; acquire: the last block to arrive reads the count
        // every other block's arrival released, so it sees all of their partials
        const unsigned old = atom_add_acq_rel_u32(&ctrl->count, 1u);
        const unsigned target = sc.gen + 1u;
        int ok = 1;
        if (old == (unsigned)(nb - 1)) {
            ctrl->count = 0u;
            st_release_u32(&ctrl->gen, target);  // orders the reset before the next round's arrivals
        } else {
            long long t0 = clock64();
            unsigned spins = 0;
            while (ld_acquire_u32(&ctrl->gen) != target) {
                if (((++spins) & 63u) == 0u) {
                    if (ld_volatile_i32(&ctrl->abort)) {
                        ok = 0;
                        break;
                    }
                    if (clock64() - t0 > timeout_cycles) {
                        atomicExch(&ctrl->status, kErrTimeout);
                        atomicExch(&ctrl->abort, 1);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        sc.gen = target;
        sc.flag = ok;
    }
    __syncthreads();
    if (!sc.flag) return false;
    const int lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
    // Warp w sums values w, w + nw, ...; it issues the loads of up to kGatherVals values
    // (kGatherPer blocks per lane each) before adding any, so the round pays the latency of
    // the partials' reads once rather than once per value.  Lane l adds blocks l, l + 32,
    // ... in that order and the lanes combine by the same tree for every value.
    constexpr int kGatherVals = 5, kGatherPer = 5;
    for (int j0 = 0; j0 * nw < nv; j0 += kGatherVals) {
        DF acc[kGatherVals];
#pragma unroll
        for (int j = 0; j < kGatherVals; ++j) acc[j] = df_zero();
        for (int b0 = 0; b0 < nb; b0 += 32 * kGatherPer) {
            float2 buf[kGatherVals][kGatherPer];
#pragma unroll
            for (int j = 0; j < kGatherVals; ++j) {
                const int i = warp + nw * (j0 + j);
#pragma unroll
                for (int k = 0; k < kGatherPer; ++k) {
                    const int b = b0 + lane + 32 * k;
                    buf[j][k] = (i < nv && b < nb) ? __ldcg(&part->v[i][b]) : make_float2(0.0f, 0.0f);
                }
            }
#pragma unroll
            for (int j = 0; j < kGatherVals; ++j)
#pragma unroll
                for (int k = 0; k < kGatherPer; ++k) acc[j] = df_add(acc[j], DF{buf[j][k].x, buf[j][k].y});
        }
#pragma unroll
        for (int j = 0; j < kGatherVals; ++j) {
            const int i = warp + nw * (j0 + j);
            const DF r = warp_reduce_df(acc[j]);
            if (lane == 0 && i < nv) sc.tot[i] = r;
        }
    }
    // maxima: the same batching (a maximum does not depend on the order)
    for (int j0 = 0; j0 * nw < nm; j0 += kGatherVals) {
        float acc[kGatherVals];
#pragma unroll
        for (int j = 0; j < kGatherVals; ++j) acc[j] = -INFINITY;
        for (int b0 = 0; b0 < nb; b0 += 32 * kGatherPer) {
            float buf[kGatherVals][kGatherPer];
#pragma unroll
            for (int j = 0; j < kGatherVals; ++j) {
                const int i = warp + nw * (j0 + j);
#pragma unroll
                for (int k = 0; k < kGatherPer; ++k) {
                    const int b = b0 + lane + 32 * k;
                    buf[j][k] = (i < nm && b < nb) ? __ldcg(&part->mx[i][b]) : -INFINITY;
                }
            }
#pragma unroll
            for (int j = 0; j < kGatherVals; ++j)
#pragma unroll
                for (int k = 0; k < kGatherPer; ++k) acc[j] = fmaxf(acc[j], buf[j][k]);
        }
#pragma unroll
        for (int j = 0; j < kGatherVals; ++j) {
            const int i = warp + nw * (j0 + j);
            const float r = warp_reduce_max(acc[j]);
            if (lane == 0 && i < nm) sc.totmax[i] = r;
        }
    }
    __syncthreads();
    return true;
}

template <class Update>
__device__ bool grid_allreduce_update(GridCtrl* ctrl, Partials* part2, BlockScratch& sc, int nv, int nm,
                                      long long timeout_cycles, Update&& update) {
    if (!grid_round_gather(ctrl, part2, sc, nv, nm, timeout_cycles)) return false;
    const int tid = threadIdx.x;
    if (tid < 32) {
        update(sc);
        __syncwarp();
    }
    if (tid == 0 && blockIdx.x == 0) {
        volatile GridCtrl* vc = ctrl;
        const int k = vc->ntrace;
        if (k >= 0 && k < 62) {
            vc->trace[k] = globaltimer_ns();
            vc->ntrace = k + 1;
        }
    }
    __syncthreads();
    return true;
}

// Cluster-wide reduction of sc.tot / sc.totmax followed by the scalar update, for the CTAs
// of one thread-block cluster.  After a cluster barrier the first CTA reads every CTA's
// block totals through distributed shared memory (lane r of a warp reads rank r, fixed
// order: deterministic), runs update(sc) on its warp 0, and a second barrier publishes
// the result.  The barriers are the hardware's: they complete when every CTA of the
// cluster arrives, as every CTA runs the same sequence of phases.
template <class Update>
__device__ void cluster_reduce_update(BlockScratch& sc, int nv, int nm, Update&& update) {
    namespace cgn = cooperative_groups;
    cgn::cluster_group cl = cgn::this_cluster();
    cl.sync();
    if (cl.block_rank() == 0) {
        const int S = (int)cl.num_blocks();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
        for (int i = warp; i < nv; i += nw) {
            DF v = df_zero();
            if (lane < S) v = cl.map_shared_rank(&sc, lane)->tot[i];
            v = warp_reduce_df(v);
            __syncwarp();
            if (lane == 0) sc.tot[i] = v;
        }
        for (int i = warp; i < nm; i += nw) {
            float v = -INFINITY;
            if (lane < S) v = cl.map_shared_rank(&sc, lane)->totmax[i];
            v = warp_reduce_max(v);
            __syncwarp();
            if (lane == 0) sc.totmax[i] = v;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            update(sc);
            __syncwarp();
        }
        __syncthreads();
    }
    cl.sync();
}

// Every block calls this once at kernel start, before its first grid_reduce_update: the
// round counter is read while no round can have completed (this block has not arrived).
__device__ __forceinline__ void grid_sync_init(GridCtrl* ctrl, BlockScratch& sc) {
    if (threadIdx.x == 0) sc.gen = ld_acquire_u32(&ctrl->gen);
    __syncthreads();
}

// Contiguous chunk [cb, ce) of [s, e) owned by block `blk` of `nb`, multiple of 4 long.
__device__ __forceinline__ void block_chunk(int64_t s, int64_t e, int blk, int nb, int64_t& cb, int64_t& ce) {
    seg_chunk(s, e, blk, nb, cb, ce);
}

}  // namespace pgdto
