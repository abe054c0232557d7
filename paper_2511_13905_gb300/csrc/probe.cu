// probe.cu -- read-bandwidth probe used to place the root-search passes on a roofline.
//
// The projection passes re-read the trial point and the constraint coefficients several
// times per step; when that working set fits the L2 cache their bound is the L2 read
// rate, not the HBM rate.  pgdto_probe_read times nothing itself: it launches one plain
// streaming read of a buffer (128-bit loads, grid-stride, a sum per block so the loads
// are not removed), and the caller times repeated launches with CUDA events.  A buffer
// well under the L2 size, read again and again, gives the L2 read rate; one far larger
// than L2 gives the HBM read rate.  The paper has no counterpart; this is measurement
// tooling, not part of the optimizer step.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pgdto.h"

namespace {

constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads) probe_read_kernel(const float4* __restrict__ buf, int64_t n4,
                                                                 float* __restrict__ out) {
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four independent 16-byte loads in flight per thread per iteration
    for (; i + 3 * stride < n4; i += 4 * stride) {
        const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
        const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
        acc += (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w) + (c.x + c.y + c.z + c.w) + (d.x + d.y + d.z + d.w);
    }
    for (; i < n4; i += stride) {
        const float4 a = __ldcg(buf + i);
        acc += a.x + a.y + a.z + a.w;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float ws[kProbeThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < kProbeThreads / 32; ++w) s += ws[w];
        out[blockIdx.x] = s;
    }
}

}  // namespace

extern "C" pgdto_status pgdto_probe_read(const float* buf, int64_t n, float* out, int blocks, void* cuda_stream) {
    if (!buf || !out || n < 4 || (n & 3) || blocks < 1 || (reinterpret_cast<uintptr_t>(buf) & 15u))
        return PGDTO_ERR_ARG;
    probe_read_kernel<<<blocks, kProbeThreads, 0, (cudaStream_t)cuda_stream>>>(reinterpret_cast<const float4*>(buf),
                                                                              n / 4, out);
    return cudaGetLastError() == cudaSuccess ? PGDTO_OK : PGDTO_ERR_CUDA;
}
