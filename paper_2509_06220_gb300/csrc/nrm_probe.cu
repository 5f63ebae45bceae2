// nrm_probe.cu -- register-only throughput probes of the SM pipes that bound
// the tree kernels (measurement only; the paper has no counterpart).
//
// The roofline of the binary64 tree is set by the FP64 pipe (one DFMA and one
// DMUL per v1_hypot) and by instruction issue, not by HBM.  The nominal FP64
// rate of a GB300 is not the rate this pipe sustains, so the benchmark
// measures it: every thread runs 8 independent dependency chains of one
// operation kind, 4 iterations unrolled, and the caller times the launch
// with CUDA events.  The values stay finite and normal, nothing is read from
// or written to memory except one store that never happens (it keeps the
// chains alive through the optimiser).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/nrm.h"

namespace {

constexpr int CHAINS = 8, UNROLL = 4;

template <int KIND> __device__ __forceinline__ double step_d(double a, double b, double c) {
    if constexpr (KIND == 0) return __fma_rn(a, b, c);
    else return __dmul_rn(a, b);
}

template <int KIND> __global__ void __launch_bounds__(256) fp64_probe_kernel(int64_t iters, double *sink) {
    double a[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) a[j] = 1.0 + (threadIdx.x + 37 * j) * 0x1p-20;
    // a -> a b + c contracts towards c / (1 - b) = 1; a -> a b drifts by
    // (1 - 2^-40)^(4 iters), far from underflow for any iteration count used
    const double b = 1.0 - 0x1p-40, c = 0x1p-40;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) a[j] = step_d<KIND>(a[j], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += a[j];
    if (s == -1.0) *sink = s; // never true: the chains must be computed
}

__global__ void __launch_bounds__(256) fp32_probe_kernel(int64_t iters, double *sink) {
    float a[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) a[j] = 1.0f + (threadIdx.x + 37 * j) * 0x1p-20f;
    const float b = 1.0f - 0x1p-20f, c = 0x1p-20f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) a[j] = __fmaf_rn(a[j], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += a[j];
    if (s == -1.0f) *sink = s;
}

} // namespace

extern "C" nrm_status nrm_probe_pipe(int32_t kind, int64_t iters, int32_t blocks_per_sm, double *sink,
                                     int64_t *thread_ops, void *stream) {
    if (kind < 0 || kind > 2 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !sink) return NRM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return NRM_EDEVICE;
    const unsigned blocks = (unsigned)(sms * blocks_per_sm);
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) fp64_probe_kernel<0><<<blocks, 256, 0, s>>>(iters, sink);
    else if (kind == 1) fp64_probe_kernel<1><<<blocks, 256, 0, s>>>(iters, sink);
    else fp32_probe_kernel<<<blocks, 256, 0, s>>>(iters, sink);
    if (thread_ops) *thread_ops = (int64_t)blocks * 256 * iters * UNROLL * CHAINS;
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}
