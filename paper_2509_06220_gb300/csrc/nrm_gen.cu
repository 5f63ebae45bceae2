// nrm_gen.cu -- seeded synthetic inputs on the device (not part of the
// method): the SplitMix64 counter hash of Steele, Lea and Flood (OOPSLA
// 2014) keyed by (seed, vector id, element index), and bit construction of
// each element (random sign, uniform fraction, exponent uniform in
// [emin, emax]).  The Python module paper_2509_06220_gb300/inputs.py
// implements the same definition on the host.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/nrm.h"

namespace {

constexpr uint64_t GOLD = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t key_of(uint64_t seed, uint64_t vec) {
    return mix64(seed ^ mix64((vec + 1) * GOLD));
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLD); }

__device__ __forceinline__ double elem_d(uint64_t u, int emin, uint64_t span) {
    const uint64_t e = (((u >> 52) & 0x7FFull) * span) >> 11;
    const uint64_t biased = (uint64_t)((int64_t)e + emin + 1023);
    const uint64_t b = (u & 0x8000000000000000ull) | (biased << 52) | (u & ((1ull << 52) - 1));
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ float elem_s(uint64_t u, int emin, uint64_t span) {
    const uint64_t e = (((u >> 23) & 0xFFFFull) * span) >> 16;
    const uint32_t biased = (uint32_t)((int64_t)e + emin + 127);
    const uint32_t b = ((uint32_t)(u >> 63) << 31) | (biased << 23) | (uint32_t)(u & ((1u << 23) - 1));
    return __int_as_float((int)b);
}

template <typename T>
__global__ void gen_kernel(T *x, int64_t n, uint64_t key, int64_t start, int emin, uint64_t span) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t u = draw(key, (uint64_t)(start + i));
        if constexpr (sizeof(T) == 8) x[i] = elem_d(u, emin, span);
        else x[i] = elem_s(u, emin, span);
    }
}

template <typename T>
__global__ void gen_ragged_kernel(T *x, int64_t x_len, const int64_t *off, int64_t B, uint64_t seed, int emin,
                                  uint64_t span) {
    for (int64_t v = blockIdx.x; v < B; v += gridDim.x) {
        const int64_t a = off[v], b = off[v + 1];
        if (a < 0 || b < a || b > x_len) continue; // malformed vector: left untouched
        const uint64_t key = key_of(seed, (uint64_t)v);
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            const uint64_t u = draw(key, (uint64_t)(i - a));
            if constexpr (sizeof(T) == 8) x[i] = elem_d(u, emin, span);
            else x[i] = elem_s(u, emin, span);
        }
    }
}

bool range_ok(nrm_dtype dt, int emin, int emax) {
    if (dt == NRM_F64) return -1022 <= emin && emin <= emax && emax <= 1023;
    if (dt == NRM_F32) return -126 <= emin && emin <= emax && emax <= 127;
    return false;
}

} // namespace

extern "C" nrm_status nrm_gen(nrm_dtype dtype, void *x, int64_t n, uint64_t seed, uint64_t vec, int64_t start,
                              int32_t emin, int32_t emax, void *stream) {
    if (n < 0 || start < 0 || (n > 0 && !x) || !range_ok(dtype, emin, emax)) return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const uint64_t key = key_of(seed, vec);
    const uint64_t span = (uint64_t)(emax - emin + 1);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 32);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == NRM_F64) gen_kernel<double><<<(unsigned)blocks, 256, 0, s>>>((double *)x, n, key, start, emin, span);
    else gen_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((float *)x, n, key, start, emin, span);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

extern "C" nrm_status nrm_gen_ragged(nrm_dtype dtype, void *x, int64_t x_len, const int64_t *offsets, int64_t B,
                                     uint64_t seed, int32_t emin, int32_t emax, void *stream) {
    if (B < 0 || x_len < 0 || (B > 0 && !offsets) || (x_len > 0 && !x) || !range_ok(dtype, emin, emax))
        return NRM_EINVAL;
    if (B == 0) return NRM_OK;
    const uint64_t span = (uint64_t)(emax - emin + 1);
    const unsigned blocks = (unsigned)std::min<int64_t>(B, 152 * 16);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == NRM_F64) gen_ragged_kernel<double><<<blocks, 256, 0, s>>>((double *)x, x_len, offsets, B, seed, emin, span);
    else gen_ragged_kernel<float><<<blocks, 256, 0, s>>>((float *)x, x_len, offsets, B, seed, emin, span);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

// ---------------------------------------------------------------------------
// segment generator for the server: one launch fills every device-generated
// request of a step (vector id = request id), same elements as nrm_gen
// ---------------------------------------------------------------------------
#include "nrm_internal.h"

uint64_t nrm_gen_key(uint64_t seed, uint64_t vec) { return key_of(seed, vec); }

namespace {
// Tiles of GEN_TILE consecutive elements of the concatenated segments: the
// segment of a tile's first element is found once per tile (the same
// binary search in every thread of the block, uniform loads), and each
// thread then walks its elements of the tile in order, stepping to the next
// segment where one ends (segments are long: a tile rarely crosses one).
constexpr int GEN_TILE = 4096;
__global__ void gen_segments_kernel(const NrmGenSeg *segs, const int64_t *cum, int64_t count, int64_t total,
                                    void *arena) {
    for (int64_t t0 = (int64_t)blockIdx.x * GEN_TILE; t0 < total; t0 += (int64_t)gridDim.x * GEN_TILE) {
        int64_t lo = 0, hi = count; // last segment with cum <= t0
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(cum + mid) <= t0) lo = mid;
            else hi = mid;
        }
        const int64_t t1 = t0 + GEN_TILE < total ? t0 + GEN_TILE : total;
        int64_t seg = lo;
        int64_t base = __ldg(cum + seg);
        int64_t end = seg + 1 < count ? __ldg(cum + seg + 1) : total;
        NrmGenSeg sg = segs[seg];
        for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            while (e >= end) {
                ++seg;
                base = end;
                end = seg + 1 < count ? __ldg(cum + seg + 1) : total;
                sg = segs[seg];
            }
            const int64_t i = e - base;
            const uint64_t u = draw(sg.key, (uint64_t)i);
            if (sg.dtype == NRM_F64) ((double *)arena)[sg.start + i] = elem_d(u, sg.emin, (uint64_t)sg.span);
            else ((float *)arena)[sg.start + i] = elem_s(u, sg.emin, (uint64_t)sg.span);
        }
    }
}
} // namespace

nrm_status nrm_gen_segments(const NrmGenSeg *segs_dev, const int64_t *cum_dev, int64_t count, int64_t total,
                            void *arena, cudaStream_t s) {
    if (count <= 0 || total <= 0) return NRM_OK;
    const int64_t blocks = std::min<int64_t>((total + GEN_TILE - 1) / GEN_TILE, 152 * 8);
    gen_segments_kernel<<<(unsigned)blocks, 256, 0, s>>>(segs_dev, cum_dev, count, total, arena);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}
