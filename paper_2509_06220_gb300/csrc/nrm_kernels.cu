// nrm_kernels.cu -- the C ABI declared in include/nrm.h (arXiv 2509.06220):
// contexts and their workspace, argument checks, the single-vector,
// strided, matrix and batch entry points (the tree kernels themselves are in
// nrm_tree.cuh, instantiated per element type in nrm_tree_d.cu and
// nrm_tree_s.cu), and the elementwise test hooks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nrm.h"
#include "nrm_device.cuh"
#include "nrm_internal.h"

#include "nrm_tree.cuh"


using namespace nrm;

// context --------------------------------------------------------------------


// Grow the workspace to `bytes` and the ticket array to `tickets` counters.
// Tickets are zeroed when allocated and are returned to zero by every call
// (each node's second arriver resets its ticket), so they never need
// clearing between calls.  A captured graph holds the addresses of the
// buffers it was captured with, so while the context has graphs an outgrown
// buffer is retired (freed with the context) instead of freed.
static void release_buffer(nrm_ctx *c, void *p) {
    if (!p) return;
    if (c->graphs.empty()) cudaFree(p);
    else c->retired.push_back(p);
}

nrm_status nrm_ctx_ensure(nrm_ctx *c, size_t bytes, int64_t tickets) {
    if (bytes <= c->ws_bytes && tickets <= c->tickets_cap) return NRM_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return set_cuda_err(c, e, "cudaSetDevice");
    e = cudaDeviceSynchronize(); // the old buffers may still be in use
    if (e != cudaSuccess) return set_cuda_err(c, e, "cudaDeviceSynchronize");
    if (bytes > c->ws_bytes) {
        release_buffer(c, c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
        size_t want = std::max(bytes, (size_t)1 << 20);
        if (nrm_test_fail_alloc()) return NRM_ENOMEM;
        e = cudaMalloc(&c->ws, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->ws = nullptr;
            return set_cuda_err(c, e, "cudaMalloc(workspace)");
        }
        c->ws_bytes = want;
    }
    if (tickets > c->tickets_cap) {
        release_buffer(c, c->tickets);
        c->tickets = nullptr;
        c->tickets_cap = 0;
        int64_t want = std::max<int64_t>(tickets, 1 << 16);
        if (nrm_test_fail_alloc()) return NRM_ENOMEM;
        e = cudaMalloc(&c->tickets, (size_t)want * sizeof(unsigned));
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->tickets = nullptr;
            return set_cuda_err(c, e, "cudaMalloc(tickets)");
        }
        e = cudaMemset(c->tickets, 0, (size_t)want * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return set_cuda_err(c, e, "cudaMemset(tickets)");
        c->tickets_cap = want;
    }
    return NRM_OK;
}

extern "C" nrm_status nrm_create(nrm_ctx **ctx, int device) {
    if (!ctx) return NRM_EINVAL;
    *ctx = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return NRM_EDEVICE;
    }
    nrm_ctx *c = new nrm_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return NRM_EDEVICE;
    }
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    c->sms = prop.multiProcessorCount;
    // defaults from sweeps on GB300 at n = 2^28 with the item cursor (the
    // autotuner refines them per shape): items of 2^7 rows, 4 warps a block
    // (for one binary64 vector of 2^28, items of 2^8 rows are 3 % faster at
    // the 80-register cap, but they halve the items of a batch of shorter
    // vectors)
    c->tune[NRM_F32] = nrm_tuning{2, 4, 7, 16};
    c->tune[NRM_F64] = nrm_tuning{2, 4, 7, 8};
    nrm_status s = nrm_ctx_ensure(c, (size_t)4 << 20, 1 << 16);
    if (s != NRM_OK) {
        delete c;
        return s;
    }
    *ctx = c;
    return NRM_OK;
}

extern "C" nrm_status nrm_destroy(nrm_ctx *ctx) {
    if (!ctx) return NRM_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (nrm_graph *g : ctx->graphs) nrm_graph_free(g);
    ctx->graphs.clear();
    nrm_host_free(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->tickets) cudaFree(ctx->tickets);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->node_args) cudaFree(ctx->node_args);
    for (void *p : ctx->retired) cudaFree(p);
    delete ctx;
    return NRM_OK;
}

extern "C" const char *nrm_status_string(nrm_status s) {
    switch (s) {
    case NRM_OK: return "NRM_OK";
    case NRM_EINVAL: return "NRM_EINVAL";
    case NRM_ENOMEM: return "NRM_ENOMEM";
    case NRM_ECUDA: return "NRM_ECUDA";
    case NRM_ETIMEOUT: return "NRM_ETIMEOUT";
    case NRM_EBUDGET: return "NRM_EBUDGET";
    case NRM_EDEVICE: return "NRM_EDEVICE";
    default: return "NRM_UNKNOWN";
    }
}

extern "C" const char *nrm_last_error(const nrm_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

extern "C" nrm_status nrm_reserve(nrm_ctx *ctx, size_t bytes) {
    if (!ctx) return NRM_EINVAL;
    // slots need 1 KiB per ticket node: reserve tickets for what fits
    return nrm_ctx_ensure(ctx, bytes, (int64_t)(bytes / 1024) + 1);
}

static bool tuning_ok(const nrm_tuning *t) {
    if (t->group_log2 < 2 || t->group_log2 > 3) return false;
    if (t->warps_per_block != 4 && t->warps_per_block != 8 && t->warps_per_block != 16) return false;
    if (t->item_log2 < t->group_log2 || t->item_log2 > t->group_log2 + MAXL) return false;
    if (t->blocks_per_sm < 1 || t->blocks_per_sm > 16) return false;
    return true;
}

extern "C" nrm_status nrm_get_tuning(const nrm_ctx *ctx, nrm_tuning *t) {
    if (!ctx || !t) return NRM_EINVAL;
    *t = ctx->tune[NRM_F64];
    return NRM_OK;
}

extern "C" nrm_status nrm_set_tuning(nrm_ctx *ctx, const nrm_tuning *t) {
    if (!ctx || !t || !tuning_ok(t)) return NRM_EINVAL;
    ctx->tune[NRM_F32] = *t;
    ctx->tune[NRM_F64] = *t;
    return NRM_OK;
}

extern "C" nrm_status nrm_get_tuning_for(const nrm_ctx *ctx, nrm_dtype dtype, nrm_tuning *t) {
    if (!ctx || !t || (dtype != NRM_F32 && dtype != NRM_F64)) return NRM_EINVAL;
    *t = ctx->tune[dtype];
    return NRM_OK;
}

extern "C" nrm_status nrm_set_tuning_for(nrm_ctx *ctx, nrm_dtype dtype, const nrm_tuning *t) {
    if (!ctx || !t || (dtype != NRM_F32 && dtype != NRM_F64) || !tuning_ok(t)) return NRM_EINVAL;
    ctx->tune[dtype] = *t;
    return NRM_OK;
}

extern "C" uint64_t nrm_kernel_launches(const nrm_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" nrm_status nrm_test_read_tickets(const nrm_ctx *ctx, uint32_t *host, int64_t count) {
    if (!ctx || !host || count < 0 || count > ctx->tickets_cap) return NRM_EINVAL;
    cudaError_t e = cudaMemcpy(host, ctx->tickets, (size_t)count * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? NRM_OK : NRM_ECUDA;
}



nrm_status nrm_plan_single(const nrm_ctx *c, nrm_dtype dt, int64_t n, VecPlan *pl) {
    return plan_single(c, n, dt == NRM_F64 ? 64 : 128, *pl) ? NRM_OK : NRM_EINVAL;
}

nrm_status nrm_run_single_range(nrm_ctx *c, nrm_dtype dt, const void *x, int64_t n, double p, void *out,
                                cudaStream_t s, const VecPlan *pl, int64_t item_lo, int64_t item_hi) {
    if (dt == NRM_F64)
        return run_single_x(c, (const double *)x, n, p, (double *)out, s, item_lo, item_hi, pl);
    return run_single_x(c, (const float *)x, n, (float)p, (float *)out, s, item_lo, item_hi, pl);
}

template <typename T> static nrm_status check_args(nrm_ctx *c, const T *x, int64_t n, T p, T *out) {
    if (!c || !out || n < 0 || (n > 0 && !x)) return NRM_EINVAL;
    if (!(p > T(0))) return NRM_EINVAL; // also rejects NaN
    return NRM_OK;
}

template <typename T> static nrm_status nrm_entry(nrm_ctx *c, const T *x, int64_t n, T p, T *out, void *stream) {
    nrm_status st = check_args<T>(c, x, n, p, out);
    if (st != NRM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return set_cuda_err(c, cudaMemsetAsync(out, 0, sizeof(T), s), "cudaMemsetAsync");
    return run_single_x(c, x, n, p, out, s, 0, 0, nullptr);
}

extern "C" nrm_status nrmf_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream) {
    return nrm_entry<float>(ctx, x, n, 2.0f, out, stream);
}
extern "C" nrm_status nrmf_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream) {
    return nrm_entry<double>(ctx, x, n, 2.0, out, stream);
}
// Z with A for the final reduction (Section 3's recommended xNRMF)
template <typename T> static nrm_status za_entry(nrm_ctx *c, const T *x, int64_t n, T *out, void *stream) {
    nrm_status st = check_args<T>(c, x, n, T(2), out);
    if (st != NRM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return set_cuda_err(c, cudaMemsetAsync(out, 0, sizeof(T), s), "cudaMemsetAsync");
    return run_single_x(c, x, n, T(2), out, s, 0, 0, nullptr, 1, 1);
}

// xNRMF with the exponent-scaled hypotenuse K2 (a hypot[f] variant, Section 2)
template <typename T> static nrm_status es_entry(nrm_ctx *c, const T *x, int64_t n, T *out, void *stream) {
    nrm_status st = check_args<T>(c, x, n, T(2), out);
    if (st != NRM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return set_cuda_err(c, cudaMemsetAsync(out, 0, sizeof(T), s), "cudaMemsetAsync");
    return run_single_x(c, x, n, T(2), out, s, 0, 0, nullptr, 1, 2);
}

extern "C" nrm_status nrmf_es_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream) {
    return es_entry<float>(ctx, x, n, out, stream);
}
extern "C" nrm_status nrmf_es_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream) {
    return es_entry<double>(ctx, x, n, out, stream);
}

extern "C" nrm_status nrmf_za_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream) {
    return za_entry<float>(ctx, x, n, out, stream);
}
extern "C" nrm_status nrmf_za_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream) {
    return za_entry<double>(ctx, x, n, out, stream);
}

extern "C" nrm_status nrmp_s(nrm_ctx *ctx, const float *x, int64_t n, float p, float *out, void *stream) {
    return nrm_entry<float>(ctx, x, n, p, out, stream);
}
extern "C" nrm_status nrmp_d(nrm_ctx *ctx, const double *x, int64_t n, double p, double *out, void *stream) {
    return nrm_entry<double>(ctx, x, n, p, out, stream);
}

// strided vectors and matrices (Sections 3 and 3.1) ------------------------------

extern "C" nrm_status nrm_strided(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t n, int64_t incx, double p,
                                  void *out, void *stream) {
    if (!ctx || !out || n < 0 || (n > 0 && !x) || incx == 0 || (dtype != NRM_F32 && dtype != NRM_F64))
        return NRM_EINVAL;
    if (!(p > 0.0) || (dtype == NRM_F32 && !((float)p > 0.0f))) return NRM_EINVAL;
    const size_t es = dtype == NRM_F64 ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return set_cuda_err(ctx, cudaMemsetAsync(out, 0, es, s), "cudaMemsetAsync");
    const int64_t step = incx < 0 ? -incx : incx;
    if (n > 1 && step > INT64_MAX / (n - 1)) return NRM_EINVAL;
    // logical element i is x[i incx] (incx > 0) or x[(n-1-i) |incx|] (incx < 0)
    const char *first = (const char *)x + (incx < 0 ? (size_t)((n - 1) * step) * es : 0);
    if (dtype == NRM_F64)
        return run_single_x(ctx, (const double *)first, n, p, (double *)out, s, 0, 0, nullptr, incx);
    return run_single_x(ctx, (const float *)first, n, (float)p, (float *)out, s, 0, 0, nullptr, incx);
}

namespace {
__global__ void fill_columns_kernel(int64_t *starts, int64_t *lens, int64_t N, int64_t M, int64_t lda) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        starts[j] = j * lda;
        lens[j] = M;
    }
}
} // namespace

extern "C" nrm_status nrm_matrix(nrm_ctx *ctx, nrm_dtype dtype, const void *A, int64_t M, int64_t N, int64_t lda,
                                 double p, void *out, void *stream) {
    if (!ctx || !out || M < 0 || N < 0 || lda < (M > 1 ? M : 1) || (dtype != NRM_F32 && dtype != NRM_F64))
        return NRM_EINVAL;
    if (M > 0 && N > 0 && !A) return NRM_EINVAL;
    if (!(p > 0.0) || (dtype == NRM_F32 && !((float)p > 0.0f))) return NRM_EINVAL;
    if (N > 1 && lda > INT64_MAX / N) return NRM_EINVAL;
    const size_t es = dtype == NRM_F64 ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    if (M == 0 || N == 0) return set_cuda_err(ctx, cudaMemsetAsync(out, 0, es, s), "cudaMemsetAsync");
    // contiguous storage: the array is one vector of M N elements (Section 3.1)
    if (lda == M || N == 1) return nrm_run_single_range(ctx, dtype, A, M * N, p, out, s, nullptr, 0, 0);
    // otherwise: the norm of every column, then the norm of the N column norms
    const size_t need = (size_t)N * (16 + es) + 512;
    if (need > ctx->aux_bytes) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_cuda_err(ctx, e, "cudaStreamSynchronize");
        if (ctx->aux) cudaFree(ctx->aux);
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
        if (nrm_test_fail_alloc()) return NRM_ENOMEM;
        e = cudaMalloc(&ctx->aux, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_cuda_err(ctx, e, "cudaMalloc(aux)");
        }
        ctx->aux_bytes = need;
    }
    int64_t *starts = (int64_t *)ctx->aux;
    int64_t *lens = starts + N;
    void *colnorm = (void *)(((uintptr_t)(lens + N) + 255) & ~(uintptr_t)255);
    const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 1024);
    fill_columns_kernel<<<blocks, 256, 0, s>>>(starts, lens, N, M, lda);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_err(ctx, e, "fill_columns_kernel");
    nrm_status st = nrm_batch_impl(ctx, dtype, A, (N - 1) * lda + M, starts, N, p, nullptr, colnorm, nullptr, s, lens);
    if (st != NRM_OK) return st;
    return nrm_run_single_range(ctx, dtype, colnorm, N, p, out, s, nullptr, 0, 0);
}

// batch -----------------------------------------------------------------------


int64_t nrm_batch_tickets(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B, bool per_vector_p) {
    return batch_nodes_bound(c, x_len, B, dt == NRM_F64 ? 64 : 128, per_vector_p);
}

size_t nrm_batch_ws_bytes(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B, bool per_vector_p) {
    const int P = dt == NRM_F64 ? 64 : 128;
    return layout_for(batch_nodes_bound(c, x_len, B, P, per_vector_p), B).end;
}

extern "C" size_t nrm_workspace_bytes(const nrm_ctx *ctx, nrm_dtype dtype, int64_t x_len, int64_t B) {
    if (!ctx) return 0;
    if (B <= 1) {
        VecPlan pl;
        if (!plan_single(ctx, std::max<int64_t>(x_len, 1), dtype == NRM_F64 ? 64 : 128, pl)) return 0;
        return layout_for((int64_t(1) << pl.dw) - 1, 1).end;
    }
    return nrm_batch_ws_bytes(ctx, dtype, x_len, B);
}


nrm_status nrm_batch_impl(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *offsets,
                          int64_t B, double p, const double *p_dev, void *out, int32_t *status, cudaStream_t s,
                          const int64_t *lens) {
    if (!ctx || B < 0 || x_len < 0 || (dtype != NRM_F32 && dtype != NRM_F64)) return NRM_EINVAL;
    if (B > 0 && (!offsets || !out)) return NRM_EINVAL;
    if (x_len > 0 && !x) return NRM_EINVAL;
    if (!p_dev && !(p > 0.0)) return NRM_EINVAL; // with p_dev, p is ignored and checked per vector
    if (B == 0) return NRM_OK;
    if (dtype == NRM_F64)
        return run_batch_x(ctx, (const double *)x, x_len, offsets, lens, B, p_dev ? 2.0 : p, p_dev,
                                 (double *)out, status, s);
    const float pf = p_dev ? 2.0f : (float)p;
    if (!(pf > 0.0f)) return NRM_EINVAL;
    return run_batch_x(ctx, (const float *)x, x_len, offsets, lens, B, pf, p_dev, (float *)out, status, s);
}

// sharding across devices (Section 2, Eq. hr) ----------------------------------
//
// Norms of disjoint parts combine by one more combine, so a vector split at
// the nodes of depth dg of its canonical row tree (rank j holds node j's
// rows) gives, node by node, the lane partials of those subtrees; combining
// the 2^dg lane vectors through the tree's top dg levels and reducing the
// lanes reproduces the one-device result bit for bit.

extern "C" nrm_status nrm_shard_range(nrm_dtype dtype, int64_t n, int32_t dg, int64_t j, int64_t *first,
                                      int64_t *count) {
    if ((dtype != NRM_F32 && dtype != NRM_F64) || n < 0 || dg < 0 || dg > NRM_SHARD_MAX_DEPTH || j < 0 ||
        j >= (int64_t(1) << dg) || !first || !count)
        return NRM_EINVAL;
    const int64_t P = dtype == NRM_F64 ? 64 : 128;
    const int64_t m = (n + P - 1) / P;
    // node j at depth dg of the ceil-split tree over m rows: rows
    // ceil((m - brev_dg(j)) / 2^dg) (zero when brev_dg(j) >= m), first row
    // from the walk down from the root (left child: ceil of half the rows)
    uint32_t b = 0;
    for (int l = 0; l < dg; ++l) b |= (uint32_t)((j >> l) & 1) << (dg - 1 - l);
    const int64_t rows = (int64_t)b >= m ? 0 : ((m - (int64_t)b) + (int64_t(1) << dg) - 1) >> dg;
    int64_t start = 0, size = m;
    for (int l = dg - 1; l >= 0; --l) {
        const int64_t left = (size + 1) >> 1;
        if ((j >> l) & 1) {
            start += left;
            size -= left;
        } else {
            size = left;
        }
    }
    *first = std::min(start * P, n);
    *count = rows == 0 ? 0 : std::min(rows * P, n - start * P);
    return NRM_OK;
}

namespace {
__global__ void node_args_kernel(int64_t *off, double *pd, int64_t n, double p) {
    off[0] = 0;
    off[1] = n;
    pd[0] = p;
}

// One warp: node (d - 1, i) = combine(node (d, 2i), node (d, 2i + 1)) for
// d = dg .. 1, in place (pair i overwrites slot i after reading 2i and
// 2i + 1, in increasing i, so nothing is read after it was overwritten); a
// node without rows passes its sibling through.  Each thread touches only its
// own V lanes of every node, so no synchronisation is needed.  Then R over
// the lanes of the root.
template <typename T, class Op>
__global__ void combine_nodes_kernel(T *lanes, int dg, int64_t m, Op op, T *out) {
    constexpr int V = Geo<T>::V;
    constexpr int P = Geo<T>::P;
    const int lane = threadIdx.x & 31;
    for (int d = dg; d >= 1; --d) {
        for (uint32_t i = 0; i < (1u << (d - 1)); ++i) {
            const bool a = node_rows(m, 2 * i, d) > 0, b = node_rows(m, 2 * i + 1, d) > 0;
            T *dst = lanes + (size_t)i * P + lane * V;
            const T *l = lanes + (size_t)(2 * i) * P + lane * V;
            const T *r = lanes + (size_t)(2 * i + 1) * P + lane * V;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const T x = l[j], y = r[j];
                dst[j] = (a && b) ? op(x, y) : (a ? x : y);
            }
        }
    }
    T r[V];
#pragma unroll
    for (int j = 0; j < V; ++j) r[j] = lanes[lane * V + j];
    const T res = lane_reduce<T, Op>(r, op, lane);
    if (lane == 0) *out = res;
}
} // namespace

extern "C" nrm_status nrm_node_lanes(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t count, double p,
                                     void *lanes, void *stream) {
    if (!ctx || !lanes || count < 0 || (count > 0 && !x) || (dtype != NRM_F32 && dtype != NRM_F64) || !(p > 0.0) ||
        (dtype == NRM_F32 && !((float)p > 0.0f)))
        return NRM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dtype == NRM_F64 ? 8 : 4;
    if (count == 0) return set_cuda_err(ctx, cudaMemsetAsync(lanes, 0, 512, s), "cudaMemsetAsync(lanes)");
    if (!ctx->node_args) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_cuda_err(ctx, e, "cudaStreamSynchronize");
        if (nrm_test_fail_alloc()) return NRM_ENOMEM;
        e = cudaMalloc(&ctx->node_args, 256);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->node_args = nullptr;
            return set_cuda_err(ctx, e, "cudaMalloc(node_args)");
        }
    }
    int64_t *off = (int64_t *)ctx->node_args;
    double *pd = (double *)((char *)ctx->node_args + 64);
    void *one = (char *)ctx->node_args + 128;
    node_args_kernel<<<1, 1, 0, s>>>(off, pd, count, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_err(ctx, e, "node_args_kernel");
    (void)es;
    if (dtype == NRM_F64)
        return run_batch_x(ctx, (const double *)x, count, off, nullptr, 1, 2.0, pd, (double *)one, nullptr, s,
                           (double *)lanes);
    return run_batch_x(ctx, (const float *)x, count, off, nullptr, 1, 2.0f, pd, (float *)one, nullptr, s,
                       (float *)lanes);
}

extern "C" nrm_status nrm_combine_nodes(nrm_ctx *ctx, nrm_dtype dtype, void *lanes, int32_t dg, int64_t n, double p,
                                        void *out, void *stream) {
    if (!ctx || !lanes || !out || n < 0 || dg < 0 || dg > NRM_SHARD_MAX_DEPTH ||
        (dtype != NRM_F32 && dtype != NRM_F64) || !(p > 0.0) || (dtype == NRM_F32 && !((float)p > 0.0f)))
        return NRM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t P = dtype == NRM_F64 ? 64 : 128;
    if (n == 0) return set_cuda_err(ctx, cudaMemsetAsync(out, 0, dtype == NRM_F64 ? 8 : 4, s), "cudaMemsetAsync");
    const int64_t m = (n + P - 1) / P;
    cudaError_t e;
    if (dtype == NRM_F64)
        e = with_op<double>(p, [&](auto op) {
            combine_nodes_kernel<double><<<1, 32, 0, s>>>((double *)lanes, dg, m, op, (double *)out);
            return cudaGetLastError();
        });
    else
        e = with_op<float>((float)p, [&](auto op) {
            combine_nodes_kernel<float><<<1, 32, 0, s>>>((float *)lanes, dg, m, op, (float *)out);
            return cudaGetLastError();
        });
    return set_cuda_err(ctx, e, "combine_nodes_kernel");
}

extern "C" nrm_status nrm_batch_segments(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len,
                                         const int64_t *starts, const int64_t *lengths, int64_t B, double p,
                                         const double *p_dev, void *out, int32_t *status, void *stream) {
    if (B > 0 && !lengths) return NRM_EINVAL;
    return nrm_batch_impl(ctx, dtype, x, x_len, starts, B, p, p_dev, out, status, (cudaStream_t)stream, lengths);
}

extern "C" nrm_status nrm_batch(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len,
                                const int64_t *offsets, int64_t B, double p, const double *p_dev, void *out,
                                int32_t *status, void *stream) {
    return nrm_batch_impl(ctx, dtype, x, x_len, offsets, B, p, p_dev, out, status, (cudaStream_t)stream);
}


// ---------------------------------------------------------------------------
// test hook: k1_exact (binary64 v1_hypot without the FP64 pipe) against the
// FP64 k1 on generated operand pairs; counts bitwise differences
// (two NaNs count as equal).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint64_t th_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double th_make(uint64_t sign, int64_t biased_exp, uint64_t frac) {
    return __longlong_as_double((long long)((sign << 63) | ((uint64_t)biased_exp << 52) | (frac & 0x000fffffffffffffull)));
}

__device__ __forceinline__ uint64_t th_frac(uint64_t u, int kind) {
    switch (kind & 7) {
    case 0: return 0;
    case 1: return 0x000fffffffffffffull;
    case 2: return 1;
    case 3: return 1ull << 51;
    case 4: return u | 0xfffffull;          // low bits all ones
    case 5: return u & ~0xfffffull;         // low bits all zeros
    case 6: return 0x000fffffffffffffull - (u & 0xff);
    default: return u;
    }
}

// operand pair i of family `mode` for the compare tests (see
// nrm_test_k1d_compare in include/nrm.h for the families)
__device__ __forceinline__ void k1d_pair(uint64_t seed, int64_t i, int mode, double &x, double &y) {
    const uint64_t u1 = th_mix(seed + (uint64_t)(4 * i + 1) * 0x9E3779B97F4A7C15ull);
    const uint64_t u2 = th_mix(seed + (uint64_t)(4 * i + 2) * 0x9E3779B97F4A7C15ull);
    const uint64_t u3 = th_mix(seed + (uint64_t)(4 * i + 3) * 0x9E3779B97F4A7C15ull);
    const int64_t e1 = 1023 - 40 + (int64_t)(u3 % 81);
    switch (mode) {
    case 0: { // moderate: exponent gap 0..32
        const int64_t dd = (int64_t)((u3 >> 20) % 33);
        x = th_make(u1 >> 63, e1, u1);
        y = th_make(u2 >> 63, e1 - dd, u2);
        break;
    }
    case 1: { // close values: gap -1, 0, +1
        const int64_t dd = (int64_t)((u3 >> 20) % 3) - 1;
        x = th_make(u1 >> 63, e1, u1);
        y = th_make(u2 >> 63, e1 + dd, ((u3 >> 30) & 1) ? (u1 + ((u2 >> 40) - (1ull << 23))) : u2);
        break;
    }
    case 2: { // edge significands, gap 0..30
        const int64_t dd = (int64_t)((u3 >> 20) % 31);
        x = th_make(u1 >> 63, e1, th_frac(u1, (int)(u3 >> 40)));
        y = th_make(u2 >> 63, e1 - dd, th_frac(u2, (int)(u3 >> 44)));
        break;
    }
    case 3: // raw bit patterns: every class (inf, NaN, subnormal, zero, extremes)
        x = __longlong_as_double((long long)u1);
        y = __longlong_as_double((long long)(((u3 >> 10) & 1) ? u2 : (u1 ^ (u2 & 0xffffull))));
        break;
    case 4: { // extremes: near the largest and the smallest normal exponent
        const int64_t ex = ((u3 >> 9) & 1) ? 2046 - (int64_t)((u3 >> 12) % 4) : 1 + (int64_t)((u3 >> 12) % 4);
        const int64_t dd = (int64_t)((u3 >> 20) % 31);
        x = th_make(0, ex, u1);
        y = th_make(0, ex - dd > 0 ? ex - dd : 0, u2);
        break;
    }
    case 5: { // gaps around the S = 1 shortcut
        const int64_t dd = 25 + (int64_t)((u3 >> 20) % 5);
        x = th_make(0, e1, th_frac(u1, (int)(u3 >> 40)));
        y = th_make(0, e1 - dd, th_frac(u2, (int)(u3 >> 44)));
        break;
    }
    default: { // equal or nearly equal values (S near 2)
        x = th_make(0, e1, u1);
        y = th_make(0, e1, u1 - (u2 & 0x3ff) + ((u2 >> 12) & 0x3ff));
        break;
    }
    }
}

// mode 0..6: k1_exact on family `mode`; mode 8..14: k1_exact_fast on family
// mode - 8, for the pairs inside its range [2^-500, 2^502) (others skipped)
__device__ __forceinline__ bool in_fast_range(double x, double y) {
    const uint32_t hx = (uint32_t)((uint64_t)__double_as_longlong(x) >> 32) & 0x7fffffffu;
    const uint32_t hy = (uint32_t)((uint64_t)__double_as_longlong(y) >> 32) & 0x7fffffffu;
    const uint32_t lo = (uint32_t)(1023 - 500) << 20, hi = (uint32_t)(1023 + 502) << 20;
    return hx >= lo && hx < hi && hy >= lo && hy < hi;
}
__global__ void k1d_compare_kernel(uint64_t seed, int64_t n, int mode, unsigned long long *bad, double *example) {
    const bool pair = mode >= 16;
    const bool fast = mode >= 8;
    const int fam = mode & 7;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x, y;
        k1d_pair(seed, i, fam, x, y);
        if (fast && !in_fast_range(x, y)) continue;
        if (pair) {
            // the paired form on pair i and a second pair of the family,
            // against the FP64 form of each
            double x2, y2, a, a2;
            k1d_pair(seed ^ 0x5bd1e9955bd1e995ull, i, fam, x2, y2);
            if (!in_fast_range(x2, y2)) continue;
            k1_exact_fast2(x, y, x2, y2, a, a2);
            const double b = k1(x, y), b2 = k1(x2, y2);
            const bool same = __double_as_longlong(a) == __double_as_longlong(b) &&
                              __double_as_longlong(a2) == __double_as_longlong(b2);
            if (!same && atomicAdd(bad, 1ull) == 0ull) {
                example[0] = x;
                example[1] = y;
                example[2] = a;
                example[3] = b;
            }
            continue;
        }
        const double a = fast ? k1_exact_fast(x, y) : k1_exact(x, y), b = k1(x, y);
        const bool same = (__double_as_longlong(a) == __double_as_longlong(b)) || (isnan(a) && isnan(b));
        if (!same) {
            if (atomicAdd(bad, 1ull) == 0ull) {
                example[0] = x;
                example[1] = y;
                example[2] = a;
                example[3] = b;
            }
        }
    }
}

} // namespace

// Elementwise pow and v1_lp of the tree kernels, for parity tests against
// the oracle on chosen operands.
template <typename T> __global__ void pow_eval_kernel(const T *x, const T *y, T *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = pw(x[i], y[i]);
}
__global__ void powr_eval_kernel(const double *x, const double *y, double *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = powr_d(x[i], y[i]);
}
template <typename T> __global__ void lp_eval_kernel(OpLp<T> op, const T *x, const T *y, T *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = op(x[i], y[i]);
}

extern "C" nrm_status nrm_test_pow(nrm_dtype dtype, const void *x, const void *y, void *out, int64_t n,
                                   void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out)) || (dtype != NRM_F64 && dtype != NRM_F32)) return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == NRM_F64)
        pow_eval_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>((const double *)x, (const double *)y,
                                                                        (double *)out, n);
    else
        pow_eval_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>((const float *)x, (const float *)y,
                                                                       (float *)out, n);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

template <typename T, class Op> __global__ void combine_eval_kernel(Op op, const T *x, const T *y, T *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = op(x[i], y[i]);
}

extern "C" nrm_status nrm_test_combine(nrm_dtype dtype, double p, const void *x, const void *y, void *out, int64_t n,
                                       void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out)) || !(p > 0.0) || (dtype != NRM_F64 && dtype != NRM_F32))
        return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    cudaError_t e;
    if (dtype == NRM_F64)
        e = with_op<double>(p, [&](auto op) {
            combine_eval_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(op, (const double *)x,
                                                                             (const double *)y, (double *)out, n);
            return cudaGetLastError();
        });
    else
        e = with_op<float>((float)p, [&](auto op) {
            combine_eval_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(op, (const float *)x,
                                                                            (const float *)y, (float *)out, n);
            return cudaGetLastError();
        });
    return e == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

template <typename T> __global__ void k2_eval_kernel(const T *x, const T *y, T *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = k2(x[i], y[i]);
}

extern "C" nrm_status nrm_test_k2(nrm_dtype dtype, const void *x, const void *y, void *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out)) || (dtype != NRM_F64 && dtype != NRM_F32)) return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == NRM_F64)
        k2_eval_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>((const double *)x, (const double *)y,
                                                                      (double *)out, n);
    else
        k2_eval_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>((const float *)x, (const float *)y,
                                                                     (float *)out, n);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

extern "C" nrm_status nrm_test_powr(const double *x, const double *y, double *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out))) return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    powr_eval_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(x, y, out, n);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

extern "C" nrm_status nrm_test_lp(nrm_dtype dtype, double p, const void *x, const void *y, void *out, int64_t n,
                                  void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out)) || !(p > 0.0) || (dtype != NRM_F64 && dtype != NRM_F32))
        return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == NRM_F64) {
        OpLp<double> op;
        op.set(p * 0.5, 1.0 / p);
        lp_eval_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(op, (const double *)x, (const double *)y,
                                                                       (double *)out, n);
    } else {
        OpLp<float> op;
        const float pf = (float)p;
        op.set(pf * 0.5f, 1.0f / pf);
        lp_eval_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(op, (const float *)x, (const float *)y,
                                                                      (float *)out, n);
    }
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

// Exhaustive checks of k1f_fast's steps against the correctly rounded
// operations.  mode 0: sqrtf_fast(S) == RN(sqrt(S)) for the 2^23 + 1 values
// S in [1, 2] (index i: S = 1 + i 2^-23).  mode 1: the FP32 reciprocal
// estimate scales exactly with the exponent: for significand index i and
// exponent e in [-88, 124], bits(rcp(M 2^e)) = bits(rcp(M)) - e 2^23.
// mode 2: divf_fast(a, b) == RN(a/b) for the significand pairs a, b in
// [1, 2) (index i: a = 1 + (i >> 23) 2^-23, b = 1 + (i & (2^23-1)) 2^-23).
// Indices [start, start + count) of the mode's range; mismatches are added
// to *bad and the last one's operands stored in example[0..1].
__global__ void k1f_exhaustive_kernel(int mode, uint64_t start, uint64_t count, unsigned long long *bad,
                                      float *example) {
    unsigned long long nb = 0;
    float ex0 = 0.0f, ex1 = 0.0f;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = start + t;
        if (mode == 0 || mode == 3) {
            if (i > (mode == 0 ? (1ull << 23) : 3 * (1ull << 23) - 1)) continue;
            const float S = __uint_as_float(0x3f800000u + (uint32_t)i);
            if (__float_as_uint(sqrtf_fast(S)) != __float_as_uint(__fsqrt_rn(S))) {
                ++nb;
                ex0 = S;
            }
        } else if (mode == 1) {
            const uint32_t f = (uint32_t)(i & 0x7fffffu);
            const int e = (int)(i >> 23) - 88;
            if (e > 124) continue;
            const float M0 = __uint_as_float(0x3f800000u | f);
            const float Me = __uint_as_float((uint32_t)(127 + e) << 23 | f);
            const int b0 = (int)__float_as_uint(rcp_approx(M0));
            const int be = (int)__float_as_uint(rcp_approx(Me));
            if (be != b0 - e * (1 << 23)) {
                ++nb;
                ex0 = Me;
            }
        } else {
            if (i >= (1ull << 46)) continue;
            const float a = __uint_as_float(0x3f800000u | (uint32_t)(i >> 23));
            const float b = __uint_as_float(0x3f800000u | (uint32_t)(i & 0x7fffffu));
            if (__float_as_uint(divf_fast(a, b)) != __float_as_uint(__fdiv_rn(a, b))) {
                ++nb;
                ex0 = a;
                ex1 = b;
            }
        }
    }
    if (nb) {
        atomicAdd(bad, nb);
        example[0] = ex0;
        example[1] = ex1;
    }
}

extern "C" nrm_status nrm_test_k1f_exhaustive(int32_t mode, uint64_t start, uint64_t count, unsigned long long *bad,
                                              float *example, void *stream) {
    if (mode < 0 || mode > 3 || !bad || !example) return NRM_EINVAL;
    if (count == 0) return NRM_OK;
    k1f_exhaustive_kernel<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(mode, start, count, bad, example);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

// k2_exact_fast against k2 (FP64 square root) on the k1d_compare families,
// for pairs inside the fast form's range [2^-500, 2^502) (others skipped).
__global__ void k2d_compare_kernel(uint64_t seed, int64_t n, int mode, unsigned long long *bad, double *example) {
    unsigned long long nb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x, y;
        k1d_pair(seed, i, mode, x, y);
        const uint32_t hx = (uint32_t)((uint64_t)__double_as_longlong(x) >> 32) & 0x7fffffffu;
        const uint32_t hy = (uint32_t)((uint64_t)__double_as_longlong(y) >> 32) & 0x7fffffffu;
        const uint32_t lo = (uint32_t)(1023 - 500) << 20, hi = (uint32_t)(1023 + 502) << 20;
        if (hx < lo || hx >= hi || hy < lo || hy >= hi) continue;
        const double a = k2_exact_fast(x, y), b = k2(x, y);
        if (__double_as_longlong(a) != __double_as_longlong(b)) {
            ++nb;
            example[0] = x;
            example[1] = y;
            example[2] = a;
            example[3] = b;
        }
    }
    if (nb) atomicAdd(bad, nb);
}

extern "C" nrm_status nrm_test_k2d_compare(uint64_t seed, int64_t n, int32_t mode, unsigned long long *bad,
                                           double *example, void *stream) {
    if (n < 0 || !bad || !example || mode < 0 || mode > 6) return NRM_EINVAL;
    k2d_compare_kernel<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(seed, n, mode, bad, example);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}

extern "C" nrm_status nrm_test_k1d_compare(uint64_t seed, int64_t n, int32_t mode, unsigned long long *bad,
                                           double *example, void *stream) {
    if (n < 0 || !bad || !example || mode < 0 || mode > 22 || (mode & 7) == 7) return NRM_EINVAL;
    k1d_compare_kernel<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(seed, n, mode, bad, example);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}
