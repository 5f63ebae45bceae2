// nrm_runtime.cu -- host runtime around the tree kernels: CUDA-graph capture
// of the ragged batch, the end-to-end call on host buffers (chunked copies
// overlapped with the tree computation), and the host-side fault hook.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "../../include/nrm.h"
#include "nrm_device.cuh"
#include "nrm_internal.h"

using nrm::VecPlan;

// --- host-side fault injection (tests only): the next `count` workspace
// allocations report NRM_ENOMEM without calling cudaMalloc. -----------------
static std::atomic<int> g_fail_alloc{0};

extern "C" void nrm_test_inject_alloc_failures(int count) { g_fail_alloc.store(count < 0 ? 0 : count); }

bool nrm_test_fail_alloc() {
    int v = g_fail_alloc.load();
    while (v > 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return true;
    }
    return false;
}

// --- graphs ---------------------------------------------------------------
void nrm_graph_free(nrm_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

extern "C" nrm_status nrm_batch_graph(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len,
                                      const int64_t *offsets, int64_t B, double p, const double *p_dev, void *out,
                                      int32_t *status, nrm_graph **graph) {
    if (!ctx || !graph) return NRM_EINVAL;
    *graph = nullptr;
    if (B <= 0 || !offsets || !out || x_len < 0 || (x_len > 0 && !x) || (!p_dev && !(p > 0.0)) ||
        (dtype != NRM_F32 && dtype != NRM_F64))
        return NRM_EINVAL;
    nrm_status st = nrm_ctx_ensure(ctx, nrm_batch_ws_bytes(ctx, dtype, x_len, B, p_dev != nullptr),
                                   nrm_batch_tickets(ctx, dtype, x_len, B, p_dev != nullptr));
    if (st != NRM_OK) return st;
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        ctx->err = cudaGetErrorString(e);
        return NRM_ECUDA;
    }
    nrm_graph *g = new nrm_graph{ctx, nullptr, nullptr};
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = nrm_batch_impl(ctx, dtype, x, x_len, offsets, B, p, p_dev, out, status, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
        if (st == NRM_OK && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && st == NRM_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(s);
    if (st != NRM_OK || e != cudaSuccess) {
        if (e != cudaSuccess) ctx->err = std::string("graph capture: ") + cudaGetErrorString(e);
        nrm_graph_free(g);
        return st != NRM_OK ? st : NRM_ECUDA;
    }
    ctx->graphs.push_back(g);
    *graph = g;
    return NRM_OK;
}

extern "C" nrm_status nrm_graph_launch(nrm_graph *graph, void *stream) {
    if (!graph || !graph->exec) return NRM_EINVAL;
    cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        graph->ctx->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
        return NRM_ECUDA;
    }
    graph->ctx->launches += 2;
    return NRM_OK;
}

extern "C" nrm_status nrm_graph_destroy(nrm_graph *graph) {
    if (!graph) return NRM_OK;
    nrm_ctx *c = graph->ctx;
    auto it = std::find(c->graphs.begin(), c->graphs.end(), graph);
    if (it != c->graphs.end()) c->graphs.erase(it);
    nrm_graph_free(graph);
    return NRM_OK;
}

// --- end-to-end call on host buffers -----------------------------------------
void nrm_host_free(nrm_ctx *c) {
    if (c->stage) cudaFree(c->stage);
    if (c->out_dev) cudaFree(c->out_dev);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    for (cudaStream_t &cs : c->s_copy) {
        if (cs) cudaStreamDestroy(cs);
        cs = nullptr;
    }
    if (c->s_comp) cudaStreamDestroy(c->s_comp);
    c->stage = nullptr;
    c->out_dev = nullptr;
    c->s_comp = nullptr;
    c->stage_bytes = 0;
}

// first row of work item i at depth dw of the row tree over m rows (the same
// root-to-node walk the kernel does)
static int64_t host_node_start(int64_t m, uint32_t j, int d) {
    int64_t start = 0, size = m;
    for (int l = d - 1; l >= 0; --l) {
        const int64_t left = (size + 1) >> 1;
        if ((j >> l) & 1u) {
            start += left;
            size -= left;
        } else {
            size = left;
        }
    }
    return start;
}

// host->device copies go in kChunks pieces; each piece's work items start
// as soon as that piece has arrived.  (More copy streams gave no more
// bandwidth on GB300: pinned H2D measured ~210 GB/s with 1 to 8 streams.)
static const int kChunks = 8;
static const int kCopyStreams = 1;

extern "C" nrm_status nrm_host(nrm_ctx *ctx, nrm_dtype dtype, const void *x_host, int64_t n, double p,
                               void *out_host) {
    if (!ctx || !out_host || n < 0 || (n > 0 && !x_host) || (dtype != NRM_F32 && dtype != NRM_F64))
        return NRM_EINVAL;
    if (!(p > 0.0) || (dtype == NRM_F32 && !((float)p > 0.0f))) return NRM_EINVAL;
    const size_t es = dtype == NRM_F64 ? 8 : 4;
    const int P = dtype == NRM_F64 ? 64 : 128;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return NRM_ECUDA;
    if (!ctx->s_comp) {
        for (int i = 0; i < kCopyStreams; ++i) cudaStreamCreateWithFlags(&ctx->s_copy[i], cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking);
        ctx->ev.resize(kChunks);
        for (auto &ev : ctx->ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (cudaMalloc(&ctx->out_dev, 16) != cudaSuccess) {
            cudaGetLastError();
            return NRM_ENOMEM;
        }
    }
    if (n == 0) {
        memset(out_host, 0, es);
        return NRM_OK;
    }
    const size_t need = (size_t)n * es;
    if (need > ctx->stage_bytes) {
        if (ctx->stage) {
            cudaDeviceSynchronize();
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        if (nrm_test_fail_alloc()) return NRM_ENOMEM;
        e = cudaMalloc(&ctx->stage, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->err = "cudaMalloc(stage): " + std::string(cudaGetErrorString(e));
            return NRM_ENOMEM;
        }
        ctx->stage_bytes = need;
    }
    VecPlan pl;
    nrm_status st = nrm_plan_single(ctx, dtype, n, &pl);
    if (st != NRM_OK) return st;
    // make sure the workspace exists before queueing anything
    st = nrm_ctx_ensure(ctx, nrm_workspace_bytes(ctx, dtype, n, 1), (int64_t(1) << pl.dw));
    if (st != NRM_OK) return st;
    const int64_t items = int64_t(1) << pl.dw;
    const int64_t chunks = std::min<int64_t>(kChunks, items);
    for (int64_t c = 0; c < chunks; ++c) {
        const int64_t i0 = items * c / chunks, i1 = items * (c + 1) / chunks;
        const int64_t r0 = host_node_start(pl.m, (uint32_t)i0, pl.dw);
        const int64_t r1 = (i1 == items) ? pl.m : host_node_start(pl.m, (uint32_t)i1, pl.dw);
        const int64_t e0 = r0 * P, e1 = std::min<int64_t>(n, r1 * P);
        cudaStream_t cs = ctx->s_copy[c % kCopyStreams];
        e = cudaMemcpyAsync((char *)ctx->stage + e0 * es, (const char *)x_host + e0 * es, (size_t)(e1 - e0) * es,
                            cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) break;
        cudaEventRecord(ctx->ev[c], cs);
        cudaStreamWaitEvent(ctx->s_comp, ctx->ev[c], 0);
        st = nrm_run_single_range(ctx, dtype, ctx->stage, n, p, ctx->out_dev, ctx->s_comp, &pl, i0, i1);
        if (st != NRM_OK) break;
    }
    if (e == cudaSuccess && st == NRM_OK)
        e = cudaMemcpyAsync(out_host, ctx->out_dev, es, cudaMemcpyDeviceToHost, ctx->s_comp);
    cudaError_t e2 = cudaStreamSynchronize(ctx->s_comp);
    for (cudaStream_t cs : ctx->s_copy) cudaStreamSynchronize(cs);
    if (st != NRM_OK) return st;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        ctx->err = std::string("nrm_host: ") + cudaGetErrorString(e);
        return NRM_ECUDA;
    }
    return NRM_OK;
}

// --- autotuner -------------------------------------------------------------
// Times every tuning candidate on a synthetic problem of the caller's shape
// and keeps the fastest for that element type.  Candidates only change how
// the fixed tree is mapped onto warps, never a result bit.
extern "C" nrm_status nrm_autotune(nrm_ctx *ctx, nrm_dtype dtype, const int64_t *lengths_host, int64_t B,
                                   nrm_tuning *best_out) {
    if (!ctx || !lengths_host || B < 1 || (dtype != NRM_F32 && dtype != NRM_F64)) return NRM_EINVAL;
    std::vector<int64_t> off((size_t)B + 1, 0);
    for (int64_t i = 0; i < B; ++i) {
        if (lengths_host[i] < 0) return NRM_EINVAL;
        off[(size_t)i + 1] = off[(size_t)i] + lengths_host[i];
    }
    const int64_t total = off[(size_t)B];
    const size_t es = dtype == NRM_F64 ? 8 : 4;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NRM_ECUDA;
    void *x = nullptr, *out = nullptr;
    int64_t *offd = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    nrm_status st = NRM_OK;
    if (cudaMalloc(&x, (size_t)std::max<int64_t>(total, 1) * es) != cudaSuccess ||
        cudaMalloc(&out, (size_t)B * es) != cudaSuccess ||
        cudaMalloc((void **)&offd, (size_t)(B + 1) * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        st = NRM_ENOMEM;
    }
    if (st == NRM_OK) {
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaMemcpyAsync(offd, off.data(), (size_t)(B + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        st = nrm_gen_ragged(dtype, x, total, offd, B, 0x5eedull, -20, 20, s);
    }
    const nrm_tuning saved = ctx->tune[dtype];
    nrm_tuning best = saved;
    float best_ms = 1e30f;
    auto run = [&](void) -> nrm_status {
        if (B == 1) return nrm_run_single_range(ctx, dtype, x, total, 2.0, out, s, nullptr, 0, 0);
        return nrm_batch_impl(ctx, dtype, x, total, offd, B, 2.0, nullptr, out, nullptr, s);
    };
    for (int G = 2; G <= 3 && st == NRM_OK; ++G)
        for (int wpb : {4, 8, 16})
            for (int k = G + 2; k <= G + 7 && st == NRM_OK; ++k)
                for (int bps : {2, 4, 8, 16}) {
                    ctx->tune[dtype] = nrm_tuning{G, wpb, k, bps};
                    if (total == 0) break;
                    st = run(); // warm-up (and workspace growth)
                    if (st != NRM_OK) break;
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < 3 && st == NRM_OK; ++r) st = run();
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) st = NRM_ECUDA;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (st == NRM_OK && ms < best_ms) {
                        best_ms = ms;
                        best = ctx->tune[dtype];
                    }
                }
    ctx->tune[dtype] = (st == NRM_OK) ? best : saved;
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (x) cudaFree(x);
    if (out) cudaFree(out);
    if (offd) cudaFree(offd);
    if (best_out) *best_out = ctx->tune[dtype];
    return st;
}

extern "C" nrm_status nrm_tune(nrm_ctx *ctx, nrm_dtype dtype, const int64_t *lengths_host, int64_t B) {
    return nrm_autotune(ctx, dtype, lengths_host, B, nullptr);
}
