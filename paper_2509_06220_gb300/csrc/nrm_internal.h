// nrm_internal.h -- host-side declarations shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nrm.h"

namespace nrm {
struct VecPlan;
}

struct nrm_graph {
    nrm_ctx *ctx;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

struct nrm_ctx {
    int device = 0;
    int sms = 1;
    void *ws = nullptr;        // partial-norm slots, batch plans, totals, cursor
    size_t ws_bytes = 0;
    unsigned *tickets = nullptr; // one counter per internal tree node; all zero between calls
    int64_t tickets_cap = 0;
    void *aux = nullptr; // matrix norms: column starts, lengths and norms
    size_t aux_bytes = 0;
    void *node_args = nullptr; // nrm_node_lanes: the one-vector offsets, p and output (256 bytes)
    nrm_tuning tune[2]{}; // per element type: [NRM_F32], [NRM_F64]
    std::string err;
    uint64_t launches = 0;
    std::vector<nrm_graph *> graphs;
    // buffers outgrown while graphs existed: a captured graph keeps their
    // addresses, so they are freed with the context, not on growth
    std::vector<void *> retired;
    // end-to-end (host buffer) staging
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t s_copy[4] = {nullptr, nullptr, nullptr, nullptr}, s_comp = nullptr;
    std::vector<cudaEvent_t> ev;
    void *out_dev = nullptr;
};

nrm_status nrm_ctx_ensure(nrm_ctx *c, size_t bytes, int64_t tickets = 0);
nrm_status nrm_plan_single(const nrm_ctx *c, nrm_dtype dt, int64_t n, nrm::VecPlan *pl);
nrm_status nrm_run_single_range(nrm_ctx *c, nrm_dtype dt, const void *x, int64_t n, double p, void *out,
                                cudaStream_t s, const nrm::VecPlan *pl, int64_t item_lo, int64_t item_hi);
nrm_status nrm_batch_impl(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *offsets,
                          int64_t B, double p, const double *p_dev, void *out, int32_t *status, cudaStream_t s,
                          const int64_t *lens = nullptr);
// workspace and ticket counters of a batch (per_vector_p: a p per vector)
size_t nrm_batch_ws_bytes(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B, bool per_vector_p = false);
int64_t nrm_batch_tickets(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B, bool per_vector_p = false);
void nrm_graph_free(nrm_graph *g);
void nrm_host_free(nrm_ctx *c);
bool nrm_test_fail_alloc();

// one device-generated input segment of a server step (element offset in the
// arena viewed as the segment's type, length, generator key and range)
struct NrmGenSeg {
    int64_t start, n;
    uint64_t key;
    int32_t emin, span, dtype, pad;
};
uint64_t nrm_gen_key(uint64_t seed, uint64_t vec);
nrm_status nrm_gen_segments(const NrmGenSeg *segs_dev, const int64_t *cum_dev, int64_t count, int64_t total,
                            void *arena, cudaStream_t s);
