// nrm_kernels.cu -- xNRMF / xNRMP tree kernels for sm_103a and the C ABI
// declared in include/nrm.h (arXiv 2509.06220, Listings 1, 2, 4, 5).
//
// Mapping of the paper's vectorised recursion onto the GPU
// ---------------------------------------------------------
// * A vector's elements form rows of P lanes (P = 64 for binary64, 128 for
//   binary32; one 512-byte row).  One warp holds one row in registers: thread
//   t owns lanes [V t, V t + V), loaded with one 16-byte load.
// * The ceil-split tree over the m rows (Listing 4's recursion on vectors)
//   is embedded in a perfect tree of depth D = ceil(lg m): slot j holds a
//   row iff brev_D(j) < m; a node with an empty child passes the other
//   through, so the embedding computes exactly Listing 4's tree.
// * The tree is cut at depth dw into 2^dw work items; a warp evaluates one
//   item (a subtree of 2^k slots) with groups of 2^G slots combined in
//   registers and a binary-counter stack above them.
// * Above the cut, each internal node has a ticket.  The warp that finishes a
//   child stores its 512-byte row of partial norms, fences, and increments
//   the parent's ticket; the second arriver combines the two children (left
//   operand = left child) and climbs on.  Whoever combines the root reduces
//   the P lanes with R's contiguous pairing (in-thread, then warp shuffles)
//   and writes the result.  The arrival order never changes a bit.
// * The second arriver resets the ticket, so tickets are zero between calls.
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

namespace nrm {

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
template <typename T> struct TreeArgs {
    const T *x;
    T *out;
    const VecPlan *plans; // batch: device plans; nullptr: single vector `one`
    VecPlan one;
    int64_t B;
    int64_t item_lo, item_hi;      // single vector: item range of this launch
    const int64_t *total_items;    // batch: written by the plan kernel
    unsigned long long *cursor;    // batch: dynamic work cursor (zeroed by plan)
    unsigned *tickets;
    T *slots;
    int levels;                    // counter-stack rows per warp: max k - G of the launch
};

// R over the P lanes held by the warp (Listing 1 with contiguous pairing):
// first inside the thread, then across threads by xor-shuffles.
template <typename T, class Op>
__device__ __forceinline__ T lane_reduce(const T (&r)[Geo<T>::V], const Op &op, int lane) {
    T v;
    if constexpr (Geo<T>::V == 2) {
        v = op(r[0], r[1]);
    } else {
        v = op(op(r[0], r[1]), op(r[2], r[3]));
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T o = __shfl_xor_sync(FULL, v, off);
        v = (lane & off) ? op(o, v) : op(v, o);
    }
    return v;
}

template <typename T>
__device__ __forceinline__ void store_row(T *dst, const T (&r)[Geo<T>::V]) {
    if constexpr (Geo<T>::V == 2) {
        __stcg(reinterpret_cast<double2 *>(dst), make_double2(r[0], r[1]));
    } else {
        __stcg(reinterpret_cast<float4 *>(dst), make_float4(r[0], r[1], r[2], r[3]));
    }
}

template <typename T>
__device__ __forceinline__ void load_slot(const T *src, T (&r)[Geo<T>::V]) {
    if constexpr (Geo<T>::V == 2) {
        const double2 v = __ldcg(reinterpret_cast<const double2 *>(src));
        r[0] = v.x;
        r[1] = v.y;
    } else {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(src));
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    }
}

// The register cap comes from the combine (Op::kMaxRegs): the trees are
// latency-bound, so more resident warps pay more than per-thread ILP (a
// sweep on GB300 found 64 registers best for v1_hypot in both precisions).
// FinalA: reduce the P lane partials with the correctly rounded hypot (the
// algorithm A; Z with A is the paper's recommended xNRMF) instead of op.
// stages of the cp.async ring of work items (Op::kStages, default none)
template <class Op, class = void> struct StagesOf {
    static constexpr int value = 0;
};
template <class Op> struct StagesOf<Op, std::void_t<decltype(Op::kStages)>> {
    static constexpr int value = Op::kStages;
};

// dynamic shared memory of a tree block: per warp, the counter stack of
// `levels` rows (k - G for the deepest work item of the launch, at most
// MAXL) and the ring of StagesOf<Op> groups of 2^G rows (512 bytes a row)
template <int G, class Op> constexpr size_t tree_smem_bytes(int wpb, int levels) {
    return (size_t)wpb * ((size_t)levels * 512 + (size_t)StagesOf<Op>::value * (1u << G) * 512);
}

// stack rows for work items of at most 2^kmax rows
static int stack_levels(int kmax, int G) { return std::max(0, std::min(MAXL, kmax - G)); }

template <typename T, int G, class Op, bool FinalA = false>
__global__ void __maxnreg__(Op::kMaxRegs) tree_kernel(TreeArgs<T> a, Op op) {
    constexpr int V = Geo<T>::V;
    constexpr int P = Geo<T>::P;
    const int lane = threadIdx.x & 31;
    const int64_t wglobal = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool batch = a.plans != nullptr;
    const int64_t total = batch ? *a.total_items : a.item_hi;
    extern __shared__ __align__(16) unsigned char nrm_smem[];
    T *stk = reinterpret_cast<T *>(nrm_smem) + (threadIdx.x >> 5) * (a.levels * P);
    constexpr int NS = StagesOf<Op>::value;
    typename Geo<T>::vec *ring = reinterpret_cast<typename Geo<T>::vec *>(
        nrm_smem + (size_t)(blockDim.x >> 5) * a.levels * 512 + (size_t)(threadIdx.x >> 5) * (NS * (1u << G) * 512));

    int64_t gi;
    if (batch) {
        unsigned long long g0 = 0;
        if (lane == 0) g0 = atomicAdd(a.cursor, 1ull);
        gi = (int64_t)__shfl_sync(FULL, g0, 0);
    } else {
        gi = a.item_lo + wglobal;
    }
    while (gi < total) {
        // locate the vector owning global item gi
        int64_t v = 0;
        VecPlan pl;
        if (batch) {
            int64_t lo = 0, hi = a.B; // last v with item_base <= gi
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (a.plans[mid].item_base <= gi) lo = mid;
                else hi = mid;
            }
            v = lo;
            pl = a.plans[v];
        } else {
            pl = a.one;
        }
        const T *xv = a.x + pl.x_off;
        const bool aligned = pl.stride == 1 && ((uintptr_t)xv & 15u) == 0;
        const uint32_t i = (uint32_t)(gi - pl.item_base);
        const int64_t t = node_rows(pl.m, i, pl.dw);
        const int64_t start = node_start(pl.m, i, pl.dw);
        T r[V];
        bool done = false;
        if constexpr (NS > 0) {
            if (pl.stride == 1 && pl.k > G && t >= (int64_t(1) << (pl.k - G))) {
                const bool tail = (start + t) * P > pl.n;
                if (t == (int64_t(1) << pl.k)) {
                    if (aligned)
                        done = item_tree_async<T, G, Op, NS, true, 1>(xv, pl.n, start, t, pl.k, lane, true, tail, op,
                                                                      stk, ring, r);
                    else
                        done = item_tree_async<T, G, Op, NS, true, 0>(xv, pl.n, start, t, pl.k, lane, false, tail, op,
                                                                      stk, ring, r);
                } else {
                    done = item_tree_async<T, G, Op, NS, false, -1>(xv, pl.n, start, t, pl.k, lane, aligned, tail, op,
                                                                    stk, ring, r);
                }
            }
        }
        if (!done) item_tree<T, G, Op>(xv, pl.n, start, t, pl.k, lane, aligned, pl.stride, op, stk, r);

        // climb the ticket tree above the cut
        uint32_t h = (1u << pl.dw) + i;
        bool root = true;
        while (h > 1) {
            T *mine = a.slots + ((size_t)(2 * pl.node_base + h - 2) * P) + lane * V;
            store_row<T>(mine, r);
            __threadfence();
            __syncwarp();
            unsigned tk = 0;
            unsigned *ticket = a.tickets + (pl.node_base + (h >> 1) - 1);
            if (lane == 0) tk = atomicAdd(ticket, 1u);
            tk = __shfl_sync(FULL, tk, 0);
            if (tk == 0) {
                root = false; // the sibling is still running; it climbs on
                break;
            }
            if (lane == 0) atomicExch(ticket, 0u);
            __threadfence();
            T sib[V];
            load_slot<T>(a.slots + ((size_t)(2 * pl.node_base + (h ^ 1u) - 2) * P) + lane * V, sib);
            if (h & 1u) {
#pragma unroll
                for (int j = 0; j < V; ++j) r[j] = op(sib[j], r[j]);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) r[j] = op(r[j], sib[j]);
            }
            h >>= 1;
        }
        if (root) {
            T res;
            if constexpr (FinalA) res = lane_reduce<T, OpCrHypot<T>>(r, OpCrHypot<T>{}, lane);
            else res = lane_reduce<T, Op>(r, op, lane);
            if (lane == 0) a.out[batch ? pl.out_idx : v] = res;
        }
        if (batch) {
            unsigned long long g1 = 0;
            if (lane == 0) g1 = atomicAdd(a.cursor, 1ull);
            gi = (int64_t)__shfl_sync(FULL, g1, 0);
        } else {
            gi += nwarps;
        }
    }
}

// ---------------------------------------------------------------------------
// batch planning (one block): offsets -> per-vector plans, prefix sums of
// work items and ticket nodes, statuses, outputs of empty / bad vectors, and
// the reset of the work cursor
// ---------------------------------------------------------------------------
// Vector v is x[off[v] .. off[v+1]) when lens == nullptr (consecutive
// vectors), else the segment x[off[v] .. off[v] + lens[v]).
template <typename T>
__global__ void __launch_bounds__(1024) plan_kernel(const int64_t *__restrict__ off, const int64_t *__restrict__ lens,
                                                    int64_t B, int64_t x_len,
                                                    int kitem, int dwmax, int kmax, int64_t node_cap,
                                                    VecPlan *plans, int64_t *totals, unsigned long long *cursor,
                                                    T *out, int32_t *status) {
    constexpr int P = Geo<T>::P;
    __shared__ int64_t s_items[1024], s_nodes[1024];
    const int tid = threadIdx.x;
    const int64_t per = (B + blockDim.x - 1) / blockDim.x;
    const int64_t v0 = min(B, tid * per), v1 = min(B, v0 + per);
    int kk = kitem; // work-item depth; deepened below if the tickets would not fit
    auto plan_of = [&](int64_t v, VecPlan &pl, int64_t &items, int64_t &nodes, int32_t &st) {
        const int64_t a = off[v];
        const int64_t b = lens ? ((lens[v] >= 0 && a <= x_len - lens[v]) ? a + lens[v] : -1) : off[v + 1];
        pl = VecPlan{};
        items = 0;
        nodes = 0;
        st = NRM_OK;
        if (a < 0 || b < a || b > x_len) {
            st = NRM_EINVAL;
            return;
        }
        const int64_t n = b - a;
        pl.x_off = a;
        pl.n = n;
        pl.stride = 1;
        if (n == 0) return;
        pl.m = (n + P - 1) / P;
        pl.D = ceil_log2_i64(pl.m);
        int k = min(pl.D, kk);
        if (pl.D - k > dwmax) k = pl.D - dwmax;
        if (k > kmax) {
            st = NRM_EINVAL; // larger than the tree kernel supports (> 2^33 rows)
            return;
        }
        pl.k = k;
        pl.dw = pl.D - k;
        items = int64_t(1) << pl.dw;
        nodes = items - 1;
    };
    int64_t si, sn;
    for (;;) {
        si = 0;
        sn = 0;
        for (int64_t v = v0; v < v1; ++v) {
            VecPlan pl;
            int64_t it, nd;
            int32_t st;
            plan_of(v, pl, it, nd, st);
            si += it;
            sn += nd;
        }
        s_items[tid] = si;
        s_nodes[tid] = sn;
        __syncthreads();
        // Hillis-Steele inclusive scan over the 1024 partial sums
        for (int d = 1; d < 1024; d <<= 1) {
            int64_t ai = 0, an = 0;
            if (tid >= d) {
                ai = s_items[tid - d];
                an = s_nodes[tid - d];
            }
            __syncthreads();
            s_items[tid] += ai;
            s_nodes[tid] += an;
            __syncthreads();
        }
        // segments may overlap, so their nodes are not bounded by x_len:
        // deeper work items need fewer tickets (the tree is unchanged)
        if (s_nodes[blockDim.x - 1] <= node_cap || kk >= kmax) break;
        __syncthreads();
        ++kk;
    }
    // If even the deepest work items need more ticket nodes than the
    // workspace holds, no vector is computed and all report NRM_ENOMEM.
    const bool overflow = s_nodes[blockDim.x - 1] > node_cap;
    const int64_t total_items = s_items[blockDim.x - 1], total_nodes = s_nodes[blockDim.x - 1];
    const int64_t nb0 = s_nodes[tid] - sn; // this thread's first ticket node (vector order)
    const int64_t ib0 = s_items[tid] - si; // its first work item in vector order
    // statuses and the outputs of empty or bad vectors
    for (int64_t v = v0; v < v1; ++v) {
        VecPlan pl;
        int64_t it, nd;
        int32_t st;
        plan_of(v, pl, it, nd, st);
        if (overflow && st == NRM_OK) st = NRM_ENOMEM;
        if (status) status[v] = st;
        if (st != NRM_OK) out[v] = T(NAN);
        else if (pl.n == 0) out[v] = T(0);
    }
    // Work order: the persistent grid takes work items in index order, so
    // the vectors are numbered longest first (a counting sort on n in
    // quarter-octave classes, the last bucket for vectors without work
    // items) and the
    // plans stored in that order, their item bases increasing with the index,
    // each with its vector's output index.  Within a bucket the order comes
    // from one 64-bit atomic per vector that returns its slot (high 20 bits)
    // and its first item (low 44 bits) together, so it may differ between
    // calls: it decides which warp computes a subtree, never the tree.
    // Ticket nodes keep the vector order.
    // classes of a quarter octave: floor(log2 n) and the next two bits of n
    constexpr int NB = 4 * 41 + 1;
    __shared__ unsigned long long s_cnt[NB];
    __shared__ int64_t s_vbase[NB], s_ibase[NB];
    const bool sorted = B < (int64_t(1) << 20) && total_items < (int64_t(1) << 44);
    auto bucket_of = [&](int64_t n, int64_t items) {
        if (items == 0 || overflow) return NB - 1;
        const int lg = 63 - __clzll((long long)n); // n >= 1
        const int cls = lg >= 40 ? 4 * 40 + 3 : 4 * lg + (lg >= 2 ? (int)((n >> (lg - 2)) & 3) : 0);
        return NB - 2 - cls;
    };
    __syncthreads(); // every reader of the scans above is done
    for (int q = tid; q < NB; q += blockDim.x) s_cnt[q] = 0ull;
    __syncthreads();
    if (sorted) {
        for (int64_t v = v0; v < v1; ++v) {
            VecPlan pl;
            int64_t it, nd;
            int32_t st;
            plan_of(v, pl, it, nd, st);
            atomicAdd(&s_cnt[bucket_of(pl.n, it)], (1ull << 44) | (unsigned long long)(overflow ? 0 : it));
        }
    }
    __syncthreads();
    if (tid == 0) {
        int64_t vb = 0, ibs = 0;
        for (int q = 0; q < NB; ++q) {
            s_vbase[q] = vb;
            s_ibase[q] = ibs;
            vb += (int64_t)(s_cnt[q] >> 44);
            ibs += (int64_t)(s_cnt[q] & ((1ull << 44) - 1));
            s_cnt[q] = 0ull;
        }
    }
    __syncthreads();
    int64_t nbr = nb0, ib_unsorted = ib0;
    for (int64_t v = v0; v < v1; ++v) {
        VecPlan pl;
        int64_t it, nd;
        int32_t st;
        plan_of(v, pl, it, nd, st);
        if (overflow) it = 0;
        pl.node_base = nbr;
        pl.out_idx = v;
        if (sorted) {
            const int q = bucket_of(pl.n, it);
            const unsigned long long got = atomicAdd(&s_cnt[q], (1ull << 44) | (unsigned long long)it);
            pl.item_base = s_ibase[q] + (int64_t)(got & ((1ull << 44) - 1));
            plans[s_vbase[q] + (int64_t)(got >> 44)] = pl;
        } else {
            pl.item_base = ib_unsorted;
            plans[v] = pl;
            ib_unsorted += it;
        }
        nbr += nd;
    }
    if (tid == blockDim.x - 1) {
        totals[0] = overflow ? 0 : total_items;
        totals[1] = total_nodes;
        *cursor = 0ull;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int DW_MAX = 20;

template <typename T> constexpr int P_of() { return Geo<T>::P; }

// Workspace layout of one call (the tickets live in their own buffer, see
// nrm_ctx::tickets, so that no other data ever occupies a ticket).
struct Layout {
    size_t slots, plans, totals, cursor, end;
};

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

static Layout layout_for(int64_t nodes, int64_t B) {
    Layout L;
    L.slots = 0;
    L.plans = align256(512 * (size_t)std::max<int64_t>(2 * nodes, 1));
    L.totals = L.plans + align256(sizeof(VecPlan) * (size_t)std::max<int64_t>(B, 1));
    L.cursor = L.totals + 256;
    L.end = L.cursor + 256;
    return L;
}

} // namespace nrm

using namespace nrm;

// context --------------------------------------------------------------------

static nrm_status set_cuda_err(nrm_ctx *c, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return NRM_OK;
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    if (e == cudaErrorMemoryAllocation) return NRM_ENOMEM;
    return NRM_ECUDA;
}

// Grow the workspace to `bytes` and the ticket array to `tickets` counters.
// Tickets are zeroed when allocated and are returned to zero by every call
// (each node's second arriver resets its ticket), so they never need
// clearing between calls.
nrm_status nrm_ctx_ensure(nrm_ctx *c, size_t bytes, int64_t tickets) {
    if (bytes <= c->ws_bytes && tickets <= c->tickets_cap) return NRM_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return set_cuda_err(c, e, "cudaSetDevice");
    e = cudaDeviceSynchronize(); // the old buffers may still be in use
    if (e != cudaSuccess) return set_cuda_err(c, e, "cudaDeviceSynchronize");
    if (bytes > c->ws_bytes) {
        if (c->ws) cudaFree(c->ws);
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
        if (c->tickets) cudaFree(c->tickets);
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
    // defaults from a sweep on GB300 at n = 2^28 (the autotuner refines them)
    c->tune[NRM_F32] = nrm_tuning{2, 4, 9, 16};
    c->tune[NRM_F64] = nrm_tuning{2, 8, 9, 16};
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

// single-vector planning ------------------------------------------------------

// Plan of one vector of n elements with P lanes: cut depth dw so that there
// are enough work items to fill the GPU (at least min_items when the tree is
// deep enough) but items no smaller than 2^G rows and no more than 2^DW_MAX.
static bool plan_single(const nrm_ctx *c, int64_t n, int P, VecPlan &pl) {
    const nrm_tuning &tu = c->tune[P == 64 ? NRM_F64 : NRM_F32];
    pl = VecPlan{};
    pl.n = n;
    pl.stride = 1;
    pl.m = (n + P - 1) / P;
    pl.D = ceil_log2_i64(pl.m);
    const int G = tu.group_log2;
    const int64_t min_items = (int64_t)c->sms * tu.warps_per_block * 2;
    int dw_fill = ceil_log2_i64(min_items);
    int dw = std::max(pl.D - tu.item_log2, dw_fill);
    dw = std::min(dw, pl.D - G);
    dw = std::max(dw, 0);
    dw = std::min(dw, DW_MAX);
    int k = pl.D - dw;
    if (k > G + MAXL) return false;
    pl.k = k;
    pl.dw = dw;
    return true;
}

template <typename T> static const nrm_tuning &tune_of(const nrm_ctx *c) {
    return c->tune[sizeof(T) == 8 ? NRM_F64 : NRM_F32];
}

template <typename T, class Op, bool FinalA = false>
static cudaError_t launch_tree(nrm_ctx *c, const TreeArgs<T> &a, const Op &op, int64_t grid_warps,
                               cudaStream_t s) {
    const nrm_tuning &tu = tune_of<T>(c);
    const int wpb = tu.warps_per_block;
    int occ = 0;
    int64_t blocks = 0;
    cudaError_t e = cudaSuccess;
    switch (tu.group_log2) {
#define NRM_LAUNCH_G(GG)                                                                                    \
    case GG: {                                                                                              \
        const size_t smem = tree_smem_bytes<GG, Op>(wpb, a.levels);                                        \
        cudaFuncSetAttribute(tree_kernel<T, GG, Op, FinalA>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                             (int)smem);                                                                    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tree_kernel<T, GG, Op, FinalA>, wpb * 32, smem); \
        occ = std::max(1, std::min(occ, tu.blocks_per_sm));                                                \
        blocks = std::max<int64_t>(1, std::min<int64_t>((grid_warps + wpb - 1) / wpb, (int64_t)c->sms * occ)); \
        tree_kernel<T, GG, Op, FinalA><<<(unsigned)blocks, wpb * 32, smem, s>>>(a, op);                     \
        e = cudaGetLastError();                                                                             \
        break;                                                                                              \
    }
        NRM_LAUNCH_G(2)
        NRM_LAUNCH_G(3)
#undef NRM_LAUNCH_G
    default: return cudaErrorInvalidValue;
    }
    c->launches++;
    return e;
}

// p -> combine op dispatch (Section 4): 2 -> v1_hypot, 1 -> sumabs,
// inf -> maxabs, other -> v1_lp with p/2 and 1/p rounded once in T.  From
// the cut-off p' on (Section 4) pow(Z, 1/p) is 1 for every Z in [1, 2], so
// v1_lp returns max(|x|, |y|): p >= 2^53 (binary64) / 2^24 (binary32) takes
// the maxabs code, which gives the same bits.
template <typename T, class F> static cudaError_t with_op(T p, F &&f) {
    const T cut = sizeof(T) == 8 ? T(9007199254740992.0) : T(16777216.0f);
    if (p == T(2)) return f(OpHypot<T>{});
    if (p == T(1)) return f(OpSumAbs<T>{});
    if (p >= cut) return f(OpMaxAbs<T>{});
    OpLp<T> o;
    o.h = p * T(0.5);
    o.ip = T(1) / p;
    return f(o);
}

template <typename T>
static nrm_status run_single(nrm_ctx *c, const T *x, int64_t n, T p, T *out, cudaStream_t s, int64_t item_lo,
                             int64_t item_hi, const VecPlan *plan_in, int64_t stride = 1, int variant = 0) {
    VecPlan pl;
    if (plan_in) pl = *plan_in;
    else if (!plan_single(c, n, P_of<T>(), pl)) return NRM_EINVAL;
    if (!plan_in) pl.stride = stride;
    const int64_t items = int64_t(1) << pl.dw;
    const int64_t nodes = items - 1;
    Layout L = layout_for(nodes, 1);
    nrm_status st = nrm_ctx_ensure(c, L.end, nodes);
    if (st != NRM_OK) return st;
    TreeArgs<T> a{};
    a.x = x;
    a.out = out;
    a.plans = nullptr;
    a.one = pl;
    a.B = 1;
    a.item_lo = plan_in ? item_lo : 0;
    a.item_hi = plan_in ? item_hi : items;
    a.total_items = nullptr;
    a.cursor = nullptr;
    a.tickets = c->tickets;
    a.slots = reinterpret_cast<T *>((char *)c->ws + L.slots);
    a.levels = stack_levels(pl.k, tune_of<T>(c).group_log2);
    const int64_t warps = a.item_hi - a.item_lo;
    cudaError_t e;
    // variant 0: the combine of p; 1: Z with A (cr_hypot for the lane
    // reduction); 2: the exponent-scaled hypotenuse K2 throughout
    if (variant == 1) e = launch_tree<T, OpHypot<T>, true>(c, a, OpHypot<T>{}, warps, s);
    else if (variant == 2) e = launch_tree<T, OpHypot2<T>>(c, a, OpHypot2<T>{}, warps, s);
    else e = with_op<T>(p, [&](auto op) { return launch_tree<T>(c, a, op, warps, s); });
    return set_cuda_err(c, e, "tree_kernel launch");
}

nrm_status nrm_plan_single(const nrm_ctx *c, nrm_dtype dt, int64_t n, VecPlan *pl) {
    return plan_single(c, n, dt == NRM_F64 ? 64 : 128, *pl) ? NRM_OK : NRM_EINVAL;
}

nrm_status nrm_run_single_range(nrm_ctx *c, nrm_dtype dt, const void *x, int64_t n, double p, void *out,
                                cudaStream_t s, const VecPlan *pl, int64_t item_lo, int64_t item_hi) {
    if (dt == NRM_F64)
        return run_single<double>(c, (const double *)x, n, p, (double *)out, s, item_lo, item_hi, pl);
    return run_single<float>(c, (const float *)x, n, (float)p, (float *)out, s, item_lo, item_hi, pl);
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
    return run_single<T>(c, x, n, p, out, s, 0, 0, nullptr);
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
    return run_single<T>(c, x, n, T(2), out, s, 0, 0, nullptr, 1, 1);
}

// xNRMF with the exponent-scaled hypotenuse K2 (a hypot[f] variant, Section 2)
template <typename T> static nrm_status es_entry(nrm_ctx *c, const T *x, int64_t n, T *out, void *stream) {
    nrm_status st = check_args<T>(c, x, n, T(2), out);
    if (st != NRM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return set_cuda_err(c, cudaMemsetAsync(out, 0, sizeof(T), s), "cudaMemsetAsync");
    return run_single<T>(c, x, n, T(2), out, s, 0, 0, nullptr, 1, 2);
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
        return run_single<double>(ctx, (const double *)first, n, p, (double *)out, s, 0, 0, nullptr, incx);
    return run_single<float>(ctx, (const float *)first, n, (float)p, (float *)out, s, 0, 0, nullptr, incx);
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
    nrm_status st = nrm_batch_impl(ctx, dtype, A, (N - 1) * lda + M, starts, N, p, colnorm, nullptr, s, lens);
    if (st != NRM_OK) return st;
    return nrm_run_single_range(ctx, dtype, colnorm, N, p, out, s, nullptr, 0, 0);
}

// batch -----------------------------------------------------------------------

// (for segments that may overlap, the plan kernel's overflow guard applies)
static int64_t batch_nodes_bound(const nrm_ctx *c, int64_t x_len, int64_t B, int P) {
    // sum over vectors of 2^dw - 1 < 2 (m_v / 2^k) summed, m_v <= n_v/P + 1
    const int k = c->tune[P == 64 ? NRM_F64 : NRM_F32].item_log2;
    const int64_t rows = x_len / P + B + 1;
    return (2 * rows >> k) + 2;
}

int64_t nrm_batch_tickets(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B) {
    return batch_nodes_bound(c, x_len, B, dt == NRM_F64 ? 64 : 128);
}

size_t nrm_batch_ws_bytes(const nrm_ctx *c, nrm_dtype dt, int64_t x_len, int64_t B) {
    const int P = dt == NRM_F64 ? 64 : 128;
    return layout_for(batch_nodes_bound(c, x_len, B, P), B).end;
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

template <typename T>
static nrm_status run_batch(nrm_ctx *c, const T *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                            int64_t B, T p, T *out, int32_t *status, cudaStream_t s) {
    constexpr int P = Geo<T>::P;
    const int64_t nodes_bound = batch_nodes_bound(c, x_len, B, P);
    Layout L = layout_for(nodes_bound, B);
    nrm_status st = nrm_ctx_ensure(c, L.end, nodes_bound);
    if (st != NRM_OK) return st;
    char *ws = (char *)c->ws;
    VecPlan *plans = reinterpret_cast<VecPlan *>(ws + L.plans);
    int64_t *totals = reinterpret_cast<int64_t *>(ws + L.totals);
    unsigned long long *cursor = reinterpret_cast<unsigned long long *>(ws + L.cursor);
    const nrm_tuning &tu = tune_of<T>(c);
    // Deepest work item: vectors of offsets never overlap, so the ticket
    // bound holds at item_log2 and a vector's k is at most item_log2 or
    // D - DW_MAX for the longest possible vector (x_len elements); the plan
    // kernel reports NRM_EINVAL for any vector deeper than kmax.  Segments
    // may overlap and deepen their items, up to G + MAXL.
    int kmax = tu.group_log2 + MAXL;
    if (!lens) {
        const int dmax = ceil_log2_i64(std::max<int64_t>(1, (x_len + P - 1) / P));
        kmax = std::min(kmax, std::max(std::min(dmax, tu.item_log2), dmax - DW_MAX));
        kmax = std::max(kmax, tu.group_log2);
    }
    plan_kernel<T><<<1, 1024, 0, s>>>(off, lens, B, x_len, tu.item_log2, DW_MAX, kmax, nodes_bound, plans, totals,
                                      cursor, out, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_err(c, e, "plan_kernel launch");
    TreeArgs<T> a{};
    a.x = x;
    a.out = out;
    a.plans = plans;
    a.B = B;
    a.total_items = totals;
    a.cursor = cursor;
    a.tickets = c->tickets;
    a.slots = reinterpret_cast<T *>(ws + L.slots);
    a.levels = stack_levels(kmax, tu.group_log2);
    const int64_t persistent = (int64_t)c->sms * 64 * tu.warps_per_block; // capped by occupancy
    e = with_op<T>(p, [&](auto op) { return launch_tree<T>(c, a, op, persistent, s); });
    return set_cuda_err(c, e, "tree_kernel launch (batch)");
}

nrm_status nrm_batch_impl(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *offsets,
                          int64_t B, double p, void *out, int32_t *status, cudaStream_t s, const int64_t *lens) {
    if (!ctx || B < 0 || x_len < 0 || (dtype != NRM_F32 && dtype != NRM_F64)) return NRM_EINVAL;
    if (B > 0 && (!offsets || !out)) return NRM_EINVAL;
    if (x_len > 0 && !x) return NRM_EINVAL;
    if (!(p > 0.0)) return NRM_EINVAL;
    if (B == 0) return NRM_OK;
    if (dtype == NRM_F64)
        return run_batch<double>(ctx, (const double *)x, x_len, offsets, lens, B, p, (double *)out, status, s);
    const float pf = (float)p;
    if (!(pf > 0.0f)) return NRM_EINVAL;
    return run_batch<float>(ctx, (const float *)x, x_len, offsets, lens, B, pf, (float *)out, status, s);
}

extern "C" nrm_status nrm_batch_segments(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len,
                                         const int64_t *starts, const int64_t *lengths, int64_t B, double p,
                                         void *out, int32_t *status, void *stream) {
    if (B > 0 && !lengths) return NRM_EINVAL;
    return nrm_batch_impl(ctx, dtype, x, x_len, starts, B, p, out, status, (cudaStream_t)stream, lengths);
}

extern "C" nrm_status nrm_batch(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len,
                                const int64_t *offsets, int64_t B, double p, void *out, int32_t *status,
                                void *stream) {
    return nrm_batch_impl(ctx, dtype, x, x_len, offsets, B, p, out, status, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// nrmf_d_noalloc: xNRMF in binary64 without any allocation.
//
// Some callers cannot call cudaMalloc: cudaMalloc and cudaFree can
// synchronise the whole device, which a latency-critical loop cannot
// afford, and some applications give all device memory to their own
// allocator or run under a fixed budget that forbids allocations outside it.
// This entry point therefore needs no context.  Its scratch (the tree's
// ticket counters and partial-norm slots) is the file-scope array below,
// created when the library is loaded onto a device and held until the
// process exits.  It is shared by every call on that device and keeps the
// last call's contents; the tickets are cleared on the stream at the start of
// each call.  The array's device address is looked up once per device; a
// cudaDeviceReset destroys the array with the context, after which this
// entry point must not be called again in the process.
// ---------------------------------------------------------------------------
namespace {

// Size limit: n <= 2^29 gives m <= 2^23 rows, a row tree of depth D <= 23,
// and with at most 2^11 work items each item holds k = D - dw <= 12 =
// NA_G + MAXL levels, the deepest the counter stack supports.
constexpr int NA_DW_MAX = 11;                                // at most 2^11 work items
constexpr int64_t NA_NODES = (int64_t(1) << NA_DW_MAX) - 1;  // internal tree nodes
constexpr size_t NA_TICKET_BYTES = 8192;                     // >= NA_NODES * 4, slot-aligned
constexpr size_t NA_SLOT_BYTES = (size_t)2 * NA_NODES * 512; // one 512-byte row per child node
constexpr int NA_G = 2, NA_WPB = 4;
static_assert(NA_TICKET_BYTES >= (size_t)NA_NODES * 4 && NA_TICKET_BYTES % 512 == 0, "ticket area");
static_assert(NA_DW_MAX + NA_G + MAXL >= 23, "n = 2^29 (2^23 rows) must fit the scratch and the stack");
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char nrm_noalloc_scratch[NA_TICKET_BYTES + NA_SLOT_BYTES];

struct NaDevice {
    bool ready = false;
    unsigned char *scratch = nullptr; // device address of nrm_noalloc_scratch
    int sms = 0;
    int occ = 1;
};
NaDevice na_devices[NA_MAX_DEVICES];
std::mutex na_mutex;

// One-time set-up per device, with that device current: look up the
// device address of the scratch array (host code cannot use the symbol
// itself) and the occupancy of the kernel.
nrm_status na_setup(int dev, NaDevice **out) {
    std::lock_guard<std::mutex> lock(na_mutex);
    NaDevice &d = na_devices[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, nrm_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return NRM_ECUDA;
        }
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return NRM_ECUDA;
        int occ = 0;
        const size_t smem = tree_smem_bytes<NA_G, OpHypot<double>>(NA_WPB, MAXL);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tree_kernel<double, NA_G, OpHypot<double>>,
                                                          NA_WPB * 32, smem);
        if (e != cudaSuccess) return NRM_ECUDA;
        d.occ = std::max(1, occ);
        d.scratch = static_cast<unsigned char *>(p);
        d.ready = true;
    }
    *out = &d;
    return NRM_OK;
}

} // namespace

extern "C" nrm_status nrmf_d_noalloc(const double *x, int64_t n, double *out, void *stream) {
    if (!out || n < 0 || (n > 0 && !x)) return NRM_EINVAL;
    if (n > NRM_NOALLOC_MAX_N) return NRM_EINVAL; // the tree would need more scratch than the array holds
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(double), s) == cudaSuccess ? NRM_OK : NRM_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return NRM_EDEVICE;
    NaDevice *d = nullptr;
    nrm_status st = na_setup(dev, &d);
    if (st != NRM_OK) return st;

    // the same tree as nrmf_d; only the cut depth is capped by the scratch size
    VecPlan pl{};
    pl.n = n;
    pl.stride = 1;
    pl.m = (n + 63) / 64;
    pl.D = ceil_log2_i64(pl.m);
    int dw = std::max(pl.D - 7, ceil_log2_i64((int64_t)d->sms * NA_WPB * 2));
    dw = std::min(dw, pl.D - NA_G);
    dw = std::max(dw, 0);
    dw = std::min(dw, NA_DW_MAX);
    pl.dw = dw;
    pl.k = pl.D - dw;
    if (pl.k > NA_G + MAXL) return NRM_EINVAL;
    const int64_t items = int64_t(1) << dw;
    const int64_t nodes = items - 1;

    unsigned *tickets = reinterpret_cast<unsigned *>(d->scratch);
    double *slots = reinterpret_cast<double *>(d->scratch + NA_TICKET_BYTES);
    if (nodes > 0 && cudaMemsetAsync(tickets, 0, (size_t)nodes * sizeof(unsigned), s) != cudaSuccess)
        return NRM_ECUDA;
    TreeArgs<double> a{};
    a.x = x;
    a.out = out;
    a.plans = nullptr;
    a.one = pl;
    a.B = 1;
    a.item_lo = 0;
    a.item_hi = items;
    a.tickets = tickets;
    a.slots = slots;
    a.levels = MAXL;
    const size_t smem = tree_smem_bytes<NA_G, OpHypot<double>>(NA_WPB, MAXL);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((items + NA_WPB - 1) / NA_WPB,
                                                                  (int64_t)d->sms * d->occ));
    tree_kernel<double, NA_G, OpHypot<double>><<<(unsigned)blocks, NA_WPB * 32, smem, s>>>(a, OpHypot<double>{});
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
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
__global__ void k1d_compare_kernel(uint64_t seed, int64_t n, int mode, unsigned long long *bad, double *example) {
    const bool fast = mode >= 8;
    const int fam = mode & 7;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x, y;
        k1d_pair(seed, i, fam, x, y);
        if (fast) {
            const uint32_t hx = (uint32_t)((uint64_t)__double_as_longlong(x) >> 32) & 0x7fffffffu;
            const uint32_t hy = (uint32_t)((uint64_t)__double_as_longlong(y) >> 32) & 0x7fffffffu;
            const uint32_t lo = (uint32_t)(1023 - 500) << 20, hi = (uint32_t)(1023 + 502) << 20;
            if (hx < lo || hx >= hi || hy < lo || hy >= hi) continue;
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

extern "C" nrm_status nrm_test_lp(nrm_dtype dtype, double p, const void *x, const void *y, void *out, int64_t n,
                                  void *stream) {
    if (n < 0 || (n > 0 && (!x || !y || !out)) || !(p > 0.0) || (dtype != NRM_F64 && dtype != NRM_F32))
        return NRM_EINVAL;
    if (n == 0) return NRM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == NRM_F64) {
        OpLp<double> op;
        op.h = p * 0.5;
        op.ip = 1.0 / p;
        lp_eval_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(op, (const double *)x, (const double *)y,
                                                                       (double *)out, n);
    } else {
        OpLp<float> op;
        const float pf = (float)p;
        op.h = pf * 0.5f;
        op.ip = 1.0f / pf;
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
    if (n < 0 || !bad || !example || mode < 0 || mode > 14 || mode == 7) return NRM_EINVAL;
    k1d_compare_kernel<<<152 * 16, 256, 0, (cudaStream_t)stream>>>(seed, n, mode, bad, example);
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}
