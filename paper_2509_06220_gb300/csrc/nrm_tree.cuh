// nrm_tree.cuh -- the xNRMF / xNRMP tree kernels for sm_103a, their batch
// planner and their host-side launchers (arXiv 2509.06220, Listings 1, 2, 4,
// 5).  Internal: the kernels of each element type are instantiated in their
// own translation unit (nrm_tree_d.cu, nrm_tree_s.cu; the batch kernel with
// one p per vector in nrm_tree_mixed.cu), and nrm_kernels.cu calls them
// through run_single_x / run_batch_x.
//
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
#pragma once

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
    const int64_t *bases; // batch: the plans' item bases, compact (the owner search reads these)
    VecPlan one;
    int64_t B;
    int64_t item_lo, item_hi;      // single vector: item range of this launch
    const int64_t *total_items;    // batch: written by the plan kernel
    unsigned long long *cursor;    // batch: dynamic work cursor (zeroed by plan)
    unsigned *item_cursor;         // single vector: dynamic item cursor (zero between launches), or
                                   // nullptr for a static assignment (warp w takes items w, w + nwarps, ...)
    unsigned *tickets;
    T *slots;
    int levels;                    // counter-stack rows per warp: max k - G of the launch
    T *lanes;                      // batch with a p per vector, B = 1: the root stores its P lane partials here
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

// Ordering of the ticket tree: the warp that finishes a child stores its row,
// then a device-scope acquire-release fence, then increments the parent's
// ticket (relaxed); the second arriver reads the ticket, fences again and
// loads its sibling's row -- fence-to-fence message passing, which needs no
// sequentially consistent fence.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// One work item: global item gi, the item's subtree (index gi - item_base
// at depth dw of vector v's row tree, plan pl), the climb of the ticket tree
// above the cut, and -- for whoever combines the root -- the lane reduction
// and the store of the result.
// stk: this warp's counter stack; ring: its cp.async ring (ops with stages).
// MayStoreLanes: when a.lanes is set, the root's P lane partials are stored
// there (a shard's node of the row tree) instead of being reduced.
template <typename T, int G, class Op, bool FinalA, bool MayStoreLanes = false>
__device__ __forceinline__ void process_item(const TreeArgs<T> &a, const VecPlan &pl, int64_t v, int64_t gi,
                                             int lane, bool batch, const Op &op, T *stk,
                                             typename Geo<T>::vec *ring) {
    constexpr int V = Geo<T>::V;
    constexpr int P = Geo<T>::P;
    constexpr int NS = StagesOf<Op>::value;
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
        fence_acq_rel_gpu(); // release this row before the ticket
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
        fence_acq_rel_gpu(); // acquire the sibling's row after the ticket
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
        if constexpr (MayStoreLanes) {
            if (a.lanes) {
                store_row<T>(a.lanes + lane * V, r);
                return;
            }
        }
        T res;
        if constexpr (FinalA) res = lane_reduce<T, OpCrHypot<T>>(r, OpCrHypot<T>{}, lane);
        else res = lane_reduce<T, Op>(r, op, lane);
        if (lane == 0) a.out[batch ? pl.out_idx : v] = res;
    }
}

// the plan of the vector owning global item gi (last v with item_base <= gi)
// (a binary search over the compact item bases, read through the read-only
// cache: 8 bytes a plan instead of one 88-byte plan per step)
template <typename T> __device__ __forceinline__ int64_t owner_of(const TreeArgs<T> &a, int64_t gi) {
    int64_t lo = 0, hi = a.B;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(a.bases + mid) <= gi) lo = mid;
        else hi = mid;
    }
    return lo;
}

// this warp's counter stack (a.levels rows) and ring (NS groups of 2^G rows)
// in the block's dynamic shared memory: all stacks first, then the rings
template <typename T, int G, int NS>
__device__ __forceinline__ void warp_smem(const TreeArgs<T> &a, T *&stk, typename Geo<T>::vec *&ring) {
    extern __shared__ __align__(16) unsigned char nrm_smem[];
    stk = reinterpret_cast<T *>(nrm_smem) + (threadIdx.x >> 5) * (a.levels * Geo<T>::P);
    ring = reinterpret_cast<typename Geo<T>::vec *>(nrm_smem + (size_t)(blockDim.x >> 5) * a.levels * 512 +
                                                    (size_t)(threadIdx.x >> 5) * (NS * (1u << G) * 512));
}

template <typename T, int G, class Op, bool FinalA = false>
__global__ void __maxnreg__(Op::kMaxRegs) tree_kernel(TreeArgs<T> a, Op op) {
    const int lane = threadIdx.x & 31;
    const int64_t wglobal = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool batch = a.plans != nullptr;
    const int64_t total = batch ? *a.total_items : a.item_hi;
    T *stk;
    typename Geo<T>::vec *ring;
    warp_smem<T, G, StagesOf<Op>::value>(a, stk, ring);

    // Work order.  Batch: the atomic cursor.  Single vector: items of one
    // size, taken from the item cursor in index order, so that the last
    // round of items spreads over all SMs (a static stride left whole SMs
    // idle while others ran their last items); the warp that draws the last
    // value (total - item_lo + nwarps - 1: every other draw happened before
    // it) returns the cursor to zero for the next launch.
    const bool dyn = !batch && a.item_cursor != nullptr;
    int64_t gi;
    if (batch) {
        unsigned long long g0 = 0;
        if (lane == 0) g0 = atomicAdd(a.cursor, 1ull);
        gi = (int64_t)__shfl_sync(FULL, g0, 0);
    } else if (dyn) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(a.item_cursor, 1u);
        gi = a.item_lo + (int64_t)__shfl_sync(FULL, g0, 0);
    } else {
        gi = a.item_lo + wglobal;
    }
    while (gi < total) {
        int64_t v = 0;
        VecPlan pl;
        if (batch) {
            v = owner_of<T>(a, gi);
            pl = a.plans[v];
        } else {
            pl = a.one;
        }
        process_item<T, G, Op, FinalA>(a, pl, v, gi, lane, batch, op, stk, ring);
        if (batch) {
            unsigned long long g1 = 0;
            if (lane == 0) g1 = atomicAdd(a.cursor, 1ull);
            gi = (int64_t)__shfl_sync(FULL, g1, 0);
        } else if (dyn) {
            unsigned g1 = 0;
            if (lane == 0) g1 = atomicAdd(a.item_cursor, 1u);
            gi = a.item_lo + (int64_t)__shfl_sync(FULL, g1, 0);
        } else {
            gi += nwarps;
        }
    }
    if (dyn && lane == 0 && gi - a.item_lo == total - a.item_lo + nwarps - 1) *a.item_cursor = 0u;
}

// A ragged batch with a p per vector: the same persistent loop, each work
// item combined with its vector's op (a warp-uniform switch: an item belongs
// to one vector), so every result is bitwise that of the single-p kernel for
// that vector's p.  Register cap: v1_lp's in both precisions (binary64 64:
// its pows are out-of-line calls, and 64 registers keep twice the warps of
// 128 resident; at binary32 v1_hypot's 72 the binary32 v1_lp spills: 2.33
// ms against 1.46 ms).
template <typename T> struct MixedRegs {
    static constexpr int value = OpLp<T>::kMaxRegs;
};
template <typename T, int G>
__global__ void __maxnreg__(MixedRegs<T>::value) tree_kernel_mixed(TreeArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t total = *a.total_items;
    T *stk;
    typename Geo<T>::vec *ring; // sized for the largest ring of the ops (v1_hypot's)
    warp_smem<T, G, StagesOf<OpHypot<T>>::value>(a, stk, ring);
    unsigned long long g0 = 0;
    if (lane == 0) g0 = atomicAdd(a.cursor, 1ull);
    int64_t gi = (int64_t)__shfl_sync(FULL, g0, 0);
    while (gi < total) {
        const int64_t v = owner_of<T>(a, gi);
        const VecPlan pl = a.plans[v];
        switch (pl.op) {
        case OP_HYPOT:
            process_item<T, G, OpHypot<T>, false, true>(a, pl, v, gi, lane, true, OpHypot<T>{}, stk, ring);
            break;
        case OP_LP: {
            OpLp<T> o;
            o.set((T)pl.h, (T)pl.ip);
            process_item<T, G, OpLp<T>, false, true>(a, pl, v, gi, lane, true, o, stk, ring);
            break;
        }
        case OP_SUMABS:
            process_item<T, G, OpSumAbs<T>, false, true>(a, pl, v, gi, lane, true, OpSumAbs<T>{}, stk, ring);
            break;
        default:
            process_item<T, G, OpMaxAbs<T>, false, true>(a, pl, v, gi, lane, true, OpMaxAbs<T>{}, stk, ring);
            break;
        }
        unsigned long long g1 = 0;
        if (lane == 0) g1 = atomicAdd(a.cursor, 1ull);
        gi = (int64_t)__shfl_sync(FULL, g1, 0);
    }
}

// ---------------------------------------------------------------------------
// batch planning (one block): offsets -> per-vector plans, prefix sums of
// work items and ticket nodes, statuses, outputs of empty / bad vectors, and
// the reset of the work cursor
// ---------------------------------------------------------------------------
// Vector v is x[off[v] .. off[v+1]) when lens == nullptr (consecutive
// vectors), else the segment x[off[v] .. off[v] + lens[v]).
// Per-vector p (pdev != nullptr): vector v's p is pdev[v] rounded to T;
// its combine follows the rule of one p per call (Section 4): 2 -> v1_hypot,
// 1 -> sumabs, at or above the cut-off p' -> maxabs, otherwise v1_lp with
// h = p/2 and ip = 1/p rounded in T; p <= 0 or NaN is NRM_EINVAL.
template <typename T> __device__ __forceinline__ bool plan_op(double pd, VecPlan &pl) {
    const T p = (T)pd;
    if (!(p > T(0))) return false;
    const T cut = sizeof(T) == 8 ? T(9007199254740992.0) : T(16777216.0f);
    pl.h = 0.0;
    pl.ip = 0.0;
    if (p == T(2)) pl.op = OP_HYPOT;
    else if (p == T(1)) pl.op = OP_SUMABS;
    else if (p >= cut) pl.op = OP_MAXABS;
    else {
        pl.op = OP_LP;
        pl.h = (double)rmul(p, T(0.5));
        pl.ip = (double)rdiv(T(1), p);
    }
    return true;
}

constexpr int LP_FINER = 2;

// Inclusive scan of v over the 1024 threads of the block (warp shuffles,
// then the 32 warp totals); *total receives the block's sum.  s_warp: 32
// shared slots.  Every thread of the block must call it.
__device__ __forceinline__ int64_t block_scan_1024(int64_t v, int64_t *s_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += s_warp[warp - 1];
    *total = s_warp[31];
    __syncthreads(); // s_warp may be reused
    return v;
}

// plans are stored as six 16-byte words (VecPlan is padded to 96 bytes)
__device__ __forceinline__ void store_plan(VecPlan *dst, const VecPlan &pl) {
    static_assert(sizeof(VecPlan) == 96, "VecPlan is six 16-byte words");
    const int4 *src = reinterpret_cast<const int4 *>(&pl);
    int4 *d = reinterpret_cast<int4 *>(dst);
#pragma unroll
    for (int w = 0; w < 6; ++w) __stcg(d + w, src[w]);
}

// One block of 1024 threads.  Thread t handles the vectors of one
// contiguous chunk, [t c, (t + 1) c) with c = ceil(B / 1024), so that each
// prefix sum (ticket nodes in vector order, item bases in plan order) is a
// single block scan of the threads' chunk totals; a chunk is read two
// vectors at a time, their offset loads issued together.
template <typename T>
__global__ void __launch_bounds__(1024) plan_kernel(const int64_t *__restrict__ off, const int64_t *__restrict__ lens,
                                                    const double *__restrict__ pdev, int64_t B, int64_t x_len,
                                                    int kitem, int dwmax, int kmax, int64_t node_cap,
                                                    VecPlan *plans, int64_t *bases, int64_t *totals,
                                                    unsigned long long *cursor,
                                                    T *out, int32_t *status) {
    constexpr int P = Geo<T>::P;
    constexpr int U = 2; // vectors whose loads are issued together
    __shared__ int64_t s_warp[32];
    const int tid = threadIdx.x;
    const int64_t C = (B + 1023) / 1024;
    const int64_t v0 = min((int64_t)tid * C, B), v1 = min(v0 + C, B);
    int kk = kitem; // work-item depth; deepened below if the tickets would not fit
    // a vector's segment [a, b) (b = -1 for a bad length) and p
    struct Seg {
        int64_t a, b;
        double p;
    };
    auto load_seg = [&](int64_t v) {
        Seg g;
        g.a = off[v];
        if (lens) {
            const int64_t l = lens[v];
            g.b = (l >= 0 && g.a <= x_len - l) ? g.a + l : -1;
        } else {
            g.b = off[v + 1];
        }
        g.p = pdev ? pdev[v] : 2.0;
        return g;
    };
    auto plan_of = [&](const Seg &g, VecPlan &pl, int64_t &items, int64_t &nodes, int32_t &st) {
        const int64_t a = g.a, b = g.b;
        pl = VecPlan{};
        items = 0;
        nodes = 0;
        st = NRM_OK;
        if (a < 0 || b < a || b > x_len || (pdev && !plan_op<T>(g.p, pl))) {
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
        // with a p per vector, v1_lp vectors take items LP_FINER levels
        // smaller: their combine is many times costlier, so a batch of them
        // is otherwise one wave of long items at the kernel's register cap
        int k = min(pl.D, (pdev && pl.op == OP_LP) ? max(kk - LP_FINER, 0) : kk);
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
    // Work order: the persistent grid takes work items in index order, so
    // the vectors are numbered longest first: a counting sort on n in
    // quarter-octave classes (floor(log2 n) and its next two bits; the last
    // class for vectors without work items), the plans stored in that order
    // with their output index, and their item bases increasing with the
    // plan index.  With a p per vector the classes are ordered by combine
    // first (v1_lp, v1_hypot, maxabs, sumabs: the costliest first).  Within
    // a class the order comes from shared-memory atomics, so it may differ
    // between calls: it decides which warp computes a subtree, never the
    // tree.  Ticket nodes keep the vector order.
    constexpr int NL = 4 * 41 + 1;   // length classes
    constexpr int NB = 4 * NL;       // (combine, length) classes, NB <= 1024
    __shared__ unsigned s_cnt[NB], s_cur[NB];
    __shared__ int64_t s_vbase[NB];
    // item counts of the plans in plan order (the first PLAN_SMEM of them;
    // the rest are read back from the plans)
    constexpr int PLAN_SMEM = 8192;
    __shared__ int32_t s_items[PLAN_SMEM];
    auto bucket_of = [&](const VecPlan &pl, int64_t items) {
        if (items == 0) return NB - 1;
        const int64_t n = pl.n;
        const int lg = 63 - __clzll((long long)n); // n >= 1
        const int cls = lg >= 40 ? 4 * 40 + 3 : 4 * lg + (lg >= 2 ? (int)((n >> (lg - 2)) & 3) : 0);
        const int rank = !pdev ? 0 : pl.op == OP_LP ? 0 : pl.op == OP_HYPOT ? 1 : pl.op == OP_MAXABS ? 2 : 3;
        return rank * NL + (NL - 2 - cls);
    };
    // One pass: the ticket nodes of all vectors and the class counts.
    // Segments may overlap, so their nodes are not bounded by x_len: if the
    // nodes exceed the workspace, deeper work items need fewer of them (the
    // tree is unchanged), and the pass is repeated at the next depth.
    int64_t total_nodes, node_excl;
    for (;;) {
        for (int q = tid; q < NB; q += 1024) s_cnt[q] = s_cur[q] = 0u;
        __syncthreads();
        int64_t tn = 0;
        for (int64_t j0 = 0; j0 < C; j0 += U) {
            Seg g[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (v0 + j0 + u < v1) g[u] = load_seg(v0 + j0 + u);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool valid = v0 + j0 + u < v1;
                int64_t it = 0, nd = 0;
                int q = NB; // no class
                if (valid) {
                    VecPlan pl;
                    int32_t st;
                    plan_of(g[u], pl, it, nd, st);
                    q = bucket_of(pl, it);
                }
                if (valid) atomicAdd(&s_cnt[q], 1u);
                tn += nd;
            }
        }
        int64_t sn;
        const int64_t incl = block_scan_1024(tn, s_warp, &sn);
        node_excl = incl - tn;
        total_nodes = sn;
        if (total_nodes <= node_cap || kk >= kmax) break;
        ++kk;
    }
    // If even the deepest work items need more ticket nodes than the
    // workspace holds, no vector is computed and all report NRM_ENOMEM (all
    // in the last class, without work items).
    const bool overflow = total_nodes > node_cap;
    if (overflow)
        for (int q = tid; q < NB; q += 1024) s_cnt[q] = q == NB - 1 ? (unsigned)B : 0u;
    __syncthreads();
    // first plan index of every class: an exclusive scan over the classes
    {
        const int64_t c = tid < NB ? (int64_t)s_cnt[tid] : 0;
        int64_t tot;
        const int64_t incl = block_scan_1024(c, s_warp, &tot);
        if (tid < NB) s_vbase[tid] = incl - c;
        __syncthreads();
    }
    // the plans, in class order, with their item counts in item_base for
    // now; statuses and the outputs of empty or bad vectors
    int64_t nbase = node_excl; // ticket nodes of the vectors before this one
    for (int64_t j0 = 0; j0 < C; j0 += U) {
        Seg g[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (v0 + j0 + u < v1) g[u] = load_seg(v0 + j0 + u);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t v = v0 + j0 + u;
            const bool valid = v < v1;
            VecPlan pl;
            int64_t it = 0, nd = 0;
            int q = NB;
            if (valid) {
                int32_t st;
                plan_of(g[u], pl, it, nd, st);
                if (overflow) {
                    it = 0;
                    if (st == NRM_OK) st = NRM_ENOMEM;
                }
                if (status) status[v] = st;
                if (st != NRM_OK) out[v] = T(NAN);
                else if (pl.n == 0) out[v] = T(0);
                q = bucket_of(pl, it);
            }
            if (valid) {
                pl.node_base = nbase;
                pl.out_idx = v;
                pl.item_base = it;
                const int64_t slot = s_vbase[q] + atomicAdd(&s_cur[q], 1u);
                store_plan(plans + slot, pl);
                if (slot < PLAN_SMEM) s_items[slot] = (int32_t)it;
            }
            nbase += nd;
        }
    }
    __syncthreads(); // the plans are written (visible within the block)
    // item bases in plan order: thread t takes the plan slots [t c, (t + 1) c)
    auto items_at = [&](int64_t sl) { return sl < PLAN_SMEM ? (int64_t)s_items[sl] : plans[sl].item_base; };
    int64_t ci = 0;
    for (int64_t sl = v0; sl < v1; ++sl) ci += items_at(sl);
    int64_t total_items;
    const int64_t iincl = block_scan_1024(ci, s_warp, &total_items);
    int64_t run = iincl - ci;
    for (int64_t sl = v0; sl < v1; ++sl) {
        const int64_t c = items_at(sl);
        plans[sl].item_base = run;
        bases[sl] = run;
        run += c;
    }
    if (tid == 0) {
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
    size_t slots, plans, bases, totals, cursor, end;
};

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

static Layout layout_for(int64_t nodes, int64_t B) {
    Layout L;
    L.slots = 0;
    L.plans = align256(512 * (size_t)std::max<int64_t>(2 * nodes, 1));
    L.bases = L.plans + align256(sizeof(VecPlan) * (size_t)std::max<int64_t>(B, 1));
    L.totals = L.bases + align256(sizeof(int64_t) * (size_t)std::max<int64_t>(B, 1));
    L.cursor = L.totals + 256;
    L.end = L.cursor + 256;
    return L;
}


// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static nrm_status set_cuda_err(nrm_ctx *c, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return NRM_OK;
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    if (e == cudaErrorMemoryAllocation) return NRM_ENOMEM;
    return NRM_ECUDA;
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
    // a short vector: items of at least 2^(G+2) rows (filling the GPU with
    // items of one group made the ticket tree above them the critical path)
    dw = std::min(dw, std::max(pl.D - G - 2, 0));
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
    o.set(p * T(0.5), T(1) / p);
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
    // the tickets of the nodes, and one more counter (the buffer's last) as
    // the item cursor: every call leaves both at zero
    nrm_status st = nrm_ctx_ensure(c, L.end, nodes + 1);
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
    a.item_cursor = c->tickets + (c->tickets_cap - 1);
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

// (for segments that may overlap, the plan kernel's overflow guard applies)
static int64_t batch_nodes_bound(const nrm_ctx *c, int64_t x_len, int64_t B, int P, bool per_vector_p = false) {
    // sum over vectors of 2^dw - 1 < 2 (m_v / 2^k) summed, m_v <= n_v/P + 1
    // (with a p per vector, v1_lp items are LP_FINER levels smaller)
    const int k = std::max(0, c->tune[P == 64 ? NRM_F64 : NRM_F32].item_log2 - (per_vector_p ? LP_FINER : 0));
    const int64_t rows = x_len / P + B + 1;
    return (2 * rows >> k) + 2;
}

// The batch kernel with one p per vector, launched from nrm_tree_mixed.cu.
cudaError_t launch_mixed(nrm_ctx *c, const TreeArgs<double> &a, int64_t grid_warps, cudaStream_t s);
cudaError_t launch_mixed(nrm_ctx *c, const TreeArgs<float> &a, int64_t grid_warps, cudaStream_t s);

template <typename T>
static cudaError_t launch_tree_mixed(nrm_ctx *c, const TreeArgs<T> &a, int64_t grid_warps, cudaStream_t s) {
    const nrm_tuning &tu = tune_of<T>(c);
    const int wpb = tu.warps_per_block;
    int occ = 0;
    int64_t blocks = 0;
    cudaError_t e = cudaSuccess;
    switch (tu.group_log2) {
#define NRM_LAUNCH_MIXED(GG)                                                                                \
    case GG: {                                                                                              \
        const size_t smem = tree_smem_bytes<GG, OpHypot<T>>(wpb, a.levels); /* the largest of the ops */   \
        cudaFuncSetAttribute(tree_kernel_mixed<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tree_kernel_mixed<T, GG>, wpb * 32, smem);      \
        occ = std::max(1, std::min(occ, tu.blocks_per_sm));                                                \
        blocks = std::max<int64_t>(1, std::min<int64_t>((grid_warps + wpb - 1) / wpb, (int64_t)c->sms * occ)); \
        tree_kernel_mixed<T, GG><<<(unsigned)blocks, wpb * 32, smem, s>>>(a);                               \
        e = cudaGetLastError();                                                                             \
        break;                                                                                              \
    }
        NRM_LAUNCH_MIXED(2)
        NRM_LAUNCH_MIXED(3)
#undef NRM_LAUNCH_MIXED
    default: return cudaErrorInvalidValue;
    }
    c->launches++;
    return e;
}

template <typename T>
static nrm_status run_batch(nrm_ctx *c, const T *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                            int64_t B, T p, const double *p_dev, T *out, int32_t *status, cudaStream_t s,
                            T *lanes = nullptr) {
    constexpr int P = Geo<T>::P;
    const int64_t nodes_bound = batch_nodes_bound(c, x_len, B, P, p_dev != nullptr);
    Layout L = layout_for(nodes_bound, B);
    nrm_status st = nrm_ctx_ensure(c, L.end, nodes_bound);
    if (st != NRM_OK) return st;
    char *ws = (char *)c->ws;
    VecPlan *plans = reinterpret_cast<VecPlan *>(ws + L.plans);
    int64_t *bases = reinterpret_cast<int64_t *>(ws + L.bases);
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
    plan_kernel<T><<<1, 1024, 0, s>>>(off, lens, p_dev, B, x_len, tu.item_log2, DW_MAX, kmax, nodes_bound, plans,
                                      bases, totals, cursor, out, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_err(c, e, "plan_kernel launch");
    TreeArgs<T> a{};
    a.x = x;
    a.out = out;
    a.plans = plans;
    a.bases = bases;
    a.B = B;
    a.total_items = totals;
    a.cursor = cursor;
    a.tickets = c->tickets;
    a.slots = reinterpret_cast<T *>(ws + L.slots);
    a.levels = stack_levels(kmax, tu.group_log2);
    a.lanes = lanes; // used by the p-per-vector kernel only (p_dev set, B = 1)
    const int64_t persistent = (int64_t)c->sms * 64 * tu.warps_per_block; // capped by occupancy
    if (p_dev) e = launch_mixed(c, a, persistent, s);
    else e = with_op<T>(p, [&](auto op) { return launch_tree<T>(c, a, op, persistent, s); });
    return set_cuda_err(c, e, "tree_kernel launch (batch)");
}

// The single-vector and batch entry points of each element type (defined in
// nrm_tree_d.cu and nrm_tree_s.cu).
nrm_status run_single_x(nrm_ctx *c, const double *x, int64_t n, double p, double *out, cudaStream_t s,
                        int64_t item_lo, int64_t item_hi, const VecPlan *plan_in, int64_t stride = 1,
                        int variant = 0);
nrm_status run_single_x(nrm_ctx *c, const float *x, int64_t n, float p, float *out, cudaStream_t s, int64_t item_lo,
                        int64_t item_hi, const VecPlan *plan_in, int64_t stride = 1, int variant = 0);
// lanes (p_dev set, B = 1): store the vector's P lane partials there, no lane reduction
nrm_status run_batch_x(nrm_ctx *c, const double *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                       int64_t B, double p, const double *p_dev, double *out, int32_t *status, cudaStream_t s,
                       double *lanes = nullptr);
nrm_status run_batch_x(nrm_ctx *c, const float *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                       int64_t B, float p, const double *p_dev, float *out, int32_t *status, cudaStream_t s,
                       float *lanes = nullptr);

} // namespace nrm
