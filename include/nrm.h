/*
 * nrm.h -- C ABI of the GB300 (sm_103a) library for xNRMF / xNRMP
 * (V. Novakovic, "Recursive vectorized computation of the vector p-norm",
 * arXiv 2509.06220).
 *
 * What every entry point computes
 * -------------------------------
 * The norm of an array x[0..n) is the paper's vectorised recursion Z
 * (Listing 4, Section 3) with a fixed lane count P, followed by a final
 * recursive reduction R (Listing 1) of the P lane partial norms:
 *
 *   rows     : row r holds x[r*P .. r*P+P), the last row zero-padded
 *              (Listing 4's masked TAIL load); m = ceil(n/P) rows;
 *   row tree : the rows are combined lane by lane with Listing 1's split
 *              (left part ceil(m/2) rows, right part floor(m/2));
 *   lanes    : the P lane results are combined by R with contiguous
 *              pairing (lanes 2i and 2i+1 first);
 *   combine  : p = 2 -> v1_hypot (Listing 2, the algorithm H); p = 1 ->
 *              |x|+|y| (Eq. vp1); p = inf -> max(|x|,|y|) (Eq. vpI);
 *              other p > 0 -> v1_lp (Listing 5) with p/2 and 1/p computed
 *              once per call and the library's own pow.
 *
 * P = 64 for binary64 (the D routines) and P = 128 for binary32 (S), i.e.
 * one 512-byte row.  Section 3 notes that the vectorised results are
 * reproducible only for a fixed lane count; with P fixed, every result of
 * this library is bitwise identical across launches, grid sizes, tuning
 * parameters, batch composition, input alignment and streams.  All
 * arithmetic is IEEE round-to-nearest-even in the input's format, with no
 * contraction beyond the paper's explicit fma, and subnormals are kept.
 *
 * Conventions
 * -----------
 * - Pointers named x, out, offsets, status are DEVICE pointers owned by the
 *   caller unless the name ends in _host.  Inputs must stay valid and
 *   unmodified until the work queued on `stream` has finished.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls are asynchronous and stream-ordered; results stay on
 *   the device.
 * - A context owns device workspace (tickets and partial-norm slots) that
 *   calls reuse.  One context may be used from one host thread at a time and
 *   its calls must be ordered on one stream (or externally synchronised);
 *   use one context per concurrent stream.
 * - Argument errors are reported synchronously by the return value and
 *   enqueue nothing.  NRM_ECUDA means a CUDA call failed; nrm_last_error()
 *   returns its message.  No entry point traps or hangs the GPU.
 * - Inputs are expected to be finite.  Infinite entries give +inf.  A NaN is
 *   handled exactly as Listing 2 does (fmin/fmax return the other operand),
 *   which this library reproduces bit for bit up to the NaN payload.
 */
#ifndef NRM_H
#define NRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef int32_t nrm_status;
#define NRM_OK 0
#define NRM_EINVAL (-1)   /* bad argument (NULL pointer, n < 0, p <= 0 or NaN, ...) */
#define NRM_ENOMEM (-2)   /* device workspace could not be allocated */
#define NRM_ECUDA (-3)    /* a CUDA runtime call failed (see nrm_last_error) */
#define NRM_ETIMEOUT (-4) /* a bounded wait ran out */
#define NRM_EBUDGET (-5)  /* a request can never fit the serving memory budget */
#define NRM_EDEVICE (-6)  /* no usable CUDA device */

/* Element types. */
typedef int32_t nrm_dtype;
#define NRM_F32 0 /* binary32, P = 128 lanes (the S routines) */
#define NRM_F64 1 /* binary64, P = 64 lanes (the D routines) */

typedef struct nrm_ctx nrm_ctx;

/* Tuning knobs.  None of them changes any result bit; they only change how
 * the fixed tree is mapped onto warps. */
typedef struct {
    int32_t group_log2;      /* rows loaded per warp before combining: 2^g, g in 2..3 */
    int32_t warps_per_block; /* 4, 8 or 16 */
    int32_t item_log2;       /* rows per warp work item: 2^k slots, k in g..g+10 */
    int32_t blocks_per_sm;   /* persistent-grid residency target, 1..16 */
} nrm_tuning;

/* Create a context on CUDA device `device` (the device is made current on
 * the calling thread).  *ctx receives the handle.  Returns NRM_EDEVICE if the
 * device does not exist, NRM_ENOMEM if the initial workspace cannot be
 * allocated. */
nrm_status nrm_create(nrm_ctx **ctx, int device);

/* Destroy a context after synchronising its device; frees its workspace and
 * captured graphs.  NULL is accepted. */
nrm_status nrm_destroy(nrm_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *nrm_status_string(nrm_status s);

/* Message of the last CUDA error seen by this context ("" if none). */
const char *nrm_last_error(const nrm_ctx *ctx);

/* Ensure at least `bytes` of workspace are allocated (synchronous).  Call
 * this before capturing library calls into a CUDA graph, since growth
 * allocates. */
nrm_status nrm_reserve(nrm_ctx *ctx, size_t bytes);

/* Workspace bytes a call with the given shape needs under the current
 * tuning (single vector: B = 1, x_len = n). */
size_t nrm_workspace_bytes(const nrm_ctx *ctx, nrm_dtype dtype, int64_t x_len, int64_t B);

/* Tuning of the binary64 kernels (nrm_get_tuning) / of both element types
 * (nrm_set_tuning); the _for forms address one element type.  A setter
 * returns NRM_EINVAL (and keeps the old values) if a field is out of range. */
nrm_status nrm_get_tuning(const nrm_ctx *ctx, nrm_tuning *t);
nrm_status nrm_set_tuning(nrm_ctx *ctx, const nrm_tuning *t);
nrm_status nrm_get_tuning_for(const nrm_ctx *ctx, nrm_dtype dtype, nrm_tuning *t);
nrm_status nrm_set_tuning_for(nrm_ctx *ctx, nrm_dtype dtype, const nrm_tuning *t);

/*
 * xNRMF (Section 3, the recommended Z + recursive final reduction, with
 * v1_hypot of Listing 2 at every node): *out = ||x[0..n)||_F.
 *   x   : device pointer to n contiguous elements, any element alignment;
 *   n   : number of elements, n >= 0; n == 0 gives +0 (Listing 1 assumes
 *         n > 0; +0 is the norm of the empty array);
 *   out : device pointer to one element, written asynchronously.
 * Errors: NRM_EINVAL for ctx == NULL, out == NULL, n < 0, or x == NULL
 * with n > 0.
 */
nrm_status nrmf_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream);
nrm_status nrmf_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream);

/*
 * xNRMF as the paper recommends it (Section 3): the same vector recursion Z
 * with v1_hypot, but the final reduction of the P lane partials uses the
 * algorithm A -- R with the correctly rounded hypot RN(sqrt(x^2+y^2))
 * (cr_hypot, Section 2), computed exactly with integer arithmetic -- instead
 * of v1_hypot.  Arguments and errors as nrmf_*.
 */
nrm_status nrmf_za_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream);
nrm_status nrmf_za_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream);

/*
 * xNRMF with another hypot[f] (Section 2 admits any hypotenuse that avoids
 * undue overflow and underflow, is monotone in |x| and |y| and accurate to a
 * small multiple of eps): the exponent-scaled hypotenuse K2 in place of
 * v1_hypot in the whole tree (Z and the final reduction R of Section 3).
 * With m = min(|x|,|y|), M = max (a NaN operand is missing data) and k the
 * binade of M (the lowest normal binade for a subnormal M):
 *   a = M 2^-k, b = RN(m 2^-k), S = RN(fma(a, a, RN(b b))), s = RN(sqrt(S)),
 *   K2 = RN(s 2^k);  K2 = +0 for M = 0 and +inf for M = inf.
 * No division; relative error at most 1.75 eps + O(eps^2) per combine
 * without underflow; K2(a, 0) = |a| exactly.  A different set of bits from
 * nrmf_* (another hypot), bitwise reproducible and equal to the oracle's
 * or_nrm_es_*.  Arguments and errors as nrmf_*.
 */
nrm_status nrmf_es_s(nrm_ctx *ctx, const float *x, int64_t n, float *out, void *stream);
nrm_status nrmf_es_d(nrm_ctx *ctx, const double *x, int64_t n, double *out, void *stream);

/*
 * xNRMP (Section 4): *out = ||x[0..n)||_p by the same tree with the combine
 * chosen by p: p == 2 is exactly xNRMF; p == 1 sums |x| (Eq. vp1); p == +inf
 * takes max |x| (Eq. vpI); otherwise v1_lp (Listing 5, Eqs. sp and qp) with
 * h = p*0.5 and ip = 1/p rounded once in the element type.  0 < p < 1 gives
 * the quasi-norm the paper mentions.  Errors as nrmf_*, plus NRM_EINVAL for
 * p <= 0 or p NaN.
 */
nrm_status nrmp_s(nrm_ctx *ctx, const float *x, int64_t n, float p, float *out, void *stream);
nrm_status nrmp_d(nrm_ctx *ctx, const double *x, int64_t n, double p, double *out, void *stream);

/*
 * Strided vector (Section 3 leaves BLAS's incx to future work; done here):
 * ||(x_0, ..., x_{n-1})||_p with x_i = x[i incx] for incx > 0 and
 * x_i = x[(n-1-i) |incx|] for incx < 0 (BLAS order: the elements are taken
 * backwards), by the same tree as nrmp_* on that logical vector.  x is the
 * lowest-addressed element in both cases.  Errors: NRM_EINVAL for incx == 0
 * and as nrmp_*.
 */
nrm_status nrm_strided(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t n, int64_t incx, double p, void *out,
                       void *stream);

/*
 * Norm of a column-major M x N matrix A with leading dimension lda >= M
 * (Section 3.1): when lda == M (or N == 1) the elements are contiguous and
 * the matrix is the one vector A[0 .. M N); otherwise the N column norms
 * are computed (as one segment batch) and their norm by the same tree gives
 * the result (for any p: ||A||_p^p is the sum of the columns' p-th powers).
 * Higher-dimensional arrays A(lda, N2, ..., Nk) are the case N = N2...Nk.
 * out: device pointer to one element.  Uses context scratch of N
 * (16 + sizeof(element)) bytes.  Errors: NRM_EINVAL for M, N < 0, lda <
 * max(M, 1), NULL pointers, bad p or dtype.
 */
nrm_status nrm_matrix(nrm_ctx *ctx, nrm_dtype dtype, const void *A, int64_t M, int64_t N, int64_t lda, double p,
                      void *out, void *stream);

/*
 * Ragged batch (the paper's per-column norms of Section 3.1, here for a
 * batch of independent vectors): for i in [0, B),
 *   out[i] = ||x[offsets[i] .. offsets[i+1])||_{p_i}
 * with the same tree as nrmp_* (p_i is rounded to the element type first).
 *   x       : device pointer to x_len elements of `dtype`;
 *   offsets : device pointer to B+1 int64 element offsets (not bytes);
 *   p       : the p of every vector when p_dev is NULL (xNRMP's p, Section 4);
 *   p_dev   : NULL, or a device pointer to B doubles, p_i = p_dev[i] (p is
 *             then ignored): one launch serves vectors with different p,
 *             each combined with the combine nrmp_* takes for its p;
 *   out     : device pointer to B elements of `dtype`;
 *   status  : device pointer to B int32 (may be NULL): NRM_OK per vector,
 *             or NRM_EINVAL where offsets[i] < 0, offsets[i+1] < offsets[i],
 *             offsets[i+1] > x_len, or p_dev[i] (rounded) is <= 0 or NaN --
 *             that vector's out[i] is then NaN.  Bad offsets and p are
 *             detected on the device; nothing traps.  If overlapping offsets
 *             would need more workspace than x_len implies, every vector
 *             reports NRM_ENOMEM (out NaN).
 * Work is distributed by a device-side plan and one persistent launch; every
 * out[i] is bitwise identical to nrmp_* on that vector alone with p_i.
 * Errors (synchronous): NRM_EINVAL for bad dtype, B < 0, x_len < 0, NULL
 * offsets/out with B > 0, or (p_dev NULL) p <= 0 or NaN.
 */
nrm_status nrm_batch(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *offsets,
                     int64_t B, double p, const double *p_dev, void *out, int32_t *status, void *stream);

/*
 * Batch of segments: out[i] = ||x[starts[i] .. starts[i] + lengths[i])||_{p_i}
 * (device arrays of B int64 each), the same tree, p / p_dev and guarantees
 * as nrm_batch; segments may lie anywhere in x (a device arena) and in any
 * order.  A segment with starts[i] < 0, lengths[i] < 0 or starts[i] +
 * lengths[i] > x_len gives NaN and NRM_EINVAL in status[i].
 */
nrm_status nrm_batch_segments(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *starts,
                              const int64_t *lengths, int64_t B, double p, const double *p_dev, void *out,
                              int32_t *status, void *stream);

/*
 * The same batch captured once into a CUDA graph (plan kernel + tree
 * kernel) and replayed with nrm_graph_launch; each replay reads the current
 * contents of x, offsets and p_dev (when not NULL).  The context's workspace
 * is sized for x_len and B at capture time; if later calls on the context
 * grow its workspace, the buffers the graph was captured with stay
 * allocated until the context is destroyed, so the graph remains valid (do
 * not replay it concurrently with other calls on the same context).  *graph
 * receives an opaque handle owned by ctx.
 */
typedef struct nrm_graph nrm_graph;
nrm_status nrm_batch_graph(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t x_len, const int64_t *offsets,
                           int64_t B, double p, const double *p_dev, void *out, int32_t *status, nrm_graph **graph);
nrm_status nrm_graph_launch(nrm_graph *graph, void *stream);
nrm_status nrm_graph_destroy(nrm_graph *graph);

/*
 * Sharding one vector across 2^dg devices (Section 2, Eq. hr: the norms of
 * disjoint parts combine by one more hypot; Section 3.1 reduces per-column
 * norms the same way).  The vector's row tree (see the top of this file) is
 * cut at depth dg: device j holds the elements of node j, computes that
 * node's P lane partials (one 512-byte row) with nrm_node_lanes, the 2^dg
 * rows are gathered (512 bytes per device, e.g. one all-gather), and
 * nrm_combine_nodes combines them through the tree's top dg levels and
 * reduces the lanes: the result is bitwise the one-device nrmp_* result.
 *
 * nrm_shard_range (host only, no device work): node j of depth dg of the
 * tree over n elements of `dtype` holds elements [*first, *first + *count)
 * (count 0 when the node has no rows, i.e. n is below 2^dg rows' worth).
 * NRM_EINVAL for a bad dtype, n < 0, dg outside [0, NRM_SHARD_MAX_DEPTH],
 * j outside [0, 2^dg) or NULL outputs.
 */
#define NRM_SHARD_MAX_DEPTH 16
nrm_status nrm_shard_range(nrm_dtype dtype, int64_t n, int32_t dg, int64_t j, int64_t *first, int64_t *count);

/*
 * The P lane partials of one node: Z of Listing 4 over the node's `count`
 * elements x[0..count) (device pointer, any element alignment) with the
 * combine of p (as nrmp_*), without the final lane reduction; lanes: device
 * pointer to P elements of `dtype` (512 bytes), written asynchronously
 * (zeros when count == 0).  Uses the context's workspace.  Errors as
 * nrmp_*, plus NRM_EINVAL for lanes == NULL.
 */
nrm_status nrm_node_lanes(nrm_ctx *ctx, nrm_dtype dtype, const void *x, int64_t count, double p, void *lanes,
                          void *stream);

/*
 * Combine the 2^dg node rows lanes[j P .. j P + P) (device, in node order j;
 * overwritten: the buffer holds intermediate rows afterwards) of a vector of
 * n elements through the top dg levels of its row tree -- the left node is
 * the left operand, a node without rows passes its sibling through -- and
 * reduce the root's P lanes by R (Listing 1, contiguous pairing): *out (one
 * device element) = ||x||_p, bitwise equal to nrmp_* on the whole vector.
 * Errors: NRM_EINVAL for NULL pointers, n < 0, dg outside
 * [0, NRM_SHARD_MAX_DEPTH], a bad dtype, p <= 0 or NaN.
 */
nrm_status nrm_combine_nodes(nrm_ctx *ctx, nrm_dtype dtype, void *lanes, int32_t dg, int64_t n, double p, void *out,
                             void *stream);

/*
 * End-to-end call on HOST buffers: copies x_host[0..n) to the device in
 * chunks that overlap with the tree computation, computes ||x||_p as
 * nrmp_*, and copies the result to *out_host; returns when it is there.
 * x_host may be pageable or pinned (pinned is faster).  Errors as nrmp_*.
 */
nrm_status nrm_host(nrm_ctx *ctx, nrm_dtype dtype, const void *x_host, int64_t n, double p, void *out_host);

/*
 * Seeded synthetic input generator (not part of the method): fills
 * x[0..n) with elements start..start+n-1 of vector `vec` of `seed`, built
 * bit by bit from the SplitMix64 counter hash: sign bit random, fraction
 * uniform on the format's grid, exponent uniform in [emin, emax] (normal
 * range of the format).  nrm_gen_ragged fills a concatenated batch of x_len
 * elements, element j of vector i drawn from vector id i; vectors whose
 * offsets are malformed are skipped.  Errors: NRM_EINVAL for a bad dtype,
 * n < 0 or an exponent range outside the normal range.
 */
nrm_status nrm_gen(nrm_dtype dtype, void *x, int64_t n, uint64_t seed, uint64_t vec, int64_t start, int32_t emin,
                   int32_t emax, void *stream);
nrm_status nrm_gen_ragged(nrm_dtype dtype, void *x, int64_t x_len, const int64_t *offsets, int64_t B, uint64_t seed,
                          int32_t emin, int32_t emax, void *stream);

/*
 * xNRMF in binary64 that allocates nothing (the paper has no counterpart;
 * this is a deployment variant of nrmf_d).  *out = ||x[0..n)||_F with the
 * same tree, hence bitwise the same result as nrmf_d.
 *
 * For callers that cannot call cudaMalloc: cudaMalloc and cudaFree can
 * synchronise the whole device, which latency-critical loops cannot afford,
 * and some applications hand all device memory to their own allocator or to
 * a fixed budget and forbid allocations outside it.  No context is needed.
 *   x     : device pointer to n binary64 elements (any element alignment);
 *   n     : 0 <= n <= NRM_NOALLOC_MAX_N; n == 0 gives +0;
 *   out   : device pointer to one binary64, written asynchronously;
 *   stream: cudaStream_t as void* (NULL = legacy default stream).
 * Scratch: a static device array of about 2 MiB inside the library (8 KiB
 * of ticket counters and 2 (2^11 - 1) partial-norm rows of 512 bytes),
 * created on every device that loads the library and held until the process
 * exits.  The first call on each device looks up that array's address (with
 * the device current); make that first call before any stream capture.  A
 * cudaDeviceReset destroys the array with the device's context: do not call
 * this entry point after one in the same process.  All
 * calls on a device share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * give wrong results -- order them on one stream.
 * Errors: NRM_EINVAL for out == NULL, n < 0, x == NULL with n > 0, or
 * n > NRM_NOALLOC_MAX_N (the tree would need more scratch than the array
 * holds); NRM_EDEVICE if no device is current; NRM_ECUDA if a CUDA call
 * fails.  It calls no cudaMalloc, cudaFree or allocating library routine.
 */
#define NRM_NOALLOC_MAX_N (INT64_C(1) << 29)
nrm_status nrmf_d_noalloc(const double *x, int64_t n, double *out, void *stream);

/*
 * Autotuner: times every tuning candidate (group 2^g rows, warps per block,
 * work-item depth, residency) on a synthetic problem of the given shape --
 * one vector of lengths_host[0] elements when B == 1, else a ragged batch
 * of B vectors with these lengths -- and keeps the fastest for `dtype` in
 * ctx (also returned in *best when best != NULL).  Tuning never changes a
 * result bit.  Allocates temporary device memory for the synthetic input;
 * synchronous.  Errors: NRM_EINVAL (bad arguments), NRM_ENOMEM, NRM_ECUDA.
 */
nrm_status nrm_autotune(nrm_ctx *ctx, nrm_dtype dtype, const int64_t *lengths_host, int64_t B, nrm_tuning *best);

/* nrm_autotune without the tuning read-back (best = NULL): the name of the
 * autotuner in the library's interface sketch.  Same arguments, effects and
 * errors. */
nrm_status nrm_tune(nrm_ctx *ctx, nrm_dtype dtype, const int64_t *lengths_host, int64_t B);

/*
 * Continuous-batching server.  Requests (element type, p, length; input
 * copied from the host or generated on the device) are submitted at any
 * time; a worker thread admits them in FIFO order as soon as their input
 * fits in the device arena, and launches steps on `nstreams` streams as
 * they free up, so steps overlap on the device and later arrivals join the
 * next step.  A step computes up to `max_batch` requests, grouped by element
 * type, with one nrm_batch_segments per type (one p per request); every
 * result is bitwise the same as the request computed alone.  The budget covers the input arena and the
 * streams' tree workspaces, which are reserved at creation (the loop never
 * allocates).  Latency is measured from arrival to the result on the host.
 */
typedef struct nrm_srv nrm_srv;

typedef struct {
    nrm_dtype dtype;       /* NRM_F32 or NRM_F64 */
    int32_t emin, emax;    /* device-generated input: exponent range of nrm_gen */
    double p;              /* > 0; 2 = xNRMF */
    int64_t n;             /* elements */
    const void *x_host;    /* input on the host (copied at launch), or NULL: */
    uint64_t seed;         /*   generate with nrm_gen(seed, vector id = request id) */
    double arrival_s;      /* nrm_srv_replay only: arrival time from the trace start */
} nrm_request;

typedef struct {
    int64_t submitted, admitted, rejected, completed;
    int64_t steps, launches;     /* steps launched; kernel launches (2 per group) */
    int64_t max_queue;           /* most requests waiting for memory at once */
    int64_t peak_bytes, arena_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms; /* arrival -> result on the host */
    double wall_s, norms_per_s, elements_per_s;
    double host_launch_s; /* worker time spent issuing steps (copies, generator, plan and tree launches) */
    double host_retire_s; /* worker time spent retiring finished steps */
    double gpu_step_s;    /* sum over steps of their duration on the device (steps on several streams overlap) */
} nrm_srv_report;

/* Create a server on `device` with a device-memory budget (bytes, inputs +
 * workspaces), nstreams in 1..16, max_batch >= 1 requests per step.
 * NRM_EBUDGET if the workspaces leave no room for inputs. */
nrm_status nrm_srv_create(nrm_srv **srv, int device, size_t budget_bytes, int nstreams, int max_batch);
/* Submit one request; *id receives its id.  NRM_EBUDGET if its input can
 * never fit the arena (counted as rejected); NRM_EINVAL for bad fields.
 * A host input must stay valid until the request is done. */
nrm_status nrm_srv_submit(nrm_srv *srv, const nrm_request *req, uint64_t *id);
/* *done = 1 once the request finished; then *norm (widened to double) and
 * *status (NRM_OK or the error) are set. */
nrm_status nrm_srv_poll(nrm_srv *srv, uint64_t id, double *norm, int32_t *status, int32_t *done);
/* Wait until every submitted request is done (NRM_ETIMEOUT after timeout_s). */
nrm_status nrm_srv_drain(nrm_srv *srv, double timeout_s);
nrm_status nrm_srv_report_get(nrm_srv *srv, nrm_srv_report *rep);
/* Replay a trace: submit reqs[i] at its arrival_s (busy-waiting on the
 * host clock), drain, and return each norm and latency (ms) plus the report.
 * Rejected requests give NaN and latency -1. */
nrm_status nrm_srv_replay(nrm_srv *srv, const nrm_request *reqs, int64_t count, double *norms, double *latency_ms,
                          nrm_srv_report *rep);
/* Stop the worker after the queued requests finish, and free everything. */
nrm_status nrm_srv_destroy(nrm_srv *srv);

/* Number of tree-kernel launches this context has issued (for accounting). */
uint64_t nrm_kernel_launches(const nrm_ctx *ctx);

/* Host-side fault injection for tests (no GPU involvement): the next `count`
 * workspace or staging allocations of any context fail with NRM_ENOMEM
 * without calling cudaMalloc.  count <= 0 disarms it. */
void nrm_test_inject_alloc_failures(int count);

/* Test hook: evaluate the binary64 v1_hypot two ways on n generated operand
 * pairs (family `mode`, 0..6: moderate exponent gaps, close values, edge
 * significands, raw bit patterns, extreme exponents, gaps near 2^-27, equal
 * values) -- the integer/FP32 form the tree kernels use and the FP64-pipe
 * form -- and add the number of bitwise differences to *bad (device
 * pointer); example (device, 4 doubles) receives the first differing
 * x, y and both results.  mode 8..14: family mode - 8 with the branch-free
 * form of checked groups, on the pairs inside its range [2^-500, 2^502)
 * (others skipped); mode 16..22: the same with the paired branch-free form
 * (two operand pairs at once, as the tree kernels combine two lanes),
 * against the FP64 form of each pair.  NRM_EINVAL for another mode. */
nrm_status nrm_test_k1d_compare(uint64_t seed, int64_t n, int32_t mode, unsigned long long *bad, double *example,
                                void *stream);

/* Test hook: evaluate the library's pow (the pow of Listing 5, Section 4)
 * elementwise, out[i] = pow(x[i], y[i]), with the same device code the
 * xNRMP tree kernels use; x, y and out are device arrays of n elements of
 * `dtype` (NRM_F64: the fixed-point integer pow, NRM_F32: the binary32
 * double-word pow).  Asynchronous on `stream`; NRM_EINVAL for n < 0, null
 * arrays or an unknown dtype. */
nrm_status nrm_test_pow(nrm_dtype dtype, const void *x, const void *y, void *out, int64_t n, void *stream);

/* Test hook: the binary64 pow that v1_lp uses for 1 < p <= 2^17 (Listing 5,
 * Section 4, with the pow restricted to the two domains of v1_lp: x in
 * [0, 1) with y in [1/2, 2^16], or x in [1, 2] with y in [2^-17, 1]; a result
 * below 2^-28 is returned as +0), elementwise out[i] = pow(x[i], y[i]) with
 * the device code of the xNRMP tree kernels.  x, y and out are device
 * arrays of n binary64 values; the caller keeps the operands in that
 * domain (outside it the values are unspecified, nothing is read or
 * written beyond the n elements).  Asynchronous on `stream`; NRM_EINVAL for
 * n < 0 or null arrays. */
nrm_status nrm_test_powr(const double *x, const double *y, double *out, int64_t n, void *stream);

/* Test hook: v1_lp (Listing 5, Section 4's Eq. sp) elementwise with
 * h = p/2 and ip = 1/p rounded in `dtype`, out[i] = v1_lp(x[i], y[i]),
 * exactly as the xNRMP tree kernels combine (for binary64 the integer
 * quotient and pow, with the FP64 form for inf, NaN and subnormal
 * operands).  Device arrays of n elements; asynchronous on `stream`;
 * NRM_EINVAL for n < 0, null arrays, p <= 0 or NaN, or an unknown dtype. */
nrm_status nrm_test_lp(nrm_dtype dtype, double p, const void *x, const void *y, void *out, int64_t n, void *stream);

/* Test hook: the combine the xNRMP tree kernels apply for this p, elementwise:
 * out[i] = K_p(x[i], y[i]) with K_2 = v1_hypot (Listing 2), K_1 = |x| + |y|
 * (Eq. vp1), K_p = max(|x|, |y|) for p at or above the cut-off p' (Eq. vpI,
 * Section 4) and v1_lp (Listing 5) otherwise, in the forms the kernels use
 * (binary64 v1_hypot and v1_lp without the FP64 divide, square root and
 * pow).  Device arrays of n elements of
 * `dtype`; asynchronous on `stream`; NRM_EINVAL for n < 0, null arrays,
 * p <= 0 or NaN, or an unknown dtype. */
nrm_status nrm_test_combine(nrm_dtype dtype, double p, const void *x, const void *y, void *out, int64_t n,
                            void *stream);

/* Test hook: exhaustive checks of the steps of the branch-free binary32
 * v1_hypot (Listing 2) that the tree kernels use on checked groups, against
 * the correctly rounded operations.  mode 0: the square root on the
 * 2^23 + 1 values S in [1, 2] (index i: S = 1 + i 2^-23); mode 1: the FP32
 * reciprocal estimate's exact scaling with the exponent e in [-88, 124]
 * (index i: significand i mod 2^23, e = i / 2^23 - 88); mode 2: the division
 * on the 2^46 significand pairs (index i: a = 1 + (i / 2^23) 2^-23,
 * b = 1 + (i mod 2^23) 2^-23).  Checks indices [start, start + count);
 * mismatches are added to *bad (device) and the operands of one of them
 * stored in example[0..1] (device).  Asynchronous; NRM_EINVAL for a bad mode
 * or null pointers. */
nrm_status nrm_test_k1f_exhaustive(int32_t mode, uint64_t start, uint64_t count, unsigned long long *bad,
                                   float *example, void *stream);
/* (mode 3 of nrm_test_k1f_exhaustive: the same square root on the 3 2^23
 * values S in [1, 8), index i: S = (1 + (i mod 2^23) 2^-23) 2^(i / 2^23),
 * the range K2's binary32 form uses.) */

/* Test hook: K2 (see nrmf_es_*) elementwise in the general form the trees
 * use outside checked groups: out[i] = K2(x[i], y[i]) on device arrays of n
 * elements of `dtype`.  Asynchronous; NRM_EINVAL for n < 0, null arrays or
 * an unknown dtype. */
nrm_status nrm_test_k2(nrm_dtype dtype, const void *x, const void *y, void *out, int64_t n, void *stream);

/* Test hook: the branch-free binary64 K2 of the checked groups (integer
 * square root, exact scalings) against the general form (FP64 square root)
 * on n operand pairs of family `mode` (the families of
 * nrm_test_k1d_compare), for the pairs inside its range [2^-500, 2^502);
 * bitwise differences are added to *bad and one of them stored in
 * example[0..3] (x, y, both results; device pointers).  Asynchronous. */
nrm_status nrm_test_k2d_compare(uint64_t seed, int64_t n, int32_t mode, unsigned long long *bad, double *example,
                                void *stream);

/* Test hook: copy the first `count` ticket counters of the context's
 * workspace to host memory (synchronous).  Between calls they are all zero. */
nrm_status nrm_test_read_tickets(const nrm_ctx *ctx, uint32_t *host, int64_t count);

/*
 * Measurement hook (the paper has no counterpart): a register-only
 * throughput probe of one SM pipe, with which the benchmark measures the
 * ceiling it holds the tree kernels to instead of assuming a nominal rate.
 *   kind          : 0 = binary64 fma (DFMA), 1 = binary64 multiply (DMUL),
 *                   2 = binary32 fma (FFMA);
 *   iters         : >= 1; every thread runs 8 independent dependency chains
 *                   of 4 iters operations each;
 *   blocks_per_sm : 1..8 blocks of 256 threads per SM of the current device;
 *   sink          : device pointer to one double, never written in practice
 *                   (it keeps the chains alive through the optimiser);
 *   thread_ops    : host pointer (may be NULL) that receives the number of
 *                   operations the launch performs.
 * Asynchronous on `stream`; time it with CUDA events on that stream.
 * Errors: NRM_EINVAL for a bad kind, iters < 1, blocks_per_sm outside 1..8
 * or sink == NULL; NRM_EDEVICE without a current device.
 */
nrm_status nrm_probe_pipe(int32_t kind, int64_t iters, int32_t blocks_per_sm, double *sink, int64_t *thread_ops,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NRM_H */
