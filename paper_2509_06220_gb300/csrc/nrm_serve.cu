// nrm_serve.cu -- continuous-batching request server for xNRMF / xNRMP.
//
// Requests (element type, p, length, input from the host or generated on the
// device) arrive at any time.  A worker thread runs the loop
//   retire finished steps -> admit waiting requests into free device memory
//   -> launch the next step on every idle stream,
// so requests that arrive while others are on the GPU join the next step as
// soon as memory frees up, and steps on different streams overlap on the
// device.  A step groups its requests by element type and computes each
// group with one segment batch (nrm_batch_segments, with one p per request
// when the group's p differ) over the request inputs, which live in one
// device arena: every result is bitwise the result of the same request
// computed alone (the tree depends on the vector and its p only).
//
// Memory: the budget covers the arena (inputs) and each stream's tree
// workspace, which is reserved up front so the loop never allocates.  A
// request larger than the arena is rejected at submission (NRM_EBUDGET);
// others wait in FIFO order until their input fits.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/nrm.h"
#include "nrm_internal.h"

namespace {

using clk = std::chrono::steady_clock;

double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// first-fit allocator over [0, size) in 256-byte units, coalescing on free
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    int64_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return (int64_t)off;
            }
        }
        return -1;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

struct Req {
    uint64_t id = 0;
    nrm_request r{};
    clk::time_point t_arrival;
    clk::time_point t_done;
    int64_t off = -1;    // arena byte offset of the input
    size_t res_byte = 0; // byte position of the result in the lane's output block
    double result = 0.0;
    int32_t status = NRM_OK;
    bool done = false;
};

size_t elem_size(nrm_dtype dt) { return dt == NRM_F64 ? 8 : 4; }
size_t req_bytes(const Req *q) { return (size_t)q->r.n * elem_size(q->r.dtype); }

struct Lane {
    nrm_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr; // timing: start and end of the step on the device
    double *h_p = nullptr, *d_p = nullptr;  // per-request p of a step (groups with mixed p)
    int64_t *h_starts = nullptr, *h_lens = nullptr, *d_starts = nullptr, *d_lens = nullptr;
    double *h_out = nullptr, *d_out = nullptr; // results widened per group slot (8 bytes each)
    int32_t *h_status = nullptr, *d_status = nullptr;
    NrmGenSeg *h_segs = nullptr, *d_segs = nullptr; // device-generated inputs of a step
    int64_t *h_cum = nullptr, *d_cum = nullptr;
    std::vector<Req *> batch;
    bool busy = false;
};

} // namespace

struct nrm_srv {
    int device = 0;
    int max_batch = 1024;
    size_t budget = 0, arena_bytes = 0;
    void *arena_ptr = nullptr;
    Arena arena;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<Req *> pending, admitted;
    // every request by id (ids are consecutive from 0); a deque grows without
    // the rehash pauses of a hash map, which stalled the loop for ~0.1 s once
    // a trace reached 1.5 M requests
    std::deque<Req *> reqs;
    uint64_t next_id = 0;
    std::thread worker;
    std::atomic<bool> stop{false};
    // statistics
    int64_t submitted = 0, rejected = 0, completed = 0; // under mu
    int64_t finished = 0;                               // under mu: requests done (completed or failed)
    double host_launch_s = 0, host_retire_s = 0, gpu_step_s = 0; // worker-written, read under mu
    std::atomic<int64_t> steps{0}, launches{0}, elements{0}, peak_bytes{0}; // worker-written
    int64_t max_queue = 0;
    std::deque<double> lat_ms;
    clk::time_point t_first, t_last;
    bool any = false;
    nrm_status fatal = NRM_OK;
};

namespace {

// results of a group of one element type are written as that type into the
// lane's d_out slots; widen them to double on the host
void retire(nrm_srv *s, Lane &ln) {
    const clk::time_point now = clk::now();
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ln.t0, ln.t1) == cudaSuccess) s->gpu_step_s += ms * 1e-3;
    for (size_t i = 0; i < ln.batch.size(); ++i) {
        Req *q = ln.batch[i];
        const char *src = (const char *)ln.h_out + q->res_byte;
        if (q->r.dtype == NRM_F64) std::memcpy(&q->result, src, sizeof(double));
        else {
            float f;
            std::memcpy(&f, src, sizeof(float));
            q->result = (double)f;
        }
        q->status = ln.h_status[i];
        q->t_done = now;
        q->done = true;
        if (q->off >= 0) s->arena.release((size_t)q->off, req_bytes(q));
        s->completed++;
        s->finished++;
        s->lat_ms.push_back(secs(q->t_arrival, now) * 1e3);
        s->t_last = now;
    }
    ln.batch.clear();
    ln.busy = false;
    s->host_retire_s += secs(now, clk::now());
    s->cv_done.notify_all();
}

nrm_status launch_step(nrm_srv *s, Lane &ln) {
    // take up to max_batch admitted requests, FIFO
    const size_t take = std::min(s->admitted.size(), (size_t)s->max_batch);
    ln.batch.assign(s->admitted.begin(), s->admitted.begin() + take);
    s->admitted.erase(s->admitted.begin(), s->admitted.begin() + take);
    // order by type so that each group is a contiguous slot range
    std::stable_sort(ln.batch.begin(), ln.batch.end(),
                     [](const Req *a, const Req *b) { return a->r.dtype < b->r.dtype; });
    if (cudaEventRecord(ln.t0, ln.stream) != cudaSuccess) return NRM_ECUDA;
    const size_t B = ln.batch.size();
    int64_t ng = 0, gtotal = 0;
    for (size_t i = 0; i < B; ++i) {
        Req *q = ln.batch[i];
        const size_t es = elem_size(q->r.dtype);
        ln.h_starts[i] = q->r.n > 0 ? q->off / (int64_t)es : 0;
        ln.h_lens[i] = q->r.n;
        ln.h_p[i] = q->r.p;
        s->elements += q->r.n;
        if (q->r.n == 0) continue;
        if (q->r.x_host) {
            void *dst = (char *)s->arena_ptr + q->off;
            if (cudaMemcpyAsync(dst, q->r.x_host, req_bytes(q), cudaMemcpyHostToDevice, ln.stream) != cudaSuccess)
                return NRM_ECUDA;
        } else {
            NrmGenSeg &g = ln.h_segs[ng];
            g.start = ln.h_starts[i];
            g.n = q->r.n;
            g.key = nrm_gen_key(q->r.seed, q->id);
            g.emin = q->r.emin;
            g.span = q->r.emax - q->r.emin + 1;
            g.dtype = q->r.dtype;
            ln.h_cum[ng] = gtotal;
            gtotal += q->r.n;
            ++ng;
        }
    }
    if (cudaMemcpyAsync(ln.d_starts, ln.h_starts, B * sizeof(int64_t), cudaMemcpyHostToDevice, ln.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(ln.d_lens, ln.h_lens, B * sizeof(int64_t), cudaMemcpyHostToDevice, ln.stream) != cudaSuccess ||
        cudaMemcpyAsync(ln.d_p, ln.h_p, B * sizeof(double), cudaMemcpyHostToDevice, ln.stream) != cudaSuccess)
        return NRM_ECUDA;
    if (ng > 0) {
        if (cudaMemcpyAsync(ln.d_segs, ln.h_segs, (size_t)ng * sizeof(NrmGenSeg), cudaMemcpyHostToDevice, ln.stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(ln.d_cum, ln.h_cum, (size_t)ng * sizeof(int64_t), cudaMemcpyHostToDevice, ln.stream) !=
                cudaSuccess)
            return NRM_ECUDA;
        nrm_status st = nrm_gen_segments(ln.d_segs, ln.d_cum, ng, gtotal, s->arena_ptr, ln.stream);
        if (st != NRM_OK) return st;
    }
    size_t g0 = 0;
    while (g0 < B) {
        size_t g1 = g0 + 1;
        bool one_p = true; // every request of the group has the same p: no per-vector p needed
        while (g1 < B && ln.batch[g1]->r.dtype == ln.batch[g0]->r.dtype) {
            one_p = one_p && ln.batch[g1]->r.p == ln.batch[g0]->r.p;
            ++g1;
        }
        const nrm_dtype dt = ln.batch[g0]->r.dtype;
        const size_t es = elem_size(dt);
        // the group's results are packed values of type dt starting at byte
        // 8 g0 of the output block (it has 8 bytes per request)
        for (size_t j = g0; j < g1; ++j) ln.batch[j]->res_byte = g0 * 8 + (j - g0) * es;
        nrm_status st = nrm_batch_segments(ln.ctx, dt, s->arena_ptr, (int64_t)(s->arena_bytes / es),
                                           ln.d_starts + g0, ln.d_lens + g0, (int64_t)(g1 - g0), ln.batch[g0]->r.p,
                                           one_p ? nullptr : ln.d_p + g0, (char *)ln.d_out + g0 * 8,
                                           ln.d_status + g0, ln.stream);
        if (st != NRM_OK) return st;
        s->launches += 2;
        g0 = g1;
    }
    if (cudaMemcpyAsync(ln.h_out, ln.d_out, B * 8, cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess ||
        cudaMemcpyAsync(ln.h_status, ln.d_status, B * sizeof(int32_t), cudaMemcpyDeviceToHost, ln.stream) !=
            cudaSuccess ||
        cudaEventRecord(ln.t1, ln.stream) != cudaSuccess || cudaEventRecord(ln.ev, ln.stream) != cudaSuccess)
        return NRM_ECUDA;
    ln.busy = true;
    s->steps++;
    return NRM_OK;
}

void worker_loop(nrm_srv *s) {
    cudaSetDevice(s->device);
    std::deque<Req *> waiting; // worker-owned FIFO of requests not yet admitted
    for (;;) {
        bool progress = false;
        // retire finished steps (request fields are read by poll: hold the lock)
        for (Lane &ln : s->lanes) {
            if (ln.busy && cudaEventQuery(ln.ev) == cudaSuccess) {
                std::lock_guard<std::mutex> lk(s->mu);
                retire(s, ln);
                progress = true;
            }
        }
        bool stopping;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->pending.empty()) {
                waiting.push_back(s->pending.front());
                s->pending.pop_front();
            }
            stopping = s->stop.load();
        }
        // admit in FIFO order while the inputs fit (arena: worker only)
        while (!waiting.empty()) {
            Req *q = waiting.front();
            const int64_t off = q->r.n > 0 ? s->arena.alloc(req_bytes(q)) : 0;
            if (off < 0) break;
            q->off = q->r.n > 0 ? off : -1;
            s->admitted.push_back(q);
            waiting.pop_front();
            progress = true;
        }
        s->peak_bytes.store((int64_t)s->arena.peak());
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->max_queue = std::max<int64_t>(s->max_queue, (int64_t)waiting.size());
        }
        for (Lane &ln : s->lanes) {
            if (!ln.busy && !s->admitted.empty()) {
                const clk::time_point h0 = clk::now();
                nrm_status st = launch_step(s, ln);
                const double hs = secs(h0, clk::now());
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->host_launch_s += hs;
                }
                if (st != NRM_OK) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->fatal = st;
                    for (Req *q : ln.batch) {
                        q->status = st;
                        q->done = true;
                        q->t_done = clk::now();
                        s->finished++;
                    }
                    ln.batch.clear();
                    s->cv_done.notify_all();
                }
                progress = true;
            }
        }
        bool idle = waiting.empty() && s->admitted.empty();
        for (Lane &ln : s->lanes) idle = idle && !ln.busy;
        if (stopping && idle) {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->pending.empty()) return;
        }
        if (!progress) std::this_thread::yield();
    }
}

} // namespace

extern "C" nrm_status nrm_srv_create(nrm_srv **srv, int device, size_t budget_bytes, int nstreams, int max_batch) {
    if (!srv || nstreams < 1 || nstreams > 16 || max_batch < 1 || max_batch > (1 << 20)) return NRM_EINVAL;
    *srv = nullptr;
    nrm_srv *s = new nrm_srv();
    s->device = device;
    s->budget = budget_bytes;
    s->max_batch = max_batch;
    s->lanes.resize((size_t)nstreams);
    size_t reserved = 0;
    nrm_status st = NRM_OK;
    for (Lane &ln : s->lanes) {
        st = nrm_create(&ln.ctx, device);
        if (st != NRM_OK) break;
        // the steps' batches take items of 2^9 rows: the finer items of the
        // single-vector defaults would multiply the slot workspace that is
        // reserved below for every stream
        const nrm_tuning bt[2] = {nrm_tuning{2, 4, 9, 16}, nrm_tuning{2, 8, 9, 16}};
        nrm_set_tuning_for(ln.ctx, NRM_F32, &bt[0]);
        nrm_set_tuning_for(ln.ctx, NRM_F64, &bt[1]);
        // reserve the largest workspace a step can need: every element of
        // the arena in one batch of the narrowest type (most rows)
        const int64_t max_elems = (int64_t)(budget_bytes / 4);
        const size_t ws = std::max(nrm_batch_ws_bytes(ln.ctx, NRM_F32, max_elems, max_batch, true),
                                   nrm_batch_ws_bytes(ln.ctx, NRM_F64, max_elems / 2, max_batch, true));
        const int64_t tk = std::max(nrm_batch_tickets(ln.ctx, NRM_F32, max_elems, max_batch, true),
                                    nrm_batch_tickets(ln.ctx, NRM_F64, max_elems / 2, max_batch, true));
        st = nrm_ctx_ensure(ln.ctx, ws, tk);
        if (st != NRM_OK) break;
        reserved += ws + (size_t)tk * 4;
        if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&ln.t0) != cudaSuccess || cudaEventCreate(&ln.t1) != cudaSuccess ||
            cudaMallocHost(&ln.h_p, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMalloc(&ln.d_p, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMallocHost(&ln.h_starts, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMallocHost(&ln.h_lens, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMallocHost(&ln.h_out, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMallocHost(&ln.h_status, (size_t)max_batch * 4) != cudaSuccess ||
            cudaMalloc(&ln.d_starts, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMalloc(&ln.d_lens, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMalloc(&ln.d_out, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMalloc(&ln.d_status, (size_t)max_batch * 4) != cudaSuccess ||
            cudaMallocHost(&ln.h_segs, (size_t)max_batch * sizeof(NrmGenSeg)) != cudaSuccess ||
            cudaMallocHost(&ln.h_cum, (size_t)max_batch * 8) != cudaSuccess ||
            cudaMalloc(&ln.d_segs, (size_t)max_batch * sizeof(NrmGenSeg)) != cudaSuccess ||
            cudaMalloc(&ln.d_cum, (size_t)max_batch * 8) != cudaSuccess) {
            cudaGetLastError();
            st = NRM_ENOMEM;
            break;
        }
        reserved += (size_t)max_batch * (20 + 8 + 8 + sizeof(NrmGenSeg));
    }
    if (st == NRM_OK) {
        if (reserved + (1u << 20) > budget_bytes) st = NRM_EBUDGET; // no room left for inputs
        else {
            s->arena_bytes = (budget_bytes - reserved) & ~size_t(255);
            if (cudaMalloc(&s->arena_ptr, s->arena_bytes) != cudaSuccess) {
                cudaGetLastError();
                st = NRM_ENOMEM;
            }
        }
    }
    if (st != NRM_OK) {
        nrm_srv_destroy(s);
        return st;
    }
    s->arena.reset(s->arena_bytes);
    s->worker = std::thread(worker_loop, s);
    *srv = s;
    return NRM_OK;
}

extern "C" nrm_status nrm_srv_destroy(nrm_srv *s) {
    if (!s) return NRM_OK;
    if (s->worker.joinable()) {
        s->stop.store(true);
        s->worker.join();
    }
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (Lane &ln : s->lanes) {
        if (ln.ev) cudaEventDestroy(ln.ev);
        if (ln.t0) cudaEventDestroy(ln.t0);
        if (ln.t1) cudaEventDestroy(ln.t1);
        if (ln.h_p) cudaFreeHost(ln.h_p);
        if (ln.d_p) cudaFree(ln.d_p);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.h_starts) cudaFreeHost(ln.h_starts);
        if (ln.h_lens) cudaFreeHost(ln.h_lens);
        if (ln.h_out) cudaFreeHost(ln.h_out);
        if (ln.h_status) cudaFreeHost(ln.h_status);
        if (ln.d_starts) cudaFree(ln.d_starts);
        if (ln.d_lens) cudaFree(ln.d_lens);
        if (ln.d_out) cudaFree(ln.d_out);
        if (ln.d_status) cudaFree(ln.d_status);
        if (ln.h_segs) cudaFreeHost(ln.h_segs);
        if (ln.h_cum) cudaFreeHost(ln.h_cum);
        if (ln.d_segs) cudaFree(ln.d_segs);
        if (ln.d_cum) cudaFree(ln.d_cum);
        if (ln.ctx) nrm_destroy(ln.ctx);
    }
    if (s->arena_ptr) cudaFree(s->arena_ptr);
    for (Req *q : s->reqs) delete q;
    delete s;
    return NRM_OK;
}

static nrm_status submit_at(nrm_srv *s, const nrm_request *r, clk::time_point t_arrival, uint64_t *id) {
    if (!s || !r || r->n < 0 || (r->dtype != NRM_F32 && r->dtype != NRM_F64) || !(r->p > 0.0)) return NRM_EINVAL;
    if (r->dtype == NRM_F32 && !((float)r->p > 0.0f)) return NRM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->any) {
        s->t_first = t_arrival;
        s->any = true;
    }
    s->submitted++;
    if ((size_t)r->n * elem_size(r->dtype) > s->arena_bytes) { // can never fit
        s->rejected++;
        return NRM_EBUDGET;
    }
    Req *q = new Req();
    q->id = s->next_id++;
    q->r = *r;
    q->t_arrival = t_arrival;
    s->reqs.push_back(q); // at index q->id
    s->pending.push_back(q);
    if (id) *id = q->id;
    return NRM_OK;
}

extern "C" nrm_status nrm_srv_submit(nrm_srv *s, const nrm_request *r, uint64_t *id) {
    return submit_at(s, r, clk::now(), id);
}

extern "C" nrm_status nrm_srv_poll(nrm_srv *s, uint64_t id, double *norm, int32_t *status, int32_t *done) {
    if (!s || !done) return NRM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= (uint64_t)s->reqs.size()) return NRM_EINVAL;
    const Req *q = s->reqs[(size_t)id];
    *done = q->done ? 1 : 0;
    if (q->done) {
        if (norm) *norm = q->result;
        if (status) *status = q->status;
    }
    return NRM_OK;
}

extern "C" nrm_status nrm_srv_drain(nrm_srv *s, double timeout_s) {
    if (!s) return NRM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    while (s->finished < (int64_t)s->reqs.size()) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return NRM_ETIMEOUT;
    }
    return s->fatal;
}

extern "C" nrm_status nrm_srv_report_get(nrm_srv *s, nrm_srv_report *rep) {
    if (!s || !rep) return NRM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(rep, 0, sizeof(*rep));
    rep->submitted = s->submitted;
    rep->rejected = s->rejected;
    rep->completed = s->completed;
    rep->admitted = s->submitted - s->rejected;
    rep->steps = s->steps.load();
    rep->launches = s->launches.load();
    rep->max_queue = s->max_queue;
    rep->peak_bytes = s->peak_bytes.load();
    rep->arena_bytes = (int64_t)s->arena_bytes;
    rep->host_launch_s = s->host_launch_s;
    rep->host_retire_s = s->host_retire_s;
    rep->gpu_step_s = s->gpu_step_s;
    std::vector<double> v(s->lat_ms.begin(), s->lat_ms.end());
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        rep->p50_ms = pct(0.50);
        rep->p99_ms = pct(0.99);
        rep->max_ms = v.back();
        double sum = 0;
        for (double d : v) sum += d;
        rep->mean_ms = sum / (double)v.size();
    }
    if (s->any && s->completed > 0) {
        rep->wall_s = secs(s->t_first, s->t_last);
        if (rep->wall_s > 0) {
            rep->norms_per_s = (double)s->completed / rep->wall_s;
            rep->elements_per_s = (double)s->elements.load() / rep->wall_s;
        }
    }
    return NRM_OK;
}

extern "C" nrm_status nrm_srv_replay(nrm_srv *s, const nrm_request *reqs, int64_t count, double *norms,
                                     double *latency_ms, nrm_srv_report *rep) {
    if (!s || (count > 0 && !reqs)) return NRM_EINVAL;
    std::vector<uint64_t> ids((size_t)count, UINT64_MAX);
    const clk::time_point t0 = clk::now();
    for (int64_t i = 0; i < count; ++i) {
        const clk::time_point ta =
            t0 + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(reqs[i].arrival_s));
        while (clk::now() < ta) {
        }
        uint64_t id = 0;
        if (submit_at(s, &reqs[i], ta, &id) == NRM_OK) ids[(size_t)i] = id;
    }
    nrm_status st = nrm_srv_drain(s, 3600.0);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int64_t i = 0; i < count; ++i) {
            const uint64_t id = ids[(size_t)i];
            Req *q = id == UINT64_MAX ? nullptr : s->reqs[(size_t)id];
            if (norms) norms[i] = q ? q->result : __builtin_nan("");
            if (latency_ms) latency_ms[i] = q ? secs(q->t_arrival, q->t_done) * 1e3 : -1.0;
        }
    }
    if (rep) nrm_srv_report_get(s, rep);
    return st;
}
