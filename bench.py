#!/usr/bin/env python3
"""Benchmark: DNRMF and SNRMF on single vectors of n = 2^28 elements.

One step is one pass of the hot path over one batch of synthetic input:
xNRMF of a binary64 vector of 2^28 elements (2 GiB) followed by xNRMF of a
binary32 vector of 2^28 elements (1 GiB), both resident in HBM (together 24x
the L2, so no flush is needed between steps).  The metric is GB/s of input
consumed per second of device time.

Printed as one JSON line (rank 0):
  value      whole-job GB/s (all ranks) with inputs already in HBM;
  e2e        the same metric through the C ABI's host-buffer entry point
             (nrm_host: pinned host input, chunked H2D copies overlapped with
             the tree, result read back), copies inside the timed region;
  roofline   for the dominant kernel (the binary64 tree kernel): the slowest
             of four floors -- its bytes at the measured HBM copy rate, its
             FP64 instructions (one DFMA and one DMUL per v1_hypot) at the
             FP64 rate measured here by a register-only probe, its
             thread-instructions (ncu count per element) at the issue rate
             of 4 warp-instructions per SM per clock, and its ALU-pipe
             instructions (ncu count) at 64 lanes per SM per clock --
             against its CUDA-event launch time;
  cpu_baseline  the C oracle on the same step, on all host cores (its thread
             driver) and on one;
  parts      per-precision figures, the hypot variants, config 0 (one FP64
             vector of 2^20: median launch and end-to-end latency), config 2
             (4096 ragged vectors, lengths log-uniform in [1, 2^18]: graph
             replay of the persistent launch against one launch per vector,
             both captured in CUDA graphs), config 3 (1024 vectors of 2^16,
             p in {1, 1.5, 3, 7.5}, one batch per p and one with a p per
             vector) and config 4 (the serving trace: Poisson arrivals at
             50k/s for 60 s through the continuous-batching server, the
             one-request-per-launch form on a prefix, the closed-loop
             capacity and a run below it).
Multi-GPU (torchrun): every rank computes its own pair of vectors (seed
1 + rank); there is no data-path collective ("weak" scaling).
The headline vectors run on a context of their own (work items of 2^8 rows,
what nrm_tune picks for one vector of 2^28 in either precision); the other configs
use the library's defaults or contexts autotuned for their shapes.
--impl reference times the oracle (the reference arm) on a bounded sample
of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 28
BYTES_D = N * 8
BYTES_S = N * 4
METRIC = "DNRMF+SNRMF GB/s at n=2^28 (FP64 2 GiB + FP32 1 GiB per step)"
WORKLOAD = ("xNRMF of one FP64 and one FP32 vector of n=2^28 each, x_i = s*m*2^e, s=+-1, m uniform in [1,2), "
            "e uniform in [-20,20], seed 1 (+rank)")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Figures from ncu captures of the kernel build they were taken on (their
# summaries are committed beside the code); set the flag to False whenever
# the binary64 tree kernel changes, and re-capture.
NCU_VALID = True
TRAFFIC_D_2E28 = 2149.612544e6 + 45.566976e6  # DNRMF: DRAM read + write of one launch at n = 2^28
TRAFFIC_S_2E28 = 1079.169280e6 + 18.969856e6  # SNRMF: the same
INST_PER_ELEM_D = 141.3  # DNRMF: smsp__inst_executed.sum x 32 / n at n = 2^26 (thread-instructions per element)
ALU_PER_ELEM_D = 72.86   # DNRMF: sm__inst_executed_pipe_alu.sum x 32 / n at n = 2^26 (the ALU pipe: 64 lanes an SM)
ALU_PER_SM_CLK = 64
FP64_PER_COMBINE_D = 2   # DNRMF: one DFMA (S = 1 + Q^2) and one DMUL (h = M s) per v1_hypot
ISSUE_PER_SM_CLK = 4 * 32  # thread-instructions an SM issues per clock (4 schedulers x 1 warp-instruction)

SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + SMI_FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [t.strip() for t in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        top = max(sm)
        loaded = [v for v in sm if v >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def aggregate(total_ms, world, steps, bytes_per_step, pg=None, device=None):
    """Whole-job figures across ranks: every rank runs its own problem
    (weak scaling, no data-path collective); the step time is the MAX over
    ranks of each rank's timed region and the value counts the bytes of all
    ranks.  Returns (max_total_ms, value_GBps)."""
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps * bytes_per_step / (total_ms * 1e-3) / 1e9


def run_reference(args):
    """The oracle (plain serial C) on a bounded sample of the workload, on
    all host cores: each step computes xNRMF of the first 2^26 elements of
    the FP64 and of the FP32 vector (the same generator) with the oracle's
    thread driver (the top splits of the same tree on separate threads)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2509_06220_gb300 import inputs
    ns = 1 << 26
    nproc = os.cpu_count() or 1
    threads = 1 << max(0, (nproc - 1).bit_length()) if nproc > 1 else 1
    xd = inputs.vector(ns, seed=1, vec=0, dtype=np.float64)
    xs = inputs.vector(ns, seed=1, vec=0, dtype=np.float32)
    for _ in range(args.warmup):
        oracle.nrm_par(xd, threads=threads)
        oracle.nrm_par(xs, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.nrm_par(xd, threads=threads)
        oracle.nrm_par(xs, threads=threads)
    dt = time.perf_counter() - t0
    gbs = args.steps * ns * 12 / dt / 1e9
    sample = ("first 2^26 elements of each vector per step (FP64 + FP32), oracle thread driver on %d threads "
              "(%d host cores, %s)" % (threads, nproc, cpu_model()))
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "sample_n": ns},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.split(":")[0].strip() in ("Model name", "Model"):
                v = l.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu part")):
                return l.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def event_ms(torch, fn, reps):
    """Average device time of fn() over reps calls, CUDA events on the
    current stream, after one untimed call."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def roofline_d(ms, n, fp64_rate, fp64_src, hbm_gbs, hbm_src, sms, sm_mhz):
    """The roofline of one DNRMF launch of n elements taking ms: the slowest
    of its floors (HBM bytes, FP64 instructions, issued instructions, ALU-pipe
    instructions); the fraction is that floor's time over the launch time."""
    floors = {"hbm": n * 8 / (hbm_gbs * 1e9) * 1e3,
              "fp64_pipe": FP64_PER_COMBINE_D * (n - 1) / fp64_rate * 1e3,
              "issue": INST_PER_ELEM_D * n / (sms * ISSUE_PER_SM_CLK * sm_mhz * 1e6) * 1e3,
              "alu_pipe": ALU_PER_ELEM_D * n / (sms * ALU_PER_SM_CLK * sm_mhz * 1e6) * 1e3}
    if not NCU_VALID:
        floors.pop("issue")
        floors.pop("alu_pipe")
    bind = max(floors, key=floors.get)
    if bind == "hbm":
        r = {"bound": "hbm", "achieved": n * 8 / (ms * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
             "peak_source": hbm_src}
    elif bind == "fp64_pipe":
        r = {"bound": "alu", "achieved": FP64_PER_COMBINE_D * (n - 1) / (ms * 1e-3) / 1e9, "peak": fp64_rate / 1e9,
             "unit": "G FP64 instructions/s (DFMA + DMUL, one each per v1_hypot)", "peak_source": fp64_src}
    elif bind == "issue":
        r = {"bound": "alu", "achieved": INST_PER_ELEM_D * n / (ms * 1e-3) / 1e9,
             "peak": sms * ISSUE_PER_SM_CLK * sm_mhz / 1e3,
             "unit": "G thread-instructions/s issued (%.1f per element, ncu)" % INST_PER_ELEM_D,
             "peak_source": "%d SMs x 4 warp-instructions per clock x %.0f MHz (the maximum SM clock)" % (sms, sm_mhz)}
    else:
        r = {"bound": "alu", "achieved": ALU_PER_ELEM_D * n / (ms * 1e-3) / 1e9,
             "peak": sms * ALU_PER_SM_CLK * sm_mhz / 1e3,
             "unit": "G thread-instructions/s on the ALU pipe (%.2f per element, ncu)" % ALU_PER_ELEM_D,
             "peak_source": "%d SMs x 64 ALU lanes x %.0f MHz (the maximum SM clock)" % (sms, sm_mhz)}
    r["frac"] = r["achieved"] / r["peak"]
    r["binding_floor"] = bind
    r["floors_ms"] = floors
    r["launch_ms"] = ms
    return r


def time_config0(nrm, torch, ctx, dev):
    """Config 0: DNRMF on one FP64 vector of 2^20 (seed 0): the median of 200
    launches timed one by one with CUDA events, and the median end-to-end
    latency of 100 calls through the host-buffer entry point (pinned input,
    result on the host), both bitwise against the oracle."""
    import numpy as np

    import oracle
    n = 1 << 20
    x = nrm.nrm_gen(n, 0, 0, torch.float64, device=dev)
    out = torch.empty((), dtype=torch.float64, device=dev)
    for _ in range(5):
        nrm.nrmf(x, out=out, ctx=ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        nrm.nrmf(x, out=out, ctx=ctx)
        b.record()
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    hx = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hx.copy_(x)
    lat = []
    for i in range(105):
        t0 = time.perf_counter()
        v = nrm.nrm_host(hx, ctx=ctx, device=dev.index or 0)
        if i >= 5:
            lat.append((time.perf_counter() - t0) * 1e3)
    lat.sort()
    want = oracle.nrm(hx.numpy())
    return {"n": n, "launches": len(ms), "median_ms": ms[len(ms) // 2], "p10_ms": ms[len(ms) // 10],
            "p90_ms": ms[9 * len(ms) // 10], "GBps_median": n * 8 / (ms[len(ms) // 2] * 1e-3) / 1e9,
            "e2e_calls": len(lat), "e2e_median_ms": lat[len(lat) // 2], "e2e_p90_ms": lat[9 * len(lat) // 10],
            "bitwise_equal_oracle": bool(np.float64(out.item()).tobytes() == want.tobytes()
                                         and np.float64(v).tobytes() == want.tobytes())}


def time_batch(nrm, torch, ctx, dev):
    """Config 2: a ragged batch of 4096 vectors, lengths log-uniform in
    [1, 2^18], FP64 and FP32: replays of the captured persistent launch
    against the 4096 single-vector launches captured into one CUDA graph
    (so neither side pays host launch overhead), bitwise equal."""
    import numpy as np

    from paper_2509_06220_gb300 import inputs
    L = inputs.ragged_lengths(4096, seed=0)
    off = np.zeros(4097, np.int64)
    np.cumsum(L, out=off[1:])
    offd = torch.from_numpy(off).to(dev)
    out = {}
    for name, td in (("f64", torch.float64), ("f32", torch.float32)):
        x = nrm.nrm_gen_ragged(offd, seed=0, dtype=td)
        # the batch runs on a context autotuned for this shape (group size,
        # warps per block, item depth, blocks per SM); the one-launch-per-
        # vector form keeps the single-vector tuning of `ctx`
        bctx = nrm.Context(0)
        tuned = bctx.autotune(nrm.NRM_F64 if td == torch.float64 else nrm.NRM_F32, L)
        g = nrm.nrm_batch_graph(x, offd, ctx=bctx)
        t_graph = event_ms(torch, g.launch, 20)
        single = torch.empty(4096, dtype=td, device=dev)
        views = [x[off[i]:off[i + 1]] for i in range(4096)]

        def singles():
            for i in range(4096):
                nrm.nrmf(views[i], out=single[i], ctx=ctx)

        singles()  # sizes the workspace before the capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        singles()
        torch.cuda.synchronize()
        t_loop = (time.perf_counter() - t0) * 1e3
        cg = torch.cuda.CUDAGraph()
        form = "4096 nrmf_* launches captured in one CUDA graph"
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                with torch.cuda.graph(cg, stream=s, capture_error_mode="thread_local"):
                    singles()
            torch.cuda.synchronize()
            t_single = event_ms(torch, cg.replay, 3)
        except RuntimeError as e:  # capture refused: time the launches from the host loop instead
            form = "4096 nrmf_* launches from a host loop (graph capture failed: %s)" % str(e)[:120]
            t_single = t_loop
        same = bool(torch.equal(single.view(torch.int64 if td == torch.float64 else torch.int32),
                                g.out.view(torch.int64 if td == torch.float64 else torch.int32)))
        out["batch_" + name] = {"norms_per_s": 4096 / (t_graph * 1e-3), "ms_per_batch": t_graph,
                                "elements": int(off[-1]), "GBps": off[-1] * x.element_size() / (t_graph * 1e-3) / 1e9,
                                "one_launch_per_vector_ms": t_single,
                                "one_launch_per_vector_norms_per_s": 4096 / (t_single * 1e-3),
                                "one_launch_per_vector_form": form,
                                "host_loop_ms": t_loop, "bitwise_equal_to_single": same, "tuning": tuned}
        del cg
        g.close()
        bctx.close()
        del x
    return out


def time_config3(nrm, torch, dev):
    """Config 3: batched xNRMP, 1024 vectors of 2^16 elements (e in [-8, 8]),
    FP64 and FP32, one captured batch per p in {1, 1.5, 3, 7.5} and one batch
    with the four p assigned per vector in turn (the p_dev form)."""
    import numpy as np
    B, n = 1024, 1 << 16
    off = torch.arange(0, (B + 1) * n, n, dtype=torch.int64, device=dev)
    res = {}
    for name, td in (("f64", torch.float64), ("f32", torch.float32)):
        x = nrm.nrm_gen_ragged(off, seed=3, dtype=td, emin=-8, emax=8)
        r = {}
        outs = {}
        for p in (1.0, 1.5, 3.0, 7.5):
            g = nrm.nrm_batch_graph(x, off, p)
            ms = event_ms(torch, g.launch, 10)
            outs[p] = g.out.clone()
            g.close()
            r["p=%g" % p] = {"ms": ms, "norms_per_s": B / (ms * 1e-3), "Gelem_per_s": B * n / (ms * 1e-3) / 1e9}
        pv = torch.tensor(np.tile([1.0, 1.5, 3.0, 7.5], B // 4), dtype=torch.float64, device=dev)
        g = nrm.nrm_batch_graph(x, off, pv)
        ms = event_ms(torch, g.launch, 10)
        mixed = g.out.clone()
        g.close()
        same = all(torch.equal(mixed[i::4], outs[p][i::4]) for i, p in enumerate((1.0, 1.5, 3.0, 7.5)))
        r["p_per_vector"] = {"ms": ms, "norms_per_s": B / (ms * 1e-3), "Gelem_per_s": B * n / (ms * 1e-3) / 1e9,
                             "bitwise_equal_to_one_p_batches": bool(same)}
        res[name] = r
        del x
    return res


def _replay(nrm, tr, nstreams, max_batch):
    srv = nrm.Server(budget_bytes=8 << 30, nstreams=nstreams, max_batch=max_batch)
    try:
        v, lat, rep = srv.replay(tr)
    finally:
        srv.close()
    return v, lat, rep


REPORT_KEYS = ("completed", "rejected", "max_queue", "steps", "launches", "p50_ms", "p99_ms", "mean_ms", "max_ms",
               "wall_s", "norms_per_s", "elements_per_s", "peak_bytes", "arena_bytes")


def _serve_summary(nrm, tr, lat, rep, window_s=10.0):
    import numpy as np
    rec = nrm.trace_records(tr)
    arr = rec["arrival_s"]
    out = {k: rep[k] for k in REPORT_KEYS}
    steps = max(rep["steps"], 1)
    out["host_launch_ms_per_step"] = rep["host_launch_s"] * 1e3 / steps
    out["host_retire_ms_per_step"] = rep["host_retire_s"] * 1e3 / steps
    out["host_us_per_request"] = (rep["host_launch_s"] + rep["host_retire_s"]) * 1e6 / max(rep["completed"], 1)
    out["gpu_ms_per_step"] = rep["gpu_step_s"] * 1e3 / steps
    out["requests_per_step"] = rep["completed"] / steps
    out["launches_per_step"] = rep["launches"] / steps
    T = float(arr[-1]) if arr.size else 0.0
    if T >= 2 * window_s:
        first = lat[arr < window_s]
        last = lat[arr >= T - window_s]
        p_first, p_last = float(np.percentile(first, 99)), float(np.percentile(last, 99))
        out["p99_first_%gs_ms" % window_s] = p_first
        out["p99_last_%gs_ms" % window_s] = p_last
        out["p99_bounded"] = bool(p_last <= 1.5 * p_first)
        # p99 of every window of arrivals, and the time of the slowest request
        edges = np.arange(0.0, T + window_s, window_s)
        out["p99_by_window_ms"] = [round(float(np.percentile(lat[(arr >= a) & (arr < a + window_s)], 99)), 3)
                                   for a in edges[:-1] if ((arr >= a) & (arr < a + window_s)).any()]
        out["max_latency_arrival_s"] = float(arr[int(np.argmax(lat))])
    return out


def time_serving(nrm, seconds, rate, baseline_seconds, saturation):
    """Config 4: Poisson arrivals at `rate`/s for `seconds`, lengths
    log-uniform in [2^4, 2^24], FP32/FP64 1:1, p = 2 (80 %) else 1.5 or 3;
    inputs generated on the device at admission; 8 GiB budget.  The trace
    through the continuous-batching server; the one-request-per-launch form
    on its first `baseline_seconds`; then the closed-loop capacity (a
    backlog of the trace's first 3 s, all arriving at once) and a 20 s run
    at 90 % of that capacity.  p99 is "bounded" when the p99 of the last
    10 s of arrivals (5 s for the 20 s run) is at most 1.5x that of the
    first."""
    import numpy as np
    res = {}
    tr = nrm.serving_trace(rate, seconds, seed=0)
    rec = nrm.trace_records(tr)
    v, lat, rep = _replay(nrm, tr, 4, 256)
    res["batched"] = _serve_summary(nrm, tr, lat, rep)
    nb = int(np.searchsorted(rec["arrival_s"], baseline_seconds))
    if nb > 0:
        pre = (nrm.Request * nb).from_buffer_copy(rec[:nb].tobytes())
        vb, latb, repb = _replay(nrm, pre, 1, 1)
        res["one_request_per_launch"] = _serve_summary(nrm, pre, latb, repb)
        res["one_request_per_launch"]["trace_prefix_s"] = baseline_seconds
        # the batched server on the same prefix alone, for the like-for-like p99
        vp, latp, repp = _replay(nrm, pre, 4, 256)
        res["batched_on_prefix"] = _serve_summary(nrm, pre, latp, repp)
        res["bitwise_equal"] = bool(vb.tobytes() == v[:nb].tobytes() == vp.tobytes())
    if saturation:
        nbk = int(np.searchsorted(rec["arrival_s"], min(3.0, seconds)))
        back = rec[:nbk].copy()
        back["arrival_s"] = 0.0
        bt = (nrm.Request * nbk).from_buffer_copy(back.tobytes())
        _, _, repc = _replay(nrm, bt, 4, 256)
        cap = repc["completed"] / max(repc["wall_s"], 1e-9)
        sat = {"closed_loop_norms_per_s": cap, "backlog_requests": nbk}
        r2 = 0.9 * cap
        tr2 = nrm.serving_trace(r2, 20.0, seed=1)
        _, lat2, rep2 = _replay(nrm, tr2, 4, 256)
        sat["run_at_90pct"] = dict(_serve_summary(nrm, tr2, lat2, rep2, window_s=5.0), rate_per_s=r2, seconds=20.0)
        res["saturation"] = sat
    L = rec["n"]
    res["trace"] = {"rate_per_s": rate, "seconds": seconds, "requests": len(tr), "mean_length": float(L.mean()),
                    "offered_elements_per_s": float(L.sum() / seconds)}
    return res


def run_capture(args):
    """The launches of one part of the benchmark alone, for ncu launch lists
    (prints one JSON line of its own timings; not a benchmark line)."""
    import numpy as np
    import torch

    import paper_2509_06220_gb300 as nrm
    from paper_2509_06220_gb300 import inputs
    dev = torch.device("cuda", 0)
    res = {"capture": args.capture}
    if args.capture == "batch":
        L = inputs.ragged_lengths(4096, seed=0)
        off = np.zeros(4097, np.int64)
        np.cumsum(L, out=off[1:])
        offd = torch.from_numpy(off).to(dev)
        for name, td, code in (("f64", torch.float64, nrm.NRM_F64), ("f32", torch.float32, nrm.NRM_F32)):
            x = nrm.nrm_gen_ragged(offd, seed=0, dtype=td)
            bctx = nrm.Context(0)
            tuned = bctx.autotune(code, L)
            g = nrm.nrm_batch_graph(x, offd, ctx=bctx)
            res[name] = {"tuning": tuned, "ms_per_batch": event_ms(torch, g.launch, max(args.steps, 1))}
            g.close()
            bctx.close()
    else:
        tr = nrm.serving_trace(args.serve_rate, args.serve_seconds, seed=0)
        back = nrm.trace_records(tr).copy()
        back["arrival_s"] = 0.0
        bt = (nrm.Request * len(back)).from_buffer_copy(back.tobytes())
        _, _, rep = _replay(nrm, bt, 4, 256)
        res["serve"] = {"requests": rep["completed"], "norms_per_s": rep["completed"] / max(rep["wall_s"], 1e-9),
                        "elements_per_s": rep["elements_per_s"]}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip configs 0, 2 and 3 and the hypot variants")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the serving trace (config 4 runs 60 s; 0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=50000.0)
    ap.add_argument("--serve-baseline-seconds", type=float, default=0.5,
                    help="prefix of the trace served one request per launch")
    ap.add_argument("--no-saturation", action="store_true")
    ap.add_argument("--log2n", type=int, default=28,
                    help="vector length 2^k (28 is the benchmark; smaller only for profiling captures)")
    ap.add_argument("--n", type=int, default=0,
                    help="vector length n, overriding --log2n (profiling captures of other shapes)")
    ap.add_argument("--p", type=float, default=2.0,
                    help="xNRMP with this p instead of xNRMF (profiling captures of the p-norm kernels; "
                         "the e2e, batch, serving and oracle legs and the v1_hypot roofline are left out)")
    ap.add_argument("--capture", default="", choices=["", "batch", "serve"],
                    help="profiling captures: 'batch' replays only the autotuned config-2 batch graphs (--steps "
                         "replays per type), 'serve' serves only a backlog of the config-4 trace's first "
                         "--serve-seconds seconds, all arriving at once")
    args = ap.parse_args()
    if args.capture:
        run_capture(args)
        return
    if args.p != 2.0:
        args.no_e2e = args.no_cpu_baseline = args.no_batch = True
        args.serve_seconds = 0
    global N, BYTES_D, BYTES_S
    N = args.n if args.n > 0 else 1 << args.log2n
    BYTES_D, BYTES_S = N * 8, N * 4
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    import paper_2509_06220_gb300 as nrm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            t = torch.zeros(1, device=dev)
            pg.all_reduce(t)
        torch.cuda.synchronize()

    ctx = nrm.context(local)
    # The headline vectors run on a context of their own: work items of 2^8
    # rows, 4 warps a block, up to 8 (binary64; its 80-register cap lets 6
    # reside) or 16 (binary32) blocks an SM, the settings sweeps at n = 2^28
    # and nrm_tune for one vector of 2^28 pick; the library defaults (items of
    # 2^7 rows, better for batches of shorter vectors) stay on `ctx` for
    # configs 0, 2 and 3.
    hctx = nrm.Context(local)
    hctx.set_tuning(group_log2=2, warps_per_block=4, item_log2=8, blocks_per_sm=8, dtype=nrm.NRM_F64)
    hctx.set_tuning(group_log2=2, warps_per_block=4, item_log2=8, blocks_per_sm=16, dtype=nrm.NRM_F32)
    # the FP64 pipe's measured rate (register-only DFMA chains), before the
    # timed region
    fp64_rate = nrm.probe_pipe(nrm.PIPE_DFMA, iters=4096, blocks_per_sm=8)
    seed = 1 + rank
    xd = nrm.nrm_gen(N, seed, 0, torch.float64, device=dev)
    xs = nrm.nrm_gen(N, seed, 0, torch.float32, device=dev)
    od = torch.empty((), dtype=torch.float64, device=dev)
    os_ = torch.empty((), dtype=torch.float32, device=dev)
    if args.p == 2.0:
        def step(x, o):
            nrm.nrmf(x, out=o, ctx=hctx)
    else:
        def step(x, o):
            nrm.nrmp(x, args.p, out=o, ctx=hctx)
    for _ in range(args.warmup):
        step(xd, od)
        step(xs, os_)
    torch.cuda.synchronize()

    K = args.steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    launches0 = hctx.launches
    with ClockSampler(local) as clk:
        barrier()
        evs[0].record()
        for i in range(K):
            step(xd, od)
            evs[2 * i + 1].record()
            step(xs, os_)
            evs[2 * i + 2].record()
        barrier()
    launches = hctx.launches - launches0
    total_ms = evs[0].elapsed_time(evs[2 * K])
    d_ms = [evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(K)]
    s_ms = [evs[2 * i + 1].elapsed_time(evs[2 * i + 2]) for i in range(K)]
    total_ms, value = aggregate(total_ms, world, K, BYTES_D + BYTES_S, pg, dev)
    ms_step = total_ms / K
    d_avg = statistics.mean(d_ms)
    s_avg = statistics.mean(s_ms)
    clocks = clk.summary()

    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    hbm_src = "measured hbm_gbs (copy)" if hbm_peak else "fallback 6800 GB/s"
    hbm_peak = hbm_peak or 6800.0
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    d_bytes_gbs = BYTES_D / (d_avg * 1e-3) / 1e9
    s_bytes_gbs = BYTES_S / (s_avg * 1e-3) / 1e9
    roof = roofline_d(d_avg, N, fp64_rate, "measured here: nrm_probe_pipe DFMA chains, %d SMs x 8 blocks" % sms,
                      hbm_peak, hbm_src, sms, sm_max)
    # DRAM bytes read+written per launch from an ncu capture at n = 2^28, in
    # proportion to n otherwise
    roof["traffic"] = TRAFFIC_D_2E28 * (N / float(1 << 28)) if NCU_VALID else None
    roof["kernel"] = "tree_kernel<double,%d,OpHypot>" % hctx.tuning_for(nrm.NRM_F64).group_log2
    roof["hbm_view"] = {"achieved": d_bytes_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": d_bytes_gbs / hbm_peak}
    roof["note"] = ("algorithmic view of Listing 2: 7 IEEE operations per v1_hypot = %.1f Gop/s; this kernel "
                    "computes the same correctly rounded results with integer/FP32 instructions plus one DFMA and "
                    "one DMUL, so the floors above price the instructions it executes" %
                    (7 * (N - 1) / (d_avg * 1e-3) / 1e9))
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "bytes_per_step": BYTES_D + BYTES_S,
                       "l2": "inputs (3 GiB) exceed the 129 MB L2; no flush", "parallelism": "replicas" if world > 1
                       else "single GPU"},
            "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
            "parts": {"dnrmf": {"ms": d_avg, "GBps": d_bytes_gbs, "Gelem_per_s": N / (d_avg * 1e-3) / 1e9,
                                "Ghypot_per_s": (N - 1) / (d_avg * 1e-3) / 1e9},
                      "snrmf": {"ms": s_avg, "GBps": s_bytes_gbs, "Gelem_per_s": N / (s_avg * 1e-3) / 1e9,
                                "hbm_frac": s_bytes_gbs / hbm_peak,
                                "traffic": TRAFFIC_S_2E28 * (N / float(1 << 28)) if NCU_VALID else None},
                      "fp64_probe_Gops": fp64_rate / 1e9}}
    if args.p != 2.0:
        # a p-norm capture: the roofline above prices v1_hypot
        line["config"]["p"] = args.p
        line["roofline"] = None

    # the other hypot variants on the same vectors (not the headline): Z with
    # A for the final reduction, and the exponent-scaled hypotenuse K2
    if rank == 0 and not args.no_batch:
        variants = {}
        vod, vos = torch.empty_like(od), torch.empty_like(os_)
        for name, fn in (("za", nrm.nrmf_za), ("es", nrm.nrmf_es)):
            for tag, x, o in (("d", xd, vod), ("s", xs, vos)):
                ms = event_ms(torch, lambda: fn(x, out=o, ctx=hctx), 5)
                variants["%snrmf_%s" % (tag, name)] = {"ms": ms, "GBps": N * x.element_size() / (ms * 1e-3) / 1e9}
        line["parts"]["variants"] = variants

    # end to end through the host-buffer entry point
    if not args.no_e2e:
        hd = torch.empty(N, dtype=torch.float64, pin_memory=True)
        hs = torch.empty(N, dtype=torch.float32, pin_memory=True)
        hd.copy_(xd)
        hs.copy_(xs)
        nrm.nrm_host(hd, ctx=hctx, device=local)
        nrm.nrm_host(hs, ctx=hctx, device=local)
        reps = 5
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            vd = nrm.nrm_host(hd, ctx=hctx, device=local)
            vs = nrm.nrm_host(hs, ctx=hctx, device=local)
        barrier()
        te = time.perf_counter() - t0
        if pg is not None:
            t = torch.tensor([te], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            te = float(t.item())
        line["e2e"] = {"value": world * reps * (BYTES_D + BYTES_S) / te / 1e9, "unit": "GB/s",
                       "h2d_bytes_per_step": BYTES_D + BYTES_S, "d2h_bytes_per_step": 12,
                       "ms_per_step": te / reps * 1e3}
        assert np.float64(vd).tobytes() == np.float64(od.item()).tobytes()
        del hd, hs

    if not args.no_batch and rank == 0:
        line["parts"]["config0"] = time_config0(nrm, torch, ctx, dev)
        line["parts"].update(time_batch(nrm, torch, ctx, dev))
        line["parts"]["config3"] = time_config3(nrm, torch, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        hxd = xd.cpu().numpy()
        hxs = xs.cpu().numpy()
        nproc = os.cpu_count() or 1
        t0 = time.perf_counter()
        vd = oracle.nrm_par(hxd, threads=nproc)
        vs = oracle.nrm_par(hxs, threads=nproc)
        tp = time.perf_counter() - t0
        t0 = time.perf_counter()
        vd1 = oracle.nrm(hxd)
        vs1 = oracle.nrm(hxs)
        tc = time.perf_counter() - t0
        same = (vd.tobytes() == vd1.tobytes() == np.float64(od.item()).tobytes()
                and vs.tobytes() == vs1.tobytes() == np.float32(os_.item()).tobytes())
        line["cpu_baseline"] = {"value": (BYTES_D + BYTES_S) / tp / 1e9, "unit": "GB/s",
                                "cores": 1 << max(0, (nproc - 1).bit_length()) if nproc > 1 else 1,
                                "kind": "oracle", "nproc": nproc, "cpu_model": cpu_model(),
                                "sample": "one full step (FP64 and FP32 vectors of 2^28) by the oracle's thread "
                                          "driver (the top splits of the same tree on separate threads), %.2f s" % tp,
                                "single_core": {"value": (BYTES_D + BYTES_S) / tc / 1e9, "unit": "GB/s",
                                                "cores": 1, "seconds": tc},
                                "bitwise_equal": bool(same)}
    if args.serve_seconds > 0 and rank == 0:
        del xd, xs
        torch.cuda.empty_cache()
        line["parts"]["serve"] = time_serving(nrm, args.serve_seconds, args.serve_rate, args.serve_baseline_seconds,
                                              not args.no_saturation)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
