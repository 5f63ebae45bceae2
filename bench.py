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
  roofline   for the dominant kernel (the binary64 tree kernel): its
             algorithmic work per launch over its CUDA-event launch time,
             against the measured or unit-count peak;
  cpu_baseline  the C oracle on the same step, single-threaded;
  parts      per-precision figures and the ragged-batch workload (4096
             vectors, log-uniform lengths in [1, 2^18]) as graph replays
             versus one launch per vector.
Multi-GPU (torchrun): every rank computes its own pair of vectors (seed
1 + rank); there is no data-path collective ("weak" scaling).
--impl reference times the oracle (the reference arm for this build) on a
bounded sample of the same workload on the host cores.
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
# the ncu traffic figures in profiles/ belong to the kernel build they were
# captured on; set to False whenever the binary64 tree kernel changes
TRAFFIC_VALID = True
TRAFFIC_D_2E28 = 2149.706496e6 + 27.048448e6  # DNRMF: DRAM read + write of one launch at n = 2^28
TRAFFIC_S_2E28 = 1075.587584e6 + 8.574976e6  # SNRMF: the same

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
    """The oracle (plain serial C) on a bounded sample of the workload:
    each step computes xNRMF of the first 2^25 elements of the FP64 and of
    the FP32 vector (the same generator), single-threaded."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2509_06220_gb300 import inputs
    ns = 1 << 25
    xd = inputs.vector(ns, seed=1, vec=0, dtype=np.float64)
    xs = inputs.vector(ns, seed=1, vec=0, dtype=np.float32)
    for _ in range(args.warmup):
        oracle.nrm(xd)
        oracle.nrm(xs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.nrm(xd)
        oracle.nrm(xs)
    dt = time.perf_counter() - t0
    gbs = args.steps * ns * 12 / dt / 1e9
    sample = "first 2^25 elements of each vector per step (FP64 + FP32), oracle single-threaded"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "sample_n": ns},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_batch(nrm, torch, ctx, dev):
    """Ragged batch of 4096 FP64 vectors, lengths log-uniform in [1, 2^18]:
    graph replay of the persistent launch versus one launch per vector."""
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
        for _ in range(3):
            g.launch()
        torch.cuda.synchronize()
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.launch()
        e1.record()
        torch.cuda.synchronize()
        t_graph = e0.elapsed_time(e1) / reps
        single = torch.empty(4096, dtype=td, device=dev)
        views = [x[off[i]:off[i + 1]] for i in range(4096)]
        for i in range(4096):
            nrm.nrmf(views[i], out=single[i], ctx=ctx)
        torch.cuda.synchronize()
        e0.record()
        for i in range(4096):
            nrm.nrmf(views[i], out=single[i], ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        t_single = e0.elapsed_time(e1)
        same = bool(torch.equal(single.view(torch.int64 if td == torch.float64 else torch.int32),
                                g.out.view(torch.int64 if td == torch.float64 else torch.int32)))
        out["batch_" + name] = {"norms_per_s": 4096 / (t_graph * 1e-3), "ms_per_batch": t_graph,
                                "elements": int(off[-1]), "GBps": off[-1] * x.element_size() / (t_graph * 1e-3) / 1e9,
                                "one_launch_per_vector_ms": t_single,
                                "one_launch_per_vector_norms_per_s": 4096 / (t_single * 1e-3),
                                "bitwise_equal_to_single": same, "tuning": tuned}
        g.close()
        bctx.close()
        del x
    return out


def time_serving(nrm, seconds, rate):
    """Serving (config 4): Poisson arrivals at `rate`/s for `seconds`,
    lengths log-uniform in [2^4, 2^24], FP32/FP64 1:1, p = 2 (80 %) else
    1.5 or 3; inputs generated on the device at admission; 8 GiB budget.
    The same trace through the continuous-batching server and through the
    one-request-per-launch form."""
    import numpy as np
    tr = nrm.serving_trace(rate, seconds, seed=0)
    res, norms = {}, {}
    for name, (ns, mb) in (("batched", (4, 256)), ("one_request_per_launch", (1, 1))):
        srv = nrm.Server(budget_bytes=8 << 30, nstreams=ns, max_batch=mb)
        v, lat, rep = srv.replay(tr)
        srv.close()
        norms[name] = v
        res[name] = {k: rep[k] for k in ("completed", "rejected", "max_queue", "steps", "launches", "p50_ms",
                                           "p99_ms", "mean_ms", "max_ms", "wall_s", "norms_per_s", "elements_per_s",
                                           "peak_bytes", "arena_bytes")}
    L = np.array([tr[i].n for i in range(len(tr))])
    res["trace"] = {"rate_per_s": rate, "seconds": seconds, "requests": len(tr), "mean_length": float(L.mean()),
                    "offered_elements_per_s": float(L.sum() / seconds)}
    res["bitwise_equal"] = bool(norms["batched"].tobytes() == norms["one_request_per_launch"].tobytes())
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=1.0,
                    help="length of the serving trace (config 4 runs 60 s; 0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=50000.0)
    ap.add_argument("--log2n", type=int, default=28,
                    help="vector length 2^k (28 is the benchmark; smaller only for profiling captures)")
    ap.add_argument("--n", type=int, default=0,
                    help="vector length n, overriding --log2n (profiling captures of other shapes)")
    ap.add_argument("--p", type=float, default=2.0,
                    help="xNRMP with this p instead of xNRMF (profiling captures of the p-norm kernels; "
                         "the e2e, batch, serving and oracle legs and the v1_hypot roofline are left out)")
    args = ap.parse_args()
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
    seed = 1 + rank
    xd = nrm.nrm_gen(N, seed, 0, torch.float64, device=dev)
    xs = nrm.nrm_gen(N, seed, 0, torch.float32, device=dev)
    od = torch.empty((), dtype=torch.float64, device=dev)
    os_ = torch.empty((), dtype=torch.float32, device=dev)
    if args.p == 2.0:
        def step(x, o):
            nrm.nrmf(x, out=o, ctx=ctx)
    else:
        def step(x, o):
            nrm.nrmp(x, args.p, out=o, ctx=ctx)
    for _ in range(args.warmup):
        step(xd, od)
        step(xs, os_)
    torch.cuda.synchronize()

    K = args.steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    launches0 = ctx.launches
    with ClockSampler(local) as clk:
        barrier()
        evs[0].record()
        for i in range(K):
            step(xd, od)
            evs[2 * i + 1].record()
            step(xs, os_)
            evs[2 * i + 2].record()
        barrier()
    launches = ctx.launches - launches0
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
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    # Compute roofline of the dominant kernel (binary64 tree): 7 IEEE
    # operations per v1_hypot (Listing 2's one-statement-one-instruction
    # count) against GB300's FP64 rate from unit counts and clocks: SMs x 2
    # FP64 FMA per clock x the maximum SM clock (1.25 TFLOP/s).  The HBM view
    # of the same kernel is reported in parts.
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_ops_peak = sms * 2 * sm_max * 1e6
    hypot_d = N - 1
    d_bytes_gbs = BYTES_D / (d_avg * 1e-3) / 1e9
    s_bytes_gbs = BYTES_S / (s_avg * 1e-3) / 1e9
    achieved_ops = 7 * hypot_d / (d_avg * 1e-3)
    # DRAM bytes read+written per launch from an ncu capture at n = 2^28
    # (profiles/tree_kernel_nrmf_2e28_dram.md), in proportion to n otherwise
    traffic = TRAFFIC_D_2E28 * (N / float(1 << 28)) if TRAFFIC_VALID else None
    roof = {"bound": "alu", "achieved": achieved_ops / 1e9, "peak": fp64_ops_peak / 1e9,
            "unit": "Gop/s (FP64, 7 per v1_hypot)", "frac": achieved_ops / fp64_ops_peak, "traffic": traffic,
            "kernel": "tree_kernel<double,%d,OpHypot>" % ctx.tuning_for(nrm.NRM_F64).group_log2,
            "peak_source": "unit counts x clock (%d SMs x 2 x %.0f MHz)" % (sms, sm_max), "launch_ms": d_avg,
            "hbm_view": {"achieved": d_bytes_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": d_bytes_gbs / hbm_peak,
                         "peak_source": peak_src + " hbm_gbs"},
            "note": "frac > 1 is possible: the roofline prices v1_hypot at 7 FP64 operations (one of them a "
                    "division, one a square root); this kernel computes the same correctly rounded results with "
                    "integer/FP32 instructions plus one DFMA and one DMUL (bitwise parity with the oracle)"}
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "bytes_per_step": BYTES_D + BYTES_S,
                       "l2": "inputs (3 GiB) exceed the 129 MB L2; no flush", "parallelism": "replicas" if world > 1
                       else "single GPU"},
            "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
            "parts": {"dnrmf": {"ms": d_avg, "GBps": d_bytes_gbs, "Gelem_per_s": N / (d_avg * 1e-3) / 1e9,
                                "Ghypot_per_s": hypot_d / (d_avg * 1e-3) / 1e9,
                                "fp64_pipe_peak_Gops": fp64_ops_peak / 1e9},
                      "snrmf": {"ms": s_avg, "GBps": s_bytes_gbs, "Gelem_per_s": N / (s_avg * 1e-3) / 1e9,
                                "hbm_frac": s_bytes_gbs / hbm_peak,
                                "traffic": TRAFFIC_S_2E28 * (N / float(1 << 28)) if TRAFFIC_VALID else None}}}
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
                fn(x, out=o, ctx=ctx)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(5):
                    fn(x, out=o, ctx=ctx)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 5
                variants["%snrmf_%s" % (tag, name)] = {"ms": ms, "GBps": N * x.element_size() / (ms * 1e-3) / 1e9}
        line["parts"]["variants"] = variants

    # end to end through the host-buffer entry point
    if not args.no_e2e:
        hd = torch.empty(N, dtype=torch.float64, pin_memory=True)
        hs = torch.empty(N, dtype=torch.float32, pin_memory=True)
        hd.copy_(xd)
        hs.copy_(xs)
        nrm.nrm_host(hd, ctx=ctx, device=local)
        nrm.nrm_host(hs, ctx=ctx, device=local)
        reps = 5
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            vd = nrm.nrm_host(hd, ctx=ctx, device=local)
            vs = nrm.nrm_host(hs, ctx=ctx, device=local)
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
        line["parts"].update(time_batch(nrm, torch, ctx, dev))

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        hxd = xd.cpu().numpy()
        hxs = xs.cpu().numpy()
        t0 = time.perf_counter()
        vd = oracle.nrm(hxd)
        vs = oracle.nrm(hxs)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": (BYTES_D + BYTES_S) / tc / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "one full step (FP64 and FP32 vectors of 2^28), single thread, %.1f s" % tc,
                                "bitwise_equal": bool(vd.tobytes() == np.float64(od.item()).tobytes()
                                                      and vs.tobytes() == np.float32(os_.item()).tobytes())}
    if args.serve_seconds > 0 and rank == 0:
        del xd, xs
        torch.cuda.empty_cache()
        line["parts"]["serve"] = time_serving(nrm, args.serve_seconds, args.serve_rate)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
