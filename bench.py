"""EM throughput benchmark: units = N * N_G * D per EM iteration.

Workload: a seeded synthetic diagonal GMM with N = 2,000,000 samples, D = 60
(speech-like: 20 base dims + deltas + delta-deltas), N_G = 256; k-means
initialisation (10 iterations) outside the timed region, then each timed
step is ONE EM iteration (fused E+M data pass, FP64 reduce, update, floor,
operands of the next E-step) through the library's C ABI (gmm_em_iterate).
X (480 MB) is larger than the 129 MB L2, so every step streams it from HBM.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the only reference implementation there is) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM iters/sec (N·N_G·D/s) at D=60,N_G=256; BF16-TC vs FP32 at stated ΔLL"
UNIT = "N·N_G·D/s"
N_FULL, D_FULL, G_FULL = 2_000_000, 60, 256
# DRAM bytes (read + write) of one tensor-core EM pass on the full workload:
# ncu dram__bytes of the screen, exact and M-step kernels at N = 1,000,000
# (948 MB in one capture), scaled by the samples (traffic grows in
# proportion).  Re-measure whenever those kernels change.
TC_PASS_TRAFFIC = 948.4e6 * 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []          # (arrival time, line)
        self.window = None       # (t0, t1): only samples that arrive inside count

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        """The timed region, in time.perf_counter() seconds."""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if self.window and not (self.window[0] <= ts <= self.window[1]):
                continue
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_data(n=None):
    """The c2 workload (N = 2,000,000, D = 60, N_G = 256), or its first n samples."""
    from paper_1707_09094_gb300 import synth
    X, _, _ = synth.make("c2")
    return X if n is None else np.ascontiguousarray(X[:n])


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(X, target_s: float = 12.0, threads: int = 0):
    """FP64 oracle EM iteration (MapReduce chunks over `threads` host cores,
    0 = all) on a bounded prefix of the workload; returns (units/s, cores,
    sample text)."""
    import oracle
    all_cores = oracle.num_threads() if threads == 0 else None
    if threads:
        oracle.set_threads(threads)
    cores = oracle.num_threads()
    G = G_FULL
    rng = np.random.default_rng(5)
    n = 20000
    start = None
    while True:
        Xs = X[:n]
        if start is None:
            idx = rng.choice(n, G, replace=False)
            start = (Xs[idx].astype(np.float64), np.ones((G, X.shape[1])), np.full(G, 1.0 / G))
        t0 = time.perf_counter()
        oracle.em_iterate(Xs, *start, 1, 1e-10, n_chunks=cores * 4)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or n >= X.shape[0]:
            break
        n = min(X.shape[0], int(n * max(2.0, target_s / 4 / max(dt, 1e-3))))
    units = n * G * X.shape[1]
    del all_cores
    return units / dt, cores, "1 FP64 EM iteration on the first %d of %d samples (D=%d, N_G=%d), %d OpenMP " \
                              "threads, %.2f s" % (n, X.shape[0], X.shape[1], G, cores, dt)


def cpu_e1_learn(threads: int, n: int):
    """The paper's speed-up workload E1 (N=1e6, D=100, N_G=100; 10 k-means +
    10 EM iterations, Sec. 5.1) by the FP64 oracle on `threads` host cores,
    timed on the first n samples of a seeded c1-style mixture of that shape
    and scaled to N=1e6 (both phases are linear in N)."""
    import oracle

    from paper_1707_09094_gb300 import synth
    N, D, G = E1_SHAPE
    rng = np.random.default_rng(2000 + len(TABLE1_SHAPES))
    X, _ = synth._draw(rng, synth.mixture_c1(rng, D, G), n)
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.learn(X, G, seed=1, km_iter=10, em_iter=10, n_chunks=max(threads, 1) * 4)
    dt = time.perf_counter() - t0
    return {"threads": threads, "samples_timed": n, "timed_s": dt, "learn_s_scaled_to_1e6": dt * N / n}


def cpu_baseline_line(X, rate_cores, cores, sample):
    """The oracle on the host: all cores (the headline figure), one core, the
    CPU model, and the E1 learn time beside the paper's own E1 numbers."""
    import oracle
    r1, _, s1 = cpu_oracle_rate(X, target_s=8.0, threads=1)
    e1_all = cpu_e1_learn(cores, 60_000)
    e1_one = cpu_e1_learn(1, 12_000)
    oracle.set_threads(cores)
    return {"value": rate_cores, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model(),
            "one_core": {"value": r1, "unit": UNIT, "sample": s1},
            "e1_learn": {"all_cores": e1_all, "one_core": e1_one,
                         "paper_s": {"1_thread": 272.0, "16_threads": 27.0,
                                     "paper_hardware": "2x Xeon E5-2620 v4, 16 cores (FP64, Armadillo gmm_diag)"},
                         "note": "10 k-means + 10 EM iterations at N=1e6, D=100, N_G=100, timed on a prefix and "
                                 "scaled by N"}}


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """Slowest rank's time (the job ends when the last replica ends)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Units all replicas processed per second (each rank runs the whole workload)."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def c2_config(N, D, G, head, world, x_bytes):
    """The `config` object of the bench line (both arms)."""
    return {"workload": "c2 EM iteration (fused E+M pass + FP64 reduce/update): N=%d D=%d N_G=%d, "
                        "k-means-initialised, E-step %s" % (N, D, G, head),
            "N": N, "D": D, "N_G": G, "form": head,
            "l2": "inputs larger than L2 (X = %.0f MB)" % (x_bytes / 1e6),
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """The FP64 CPU oracle on the host cores, the same metric and config:
    every step is one oracle EM iteration (MapReduce chunks over all cores)
    on a prefix of the workload sized so the whole run takes about a minute;
    value = units of that prefix / its median step time, ms_per_step the
    measured step time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    X = make_data()
    N, D = X.shape
    G = G_FULL
    cores = oracle.num_threads()
    target = max(0.5, 60.0 / max(args.steps + args.warmup, 1))
    _, _, sample = cpu_oracle_rate(X, target_s=4 * target)    # sizes the prefix: one step ~ target seconds
    n = int(sample.split("first ")[1].split(" ")[0])
    rng = np.random.default_rng(5)
    idx = rng.choice(n, G, replace=False)
    Xs = X[:n]
    start = (Xs[idx].astype(np.float64), np.ones((G, D)), np.full(G, 1.0 / G))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.em_iterate(Xs, *start, 1, 1e-10, n_chunks=cores * 4)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    units = n * G * D
    v = units / statistics.median(times)
    head = args.forms[-1] if args.forms else "bf16"
    smp = "each step: 1 FP64 EM iteration on the first %d of %d samples (D=%d, N_G=%d), %d OpenMP threads" % (
        n, N, D, G, cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "units_per_step": units, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": c2_config(N, D, G, head, 1, X.nbytes),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp,
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1707_09094_gb300 import GMM, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    X = make_data(args.n)
    Xd = torch.from_numpy(X).cuda()
    N, D = X.shape
    G = G_FULL
    units = N * G * D
    stream = torch.cuda.current_stream()

    # k-means initialisation (not timed), shared by every form
    base = GMM().learn(Xd, G, km_iter=10, em_iter=0, seed=1002, var_floor=1e-10)
    start = base.get_params()

    def em_model():
        g = GMM().set_params(*start)
        g.em_iterate(Xd, 0, recompute_center=True)   # global centre for the tensor-core forms
        return g

    # quality: 10 EM iterations per form from the same start, judged on the same evaluator
    quality = {}
    for prec in args.forms:
        g = em_model()
        try:
            g.em_iterate(Xd, 10, prec=prec)
        except Exception as e:  # noqa: BLE001  (form not available on this build)
            quality[prec] = {"error": str(e)}
            continue
        quality[prec] = {"avg_log_p": base_eval(base, g, Xd)}
    ref_ll = quality.get("fp32", {}).get("avg_log_p")

    def time_form(prec, host_input=False):
        g = em_model()
        Xin = X if not host_input else torch.from_numpy(X).pin_memory()
        with ClockSampler(local) as cs:   # started before the warm-up: sampling is live when timing starts
            for _ in range(args.warmup):
                g.set_params(*start)
                g.em_iterate(Xin if host_input else Xd, 1, prec=prec)
            g.set_params(*start)
            g.profile(True)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                g.em_iterate(Xin if host_input else Xd, 1, prec=prec)
            ev1.record(stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            wall = t1 - t0
            cs.mark(t0, t1)
            time.sleep(2.5 * cs.interval_ms / 1e3)   # let the last samples of the window arrive
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
        pass_ms, pass_n, launches = g.profile_read()
        extra = {}
        if prec == "bf16":
            cyc = g.phase_cycles()
            tot = max(sum(cyc), 1)
            names = ["build_next_operand", "sync_operand_ready", "wait_mma", "screen_pass1", "candidate_lists"]
            n_scr, kept, dense = g.screen_stats()
            extra = {"screen_phase_share": {k: c / tot for k, c in zip(names, cyc)},
                     "candidates_per_sample": kept / max(n_scr, 1), "dense_fallbacks": dense}
        g.profile(False)
        return {"ms": ms, "wall_s": wall, "pass_ms": pass_ms, "pass_n": pass_n, "launches": launches,
                "clocks": cs.summary(), **extra}

    # k-means (Sec. 3) pass throughput, both forms, and one whole learn(), reported beside the EM metric
    from paper_1707_09094_gb300._lib import GMM_DEBUG_KM_FORM

    def km_time(form):
        km = GMM().set_params(*start)
        km.debug_set(GMM_DEBUG_KM_FORM, form)
        km.kmeans(Xd, 1, return_assign=False)
        km.set_params(*start)
        km.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        km.kmeans(Xd, 5, return_assign=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms, n, _ = km.profile_read()
        return ms / max(n, 1), wall * 1e3 / 5, km.km_screen_stats()

    km_tc = km_time(0)
    km_cc = km_time(1)
    learn_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        GMM().learn(Xd, G, km_iter=10, em_iter=10, seed=1002, prec=args.forms[-1])
        torch.cuda.synchronize()
        learn_t.append(time.perf_counter() - t0)

    results = {}
    for prec in args.forms:
        if "error" in quality.get(prec, {}):
            continue
        results[prec] = time_form(prec)
    head = args.forms[-1] if args.forms[-1] in results else "fp32"
    r = results[head]
    e2e = time_form(head, host_input=True)
    h2d_gbs = plain_copy_gbs(X, Xd)
    step_ms = r["ms"] / args.steps
    value = whole_job_rate(units, world, step_ms)

    peaks, peak_src = _peaks()
    pass_ms = r["pass_ms"] / max(r["pass_n"], 1)
    if head == "fp32":
        # CUDA-core form: 4 FMA per (i, g, d) (E: 2, M: 2); peak = 152 SMs x 128 FMA/clk x 2 flop x max clock
        flops = 8.0 * units
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (pass_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s clock)" %
                               (peaks.get("sm_max_mhz", 2070.0), peak_src)}
    else:
        flops = 8.0 * units   # algorithmic: E 2 MAC + M 2 MAC per (i, g, d)
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": flops / (pass_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "bf16_tflops (%s)" % peak_src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = (args.traffic * N / N_FULL if args.traffic and head == "bf16" else None)
    roof["kernel_ms"] = pass_ms

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16"}[head],
        "data": "synthetic",
        "config": c2_config(N, D, G, head, world, X.nbytes),
        "roofline": roof,
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "e2e": {"value": world * units / (e2e["ms"] / args.steps * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": 8 + 32,
                "ms_per_step": e2e["ms"] / args.steps,
                "plain_h2d_copy_gbs": h2d_gbs,
                "plain_h2d_copy_ms": X.nbytes / (h2d_gbs * 1e9) * 1e3,
                "note": "plain_h2d_copy: one cudaMemcpyAsync of the same pinned X, the copy engine's rate here"},
        "kmeans": kmeans_line(km_tc, km_cc, units, N * (D + 1) * 4, peaks, peak_src),
        "learn_10km_10em_s": min(learn_t),
        "forms": {p: {"value": world * units / (results[p]["ms"] / args.steps * 1e-3),
                      "ms_per_step": results[p]["ms"] / args.steps,
                      "pass_ms": results[p]["pass_ms"] / max(results[p]["pass_n"], 1),
                      "avg_log_p_after_10_em": quality[p]["avg_log_p"],
                      "delta_ll_vs_fp32": (quality[p]["avg_log_p"] - ref_ll) if ref_ll is not None else None,
                      **{k: results[p][k] for k in ("screen_phase_share", "candidates_per_sample", "dense_fallbacks")
                         if k in results[p]}}
                  for p in results},
    }
    if not args.no_batched:
        line["batched_512"] = run_batched_leg()
    if not args.no_init_net:
        line["init_net"] = run_init_net_leg(peaks, peak_src)
        line["init_net_c5"] = run_init_net_c5_leg()
    if not args.no_table1:
        line["table1_em_tol"] = run_table1_leg()
    if not args.no_c3:
        line["c3"] = run_c3_leg(peaks, peak_src)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(X)
        line["cpu_baseline"] = cpu_baseline_line(X, rate, cores, sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# The shapes (N, D, N_G) of the paper's Table 1 datasets (Sec. 5.2; the UCI
# data itself is not available, seeded c1-style mixtures of these shapes stand
# in for it) and of its speed-up experiment E1 (Sec. 5.1).
TABLE1_SHAPES = [(2048, 10, 5), (2534, 72, 6), (6497, 11, 30), (37749, 32, 50), (100000, 2, 6),
                 (150000, 78, 30), (581012, 55, 21), (1000000, 10, 25)]
E1_SHAPE = (1000000, 100, 100)


def run_table1_leg(em_tol=1e-6, max_iter=250):
    """Convergence-driven learn (k-means 10, EM until the mean-LL gain is below
    em_tol, at most 250 iterations) on Table-1-shaped synthetic data, per
    E-step form: EM iterations to converge, final mean log-likelihood, time."""
    import torch

    from paper_1707_09094_gb300 import GMM, synth
    rows = []
    for r, (N, D, G) in enumerate(TABLE1_SHAPES + [E1_SHAPE]):
        rng = np.random.default_rng(2000 + r)
        X, _ = synth._draw(rng, synth.mixture_c1(rng, D, G), N)
        Xd = torch.from_numpy(X).cuda()
        for prec in ("fp32", "bf16"):
            if prec == "bf16" and (D > 64 or G > 256):
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = GMM().learn(Xd, G, km_iter=10, em_iter=max_iter, em_tol=em_tol, seed=2000 + r, prec=prec)
            torch.cuda.synchronize()
            rows.append({"N": N, "D": D, "N_G": G, "form": prec, "em_iters": len(g.ll_history()),
                         "final_ll": float(g.avg_log_p(Xd)), "learn_s": time.perf_counter() - t0})
    return {"em_tol": em_tol, "max_em_iter": max_iter, "runs": rows}


def kmeans_line(tc, cc, units, bytes_alg, peaks, peak_src):
    """k-means map pass (operands, assignment, sorted statistics), per form.
    Algorithmic work: 1 MAC per (i, g, d) (the expanded score x.mu) and the
    bytes X once + one assignment per sample.  The tensor-core form issues 3
    BF16 MMAs per MAC (split operands); the CUDA-core form 1 FP32 FMA."""
    (tc_ms, tc_wall, (scr, dfr, f64)), (cc_ms, cc_wall, _) = tc, cc
    tens = peaks["bf16_tflops"]
    alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"form": "tensor cores: split-BF16 screen, exact FP32/FP64 decision of the rest",
            "pass_ms": tc_ms, "units_per_s": units / (tc_ms * 1e-3), "iterations_wall_ms": tc_wall,
            "deferred_per_sample": dfr / max(scr, 1), "fp64_per_sample": f64 / max(scr, 1),
            "roofline": {"bound": "tensor", "achieved": 2.0 * units / (tc_ms * 1e-3) / 1e12, "peak": tens,
                         "unit": "TFLOP/s", "frac": 2.0 * units / (tc_ms * 1e-3) / 1e12 / tens,
                         "peak_source": "bf16_tflops (%s); algorithmic 2 flop per (i, g, d)" % peak_src},
            "hbm": {"achieved": bytes_alg / (tc_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": bytes_alg / (tc_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                    "note": "algorithmic bytes: X once + one int32 assignment per sample"},
            "cuda_core_form": {"pass_ms": cc_ms, "iterations_wall_ms": cc_wall,
                               "roofline": {"bound": "alu", "achieved": 2.0 * units / (cc_ms * 1e-3) / 1e12,
                                            "peak": alu, "unit": "TFLOP/s",
                                            "frac": 2.0 * units / (cc_ms * 1e-3) / 1e12 / alu,
                                            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz"
                                                           % peaks.get("sm_max_mhz", 2070.0)}}}


def run_batched_leg():
    """Batched form: 512 independent fits (N log-uniform in [1000, 200000],
    D in {13,39,64}, N_G in {8..128}), k-means(10) + EM(10) each, one call."""
    import torch

    from paper_1707_09094_gb300 import learn_batched, synth
    Xs, Gs, units = [], [], 0
    for j in range(512):
        X, _, mix = synth.batched_fit(j)
        Xs.append(torch.from_numpy(X).cuda())
        Gs.append(mix.means.shape[0])
        units += X.shape[0] * X.shape[1] * mix.means.shape[0]
    learn_batched(Xs, Gs, km_iter=10, em_iter=10, seed=40000)     # autotunes this bucket
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    models = learn_batched(Xs, Gs, km_iter=10, em_iter=10, seed=40000)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_tot = int(sum(x.shape[0] for x in Xs))
    return {"fits": 512, "samples": n_tot, "km_iter": 10, "em_iter": 10, "learn_s": dt,
            "fits_per_s": 512 / dt, "units_per_iter": units,
            "units_per_s_20_iters": 20 * units / dt,
            "mean_final_ll": float(np.mean([m.ll_history()[-1] for m in models]))}


def run_init_net_leg(peaks, peak_src, B=16, P=4096, steps=10, warmup=3):
    """Learned initialiser: Adam training steps of the set encoder at
    D=32, N_G=32 (per point 32-256-256-256, mean pool, 256-512-512-512-2080),
    B sets of P points per step, on synthetic sets with synthetic targets."""
    import torch

    from paper_1707_09094_gb300 import InitNet
    D, G, Hp, Hh, Lp, Lh = 32, 32, 256, 512, 3, 3
    net = InitNet(D, G, Hp, Hh, Lp, Lh, seed=0)
    gen = torch.Generator(device="cuda").manual_seed(7)
    pts = torch.randn((B, P, D), device="cuda", generator=gen) * 2.0
    tgt = (torch.randn((B, G, D), device="cuda", generator=gen, dtype=torch.float64),
           torch.rand((B, G, D), device="cuda", generator=gen, dtype=torch.float64) + 0.5,
           torch.full((B, G), 1.0 / G, device="cuda", dtype=torch.float64))
    for _ in range(warmup):
        net.step(pts, tgt, lam=0.1, mode=2)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        net.step(pts, tgt, lam=0.1, mode=2)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # algorithmic GEMM flops: forward, input-gradient and weight-gradient
    # products of every layer (3 x 2 x MACs); point layers per point, head per set
    point_mac = D * Hp + (Lp - 1) * Hp * Hp
    head_mac = Hp * Hh + (Lh - 1) * Hh * Hh + Hh * G * (1 + 2 * D)
    flops = 6.0 * (B * P * point_mac + B * head_mac)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"sets": B, "points_per_set": P, "ms_per_step": ms, "sets_per_s": B / (ms * 1e-3),
            "points_per_s": B * P / (ms * 1e-3),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops"], "peak_source": "bf16_tflops (%s)" % peak_src,
                         "flops_per_step": flops}}


def plain_copy_gbs(X, Xd, reps=5):
    """Host-to-device rate of one plain copy of the pinned workload (the
    bound of the e2e step's input transfer)."""
    import torch
    Xh = torch.from_numpy(X).pin_memory()
    stream = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        Xd.copy_(Xh, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        best = min(best, ev0.elapsed_time(ev1))
    return X.nbytes / (best * 1e-3) / 1e9


def run_c3_leg(peaks, peak_src, steps=3, n=None):
    """The precision workload at full size (N=1e7, D=128, N_G=1024; means
    N(0, 3^2), sigma log-uniform on [0.1, 10]): k-means (2 iterations, not
    timed), then EM iterations of each form from the same start, each after
    one untimed iteration:
      bf16  the blocked tensor-core pass (split-BF16 screen over blocks of 128
            Gaussians on tcgen05, exact FP32 log-densities of the candidates,
            M-step from the kept responsibilities);
      fp32  the register-blocked two-phase CUDA-core form (log-densities
            computed once: the first phase records each block's candidates).
    Algorithmic work as the headline: 8 flop per (i, g, d); the bf16 roofline
    is against the BF16 tensor peak, the fp32 one against the FP32 FMA peak.
    n: the first n samples only (profiling captures)."""
    import torch

    from paper_1707_09094_gb300 import GMM, synth
    X, _, _ = synth.make("c3", N=n) if n else synth.make("c3")
    Xd = torch.from_numpy(X).cuda()
    N, D = X.shape
    G = 1024
    start = GMM().learn(Xd, G, km_iter=2, em_iter=0, seed=1003, var_floor=1e-10).get_params()
    units = N * G * D
    alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    out = {"N": N, "D": D, "N_G": G, "forms": {}}
    stream = torch.cuda.current_stream()
    for prec in ("bf16", "fp32"):
        g = GMM().set_params(*start)
        g.em_iterate(Xd, 1, prec=prec, var_floor=1e-10, recompute_center=True)   # warm-up
        g.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.em_iterate(Xd, steps, prec=prec, var_floor=1e-10)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        achieved = 8.0 * units / (ms * 1e-3) / 1e12
        f = {"ms_per_iteration": ms, "units_per_s": units / (ms * 1e-3), "mean_ll": g.ll_history()[-1]}
        if prec == "bf16":
            sc, kept, dense = g.screen_stats()
            f["form"] = "tensor cores (split-BF16 screen, exact FP32 candidates)"
            f["candidates_per_sample"] = kept / max(sc, 1)
            f["samples_to_fp32_form"] = dense
            peak = peaks["bf16_tflops"]
            f["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "peak_source": "bf16_tflops (%s)" % peak_src}
        else:
            f["form"] = "fp32 (register-blocked, two phases, log-densities recorded once)"
            f["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu, "unit": "TFLOP/s",
                             "frac": achieved / alu,
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s clock)"
                                            % (peaks.get("sm_max_mhz", 2070.0), peak_src)}
        out["forms"][prec] = f
    out["delta_ll_bf16_vs_fp32"] = out["forms"]["bf16"]["mean_ll"] - out["forms"]["fp32"]["mean_ll"]
    del Xd
    torch.cuda.empty_cache()
    return out


def run_init_net_c5_leg(n_train=32768, epochs=2.0, n_eval=16):
    """The learned-initialiser workload at its shape (D=32, N_G=32, 4096
    points per set), scaled down to fit the bench: n_train mixtures fitted by
    the plain method (batched k-means 10 + EM 10), Adam for `epochs`, then
    n_eval held-out mixtures of N = 1e6 fitted to convergence three ways
    (k-means seeding; the network's start; the network's means as k-means
    seeds with 3 iterations).  Paired means: data passes, final mean LL."""
    from paper_1707_09094_gb300 import init_train
    r = init_train.c5_experiment(n_train=n_train, epochs=epochs, n_eval=n_eval, eval_n=1_000_000, lr=3e-3,
                                 lam=1.0, hybrid_km=3)
    return {k: v for k, v in r.items() if k != "rows"}


def base_eval(base, g, Xd):
    return g.avg_log_p(Xd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp32,bf16",
                    help="comma list of E-step forms; the last available one is the headline")
    ap.add_argument("--traffic", type=float, default=TC_PASS_TRAFFIC,
                    help="DRAM bytes of one headline pass (ncu), per pass; 0 = not measured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-fit batched leg")
    ap.add_argument("--no-init-net", action="store_true", help="skip the learned-initialiser training leg")
    ap.add_argument("--no-table1", action="store_true", help="skip the convergence runs on Table-1 shapes")
    ap.add_argument("--no-c3", action="store_true", help="skip the full-size precision workload (N=1e7, D=128)")
    ap.add_argument("--n", type=int, default=None,
                    help="time on the first n samples only (profiling captures); the default is the full workload")
    ap.add_argument("--c3-only", action="store_true",
                    help="run only the precision-workload leg (with --n: its first n samples) and print its JSON")
    args = ap.parse_args()
    args.forms = [f for f in args.forms.split(",") if f]
    if args.impl == "reference":
        return run_reference(args)
    if args.c3_only:
        peaks, peak_src = _peaks()
        print(json.dumps(run_c3_leg(peaks, peak_src, steps=args.steps, n=args.n)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
