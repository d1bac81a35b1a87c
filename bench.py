#!/usr/bin/env python
"""Benchmark: Brouwer-Zimmermann enumeration throughput on the random [200,100] code.

One step = md_compute on G = [I_100 | R] (R from SplitMix64 seed 3, the first invertible
draw) running every level of stages g = 1..--max-stage (default 10) to completion: both
Gamma matrices, every g-row combination, ~3.9e13 codewords at g <= 10.  The metric is
codewords/s = the sum of C(k, g) over the completed levels / device time.  At N = 1 the
full computation to d (time-to-d, ~3.2e14 codewords) also runs once, after the timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-time-to-d]
    python bench.py --workload batch | --workload serve     (the batched and serving workloads alone)

At N = 1 the default run also measures, after the timed steps: the same stages on the popcount
kernels against the POPC peak measured on this GPU ("roofline_popcount"), the batch of 2048
codes with md_batch_tune's options against the per-code loop ("batch"; and under a 1e10
combination budget, "batch_budget_1e10"), and the serving trace ("serve"), each with its own
clock samples.

Under torchrun (N > 1) every rank runs an independent replica of the step on its own GPU
(the path has no cross-GPU exchange); value = all ranks' codewords / the slowest rank's
time.  --impl reference times the CPU oracle (the plain C implementation used by the
tests) on bounded samples of the same workload, on this host's cores.
"""
from __future__ import annotations

import argparse
import atexit
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
POPC_PER_SM_PER_CLK = 16          # measured on GB300 (popc.b32 throughput per SM per clock)
NOMINAL_SMS = 152
NOMINAL_MAX_MHZ = 2070.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch, from ncu captures of the present kernels
# (profiles/): the split kernel's level (8, Gamma_0) launch, a fixed staging cost that does not grow
# with the codewords; the tensor-core kernel's level (10, Gamma_0) launch, the one bench.py times
# (a one-pass capture of the full-size launch; ncu prints 3 significant digits)
SPLIT_KERNEL_TRAFFIC_BYTES = 157696 + 732160
TC_KERNEL_TRAFFIC_BYTES = 6570000000 + 13740000
TC_KERNEL_TRAFFIC_NOTE = ("dram read + write of the level (10, Gamma_0) launch, ncu (one pass): the head-slice "
                          "stream of a head table (502 MB per matrix) larger than L2; 0.0004 B per codeword")
FP8_PER_BF16 = 2.0                # nominal dense fp8 / bf16 tensor rate (4.5 / 2.25 PFLOP/s)
# the input of both arms (seed 3's first R draw is invertible, so no draw is skipped)
DATA = ("synthetic: random code G=[I_100|R], R i.i.d. Bernoulli(1/2) from SplitMix64 seed 3 "
        "(the first draw; R is invertible)")


def data_string(workload: str) -> str:
    """The `data` field of both arms for a single-code workload."""
    if workload == "rand200x100":
        return DATA
    from paper_1911_08963_gb300 import inputs
    c = inputs.SINGLE[workload]
    return ("synthetic: random code G=[I_%d|R], R i.i.d. Bernoulli(1/2) from SplitMix64 seed %d "
            "(draw %d: the first invertible R)" % (c["k"], c["seed"], c["skip"] + 1))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rand200x100")
    ap.add_argument("--max-stage", type=int, default=10)
    ap.add_argument("--filter", type=int, default=1)
    ap.add_argument("--tensor", type=int, default=1,
                    help="1 = large levels on the tensor-core kernel (default), 0 = popcount kernels only")
    ap.add_argument("--no-time-to-d", action="store_true",
                    help="skip the full computation to d (run once on rank 0 at N=1 by default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end leg (at most --steps)")
    ap.add_argument("--no-popcount", action="store_true", help="skip the popcount-kernel roofline run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch lines (all 2048 codes, and under 1e10)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving line")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--oracle-full", action="store_true",
                    help="reference arm, workloads with k <= 64: also time the complete oracle run to d "
                         "(and the 2^k brute force for k <= 32) on all host cores")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--verbose", action="store_true", help="per-level records on stderr")
    ap.add_argument("--batch-count", type=int, default=2048)
    ap.add_argument("--batch-workers", type=int, default=0,
                    help="threads running the batch's single-code computations (0 = library default 2)")
    ap.add_argument("--chunk-log2", type=int, default=0, help="log2 combinations per work item (0 = library default)")
    ap.add_argument("--batch-budget", type=float, default=1e10,
                    help="batch: per-code work budget in combinations (0 = every code)")
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-budget", type=float, default=1e11)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-heavy", type=float, default=0,
                    help="estimated work from which a request runs alone on the tensor cores "
                         "(0 = library default 2^30, -1 = never)")
    ap.add_argument("--profile-once", action="store_true",
                    help="one md_compute up to --max-stage and exit (a target for ncu captures)")
    return ap.parse_args()


# --------------------------------------------------------------------- helpers ---

class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            atexit.register(self._end)          # a leg that fails before stop() leaves none running
        except OSError:
            self.proc = None

    def _end(self):
        if self.proc and self.proc.poll() is None:
            self.proc.kill()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def gpu_index() -> int:
    """The GPU this process uses, as nvidia-smi numbers it."""
    _, _, local = dist_env()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = vis.split(",")
    if vis and local < len(parts) and parts[local].strip().isdigit():
        return int(parts[local])
    return local


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(args, n, k):
    """The `config` object shared by both arms."""
    from paper_1911_08963_gb300 import inputs
    seed = inputs.SINGLE[args.workload]["seed"] if args.workload in inputs.SINGLE else 3
    return {"workload": "random [%d,%d] seed %d, Brouwer-Zimmermann stages g=1..%d, every level complete "
                        "(or the run to d if it stops first)" % (n, k, seed, args.max_stage),
            "n": n, "k": k, "max_stage": args.max_stage, "filter": args.filter,
            "l2": "flushed between steps (512 MiB write); inputs are ~100 KB"}


def reduce_over_ranks(seconds: float, codewords: int, device: str):
    """Replicas: the slowest rank's time and all ranks' codewords (torch.distributed, any
    backend; a no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, codewords
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(codewords)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def roofline_line(args, n, k, top_g, nlaunch, per_launch_cw, per_launch_s, words):
    """Roofline of the kernel that runs the deepest stage's levels.  `words`: the packed 32-bit
    words each tensor-core product multiplies (0 for the popcount kernels)."""
    W = (n - k + 31) // 32                    # packed words of a full-rank matrix's rows
    bits = n - k                              # the columns whose weight the product counts
    if args.tensor:
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops_sustained")
        basis = "measured bf16_tflops_sustained x %.0f (nominal fp8/bf16 dense ratio)" % FP8_PER_BF16
        if not bf16:
            bf16, basis = 1700.0, "fallback sustained bf16 1.7 PFLOP/s x 2 (nominal fp8/bf16 dense ratio)"
        F = words or W
        flops_cw = 2.0 * 32 * F
        cw_rate = per_launch_cw / per_launch_s
        achieved = cw_rate * flops_cw / 1e12
        peak = bf16 * FP8_PER_BF16
        burst = peaks.get("bf16_tflops")
        line = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TC_KERNEL_TRAFFIC_BYTES,
                "traffic_note": TC_KERNEL_TRAFFIC_NOTE,
                "kernel": "tc_kernel<%d> (stage g=%d levels, %d launches timed)" % (W, top_g, nlaunch),
                "peak_basis": basis,
                "work_basis": "%d flops per codeword executed: a +-1 e4m3 inner product over the first %d of "
                              "the %d packed words (%d bits, all real columns; tcgen05.mma kind::f8f6f4, K = 32 "
                              "per instruction); the weight over fewer words bounds the full weight, rows "
                              "that pass are rechecked exactly" % (flops_cw, F, W, 32 * F),
                # the method's own work: the +-1 product over all n - k real columns of a codeword
                "method": {"flops_per_codeword": 2 * bits, "achieved": cw_rate * 2 * bits / 1e12,
                           "frac": cw_rate * 2 * bits / 1e12 / peak},
                "codewords_per_s": cw_rate,
                "peak_codewords_per_s": peak * 1e12 / flops_cw}
        if burst:
            line["frac_of_burst"] = achieved / (burst * FP8_PER_BF16)
        return line
    return popc_roofline(POPC_PER_SM_PER_CLK, NOMINAL_SMS, NOMINAL_MAX_MHZ, top_g, nlaunch, per_launch_cw,
                         per_launch_s, "16 popc/clk/SM (an earlier probe) x 152 SMs x 2070 MHz max clock")


def clock_matched(roofline, rate, sms, mhz):
    """The tensor roofline's work against the tensor pipe's own e4m3 rate on this GPU:
    md_mma_rate's flops per SM per clock x SMs x the SM clock (MHz) of the timed region."""
    peak = rate * sms * mhz * 1e6 / 1e12
    return {"peak": peak, "unit": "TFLOP/s", "flops_per_sm_per_clk": rate,
            "basis": "md_mma_rate on this GPU: %.0f e4m3 flops/clk/SM x %d SMs x %.0f MHz (median SM clock "
                     "of the timed region)" % (rate, sms, mhz),
            "frac": roofline["achieved"] / peak, "frac_method": roofline["method"]["achieved"] / peak}


def popc_roofline(per_sm_clk, sms, mhz, top_g, nlaunch, per_launch_cw, per_launch_s, basis):
    """Roofline of the popcount kernels (the split kernel of the deepest stage): one POPC per
    codeword (the popcount of the OR of the fewest packed words that bounds the weight; exact
    weights only for the rare codeword that can reach U) against the POPC pipe's peak."""
    peak = per_sm_clk * sms * mhz * 1e6 / 1e9                                        # Gpopc/s
    achieved = per_launch_cw / per_launch_s / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpopc/s", "frac": achieved / peak,
            "traffic": SPLIT_KERNEL_TRAFFIC_BYTES,
            "traffic_note": "dram read + write of the level (8, Gamma_0) launch of the same kernel, ncu: a fixed "
                            "staging cost (rows, pair table, state atomics) that does not grow with codewords",
            "kernel": "split_kernel (stage g=%d levels, %d launches timed)" % (top_g, nlaunch),
            "peak_basis": basis,
            "work_basis": "1 popc per codeword: popcount of the OR of the packed words, exact weight "
                          "only for codewords that can reach U"}


def measured_peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ CPU oracle ---

def oracle_sample_rate(G, n, k, g, seconds, threads):
    """Codewords/s of the CPU oracle on a bounded prefix of level (g, 0), sized to take
    about `seconds` on `threads` threads.  Returns (rate, codewords, seconds)."""
    import oracle
    gams, _, _ = oracle.gammas(G, n, k)
    total = math.comb(k, g)
    probe = min(total, 2_000_000 * threads)
    t0 = time.perf_counter()
    oracle.scan(gams[0], n, k, g, 0, probe, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-3)
    size = min(total, max(probe, int(probe / dt * seconds)))
    t0 = time.perf_counter()
    oracle.scan(gams[0], n, k, g, 0, size, threads=threads)
    dt = time.perf_counter() - t0
    return size / dt, size, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1911_08963_gb300 import inputs
    oracle.build()
    G, n, k = inputs.single_code(args.workload)
    threads = os.cpu_count() or 1
    g = args.max_stage
    per_step = 2.0 if args.oracle_full else max(2.0, 120.0 / max(1, args.steps + args.warmup))
    rates = []
    for i in range(args.warmup + args.steps):
        rate, size, dt = oracle_sample_rate(G, n, k, g, per_step, threads)
        if i >= args.warmup:
            rates.append((size, dt))
    cw = sum(s for s, _ in rates)
    sec = sum(t for _, t in rates)
    value = cw / sec
    line = {
        "impl": "reference", "metric": "codewords/s", "value": value, "unit": "codewords/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": data_string(args.workload),
        "config": workload_config(args, n, k),
        "cpu_baseline": {"value": value, "unit": "codewords/s", "cores": threads, "kind": "oracle",
                         "sample": "colex-rank prefix of level (g=%d, Gamma_1), %d combinations per step"
                                   % (g, rates[0][0])},
        "e2e": {"value": value, "unit": "codewords/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if args.oracle_full and k <= 64:
        # the whole computation on the host cores: Alg. 1 to d, and for k <= 32 the definition
        t0 = time.perf_counter()
        res = oracle.bz(G, n, k, threads=threads)
        full = {"d": res.d, "seconds": time.perf_counter() - t0, "codewords": res.codewords,
                "stop_stage": res.stop[0], "threads": threads}
        if k <= 32:
            t0 = time.perf_counter()
            dbf, _ = oracle.bruteforce(G, n, k, threads=threads)
            full["bruteforce"] = {"d": dbf, "seconds": time.perf_counter() - t0, "messages": (1 << k) - 1}
        line["oracle_full"] = full
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- GPU arm -------

def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the GPU path has no CPU fallback)")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_08963_gb300 import binding as B
    from paper_1911_08963_gb300 import inputs

    G, n, k = inputs.single_code(args.workload)
    stream = torch.cuda.current_stream()
    opt = B.md_options_init(max_stage=args.max_stage, filter=args.filter, tensor=args.tensor,
                            stream=stream.cuda_stream)
    h = B.md_create(G, n, k, opt)
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step():
        d, wit = B.md_compute(h, n)
        return d, B.md_info_get(h), B.md_levels(h, with_time=True)

    for _ in range(args.warmup):
        step()
        l2_flush.zero_()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index())
    sampler.start()
    ev = []
    infos = []
    lev_all = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d, info, levels = step()
        e1.record(stream)
        ev.append((e0, e1))
        infos.append(info)
        lev_all.append(levels)
        l2_flush.zero_()                  # outside the events: the next step starts with a cold L2
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    cw = sum(i["codewords"] for i in infos)
    launches = sum(i["gpu_launches"] for i in infos)
    total_s, cw = reduce_over_ranks(total_s, cw, "cuda")
    value = cw / total_s

    # roofline of the dominant kernel: the enumeration kernels of the deepest stage
    top_g = max(lv[0] for lv in lev_all[0])
    top = [lv for levels in lev_all for lv in levels if lv[0] == top_g]
    top_cw = sum(lv[4] for lv in top)
    top_s = sum(lv[5] for lv in top)
    per_launch_cw = top_cw / len(top)
    per_launch_s = top_s / len(top)
    roofline = roofline_line(args, n, k, top_g, len(top), per_launch_cw, per_launch_s, max(lv[6] for lv in top))

    line = {
        "metric": "codewords/s", "value": value, "unit": "codewords/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": data_string(args.workload),
        "config": dict(workload_config(args, n, k), codewords_per_step=infos[0]["codewords"],
                       parallelism="replicas" if ws > 1 else "single GPU"),
        "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
        "d_after_stages": infos[0]["d"],
    }

    if rank == 0 and roofline.get("bound") == "tensor":
        # the tensor pipe's fp8 rate measured on this GPU (after the timed region), at the SM
        # clock the timed region ran at: a second denominator beside the cuBLAS-derived peak
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or measured_peaks().get("sm_max_mhz") or NOMINAL_MAX_MHZ
        try:
            roofline["clock_matched"] = clock_matched(roofline, B.md_mma_rate(), sms, mhz)
        except B.MDError as e:                  # the headline line is printed either way
            roofline["clock_matched"] = {"error": str(e)}

    def leg(key, fn):
        """A measurement after the timed steps: its failure is recorded under its key, and the
        line (with the timed value) is printed all the same."""
        try:
            fn()
        except Exception as e:                  # noqa: BLE001 -- reported in the JSON line
            line[key] = {"error": "%s: %s" % (type(e).__name__, e)}

    def e2e_leg():
        # end to end through the C ABI from host buffers: create (host G), compute, destroy
        opt_e = B.md_options_init(max_stage=args.max_stage, filter=args.filter, tensor=args.tensor)
        times, h2d, d2h, cwe = [], 0, 0, 0
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            hh = B.md_create(G, n, k, opt_e)
            B.md_compute(hh, n)
            inf = B.md_info_get(hh)
            B.md_destroy(hh)
            times.append(time.perf_counter() - t0)
            h2d += inf["h2d_bytes"] + G.nbytes
            d2h += inf["d2h_bytes"]
            cwe += inf["codewords"]
        line["e2e"] = {"value": cwe / sum(times), "unit": "codewords/s", "steps": e2e_steps,
                       "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps}

    def cpu_leg():
        threads = os.cpu_count() or 1
        rate, size, dt = oracle_sample_rate(G, n, k, args.max_stage, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": rate, "unit": "codewords/s", "cores": threads, "kind": "oracle",
                                "sample": "colex-rank prefix of level (g=%d, Gamma_1): %d combinations, %.1f s"
                                          % (args.max_stage, size, dt)}

    def time_to_d_leg():
        opt_f = B.md_options_init(filter=args.filter, tensor=args.tensor, stream=stream.cuda_stream)
        hf = B.md_create(G, n, k, opt_f)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        dfull, wit = B.md_compute(hf, n)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        inf = B.md_info_get(hf)
        B.md_destroy(hf)
        line["time_to_d"] = {"d": dfull, "seconds_device": e0.elapsed_time(e1) * 1e-3, "seconds_wall": wall,
                             "codewords": inf["codewords"], "stop_stage": inf["stop_g"],
                             "complete": inf["complete"]}

    def popcount_leg():
        # the popcount kernels on the same workload (md_options.tensor = 0), against the POPC
        # peak measured on this GPU: its rate per SM and clock x SMs x the SM clock
        per_sm_clk = B.md_popc_rate()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        sampler = ClockSampler(gpu_index())
        sampler.start()
        hp = B.md_create(G, n, k, B.md_options_init(max_stage=args.max_stage, filter=args.filter, tensor=0,
                                                    stream=stream.cuda_stream))
        B.md_compute(hp, n)
        info_p = B.md_info_get(hp)
        lev_p = B.md_levels(hp, with_time=True)
        B.md_destroy(hp)
        clocks_p = sampler.stop()
        gtop = max(lv[0] for lv in lev_p)
        top_p = [lv for lv in lev_p if lv[0] == gtop]
        mhz = clocks_p.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or NOMINAL_MAX_MHZ
        rp = popc_roofline(per_sm_clk, sms, mhz, gtop, len(top_p), sum(lv[4] for lv in top_p) / len(top_p),
                           sum(lv[5] for lv in top_p) / len(top_p),
                           "md_popc_rate on this GPU: %.2f popc/clk/SM x %d SMs x %.0f MHz max SM clock"
                           % (per_sm_clk, sms, mhz))
        rp.update({"popc_per_sm_per_clk": per_sm_clk, "codewords_per_s": info_p["codewords"] / info_p["seconds_device"],
                   "clocks": clocks_p, "run": "md_compute with tensor = 0, stages g <= %d" % args.max_stage})
        line["roofline_popcount"] = rp

    def batch_leg():
        import tempfile
        cache = os.path.join(tempfile.gettempdir(), "md_tune_bench_%d.json" % os.getpid())
        try:
            line["batch"] = batch_measure(args, B, inputs, 0, cache)
            line["batch_budget_1e10"] = batch_measure(args, B, inputs, int(1e10), cache)
        finally:
            if os.path.exists(cache):
                os.remove(cache)

    def serve_leg():
        line["serve"] = serve_measure(args, B, inputs)

    if rank == 0 and not args.no_e2e:
        leg("e2e", e2e_leg)
    if rank == 0 and ws == 1 and not args.no_cpu:
        leg("cpu_baseline", cpu_leg)
    if rank == 0 and ws == 1 and not args.no_time_to_d:
        leg("time_to_d", time_to_d_leg)
    if rank == 0 and ws == 1 and args.tensor and not args.no_popcount and args.workload == "rand200x100":
        leg("roofline_popcount", popcount_leg)
    if rank == 0 and ws == 1 and not args.no_batch:
        leg("batch", batch_leg)
    if rank == 0 and ws == 1 and not args.no_serve:
        leg("serve", serve_leg)

    if args.verbose and rank == 0:
        for lv in lev_all[0]:
            sys.stderr.write("level g=%d j=%d weight=%d rank=%d count=%d kernel=%.4f s  %.3e cw/s\n"
                             % (lv[0], lv[1], lv[2], lv[3], lv[4], lv[5], lv[4] / max(lv[5], 1e-9)))
    B.md_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def batch_measure(args, B, inputs, budget, tune_cache=None):
    """The uneven batch (seed 4): md_batch with options picked by md_batch_tune against one
    md_compute per code (the per-code launch loop), same GPU and stream, clocks sampled over
    both.  budget = per-code estimated work limit (0 = every code)."""
    import torch
    codes = inputs.batch_codes(count=args.batch_count)
    base = B.md_options_init(work_budget=budget, batch_workers=args.batch_workers)
    t0 = time.perf_counter()
    opt = B.md_batch_tune(codes, base, tune_cache)
    t_tune = time.perf_counter() - t0
    opt_loop = B.md_options_init(work_budget=budget, batch_mode=1)
    B.md_batch(codes[:64], opt)                    # warm-up (module load, first allocations)
    B.md_batch(codes[:64], opt_loop)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index())
    sampler.start()
    t0 = time.perf_counter()
    d_b, w_b, st_b = B.md_batch(codes, opt)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    d_l, w_l, st_l = B.md_batch(codes, opt_loop)
    t_loop = time.perf_counter() - t0
    clocks = sampler.stop()
    same = d_b == d_l and st_b == st_l and all((x == y).all() for x, y in zip(w_b, w_l))
    done = sum(1 for s_ in st_b if s_ == B.MD_OK)
    skipped = sum(1 for s_ in st_b if s_ == B.MD_EBUDGET)
    hist = {}
    for (G, n, k), s_ in zip(codes, st_b):
        key = "n%d-%d" % (n // 25 * 25, n // 25 * 25 + 24)
        h = hist.setdefault(key, [0, 0])
        h[0 if s_ == B.MD_OK else 1] += 1
    return {"metric": "codes/s (batched vs per-code loop)", "value": done / t_batch, "unit": "codes/s",
            "per_code_loop": done / t_loop, "speedup": t_loop / t_batch, "codes": len(codes), "completed": done,
            "skipped_over_budget": skipped, "seconds_batched": t_batch, "seconds_loop": t_loop,
            "identical_results": same, "higher_is_better": True, "n_gpus": 1, "clocks": clocks,
            "tuned": {"chunk_log2": opt.chunk_log2, "blocks_per_sm": opt.blocks_per_sm,
                      "batch_heavy": opt.batch_heavy, "seconds": t_tune},
            "config": {"workload": "%d random codes, seed 4, n~U{48..160}, k~U{n/3..n/2}" % len(codes),
                       "work_budget": budget, "batch_workers": opt.batch_workers or 2,
                       "histogram_done_skipped_by_n": hist}}


def serve_measure(args, B, inputs):
    """Poisson stream (seed 5, 200 requests/s) through the continuous-batching server; requests
    whose estimated work exceeds the budget are refused at submission (admission by work)."""
    trace = inputs.serving_trace(args.serve_count)
    heavy = 2 ** 64 - 1 if args.serve_heavy < 0 else int(args.serve_heavy)
    s = B.md_server_create(slots=args.serve_slots, work_budget=int(args.serve_budget), heavy=heavy)
    # warm-up: a few small codes through the server
    for t, G, n, k in trace[:8]:
        try:
            tk = B.md_server_submit(s, G, n, k)
            while B.md_server_poll(s, tk, n) is None:
                time.sleep(0.0005)
        except B.MDError:
            pass
    outstanding = {}
    lat = []
    rejected = 0
    lock = threading.Lock()
    stop = [False]
    sampler = ClockSampler(gpu_index())
    sampler.start()
    start = time.perf_counter()

    def poller():
        while not stop[0] or outstanding:
            with lock:
                items = list(outstanding.items())
            for tk, (arr, n) in items:
                r = B.md_server_poll(s, tk, n)
                if r is not None:
                    now = time.perf_counter() - start
                    with lock:
                        del outstanding[tk]
                        lat.append((now - arr, r[2]))
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    for arr, G, n, k in trace:
        delay = arr - (time.perf_counter() - start)
        if delay > 0:
            time.sleep(delay)
        try:
            tk = B.md_server_submit(s, G, n, k)
            with lock:
                outstanding[tk] = (arr, n)
        except B.MDError as e:
            if e.code != B.MD_EBUDGET:
                raise
            rejected += 1
    stop[0] = True
    th.join()
    makespan = time.perf_counter() - start
    clocks = sampler.stop()
    B.md_server_destroy(s)
    ok = sorted(x for x, st in lat if st == B.MD_OK)
    p = lambda q: ok[min(len(ok) - 1, int(q * len(ok)))] if ok else None
    return {"metric": "serving latency p50/p99 and codes/s", "value": len(ok) / makespan, "unit": "codes/s",
            "p50_ms": p(0.50) * 1e3 if ok else None, "p99_ms": p(0.99) * 1e3 if ok else None,
            "completed": len(ok), "rejected_over_budget": rejected, "requests": len(trace),
            "makespan_s": makespan, "trace_s": trace[-1][0], "higher_is_better": True, "n_gpus": 1,
            "clocks": clocks,
            "config": {"workload": "Poisson arrivals 200/s, seed 5, n~U{64..200}, k=n/2+U{-8..8}",
                       "work_budget": int(args.serve_budget), "slots": args.serve_slots,
                       "heavy": "never" if args.serve_heavy < 0 else int(args.serve_heavy) or 2 ** 30}}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_08963_gb300 import binding as B
    from paper_1911_08963_gb300 import inputs
    print(json.dumps(batch_measure(args, B, inputs, int(args.batch_budget))), flush=True)
    return 0


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_08963_gb300 import binding as B
    from paper_1911_08963_gb300 import inputs
    print(json.dumps(serve_measure(args, B, inputs)), flush=True)
    return 0


def run_profile_once(args):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_08963_gb300 import binding as B
    from paper_1911_08963_gb300 import inputs
    G, n, k = inputs.single_code(args.workload)
    h = B.md_create(G, n, k, B.md_options_init(max_stage=args.max_stage, filter=args.filter, tensor=args.tensor))
    d, _ = B.md_compute(h, n)
    info = B.md_info_get(h)
    B.md_destroy(h)
    print(json.dumps({"workload": args.workload, "max_stage": args.max_stage, "d": d,
                      "codewords": info["codewords"], "seconds_device": info["seconds_device"]}))
    return 0


def main():
    args = parse()
    if args.profile_once:
        return run_profile_once(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
