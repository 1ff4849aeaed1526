#!/usr/bin/env python3
"""Throughput of the N-FHMM variational sweep on GB300: frame-iterations/s.

One step = one separation job of the paper-size workload (S=2 sources, N=40
dictionaries of K=10 elements, F=513 bins, T=3000 frames) taken through the
whole hot path: initial state from the job's inputs, 50 sweeps (Eq. 6,
Eqs. 7 and 8, forward-backward per source) and the variational bound.
frame-iterations per step = T * 50.

* ``value``: inputs already resident in HBM; the step runs through the
  library's C ABI from device pointers.  L2 (129 MB) is flushed by a 256 MB
  write before every timed step; each step is timed with CUDA events on the
  stream that launches it.
* ``e2e``: the same step through the same public API from pinned host
  buffers: host->device copies of V, W, A, pi and the device->host read of the
  posteriors and bound are inside the timed region.
* ``roofline``: the stage with the largest summed CUDA-event time inside the
  timed region, its algorithmic flops or bytes per launch over its mean
  launch time, against the measured peaks.
* ``cpu_baseline``: the FP64 oracle on a bounded sample of the same
  workload, timed on this host's cores (rank 0, one GPU only).

The default run (one GPU) adds three sub-lines to the same JSON line, each
timed the same way with its own clock record: ``batched_fp32`` and
``batched_bf16`` (64 jobs, T ~ U[500, 8000], one batch; the BF16 form is
the precision form of the contractions) and ``serving`` (Poisson arrivals
at 200 jobs/s for 5 s through continuous batching, with p50/p99 latency).

``--impl reference`` times the FP64 oracle alone (the reference arm).
Multi-GPU (torchrun): each rank runs its own independent jobs (replicas, no
collective on the data path); ``value`` is all ranks' frame-iterations over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VI frame·iterations/s (S=2,N=40,K=10,F=513) vs roofline; p50/p99 job latency"
UNIT = "frame·iterations/s"
SWEEPS = 50
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
TF32_OVER_BF16 = 1.1 / 2.25                              # nominal dense ratio
# stage events bracket every PROFILE_STRIDE-th sweep of the timed region
# (the rest replay the same one-sweep graph without events)
PROFILE_STRIDE = 10
TIMED_NOTE = f"stages of every {PROFILE_STRIDE}th sweep bracketed by CUDA events"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--sweeps", type=int, default=SWEEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run one context for 3 sweeps and exit (a small case for ncu)")
    ap.add_argument("--fb-mode", type=int, default=None,
                    help="the forward-backward form (0 scan, k >= 1 sequential with k chains "
                         "per block): with --ncu-case --workload batched instead of the "
                         "autotuner's choice; with --workload serving for the serving batches "
                         "(default: the scan)")
    ap.add_argument("--fb-chunk", type=int, default=None,
                    help="single workload: frames per forward-backward chunk instead of the "
                         "autotuner's choice (for profiler runs)")
    ap.add_argument("--fb-group", type=int, default=None,
                    help="with --fb-chunk: chunks per group (0: none)")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "serving", "exact"],
                    help="single: one S2 N40 K10 F513 T3000 job per step (the headline); "
                         "batched: 64 jobs, T ~ U[500, 8000], in one batch per step; "
                         "serving: Poisson arrivals served by continuous batching; "
                         "exact: exact-inference EM iteration against a variational sweep")
    ap.add_argument("--exact-frames", type=int, default=3000)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-saturate", action="store_true",
                    help="serving: every request queued at the start (peak throughput)")
    ap.add_argument("--no-extras", action="store_true",
                    help="single workload only: skip the batched and serving sub-lines")
    ap.add_argument("--extra-steps", type=int, default=4,
                    help="timed steps of each batched sub-line (after 3 warm-up steps)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_seed(rank: int) -> int:
    """Each rank separates its own job: the replicas share no data."""
    return rank


def aggregate(frame_its_per_rank: float, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job frame-iterations/s: all ranks' work over the slowest rank's time."""
    return world * frame_its_per_rank * steps / (slowest_ms / 1e3)


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks(probe=None):
    """Roofline denominators: MEASURED_PEAKS.json (else the fallback), and
    the tensor-core rates measured in this run by nfhmm_mma_rate (probe)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        out = {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
               "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
               "source": "measured"}
    else:
        out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
               "source": "fallback"}
    if probe:
        out["tf32_probe"] = probe.get("tf32")
        out["probe_record"] = probe
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_single_thread(seconds_hint: float = 8.0):
    """The oracle timed with its BLAS held to one thread: a child process
    started with OPENBLAS_NUM_THREADS=1 (the BLAS reads it at load time)."""
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(seconds_hint=%r)))" % (ROOT, seconds_hint))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=120)
        v, _, sample = json.loads(r.stdout.strip().splitlines()[-1])
        return v, sample
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None, None


def cpu_baseline_record():
    """The FP64 oracle on the host: all cores, and one BLAS thread."""
    v, cores, sample = oracle_sample(seconds_hint=12.0)
    v1, sample1 = oracle_sample_single_thread(seconds_hint=8.0)
    rec = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
           "cpu_model": cpu_model(), "os_cpu_count": os.cpu_count()}
    if v1 is not None:
        rec["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                "blas_threads": "OPENBLAS_NUM_THREADS=1", "sample": sample1}
    return rec


def oracle_sample(seconds_hint: float = 20.0, sweeps: int = None):
    """Time the FP64 oracle on the paper-size workload (a bounded number of
    sweeps from the initial state).  Returns (frame-its/s, cores, sample)."""
    import numpy as np  # noqa: F401
    from oracle import vi
    from paper_1206_6468_gb300 import synth
    p = synth.make_problem(seed=0, **synth.PAPER_SIZE)
    B = vi.element_mask(p.S, p.N, p.K)
    counts, dhat = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    t0 = time.perf_counter()
    n = 0
    while True:
        st = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, counts, dhat, B)
        counts, dhat = st["counts"], st["dhat"]
        n += 1
        el = time.perf_counter() - t0
        if (sweeps is not None and n >= sweeps) or (sweeps is None and el >= seconds_hint):
            break
    vi.bound(p.V, p.W, st["alpha"], st["logZ"], p.gamma, p.S, p.K, Vhat=st["Vhat"])
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    return p.T * n / el, cores, f"{n} sweeps + bound of S2 N40 K10 F513 T3000 (FP64 NumPy)"


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import vi
    from paper_1206_6468_gb300 import synth
    p = synth.make_problem(seed=0, **synth.PAPER_SIZE)
    B = vi.element_mask(p.S, p.N, p.K)
    counts, dhat = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, counts, dhat, B)
        counts, dhat = st["counts"], st["dhat"]
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
    tot = sum(times)
    value = p.T * len(times) / tot
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    sample = "one sweep of S2 N40 K10 F513 T3000 per step (FP64 NumPy oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "S2 N40 K10 F513 T3000, one sweep per step", "S": 2,
                       "N": 40, "K": 10, "F": 513, "T": 3000},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def stage_cost(stage, p, precision, tc):
    """Algorithmic work per launch of one stage: (bound, amount, unit, peak_key)."""
    S, N, K, F, T = p.S, p.N, p.K, p.F, p.T
    M = S * N * K
    if stage in ("gemm1", "gemm2"):
        flops = 2.0 * T * F * M
        if tc:
            return "tensor", flops, "TFLOP/s"
        return "alu", flops, "TFLOP/s"
    if stage == "weights":
        # counts in, w (float) and the contraction operand out (bf16: 2 bytes,
        # split tf32: 8), d-hat in and phi-hat out; alpha-hat is stored by the
        # last sweep of a run only
        op = (2 if precision == "bf16" else 8) if tc else 0
        return "hbm", 4.0 * (2 * T * M + 2 * S * T * N) + op * T * M, "GB/s"
    if stage == "fb":
        return "hbm", 4.0 * (2 * S * T * N + S * N * N), "GB/s"
    if stage == "bound":
        return "hbm", 4.0 * T * M, "GB/s"
    return "hbm", 0.0, "GB/s"


def csrc_digest():
    """sha256 over every kernel and header source of the library."""
    import hashlib
    d = os.path.join(ROOT, "paper_1206_6468_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def measured_traffic(stage, workload):
    """DRAM bytes per stage invocation from the committed ncu summary
    profiles/traffic_<workload>.txt, or None when the library's sources
    changed since the counters were taken (the summary records their
    sha256)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    want = val = None
    for line in open(path):
        parts = line.split()
        if len(parts) == 2 and parts[0] == "csrc_sha256":
            want = parts[1]
        if len(parts) == 3 and parts[0] == "stage" and parts[1] == stage:
            val = float(parts[2])
    if want is None or val is None or want != csrc_digest():
        return None
    return val


def fb_serial_steps(longest, mode, L, G):
    """Frame steps on the forward-backward's critical path: the longest
    chain's frames for the sequential form; for the scan, a chunk's frames
    twice (products, replay) plus the scan across the longest chain's chunks
    (over groups and within one when grouped)."""
    if mode > 0:
        return longest, "sequential"
    C = -(-longest // L)
    return 2 * L + (G + -(-C // G) if G >= 2 else C), "scan"


def tensor_peak(precision, peaks):
    """(peak TFLOP/s, note) of a tensor-core contraction of this precision.
    The split-TF32 (FP32) form runs tf32 MMAs: their rate measured in this run
    by nfhmm_mma_rate, else the measured bf16 sustained rate x the nominal
    1.1/2.25 tf32/bf16 ratio; it issues three tf32 MMAs per product, so its
    own ceiling is a third of the peak (reported beside it)."""
    if precision == "bf16":
        return peaks["bf16_tflops_sustained"], f"{peaks['source']} bf16 sustained (MEASURED_PEAKS.json)"
    if peaks.get("tf32_probe"):
        return peaks["tf32_probe"], "tf32 MMA rate measured in this run (nfhmm_mma_rate, burst)"
    return (peaks["bf16_tflops_sustained"] * TF32_OVER_BF16,
            f"{peaks['source']} bf16 sustained x 1.1/2.25 (tf32)")


def stage_rooflines(prof, T, S, N, K, F, precision, tc, peaks, fb_path=None):
    """Achieved against peak for every sweep stage, from the same live
    events (the contractions run beside the forward-backward, so their times
    include sharing the SMs with it).  fb_path = (serial steps, form): the
    forward-backward also gets its critical-path model, the live time per
    serial frame step."""
    class _P:
        pass
    q = _P()
    q.S, q.N, q.K, q.F, q.T = S, N, K, F, T
    out = {}
    for st in ("weights", "gemm1", "gemm2", "fb"):
        ms, inv, _ = prof.get(st, (0.0, 0, 0))
        if inv <= 0 or ms <= 0:
            continue
        bound_kind, amount, unit = stage_cost(st, q, precision, tc)
        avg_s = ms / 1e3 / inv
        extra = {}
        if unit == "TFLOP/s":
            achieved = amount / avg_s / 1e12
            if bound_kind == "tensor":
                peak, _ = tensor_peak(precision, peaks)
                if precision == "fp32":
                    extra = {"mmas_per_product": 3, "split_tf32_ceiling": round(peak / 3, 1),
                             "frac_of_split_ceiling": round(3 * achieved / peak, 4)}
            else:
                peak = FP32_SIMT_PEAK_TFLOPS
        else:
            achieved = amount / avg_s / 1e9
            peak = peaks["hbm_gbs"]
        out[st] = {"bound": bound_kind, "achieved": round(achieved, 2), "peak": round(peak, 1),
                   "unit": unit, "frac": round(achieved / peak, 4), "ms": round(1e3 * avg_s, 4)}
        out[st].update(extra)
        if st == "fb" and fb_path:
            out[st]["critical_path"] = {"form": fb_path[1], "serial_steps": int(fb_path[0]),
                                        "ns_per_step": round(1e9 * avg_s / fb_path[0], 1)}
    return out


def roofline_of(prof, T, S, N, K, F, precision, tc, peaks, sweeps_run, traffic_workload=None,
                fb_path=None):
    """Roofline object of the stage with the largest summed event time."""
    class _P:
        pass
    q = _P()
    q.S, q.N, q.K, q.F, q.T = S, N, K, F, T
    dom = max((s for s in prof if s != "init"), key=lambda s: prof[s][0])
    dom_ms, dom_inv, dom_launches = prof[dom]
    bound_kind, amount, unit = stage_cost(dom, q, precision, tc)
    avg_s = dom_ms / 1e3 / max(dom_inv, 1)
    if unit == "TFLOP/s":
        achieved = amount / avg_s / 1e12
        if bound_kind == "tensor":
            peak, note = tensor_peak(precision, peaks)
        else:
            peak = FP32_SIMT_PEAK_TFLOPS
            note = "derived FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 x 2.07 GHz"
    else:
        achieved = amount / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        note = f"{peaks['source']} HBM copy bandwidth"
    out = {"bound": bound_kind, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak,
           "traffic": measured_traffic(dom, traffic_workload) if traffic_workload else None,
           "peak_source": note, "launch_ms": 1e3 * avg_s,
           "launches_per_invocation": dom_launches / max(sweeps_run, 1),
           "stage_ms_per_invocation": {s: round(prof[s][0] / max(prof[s][1], 1), 4)
                                       for s in prof},
           "timed_sweeps": TIMED_NOTE}
    if dom == "fb" and fb_path:
        # a serial chain: its latency, not HBM, is what limits it
        out["limit"] = {"kind": "serial chain (critical path)", "form": fb_path[1],
                        "serial_frame_steps": int(fb_path[0]),
                        "ns_per_step": round(1e9 * avg_s / fb_path[0], 1)}
    return out


def timed_steps(fn, n, world, flush, stream):
    """n steps of fn, each timed by CUDA events on the launching stream,
    with L2 flushed (a 256 MB write) before each; barrier and synchronise on
    both sides."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n)]
    barrier(world)
    torch.cuda.synchronize()
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return [e0.elapsed_time(e1) for e0, e1 in evs]


def batched_jobs(rank, n_jobs=64):
    from paper_1206_6468_gb300 import synth
    lengths = synth.batched_lengths(n_jobs, 500, 8000, seed=job_seed(rank))
    jobs = synth.make_jobs(2, 40, 10, 513, lengths, self_prob=0.95, energy_sigma=1.5,
                           seed=job_seed(rank))
    return lengths, jobs


def run_batched(args, rank, world, local, precision=None, data=None, steps=None, warmup=None):
    """64 jobs of T ~ U[500, 8000] frames sharing one S2 N40 K10 F513 model,
    run as one batch: one step = initial state + 50 sweeps + bound of all.
    Returns the line (None for --ncu-case)."""
    import torch

    from paper_1206_6468_gb300 import nfhmm
    precision = precision or args.precision
    steps = steps or args.steps
    warmup = max(3, warmup or args.warmup)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lengths, jobs = data or batched_jobs(rank, 16 if args.ncu_case else 64)
    f32 = {"V": jobs.stacked_V()}
    for k in ("W", "A", "pi"):
        f32[k] = np.ascontiguousarray(getattr(jobs, k), dtype=np.float32)
    T = int(lengths.sum())
    d_in = {k: torch.from_numpy(v).to(dev) for k, v in f32.items()}
    h_in = {k: torch.from_numpy(v).pin_memory() for k, v in f32.items()}
    h_dhat = torch.empty((jobs.S, T, jobs.N), dtype=torch.float32).pin_memory()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ctx = nfhmm.VIContext(d_in["V"], d_in["W"], d_in["A"], d_in["pi"], jobs.S, jobs.N, jobs.K,
                          precision=precision, job_frames=lengths.tolist())
    sweeps = args.sweeps
    if args.ncu_case:
        # the form the bench runs (one sweep, the autotuner), or the one asked
        # for, then three sweeps
        if args.fb_mode is None:
            ctx.sweep(1)
            print("autotuned:", ctx.autotune(reps=1), flush=True)
        else:
            ctx.set_option("fb_mode", args.fb_mode)
        print("bound after 3 sweeps:", ctx.sweep(3, bound=True), flush=True)
        ctx.close()
        return None
    # forward-backward geometry picked by the library's autotuner on these
    # jobs (one sweep first: it times whole sweeps from the current state)
    ctx.sweep(1)
    tuned = ctx.autotune(reps=3)

    def step_device():
        ctx.reinit(d_in["V"], d_in["W"], d_in["A"], d_in["pi"])
        return ctx.sweep(sweeps, bound=True)

    def step_e2e():
        ctx.reinit(h_in["V"], h_in["W"], h_in["A"], h_in["pi"])
        L = ctx.sweep(sweeps, bound=True)
        ctx.posteriors(out=h_dhat)
        return L

    ctx.set_option("profile_stride", PROFILE_STRIDE)
    ctx.profile_enable(True)
    for _ in range(warmup):
        step_device()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    for st in nfhmm.STAGES:
        ctx.profile_read(st, reset=True)
    l0 = ctx.kernel_launches()
    ms = timed_steps(step_device, steps, world, flush, stream)
    launches = ctx.kernel_launches() - l0
    prof = {st: ctx.profile_read(st, reset=True) for st in nfhmm.STAGES}
    for _ in range(2):
        step_e2e()
    ms_e2e = timed_steps(step_e2e, steps, world, flush, stream)
    ctx.profile_enable(False)
    clocks = sampler.stop()
    tot_ms = max_over_ranks(sum(ms), world)
    tot_e2e = max_over_ranks(sum(ms_e2e), world)
    fit = T * sweeps
    peaks = load_peaks(getattr(args, "_tensor_probe", None))
    tc = bool(ctx.query("tensor_cores"))
    fb_path = fb_serial_steps(int(lengths.max()), ctx.query("fb_mode"), ctx.query("fb_chunk"),
                              ctx.query("fb_group"))
    line = {
        "metric": METRIC, "value": aggregate(fit, steps, world, tot_ms), "unit": UNIT,
        "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": tot_ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "bf16",
        "data": "synthetic",
        "config": {"workload": f"batched: {len(lengths)} jobs, T ~ U[500, 8000] (sum {T}), "
                               f"S2 N40 K10 F513, {sweeps} sweeps + bound per step",
                   "jobs": len(lengths), "frames": T, "sweeps_per_step": sweeps,
                   "precision": precision, "contractions": "tcgen05" if tc else "fp32 SIMT",
                   "l2": "inputs larger than L2; flushed between steps (256 MB write)",
                   "fb_geometry": {"chunk": tuned["fb_chunk"], "group": tuned["fb_group"],
                                   "mode": "sequential x%d" % tuned["fb_mode"]
                                   if tuned["fb_mode"] else "scan",
                                   "picked_by": "nfhmm_autotune",
                                   "sweep_us": round(tuned["us"], 1)},
                   "contraction_tiles": dict(tuned.get("tiles") or {}, picked_by="nfhmm_autotune"),
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline_of(prof, T, 2, 40, 10, 513, precision, tc, peaks, steps * sweeps,
                                fb_path=fb_path),
        "roofline_by_stage": stage_rooflines(prof, T, 2, 40, 10, 513, precision, tc, peaks,
                                             fb_path),
        "e2e": {"value": aggregate(fit, steps, world, tot_e2e), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(v.numel() * 4 for v in h_in.values())),
                "d2h_bytes_per_step": int(h_dhat.numel() * 4 + 8)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    ctx.close()
    del d_in, h_in, h_dhat, flush
    torch.cuda.empty_cache()
    return line


def run_serving(args, rank, world, local):
    """Continuous batching: requests arrive as a Poisson process (rate
    --serve-rate per second for --serve-seconds), T log-uniform in
    [200, 10000], half on an S=2 and half on an S=3 model (N40 K10 F513);
    each runs until its bound moves by less than 1e-5 relative or 100 sweeps.
    Returns the line."""
    import torch

    from paper_1206_6468_gb300 import nfhmm, synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rng = np.random.Generator(np.random.PCG64(1000 + job_seed(rank)))
    pool_n, t_max = 8, 10000
    models = [synth.make_jobs(S, 40, 10, 513, [t_max] * pool_n, self_prob=0.95,
                              energy_sigma=1.5, seed=100 * S + job_seed(rank)) for S in (2, 3)]
    # request spectrograms arrive in pinned host buffers, as a serving front end would hold them
    pools = [[torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).pin_memory().numpy()
              for v in m.V] for m in models]
    n_req = int(rng.poisson(args.serve_rate * args.serve_seconds))
    arrivals = np.sort(rng.uniform(0.0, args.serve_seconds, size=n_req))
    Ts = np.exp(rng.uniform(np.log(200), np.log(t_max), size=n_req)).astype(int)
    which = rng.integers(0, 2, size=n_req)
    item = rng.integers(0, pool_n, size=n_req)
    reqs = [(int(which[r]), pools[which[r]][item[r]][:Ts[r]], float(arrivals[r]))
            for r in range(n_req)]
    capacity, max_jobs = 1 << 17, 512

    def batches():
        out = [nfhmm.Batch(np.ascontiguousarray(m.W, dtype=np.float32),
                           np.ascontiguousarray(m.A, dtype=np.float32),
                           np.ascontiguousarray(m.pi, dtype=np.float32), m.S, m.N, m.K,
                           capacity=capacity, max_jobs=max_jobs, precision=args.precision)
               for m in models]
        if args.fb_mode is not None:
            for b in out:
                b.set_option("fb_mode", args.fb_mode)
        return out

    warm = batches()
    nfhmm.serve(warm, reqs[:8], max_sweeps=5, realtime=False, want_posteriors=False)
    for b in warm:
        b.close()
    bs = batches()
    l0 = sum(b.kernel_launches() for b in bs)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    t0 = time.perf_counter()
    res, _ = nfhmm.serve(bs, reqs, rel_tol=1e-5, max_sweeps=100,
                         realtime=not args.serve_saturate, want_posteriors=True)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    launches = sum(b.kernel_launches() for b in bs) - l0
    ok = [r for r in res if r["status"] == nfhmm.OK]
    fit = sum(Ts[i] * res[i]["sweeps"] for i in range(n_req) if res[i]["status"] == nfhmm.OK)
    lat = np.array([(r["done_s"] - (0.0 if args.serve_saturate else arrivals[i])) * 1e3
                    for i, r in enumerate(res) if r["status"] == nfhmm.OK])
    value = fit / wall
    line = {
        "metric": METRIC, "value": value * world, "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
        "data": "synthetic",
        "config": {"workload": ("serving, all queued at start" if args.serve_saturate else
                                f"serving, Poisson {args.serve_rate:g} jobs/s for "
                                f"{args.serve_seconds:g} s") +
                               ", T log-uniform [200, 10000], S in {2, 3}, N40 K10 F513, "
                               "until |dL| < 1e-5 |L| or 100 sweeps",
                   "requests": n_req, "completed": len(ok), "frames": int(Ts.sum()),
                   "batch_capacity_frames": capacity, "max_jobs": max_jobs,
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "fb_mode": "sequential x%d" % args.fb_mode if args.fb_mode else "scan",
                   "timing": "host wall clock from the first arrival to the last result "
                             "(latency = result time - arrival time)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "sweeps": {"mean": float(np.mean([r["sweeps"] for r in ok])),
                   "max": int(max(r["sweeps"] for r in ok))},
        "e2e": {"value": value * world, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(Ts) * 513 * 4),
                "d2h_bytes_per_step": int(sum(Ts[i] * (2 + which[i]) * 40 * 4 for i in range(n_req)))},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    for b in bs:
        b.close()
    return line


def run_exact(args, rank, world, local):
    """Per-iteration time of exact inference in the original N-FHMM (EM over
    the N^S joint states) against a variational sweep on the same
    spectrogram, at the configurations of Section 5's comparison: S=2 sources
    of N=20 dictionaries with K=30 elements (exact inference's best) and
    K=20 (the variational method's best); F=513, T frames."""
    import torch

    from paper_1206_6468_gb300 import nfhmm, synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    T = args.exact_frames
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    res = {}
    sampler = ClockSampler(local)
    sampler.start()
    for K in (30, 20):
        p = synth.make_problem(S=2, N=20, K=K, F=513, T=T, self_prob=0.95, energy_sigma=1.5,
                               seed=job_seed(rank))
        f = {k: torch.from_numpy(v).to(dev) for k, v in p.as_f32().items()}
        ctx = nfhmm.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K,
                              precision=args.precision)
        ctx.sweep(5)
        vi_ms = timed(lambda: ctx.sweep(1), 50)
        ctx.close()
        x = nfhmm.ExactNFHMM(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K,
                             precision=args.precision)
        x.iterate(2, loglik=False)
        ex_ms = timed(lambda: x.iterate(1, loglik=False), 5)
        ll = x.iterate(1)
        x.close()
        res[K] = {"vi_ms_per_sweep": vi_ms, "exact_ms_per_iteration": ex_ms,
                  "exact_over_vi": ex_ms / vi_ms, "exact_loglik": ll}
    clocks = sampler.stop()
    line = {
        "metric": "exact N-FHMM EM iteration time / variational sweep time", "value":
            res[30]["exact_ms_per_iteration"] / res[20]["vi_ms_per_sweep"],
        "unit": "x", "n_gpus": world, "steps": 5, "warmup": 2,
        "ms_per_step": res[30]["exact_ms_per_iteration"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "bf16", "data": "synthetic",
        "config": {"workload": f"exact vs variational, S2 N20 F513 T{T}; exact K30, "
                               "variational K20 (each method's best configuration in Section 5)",
                   "joint_states": 400, "precision": args.precision},
        "by_config": {f"K{K}": v for K, v in res.items()},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_single(args, rank, world, local):
    """One paper-size job per step: initial state, 50 sweeps, bound.  Returns
    the line (None for --ncu-case)."""
    import torch

    from paper_1206_6468_gb300 import nfhmm, synth
    assert torch.cuda.is_available(), "bench.py needs a GPU"
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = synth.make_problem(seed=job_seed(rank), **synth.PAPER_SIZE)
    f32 = p.as_f32()
    d_in = {k: torch.from_numpy(v).to(dev) for k, v in f32.items()}
    h_in = {k: torch.from_numpy(v).pin_memory() for k, v in f32.items()}
    h_dhat = torch.empty((p.S, p.T, p.N), dtype=torch.float32).pin_memory()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    ctx = nfhmm.VIContext(d_in["V"], d_in["W"], d_in["A"], d_in["pi"], p.S, p.N, p.K,
                          gamma=p.gamma, precision=args.precision)
    sweeps = args.sweeps
    if args.ncu_case:
        if args.fb_chunk is not None:
            ctx.set_option("fb_chunk", args.fb_chunk)
        if args.fb_group is not None:
            ctx.set_option("fb_group", args.fb_group)
        print("bound after 3 sweeps:", ctx.sweep(3, bound=True), flush=True)
        ctx.close()
        return None
    # forward-backward geometry picked by the library's autotuner (whole sweeps
    # from a saved state, before the warm-up; the step re-initialises anyway),
    # or given on the command line (a profiler's serialised kernels would
    # steer the autotuner elsewhere)
    ctx.sweep(1)
    if args.fb_chunk is not None:
        ctx.set_option("fb_chunk", args.fb_chunk)
        if args.fb_group is not None:
            ctx.set_option("fb_group", args.fb_group)
        tuned = {"fb_chunk": ctx.query("fb_chunk"), "fb_group": ctx.query("fb_group"),
                 "fb_mode": ctx.query("fb_mode"), "us": None, "tiles": ctx.tiles(),
                 "picked_by": "command line"}
    else:
        tuned = ctx.autotune(reps=5)

    def step_device():
        ctx.reinit(d_in["V"], d_in["W"], d_in["A"], d_in["pi"])
        return ctx.sweep(sweeps, bound=True)

    def step_e2e():
        ctx.reinit(h_in["V"], h_in["W"], h_in["A"], h_in["pi"])
        L = ctx.sweep(sweeps, bound=True)
        ctx.posteriors(out=h_dhat)
        return L

    # warm-up with profiling on, as in the timed region (the sweeps' CUDA
    # graphs, with and without stage events, are captured here)
    ctx.set_option("profile_stride", PROFILE_STRIDE)
    ctx.profile_enable(True)
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local]))
    sampler.start()
    for st in nfhmm.STAGES:
        ctx.profile_read(st, reset=True)
    l0 = ctx.kernel_launches()
    ms = timed_steps(step_device, args.steps, world, flush, stream)
    launches = ctx.kernel_launches() - l0
    prof = {st: ctx.profile_read(st, reset=True) for st in nfhmm.STAGES}
    # end-to-end through host buffers (profiling on, as above)
    for _ in range(2):
        step_e2e()
    ms_e2e = timed_steps(step_e2e, args.steps, world, flush, stream)
    ctx.profile_enable(False)
    clocks = sampler.stop()

    frames_its = p.T * sweeps
    tot_ms = max_over_ranks(sum(ms), world)
    tot_e2e = max_over_ranks(sum(ms_e2e), world)
    value = aggregate(frames_its, args.steps, world, tot_ms)
    e2e_value = aggregate(frames_its, args.steps, world, tot_e2e)

    peaks = load_peaks(getattr(args, "_tensor_probe", None))
    tc = bool(ctx.query("tensor_cores"))
    fb_path = fb_serial_steps(p.T, ctx.query("fb_mode"), ctx.query("fb_chunk"),
                              ctx.query("fb_group"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
        "data": "synthetic",
        "config": {"workload": f"S2 N40 K10 F513 T3000, {sweeps} sweeps + bound per step",
                   "S": p.S, "N": p.N, "K": p.K, "F": p.F, "T": p.T, "sweeps_per_step": sweeps,
                   "precision": args.precision, "contractions": "tcgen05" if tc else "fp32 SIMT",
                   "l2": "flushed between steps (256 MB write)",
                   "fb_geometry": {"chunk": tuned["fb_chunk"], "group": tuned["fb_group"],
                                   "mode": "sequential x%d" % tuned["fb_mode"]
                                   if tuned["fb_mode"] else "scan",
                                   "picked_by": tuned.get("picked_by", "nfhmm_autotune"),
                                   "sweep_us": round(tuned["us"], 1) if tuned["us"] else None},
                   "contraction_tiles": dict(tuned.get("tiles") or {},
                                             picked_by=tuned.get("picked_by", "nfhmm_autotune")),
                   "parallelism": f"replicas x{world}"},
        "roofline": dict(roofline_of(prof, p.T, p.S, p.N, p.K, p.F, args.precision, tc, peaks,
                                     args.steps * sweeps, f"paper_size_{args.precision}",
                                     fb_path), fb_chunk=ctx.query("fb_chunk")),
        "roofline_by_stage": stage_rooflines(prof, p.T, p.S, p.N, p.K, p.F, args.precision, tc,
                                             peaks, fb_path),
        "tensor_peaks_measured": peaks.get("probe_record"),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(v.numel() * 4 for v in h_in.values())),
                "d2h_bytes_per_step": int(h_dhat.numel() * 4 + 8)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    ctx.close()
    del d_in, h_in, h_dhat, flush
    torch.cuda.empty_cache()
    return line


SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "e2e",
            "roofline", "roofline_by_stage", "gpu_launches", "clocks", "latency_ms", "sweeps")


def sub_line(line):
    return {k: line[k] for k in SUB_KEYS if k in line}


def measure_tensor_peaks():
    """The tensor cores' dense rates measured by the library (tf32, bf16)."""
    from paper_1206_6468_gb300 import nfhmm
    rec = {}
    for prec in ("fp32", "bf16"):
        try:
            rec["tf32" if prec == "fp32" else "bf16"] = round(nfhmm.mma_rate(prec), 1)
        except nfhmm.NfhmmError:
            pass
    rec["how"] = ("nfhmm_mma_rate: every SM issues back-to-back 128x256 MMAs (K 8 tf32 / 16 "
                  "bf16) from shared memory into TMEM; CUDA events over 5 launches")
    return rec


def main():
    args = parse()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "exact":
        run_exact(args, rank, world, local)
        return
    if not args.ncu_case:
        import torch
        torch.cuda.set_device(torch.device("cuda", local))
        args._tensor_probe = measure_tensor_peaks()
    if args.workload == "batched":
        line = run_batched(args, rank, world, local)
    elif args.workload == "serving":
        line = run_serving(args, rank, world, local)
    else:
        line = run_single(args, rank, world, local)
        if line is not None and world == 1 and not args.no_extras:
            # the batched (FP32 and BF16) and serving forms, each timed as its own line
            data = batched_jobs(rank)
            b32 = run_batched(args, rank, world, local, "fp32", data, args.extra_steps, 3)
            b16 = run_batched(args, rank, world, local, "bf16", data, args.extra_steps, 3)
            del data
            sv = run_serving(args, rank, world, local)
            line["batched_fp32"] = sub_line(b32)
            line["batched_bf16"] = sub_line(b16)
            line["serving"] = sub_line(sv)
            line["bf16_batched_over_fp32_single"] = b16["value"] / line["value"]
        if line is not None and rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_record()
    if line is not None and rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
