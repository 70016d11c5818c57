"""Benchmark: forward + gradient samples/s of the fused path on one GB300.

Workload (default, ``hea20``): the large configuration of the paper's
checkpointing experiment (Sec. 4.3, Table 1) with this build's ansatz:
hardware-efficient ansatz, 20 qubits, 1,000 layers of [RZ, RY, RZ on every
qubit + CZ chain] (60,000 parameters), RY(x) encoding, L = sum_b <Z_0>_b,
1,000 samples trained in micro-batches, the checkpoint interval chosen from
free device memory. One step = forward expectations + loss + adjoint gradients
reduced per parameter (qf_train_step) over ONE micro-batch; the timed steps
walk through the micro-batches of the epoch, inputs resident in HBM. Synthetic
seeded inputs (theta ~ U[0, 2pi), x ~ U[0, pi]^20). ``--workload hea12`` (and
the others) time the smaller configurations.

Printed JSON line (rank 0): value = samples/s of the whole job, plus the
unfused one-kernel-per-gate comparator on the same GPU, the roofline of the
dominant kernel (fused adjoint pass), an end-to-end number through the
host-buffer C-ABI call, the oracle's CPU throughput, the max-abs error of
every timed path against the float64 oracle, and sampled SM clocks.

``--impl reference`` times the float64 CPU oracle instead (the reference
arm): each step is the oracle's training step on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_02804_gb300 import workloads  # noqa: E402
from paper_2603_02804_gb300.record_traffic import TABLE as TRAFFIC_FILE, sources_sha  # noqa: E402

WORKLOAD = "hea20"
FP32_LANES_PER_SM = 128
# GB300's dense FP64 rate (the complex128 path's denominator), TFLOP/s nominal
FP64_TFLOPS_NOMINAL = 1.25
PARITY_TOL = 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(workloads.WORKLOADS) + ["mixed512", "paper_hea", "fusion_sweep"])
    ap.add_argument("--qubits", type=int, default=29, help="paper_hea: number of qubits")
    ap.add_argument("--circuits", type=int, default=0, help="mixed512: first N circuits only (profiling cases)")
    ap.add_argument("--no-autotune", action="store_true", help="mixed512: 12-qubit tiles for every circuit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true")
    ap.add_argument("--no-error-check", action="store_true", help="skip the oracle error of the timed paths")
    ap.add_argument("--batch", type=int, default=0, help="override the workload's batch (profiling cases)")
    ap.add_argument("--depth", type=int, default=0, help="override the workload's depth (profiling cases)")
    ap.add_argument("--micro-batch", type=int, default=0, help="hea20: samples per step (default 100)")
    ap.add_argument("--ckpt", type=int, default=0, help="hea20: checkpoint interval (default: from memory)")
    ap.add_argument("--pergate-samples", type=int, default=32, help="hea20: samples of the per-gate comparator step")
    ap.add_argument("--tile-bits", type=int, default=0, help="plan option tile_bits (0: library default)")
    ap.add_argument("--catch-up", type=int, default=0, choices=[0, 1, 2], help="plan option catch_up")
    ap.add_argument("--fwd-ctas", type=int, default=0, choices=[0, 2, 3], help="plan option fwd_ctas")
    ap.add_argument("--autotune", action="store_true",
                    help="hea20: choose tile width, catch-up rule and forward instance with the autotuner first")
    ap.add_argument("--tc", action="store_true", help="forward rounds on the tensor cores (3xTF32)")
    ap.add_argument("--ckpt-mode", type=int, default=0, choices=[0, 1])
    ap.add_argument("--mem-save", action="store_true", help="checkpoint mode 1 with bfloat16 pass outputs")
    ap.add_argument("--no-variants", action="store_true", help="skip the tensor-core / mode-1 variant timings")
    ap.add_argument("--precision", default="complex64", choices=["complex64", "complex128"],
                    help="state precision of the timed step (complex128: float64 inputs and arithmetic)")
    return ap.parse_args()


def override(w, args):
    """A smaller case of the same workload for profiling (batch / depth)."""
    import dataclasses
    kw = {}
    if args.batch:
        kw["B"] = args.batch
        extra = dict(w.extra)
        extra["micro_batch"] = min(int(extra.get("micro_batch", args.batch)), args.batch)
        kw["extra"] = extra
    if args.depth:
        kw["d"] = args.depth
    return dataclasses.replace(w, **kw) if kw else w


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(peaks):
    """FP32 FMA peak of this GPU: SMs (queried) x 128 lanes x 2 flops x the
    maximum SM clock (from the measured peaks file)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz"


def algorithmic_flops(n, d, B):
    """Arithmetic per step in flops (a multiply or an add = 1, FMA = 2) of the
    round programs, per qubit and layer and per pair of amplitudes.
    Forward: the RY as three shears on (re, im) = 6 FMA = 12 flops, plus a
    quarter of the round's merged diagonal (one complex multiply, 6 flops, per
    amplitude for the 4 RZ runs of a round) = 3 flops; 15 in all.
    Adjoint: the RY un-applied from psi and lambda (12 FMA) and its
    Im<lambda|Y|psi> (4 FMA) = 32 flops, plus a quarter of the diagonal's
    share (two complex multiplies and Im(conj(lambda) psi) per amplitude,
    15 flops, and the signed sums) = 8 flops; 40 in all. Counting each gate
    separately, as a per-gate program must, gives 36 and 96."""
    pairs = B * (1 << (n - 1))
    return n * d * pairs * 15, n * d * pairs * 40


def per_gate_model_flops(n, d, B):
    """The per-gate work model: 6 flops per amplitude per rotation forward,
    16 per amplitude per rotation in the adjoint (un-apply psi 6, un-apply
    lambda 6, Im<lambda|P|psi> about 4), 3 rotations per qubit and layer."""
    amps = B * (1 << n)
    return 3 * n * d * amps * 6, 3 * n * d * amps * 16


def adjoint_bytes_per_amp(handle):
    """Algorithmic HBM bytes per amplitude of the plan's adjoint passes, from
    the exported program: psi and lambda read where a pass loads them (a seed
    pass makes lambda from psi), psi and lambda written where a later pass
    needs them, and 8 bytes per re-anchor from a stored state in the middle of
    a pass. Returns (mean per launch, launches)."""
    from paper_2603_02804_gb300 import qfuse
    w = [int(v) for v in qfuse.qf_plan_export(handle, 1)]
    n_pass = w[2]
    i = 3
    heads = []
    for _ in range(n_pass):
        heads.append(w[i:i + 11])
        i += 11 + 32
    n_ops = w[i]
    codes = [w[i + 1 + 2 * k] & 15 for k in range(n_ops)]
    BUF_NONE, LAM_SEED = -3, -1
    total = 0
    for op_begin, op_end, psi_src, psi_dst, lam_src, lam_dst, *_ in heads:
        b = 8                                   # psi in
        b += 8 if lam_src != LAM_SEED else 0    # lambda in
        b += 8 if psi_dst != BUF_NONE else 0    # psi out
        b += 8 if lam_dst != BUF_NONE else 0    # lambda out
        b += 8 * sum(1 for c in codes[op_begin:op_end] if c == 7)  # re-anchors
        total += b
    return total / max(n_pass, 1), n_pass


def measured_traffic(key, amps):
    """DRAM bytes (read + write) per launch of the dominant kernel, scaled to
    `amps` amplitudes per launch from an ncu capture of the current sources;
    (None, reason) when no capture of these sources exists."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no ncu capture recorded"
    with open(TRAFFIC_FILE) as f:
        tab = json.load(f)
    e = tab.get(key)
    if e is None:
        return None, f"no ncu capture recorded for {key}"
    if e.get("sources_sha") != sources_sha():
        return None, "kernel sources changed since the ncu capture"
    return e["bytes_per_amp"] * amps, e["case"]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- the oracle (CPU)
def _oracle_step(orc, c, w, theta, x, y, threads, B_total):
    """The oracle's training step on samples x (of a batch of B_total)."""
    th = theta.astype(np.float64)
    xx = x.astype(np.float64)
    if w.loss == "mse":
        E = orc.expectation(c, th, xx, w.obs, threads=threads)
        dLdE = orc.mse_dLdE(E, y) * len(E) / B_total
    else:
        dLdE = np.ones(len(xx))
    return orc.gradient(c, th, xx, w.obs, dLdE=dLdE, threads=threads)


def _oracle_sample(w, theta, x, threads, target_s):
    """Size a bounded sample of the workload for the oracle: whole samples when
    one takes well under target_s, else one sample over the first d' of the d
    layers (the oracle's cost is linear in the gate count, so one such step
    counts as d'/d of a sample). Returns (circuit, d', samples per step)."""
    from oracle import oracle as orc
    d_cal = min(w.d, 2)
    t0 = time.perf_counter()
    _oracle_step(orc, orc.hea(w.n, d_cal), w, theta[:3 * w.n * d_cal], x[:1], None if w.loss != "mse" else
                 np.ones(1, np.float32), threads, w.B)
    per_layer = (time.perf_counter() - t0) / d_cal
    if per_layer * w.d <= target_s:
        d_s = w.d
        par = max(1, threads) if w.B >= threads else 1
        B_s = int(max(1, min(w.B, par * max(1, int(target_s / max(per_layer * w.d, 1e-6))))))
    else:
        d_s = int(max(1, min(w.d, target_s / max(per_layer, 1e-9))))
        B_s = 1
    return orc.hea(w.n, d_s), d_s, B_s


def _timed_oracle_step(orc, w, theta, x, y, threads, target_s):
    """(samples/s, description, seconds) of the oracle's step on a bounded
    sample of the workload sized to about target_s on `threads` threads."""
    c, d_s, B_s = _oracle_sample(w, theta, x, threads, target_s)
    t0 = time.perf_counter()
    _oracle_step(orc, c, w, theta[:3 * w.n * d_s], x[:B_s], None if y is None else y[:B_s], threads, w.B)
    dt = time.perf_counter() - t0
    units = B_s * d_s / w.d
    what = (f"{B_s} of the {w.B} samples" if d_s == w.d else
            f"1 sample over the first {d_s} of the {w.d} layers (counted as {d_s}/{w.d} of a sample; the oracle's "
            f"time is linear in the gate count)")
    what = (f"{what} of the {w.name} workload (n={w.n}, d={w.d}), float64"
            + (f", OpenMP over {'samples' if B_s >= threads else 'amplitudes'}" if threads > 1 else ", one thread"))
    return units / dt, what, dt


def cpu_baseline(w, target_s=20.0, threads=0):
    """The float64 oracle's training step (forward, loss, adjoint gradient) on
    the host cores, over a bounded sample of the workload (about target_s),
    and on one core over a smaller sample (about target_s / 4)."""
    from oracle import oracle as orc
    orc.build()
    theta, x, y = workloads.make_inputs(w)
    threads = threads or orc.max_threads()
    value, what, dt = _timed_oracle_step(orc, w, theta, x, y, threads, target_s)
    out = {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle", "sample": what, "seconds": dt}
    if threads > 1:
        v1, what1, dt1 = _timed_oracle_step(orc, w, theta, x, y, 1, target_s / 4)
        out["single_thread"] = {"value": v1, "unit": "samples/s", "sample": what1, "seconds": dt1,
                                "speedup_on_cores": value / v1}
    return out


def cpu_baseline_spawned(w, threads):
    """cpu_baseline in a spawned process: a process holding a CUDA context and
    torch's threads slows the oracle's OpenMP threads down, so the oracle is
    timed in a clean process, on `threads` of the host cores."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        return pool.apply(cpu_baseline, (w, 20.0, threads))


def _oracle_error_worker(n, d, theta, x0, obs, threads, q):
    """(spawned process) E and dE/dtheta of one sample, full depth."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    t0 = time.perf_counter()
    g, E = orc.gradient(orc.hea(n, d), theta.astype(np.float64), x0.astype(np.float64)[None, :], obs,
                        per_sample=True, threads=threads)
    q.put((float(E[0]), g[0], time.perf_counter() - t0))


class OracleJob:
    """The oracle's E and per-sample gradient of one sample at the benchmark's
    full size, computed in a spawned process on the host cores while the GPU
    legs run (the GPU work is launched asynchronously from one thread)."""

    def __init__(self, w, theta, x0, threads):
        from oracle import oracle as orc
        orc.build()
        ctx = mp.get_context("spawn")
        self.q = ctx.Queue()
        self.p = ctx.Process(target=_oracle_error_worker, args=(w.n, w.d, theta, x0, w.obs, threads, self.q),
                             daemon=True)
        self.p.start()
        self.res = None
        self.threads = threads

    def result(self, timeout):
        if self.res is None:
            try:
                self.res = self.q.get(timeout=timeout)
            except Exception:
                self.res = False
            self.p.join(timeout=5)
            if self.p.is_alive():
                self.p.terminate()
        return self.res or None


def gpu_sample_grad(sim, theta, x0):
    """E and dE/dtheta of one sample through the path's forward and backward."""
    import torch
    E = sim.forward(theta, x0)
    g = sim.backward(theta, x0, torch.ones(1, dtype=torch.float64), per_sample=True)
    torch.cuda.synchronize()
    return float(E.cpu()[0]), g.cpu().numpy()[0]


def error_entry(ref, got, what):
    if ref is None or got is None:
        return None
    e_err = abs(got[0] - ref[0])
    g_err = float(np.max(np.abs(got[1] - ref[1])))
    return {"E": e_err, "grad": g_err, "within_1e-5": bool(e_err <= PARITY_TOL and g_err <= PARITY_TOL),
            "sample": what}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    orc.build()
    theta, x, y = workloads.make_inputs(w)
    threads = orc.max_threads()
    # each step: a bounded sample sized so that the whole run stays within minutes
    target = min(10.0, 150.0 / max(args.steps + args.warmup, 1))
    c, d_s, B_s = _oracle_sample(w, theta, x, threads, target)
    th = theta[:3 * w.n * d_s]
    for _ in range(args.warmup):
        _oracle_step(orc, c, w, th, x[:B_s], None if y is None else y[:B_s], threads, w.B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(orc, c, w, th, x[:B_s], None if y is None else y[:B_s], threads, w.B)
    dt = time.perf_counter() - t0
    units = B_s * d_s / w.d
    value = units * args.steps / dt
    what = (f"{B_s} samples of the {w.name} batch per step" if d_s == w.d else
            f"1 sample over the first {d_s} of the {w.d} layers per step, counted as {d_s}/{w.d} of a sample "
            f"(the oracle's time is linear in the gate count)")
    line = {
        "impl": "reference", "metric": "fwd+grad samples/s", "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": f"{w.name}: HEA n={w.n} d={w.d} [RZ,RY,RZ + CZ chain], RY(x) encoding, "
                               f"loss={w.loss}, obs=Z0", "sample_per_step": what},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle", "sample": what},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- large workload
def run_large(args, w):
    """n=20, d=1000, 1000 samples: one step = one micro-batch of mb samples
    (qf_train_step), the checkpoint interval chosen from free memory."""
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2603_02804_gb300 import build as qbuild
    if rank == 0:
        qbuild.build()
    if world > 1:
        dist.barrier()
    from paper_2603_02804_gb300 import dp, qfuse
    from paper_2603_02804_gb300.torch_api import Simulator

    if args.warmup < 3:
        args.warmup = 3
    peaks, peak_src = load_peaks()
    theta_np, x_np, _ = workloads.make_inputs(w)
    if rank > 0:  # weak scaling: every rank trains its own samples
        x_np = workloads.draw_x(w.B, w.n, w.seeds[1] + 1000 * rank)
    N = w.B
    mb = min(args.micro_batch or int(w.extra.get("micro_batch", 100)), N)
    n_mb = (N + mb - 1) // mb
    solo = rank == 0 and world == 1
    ncores = os.cpu_count() or 1
    job = None
    if solo and not args.no_error_check:
        job = OracleJob(w, theta_np, x_np[0], max(1, ncores - 4))

    tuned = None
    tune_s = 0.0
    knobs = dict(tile_bits=args.tile_bits, catch_up=args.catch_up, fwd_ctas=args.fwd_ctas)
    if args.autotune:
        from paper_2603_02804_gb300.autotune import Autotuner
        t_start = time.perf_counter()
        tuner = Autotuner(path=os.environ.get("QF_AUTOTUNE_CACHE"))
        knobs = tuner.choose(w.n, w.d, mb)
        tune_s = time.perf_counter() - t_start
        tuned = {"choice": knobs, "timed_shape": list(tuner.shape(w.n, w.d, mb)), "seconds": tune_s,
                 "timings_ms": next(iter(tuner.timings.values()), None)}
        torch.cuda.empty_cache()
    opts = dict(ckpt_mode=args.ckpt_mode, mem_save=args.mem_save, tc_path=args.tc, **knobs)
    free, _ = torch.cuda.mem_get_info()
    h = qfuse.qf_hea_create(w.n, w.d)
    if args.ckpt:
        c = args.ckpt
    else:
        c, _ = qfuse.qf_plan_fit(h, mb, int(0.8 * free), host_only=True, **opts)
    qfuse.qf_circuit_destroy(h)
    sim = Simulator(w.n, w.d, mb, ckpt_layers=c, obs=w.obs, **opts)
    dev = torch.device("cuda", local)
    theta = torch.from_numpy(theta_np).to(dev)
    xs = [torch.from_numpy(np.ascontiguousarray(x_np[i:i + mb])).to(dev) for i in range(0, N, mb)]
    out = sim.device_outputs()
    stream = torch.cuda.current_stream(dev)

    def step(s, k, o):
        _, _, g = s.train_step(theta, xs[k % len(xs)], loss=w.loss, out=o)
        if world > 1:
            dp.allreduce_sum(g)  # data-parallel gradient sum over ranks (NCCL)

    for k in range(args.warmup):
        step(sim, k, out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        t0.record(stream)
        for k in range(args.steps):
            step(sim, k, out)
            launches += sim.launches()
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t = torch.tensor([t0.elapsed_time(t1)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms = total_ms / args.steps
    timed_samples = sum(xs[k % len(xs)].shape[0] for k in range(args.steps))
    value = timed_samples * world / (total_ms / 1e3)

    # ---- pass-kernel timings (CUDA events around every pass launch) of 2 more steps
    K_p = 2
    qfuse.qf_profile(sim.handle, True)
    qfuse.qf_profile_read(sim.handle)
    for k in range(K_p):
        step(sim, k, out)
    prof = qfuse.qf_profile_read(sim.handle)
    qfuse.qf_profile(sim.handle, False)
    info = sim.info()
    passes = info["n_passes"]
    bwd_launch_ms = prof["bwd_ms"] / max(prof["bwd_launches"], 1)
    fwd_launch_ms = prof["fwd_ms"] / max(prof["fwd_launches"], 1)
    fwd_fl, bwd_fl = algorithmic_flops(w.n, w.d, mb)
    pg_fwd, pg_bwd = per_gate_model_flops(w.n, w.d, mb)
    fp32_peak, peak_what = fp32_peak_tflops(peaks)
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    amps = mb * (1 << w.n)
    # algorithmic bytes of one adjoint launch, averaged over the plan's passes
    bpa, _ = adjoint_bytes_per_amp(sim.handle)
    bwd_bytes = amps * bpa
    achieved = bwd_fl / passes / (bwd_launch_ms / 1e3) / 1e12
    traffic, traffic_note = measured_traffic(w.name, amps) if not (args.tc or args.ckpt_mode) else (None, "variant")
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
        "traffic": traffic, "traffic_note": traffic_note,
        "kernel": "pass_kernel<true> (fused adjoint pass)", "peak_source": f"{peak_what} (derived: FP32 FMA peak)",
        "bwd_kernel_ms": bwd_launch_ms, "fwd_kernel_ms": fwd_launch_ms,
        "flops_model": "executed arithmetic of the round programs: 15 (forward) and 40 (adjoint) flops per "
                       "amplitude pair, qubit and layer",
        "per_gate_flops_model": {"achieved": pg_bwd / passes / (bwd_launch_ms / 1e3) / 1e12,
                                 "frac": pg_bwd / passes / (bwd_launch_ms / 1e3) / 1e12 / fp32_peak,
                                 "note": "16 flops per amplitude per rotation (6 + 6 un-apply, 4 gradient), "
                                         "as a per-gate program counts them"},
        "hbm": {"achieved_gbs": bwd_bytes / (bwd_launch_ms / 1e3) / 1e9, "peak_gbs": hbm_gbs,
                "frac": bwd_bytes / (bwd_launch_ms / 1e3) / 1e9 / hbm_gbs, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": bwd_bytes, "algorithmic_bytes_per_amp": bpa},
        "fwd_kernel": {"achieved": fwd_fl / passes / (fwd_launch_ms / 1e3) / 1e12,
                       "hbm_gbs": amps * 16 / (fwd_launch_ms / 1e3) / 1e9},
        "timing": f"CUDA events on the launching stream around every pass launch of {K_p} steps run after the "
                  f"timed ones ({prof['bwd_launches']} adjoint and {prof['fwd_launches']} forward launches)",
    }

    # ---- end to end through the host-buffer call (pinned host memory)
    K_e = max(1, min(args.steps, 3))
    th_h = torch.from_numpy(theta_np).pin_memory()
    xs_h = [torch.from_numpy(np.ascontiguousarray(x_np[i:i + mb])).pin_memory() for i in range(0, N, mb)]
    outs_h = sim.host_outputs()
    sim.train_step_host(th_h, xs_h[0], loss=w.loss, out=outs_h)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(K_e):
        sim.train_step_host(th_h, xs_h[k % len(xs_h)], loss=w.loss, out=outs_h)
    e_dt = time.perf_counter() - e0
    e2e = {"value": mb * world * K_e / e_dt, "unit": "samples/s", "steps": K_e,
           "h2d_bytes_per_step": theta_np.nbytes + xs_h[0].numel() * 4,
           "d2h_bytes_per_step": 8 + 8 * mb + 8 * w.n_params}

    # ---- error of each timed path against the oracle (sample 0, full depth)
    x0 = xs[0][:1].contiguous()
    got = {"fused": gpu_sample_grad(sim, theta, x0)} if job else {}
    ws_gb = sim.ws_bytes / 1e9
    del sim, out
    torch.cuda.empty_cache()

    # ---- unfused per-gate comparator on a subset of samples
    per_gate = None
    if not args.no_per_gate and solo:
        B_pg = min(args.pergate_samples, mb)
        warm = Simulator(w.n, 2, B_pg, path="per_gate", obs=w.obs)
        warm.train_step(theta[:3 * w.n * 2], xs[0][:B_pg], loss=w.loss)
        del warm
        pg = Simulator(w.n, w.d, B_pg, path="per_gate", obs=w.obs)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pg.train_step(theta, xs[0][:B_pg], loss=w.loss)
        p1.record(stream)
        pg_launches = pg.launches()
        torch.cuda.synchronize()
        pg_ms = p0.elapsed_time(p1)
        per_gate = {"value": B_pg / (pg_ms / 1e3), "unit": "samples/s", "ms_per_step": pg_ms,
                    "gpu_launches_per_step": pg_launches,
                    "sample": f"1 step of {B_pg} samples (state {B_pg * 8 * (1 << w.n) / 1e6:.0f} MB, larger than L2), "
                              f"full depth"}
        if job:
            got["per_gate"] = gpu_sample_grad(pg, theta, x0)
        del pg
        torch.cuda.empty_cache()

    # ---- variants: tensor-core forward, checkpoint mode 1, bfloat16 storage
    variants = None
    if not args.no_variants and solo:
        variants = {}
        for name, kw in (("tc_path", dict(tc_path=True)), ("ckpt_mode_1", dict(ckpt_mode=1)),
                         ("ckpt_mode_1_mem_save", dict(ckpt_mode=1, mem_save=True))):
            if all(opts.get(k) == v for k, v in kw.items()):
                continue
            free, _ = torch.cuda.mem_get_info()
            h = qfuse.qf_hea_create(w.n, w.d)
            cv, _ = qfuse.qf_plan_fit(h, mb, int(0.8 * free), host_only=True, **kw, **knobs)
            qfuse.qf_circuit_destroy(h)
            vs = Simulator(w.n, w.d, mb, ckpt_layers=cv, obs=w.obs, **kw, **knobs)
            vo = vs.device_outputs()
            step(vs, 0, vo)
            torch.cuda.synchronize()
            K_v = 2
            qfuse.qf_profile(vs.handle, True)
            qfuse.qf_profile_read(vs.handle)
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for k in range(K_v):
                step(vs, k + 1, vo)
            v1.record(stream)
            torch.cuda.synchronize()
            vp = qfuse.qf_profile_read(vs.handle)
            v_ms = v0.elapsed_time(v1) / K_v
            variants[name] = {"value": mb / (v_ms / 1e3), "unit": "samples/s", "ms_per_step": v_ms,
                              "ckpt_layers": cv, "workspace_gb": vs.ws_bytes / 1e9,
                              "fwd_ms_per_step": vp["fwd_ms"] / K_v, "bwd_ms_per_step": vp["bwd_ms"] / K_v,
                              "device_status": qfuse.qf_device_status(stream)}
            if job:
                got[name] = gpu_sample_grad(vs, theta, x0)
            del vs, vo
            torch.cuda.empty_cache()

    cpu = None
    ref = None
    if job:
        r = job.result(timeout=600)
        if r:
            ref = (r[0], r[1])
    errors = None
    if job:
        what = f"sample 0 of micro-batch 0, E and dE/dtheta (all {w.n_params}) vs the float64 oracle, full depth"
        errors = {k: error_entry(ref, v, what) for k, v in got.items()}
        if ref is None:
            errors["note"] = "oracle did not finish in time"
        else:
            errors["oracle_seconds"] = r[2]
            errors["oracle_threads"] = job.threads
        if variants:
            for k in variants:
                variants[k]["error"] = errors.get(k)
        if per_gate:
            per_gate["error"] = errors.get("per_gate")
    if solo and not args.no_cpu_baseline:
        cpu = cpu_baseline_spawned(w, max(1, ncores - 2))

    if rank == 0:
        line = {
            "metric": "fwd+grad samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded): theta~U[0,2pi), x~U[0,pi]^n",
            "config": {"workload": f"{w.name}: HEA n={w.n} d={w.d} [RZ,RY,RZ + CZ chain] ({w.n_params} params), "
                                   f"RY(x) encoding, L=sum E, obs=Z0, complex64; {N} samples/GPU per epoch in "
                                   f"micro-batches of {mb}, one step = one micro-batch; checkpoint mode "
                                   f"{'A (re-run)' if args.ckpt_mode else 'B (reverse + re-anchor)'}, "
                                   f"interval c={c} layers from memory",
                       "micro_batch": mb, "micro_batches_per_epoch": n_mb, "ckpt_layers": c,
                       "ckpt_mode": args.ckpt_mode, "mem_save": bool(args.mem_save), "tc_path": bool(args.tc),
                       "passes_per_direction": passes, "tile_bits": info["tile_bits"], "workspace_gb": ws_gb,
                       "catch_up": info["catch_up"], "fwd_ctas": info["fwd_ctas"], "autotune": tuned,
                       "parallelism": f"dp{world}",
                       "l2": f"inputs larger than L2 (state of a micro-batch {amps * 8 / 1e6:.0f} MB)",
                       "fwd_ms_per_step": prof["fwd_ms"] / K_p, "bwd_ms_per_step": prof["bwd_ms"] / K_p},
            "error_vs_oracle": errors,
            "per_gate": per_gate,
            "speedup_vs_per_gate": (value / per_gate["value"]) if per_gate else None,
            "variants": variants,
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "peaks": {"source": peak_src, "hbm_gbs": hbm_gbs},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_mixed(args):
    """512 uneven circuits (n 8..18, d 10..200, B 1..64) trained by one
    persistent launch per step; eager steps and CUDA-graph replays timed."""
    import torch
    from paper_2603_02804_gb300 import build as qbuild
    from paper_2603_02804_gb300.autotune import Autotuner
    from paper_2603_02804_gb300.torch_api import Batch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    peaks, peak_src = load_peaks()
    circs = workloads.mixed_circuits(512, seed=104 + 1000 * rank)
    if args.circuits:
        circs = circs[:args.circuits]  # a subset of the same draw (profiling cases)
    specs = [(c.n, c.d, c.B) for c in circs]
    tuner = Autotuner(path=os.environ.get("QF_AUTOTUNE_CACHE"), kind="batch")  # JSON cache file, or in memory
    t0 = time.perf_counter()
    bt = Batch(specs, loss="sum", tile_bits=None if args.no_autotune else tuner)
    tune_s = time.perf_counter() - t0
    cat = lambda arrs: torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrs])).cuda()
    theta, x = cat([c.theta for c in circs]), cat([c.x for c in circs])
    out = bt.outputs()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.train_step(theta, x, out=out)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            starts[k].record(stream)
            bt.train_step(theta, x, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    gs = torch.cuda.Stream()
    with torch.cuda.stream(gs):
        bt.capture(theta, x, None, out, gs)
    gs.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(gs)
    for _ in range(args.steps):
        bt.replay()
    g1.record(gs)
    gs.synchronize()
    graph_ms = g0.elapsed_time(g1)
    # end to end from pinned host buffers
    th_h = theta.cpu().pin_memory()
    x_h = x.cpu().pin_memory()
    res_h = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in out]
    e0 = time.perf_counter()
    for _ in range(max(1, args.steps // 4)):
        theta.copy_(th_h, non_blocking=True)
        x.copy_(x_h, non_blocking=True)
        bt.train_step(theta, x, out=out)
        for h, d in zip(res_h, out):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
    e_dt = (time.perf_counter() - e0) / max(1, args.steps // 4)
    fl = sum(sum(algorithmic_flops(n, d, B)) for n, d, B in specs)
    ms = total_ms / args.steps
    fp32_peak, peak_what = fp32_peak_tflops(peaks)
    achieved = fl / (ms / 1e3) / 1e12
    line = {
        "metric": "fwd+grad samples/s", "value": bt.n_samples * world / (ms / 1e3), "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": "mixed512: 512 HEA circuits n~U{8..18} d~U{10..200} B~U{1..64}, L=sum E, obs=Z0, "
                               "one persistent launch per step", "samples_per_step": bt.n_samples,
                   "work_items": bt.n_items, "tile_bits": "12 (fixed)" if args.no_autotune else "autotuned", "tune_s": tune_s,
                   "l2": "inputs larger than L2 (workspace %.1f GB)" % (bt.ws_bytes / 1e9)},
        "graph": {"value": bt.n_samples * world * args.steps / (graph_ms / 1e3), "unit": "samples/s",
                  "ms_per_step": graph_ms / args.steps},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None, "peak_source": peak_what,
                     "kernel": "batch_kernel (whole step: prep + persistent + reductions)"},
        "e2e": {"value": bt.n_samples * world / e_dt, "unit": "samples/s",
                "h2d_bytes_per_step": theta.numel() * 4 + x.numel() * 4,
                "d2h_bytes_per_step": sum(t.numel() * 8 for t in out)},
        "gpu_launches": 4 * args.steps,
        "per_gate": None, "cpu_baseline": None, "clocks": clk.summary(),
        "autotune": tuner.cache,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


PAPER_SEC42_SAMPLES_PER_S = {29: 3.57}  # fused, GH200, HEA d=1 (Sec. 4.2); other hardware: context only


def run_paper(args):
    """The paper's throughput measurement (Sec. 4.2): HEA with d = 1 layer of Rx, Ry, Rz on every qubit
    and a CZ ring, applied to random normalised initial states, O = IXYZ IXYZ ..., L = sum_b E_b, the
    batch as large as fits in memory; one step = forward + loss + adjoint + gradient reduction."""
    import torch
    from paper_2603_02804_gb300 import build as qbuild
    from paper_2603_02804_gb300 import qfuse
    from paper_2603_02804_gb300.torch_api import Simulator

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    peaks, peak_src = load_peaks()
    n, d = args.qubits, 1
    rows = workloads.xyz_ring_gates(n, d)
    P = 3 * n * d
    obs = workloads.ixyz(n)
    state_bytes = (1 << n) * 8
    h = qfuse.qf_circuit_create(n, rows, P, qfuse.QF_ENC_STATE_IN)
    ws1 = qfuse.qf_plan(h, 1, host_only=True, host_staging=False)
    qfuse.qf_circuit_destroy(h)
    free, _ = torch.cuda.mem_get_info()
    B = args.batch or max(1, int(0.85 * free) // (ws1 + state_bytes))
    sim = Simulator(n, 0, B, gates=rows, n_params=P, obs=obs, encoding="state", host_staging=False)
    theta = torch.from_numpy(workloads.draw_theta(P, 401)).cuda()
    # random normalised states drawn on the device (seeded), one sample at a time
    gen = torch.Generator(device="cuda")
    gen.manual_seed(402 + 1000 * rank)
    psi0 = torch.empty(B, 1 << n, dtype=torch.complex64, device="cuda")
    for b in range(B):
        re = torch.randn(1 << n, generator=gen, device="cuda")
        im = torch.randn(1 << n, generator=gen, device="cuda")
        z = torch.complex(re, im)
        psi0[b] = z / torch.linalg.vector_norm(z)
        del re, im, z
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        sim.train_step(theta, psi0, loss="sum")
    torch.cuda.synchronize()
    qfuse.qf_profile(sim.handle, True)
    qfuse.qf_profile_read(sim.handle)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            sim.train_step(theta, psi0, loss="sum")
            launches += sim.launches()
        t1.record(stream)
        torch.cuda.synchronize()
    prof = qfuse.qf_profile_read(sim.handle)
    status = qfuse.qf_device_status(stream)
    ms = t0.elapsed_time(t1) / args.steps
    info = sim.info()
    nf = nb = info["n_passes"]
    amps = B * (1 << n)
    # algorithmic bytes: forward passes 16 B/amp (read + write psi), E 8 B/amp (psi_M once), seed 16 B/amp,
    # adjoint passes 32 B/amp (psi and lambda read + write) but the last reads only
    step_bytes = amps * (16 * nf + 8 + 16 + 32 * nb - 16)
    bwd_bytes = amps * (16 + 32 * (nb - 1) + 16)
    bwd_ms = prof["bwd_ms"] / args.steps
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    value = B * world / (ms / 1e3)
    ref = PAPER_SEC42_SAMPLES_PER_S.get(n)
    line = {
        "metric": "fwd+grad samples/s", "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / ref) if ref else None, "dtype": "f32",
        "data": "synthetic: random normalised complex Gaussian states (seeded, drawn on the device), "
                "theta~U[0,2pi)",
        "config": {"workload": f"paper_hea: n={n} d=1 [Rx,Ry,Rz + CZ ring], random initial states, "
                               f"O=IXYZ..., L=sum E, batch={B} (largest that fits)",
                   "passes_per_direction": nf, "workspace_gb": sim.ws_bytes / 1e9,
                   "baseline_note": "vs_baseline divides by the paper's GH200 number for this workload (Sec. 4.2)"
                   if ref else None, "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": bwd_bytes / (bwd_ms / 1e3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                     "frac": bwd_bytes / (bwd_ms / 1e3) / 1e9 / hbm_gbs, "traffic": None,
                     "kernel": "adjoint phase (seed + adjoint pass kernels)", "peak_source": peak_src,
                     "step": {"algorithmic_bytes": step_bytes, "achieved_gbs": step_bytes / (ms / 1e3) / 1e9,
                              "frac": step_bytes / (ms / 1e3) / 1e9 / hbm_gbs},
                     "fwd_ms_per_step": prof["fwd_ms"] / args.steps, "bwd_ms_per_step": bwd_ms},
        "gpu_launches": launches, "device_status": status, "per_gate": None, "cpu_baseline": None, "e2e": None,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_fusion_sweep(args):
    """Sec. 4.1: time of m consecutive single-qubit gates (Rx, Ry, Rz repeating) on every qubit of a
    20-qubit state, batch 100, random initial states, forward alone and forward + adjoint, as m grows."""
    import torch
    from paper_2603_02804_gb300 import build as qbuild
    from paper_2603_02804_gb300.torch_api import Simulator

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    n, B = 20, args.batch or 100
    obs = workloads.ixyz(n)
    psi0 = torch.from_numpy(workloads.draw_state(B, n, 4101)).cuda()
    stream = torch.cuda.current_stream()
    rows_out = []
    for m in (1, 3, 6, 9, 18, 36, 72):
        rows = workloads.consecutive_gates(n, m)
        P = n * m
        sim = Simulator(n, 0, B, gates=rows, n_params=P, obs=obs, encoding="state", host_staging=False)
        theta = torch.from_numpy(workloads.draw_theta(P, 4100 + m)).cuda()
        for _ in range(3):
            sim.train_step(theta, psi0, loss="sum")
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        K = args.steps
        ev[0].record(stream)
        for _ in range(K):
            sim.forward(theta, psi0)
        ev[1].record(stream)
        for _ in range(K):
            sim.train_step(theta, psi0, loss="sum")
        ev[2].record(stream)
        torch.cuda.synchronize()
        fwd = ev[0].elapsed_time(ev[1]) / K
        step = ev[1].elapsed_time(ev[2]) / K
        info = sim.info()
        rows_out.append({"m": m, "gates": n * m, "passes": info["n_passes"], "fwd_ms": fwd, "fwd_bwd_ms": step,
                         "bwd_ms": step - fwd, "fwd_us_per_gate": 1e3 * fwd / (n * m),
                         "fwd_bwd_us_per_gate": 1e3 * step / (n * m), "samples_per_s": B / (step / 1e3),
                         "workspace_gb": sim.ws_bytes / 1e9})
        del sim
    last = rows_out[-1]
    line = {"metric": "fwd+grad samples/s", "value": last["samples_per_s"], "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": 3, "ms_per_step": last["fwd_bwd_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: random normalised complex Gaussian states, theta~U[0,2pi)",
            "config": {"workload": f"fusion_sweep: n={n}, batch={B}, m consecutive Rx,Ry,Rz gates per qubit, "
                                   "O=IXYZ..., L=sum E (value at the largest m)", "l2": "inputs larger than L2"},
            "sweep": rows_out, "roofline": None, "gpu_launches": None, "cpu_baseline": None, "e2e": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- small workloads
def run_small(args, w):
    """Workloads whose batch is one step (hea12, hea16, tiny): qf_train_step
    on the whole batch, L2 flushed between the timed steps."""
    if args.warmup < 3:
        args.warmup = 3

    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2603_02804_gb300 import build as qbuild
    if rank == 0:
        qbuild.build()
    if world > 1:
        dist.barrier()
    from paper_2603_02804_gb300 import qfuse
    from paper_2603_02804_gb300.torch_api import Simulator

    peaks, peak_src = load_peaks()
    theta_np, x_np, y_np = workloads.make_inputs(w)
    # weak scaling: every rank processes its own batch of w.B samples
    if rank > 0:
        x_np = workloads.draw_x(w.B, w.n, w.seeds[1] + 1000 * rank)
    dev = torch.device("cuda", local)
    c128 = args.precision == "complex128"
    if c128:  # float64 inputs (the float32 draws, promoted exactly)
        theta_np, x_np = theta_np.astype(np.float64), x_np.astype(np.float64)
        y_np = None if y_np is None else y_np.astype(np.float64)
    theta = torch.from_numpy(theta_np).to(dev)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.from_numpy(y_np).to(dev) if y_np is not None else None
    ckpt = w.ckpt_layers or 0
    opts = dict(ckpt_mode=args.ckpt_mode, mem_save=args.mem_save, tc_path=args.tc, tile_bits=args.tile_bits,
                catch_up=args.catch_up, fwd_ctas=args.fwd_ctas)
    if c128:
        opts["precision"] = "complex128"
    sim = Simulator(w.n, w.d, w.B, ckpt_layers=ckpt, obs=w.obs, **opts)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    from paper_2603_02804_gb300 import dp

    # the oracle's per-sample E and dE/dtheta of every sample (float64)
    ref = None
    solo = rank == 0 and world == 1
    if solo and not args.no_error_check:
        from oracle import oracle as orc
        orc.build()
        t32, x32, _ = workloads.make_inputs(w)
        g_r, E_r = orc.gradient(orc.hea(w.n, w.d), t32.astype(np.float64), x32.astype(np.float64), w.obs,
                                per_sample=True)
        ref = (E_r, g_r)

    def path_error(s, inp=None):
        """Max-abs error of E and of every per-sample gradient dE_b/dtheta
        against the oracle, over the whole batch."""
        if ref is None:
            return None
        th_, x_ = (inp[0], inp[1]) if inp is not None else (theta, x)
        E = s.forward(th_, x_)
        g = s.backward(th_, x_, torch.ones(x_.shape[0], dtype=torch.float64), per_sample=True)
        torch.cuda.synchronize()
        e_err = float(np.max(np.abs(E.cpu().numpy() - ref[0])))
        g_err = float(np.max(np.abs(g.cpu().numpy() - ref[1])))
        return {"E": e_err, "grad": g_err, "within_1e-5": bool(e_err <= PARITY_TOL and g_err <= PARITY_TOL),
                "sample": f"all {x_.shape[0]} samples, E and per-sample dE/dtheta vs the float64 oracle"}

    def step(s, inp=None):
        th_, x_, y_ = inp if inp is not None else (theta, x, y)
        if not hasattr(s, "bench_out"):
            s.bench_out = s.device_outputs()  # the same buffers every step
        loss, E, g = s.train_step(th_, x_, y_, loss=w.loss, out=s.bench_out)
        if world > 1:
            dp.allreduce_sum(g)  # data-parallel gradient sum over ranks (NCCL)
        return g

    def timed(s, K, inp=None):
        """K steps, each bracketed by CUDA events after an L2 flush."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        launches = 0
        for k in range(K):
            flush.fill_(k & 255)  # evict the state from L2 between timed steps
            starts[k].record(stream)
            step(s, inp)
            ends[k].record(stream)
            launches += s.launches()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends)), launches

    def profiled(s, K, inp=None):
        """Pass-kernel timings: K more steps with CUDA events recorded around
        every pass launch (the library launches such steps one kernel at a
        time instead of replaying its recorded graph)."""
        qfuse.qf_profile(s.handle, True)
        ms, _ = timed(s, K, inp)
        p = qfuse.qf_profile_read(s.handle)
        qfuse.qf_profile(s.handle, False)
        p["ms_per_step"] = ms / K
        return p

    # the warm-up records the step's CUDA graph; the timed steps replay it
    for _ in range(args.warmup):
        step(sim)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    g0 = sim.graph_stats()
    with ClockSampler(local) as clk:
        total_ms, launches = timed(sim, args.steps)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    g1 = sim.graph_stats()
    step_graph = {"replayed_in_timed_steps": g1["replayed"] - g0["replayed"], "recorded": g1["recorded"]}
    prof = profiled(sim, args.steps)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = w.B * world * args.steps / (total_ms / 1e3)
    main_error = path_error(sim) if not c128 else None

    # ---- roofline of the dominant kernel: the fused adjoint pass kernel
    fwd_fl, bwd_fl = algorithmic_flops(w.n, w.d, w.B)
    info = sim.info()
    bwd_launch_ms = prof["bwd_ms"] / max(prof["bwd_launches"], 1)
    fwd_launch_ms = prof["fwd_ms"] / max(prof["fwd_launches"], 1)
    bwd_per_launch = bwd_fl / info["n_passes"]
    fp32_peak, peak_what = fp32_peak_tflops(peaks)
    alu_peak = FP64_TFLOPS_NOMINAL if c128 else fp32_peak
    achieved = bwd_per_launch / (bwd_launch_ms / 1e3) / 1e12
    amps_launch = w.B * (1 << w.n)
    traffic, traffic_note = (measured_traffic(w.name, amps_launch) if not (args.tc or args.ckpt_mode or c128)
                             else (None, "variant"))
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic, "traffic_note": traffic_note,
                "kernel": ("pass64_kernel<true> (fused adjoint, complex128)" if c128
                           else "pass_kernel<true> (fused adjoint)"),
                "peak_source": ("GB300 dense FP64, nominal" if c128 else f"{peak_what} (derived: FP32 FMA peak)"),
                "fwd_kernel": {"achieved": (fwd_fl / info["n_passes"]) / (fwd_launch_ms / 1e3) / 1e12,
                               "ms": fwd_launch_ms},
                "bwd_kernel_ms": bwd_launch_ms,
                "flops_model": "executed arithmetic of the round programs: 15 (forward) and 40 (adjoint) flops "
                               "per amplitude pair, qubit and layer",
                "timing": (f"CUDA events on the launching stream around every pass launch of {args.steps} "
                           f"steps run right after the timed ones (launched kernel by kernel: "
                           f"{prof['ms_per_step']:.4f} ms per step)")}
    state_bytes = w.B * (1 << w.n) * (16 if c128 else 8)
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    hbm = {"algorithmic_bytes_per_step": 4 * state_bytes,
           "achieved_gbs": 4 * state_bytes / (ms_per_step / 1e3) / 1e9,
           "peak_gbs": hbm_gbs, "peak_source": peak_src,
           "frac": 4 * state_bytes / (ms_per_step / 1e3) / 1e9 / hbm_gbs,
           "note": "state of this workload fits in L2; the path is ALU-bound, see roofline"}

    # ---- the same step with the tensor-core forward, with checkpoint mode 1 and
    # in complex128 (float64 inputs, its own FP64 roofline)
    variants = None
    if not args.no_variants and world == 1:
        variants = {}
        inp64 = tuple(None if v is None else v.double() for v in (theta, x, y))
        for name, kw in (("tc_path", dict(tc_path=True)), ("ckpt_mode_1", dict(ckpt_mode=1)),
                         ("ckpt_mode_1_mem_save", dict(ckpt_mode=1, mem_save=True)),
                         ("complex128", dict(precision="complex128"))):
            if all(opts.get(k) == v for k, v in kw.items()):
                continue
            v128 = kw.get("precision") == "complex128"
            inp = inp64 if v128 else None
            try:
                vs = Simulator(w.n, w.d, w.B, ckpt_layers=ckpt, obs=w.obs, **kw)
            except qfuse.QFError as err:
                variants[name] = {"unavailable": str(err)}
                continue
            for _ in range(args.warmup):
                step(vs, inp)
            torch.cuda.synchronize()
            K = min(args.steps, 50 if v128 else 200)
            v_ms, _ = timed(vs, K, inp)
            vp = profiled(vs, K, inp)
            variants[name] = {"value": w.B * K / (v_ms / 1e3), "unit": "samples/s", "ms_per_step": v_ms / K,
                              "fwd_ms_per_step": vp["fwd_ms"] / K, "bwd_ms_per_step": vp["bwd_ms"] / K,
                              "device_status": qfuse.qf_device_status(stream),
                              "error": path_error(vs, inp)}
            if v128:
                vi = vs.info()
                f_fl, b_fl = algorithmic_flops(w.n, w.d, w.B)
                b_ms = vp["bwd_ms"] / max(vp["bwd_launches"], 1)
                f_ms = vp["fwd_ms"] / max(vp["fwd_launches"], 1)
                ach = b_fl / vi["n_passes"] / (b_ms / 1e3) / 1e12
                variants[name]["dtype"] = "f64"
                variants[name]["roofline"] = {
                    "bound": "alu", "kernel": "pass64_kernel<true> (fused adjoint, complex128)",
                    "achieved": ach, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                    "frac": ach / FP64_TFLOPS_NOMINAL, "peak_source": "GB300 dense FP64, nominal",
                    "fwd_kernel": {"achieved": f_fl / vi["n_passes"] / (f_ms / 1e3) / 1e12, "ms": f_ms},
                    "bwd_kernel_ms": b_ms}
            del vs

    # ---- the same step captured once in a CUDA graph and replayed (the C-ABI
    # allocates and synchronises nothing after qf_plan)
    if variants is not None and not c128:
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            step(sim)
        stream.wait_stream(gs)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step(sim)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        K = min(args.steps, 200)
        g_st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        g_en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            flush.fill_(k & 255)
            g_st[k].record(stream)
            graph.replay()
            g_en[k].record(stream)
        torch.cuda.synchronize()
        g_ms = sum(a.elapsed_time(b) for a, b in zip(g_st, g_en))
        variants["cuda_graph"] = {"value": w.B * K / (g_ms / 1e3), "unit": "samples/s", "ms_per_step": g_ms / K,
                                  "note": "qf_train_step captured once with torch.cuda.graph, replayed per step"}
        del graph

    # ---- unfused per-gate comparator on the same GPU (complex64 only)
    per_gate = None
    if not args.no_per_gate and not c128:
        pg = Simulator(w.n, w.d, w.B, path="per_gate", ckpt_layers=ckpt, obs=w.obs)
        for _ in range(args.warmup):
            step(pg)
        torch.cuda.synchronize()
        pg_ms, pg_launches = timed(pg, args.steps)
        per_gate = {"value": w.B * world * args.steps / (pg_ms / 1e3), "unit": "samples/s",
                    "ms_per_step": pg_ms / args.steps, "gpu_launches_per_step": pg_launches // args.steps,
                    "error": path_error(pg)}
        del pg

    # ---- end to end through the host-buffer call (pinned host memory)
    th_h = torch.from_numpy(theta_np).pin_memory()
    x_h = torch.from_numpy(x_np).pin_memory()
    y_h = torch.from_numpy(y_np).pin_memory() if y_np is not None else None
    outs_h = sim.host_outputs()  # pinned once, written by every step
    for _ in range(2):
        sim.train_step_host(th_h, x_h, y_h, loss=w.loss, out=outs_h)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        loss_h, E_h, g_h = sim.train_step_host(th_h, x_h, y_h, loss=w.loss, out=outs_h)
    e_dt = time.perf_counter() - e0
    h2d = theta_np.nbytes + x_np.nbytes + (y_np.nbytes if y_np is not None else 0)
    d2h = 8 + 8 * w.B + 8 * w.n_params
    e2e = {"value": w.B * world * args.steps / e_dt, "unit": "samples/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    cpu = None
    if solo and not args.no_cpu_baseline:
        cpu = cpu_baseline_spawned(w, max(1, (os.cpu_count() or 1) - 2))

    if rank == 0:
        line = {
            "metric": "fwd+grad samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if c128 else "f32",
            "data": "synthetic (seeded): theta~U[0,2pi), x~U[0,pi]^n, y~{-1,+1}",
            "config": {"workload": f"{w.name}: HEA n={w.n} d={w.d} [RZ,RY,RZ + CZ chain], RY(x) encoding, "
                                   f"batch={w.B}/GPU, loss={w.loss}, obs=Z0",
                       "path": "fused", "tile_bits": info["tile_bits"], "passes": info["n_passes"],
                       "tc_path": bool(args.tc), "ckpt_mode": args.ckpt_mode, "mem_save": bool(args.mem_save),
                       "precision": args.precision,
                       "ckpt_layers": info["ckpt_layers"], "parallelism": f"dp{world}",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "error_vs_oracle": main_error,
            "per_gate": per_gate,
            "speedup_vs_per_gate": (value / per_gate["value"]) if per_gate else None,
            "variants": variants,
            "roofline": roofline,
            "hbm": hbm,
            "e2e": e2e,
            "gpu_launches": launches,
            "step_graph": step_graph,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "peaks": {"source": peak_src, "hbm_gbs": hbm_gbs},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload == "paper_hea":
        return run_paper(args)
    if args.workload == "fusion_sweep":
        return run_fusion_sweep(args)
    if args.workload == "mixed512":
        return run_mixed(args)
    w = override(workloads.WORKLOADS[args.workload], args)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "hea20":
        return run_large(args, w)
    return run_small(args, w)


if __name__ == "__main__":
    sys.exit(main())
