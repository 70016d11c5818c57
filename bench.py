"""Benchmark: forward + gradient samples/s of the fused path on one GB300.

Workload (default): hardware-efficient ansatz, 12 qubits, 20 layers of
[RZ, RY, RZ on every qubit + CZ chain], RY(x) encoding, batch 256, MSE loss
of <Z_0> against labels in {-1, +1}; one step = forward expectations + loss +
adjoint gradients reduced per parameter (qf_train_step), inputs resident in
HBM. Synthetic seeded inputs (theta ~ U[0, 2pi), x ~ U[0, pi]^12).

Printed JSON line (rank 0): value = samples/s of the whole job, plus the
unfused one-kernel-per-gate comparator on the same GPU, the roofline of the
dominant kernel (fused adjoint pass), an end-to-end number through the
host-buffer C-ABI call, the oracle's CPU throughput, and sampled SM clocks.

``--impl reference`` times the float64 CPU oracle instead (the reference
arm): each step is the oracle's training step on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_02804_gb300 import workloads  # noqa: E402

WORKLOAD = "hea12"
FP32_LANES_PER_SM = 128
N_SM = 152
# GB300's dense FP64 rate (the complex128 path's denominator), TFLOP/s nominal
FP64_TFLOPS_NOMINAL = 1.25
# DRAM bytes (read + write) of one adjoint pass launch from an ncu capture of the current kernel build
# (profiles/pass_kernels_hea12.md); None where no capture of the current build exists.
ADJOINT_TRAFFIC_BYTES = {"hea12": 16_860_160}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(workloads.WORKLOADS) + ["mixed512", "paper_hea", "fusion_sweep"])
    ap.add_argument("--qubits", type=int, default=29, help="paper_hea: number of qubits")
    ap.add_argument("--circuits", type=int, default=0, help="mixed512: first N circuits only (profiling cases)")
    ap.add_argument("--no-autotune", action="store_true", help="mixed512: 12-qubit tiles for every circuit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true")
    ap.add_argument("--batch", type=int, default=0, help="override the workload's batch (profiling cases)")
    ap.add_argument("--depth", type=int, default=0, help="override the workload's depth (profiling cases)")
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


def cpu_baseline(w, max_seconds=20.0):
    """The float64 oracle's training step (forward, MSE/sum loss, adjoint
    gradient) on the host cores, over a bounded sample of the workload."""
    from oracle import oracle as orc
    orc.build()
    theta, x, y = workloads.make_inputs(w)
    c = orc.hea(w.n, w.d)
    threads = orc.max_threads()
    # size the sample: time one sample first
    t0 = time.perf_counter()
    _oracle_step(orc, c, w, theta, x[:1], None if y is None else y[:1], threads)
    one = time.perf_counter() - t0
    per_thread = max(1, int(max_seconds / max(one, 1e-6)))
    B = int(min(w.B, max(threads, per_thread * threads // 4)))
    t0 = time.perf_counter()
    _oracle_step(orc, c, w, theta, x[:B], None if y is None else y[:B], threads)
    dt = time.perf_counter() - t0
    return {"value": B / dt, "unit": "samples/s", "cores": threads, "kind": "oracle",
            "sample": f"{B} of the {w.B} samples of one {w.name} training step (n={w.n}, d={w.d}), "
                      f"float64, OpenMP over samples"}


def _oracle_step(orc, c, w, theta, x, y, threads):
    th = theta.astype(np.float64)
    xx = x.astype(np.float64)
    if w.loss == "mse":
        E = orc.expectation(c, th, xx, w.obs, threads=threads)
        dLdE = orc.mse_dLdE(E, y) * len(E) / w.B
    else:
        dLdE = np.ones(len(xx))
    return orc.gradient(c, th, xx, w.obs, dLdE=dLdE, threads=threads)


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    orc.build()
    theta, x, y = workloads.make_inputs(w)
    c = orc.hea(w.n, w.d)
    threads = orc.max_threads()
    t0 = time.perf_counter()
    _oracle_step(orc, c, w, theta, x[:1], None if y is None else y[:1], threads)
    one = time.perf_counter() - t0
    # each step: a bounded sample sized so that the whole run stays within minutes
    budget = 120.0 / max(args.steps + args.warmup, 1)
    Bs = int(max(1, min(w.B, threads * max(1, int(budget / max(one, 1e-6))))))
    for _ in range(args.warmup):
        _oracle_step(orc, c, w, theta, x[:Bs], None if y is None else y[:Bs], threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(orc, c, w, theta, x[:Bs], None if y is None else y[:Bs], threads)
    dt = time.perf_counter() - t0
    value = Bs * args.steps / dt
    line = {
        "impl": "reference", "metric": "fwd+grad samples/s", "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": f"{w.name}: HEA n={w.n} d={w.d} batch={w.B} loss={w.loss} obs=Z0",
                   "sample_per_step": Bs},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": f"{Bs} samples of the {w.name} batch per step"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
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
    tuner = Autotuner(path=os.environ.get("QF_AUTOTUNE_CACHE"))  # JSON cache file, or in memory only
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
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
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
                     "frac": achieved / fp32_peak, "traffic": None,
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


def run_epoch(args, w):
    """Large workload (n=20, d=1000, 1000 samples): micro-batches of `mb`
    samples with the checkpoint interval chosen from free HBM; one step = one
    epoch over all samples (gradients summed over micro-batches)."""
    import torch
    from paper_2603_02804_gb300 import build as qbuild
    from paper_2603_02804_gb300 import qfuse
    from paper_2603_02804_gb300.torch_api import Simulator

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    peaks, peak_src = load_peaks()
    theta_np, x_np, _ = workloads.make_inputs(w)
    N = w.B
    mb = int(w.extra.get("micro_batch", 100))
    free, _ = torch.cuda.mem_get_info()
    opts = dict(ckpt_mode=args.ckpt_mode, mem_save=args.mem_save, tc_path=args.tc)
    h = qfuse.qf_hea_create(w.n, w.d)
    c, ws_need = qfuse.qf_plan_fit(h, mb, int(0.8 * free), host_only=True, **opts)
    qfuse.qf_circuit_destroy(h)
    sim = Simulator(w.n, w.d, mb, ckpt_layers=c, obs=w.obs, **opts)
    theta = torch.from_numpy(theta_np).cuda()
    xs = [torch.from_numpy(x_np[i:i + mb]).cuda() for i in range(0, N, mb)]
    grad = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def epoch():
        grad.zero_()
        for xb in xs:
            _, _, g = sim.train_step(theta, xb, loss=w.loss)
            grad.add_(g)

    sim.train_step(theta, xs[0], loss=w.loss)
    epoch()  # warm every kernel of the timed epoch (library and torch)
    torch.cuda.synchronize()
    qfuse.qf_profile(sim.handle, True)
    qfuse.qf_profile_read(sim.handle)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            epoch()
        t1.record(stream)
        torch.cuda.synchronize()
    prof = qfuse.qf_profile_read(sim.handle)
    ms = t0.elapsed_time(t1) / args.steps
    info = sim.info()
    fwd_fl, bwd_fl = algorithmic_flops(w.n, w.d, mb)
    bwd_ms = prof["bwd_ms"] / max(prof["bwd_launches"], 1)
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    # the adjoint phase's flops over its time (checkpoint mode 1: it also re-runs the forward)
    phase_fl = (bwd_fl + (fwd_fl if args.ckpt_mode == 1 else 0)) * len(xs) * args.steps
    ach = phase_fl / (prof["bwd_ms"] / 1e3) / 1e12
    bytes_bwd = 32 * mb * (1 << w.n)  # read + write psi and lambda per adjoint pass
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    line = {
        "metric": "fwd+grad samples/s", "value": N * world / (ms / 1e3), "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": f"{w.name}: HEA n={w.n} d={w.d}, {N} samples per step (epoch) in micro-batches "
                               f"of {mb}, L=sum E, obs=Z0", "ckpt_layers_from_memory": c,
                   "ckpt_mode": args.ckpt_mode, "mem_save": bool(args.mem_save), "tc_path": bool(args.tc),
                   "fwd_ms_per_step": prof["fwd_ms"] / args.steps, "bwd_ms_per_step": prof["bwd_ms"] / args.steps,
                   "workspace_gb": sim.ws_bytes / 1e9, "passes": info["n_passes"],
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                     "traffic": None, "kernel": ("pass_kernel<true,true> (fused adjoint)" if args.ckpt_mode == 0 else
                                                 "adjoint phase: pass_kernel<true,true> and forward re-runs"),
                     "bwd_pass_ms": bwd_ms,
                     "hbm": {"achieved_gbs": bytes_bwd / (bwd_ms / 1e3) / 1e9, "peak_gbs": hbm_gbs,
                             "frac": bytes_bwd / (bwd_ms / 1e3) / 1e9 / hbm_gbs, "peak_source": peak_src}},
        "gpu_launches": None, "per_gate": None, "cpu_baseline": None, "e2e": None, "clocks": clk.summary(),
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
    from paper_2603_02804_gb300 import qfuse
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


def main():
    args = parse()
    if args.workload == "paper_hea":
        return run_paper(args)
    if args.workload == "fusion_sweep":
        return run_fusion_sweep(args)
    if args.workload == "mixed512":
        return run_mixed(args)
    if args.workload == "hea20":
        return run_epoch(args, override(workloads.WORKLOADS["hea20"], args))
    w = override(workloads.WORKLOADS[args.workload], args)
    if args.impl == "reference":
        return run_reference(args, w)
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
    opts = dict(ckpt_mode=args.ckpt_mode, mem_save=args.mem_save, tc_path=args.tc)
    if c128:
        opts["precision"] = "complex128"
    sim = Simulator(w.n, w.d, w.B, ckpt_layers=ckpt, obs=w.obs, **opts)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    from paper_2603_02804_gb300 import dp

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

    # ---- roofline of the dominant kernel: the fused adjoint pass kernel
    fwd_fl, bwd_fl = algorithmic_flops(w.n, w.d, w.B)
    info = sim.info()
    bwd_launch_ms = prof["bwd_ms"] / max(prof["bwd_launches"], 1)
    fwd_launch_ms = prof["fwd_ms"] / max(prof["fwd_launches"], 1)
    bwd_per_launch = bwd_fl / info["n_passes"]
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    alu_peak = FP64_TFLOPS_NOMINAL if c128 else fp32_peak
    achieved = bwd_per_launch / (bwd_launch_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak,
                "traffic": ADJOINT_TRAFFIC_BYTES.get(w.name) if not (args.tc or args.ckpt_mode or c128) else None,
                "kernel": ("pass64_kernel<true> (fused adjoint, complex128)" if c128
                           else "pass_kernel<true> (fused adjoint)"),
                "peak_source": ("GB300 dense FP64, nominal" if c128 else
                                f"152 SMs x 128 FP32 lanes x 2 x {clock_mhz:.0f} MHz"),
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
            if kw == opts:
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
                              "device_status": qfuse.qf_device_status(stream)}
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
                    "ms_per_step": pg_ms / args.steps, "gpu_launches_per_step": pg_launches // args.steps}
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

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


if __name__ == "__main__":
    sys.exit(main())
