"""Benchmark: fwd+adjoint patterns*slices per second of the multislice loss and gradient.

One step is one msp_loss_grad call on the W = 128, L = 4, S = 1024 workload (c2) at the
reconstruction's starting point (V = 0, the probe guess with a 20 angstrom defocus error,
Poisson-noisy patterns): the transmissions (Sec. 2.1), the window gather, the multislice forward
through all four slices, the far-field loss and residual (Sec. 3.2), the adjoint back through
every slice, the atomic-free overlap-add of every slice's potential gradient and the probe
gradient sum.  value = S * L / (time per step).  The same run also times, on the same GPU:
  * the layer step of Algorithm 1 (msp_layer_step: the same pass, one slice's gradient and step);
  * the plain method to its final loss (msp_reconstruct): c1, 50 sweeps from V = 0 with the known
    probe; c2, sweeps of the four slice steps and one probe step from the probe guess, in the FP32
    mode and in the precise-forward mode (time to the final loss, and the final losses);
  * the full 4096-position, 8-slice workload (c3), and the precise mode's cost per pass.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl msp|reference] [--config c2|...]

--impl reference times the FP64 CPU oracle on all the host's cores (a bounded sample of the
same workload and state per step); it is a reported baseline, not the target.

--config smd_gaas times the paper's second method instead: one iteration of
Algorithm 2 (Sec. 3.4: one matrix step of Eq. Opt_Prob_Matrix, the proximal step
of every slice, the lambda update and A = lambda A(o)) on the Table 1 setting,
N = 40, all 1600 cyclic probe shifts, M = 3; value = iterations / s.
Under torchrun (N > 1) every rank runs an independent replica (the method's
positions could be sharded, but this build is single-GPU): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import synth  # noqa: E402

METRIC = "fwd+adjoint patterns·slices/s"
UNIT = "pattern·slices/s"
CFG = synth.C2


def fft_flops(S, L, W):
    """Algorithmic FLOPs of one fwd+adjoint pass: (4L-2) 2-D FFTs of W x W per position,
    5 N log2 N each (the standard complex-FFT count)."""
    n = W * W
    return S * (4 * L - 2) * 5.0 * n * math.log2(n)


def measured_traffic(kernel: str, root: str = ROOT):
    """DRAM bytes of `kernel` from its committed ncu capture (profiles/traffic.json: per kernel
    the counters, per call (all its launches in one call) or per launch as the record's `per`
    says, the workload, the command and a hash of the kernel's sources), or None if those
    sources changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(root, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha1()
        for f in rec["sources"]:
            h.update(open(os.path.join(root, f), "rb").read())
        val = rec.get("dram_bytes_per_call", rec.get("dram_bytes_per_launch"))
        return val if rec.get("source_sha1") == h.hexdigest() else None
    except Exception:
        return None


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's time: every rank contributes x, all receive the maximum."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, ms_per_step: float) -> float:
    """Whole-job pattern*slices per second: every rank processes its own replica of the
    workload each step, and the job's step takes as long as its slowest rank's."""
    return world * units_per_rank / (ms_per_step * 1e-3)


# The tcgen05 kind::tf32 pipe rate measured by this repository's micro-benchmark
# (bench.py --config peaks: M = 128, N = 256, K = 8 MMAs back to back on every SM of a GB300):
# the denominator of the tf32 contractions' roofline fractions.
TF32_MEASURED_TFLOPS = 1073.0


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(msp, torch, dev, cfg, precision=0):
    """Seeded synthetic specimen, probe guess, raster and Poisson-noisy intensities (the library's
    FP32 forward model of the true specimen, then per-position seeded counting noise)."""
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd, precision=precision)
    V_true = synth.potential_slices(cfg).astype(np.float32)
    p_true = synth.probe(cfg).astype(np.complex64)
    p_guess = synth.probe(cfg, defocus_A=cfg.defocus_guess_A or cfg.defocus_A).astype(np.complex64)
    d_pos = torch.from_numpy(pos).to(dev)
    ws = msp.make_workspace(g, dev)
    I_clean = msp.forward(g, torch.from_numpy(p_true).to(dev), torch.from_numpy(V_true).to(dev), d_pos, ws=ws)
    I_meas = synth.poisson_counts(I_clean.cpu().numpy().astype(np.float64), cfg.dose, cfg.seed).astype(np.float32)
    return g, gd, pos, d_pos, ws, V_true, p_guess, I_meas


def _oracle_chunk(job):
    """One worker's share of the CPU baseline: the oracle's loss and gradients over its positions
    (a process of a spawn pool; one numpy thread per process)."""
    gd, probe, pos, I, L, obj = job
    from oracle import msp_oracle as O
    t0 = time.perf_counter()
    O.loss_grad(dict(gd, n_pos=len(pos)), probe, pos, I, V=np.zeros((L, obj, obj)))
    return time.perf_counter() - t0


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def cpu_oracle_rate(cfg, pos, I, probe, budget_s, cores):
    """pattern*slices/s of the FP64 oracle's loss and gradients (the CPU form of one msp_loss_grad
    pass) at the reconstruction's starting point, on `cores` processes of a spawn pool (1: this
    process), on as many positions as fit `budget_s`.  Returns (rate, positions, seconds)."""
    gd = synth.geometry(cfg)
    from oracle import msp_oracle as O
    if cores <= 1:
        done, t_used, n = 0, 0.0, 2
        while done < len(pos) and t_used < budget_s:
            sub = slice(done, min(len(pos), done + n))
            t0 = time.perf_counter()
            O.loss_grad(dict(gd, n_pos=sub.stop - sub.start), probe, pos[sub], I[sub],
                        V=np.zeros((cfg.n_slices, cfg.obj, cfg.obj)))
            t_used += time.perf_counter() - t0
            done = sub.stop
            n = min(2 * n, 64)
        return done * cfg.n_slices / t_used, done, t_used
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    # positions per worker from a single-position probe of the per-position cost
    t0 = time.perf_counter()
    O.loss_grad(dict(gd, n_pos=1), probe, pos[:1], I[:1], V=np.zeros((cfg.n_slices, cfg.obj, cfg.obj)))
    per = max(time.perf_counter() - t0, 1e-3)
    k = max(1, min(len(pos) // cores if len(pos) >= cores else 1, int(budget_s / per)))
    n = min(len(pos), k * cores)
    jobs = [(gd, probe, pos[i::cores][:k], I[i::cores][:k], cfg.n_slices, cfg.obj) for i in range(cores)]
    jobs = [j for j in jobs if len(j[2])]
    with ctx.Pool(len(jobs), initializer=_single_thread_env) as pool:
        pool.map(_oracle_chunk, jobs[:1])          # start-up (imports) outside the timing
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, jobs)
        dt = time.perf_counter() - t0
    return n * cfg.n_slices / dt, n, dt


def cpu_baseline(cfg, pos, I, probe, budget_s=10.0):
    """The FP64 oracle, as it stands, on the host: one thread, and all host cores (a spawn pool over
    positions), each on a bounded sample of the workload's positions at the GPU arm's state."""
    nproc = os.cpu_count() or 1
    r1, n1, t1 = cpu_oracle_rate(cfg, pos, I, probe, budget_s, 1)
    ra, na, ta = cpu_oracle_rate(cfg, pos, I, probe, budget_s, nproc)
    return {"value": ra, "unit": UNIT, "cores": nproc, "kind": "oracle", "nproc": nproc,
            "sample": f"FP64 numpy oracle loss and gradients (all slices, probe) at V = 0 with the probe guess and "
                      f"the GPU arm's measured patterns: {na} of {len(pos)} positions of {cfg.name} on {nproc} "
                      f"processes ({ta:.1f} s); single thread: {n1} positions ({t1:.1f} s)",
            "single_thread": {"value": r1, "unit": UNIT, "cores": 1, "positions": n1, "seconds": t1},
            "all_cores": {"value": ra, "unit": UNIT, "cores": nproc, "positions": na, "seconds": ta}}


def reference_state(cfg, idx):
    """The measured patterns of scan positions `idx` of the workload, made on the host by the oracle
    (the GPU arm makes the same patterns with the library's forward model), with the same
    per-position counting noise, and the probe guess."""
    from oracle import msp_oracle as O
    pos = synth.scan_positions(cfg)[idx]
    gd = synth.geometry(cfg, n_pos=len(pos))
    I = O.forward(gd, synth.probe(cfg).astype(np.complex64), pos, V=synth.potential_slices(cfg).astype(np.float32))
    I = synth.poisson_counts(I, cfg.dose, cfg.seed, index=idx).astype(np.float32)
    probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A or cfg.defocus_A).astype(np.complex64)
    return pos, I, probe


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = CFG
    nproc = os.cpu_count() or 1
    # a sample of positions spread over the scan, patterns made once (outside the steps)
    idx = np.linspace(0, cfg.n_pos - 1, min(cfg.n_pos, 32 * nproc)).astype(int)
    pos, I, probe = reference_state(cfg, idx)
    per_step = []
    budget = max(0.5, 120.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        r, n, dt = cpu_oracle_rate(cfg, pos, I, probe, budget, nproc)
        if i >= args.warmup:
            per_step.append(r)
    value = float(np.median(per_step))
    base = {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"per step, up to {n} of {cfg.n_pos} positions of {cfg.name} (spread over the scan) on {nproc} "
                      f"processes: FP64 numpy oracle loss and gradients at V = 0 with the probe guess"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cfg.n_pos * cfg.n_slices / value * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "call": "oracle.loss_grad (all slices and the probe)",
                       "parallelism": f"cpu, {nproc} processes"},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Algorithm 2 (sparse matrix decomposition)
# ---------------------------------------------------------------------------

SMD_METRIC = "Algorithm 2 iterations/s"
SMD_UNIT = "iterations/s"


def smd_flops(n, S, M):
    """Algorithmic FLOPs of one Algorithm 2 iteration, split as (contractions, DFTs): the two
    complex contractions N^2 x N^2 x S of the matrix step (8 flops per complex multiply-add),
    and direct DFT passes of 8 N^3 flops each -- 4 per column of A P (S columns), and, per
    column of the N^2 x N^2 matrices, 8 (M - 2) for the decomposition gradient and 4 (M - 2)
    for the transfer pass (a unit impulse needs no DFT for its first propagation, and the
    adjoint wave on the first slice is needed at one pixel only)."""
    n2 = n * n
    return 2 * 8.0 * n2 * n2 * S, 8.0 * n ** 3 * (4 * S + 12 * max(M - 2, 0) * n2)


def smd_inputs(msp, torch, dev, cfg):
    """Table 1 stand-in: lattice slices exp(i sigma V), the aperture probe, every cyclic shift,
    noise-free intensities |F A P|^2 (A from the library's transfer matrix; P and F applied
    with torch, as input synthesis only)."""
    gd = synth.smd_geometry(cfg)
    n, M = cfg.obj, cfg.n_slices
    g = msp.smd_geometry(**gd)
    V = synth.potential_slices(cfg)
    truth = np.exp(1j * gd["sigma"] * V).astype(np.complex64)
    probe = synth.probe(cfg).astype(np.complex64)
    shifts = synth.cyclic_shifts(n)
    ws = msp.smd_make_workspace(g, dev)
    A_true = msp.smd_transfer(g, torch.from_numpy(truth).to(dev), 1.0, ws=ws)      # row j = column j
    p = torch.from_numpy(probe).to(dev)
    P = torch.stack([torch.roll(p, (int(a), int(b)), dims=(0, 1)).reshape(-1) for a, b in shifts], dim=1)
    B = A_true.transpose(0, 1) @ P                                                  # exit waves, N^2 x S
    I = (torch.fft.fft2(B.transpose(0, 1).reshape(-1, n, n)).abs() ** 2).float()
    torch.cuda.synchronize()
    return g, gd, ws, probe, shifts, I.cpu().numpy()


def smd_cpu_iteration(cfg, probe, shifts, I):
    """One Algorithm 2 iteration of the FP64 oracle, as it stands (dense N^2 x N^2 matrices)."""
    from oracle import msp_oracle as O
    gd = synth.smd_geometry(cfg)
    n, M = cfg.obj, cfg.n_slices
    t0 = time.perf_counter()
    F = O.dft_matrix_2d(n)
    G = O.propagator_matrix(gd, n)
    P = O.probe_matrix(probe.astype(np.complex128), shifts)
    Im = O.measurement_matrix(I.astype(np.float64))
    o = [np.ones(n * n, complex) for _ in range(M)]
    A = O.transfer_matrix(G, o)
    t1 = time.perf_counter()
    A, _ = O.matrix_step(A, F, P, Im, O.matrix_step_size(probe.astype(np.complex128)))
    O.decomposition_update(A, G, o, 1.0)
    return time.perf_counter() - t1, t1 - t0


def smd_cpu_baseline(cfg, probe, shifts, I, budget_s=60.0, max_iter=3):
    times = []
    t_start = time.perf_counter()
    cpu0 = time.process_time()
    while len(times) < max_iter and (not times or time.perf_counter() - t_start < budget_s):
        dt, _ = smd_cpu_iteration(cfg, probe, shifts, I)
        times.append(dt)
    t = float(np.median(times))
    cores = max(1, round((time.process_time() - cpu0) / max(time.perf_counter() - t_start, 1e-9)))
    return {"value": 1.0 / t, "unit": SMD_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} full Algorithm 2 iteration(s) of {cfg.name} (N = {cfg.obj}, S = {cfg.n_pos}, "
                      f"M = {cfg.n_slices}), FP64 numpy oracle with dense N^2 x N^2 matrices, multithreaded BLAS, "
                      f"median {t:.2f} s; cores = process CPU time / wall time"}


def run_smd_reference(args, rank, world):
    if rank != 0:
        return
    cfg = CFG
    import torch
    from paper_2205_03902_gb300 import msp
    if torch.cuda.is_available():
        import __graft_entry__
        __graft_entry__.build()
        _, _, _, probe, shifts, I = smd_inputs(msp, torch, torch.device("cuda", 0), cfg)
    else:
        probe = synth.probe(cfg).astype(np.complex64)
        shifts = synth.cyclic_shifts(cfg.obj)
        I = np.ones((len(shifts), cfg.obj, cfg.obj), np.float32)
    base = smd_cpu_baseline(cfg, probe, shifts, I, budget_s=60.0, max_iter=max(1, min(args.steps, 3)))
    value = base["value"]
    line = {"impl": "reference", "metric": SMD_METRIC, "value": value, "unit": SMD_UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "call": "oracle.matrix_step + oracle.decomposition_update",
                       "parallelism": f"cpu, {base['cores']} cores busy (multithreaded BLAS)"},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": SMD_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_smd(args, rank, world, local_rank):
    import torch
    from paper_2205_03902_gb300 import msp
    import __graft_entry__
    __graft_entry__.build()

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)

    cfg = CFG
    g, gd, ws, probe_h, shifts_h, I_h = smd_inputs(msp, torch, dev, cfg)
    n, M, S = cfg.obj, cfg.n_slices, cfg.n_pos
    probe = torch.from_numpy(probe_h).to(dev)
    shifts = torch.from_numpy(shifts_h).to(dev)
    I = torch.from_numpy(I_h).to(dev)
    o = torch.ones((M, n, n), dtype=torch.complex64, device=dev)     # Algorithm 2 starts at O^0 = I, lambda = 1
    lam = torch.ones(1, dtype=torch.float64, device=dev)
    A = msp.smd_transfer(g, o, 1.0, ws=ws)
    obj = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(A, o, lam, probe, shifts, I, obj):
        msp.smd_matrix_step(g, A, probe, shifts, I, ws=ws, objective=obj[0:1])
        msp.smd_decompose(g, A, o, lam, ws=ws, objective=obj[1:2])

    for _ in range(args.warmup):
        step(A, o, lam, probe, shifts, I, obj)
    torch.cuda.synchronize()
    obj_first = obj.cpu().tolist()

    msp.profile_read(reset=True)
    msp.profile_enable(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(A, o, lam, probe, shifts, I, obj)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = msp.profile_read(reset=True)
    msp.profile_enable(False)
    ms_per_step = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), dist, dev) / args.steps
    value = job_throughput(world, 1.0, ms_per_step)
    obj_last = obj.cpu().tolist()

    # ---- end to end with host buffers: the step's inputs (probe, shifts, I) copied from pinned
    # memory on a copy stream (two input sets), the slices, lambda and objectives read back ----
    h_I = torch.from_numpy(I_h).pin_memory()
    h_p = torch.from_numpy(probe_h).pin_memory()
    h_s = torch.from_numpy(shifts_h).pin_memory()
    h_o = [torch.empty((M, n, n), dtype=torch.complex64).pin_memory() for _ in range(2)]
    h_scal = [torch.empty(3, dtype=torch.float64).pin_memory() for _ in range(2)]
    sets = [dict(I=torch.empty_like(I), p=torch.empty_like(probe), s=torch.empty_like(shifts),
                 scal=torch.empty(3, dtype=torch.float64, device=dev)) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ev_copy = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    h2d = h_I.numel() * 4 + h_p.numel() * 8 + h_s.numel() * 4
    d2h = h_o[0].numel() * 8 + h_scal[0].numel() * 8

    def issue_copy(k):
        b = sets[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(ev_done[k % 2])
            b["I"].copy_(h_I, non_blocking=True)
            b["p"].copy_(h_p, non_blocking=True)
            b["s"].copy_(h_s, non_blocking=True)
            ev_copy[k % 2].record(copy_stream)

    def issue_step(k):
        b = sets[k % 2]
        stream.wait_event(ev_copy[k % 2])
        step(A, o, lam, b["p"], b["s"], b["I"], b["scal"])
        b["scal"][2:3].copy_(lam)
        h_o[k % 2].copy_(o, non_blocking=True)
        h_scal[k % 2].copy_(b["scal"], non_blocking=True)
        ev_done[k % 2].record(stream)

    e_steps = max(3, min(args.steps, 50))
    issue_copy(0)
    issue_step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issue_copy(1)
    for k in range(1, e_steps + 1):
        if k < e_steps:
            issue_copy(k + 1)
        issue_step(k)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e_steps
    assert np.isfinite(h_scal[e_steps % 2].numpy()).all()
    e2e_value = job_throughput(world, 1.0, 1e3 * max_over_ranks(e2e_s, dist, dev))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = read_peaks()
    gemm_flops, dft_flops = smd_flops(n, S, M)
    gemm_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    # the contraction runs on the tensor cores as a real tf32 product with operands split into
    # (big, small) pairs: 3 tf32 products of 8 flops per complex multiply-add, 24 N^4 S per launch
    tc_flops = 3 * gemm_flops / 2
    tf32_peak = TF32_MEASURED_TFLOPS
    achieved = tc_flops / (gemm_ms * 1e-3) / 1e12
    line = {
        "metric": SMD_METRIC, "value": value, "unit": SMD_UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "call": "msp_smd_matrix_step + msp_smd_decompose (auto steps)",
                   "N": n, "shifts": S, "slices": M,
                   "l2": "flushed between timed steps (256 MiB write outside the step events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": achieved / tf32_peak,
                     "traffic": measured_traffic("cgemm_kernel") if cfg is synth.SMD_GAAS else None,
                     "kernel": "cgemm_kernel (tcgen05 kind::tf32, 3 tf32 products per FP32 product; A P and C P^H)",
                     "kernel_ms": gemm_ms,
                     "complex_fp32_equivalent_tflops": (gemm_flops / 2) / (gemm_ms * 1e-3) / 1e12,
                     "peak_source": "measured tcgen05 kind::tf32 pipe rate (bench.py --config peaks, N = 256)"},
        "step_tflops": (gemm_flops + dft_flops) / (ms_per_step * 1e-3) / 1e12,
        "e2e": {"value": e2e_value, "unit": SMD_UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(prof["all_launches"]),
        "clocks": clocks,
        "objectives_first_timed_step": obj_first, "objectives_last_timed_step": obj_last,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = smd_cpu_baseline(cfg, probe_h, shifts_h, I_h, budget_s=30.0, max_iter=2)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# DFT as a matrix product on the tensor cores, against the fused shared-memory FFT
# ---------------------------------------------------------------------------

DFT_METRIC = "2-D DFTs/s (W = 128, tensor-core contraction)"
DFT_UNIT = "transforms/s"


def run_dft(args, rank, world, local_rank):
    """The batched 2-D DFT of msp_dft2_tc on c3's shape (S = 4096 images of 128 x 128), and, in the
    same run, the fused kernel's own FFT rate in the c3 layer step ((4L - 2) 2-D FFTs per position)."""
    import torch
    from paper_2205_03902_gb300 import msp
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg = synth.C3
    S, W = cfg.n_pos, cfg.win
    x_h = synth.random_complex((S, W, W), 7).astype(np.complex64)
    x = torch.from_numpy(x_h).to(dev)
    y = torch.empty_like(x)
    n = int(msp.lib().msp_dft2_tc_workspace_bytes(W, S))
    buf = torch.empty(n + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    ws = msp.Workspace(buf[off:off + n])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        msp.dft2_tc(x, out=y, ws=ws)
    torch.cuda.synchronize()
    msp.profile_read(reset=True)
    msp.profile_enable(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        msp.dft2_tc(x, out=y, ws=ws)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = msp.profile_read(reset=True)
    msp.profile_enable(False)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    value = S / (ms * 1e-3)
    pass_ms = prof["fused_ms"] / max(1, prof["fused_launches"])
    tc_flops = 24.0 * S * W ** 3                      # one pass: 24 M N K with M = K = W, N = S W
    tf32_peak = TF32_MEASURED_TFLOPS
    # end to end: host -> device, transform, device -> host (pinned buffers)
    x_pin = torch.from_numpy(x_h).pin_memory()
    y_pin = torch.empty_like(x_pin).pin_memory()
    e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        x.copy_(x_pin, non_blocking=True)
        msp.dft2_tc(x, out=y, ws=ws)
        y_pin.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e2e = S / ((time.perf_counter() - t0) / e_steps)
    # the fused kernel's FFT rate on the c3 layer step
    g, gd, pos, d_pos, ws3, V_true, p_guess, I_meas = make_inputs(msp, torch, dev, cfg)
    probe = torch.from_numpy(p_guess).to(dev)
    V = torch.zeros((cfg.n_slices, cfg.obj, cfg.obj), dtype=torch.float32, device=dev)
    Im = torch.from_numpy(I_meas).to(dev)
    for _ in range(2):
        msp.layer_step(g, probe, V, d_pos, Im, 0, ws=ws3)
    torch.cuda.synchronize()
    msp.profile_read(reset=True)
    msp.profile_enable(True)
    for _ in range(5):
        msp.layer_step(g, probe, V, d_pos, Im, 0, ws=ws3)
    torch.cuda.synchronize()
    p3 = msp.profile_read(reset=True)
    msp.profile_enable(False)
    fused_ms = p3["fused_ms"] / max(1, p3["fused_launches"])
    fft_rate = (4 * cfg.n_slices - 2) * S / (fused_ms * 1e-3)
    line = {
        "metric": DFT_METRIC, "value": value, "unit": DFT_UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"dft2_W{W}_S{S} (c3 shape)", "call": "msp_dft2_tc (two tensor-core passes)",
                   "l2": "flushed between timed steps (256 MiB write outside the step events)",
                   "parallelism": "single GPU"},
        "roofline": {"bound": "tensor", "achieved": tc_flops / (pass_ms * 1e-3) / 1e12, "peak": tf32_peak,
                     "unit": "TFLOP/s", "frac": tc_flops / (pass_ms * 1e-3) / 1e12 / tf32_peak, "traffic": None,
                     "kernel": "cgemm_kernel<false, true> (one DFT pass, tcgen05 kind::tf32, split operands)",
                     "kernel_ms": pass_ms,
                     "peak_source": "measured tcgen05 kind::tf32 pipe rate (bench.py --config peaks, N = 256)"},
        "smem_fft_comparison": {"fused_kernel": "position_kernel<128, LAYER> on the c3 layer step",
                                "fused_kernel_ms": fused_ms, "fft_transforms_per_s": fft_rate,
                                "tensor_dft_over_smem_fft": value / fft_rate},
        "e2e": {"value": e2e, "unit": DFT_UNIT, "h2d_bytes_per_step": S * W * W * 8, "d2h_bytes_per_step": S * W * W * 8},
        "gpu_launches": int(prof["all_launches"]),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        sub = x_h[:64].astype(np.complex128)
        from oracle import msp_oracle as O
        t0 = time.perf_counter()
        cpu0 = time.process_time()
        reps = 0
        while time.perf_counter() - t0 < 5.0:
            for v in sub:
                O.dft2(v)
            reps += 1
        dt = time.perf_counter() - t0
        cores = max(1, round((time.process_time() - cpu0) / dt))
        line["cpu_baseline"] = {"value": reps * len(sub) / dt, "unit": DFT_UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{reps * len(sub)} transforms of 128 x 128 with the oracle's numpy FFT, "
                                          f"{dt:.1f} s; cores = process CPU time / wall time"}
    print(json.dumps(line), flush=True)


def time_events(fn, n, stream, flush=None):
    """Mean ms of fn() over n calls, CUDA events on `stream`, L2 flushed before each (outside)."""
    import torch
    ms = 0.0
    for i in range(n):
        if flush is not None:
            flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    return ms / n


def plain_method_run(msp, torch, dev, cfg, sweeps, probe_steps, precision, stream):
    """Time to the plain method's final loss: msp_reconstruct from V = 0 and the workload's probe
    guess (the true probe when it is known), CUDA events around the whole call."""
    g, gd, pos, d_pos, ws, V_true, p_guess, I_meas = make_inputs(msp, torch, dev, cfg, precision)
    I = torch.from_numpy(I_meas).to(dev)
    plan = msp.plan(sweeps, probe_steps=probe_steps)
    out = {}
    for rep in range(2):                       # the first run warms up
        V = torch.zeros((cfg.n_slices, cfg.obj, cfg.obj), dtype=torch.float32, device=dev)
        p = torch.from_numpy(p_guess).to(dev)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h = msp.reconstruct(g, plan, p, V, d_pos, I, ws=ws)
        b.record(stream)
        b.synchronize()
        out = {"ms": a.elapsed_time(b), "sweeps": sweeps, "probe_steps_per_sweep": probe_steps,
               "passes": int(sweeps * (cfg.n_slices + probe_steps) + 1),
               "loss_first": float(h[0].item()), "loss_final": float(h[-1].item())}
    out["precision"] = {0: "fp32", 1: "fp64_forward", 2: "split_bf16_dft", 3: "double_float_forward"}[precision]
    return out


def net_macs_per_pixel(L):
    """Multiply-adds per pixel of the proposal network's forward pass (true channel counts)."""
    ch = [2 * L, 64, 64, 64, 64, 64, L]
    return sum(9 * ch[i] * ch[i + 1] for i in range(6))


def learned_proposal_run(msp, torch, dev, stream, peaks, n_train=6, sweeps=16, train_steps=1500, every=2,
                         horizon=None, held_out=(200, 201, 202)):
    """The learned-proposal form on the eight-slice workload: a corpus from plain-method
    trajectories of `n_train` seeded specimens, Adam training, the network's kernel rates, and,
    on each held-out specimen, the wall time to the plain method's final loss: learned (the
    acceptance loop) against plain (msp_reconstruct)."""
    from paper_2205_03902_gb300 import learned
    cfg5 = synth.C5
    L, N = cfg5.n_slices, cfg5.obj
    zeros = lambda: torch.zeros((L, N, N), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    corpus = learned.Corpus()
    for k in range(n_train):
        c = synth.c5_specimen(100 + k)
        g, gd, pos, d_pos, ws, _, p, I = make_inputs(msp, torch, dev, c)
        probe, I = torch.from_numpy(p).to(dev), torch.from_numpy(I).to(dev)
        states, _ = learned.plain_trajectory(g, probe, zeros(), d_pos, I, sweeps, ws=ws)
        learned.add_trajectory(corpus, g, probe, d_pos, I, states, every=every, horizon=horizon, ws=ws)
        del ws
    torch.cuda.synchronize()
    corpus_s = time.perf_counter() - t0
    sv, sg, sd = learned.input_scales(corpus)
    s = msp.net_shape(L, N, N, sv, sg, sd)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    a, b = ev()
    a.record(stream)
    params, tl = learned.train(s, corpus, train_steps, lr=1e-3, seed=0)
    b.record(stream)
    b.synchronize()
    train_ms = a.elapsed_time(b)
    # kernel rates of the network
    nws = msp.net_make_workspace(s, dev)
    out = torch.empty_like(corpus.V[0])
    msp.net_forward(s, params, corpus.V[0], corpus.G[0], out=out, ws=nws)
    fms = time_events(lambda: msp.net_forward(s, params, corpus.V[0], corpus.G[0], out=out, ws=nws), 10, stream)
    pc, m_, v_ = params.clone(), torch.zeros_like(params), torch.zeros_like(params)
    tms = time_events(lambda: msp.net_train_step(s, pc, m_, v_, 1, 1e-3, corpus.V[0], corpus.G[0], corpus.T[0],
                                                 ws=nws), 10, stream)
    P_px = N * N
    fwd_flop = 2.0 * P_px * net_macs_per_pixel(L)
    ch = [2 * L, 64, 64, 64, 64, 64, L]
    dgrad_flop = 2.0 * P_px * sum(9 * ch[i] * ch[i + 1] for i in range(1, 6))
    train_flop = 2 * fwd_flop + dgrad_flop          # forward, weight gradients, data gradients
    bf16_peak = float(peaks.get("bf16_tflops", 0.0)) or None
    # held-out specimens: plain to its final loss, then the learned loop to the same loss
    runs = []
    for spec in held_out:
        c = synth.c5_specimen(spec)
        g, gd, pos, d_pos, ws, _, p, I = make_inputs(msp, torch, dev, c)
        probe, I = torch.from_numpy(p).to(dev), torch.from_numpy(I).to(dev)
        lws = msp.learned_make_workspace(g, s, dev)
        msp.reconstruct(g, msp.plan(1), probe, zeros(), d_pos, I, ws=ws)                 # warm-up
        msp.learned_propose(g, s, params, probe, zeros(), d_pos, I, ws=ws, learn_ws=lws)
        V = zeros()
        torch.cuda.synchronize()
        a, b = ev()
        a.record(stream)
        h = msp.reconstruct(g, msp.plan(sweeps), probe, V, d_pos, I, ws=ws)
        b.record(stream)
        b.synchronize()
        plain_ms, target = a.elapsed_time(b), float(h[-1].item())
        V = zeros()
        torch.cuda.synchronize()
        a, b = ev()
        a.record(stream)
        hist = learned.reconstruct_learned(g, s, params, probe, V, d_pos, I, 2 * sweeps, target_loss=target, ws=ws,
                                           learn_ws=lws)
        b.record(stream)
        b.synchronize()
        learned_ms = a.elapsed_time(b)
        reached = hist[-1][2] <= target
        runs.append({"specimen": spec, "target_loss": target, "plain_ms": plain_ms, "plain_sweeps": sweeps,
                     "learned_ms": learned_ms if reached else None, "learned_reached": bool(reached),
                     "learned_iterations": len(hist), "accepted": int(sum(x[1] for x in hist)),
                     "learned_final_loss": hist[-1][2], "speedup": plain_ms / learned_ms if reached else None})
        del ws, lws
    all_reached = all(r["learned_reached"] for r in runs)
    plain_total = sum(r["plain_ms"] for r in runs)
    learned_total = sum(r["learned_ms"] for r in runs) if all_reached else None
    return {
        "workload": cfg5.name, "specimens": {"train": [100 + k for k in range(n_train)], "held_out": list(held_out)},
        "corpus": {"samples": len(corpus), "trajectory_sweeps": sweeps, "state_every": every,
                   "build_s": corpus_s,
                   "target": "V_K - V_k" if horizon is None else f"V_min(k+{horizon},K) - V_k",
                   "note": "k along each plain trajectory of K sweeps"},
        "scales": {"s_V": sv, "s_G": sg, "s_D": sd},
        "training": {"steps": train_steps, "ms": train_ms, "loss_first10": float(np.mean(tl[:10])),
                     "loss_last10": float(np.mean(tl[-10:]))},
        "net_forward": {"ms": fms, "tflops": fwd_flop / (fms * 1e-3) / 1e12,
                        "frac_of_bf16_peak": (fwd_flop / (fms * 1e-3) / 1e12) / bf16_peak if bf16_peak else None,
                        "flop": fwd_flop},
        "net_train_step": {"ms": tms, "tflops": train_flop / (tms * 1e-3) / 1e12,
                           "frac_of_bf16_peak": (train_flop / (tms * 1e-3) / 1e12) / bf16_peak if bf16_peak else None,
                           "flop": train_flop},
        "time_to_plain_final_loss": {"held_out_runs": runs, "plain_ms_total": plain_total,
                                     "learned_ms_total": learned_total,
                                     "speedup": plain_total / learned_total if learned_total else None},
    }


def run_msp(args, rank, world, local_rank):
    import torch
    from paper_2205_03902_gb300 import msp
    import __graft_entry__
    __graft_entry__.build()

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)

    cfg = CFG
    g, gd, pos, d_pos, ws, V_true, p_guess, I_meas_h = make_inputs(msp, torch, dev, cfg)
    S, L, W = cfg.n_pos, cfg.n_slices, cfg.win
    probe = torch.from_numpy(p_guess).to(dev)
    V = torch.zeros((L, cfg.obj, cfg.obj), dtype=torch.float32, device=dev)   # Alg. 1 starts from V = 0
    I_meas = torch.from_numpy(I_meas_h).to(dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    dV = torch.empty_like(V)
    dprobe = torch.empty_like(probe)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        msp.loss_grad(g, probe, V, d_pos, I_meas, ws=ws, loss=loss, dV=dV, dprobe=dprobe)

    msp.set_overlap_add(msp.OVERLAP_L2_REDUCE if args.overlap_add == "l2" else msp.OVERLAP_FIXED_ORDER)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    msp.profile_read(reset=True)
    msp.profile_enable(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))          # L2 flushed between timed steps (outside the events)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = msp.profile_read(reset=True)
    msp.profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, S * L, ms_per_step)
    loss_step = float(loss.item())

    # ---- end to end through the public API with host buffers (pinned), copies timed ----
    # Every step copies its inputs (patterns, potentials, probe, positions) from pinned host
    # memory and reads its results (dV, dprobe, loss) back.  As a caller would, the copy of
    # step k+1's inputs runs on a copy stream while step k computes (two input sets).
    h_I = torch.from_numpy(I_meas_h).pin_memory()
    h_V = torch.zeros((L, cfg.obj, cfg.obj), dtype=torch.float32).pin_memory()
    h_p = torch.from_numpy(p_guess).pin_memory()
    h_pos = torch.from_numpy(pos).pin_memory()
    h_dV = [torch.empty_like(h_V).pin_memory() for _ in range(2)]
    h_dp = [torch.empty_like(h_p).pin_memory() for _ in range(2)]
    h_loss = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    sets = [dict(I=torch.empty_like(I_meas), V=torch.empty_like(V), p=torch.empty_like(probe),
                 pos=torch.empty_like(d_pos), loss=torch.empty(1, dtype=torch.float64, device=dev),
                 dV=torch.empty_like(V), dp=torch.empty_like(probe)) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ev_copy = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    h2d = h_I.numel() * 4 + h_V.numel() * 4 + h_p.numel() * 8 + h_pos.numel() * 4
    d2h = h_dV[0].numel() * 4 + h_dp[0].numel() * 8 + 8

    def issue_copy(k):
        b = sets[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(ev_done[k % 2])      # step k-2 no longer reads this set
            b["I"].copy_(h_I, non_blocking=True)
            b["V"].copy_(h_V, non_blocking=True)
            b["p"].copy_(h_p, non_blocking=True)
            b["pos"].copy_(h_pos, non_blocking=True)
            ev_copy[k % 2].record(copy_stream)

    def issue_step(k):
        b = sets[k % 2]
        stream.wait_event(ev_copy[k % 2])
        msp.loss_grad(g, b["p"], b["V"], b["pos"], b["I"], ws=ws, loss=b["loss"], dV=b["dV"], dprobe=b["dp"])
        h_dV[k % 2].copy_(b["dV"], non_blocking=True)
        h_dp[k % 2].copy_(b["dp"], non_blocking=True)
        h_loss[k % 2].copy_(b["loss"], non_blocking=True)
        ev_done[k % 2].record(stream)

    e_steps = max(3, min(args.steps, 50))
    issue_copy(0)
    issue_step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issue_copy(1)
    for k in range(1, e_steps + 1):
        if k < e_steps:
            issue_copy(k + 1)
        issue_step(k)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e_steps
    assert np.isfinite(h_loss[e_steps % 2].numpy()).all()
    e2e_value = job_throughput(world, S * L, 1e3 * max_over_ranks(e2e_s, dist, dev))

    if rank != 0:
        sampler.stop()
        if dist:
            dist.destroy_process_group()
        return

    # ---- further measurements of this run (rank 0), clocks still sampled ----
    extra = {}
    if not args.quick:
        # the other overlap-add of the same step: reductions in L2 from the fused kernel (or the gather)
        other = msp.OVERLAP_FIXED_ORDER if args.overlap_add == "l2" else msp.OVERLAP_L2_REDUCE
        msp.set_overlap_add(other)
        step()
        msp.profile_read(reset=True)
        msp.profile_enable(True)
        oms = time_events(step, 20, stream, flush)
        po = msp.profile_read(reset=True)
        msp.profile_enable(False)
        msp.set_overlap_add(msp.OVERLAP_L2_REDUCE if args.overlap_add == "l2" else msp.OVERLAP_FIXED_ORDER)
        extra["other_overlap_add"] = {
            "overlap_add": "l2_reduce" if other == msp.OVERLAP_L2_REDUCE else "fixed_order",
            "call": "msp_loss_grad, the same step", "ms": oms, "value": S * L / (oms * 1e-3), "unit": UNIT,
            "fused_kernel_ms": po["fused_ms"] / 20, "launches_per_call": po["all_launches"] / 20}
        # the layer step of Algorithm 1 on the same state
        Vl = torch.zeros_like(V)
        lb, mu = torch.empty(1, dtype=torch.float64, device=dev), torch.empty(1, dtype=torch.float64, device=dev)
        msp.profile_read(reset=True)
        msp.profile_enable(True)
        lms = time_events(lambda: msp.layer_step(g, probe, Vl, d_pos, I_meas, 0, ws=ws, loss_before=lb, mu=mu),
                          10, stream, flush)
        pl = msp.profile_read(reset=True)
        msp.profile_enable(False)
        extra["layer_step"] = {"call": "msp_layer_step(layer=0, auto step)", "ms": lms,
                               "value": S * L / (lms * 1e-3), "unit": UNIT,
                               "fused_kernel_ms": pl["fused_ms"] / 10,
                               "fused_launches_per_call": pl["fused_launches"] / 10}
        # the precise-forward mode's cost per pass on the same state
        gp = msp.geometry(**gd, precision=msp.MSP_PRECISION_FP64_FORWARD)
        wsp = msp.make_workspace(gp, dev)
        pms = time_events(lambda: msp.loss_grad(gp, probe, V, d_pos, I_meas, ws=wsp), 3, stream, flush)
        extra["precise_forward"] = {"call": "msp_loss_grad, MSP_PRECISION_FP64_FORWARD", "ms": pms,
                                    "value": S * L / (pms * 1e-3), "unit": UNIT, "cost_vs_fp32": pms / ms_per_step}
        del wsp
        gd_ = msp.geometry(**gd, precision=msp.MSP_PRECISION_DF_FORWARD)
        wsd = msp.make_workspace(gd_, dev)
        msp.loss_grad(gd_, probe, V, d_pos, I_meas, ws=wsd)
        dms = time_events(lambda: msp.loss_grad(gd_, probe, V, d_pos, I_meas, ws=wsd), 5, stream, flush)
        extra["precise_forward_double_float"] = {"call": "msp_loss_grad, MSP_PRECISION_DF_FORWARD", "ms": dms,
                                                 "value": S * L / (dms * 1e-3), "unit": UNIT,
                                                 "cost_vs_fp32": dms / ms_per_step}
        del wsd
        # the split-BF16 precision form (tensor-core DFT passes) on the same state
        gb = msp.geometry(**gd, precision=msp.MSP_PRECISION_BF16X3_DFT)
        wsb = msp.make_workspace(gb, dev)
        msp.loss_grad(gb, probe, V, d_pos, I_meas, ws=wsb)
        msp.profile_read(reset=True)
        msp.profile_enable(True)
        bms = time_events(lambda: msp.loss_grad(gb, probe, V, d_pos, I_meas, ws=wsb), 5, stream, flush)
        msp.profile_enable(False)
        extra["split_bf16_dft"] = {"call": "msp_loss_grad, MSP_PRECISION_BF16X3_DFT", "ms": bms,
                                   "value": S * L / (bms * 1e-3), "unit": UNIT, "cost_vs_fp32": bms / ms_per_step}
        del wsb
        # the plain method to its final loss
        pm = {
            "c1_known_probe": plain_method_run(msp, torch, dev, synth.C1, 50, 0, 0, stream),
            "c2_probe_estimation_fp32": plain_method_run(msp, torch, dev, cfg, 20, 1, 0, stream),
            "c2_probe_estimation_precise": plain_method_run(msp, torch, dev, cfg, 20, 1, 1, stream),
            "c2_probe_estimation_double_float": plain_method_run(msp, torch, dev, cfg, 20, 1, 3, stream),
            "c2_probe_estimation_split_bf16": plain_method_run(msp, torch, dev, cfg, 20, 1, 2, stream),
            "c3_probe_estimation_fp32": plain_method_run(msp, torch, dev, synth.C3, 5, 1, 0, stream),
            "c3_probe_estimation_split_bf16": plain_method_run(msp, torch, dev, synth.C3, 5, 1, 2, stream),
        }

        def versus(a, b):   # form b against the FP32 form a: final loss and time
            return {"final_loss_rel_diff": abs(pm[a]["loss_final"] - pm[b]["loss_final"]) / pm[a]["loss_final"],
                    "time_ratio_over_fp32": pm[b]["ms"] / pm[a]["ms"]}

        pm["c2_precise_vs_fp32"] = versus("c2_probe_estimation_fp32", "c2_probe_estimation_precise")
        pm["c2_double_float_vs_fp32"] = versus("c2_probe_estimation_fp32", "c2_probe_estimation_double_float")
        pm["c2_split_bf16_vs_fp32"] = versus("c2_probe_estimation_fp32", "c2_probe_estimation_split_bf16")
        pm["c3_split_bf16_vs_fp32"] = versus("c3_probe_estimation_fp32", "c3_probe_estimation_split_bf16")
        extra["plain_method"] = pm
        # the full 8-slice, 4096-position workload
        c3 = synth.C3
        g3, gd3, pos3, d_pos3, ws3, _, p3g, I3 = make_inputs(msp, torch, dev, c3)
        p3 = torch.from_numpy(p3g).to(dev)
        V3 = torch.zeros((c3.n_slices, c3.obj, c3.obj), dtype=torch.float32, device=dev)
        I3d = torch.from_numpy(I3).to(dev)
        msp.loss_grad(g3, p3, V3, d_pos3, I3d, ws=ws3)
        msp.profile_read(reset=True)
        msp.profile_enable(True)
        c3ms = time_events(lambda: msp.loss_grad(g3, p3, V3, d_pos3, I3d, ws=ws3), 5, stream, flush)
        p3p = msp.profile_read(reset=True)
        msp.profile_enable(False)
        k3 = p3p["fused_ms"] / 5
        extra["c3_full"] = {"workload": c3.name, "call": "msp_loss_grad", "ms": c3ms,
                            "value": c3.n_pos * c3.n_slices / (c3ms * 1e-3), "unit": UNIT, "fused_kernel_ms": k3,
                            "fused_kernel_tflops": fft_flops(c3.n_pos, c3.n_slices, c3.win) / (k3 * 1e-3) / 1e12}
        del ws3
        g3b = msp.geometry(**gd3, precision=msp.MSP_PRECISION_BF16X3_DFT)
        ws3b = msp.make_workspace(g3b, dev)
        msp.loss_grad(g3b, p3, V3, d_pos3, I3d, ws=ws3b)
        c3b = time_events(lambda: msp.loss_grad(g3b, p3, V3, d_pos3, I3d, ws=ws3b), 3, stream, flush)
        extra["c3_full"]["split_bf16_dft"] = {"ms": c3b, "value": c3.n_pos * c3.n_slices / (c3b * 1e-3),
                                              "cost_vs_fp32": c3b / c3ms}
        del ws3b
        extra["learned_proposal"] = learned_proposal_run(msp, torch, dev, stream, read_peaks())
    clocks = sampler.stop()
    clocks["window"] = "the timed steps and the measurements of this run that follow them"

    peaks = read_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12      # TFLOP/s: SMs x FP32 lanes x FMA x clock
    # the fused kernel's time per call (a call may run it in several position batches)
    fused_ms = prof["fused_ms"] / args.steps
    fused_launches_per_call = prof["fused_launches"] / args.steps
    achieved = fft_flops(S, L, W) / (fused_ms * 1e-3) / 1e12
    kname = "position_kernel<128, LOSS_GRAD>" if W == 128 else ("position_cluster_kernel<LOSS_GRAD>" if W == 256
                                                                 else f"position_kernel<{W}, LOSS_GRAD>")
    traffic = None
    if cfg is synth.C2:
        traffic = measured_traffic("position_kernel_loss_grad" + ("_l2_reduce" if args.overlap_add == "l2" else ""))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "call": "msp_loss_grad (loss, dV of every slice, dprobe)",
                   "positions": S, "slices": L, "window": W, "object": [cfg.obj, cfg.obj],
                   "state": "V = 0, probe guess (20 A defocus error), Poisson-noisy patterns",
                   "l2": "flushed between timed steps (256 MiB write outside the step events)",
                   "overlap_add": "l2_reduce" if args.overlap_add == "l2" else "fixed_order",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic,
                     "kernel": kname + " (fused fwd+adjoint)", "kernel_ms": fused_ms,
                     "kernel_launches_per_call": fused_launches_per_call,
                     "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(prof["all_launches"]),
        "clocks": clocks,
        "loss_timed_step": loss_step,
    }
    line.update(extra)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, pos, I_meas_h, p_guess)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_peaks(args):
    """The FP32 FFMA rate and the tcgen05 kind::tf32 MMA rate per shape, from the stand-alone
    micro-benchmarks in csrc/msp_peaks.cu: the figures the kernels' fractions are read against."""
    if args.impl == "reference" or int(os.environ.get("RANK", 0)) != 0:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the pipe micro-benchmarks have no reference arm"}))
        return
    from paper_2205_03902_gb300 import build as B
    import subprocess
    exe = B.build_peaks()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        raise SystemExit("msp_peaks failed: " + r.stdout + r.stderr)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    res.update({"metric": "compute pipe peaks", "unit": "TFLOP/s", "n_gpus": 1,
                "config": {"workload": "micro-benchmarks (FFMA: 8 CTAs x 256 threads per SM, 8 chains each; "
                                       "tf32 MMA: one CTA per SM, one thread issuing 768 MMAs)"},
                "nominal_fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
                "derived_tf32_tflops": float(peaks.get("bf16_tflops", 1900.0)) * 1.1 / 2.25})
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="msp", choices=["msp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="the timed loss/gradient steps and e2e only")
    ap.add_argument("--overlap-add", default="fixed", choices=["fixed", "l2"],
                    help="how msp_loss_grad sums the window gradients of the timed steps: fixed (a gather "
                         "in scan order, bit-reproducible; the default) or l2 (reductions in L2 from the "
                         "fused kernel)")
    ap.add_argument("--train-steps", type=int, default=1500, help="Adam steps of the learned proposal (learned_c5)")
    ap.add_argument("--config", default="c2",
                    choices=sorted(synth.CONFIGS) + sorted(synth.SMD_CONFIGS) + ["dft_c3", "peaks", "learned_c5"],
                    help="workload (default c2: W = 128, L = 4, S = 1024, the benchmark configuration; "
                         "smd_gaas: Algorithm 2 on the Table 1 setting; peaks: FFMA and tcgen05 tf32 "
                         "MMA micro-benchmarks; learned_c5: the learned-proposal form alone, with "
                         "--train-steps Adam steps)")
    args = ap.parse_args()
    global CFG
    smd = args.config in synth.SMD_CONFIGS
    if args.config == "peaks":
        run_peaks(args)
        return
    if args.config == "learned_c5":
        if args.impl == "reference" or int(os.environ.get("RANK", 0)) != 0:
            if args.impl == "reference":
                print(json.dumps({"impl": "reference", "unavailable": "the learned proposal has no reference arm"}))
            return
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_2205_03902_gb300 import msp
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        r = learned_proposal_run(msp, torch, dev, torch.cuda.current_stream(), read_peaks(),
                                 train_steps=args.train_steps)
        t = r["time_to_plain_final_loss"]
        print(json.dumps({"metric": "wall time to the plain method's final loss", "value": t["learned_ms_total"],
                          "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "bf16",
                          "data": "synthetic", "config": {"workload": r["workload"]}, **r}), flush=True)
        return
    if args.config == "dft_c3":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the DFT study has no reference arm; see --config c3"}))
            return
        run_dft(args, int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
                int(os.environ.get("LOCAL_RANK", 0)))
        return
    CFG = synth.SMD_CONFIGS[args.config] if smd else synth.CONFIGS[args.config]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        (run_smd_reference if smd else run_reference)(args, rank, world)
    else:
        (run_smd if smd else run_msp)(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
