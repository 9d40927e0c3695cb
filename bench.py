"""Throughput of the per-particle Lagrangian step on GB300.

Workload (one GPU): a 256^3 periodic grid with a seeded divergence-free random
Fourier field stored in FP32, 1e9 particles in the mixed-precision storage
(int32 cell + FP32 offset, FP32 velocity, FP32 diameter), dt = 5e-4, counting
sort every 10 steps.  A "step" is one pass of the whole hot path: the
counting sort when it is due (every 10th step), then gather, integrate,
relocate and deposit for every particle.  The particle state (32 GB) is far
larger than L2, so no flush is needed between steps.

Prints one JSON line.  With --impl reference the same metric is measured for
the FP64 CPU oracle on a bounded sample of the workload on the host cores.
Launch on N GPUs: python -m torch.distributed.run --nproc-per-node N bench.py
--gpus N (each rank runs its own replica of the workload: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 1e9 particles, % HBM roofline; mixed vs FP64 at fixed error"
UNIT = "particle-steps/s"
# algorithmic bytes per particle-step of the step kernel (read + write of the particle state)
STEP_BYTES = {"mixed_f32": 32 + 28, "mixed_bf16": 26 + 22, "fp64": 56 + 48}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per particle and launch of the sorted-step
# kernel at the workload's density, keyed by the SHA-256 of the kernel's source file; a kernel whose
# source has changed since has no measured traffic (null).  Counter captures run on small cases only
# (a few GB on the device), so the figure is derived from two of them at 24 and 60 particles per cell
# (128^3 / 5.0e7 and 64^3 / 1.6e7 particles): per particle the traffic is the state's bytes plus
# per-unit costs (fluid tile, deposit-tile flush) divided by the density, and a small capture misses
# the dirty lines still in L2 when the kernel ends.  Fitted: reads 32 + 120 / rho B, writes
# 28 + 99 / rho B with ~60 MB left in L2; at the 1e9 workload's 59.6 particles per cell, 63.7 B.
STEP_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2603_26691_gb300", "csrc",
                           "step_mixed_tma.cu")
MEASURED_TRAFFIC = {
    ("cc6fd6e7278a727c5c1b8648edf045fc9ea4547380736fa09847ca45e4fe51f8", "fourier256_mixed_1e9"): 63.7,
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_rate(workload, U, n_per_thread: int, budget_s: float, threads: int = 0, warmup: int = 0,
                 steps: int = 0):
    """The FP64 oracle, as it stands, on every host core: each thread steps its own seeded sample of
    the workload (n_per_thread particles, its own source field; the C oracle runs without the GIL) for
    `steps` steps, or until budget_s of wall time when steps = 0.  Returns (particle-steps/s, threads,
    steps per thread, seconds)."""
    import concurrent.futures as cf

    import oracle
    from paper_2603_26691_gb300 import inputs

    threads = threads or (os.cpu_count() or 1)
    N = workload.grid
    G = oracle.make_grid(N, chunk_edge=workload.chunk_edge)
    U = np.ascontiguousarray(U, dtype=np.float64)
    samples = []
    for t in range(threads):
        pos, vel, d, _ = inputs.particles(workload.seed, t * n_per_thread, n_per_thread)
        samples.append([pos, vel, d, np.zeros((3, N ** 3))])
    for smp in samples:
        for _ in range(warmup):
            smp[0], smp[1], _, _ = oracle.run(G, U, smp[0], smp[1], smp[2], 1, workload.dt, src=smp[3], inplace=True)

    def work(smp, t0):
        k = 0
        while (steps and k < steps) or (not steps and time.perf_counter() - t0 < budget_s):
            smp[0], smp[1], _, _ = oracle.run(G, U, smp[0], smp[1], smp[2], 1, workload.dt, src=smp[3], inplace=True)
            k += 1
        return k

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        done = list(ex.map(lambda smp: work(smp, t0), samples))
    el = time.perf_counter() - t0
    return n_per_thread * sum(done) / el, threads, min(done), el


def cpu_baseline(workload, U, budget_s: float = 15.0, n_per_thread: int = 20000):
    """The FP64 oracle, as it stands, on a bounded sample of the workload on every host core."""
    rate, threads, steps, el = _oracle_rate(workload, U, n_per_thread, budget_s)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{threads} threads x {n_per_thread} particles of the workload x >= {steps} steps each "
                      f"(own source field per thread), {el:.1f} s"}


def run_reference(args, workload):
    """The oracle arm: same metric, FP64 CPU oracle on every host core, a bounded sample per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    U = workload.make_field()
    threads = os.cpu_count() or 1
    n_per_thread = max(1, args.ref_sample // threads)
    rate, threads, steps, el = _oracle_rate(workload, U, n_per_thread, 0.0, threads=threads, warmup=args.warmup,
                                            steps=args.steps)
    n_sample = n_per_thread * threads
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles_per_step": n_sample,
                       "precision": "fp64 (CPU oracle)", "dt": workload.dt},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n_sample} particles of the workload per step on {threads} threads "
                                       f"({n_per_thread} each, own source field per thread)"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def setup_sim(workload, n, U32, precision, device, batch=50_000_000):
    import torch

    from paper_2603_26691_gb300 import inputs
    from paper_2603_26691_gb300.sim import Sim

    sim = Sim(workload.grid, precision=precision, chunk_edge=workload.chunk_edge, device=device)
    # the bench calls the sort itself (to time it apart) at the workload's cadence; the library is
    # told the same cadence so that the step before each sort leaves its output as records for the
    # sort's gather (the library never sorts on its own here: the bench's sort always comes first)
    sim.set_params(reorder_every=workload.reorder_every)
    sim.set_fluid(torch.as_tensor(U32, device=device))
    sim.reserve(n)
    q = inputs.lognormal_qtable()
    first = 0
    while first < n:
        cnt = min(batch, n - first)
        pos, vel, d, ids = sim.gen_particles(workload.seed, first, cnt, q, vmax=workload.vmax)
        sim.add_particles(pos, d, vel, ids)
        del pos, vel, d, ids
        first += cnt
    torch.cuda.synchronize()
    return sim


# physics variants timed beside the default step: the paper's own choices (nearest-grid-point
# gather, semi-implicit Euler, Schiller-Naumann drag, containing-cell deposit) and the
# cloud-in-cell deposit
VARIANTS = {
    "paper_ngp_semi_implicit_schiller_naumann": dict(gather="ngp", integrator="semi_implicit",
                                                     drag="schiller_naumann", deposit="cell"),
    "schiller_naumann": dict(drag="schiller_naumann"),
    "cic_deposit": dict(deposit="cic"),
}


def timed_steps(sim, steps, dt, reorder_every, step_index0):
    """Run `steps` steps with the sort every `reorder_every` steps; per-kernel CUDA events."""
    import torch

    ev = []
    for s in range(steps):
        idx = step_index0 + s
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sorted_now = reorder_every > 0 and idx % reorder_every == 0
        if sorted_now:
            sim.reorder()
        e1.record()
        sim.step(1, dt)
        e2.record()
        ev.append((e0, e1, e2, sorted_now))
    return ev


# FP64 operations per particle of one adjoint step launch (adjoint_step_kernel) and of one FP64
# step launch, from ncu instruction counters (2 x DFMA + DADD + DMUL, thread instructions) on the
# adjoint workload; keyed by the SHA-256 of the kernel source, absent (null) once it changes
MEASURED_FP64_OPS = {
    # ncu instruction counters: 116 DFMA + 46.8 DADD + 70 DMUL per particle; FP64 pipe 79 % busy
    # (the cell-deposit instance adjoint_step_kernel<false>)
    ("745faef8cafcc409ab81adaf96843ca26e35db7c534e64437178455cdd04f368", "adjoint_step_kernel"): 348.8,
    # step_f64_kernel: 56 DFMA + 59 DADD + 19 DMUL per particle (2e6 particles on 128^3)
    ("8fc2e56686bddc20dfeca2e836f247c15b1f3655db751a7a9f10af9a572c8820", "step_f64_kernel"): 190.0,
}
MEASURED_FP64_PIPE = {("745faef8cafcc409ab81adaf96843ca26e35db7c534e64437178455cdd04f368", "adjoint_step_kernel"): 0.794,
                      ("8fc2e56686bddc20dfeca2e836f247c15b1f3655db751a7a9f10af9a572c8820", "step_f64_kernel"): 0.858}
F64_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2603_26691_gb300", "csrc", "step_f64.cu")


def fp64_peak(sim):
    """This GPU's FP64 FMA rate, measured by the library's FMA-chain probe (else the nominal figure)."""
    try:
        return sim.probe_fma()[0], "measured (FP64 FMA-chain probe, st_probe_fma)"
    except Exception:  # noqa: BLE001 - an older library without the probe
        return FP64_NOMINAL_GFLOPS, "nominal GB300 dense FP64"


def fp64_step_roofline(n, ms, peak=None, peak_kind=None):
    """The FP64 step kernel against the FP64 rate (its operation count from ncu, by source)."""
    import hashlib

    with open(F64_SOURCE, "rb") as f:
        key = (hashlib.sha256(f.read()).hexdigest(), "step_f64_kernel")
    ops = MEASURED_FP64_OPS.get(key)
    ach = ops * n / (ms * 1e-3) / 1e9 if ops else None
    peak = peak or FP64_NOMINAL_GFLOPS
    return {"bound": "alu", "unit": "GFLOP/s (FP64)", "fp64_ops_per_particle": ops, "achieved": ach,
            "peak": peak, "peak_kind": peak_kind or "nominal GB300 dense FP64",
            "frac": ach / peak if ach else None, "fp64_pipe_busy_ncu": MEASURED_FP64_PIPE.get(key)}
ADJOINT_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2603_26691_gb300", "csrc",
                              "adjoint.cu")
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 dense FP64, the nominal figure (no measured FP64 peak on this machine)


def run_adjoint(args, workload):
    """The adjoint workload: FP64 forward with checkpoints, then the backward sweep (recomputation of
    each segment and the adjoint step), for a loss on the time-summed source field.  One JSON line:
    forward+backward particle-steps/s, with the library's kernel timers."""
    import hashlib

    import torch

    ws, rank, local = _dist()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    n = args.n or workload.n
    U = workload.make_field()
    U32 = U.astype(np.float32)
    sim = setup_sim(workload, n, U32, "fp64", device)
    sim.set_params(reorder_every=0)
    # generation order: the FP64 adjoint adds every dL/dU product exactly, and sorted particles would
    # send a warp's adds to the same words (measured 5.5 ms per launch sorted, 5.2 ms unsorted)
    steps, ck, dt = workload.steps, workload.extra["checkpoint"], workload.dt
    gen = torch.Generator(device=device)
    gen.manual_seed(7)
    lam = torch.randn((3, sim.ncell), generator=gen, dtype=torch.float64, device=device)
    # warm-up: W short forward/backward runs of one checkpoint segment
    for _ in range(max(args.warmup, 1)):
        sim.adjoint_forward(ck, dt, ck)
        sim.adjoint_backward(lam)
    torch.cuda.synchronize()
    sim.timers(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = sim.kernel_launches
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t2 = torch.cuda.Event(enable_timing=True)
    t0.record()
    sim.adjoint_forward(steps, dt, ck)
    t1.record()
    gd, ga, gU = sim.adjoint_backward(lam)
    t2.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = sim.kernel_launches - launches0
    tm = sim.timers()
    sim.timers(False)
    fwd_ms, bwd_ms = t0.elapsed_time(t1), t1.elapsed_time(t2)
    total_ms = fwd_ms + bwd_ms
    value = n * steps / (total_ms * 1e-3)
    adj_ms, adj_n = tm["adjoint"]
    stp_ms, stp_n = tm["step"]
    with open(ADJOINT_SOURCE, "rb") as f:
        src_hash = hashlib.sha256(f.read()).hexdigest()
    ops = MEASURED_FP64_OPS.get((src_hash, "adjoint_step_kernel"))
    adj_avg = adj_ms / max(adj_n, 1)
    achieved = ops * n / (adj_avg * 1e-3) / 1e9 if ops else None
    p64, p64_kind = fp64_peak(sim)
    roofline = {"bound": "alu", "kernel": "adjoint_step_kernel", "unit": "GFLOP/s (FP64)", "peak": p64,
                "peak_kind": p64_kind, "achieved": achieved,
                "frac": achieved / p64 if achieved else None, "traffic": None,
                "fp64_ops_per_particle": ops, "launches": adj_n, "ms_per_launch": adj_avg,
                "fp64_pipe_busy_ncu": MEASURED_FP64_PIPE.get((src_hash, "adjoint_step_kernel")),
                "step_f64_kernel": {"launches": stp_n, "ms_per_launch": stp_ms / max(stp_n, 1)}}
    # end to end through the public API with host buffers: lam from host memory, the gradients to host
    lam_h = lam.cpu().numpy()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    sim.adjoint_forward(steps, dt, ck)
    hgd, hga, hgU = sim.adjoint_backward(lam_h)
    e_el = time.perf_counter() - e0
    e2e = {"value": n * steps / e_el, "unit": "particle-steps/s", "h2d_bytes_per_step": int(lam_h.nbytes),
           "d2h_bytes_per_step": int(hgd.nbytes + hgU.nbytes), "steps": 1,
           "what": "one forward (checkpointed) + backward run, lam from host, dL/dd and dL/dU to host"}
    # the same run through the cloud-in-cell deposit (the adjoint step kernel's second instance,
    # which differentiates the deposit weights too)
    sim.set_physics(deposit="cic")
    sim.timers(True)
    c0e, c1e, c2e = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0e.record()
    sim.adjoint_forward(steps, dt, ck)
    c1e.record()
    sim.adjoint_backward(lam)
    c2e.record()
    torch.cuda.synchronize()
    tmc = sim.timers()
    sim.timers(False)
    sim.set_physics()
    # ids in storage order (no run reorders), to compare per-particle gradients across handles by id
    ids64 = sim.particles(host=False)[3].long()
    cf_ms, cb_ms = c0e.elapsed_time(c1e), c1e.elapsed_time(c2e)
    cic = {"forward_ms": cf_ms, "backward_ms": cb_ms, "particle_steps_per_s": n * steps / ((cf_ms + cb_ms) * 1e-3),
           "adjoint_kernel_ms_per_launch": tmc["adjoint"][0] / max(tmc["adjoint"][1], 1),
           "step_kernel_ms_per_launch": tmc["step"][0] / max(tmc["step"][1], 1)}
    sim.close()
    # the same workload on a mixed FP32-velocity handle: the FP32 adjoint (general mixed step forward,
    # FP32 reverse step), its gradients compared with the FP64 run's
    sim32 = setup_sim(workload, n, U32, "mixed_f32", device)
    sim32.set_params(reorder_every=0)
    # sorted by cell once, before any recorded run (the recorded runs keep their storage order): the
    # particles of a warp then share stencils, and the FP32 adjoint sums their dL/dU products per
    # stencil before the exact adds (2.4 -> 0.94 ms per launch at 1e7)
    sim32.reorder()
    # the same warm-up runs as the FP64 handle's, so that both timed runs start from the same state
    # (up to the FP32 rounding of the mixed handle)
    for _ in range(max(args.warmup, 1)):
        sim32.adjoint_forward(ck, dt, ck)
        sim32.adjoint_backward(lam)
    torch.cuda.synchronize()
    sim32.timers(True)
    f0e, f1e, f2e = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    f0e.record()
    sim32.adjoint_forward(steps, dt, ck)
    f1e.record()
    gd32, ga32, gU32 = sim32.adjoint_backward(lam)
    f2e.record()
    torch.cuda.synchronize()
    tmf = sim32.timers()
    sim32.timers(False)
    ids32 = sim32.particles(host=False)[3].long()
    sim32.close()
    # the handles keep different storage orders: dL/dd compared by particle id
    gd_id, gd32_id = torch.empty_like(gd), torch.empty_like(gd)
    gd_id[ids64] = gd
    gd32_id[ids32] = gd32
    ff_ms, fb_ms = f0e.elapsed_time(f1e), f1e.elapsed_time(f2e)
    fp32 = {"forward_ms": ff_ms, "backward_ms": fb_ms, "particle_steps_per_s": n * steps / ((ff_ms + fb_ms) * 1e-3),
            "adjoint_kernel_ms_per_launch": tmf["adjoint"][0] / max(tmf["adjoint"][1], 1),
            "step_kernel_ms_per_launch": tmf["step"][0] / max(tmf["step"][1], 1),
            "grad_alpha_rel_diff_to_fp64": abs(ga32 - ga) / abs(ga),
            "grad_U_rel_l2_diff_to_fp64": float((torch.linalg.vector_norm(gU32 - gU) / torch.linalg.vector_norm(gU)).item()),
            "grad_d_rel_l2_diff_to_fp64": float((torch.linalg.vector_norm(gd32_id - gd_id) / torch.linalg.vector_norm(gd)).item()),
            "grad_d_compared_by_id": True}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        from paper_2603_26691_gb300 import inputs

        ns = 200_000  # about 9 s of oracle time (~4.7e6 particle-steps/s)
        G = oracle.make_grid(workload.grid, chunk_edge=workload.chunk_edge)
        pos, vel, d, _ = inputs.particles(workload.seed, 0, ns)
        c0 = time.perf_counter()
        oracle.adjoint(G, U, pos, vel, d, steps, dt, lam_h)
        c_el = time.perf_counter() - c0
        cpu = {"value": ns * steps / c_el, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{ns} particles x {steps} steps, forward and adjoint (single thread), {c_el:.1f} s"}
    line = {"metric": "adjoint particle-steps/s (forward with checkpoints + backward with recomputation)",
            "value": value, "unit": "particle-steps/s", "n_gpus": ws, "steps": steps, "warmup": max(args.warmup, 1),
            "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles_per_gpu": n, "dt": dt,
                       "checkpoint_every": ck, "field": "Taylor-Green + 10% random Fourier, FP32-rounded",
                       "l2": "no flush: 56 B x particles of state per step, far larger than L2",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "breakdown": {"forward_ms": fwd_ms, "backward_ms": bwd_ms, "timers": tm,
                          "grad_alpha": ga, "grad_d_norm": float(torch.linalg.vector_norm(gd).item()),
                          "cic_deposit": cic, "fp32_adjoint": fp32}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_coupled(args, workload):
    """The asynchronous two-way coupling workload: K particle steps per coupling interval in a frozen
    field, each interval's fluid update (estimated source + Jacobi sweeps) ahead of its steps.  One JSON
    line: coupled particle-steps/s, beside the same particles' uncoupled step time."""
    import torch

    ws, rank, local = _dist()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    n = args.n or workload.n
    K = workload.extra["fluid_every"]
    U32 = workload.make_field().astype(np.float32)
    sim = setup_sim(workload, n, U32, workload.precision, device)
    warm = max(1, -(-args.warmup // K))
    timed = max(1, args.steps // K)
    R = workload.reorder_every
    # the same particles stepped without the fluid update first: sorted, warm-up steps, then the
    # timed steps with a sort every R steps counted from that sort (as the coupled run below)
    sim.reorder()
    timed_steps(sim, warm * K, workload.dt, 0, 0)
    ev = timed_steps(sim, K * timed, workload.dt, R, warm * K)
    torch.cuda.synchronize()
    plain_ms = sum(e0.elapsed_time(e2) for (e0, e1, e2, _) in ev)
    # the coupled run: sorted again, then the library sorts every R steps itself
    sim.reorder()
    sim.set_params(reorder_every=R)
    sim.couple_params(rho_f=1.2, nu=workload.extra["nu"], sweeps=10, steps_per_interval=K, extrapolator="zero")
    sim.couple_run(warm, workload.dt)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    launches0 = sim.kernel_launches
    a.record()
    sim.couple_run(timed, workload.dt)
    b.record()
    torch.cuda.synchronize()
    launches = sim.kernel_launches - launches0
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    sim.close()
    steps = K * timed
    line = {"metric": "particle-steps/s, asynchronous two-way coupling (fluid update from lagged sources)",
            "value": n * steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm * K,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles_per_gpu": n,
                       "chunk_edge": workload.chunk_edge, "steps_per_interval": K, "nu": workload.extra["nu"],
                       "jacobi_sweeps": 10, "rho_f": 1.2, "extrapolator": "zero", "dt": workload.dt,
                       "reorder_every": workload.reorder_every},
            "uncoupled_ms_per_step": plain_ms / steps,
            "coupling_overhead": ms / plain_ms - 1.0,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# algorithmic bytes per particle-step of the microphysics step on mixed handles: the step kernel's state
# (cell 4, offsets 12, velocity 12, diameter 4) plus the compensated temperature and diameter residual
# (16), read and written
MICRO_BYTES = {"mixed_f32": 2 * (32 + 16), "mixed_bf16": 2 * (26 + 16)}


def run_micro(args, workload):
    """Droplet microphysics (vapour mass and heat transfer, paper Sec. 2.1) on the mixed-precision workload:
    the same particles and velocity field plus seeded fluid temperature and vapour fields; one JSON line with
    particle-steps/s, the microphysics kernel's HBM roofline and the bytes it adds per particle-step."""
    import torch

    from paper_2603_26691_gb300 import inputs

    ws, rank, local = _dist()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    n = args.n or workload.n
    precision = args.precision or workload.precision
    U32 = workload.make_field().astype(np.float32)
    T, rv = inputs.thermo_fields(workload.grid, seed=workload.field_seed + 1)
    sim = setup_sim(workload, n, U32, precision, device)
    sim.set_thermo(T, rv)
    sim.set_microphysics(True, T_init=285.0)
    R = workload.reorder_every
    W, K = max(args.warmup, 3), args.steps
    for _ in timed_steps(sim, W, workload.dt, R, 0):
        pass
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = sim.kernel_launches
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    evs = timed_steps(sim, K, workload.dt, R, W)
    b.record()
    torch.cuda.synchronize()
    launches = sim.kernel_launches - launches0
    clk = clocks.stop()
    total_ms = a.elapsed_time(b)
    step_ms = [e1.elapsed_time(e2) for (e0, e1, e2, _) in evs]
    sort_ms = [e0.elapsed_time(e1) for (e0, e1, e2, s_) in evs if s_]
    avg = sum(step_ms) / len(step_ms)
    peak, peak_kind = _peaks()
    mb = MICRO_BYTES[precision]
    achieved = mb * n / (avg * 1e-3) / 1e9
    W0, E0 = sim.micro_invariants()
    msrc = sim.micro_sources()
    sim.close()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        ns = 20000
        G = oracle.make_grid(workload.grid, chunk_edge=workload.chunk_edge)
        M = oracle.make_micro()
        pos, vel, d, _ = inputs.particles(workload.seed, 0, ns)
        Tp = np.full(ns, 285.0)
        Ud = U32.astype(np.float64).reshape(-1, 3)
        c0 = time.perf_counter()
        steps = 0
        while time.perf_counter() - c0 < args.cpu_budget:
            pos, vel, d, Tp, _, _, _ = oracle.micro_run(G, M, Ud, T.reshape(-1), rv.reshape(-1), pos, vel, d, Tp, 1,
                                                        workload.dt)
            steps += 1
        el = time.perf_counter() - c0
        cpu = {"value": ns * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{ns} particles of the workload x {steps} microphysics steps (single thread), {el:.1f} s"}
    line = {"metric": "particle-steps/s with droplet microphysics (vapour mass and heat transfer)",
            "value": n * K / (total_ms * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles_per_gpu": n, "precision": precision,
                       "dt": workload.dt, "reorder_every": R,
                       "thermo": "T 285 +- 3 K, rho_v 0.0105 kg/m^3 +- 5 % (seeded random Fourier fields)",
                       "l2": "no flush: 48 B x particles of state per step, far larger than L2"},
            "roofline": {"bound": "hbm", "kernel": "micro_mixed_kernel", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_particle_step": mb,
                         "added_bytes_per_particle_step": mb - STEP_BYTES[precision], "step_kernel_ms": avg},
            "breakdown": {"sort_ms_avg": (sum(sort_ms) / len(sort_ms)) if sort_ms else None,
                          "step_kernel_ms": [round(x, 3) for x in step_ms],
                          "water_in_droplets_kg": W0, "vapour_gained_kg": float(msrc[0].sum()),
                          "energy_gained_J": float(msrc[1].sum())},
            "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_chunks(args, workload):
    """Chunk-by-chunk streaming (paper Sec. 2.2): the particle set lives in pinned host memory as chunks,
    each pass uploads, sorts and steps and downloads every chunk, copies overlapping computation.  One
    JSON line: particle-steps/s of a pass of `--steps` steps (after a one-step pass that sorts each chunk
    from generation order), with the pass's copy and compute times from the library's CUDA events."""
    import torch

    ws, rank, local = _dist()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    from paper_2603_26691_gb300 import inputs
    from paper_2603_26691_gb300.sim import Sim

    n = args.n or workload.n
    C = args.chunk or workload.extra["chunk"]
    U32 = workload.make_field().astype(np.float32)
    sim = Sim(workload.grid, precision=workload.precision, chunk_edge=workload.chunk_edge, device=device)
    sim.set_params(reorder_every=workload.reorder_every)
    sim.set_fluid(torch.as_tensor(U32, device=device))
    sim.chunks_create(C)
    q = inputs.lognormal_qtable()
    for first in range(0, n, C):
        cnt = min(C, n - first)
        pos, vel, d, _ = sim.gen_particles(workload.seed, first, cnt, q, vmax=workload.vmax)
        sim.chunks_add(pos, d, vel)
        del pos, vel, d
    torch.cuda.synchronize()
    warm = sim.chunks_step(1, workload.dt)  # every chunk sorted once from generation order
    K = args.steps
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = sim.kernel_launches
    t0 = time.perf_counter()
    ms = sim.chunks_step(K, workload.dt)
    host_s = time.perf_counter() - t0
    launches = sim.kernel_launches - launches0
    clk = clocks.stop()
    nchunks = sim.chunks_count()[1]
    sim.close()
    state_b = 36  # 32 B of mixed FP32 state + the id per particle, each way per pass
    value = n * K / (ms["wall_ms"] * 1e-3)
    line = {"metric": "particle-steps/s, particle set streamed chunk by chunk from pinned host memory",
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": 1, "ms_per_step": ms["wall_ms"] / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles": n, "chunk_particles": C,
                       "chunks": nchunks, "dt": workload.dt, "reorder_every": workload.reorder_every,
                       "l2": "no flush: the chunks (9 GB each) are far larger than L2"},
            "e2e": {"value": n * K / host_s, "unit": UNIT, "h2d_bytes_per_step": n * state_b // K,
                    "d2h_bytes_per_step": n * state_b // K, "steps": K,
                    "what": "one pass: every chunk uploaded from pinned host memory, stepped, downloaded"},
            "breakdown": {"pass": ms, "first_pass_one_step": warm,
                          "host_link_gb_per_s": {"h2d": n * state_b / (ms["h2d_ms"] * 1e-3) / 1e9,
                                                 "d2h": n * state_b / (ms["d2h_ms"] * 1e-3) / 1e9}},
            "roofline": None, "cpu_baseline": None, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fourier256_mixed_1e9")
    ap.add_argument("--n", type=int, default=None, help="particles per GPU (default: the workload's)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--grid", type=int, default=None, help="cells per axis (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--fp64-n", type=int, default=None, help="particles for the FP64-step comparison (0 = skip)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chunk", type=int, default=None, help="particles per chunk (chunk-streaming workload)")
    ap.add_argument("--variant-steps", type=int, default=3, help="steps per physics variant (0 = skip)")
    args = ap.parse_args()

    from paper_2603_26691_gb300 import inputs

    workload = inputs.WORKLOADS[args.workload]
    if args.grid:
        import dataclasses

        workload = dataclasses.replace(workload, grid=args.grid)
    if args.impl == "reference":
        return run_reference(args, workload)
    if workload.extra and workload.extra.get("checkpoint"):
        return run_adjoint(args, workload)
    if workload.extra and workload.extra.get("fluid_every"):
        return run_coupled(args, workload)
    if workload.extra and workload.extra.get("micro"):
        return run_micro(args, workload)
    if workload.extra and workload.extra.get("chunk"):
        return run_chunks(args, workload)

    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    precision = args.precision or workload.precision
    n = args.n or workload.n
    K, W = args.steps, args.warmup
    assert W >= 3, "at least 3 warm-up steps"
    U = workload.make_field()
    U32 = U.astype(np.float32)

    sim = setup_sim(workload, n, U32, precision, device)
    dt = workload.dt
    reorder_every = workload.reorder_every
    # warm-up (sorts at step 0, 10, ... as in the timed region)
    for ev in timed_steps(sim, W, dt, reorder_every, 0):
        pass
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    clocks.start()
    time.sleep(0.3)
    launches0 = sim.kernel_launches
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    evs = timed_steps(sim, K, dt, reorder_every, W)
    t_end.record()
    torch.cuda.synchronize()
    launches = sim.kernel_launches - launches0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [e1.elapsed_time(e2) for (e0, e1, e2, _) in evs]
    sort_ms = [e0.elapsed_time(e1) for (e0, e1, e2, s) in evs if s]
    t_max = total_ms
    if ws > 1:
        t = torch.tensor([total_ms], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    value = n * ws * K / (t_max * 1e-3)

    peak, peak_kind = _peaks()
    # the step just before each sort runs the record-writing instance of the step kernel (its
    # output as 32-byte records for the sort's gather: the state read, 36 B written); the others
    # run the plain instance, the dominant kernel that the roofline below is for
    rec_step = [precision != "fp64" and reorder_every > 0 and (W + i + 1) % reorder_every == 0
                for i in range(K)]
    rec_bytes = {"mixed_f32": 68, "mixed_bf16": 62}.get(precision)  # read the state, write cells + records
    # the first step after each sort that followed a record-writing step gathers the records through
    # the sort's permutation itself (the gathering instance): read permutation, record and id (40 B),
    # write the state with diameters and the id (36 B; 30 B with BF16 velocities)
    gat_step = [precision != "fp64" and reorder_every > 1 and (W + i) % reorder_every == 0 and W + i > 0
                for i in range(K)]
    gat_bytes = {"mixed_f32": 76, "mixed_bf16": 70}.get(precision)
    plain_ms = [t for t, r, g in zip(step_ms, rec_step, gat_step) if not r and not g] or step_ms
    rec_ms = [t for t, r in zip(step_ms, rec_step) if r]
    gat_ms = [t for t, g in zip(step_ms, gat_step) if g]
    step_all_avg = sum(step_ms) / len(step_ms)
    step_avg = sum(plain_ms) / len(plain_ms)
    bytes_per_launch = STEP_BYTES[precision] * n
    achieved = bytes_per_launch / (step_avg * 1e-3) / 1e9
    traffic = None
    if precision != "fp64":
        import hashlib

        with open(STEP_SOURCE, "rb") as f:
            m = MEASURED_TRAFFIC.get((hashlib.sha256(f.read()).hexdigest(), workload.name))
        if m is not None:
            traffic = m * n
    kname = "step_f64_kernel" if precision == "fp64" else "step_mixed_tma_kernel (plain instance)"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                # the same kernel's measured DRAM bytes (ncu, this source) at the measured rate
                "frac_of_measured_traffic": (traffic / (step_avg * 1e-3) / 1e9 / peak) if traffic else None,
                "kernel": kname, "launches": len(plain_ms),
                "algorithmic_bytes_per_particle_step": STEP_BYTES[precision], "peak_kind": peak_kind,
                "step_kernel_ms": step_avg,
                "all_steps": {"step_kernel_ms_avg": step_all_avg,
                              "frac": bytes_per_launch / (step_all_avg * 1e-3) / 1e9 / peak},
                "record_steps": {"launches": len(rec_ms),
                                 "step_kernel_ms_avg": (sum(rec_ms) / len(rec_ms)) if rec_ms else None,
                                 "bytes_per_particle": rec_bytes,
                                 "frac": (rec_bytes * n / (sum(rec_ms) / len(rec_ms) * 1e-3) / 1e9 / peak)
                                 if rec_ms else None},
                "gathering_steps": {"launches": len(gat_ms),
                                    "step_kernel_ms_avg": (sum(gat_ms) / len(gat_ms)) if gat_ms else None,
                                    "bytes_per_particle": gat_bytes,
                                    "frac": (gat_bytes * n / (sum(gat_ms) / len(gat_ms) * 1e-3) / 1e9 / peak)
                                    if gat_ms else None}}

    if precision == "fp64":  # the FP64 step is bound by FP64 arithmetic, not by HBM
        roofline = dict(fp64_step_roofline(n, step_avg, *fp64_peak(sim)), kernel="step_f64_kernel", launches=len(step_ms),
                        step_kernel_ms=step_avg, hbm_frac_of_algorithmic=achieved / peak)

    # per-chunk bounding boxes of the sorted state (on demand: one read of cells and offsets)
    sim.reorder()
    cb0 = torch.cuda.Event(enable_timing=True)
    cb1 = torch.cuda.Event(enable_timing=True)
    cb0.record()
    sim.chunk_bounds()
    cb1.record()
    torch.cuda.synchronize()
    chunk_bounds_ms = cb0.elapsed_time(cb1)

    # end to end through the C ABI with host buffers: each step receives the fluid field from
    # pinned host memory and returns the per-cell sources to pinned host memory (two buffers in
    # turn, as a consumer of the results would use them), the transfers queued with the asynchronous
    # calls so that they overlap the steps, the sorts left to the library's own schedule (inside
    # st_step); the timed region ends when the last sources are in host memory.  One untimed pass of
    # the same loop first (staging buffers, first use of the transfer kernels).  Few pinned buffers:
    # with twenty, after a long test run in the same box, some of them took device -> host copies at
    # 20 GB/s instead of 193
    Uh = torch.from_numpy(U32).pin_memory()
    E = args.e2e_steps
    src_h = [torch.empty((3, sim.ncell), dtype=torch.float64).pin_memory() for _ in range(2)]
    import ctypes as C

    lib = sim.lib

    # events on the compute stream around each step's work there (step, sort when due, source
    # conversion and reset): their span against the host clock shows whether the loop kept the GPU busy
    evs_e2e = []

    def e2e_loop(asynchronous):
        evs_e2e.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if asynchronous and E > 0:
            sim.set_fluid_async(Uh)
        for s in range(E):
            if not asynchronous:
                sim._chk(lib.st_set_fluid(sim.h, C.c_void_p(Uh.data_ptr()), 0, 0), "st_set_fluid")
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record()
            sim.step(1, dt)
            if asynchronous:
                # the next step's field is queued before this step's sources: its upload then never
                # waits behind their download where both directions share a copy engine
                if s + 1 < E:
                    sim.set_fluid_async(Uh)
                sim.sources_async(src_h[s % 2], reset=True)
                eb.record()
            else:
                sim._chk(lib.st_get_sources(sim.h, C.c_void_p(src_h[s % 2].data_ptr()), 1, 0), "st_get_sources")
                eb.record()
            evs_e2e.append((ea, eb))
        sim.synchronize()
        return max(time.perf_counter() - t0, 1e-9)

    def e2e_stream_ms():
        if not evs_e2e:
            return None
        busy = sum(a.elapsed_time(b) for a, b in evs_e2e) / len(evs_e2e)
        span = evs_e2e[0][0].elapsed_time(evs_e2e[-1][1]) / len(evs_e2e)
        return {"span_per_step": span, "step_and_conversion_per_step": busy}

    torch.cuda.synchronize()
    e2e_loop(True)
    if ws > 1:
        torch.distributed.barrier()
    e_el = e2e_loop(True)
    e_stream = e2e_stream_ms()
    # the same loop with the synchronous calls (each waits for its copy), for comparison
    if ws > 1:
        torch.distributed.barrier()
    s_el = e2e_loop(False)
    s_stream = e2e_stream_ms()
    if ws > 1:  # the whole job's time: the slowest rank's
        t = torch.tensor([e_el, s_el], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e_el, s_el = float(t[0].item()), float(t[1].item())
    # this machine's host link for the same buffers (one copy each way, CUDA events): the end-to-end rate
    # depends on it, and it differs between boxes of the pool
    link = {}
    if E > 0:
        dU = torch.empty(Uh.shape, dtype=Uh.dtype, device=device)
        dS = torch.empty(src_h[0].shape, dtype=torch.float64, device=device)
        for name, dst, src_t in (("h2d_gbs", dU, Uh), ("d2h_gbs", src_h[0], dS)):
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            dst.copy_(src_t, non_blocking=True)
            ea.record()
            dst.copy_(src_t, non_blocking=True)
            eb.record()
            torch.cuda.synchronize()
            link[name] = src_t.numel() * src_t.element_size() / (ea.elapsed_time(eb) * 1e-3) / 1e9
        # and into every one of the loop's host buffers (pinned memory can land on a slower node)
        rates = []
        for b in src_h:
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record()
            b.copy_(dS, non_blocking=True)
            eb.record()
            torch.cuda.synchronize()
            rates.append(b.numel() * 8 / (ea.elapsed_time(eb) * 1e-3) / 1e9)
        link["d2h_gbs_each_buffer_min_max"] = [min(rates), max(rates)]
        del dU, dS
    e2e = {"value": n * ws * E / e_el if E > 0 else None, "unit": UNIT, "h2d_bytes_per_step": int(U32.nbytes),
           "d2h_bytes_per_step": int(src_h[0].numel() * 8), "steps": E,
           "what": "per step: fluid field H2D from pinned host, step (sort when due), sources D2H to pinned host, "
                   "queued with st_set_fluid_async / st_get_sources_async and overlapping the steps",
           "synchronous_calls_value": n * ws * E / s_el if E > 0 else None, "host_link": link,
           "wall_ms_per_step": e_el * 1e3 / E if E > 0 else None, "compute_stream_ms": e_stream,
           "synchronous_compute_stream_ms": s_stream}

    # physics variants on the same particles, sorted: the sorted-particle step kernel's physics
    # instance
    variants = None
    if args.variant_steps > 0:
        variants = {}
        for name, ph in VARIANTS.items():
            sim.set_physics(**ph)
            sim.reorder()
            sim.step(1, dt)
            ev = timed_steps(sim, args.variant_steps, dt, 0, 1)
            torch.cuda.synchronize()
            ms = sum(e1.elapsed_time(e2) for (e0, e1, e2, _) in ev) / len(ev)
            variants[name] = {"physics": ph, "step_kernel_ms": ms, "particle_steps_per_s": n / (ms * 1e-3),
                              "hbm_frac_of_algorithmic": STEP_BYTES[precision] * n / (ms * 1e-3) / 1e9 / peak,
                              "kernel": "step_mixed_tma_kernel (physics instance)"}
        sim.set_physics()
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # FP64 GPU step on the same workload, for the mixed-vs-FP64 comparison
    fp64 = None
    fp64_n = n if args.fp64_n is None else args.fp64_n
    if fp64_n > 0 and precision != "fp64":
        s64 = setup_sim(workload, fp64_n, U32, "fp64", device)
        for _ in timed_steps(s64, 1, dt, reorder_every, 0):
            pass
        torch.cuda.synchronize()
        ev64 = timed_steps(s64, args.fp64_steps, dt, 0, 1)
        torch.cuda.synchronize()
        ms64 = sum(e1.elapsed_time(e2) for (e0, e1, e2, _) in ev64) / len(ev64)
        p64, p64_kind = fp64_peak(s64)
        rate64 = fp64_n / (ms64 * 1e-3)
        fp64 = {"particles": fp64_n, "step_kernel_ms": ms64, "particle_steps_per_s": rate64,
                "mixed_step_kernel_particle_steps_per_s": n / (step_avg * 1e-3),
                "speedup_mixed_over_fp64_step_kernel": (n / (step_avg * 1e-3)) / rate64,
                "bound": "alu (FP64)", "roofline": fp64_step_roofline(fp64_n, ms64, p64, p64_kind)}
        s64.close()
        del s64
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(workload, U32.astype(np.float64), budget_s=args.cpu_budget)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": workload.name, "grid": workload.grid, "particles_per_gpu": n,
                       "precision": precision, "dt": dt, "reorder_every": reorder_every,
                       "chunk_edge": workload.chunk_edge, "field": "divergence-free random Fourier, k<=8, rms 1",
                       "l2": "no flush: 32 B x particles of state per step, far larger than L2",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "breakdown": {"step_kernel_ms_avg": step_all_avg, "sort_ms_avg": (sum(sort_ms) / len(sort_ms)) if sort_ms else None,
                          "step_kernel_ms": [round(x, 3) for x in step_ms],
                          "sorts_in_timed_region": len(sort_ms),
                          "chunk_bounds_ms": chunk_bounds_ms},
            "fp64_step": fp64, "physics_variants": variants}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
