"""Benchmark of the fused stream-collide step (site-population updates/s).

Workload (one "step" = one predictor-corrector time step over the whole grid):
256 x 256 transverse grid, dx = 0.1 fm, 8 x 8 x 12 = 768-node momentum lattice,
FP32 populations (Landau matching / EOS inversion with FP64 refinement), eta/s = 0.16,
dtau = 0.0036 fm/c from tau = 0.4 fm/c, 40 seeded Gaussian hotspots (0.4 fm,
Exp(20 GeV/fm^3), N(0, 3 fm)) on a 10 GeV/fm^3 background.
The two population arrays (402 MB) exceed the 126 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank runs an independent replica of the workload
(the single-grid step has no multi-GPU decomposition here): weak scaling.
--impl reference times the FP64 CPU oracle on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 256
ETA_S, TAU0, DTAU, DX = 0.16, 0.4, 0.0036, 0.1
# the time steps of the other workloads, each over tau 0.4 -> 4 fm/c in its
# stated number of steps: batch 200, adjoint 300, precision sweep 500
DTAU_BATCH, DTAU_ADJ, DTAU_SWEEP = 3.6 / 200, 3.6 / 300, 3.6 / 500
WORKLOAD = ("rlb-milne-2+1d 256x256 grid dx 0.1 fm, 768 nodes (8xi x 8theta x 12phi), FP32 "
            "populations, 40 hotspots on 10 GeV/fm^3")



RECORD = None  # --record PATH: every JSON line is also appended there (JSONL)


def emit(line: dict):
    """Print the benchmark's JSON line (and append it to the run record)."""
    text = json.dumps(line)
    print(text, flush=True)
    if RECORD:
        with open(RECORD, "a") as fh:
            fh.write(text + "\n")


class Ranks:
    """One process per GPU (torchrun): rank and world size from the
    environment, a process group when there is more than one rank, a barrier,
    and the maximum of a host number over ranks (the timed region of the
    slowest rank).  The replicas exchange nothing else."""

    def __init__(self, backend: str = "nccl"):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float, device: str = "cuda") -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def job_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput of weak scaling: every rank processes the same
    number of units, the job takes as long as the slowest rank."""
    return world * units_per_rank / t_max


# DRAM traffic of the stage kernel on the 256 x 256 workload: ncu
# dram__bytes_read.sum + dram__bytes_write.sum, mean of one predictor and one
# corrector launch of `bench.py --steps 3 --warmup 3 --no-cpu-baseline --no-e2e
# --no-secondary` on a GB300 (the mirror-paired kernel, the default).  It
# describes the kernel sources it was taken on (the SHA-1 of the code of the
# stage-kernel headers, comments removed) and is reported only while they are
# unchanged.
STAGE_TRAFFIC = {"sources": ("rlb_stage_mp.cuh", "rlb_stage_x2.cuh", "rlb_kernels.cuh"),
                 "sha1": "58dca9d88d17d4433154fd976ca57735f83fd842", "bytes_per_launch": 479.79e6}


def code_digest(files) -> str:
    """SHA-1 of the code of the given kernel sources with comments and
    whitespace runs removed (a comment edit does not change the kernel)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1108_5561_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()


def stage_traffic(grid: int):
    """Measured DRAM bytes per stage launch, or None (other grid, changed kernel)."""
    if grid != 256:
        return None
    ok = code_digest(STAGE_TRAFFIC["sources"]) == STAGE_TRAFFIC["sha1"]
    return STAGE_TRAFFIC["bytes_per_launch"] if ok else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if device_id:
                cmd += ["-i", device_id]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def oracle_rate(eps_window, steps, nthreads):
    """Oracle (FP64 CPU) updates/s on a window of the workload."""
    from oracle.oracle import Oracle
    ny, nx = eps_window.shape
    o = Oracle(nx=nx, ny=ny, dx=DX, eta_over_s=ETA_S)
    f, lnM = o.init_state(eps_window, nthreads)
    t0 = time.perf_counter()
    o.step(f, lnM, TAU0, DTAU, steps, nthreads)
    dt = time.perf_counter() - t0
    return nx * ny * o.nn * steps / dt, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    from paper_1108_5561_gb300.inputs import hotspots
    eps0, _, _ = hotspots(NX, NY, n=40, seed=1108)
    c = NX // 2
    win = eps0[c - 8:c + 8, c - 8:c + 8]  # 16 x 16 sample per step
    cores = os.cpu_count() or 1
    rate, dt = oracle_rate(win, args.warmup + args.steps, cores)
    line = {
        "impl": "reference", "metric": "site-population updates/s", "value": rate,
        "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / (args.warmup + args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision_of_oracle": "f64", "grid": [NX, NY],
                   "nodes_per_site": 768},
        "cpu_baseline": {"value": rate, "unit": "updates/s", "cores": cores, "kind": "oracle",
                         "sample": "16x16 central window of the 256x256 workload, one oracle "
                                   "step per benchmark step"},
        "e2e": {"value": rate, "unit": "updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    emit(line)
    return 0


BATCH_EVENTS, BATCH_EVOLUTION_STEPS = 512, 200


def batch_main(args, rank, world, local):
    """Batched events (512 events, sides U{64..192}, eta/s U(0.04, 0.3), 40
    hotspots each, FP32, 768 nodes): batched events/s = events whose full
    200-step evolution (tau 0.4 -> 1.12 fm/c at dtau 0.0036) completes per
    second, from the timed steps of the whole batch.  One launch per kernel per
    stage for all events, each step replayed as a CUDA graph, stage-kernel
    variant chosen by the autotuner on the batch."""
    import torch
    import paper_1108_5561_gb300 as rlb
    from paper_1108_5561_gb300.inputs import batch_events, hotspots

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    ranks = Ranks("nccl")
    evs = batch_events(BATCH_EVENTS, seed=1108)
    events = [rlb.Event(n, n, eta) for n, eta in evs]
    eps = np.concatenate([hotspots(n, n, n=40, seed=1108 + i)[0].reshape(-1) for i, (n, _) in enumerate(evs)])
    g = rlb.GridParams(dx=DX, prec=rlb.RLB_F32, tau0=TAU0, dtau=DTAU_BATCH)
    run = rlb.Run(g, device=local, events=events)
    run.init_grid(eps)
    run.step(1)
    chosen, tune_ms = run.autotune()
    run.step(args.warmup - 1)
    torch.cuda.synchronize()
    run.check()

    barrier = ranks.barrier

    props = torch.cuda.get_device_properties(local)
    dev_id = str(getattr(props, "uuid", "")) or None
    if dev_id and not dev_id.startswith("GPU-"):
        dev_id = "GPU-" + dev_id
    sampler = ClockSampler(dev_id) if rank == 0 else None
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t = e0.elapsed_time(e1) / 1e3
    run.set_timing(True)
    run.step(min(args.steps, 10))
    torch.cuda.synchronize()
    stage_ms, stage_n, match_ms, match_n = run.timing()
    run.set_timing(False)
    clocks = sampler.stop() if sampler else None
    run.check()
    t = ranks.max(t)
    ns, nn, b = run.ns, g.nodes, 4
    t_step = t / args.steps
    value = job_rate(BATCH_EVENTS / BATCH_EVOLUTION_STEPS, world, t_step)
    alg_bytes_launch = 2.5 * b * ns * nn + ns * (56 + 64 + 8 + 8 + 4)
    achieved = alg_bytes_launch / (stage_ms / stage_n / 1e3) / 1e9
    peak, peak_kind = peaks()

    e2e = None
    if not args.no_e2e:
        t_e2e, e2e = end_to_end(run, eps, args.steps, barrier, torch)
        e2e = {"value": world * BATCH_EVENTS * args.steps / (t_e2e * BATCH_EVOLUTION_STEPS), "unit": "events/s",
               **e2e}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        side = 64
        win, _, _ = hotspots(side, side, n=40, seed=1108)
        cores = os.cpu_count() or 1
        rate, dt = oracle_rate(win, 4, cores)
        mean_sites = ns / BATCH_EVENTS
        cpu = {"value": rate / (mean_sites * nn * BATCH_EVOLUTION_STEPS), "unit": "events/s", "cores": cores,
               "kind": "oracle",
               "sample": "one 64x64 hotspot event, 4 oracle steps (%.1f s), scaled to a mean event of the "
                         "batch (%.0f sites, 200 steps)" % (dt, mean_sites)}
    if rank == 0:
        line = {
            "metric": "batched events/s", "value": value, "unit": "events/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of %d events, square sides U{64..192}, eta/s U(0.04, 0.3), "
                                   "40 hotspots each, 768 nodes, FP32 populations, %d-step evolution"
                                   % (BATCH_EVENTS, BATCH_EVOLUTION_STEPS),
                       "events": BATCH_EVENTS, "sites": ns, "nodes_per_site": nn, "dx_fm": DX,
                       "dtau": DTAU_BATCH, "tau0": TAU0, "stage_variant": chosen, "variant_ms": tune_ms,
                       "l2": "inputs larger than L2 (two %.1f GB population arrays)" % (ns * nn * b / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                         "kernel": "stage kernel (variant %d)" % chosen,
                         "algorithmic_bytes_per_update": 5 * b,
                         "stage_ms_per_launch": stage_ms / stage_n, "match_ms_per_launch": match_ms / match_n},
            "e2e": e2e, "gpu_launches": 4 * args.steps, "clocks": clocks, "cpu_baseline": cpu,
        }
        emit(line)
    ranks.close()
    return 0


def sweep_main(args, rank, world, local):
    """Precision sweep on the 16 x 8 x 16 lattice (2048 populations per site):
    1024 x 1024 grid of 40 hotspots, eta/s 0.16, timed for FP32 and BF16
    population storage (FP32 arithmetic and moments, FP64-accurate final steps of the
    matching), plus the error of both against the FP64 oracle on a 128 x 128
    sub-run.  The JSON line's value is the BF16 rate; both rates and the errors
    are in "sweep"."""
    import torch
    import paper_1108_5561_gb300 as rlb
    from paper_1108_5561_gb300.inputs import hotspots

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    side, lat = 1024, dict(n_xi=16, n_theta=8, n_phi_half=8)
    eps0, _, _ = hotspots(side, side, n=40, seed=1108)
    stream = torch.cuda.current_stream()
    res, kern = {}, {}
    peak, peak_kind = peaks()
    sampler = ClockSampler(None) if rank == 0 else None
    for name, prec, b in (("fp32", rlb.RLB_F32, 4), ("bf16", rlb.RLB_BF16, 2)):
        g = rlb.GridParams(nx=side, ny=side, dx=DX, prec=prec, eta_over_s=ETA_S, tau0=TAU0, dtau=DTAU_SWEEP, **lat)
        run = rlb.Run(g, device=local)
        run.init_grid(eps0)
        run.step(args.warmup)
        torch.cuda.synchronize()
        run.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        run.set_timing(True)
        run.step(min(args.steps, 20))
        torch.cuda.synchronize()
        sm, sn, mm, mn = run.timing()
        run.set_timing(False)
        run.check()
        ns, nn = side * side, g.nodes
        alg = 2.5 * b * ns * nn + ns * (56 + 64 + 8 + 8 + 4)
        res[name] = {"updates_per_s": ns * nn * args.steps / t, "ms_per_step": 1e3 * t / args.steps}
        kern[name] = {"stage_ms_per_launch": sm / sn, "match_ms_per_launch": mm / mn,
                      "achieved_GBps": alg / (sm / sn / 1e3) / 1e9}
        del run
        torch.cuda.empty_cache()
    clocks = sampler.stop() if sampler else None
    # accuracy: 128 x 128 sub-run against the oracle
    sub, sub_steps = 128, args.sweep_oracle_steps
    errs = {}
    if rank == 0:
        from oracle.oracle import Oracle
        c = side // 2
        win = eps0[c - sub // 2:c + sub // 2, c - sub // 2:c + sub // 2]
        o = Oracle(nx=sub, ny=sub, dx=DX, eta_over_s=ETA_S, **lat)
        f, lnM = o.init_state(win, os.cpu_count() or 1)
        o.step(f, lnM, TAU0, DTAU_SWEEP, sub_steps, os.cpu_count() or 1)
        mo = o.moments(f, lnM, os.cpu_count() or 1)
        for name, prec in (("fp32", rlb.RLB_F32), ("bf16", rlb.RLB_BF16)):
            g = rlb.GridParams(nx=sub, ny=sub, dx=DX, prec=prec, eta_over_s=ETA_S, tau0=TAU0, dtau=DTAU_SWEEP, **lat)
            r = rlb.Run(g, device=local)
            r.init_grid(win)
            r.step(sub_steps)
            mg = r.moments()
            errs[name] = {"eps": float(np.abs(mg[:, 0] / mo[:, 0] - 1).max()),
                          "T": float(np.abs(mg[:, 1] / mo[:, 1] - 1).max()),
                          "u": float((np.abs(mg[:, 2:5] - mo[:, 2:5]).max(axis=1) /
                                      np.abs(mo[:, 2:5]).max(axis=1)).max())}
    if rank == 0:
        bf = res["bf16"]
        line = {
            "metric": "site-population updates/s", "value": bf["updates_per_s"], "unit": "updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": bf["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "precision sweep: 1024x1024 grid, 16x8x16 = 2048 populations/site, "
                                   "40 hotspots, BF16 vs FP32 storage",
                       "grid": [side, side], "nodes_per_site": 2048, "eta_over_s": ETA_S, "dtau": DTAU_SWEEP,
                       "tau0": TAU0, "l2": "inputs larger than L2 (4.3 GB BF16 / 8.6 GB FP32 per array)",
                       "parallelism": "single GPU"},
            "roofline": {"bound": "hbm", "achieved": kern["bf16"]["achieved_GBps"], "peak": peak, "unit": "GB/s",
                         "frac": kern["bf16"]["achieved_GBps"] / peak, "traffic": None, "peak_source": peak_kind,
                         "kernel": "stage_kernel_x2 <bf16, 16, 8, 16>", "algorithmic_bytes_per_update": 10},
            "sweep": {"rates": res, "kernels": kern, "oracle_subrun": {"grid": [sub, sub], "steps": sub_steps,
                                                                      "max_rel_error": errs}},
            "e2e": None, "gpu_launches": 4 * args.steps, "clocks": clocks, "cpu_baseline": None,
        }
        emit(line)
    return 0


def adjoint_main(args, rank, world, local):
    """Adjoint workload: 128 x 128 grid, 768 nodes, FP32 populations, 40
    hotspots, eta/s 0.08, 300 steps from tau 0.4 fm/c; gradient of the final
    p_perp-weighted v2 with respect to the 40 hotspot amplitudes and eta/s by the
    discrete adjoint with a checkpoint every 32 steps.  Value: time of the
    gradient with FP32 per-node adjoint arithmetic (forward with checkpoints +
    adjoint sweep) over the time of the plain forward run; the FP64-arithmetic
    gradient is timed too and the two are compared, and two amplitude components
    are checked against central finite differences of the forward run."""
    import torch
    import paper_1108_5561_gb300 as rlb
    from paper_1108_5561_gb300 import adjoint as ADJ
    from paper_1108_5561_gb300.inputs import hotspot_basis, hotspots

    torch.cuda.set_device(local)
    side, steps, every, etas = 128, args.steps, 32, 0.08
    _, amps, cen = hotspots(side, side, n=40, seed=1108)
    basis_h = hotspot_basis(side, side, cen, dx=DX)
    floor = 10.0
    g = rlb.GridParams(nx=side, ny=side, dx=DX, prec=rlb.RLB_F32, eta_over_s=etas, tau0=TAU0, dtau=DTAU_ADJ)
    run = rlb.Run(g, device=local)
    eps0 = torch.as_tensor(floor + amps @ basis_h, dtype=torch.float64, device="cuda")
    basis = torch.as_tensor(basis_h, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):  # warm-up: forward runs
        run.init_grid(eps0)
        run.step(steps)
    torch.cuda.synchronize()
    sampler = ClockSampler(None) if rank == 0 else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.init_grid(eps0)
    run.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / 1e3
    t0 = time.perf_counter()
    v2, gA, geta = ADJ.v2_gradient(run, eps0, basis, steps, every, arithmetic=rlb.RLB_F32)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, gA64, geta64 = ADJ.v2_gradient(run, eps0, basis, steps, every, arithmetic=rlb.RLB_F64)
    torch.cuda.synchronize()
    t_grad64 = time.perf_counter() - t0
    t0 = time.perf_counter()  # every step's state kept in HBM: no recompute
    ADJ.v2_gradient(run, eps0, basis, steps, 1, arithmetic=rlb.RLB_F32)
    torch.cuda.synchronize()
    t_grad1 = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    run.check()
    # finite differences of the forward run for the two largest amplitudes
    def v2_of(a):
        run.init_grid(torch.as_tensor(floor + a @ basis_h, dtype=torch.float64, device="cuda"))
        run.step(steps)
        return run.observables()[1]
    checks = []
    for i in np.argsort(-amps)[:2]:
        h = 0.05 * amps[i]
        ap, am = amps.copy(), amps.copy()
        ap[i] += h
        am[i] -= h
        fd = (v2_of(ap) - v2_of(am)) / (2 * h)
        checks.append({"hotspot": int(i), "adjoint": float(gA[i]), "adjoint_fp64": float(gA64[i]),
                       "finite_difference": float(fd),
                       "rel_diff": float(abs(gA[i] - fd) / max(abs(fd), 1e-300)),
                       "rel_diff_fp64": float(abs(gA64[i] - fd) / max(abs(fd), 1e-300))})
    if rank == 0:
        line = {
            "metric": "adjoint/forward time", "value": t_grad / t_fwd, "unit": "x",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_fwd / steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "adjoint: 128x128, 768 nodes, FP32 populations, 40 hotspots, eta/s 0.08, "
                                   "%d steps, checkpoint every %d, gradient of final p_perp-weighted v2 wrt "
                                   "40 amplitudes and eta/s (FP32 per-node adjoint arithmetic, FP64 matching "
                                   "adjoint)" % (steps, every),
                       "grid": [side, side], "dtau": DTAU_ADJ, "tau0": TAU0, "forward_s": t_fwd, "gradient_s": t_grad,
                       "gradient_fp64_s": t_grad64, "fp64_over_forward": t_grad64 / t_fwd,
                       "every_step_kept": {"gradient_s": t_grad1, "over_forward": t_grad1 / t_fwd,
                                           "device_bytes": steps * run.state_blob_size()},
                       "fp32_vs_fp64_rel": {
                           "amplitudes": float(np.linalg.norm(gA - gA64) / np.linalg.norm(gA64)),
                           "eta": float(abs(geta - geta64) / abs(geta64))},
                       "v2": v2,
                       "dv2_deta": geta, "dv2_dA_norm": float(np.linalg.norm(gA)), "fd_checks": checks,
                       "parallelism": "single GPU"},
            "roofline": None, "e2e": None, "gpu_launches": None, "clocks": clocks, "cpu_baseline": None,
        }
        emit(line)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 1000 for the grid workload, 40 for the batch)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="grid", choices=["grid", "batch", "sweep", "adjoint"],
                    help="grid: 256x256 FP32 (site-population updates/s); batch: 512 events (events/s); "
                         "sweep: 1024x1024 x 2048 nodes, BF16 vs FP32; adjoint: gradient of v2, 128x128")
    ap.add_argument("--sweep-oracle-steps", type=int, default=10,
                    help="steps of the 128x128 oracle sub-run of the sweep")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the short batch / adjoint / sweep / FP64 / ALU-peak records of the grid run")
    ap.add_argument("--grid", type=int, default=256,
                    help="grid side; the benchmark workload is 256 (smaller sides for profiling)")
    ap.add_argument("--record", default=None, help="also append the JSON line to this JSONL file")
    args = ap.parse_args()
    global RECORD
    RECORD = args.record
    if args.steps is None:
        args.steps = {"batch": 40, "sweep": 500, "adjoint": 300}.get(args.workload, 1000)
    global NX, NY
    NX = NY = args.grid
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "batch":
        return batch_main(args, rank, world, local)
    if args.workload == "sweep":
        return sweep_main(args, rank, world, local)
    if args.workload == "adjoint":
        return adjoint_main(args, rank, world, local)

    import torch
    import paper_1108_5561_gb300 as rlb
    from paper_1108_5561_gb300.inputs import hotspots

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    ranks = Ranks("nccl")
    eps0, _, _ = hotspots(NX, NY, n=40, seed=1108)
    g = rlb.GridParams(nx=NX, ny=NY, dx=DX, prec=rlb.RLB_F32, eta_over_s=ETA_S, tau0=TAU0,
                       dtau=DTAU)
    run = rlb.Run(g, device=local)
    run.init_grid(eps0)
    stream = torch.cuda.current_stream()
    run.step(args.warmup)
    torch.cuda.synchronize()
    run.check()

    barrier = ranks.barrier

    props = torch.cuda.get_device_properties(local)
    dev_id = str(getattr(props, "uuid", "")) or None
    if dev_id and not dev_id.startswith("GPU-"):
        dev_id = "GPU-" + dev_id
    sampler = ClockSampler(dev_id) if rank == 0 else None
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t = e0.elapsed_time(e1) / 1e3
    # per-kernel launch durations (CUDA events inside the library, same stream),
    # measured on a separate pass of the same steps so the timed region above
    # carries no extra events
    run.set_timing(True)
    run.step(min(args.steps, 200))
    torch.cuda.synchronize()
    stage_ms, stage_n, match_ms, match_n = run.timing()
    run.set_timing(False)
    clocks = sampler.stop() if sampler else None
    run.check()
    t = ranks.max(t)
    ns, nn = NX * NY, g.nodes
    updates = world * ns * nn * args.steps
    value = job_rate(ns * nn * args.steps, world, t)
    b = 4  # FP32 storage
    launches = 4 * args.steps  # per step: (match + stream-collide) x (predictor, corrector)
    # algorithmic bytes of one stream-collide launch: predictor reads f and writes
    # f* (2b), corrector reads f* and f and writes f (3b) per population; per site
    # 14 FP32 matching results, 16 floats of output moments, ln M in and out,
    # ln M at tau (corrector only)
    alg_bytes_launch = 2.5 * b * ns * nn + ns * (56 + 64 + 8 + 8 + 4)
    achieved = alg_bytes_launch / (stage_ms / stage_n / 1e3) / 1e9
    peak, peak_kind = peaks()

    # end to end through the library's host-buffer calls: eps0 from pinned host
    # memory, the initial condition, then every step the step itself and the
    # per-site observables into pinned host memory.
    e2e = None
    if not args.no_e2e:
        t_e2e, e2e = end_to_end(run, eps0, args.steps, barrier, torch)
        e2e = {"value": updates / t_e2e, "unit": "updates/s", **e2e}

    kern = {"stream_collide_ms_per_launch": stage_ms / stage_n,
            "match_ms_per_launch": match_ms / match_n, "timed_launches": stage_n + match_n}
    sec = None
    if rank == 0 and world == 1 and not args.no_secondary:
        del run
        torch.cuda.empty_cache()
        sec = secondary(args, local, torch, rlb)
        alu = sec["alu_peaks_tflops"]["fp32_ffma2_tflops"]
        fl = FLOPS_PER_POP_STAGE["fp32_mirror_paired"] * ns * nn / (stage_ms / stage_n / 1e3) / 1e12
        kern["alu_roofline"] = {"bound": "alu", "achieved": fl, "peak": alu, "unit": "TFLOP/s", "frac": fl / alu,
                                "peak_source": "measured (rlb_alu_peaks, packed FP32 multiply-add)",
                                "flops_per_population_stage": FLOPS_PER_POP_STAGE["fp32_mirror_paired"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c = NX // 2
        win = eps0[c - 64:c + 64, c - 64:c + 64]
        cores = os.cpu_count() or 1
        rate, dt = oracle_rate(win, 16, cores)
        cpu = {"value": rate, "unit": "updates/s", "cores": cores, "kind": "oracle",
               "sample": "128x128 central window of the workload, 16 oracle steps (%.1f s)" % dt}
    return finish(args, rank, world, t, value, achieved, peak, peak_kind, b, nn, launches, e2e,
                  clocks, cpu, ranks, kern, sec)


def end_to_end(run, eps0, steps, barrier, torch):
    """The same steps through the library's host-buffer calls: rlb_init_grid
    reads eps0 from (pinned) host memory, and after every step
    rlb_moments_async downloads the per-site observables (8 doubles per site)
    into one of two pinned host arrays while the next step runs; the timed
    region ends when rlb_moments_wait reports every download complete.  Also
    timed: the synchronous form (rlb_moments into host memory after every
    step, returning when the data is there).  Returns (seconds, the e2e record
    without its value)."""
    ns = run.ns
    host_eps = torch.from_numpy(np.ascontiguousarray(eps0).reshape(-1).copy()).pin_memory()
    host_obs = [torch.empty((ns, 8), dtype=torch.float64).pin_memory() for _ in range(2)]
    eps_np = host_eps.numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run.init_grid(eps_np)
    for k in range(steps):
        run.step(1)
        run.moments_async(host_obs[k % 2])
    run.moments_wait()
    torch.cuda.synchronize()
    barrier()
    t_e2e = time.perf_counter() - t0
    run.check()
    # the synchronous form, for the record
    obs_np = host_obs[0].numpy()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    run.init_grid(eps_np)
    for _ in range(steps):
        run.step(1)
        run.moments(out=obs_np)
    torch.cuda.synchronize()
    t_sync = time.perf_counter() - t1
    return t_e2e, {"h2d_bytes_per_step": ns * 8 / steps, "d2h_bytes_per_step": ns * 8 * 8,
                   "path": "rlb_init_grid(host eps0) once, then per step rlb_step + rlb_moments_async(pinned host "
                           "output, downloaded during the next step), rlb_moments_wait at the end",
                   "synchronous_updates_per_s": ns * run.nn * steps / t_sync,
                   "synchronous_path": "per step rlb_step + rlb_moments(host output, returns when it is there)"}


# Arithmetic per population and stage, counted from the kernels' per-node
# operations (a multiply-add = 2 flops; the FP64 exponential of the generic
# kernel counted as 20): the mirror-paired FP32 stage kernel about 80 FP32
# flops (streaming 13, radial operator and Milne term 18, polar operator on the
# even/odd parts 13, equilibrium/force/collision and the d ln M sums 26, Heun
# 5, moments 5) plus one hardware exponential; the generic FP64 kernel about 110.
FLOPS_PER_POP_STAGE = {"fp32_mirror_paired": 80, "fp64_generic": 110}


def secondary(args, local, torch, rlb):
    """Short runs of the other workloads, for the grid run's JSON line: ALU
    peaks, the FP64 32x32 run (Gaussian, eta/s 0.08, 200 steps), the 512-event
    batch, the 128x128 adjoint and the 1024x1024 BF16/FP32 sweep (a few timed
    steps each; the dedicated --workload runs time them at length)."""
    from paper_1108_5561_gb300.inputs import batch_events, hotspot_basis, hotspots, smooth_gaussian
    from paper_1108_5561_gb300 import adjoint as ADJ
    out = {}
    stream = torch.cuda.current_stream()

    def timed(run, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def stage_ms(run, steps):
        run.set_timing(True)
        run.step(steps)
        torch.cuda.synchronize()
        sm, sn, mm, mn = run.timing()
        run.set_timing(False)
        return sm / sn, mm / mn

    peaks_alu = rlb.alu_peaks(local)
    out["alu_peaks_tflops"] = peaks_alu
    # plain FP64 step: the 32x32 Gaussian run of the FP64 parity test
    g = rlb.GridParams(nx=32, ny=32, dx=0.2, prec=rlb.RLB_F64, eta_over_s=0.08, tau0=0.4, dtau=0.018)
    run = rlb.Run(g, device=local)
    run.init_grid(smooth_gaussian(32, 32))
    run.step(3)
    t = timed(run, 200)
    sms, mms = stage_ms(run, 20)
    pops = 32 * 32 * g.nodes
    fp64_rate = pops * 200 / t
    fl = FLOPS_PER_POP_STAGE["fp64_generic"] * pops / (sms / 1e3) / 1e12
    out["fp64_32x32"] = {"updates_per_s": fp64_rate, "ms_per_step": 1e3 * t / 200, "stage_ms_per_launch": sms,
                         "match_ms_per_launch": mms, "stage_fp64_tflops": fl,
                         "stage_frac_of_fp64_peak": fl / peaks_alu["fp64_dfma_tflops"]}
    del run
    # batch of 512 events
    evs = batch_events(BATCH_EVENTS, seed=1108)
    events = [rlb.Event(n, n, eta) for n, eta in evs]
    eps = np.concatenate([hotspots(n, n, n=40, seed=1108 + i)[0].reshape(-1) for i, (n, _) in enumerate(evs)])
    gb = rlb.GridParams(dx=DX, prec=rlb.RLB_F32, tau0=TAU0, dtau=DTAU_BATCH)
    run = rlb.Run(gb, device=local, events=events)
    run.init_grid(eps)
    run.step(1)
    chosen, _ = run.autotune()
    run.step(3)
    t = timed(run, 8) / 8
    sms, mms = stage_ms(run, 4)
    batch_rate = run.ns * gb.nodes / t
    out["batch_512"] = {"events_per_s": BATCH_EVENTS / BATCH_EVOLUTION_STEPS / t, "ms_per_step": 1e3 * t,
                        "updates_per_s": batch_rate, "sites": run.ns, "stage_variant": chosen,
                        "stage_ms_per_launch": sms, "match_ms_per_launch": mms,
                        "vs_fp64_32x32_updates": batch_rate / fp64_rate}
    del run, eps
    torch.cuda.empty_cache()
    # adjoint: gradient of v2 on 128x128, 300 steps, checkpoint every 32 (FP32 adjoint arithmetic)
    side, steps = 128, 300
    _, amps, cen = hotspots(side, side, n=40, seed=1108)
    basis_h = hotspot_basis(side, side, cen, dx=DX)
    ga = rlb.GridParams(nx=side, ny=side, dx=DX, prec=rlb.RLB_F32, eta_over_s=0.08, tau0=TAU0, dtau=DTAU_ADJ)
    run = rlb.Run(ga, device=local)
    eps0 = torch.as_tensor(10.0 + amps @ basis_h, dtype=torch.float64, device="cuda")
    basis = torch.as_tensor(basis_h, dtype=torch.float64, device="cuda")
    run.init_grid(eps0)
    run.step(steps)
    run.init_grid(eps0)
    t_fwd = timed(run, steps)
    ADJ.v2_gradient(run, eps0, basis, 8, 4, arithmetic=rlb.RLB_F32)  # warm-up of the adjoint kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ADJ.v2_gradient(run, eps0, basis, steps, 32, arithmetic=rlb.RLB_F32)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    # the same gradient with every step's state kept in HBM (no recompute)
    run_blob_bytes = run.state_blob_size()
    t0 = time.perf_counter()
    ADJ.v2_gradient(run, eps0, basis, steps, 1, arithmetic=rlb.RLB_F32)
    torch.cuda.synchronize()
    t_grad1 = time.perf_counter() - t0
    del run
    g64 = rlb.GridParams(nx=side, ny=side, dx=DX, prec=rlb.RLB_F64, eta_over_s=0.08, tau0=TAU0, dtau=DTAU_ADJ)
    run = rlb.Run(g64, device=local)
    run.init_grid(eps0)
    run.step(3)
    run.init_grid(eps0)
    t_fwd64 = timed(run, steps)
    del run
    out["adjoint_128x128"] = {"dtau": DTAU_ADJ, "gradient_s": t_grad, "forward_fp32_s": t_fwd,
                              "over_forward_fp32": t_grad / t_fwd,
                              "forward_fp64_s": t_fwd64, "over_forward_fp64": t_grad / t_fwd64,
                              "steps": steps, "checkpoint_every": 32,
                              "every_step_kept": {"gradient_s": t_grad1, "over_forward_fp32": t_grad1 / t_fwd,
                                                  "device_bytes": steps * run_blob_bytes}}
    # precision sweep: 1024x1024, 16x8x16 lattice
    sweep = {}
    eps0 = hotspots(1024, 1024, n=40, seed=1108)[0]
    for name, prec, b in (("fp32", rlb.RLB_F32, 4), ("bf16", rlb.RLB_BF16, 2)):
        gs = rlb.GridParams(nx=1024, ny=1024, dx=DX, prec=prec, eta_over_s=ETA_S, tau0=TAU0, dtau=DTAU_SWEEP,
                            n_xi=16, n_theta=8, n_phi_half=8)
        run = rlb.Run(gs, device=local)
        run.init_grid(eps0)
        run.step(3)
        t = timed(run, 6) / 6
        sms, _ = stage_ms(run, 4)
        ns, nn = 1024 * 1024, gs.nodes
        alg = 2.5 * b * ns * nn + ns * (56 + 64 + 8 + 8 + 4)
        sweep[name] = {"updates_per_s": ns * nn / t, "ms_per_step": 1e3 * t, "stage_ms_per_launch": sms,
                       "stage_frac_of_hbm": alg / (sms / 1e3) / 1e9 / peaks()[0]}
        del run
        torch.cuda.empty_cache()
    out["sweep_1024x1024_2048"] = sweep
    return out


def finish(args, rank, world, t, value, achieved, peak, peak_kind, b, nn, launches, e2e, clocks,
           cpu, ranks, kern, sec=None):
    if rank == 0:
        line = {
            "metric": "site-population updates/s", "value": value, "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("256x256", "%dx%d" % (NX, NY)), "grid": [NX, NY], "dx_fm": DX,
                       "nodes_per_site": nn,
                       "eta_over_s": ETA_S, "dtau": DTAU, "tau0": TAU0,
                       "l2": "inputs larger than L2 (two 201 MB population arrays)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": stage_traffic(NX),
                         "peak_source": peak_kind,
                         "kernel": "stage_kernel_mp (fused stream-collide, mirror-paired polar lines, packed FP32 pairs)",
                         "algorithmic_bytes_per_update": 5 * b, **kern},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "secondary": sec,
        }
        emit(line)
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
