"""Throughput of the unsplit CTU step on a GB300 (zone-updates per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload kh1024|sedov4096|sedov8192|rt1024] [--precision fp32|fp64]

A step is one pass of the solver's driver loop (paper §2): ghost fill, CFL time step reduced on the
device, one fused CTU step.  Default workload: the 1024 x 1024 periodic Kelvin-Helmholtz shear layer
(gamma 1.4, CFL 0.8, seeded noise in v), FP32 bulk with double energy recovery; the plain FP64 path is
measured on the same workload in the same run.  Inputs are resident in HBM when the timed region
starts; the state (17 MB in FP32) fits in L2, so L2 is flushed (256 MB write) before every timed step
and each step is timed on its own with CUDA events on the solver's stream.

--impl reference times the FP64 CPU oracle (the plain C implementation the CUDA path is checked
against) on the host cores, on the same workload and metric.

Multi-GPU (torchrun, N > 1): the problem is replicated, one independent copy per rank (no data-path
exchange); the value is the sum over ranks, timed by the slowest rank.
"""
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

# algorithmic flops per zone-update: counted with an instrumented copy of the FP64 oracle on the
# Kelvin-Helmholtz workload (+ - * / sqrt = 1 flop each): 973 per zone plus 40 per Newton iteration of
# the two-shock solver, at 4.008 solves per zone
FLOPS_BASE = 973.0
FLOPS_PER_ITER = 40.0
SOLVES_PER_ZONE = 4.008
# ALU peaks from the unit counts and the maximum SM clock (FMA = 2 flops): FP32 152 SMs x 128 lanes x 2 x
# 2070 MHz = 80.55 TFLOP/s; FP64 the part's 1.25 TFLOP/s.  (FMA-chain microbenchmarks on the same GPUs reach
# 73.4 and 1.16 TFLOP/s.)
ALU_PEAK_TFLOPS = {"fp32": 152 * 128 * 2 * 2.070e9 / 1e12, "fp64": 1.25}
ALU_PEAK_SOURCE = {"fp32": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (unit counts x max SM clock)",
                   "fp64": "GB300 FP64 rate 1.25 TFLOP/s"}


# DRAM bytes (read + write) of one launch of the FP32 fused step kernel on the KH 1024^2 workload, from an
# ncu capture of the kernel built from the sources whose SHA-256 is recorded; reported only while the
# kernel's sources are unchanged (otherwise the counters describe another kernel and traffic is null)
TRAFFIC_CAPTURE = {"bytes_per_launch": 17378816 + 1024, "issue_active": 0.7882, "warp_instructions": 79743152,
                   "sources_sha256": "472f1932619ece4588de8e4e77ed15e12edaa6738965092c67af0d80ae8ad680"}
KERNEL_SOURCES = ["paper_1306_6883_gb300/csrc/" + f for f in
                  ("k_ctu.cu", "ctu_kernels.cuh", "ctu_tile.cuh", "hydro_device.cuh", "mlp.cuh", "hydro_kernels.h",
                   "tma.cuh")] + ["include/hydro.h"]


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "note": "fallback"}


def workload(name):
    import hydro_problems as hp
    if name == "kh1024":
        return hp.kh(1024, 1024, seed=0), "kh_1024x1024_periodic"
    if name == "sedov4096":
        return hp.sedov(4096, 4096), "sedov_4096x4096_outflow"
    if name == "sedov8192":
        return hp.sedov(8192, 8192, density_noise=0.01), "sedov_8192x8192_outflow_1pct_noise"
    if name == "rt1024":
        return hp.rt(1024, 3072), "rayleigh_taylor_1024x3072_gravity_hydrostatic"
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hydro_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 250.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k in range(4) if r[3][k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------------- our arm
def time_device_path(pr, precision, steps, warmup, flush, **kw):
    """Value: steps of the driver loop (ghost cells, CFL dt, CTU step) with the state resident in HBM through
    hydro_step_fused: one launch of the fused step kernel (two sweep launches for the split variant)."""
    import torch

    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    prec = H.HYDRO_FP32 if precision == "fp32" else H.HYDRO_FP64
    s = Solver(params_for(pr, prec, **kw), pr.U)
    stream = s.stream
    for _ in range(warmup):
        s.step_fused()
    st0, stats0 = s.status()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        s.step_fused()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st, stats1 = s.status()
    t_sim, n_sim = s.time()
    tot = s.totals()
    s.close()
    solves = stats1[0] - stats0[0]
    iters = stats1[1] - stats0[1]
    launches = 2 if kw.get("split") else 1  # split: x (y) sweep, y (x) sweep folding in the dt
    return {"step_ms": step_ms, "kernel_ms": step_ms, "iters_per_solve": iters / max(solves, 1),
            "t_sim": t_sim, "totals": tot, "launches_per_step": launches}


def time_e2e(pr, precision, steps, warmup):
    """Same metric through the public C-ABI call for a run kept in host memory, hydro_step_host_chained:
    every step uploads the whole state from pinned host memory in chunks of tile-row bands, runs the fused
    step band by band as the rows arrive (its time step is the one the previous call reduced from the state
    it wrote, which is this call's input) and copies each band's rows back while later bands compute,
    returning when the new state is in host memory; the two pinned host buffers alternate as input and
    output.  The first warm-up call reduces the time step from the uploaded state (no chain yet)."""
    import torch

    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    prec = H.HYDRO_FP32 if precision == "fp32" else H.HYDRO_FP64
    dt_ = torch.float32 if precision == "fp32" else torch.float64
    s = Solver(params_for(pr, prec), pr.U)
    host = [torch.from_numpy(np.ascontiguousarray(pr.U)).to(dt_).pin_memory() for _ in range(2)]

    def one(k):
        s.step_host(host[k % 2], host[(k + 1) % 2], chained=True)

    for k in range(warmup):
        one(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(warmup, warmup + steps):  # the run goes on: each input is the previous step's output
        one(k)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    s.status()
    s.close()
    nbytes = host[0].numel() * host[0].element_size()
    return {"seconds": el, "h2d": nbytes, "d2h": nbytes}


def fp32_error(pr, steps=50):
    """Error of the FP32 path against the FP64 path after `steps` fused steps from the same initial state:
    L1 and max of |U32 - U64| per field, relative to the field's L1 norm and maximum.  The FP64 path rounds
    exactly like the oracle (bit-identical runs are a test of the suite), so this is the FP32 error against
    the oracle."""
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    out = {}
    for prec in (H.HYDRO_FP64, H.HYDRO_FP32):
        s = Solver(params_for(pr, prec), pr.U)
        s.advance(steps)
        ng = pr.ng
        out[prec] = (s.state_numpy()[:, ng:-ng, ng:-ng].astype(np.float64), s.time())
        s.status()
        s.close()
    a, (t32, _) = out[H.HYDRO_FP32]
    b, (t64, _) = out[H.HYDRO_FP64]
    d = np.abs(a - b).reshape(4, -1)
    ref = np.abs(b).reshape(4, -1)
    names = ("rho", "rho_u", "rho_v", "E")
    return {"steps": steps, "against": "FP64 GPU path (bit-identical to the oracle)",
            "l1_rel": dict(zip(names, (d.sum(1) / ref.sum(1)).tolist())),
            "max_rel": dict(zip(names, (d.max(1) / ref.max(1)).tolist())),
            "t_rel": abs(t32 - t64) / t64}


def time_ensemble(steps=100, warmup=3, n=256, seed=0):
    """The 256-member ensemble of four-quadrant problems on {64,128,256,512}^2 grids (seeded), FP32, each
    member with its own CFL dt; tile shapes autotuned per size class; `steps` steps captured in one CUDA
    graph and launched once.  The states (~0.4 GB per buffer) exceed L2."""
    import torch

    import hydro_problems as hp
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Ensemble, params_for

    probs = hp.ensemble(n, seed)
    e = Ensemble([params_for(p, H.HYDRO_FP32) for p in probs], [p.U for p in probs])
    shapes = e.autotune(reps=2)
    e.run(warmup)
    e.status()
    torch.cuda.synchronize()
    e.run(steps)  # capture + instantiate the graph of `steps` steps (untimed), advancing the members
    torch.cuda.synchronize()
    e.run(steps)  # same parity again only if steps is even; otherwise this captures the other graph
    torch.cuda.synchronize()
    s = e.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    e.run(steps)
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st, stats = e.status()
    cells = sum(p.nx * p.ny for p in probs)
    out = {"members": n, "cells": cells, "steps": steps, "ms": ms, "value": cells * steps / (ms * 1e-3),
           # per run: one dt kernel; per step: one persistent fused step kernel per distinct tile shape
           "unit": "zone-updates/s", "graph_launches": 1, "kernel_launches": 1 + steps * len(set(shapes)),
           "classes": e.classes(), "riemann_iters_per_solve": stats[1] / max(stats[0], 1)}
    e.close()
    return out


def harvest_and_train(train_steps=6000, batch=4096, lr=1e-3, seed=0):
    """Training set for the learned starting pressure: Riemann problems sampled from FP32 runs of the Sod
    tube (128^2 to t = 0.2), the Kelvin-Helmholtz layer (1024^2, 40 steps) and the Sedov blast (1024^2,
    300 steps).  Faces are kept at random (hash of face and step) and, in addition, every face past the
    network's gate (the faces the network will be asked about); training draws its minibatches from an equal
    mix of gated and other faces.  Then `train_steps` Adam steps of the library's training kernels."""
    import torch

    import hydro_problems as hp
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Model, Solver, params_for

    cap = 12_000_000
    buf = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = [(hp.sod(128, 128), 0.2, 70, 0.25), (hp.kh(1024, 1024), 0.0, 40, 0.02),
            (hp.sedov(1024, 1024), 0.0, 300, 0.005)]
    t0 = time.perf_counter()
    gate = (0.35, 1.0)  # the default gate of the learned kernels (model.set_gate)
    for pr, tmax, steps, rate in plan:
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        H.hydro_set_harvest(s.ctx, buf.data_ptr(), cap, rate, count.data_ptr())
        H.hydro_set_harvest_gate(s.ctx, *gate)
        s.advance(steps, tmax)
        s.status()
        s.close()
    n = min(int(count.item()), cap)
    data = buf[:n]
    torch.cuda.synchronize()
    t_h = time.perf_counter()
    gated = strong_mask(data)
    g = torch.Generator(device="cuda").manual_seed(seed)
    strong_set, weak_set = data[gated], data[~gated]
    k = min(weak_set.shape[0], max(strong_set.shape[0], 1))
    weak_pick = weak_set[torch.randperm(weak_set.shape[0], device="cuda", generator=g)[:k]]
    train_set = torch.cat([strong_set, weak_pick])
    train_set = train_set[torch.randperm(train_set.shape[0], device="cuda", generator=g)].contiguous()
    t1 = time.perf_counter()
    m = Model(seed=seed)
    loss = m.train(train_set, steps=train_steps, batch=batch, lr=lr, seed=seed + 1)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # iterations per face at the FP32 tolerance, acoustic vs learned start: on a held-out problem family
    # (four-quadrant problems, not in the training set) and on the training set, all faces and the faces
    # the default gate sends to the network
    cap2 = 2_000_000
    buf2 = torch.zeros((cap2, 8), dtype=torch.float32, device="cuda")
    count2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    for k in range(4):
        pr = hp.quad(512, 512, seed=1000 + k)
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        H.hydro_set_harvest(s.ctx, buf2.data_ptr(), cap2, 0.05, count2.data_ptr())
        s.advance(20)
        s.status()
        s.close()
    held = buf2[:min(int(count2.item()), cap2)]

    def strong(d):
        return d[strong_mask(d)].contiguous()

    iters = {}
    rnd = data[~gated][:2_000_000].contiguous()  # the randomly kept faces (gated ones are counted apart)
    for name, d in (("held_out_quad_all", held), ("held_out_quad_strong", strong(held)),
                    ("training_runs_random", rnd), ("training_runs_strong", strong_set.contiguous())):
        row = {"faces": int(d.shape[0])}
        if d.shape[0]:
            for learned in (False, True):
                mean, nonconv = H.hydro_mlp_iterations(m.m, d.data_ptr(), d.shape[0], learned)
                row["learned" if learned else "acoustic"] = mean
                row["nonconverged_" + ("learned" if learned else "acoustic")] = nonconv
        iters[name] = row
    return m, {"samples": n, "gated_samples": int(strong_set.shape[0]), "training_set": int(train_set.shape[0]),
               "harvest_s": t_h - t0, "curation_s": t1 - t_h, "train_steps": train_steps, "batch": batch, "train_s": t2 - t1,
               "final_minibatch_loss": loss, "iterations_per_face": iters}


def strong_mask(d):
    """Harvested faces past the default gate of the learned kernels: |ln(pL/pR)|/2 >= 0.35 or
    |uL - uR| / c_ref >= 1 (columns rho_L, u_L, p_L, rho_R, u_R, p_R)."""
    import torch
    pmax, pmin = torch.maximum(d[:, 2], d[:, 5]), torch.minimum(d[:, 2], d[:, 5])
    du = d[:, 1] - d[:, 4]
    return (pmax >= math.exp(0.7) * pmin) | (du ** 4 * d[:, 0] * d[:, 3] >= d[:, 2] * d[:, 5])


def time_learned(model, steps=20, warmup=3):
    """Config of the learned proposal: 8192^2 Sedov blast with 1 % seeded density noise, FP32, the same
    steps with the acoustic start (plain) and with the network's start (default gate, and gate always
    open); zone-updates/s and Riemann iterations per solve at the same tolerance."""
    import torch

    import hydro_problems as hp
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    pr = hp.sedov(8192, 8192, density_noise=0.01)
    out = {"workload": "sedov_8192x8192_outflow_1pct_noise", "steps": steps}
    for name, learned, gate in (("plain", False, None), ("learned", True, (0.35, 1.0)),
                                ("learned_gate_open", True, (0.0, 0.0))):
        if learned:
            model.set_gate(*gate)
        s = Solver(params_for(pr, H.HYDRO_FP32, use_learned_guess=1 if learned else 0), pr.U)
        if learned:
            H.hydro_set_riemann_model(s.ctx, model.m)
        s.advance(warmup)
        s.status()
        _, st0 = s.status()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.advance(steps)
        b.record(s.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        _, st1 = s.status()
        s.close()
        solves, iters = st1[0] - st0[0], st1[1] - st0[1]
        out[name] = {"value": pr.nx * pr.ny * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "riemann_iters_per_solve": iters / max(solves, 1)}
    model.set_gate(0.35, 1.0)
    return out


def cpu_baseline(pr, budget_s=12.0, max_steps=50):
    """The oracle as it stands (OpenMP over rows on all host cores), on whole steps of the same workload,
    for about budget_s seconds."""
    import oracle

    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    oracle.fill_ghost(p, U)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps:
        oracle.fill_ghost(p, U)
        oracle.step(p, U, oracle.cfl_dt(p, U))
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": pr.nx * pr.ny * n / el, "unit": "zone-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{n} whole steps of the {pr.nx}x{pr.ny} workload from its initial state, "
                                        f"{el:.1f} s, FP64"}


def cpu_variant(pr, steps=5, **kw):
    """The oracle beside a variant leg: `steps` whole FP64 steps of the same workload with the same options
    (split, riemann_solver, reconstruction; gravity from the problem), on all host cores."""
    import oracle

    xmin, xmax, ymin, ymax = pr.domain
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                      ymax=ymax, grav=pr.grav, riemann_solver=kw.get("riemann_solver", 0),
                      reconstruction=kw.get("reconstruction", 0))
    U = pr.U.copy()
    t0 = time.perf_counter()
    oracle.advance(p, U, nsteps=steps, split=bool(kw.get("split")))
    el = time.perf_counter() - t0
    return {"value": pr.nx * pr.ny * steps / el, "unit": "zone-updates/s", "cores": oracle.num_threads(),
            "sample": f"{steps} whole FP64 steps, {el:.2f} s"}


def run_ours(args, world, rank, local):
    import torch

    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    pr, wname = workload(args.workload)
    zones = pr.nx * pr.ny
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        main = time_device_path(pr, args.precision, args.steps, args.warmup, flush)
    barrier(world)
    other = "fp64" if args.precision == "fp32" else "fp32"
    var = time_device_path(pr, other, max(args.steps // 4, 10), args.warmup, flush)
    e2e = time_e2e(pr, args.precision, max(args.steps // 4, 10), args.warmup)
    accuracy = fp32_error(pr) if args.precision == "fp32" else None
    ens = time_ensemble() if args.precision == "fp32" else None
    rt = split = hllc = ppm = None
    if args.precision == "fp32":
        r = time_device_path(pr, "fp32", 20, args.warmup, flush, reconstruction=1)
        ppm = {"workload": wname, "steps": 20, "value": zones * 20 / (sum(r["step_ms"]) / 1e3),
               "ms_per_step": sum(r["step_ms"]) / 20, "launches_per_step": r["launches_per_step"],
               "riemann_iters_per_solve": r["iters_per_solve"],
               "step": "the fused unsplit step with piecewise-parabolic reconstruction"}
        r = time_device_path(pr, "fp32", 20, args.warmup, flush, riemann_solver=1)
        hllc = {"workload": wname, "steps": 20, "value": zones * 20 / (sum(r["step_ms"]) / 1e3),
                "ms_per_step": sum(r["step_ms"]) / 20, "launches_per_step": r["launches_per_step"],
                "step": "the fused unsplit step with the HLLC solver at every face"}
        r = time_device_path(pr, "fp32", 20, args.warmup, flush, split=1)
        split = {"workload": wname, "steps": 20, "value": zones * 20 / (sum(r["step_ms"]) / 1e3),
                 "ms_per_step": sum(r["step_ms"]) / 20, "launches_per_step": r["launches_per_step"],
                 "riemann_iters_per_solve": r["iters_per_solve"],
                 "step": "dimensionally split: x (or y) sweep, then y (or x) sweep folding in the next CFL dt"}
        prt, rtname = workload("rt1024")
        r = time_device_path(prt, "fp32", 20, args.warmup, flush)
        rt = {"workload": rtname, "steps": 20, "value": prt.nx * prt.ny * 20 / (sum(r["step_ms"]) / 1e3),
              "ms_per_step": sum(r["step_ms"]) / 20, "launches_per_step": r["launches_per_step"],
              "riemann_iters_per_solve": r["iters_per_solve"]}
        if world == 1:  # the oracle beside each variant leg, on a single-GPU run only
            ppm["cpu_oracle"] = cpu_variant(pr, reconstruction=1)
            hllc["cpu_oracle"] = cpu_variant(pr, riemann_solver=1)
            split["cpu_oracle"] = cpu_variant(pr, split=1)
            rt["cpu_oracle"] = cpu_variant(prt, steps=2)
    learned = None
    if args.precision == "fp32":
        model, training = harvest_and_train()
        learned = time_learned(model)
        learned["training"] = training
        model.close()

    t_step = sum(main["step_ms"]) / 1e3
    t_step = max_over_ranks(t_step, world)
    ms_per_step = 1e3 * t_step / args.steps
    value = world * zones * args.steps / t_step
    kern_ms = sum(main["kernel_ms"]) / len(main["kernel_ms"])
    flops_zone = FLOPS_BASE + FLOPS_PER_ITER * SOLVES_PER_ZONE * main["iters_per_solve"]
    achieved = flops_zone * zones / (kern_ms * 1e-3) / 1e12
    peak = ALU_PEAK_TFLOPS[args.precision]
    bytes_zone = 2 * 4 * (4 if args.precision == "fp32" else 8)
    hbm = _peaks().get("hbm_gbs", 6800.0)
    e2e_steps = max(args.steps // 4, 10)
    e2e_value = world * zones * e2e_steps / max_over_ranks(e2e["seconds"], world)
    var_value = zones * len(var["step_ms"]) / (sum(var["step_ms"]) / 1e3)

    if rank != 0:
        return
    line = {
        "metric": "zone-updates/s (cells x steps / s) of the unsplit CTU step",
        "value": value,
        "unit": "zone-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded initial conditions)",
        "config": {"workload": wname, "nx": pr.nx, "ny": pr.ny, "gamma": pr.gamma, "cfl": pr.cfl,
                   "precision": args.precision + ("+fp64 energy recovery" if args.precision == "fp32" else ""),
                   "step": "ghost cells (boundary map) + CTU step + CFL dt of the new state, one fused launch",
                   "l2": "flushed (256 MB write) before every timed step; per-step CUDA events",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": "ctu_step_fused_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": ALU_PEAK_SOURCE[args.precision],
                     "flops_per_zone": flops_zone, "kernel_ms": kern_ms,
                     "hbm_gbs": bytes_zone * zones / (kern_ms * 1e-3) / 1e9, "hbm_frac_of_measured": None,
                     "traffic": None, "traffic_note": None},
        "cpu_baseline": None,
        "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"], "call": "hydro_step_host_chained"},
        "gpu_launches": main["launches_per_step"] * args.steps,
        "clocks": clk.summary(),
        "variants": {other: {"value": var_value, "ms_per_step": 1e3 / var_value * zones,
                             "speedup_of_" + args.precision: value / world / var_value if args.precision == "fp32"
                             else var_value / (value / world)}},
        "riemann_iters_per_solve": main["iters_per_solve"],
        "fp32_error": accuracy,
        "ensemble": ens,
        "rayleigh_taylor": rt,
        "split_variant": split,
        "hllc_variant": hllc,
        "ppm_variant": ppm,
        "learned_proposal": learned,
    }
    line["roofline"]["hbm_frac_of_measured"] = line["roofline"]["hbm_gbs"] / hbm
    if args.precision == "fp32" and wname == "kh_1024x1024_periodic":
        if kernel_sources_sha256() == TRAFFIC_CAPTURE["sources_sha256"]:
            line["roofline"]["traffic"] = TRAFFIC_CAPTURE["bytes_per_launch"]
            line["roofline"]["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch; "
                                                "the new state stays in L2 and is written back after the launch")
            # the bound that binds: the kernel is issue-bound (share of cycles in which a warp instruction
            # issues, from the same capture), far from both the FP32 ALU and the HBM ceilings
            line["roofline"]["issue_active_ncu"] = TRAFFIC_CAPTURE["issue_active"]
            line["roofline"]["warp_instructions_per_launch_ncu"] = TRAFFIC_CAPTURE["warp_instructions"]
        else:
            line["roofline"]["traffic_note"] = "kernel sources changed since the last ncu capture"

    if world == 1:
        line["cpu_baseline"] = cpu_baseline(pr)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank, local):
    """The FP64 CPU oracle on the host cores: each timed step is one whole oracle step of the workload
    (if that is too slow for the run to end within a few minutes, a centred window of it)."""
    if rank != 0:
        return
    import oracle
    from oracle import build as obuild
    obuild.build()
    pr, wname = workload(args.workload)
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    oracle.fill_ghost(p, U)
    # probe one step to size the sample
    t0 = time.perf_counter()
    V = U.copy()
    oracle.step(p, V, oracle.cfl_dt(p, V))
    one = time.perf_counter() - t0
    budget = 150.0
    sample = f"whole {pr.nx}x{pr.ny} steps"
    if one * (args.steps + args.warmup) > budget:
        # centred window whose step fits the budget; its outer ng cells act as its ghost cells
        frac = budget / (one * (args.steps + args.warmup))
        w = max(64, int(pr.nx * np.sqrt(frac)) // 8 * 8)
        j0 = (pr.ny - w) // 2 + pr.ng
        i0 = (pr.nx - w) // 2 + pr.ng
        U = np.ascontiguousarray(U[:, j0 - pr.ng:j0 + w + pr.ng, i0 - pr.ng:i0 + w + pr.ng])
        dx = 1.0 / pr.nx
        p = oracle.params(w, w, xmax=w * dx, ymax=w * dx, gamma=pr.gamma, cfl=pr.cfl)
        sample = f"{w}x{w} centred window steps (window halo as ghost cells)"
    zones = p.nx * p.ny
    for _ in range(args.warmup):
        oracle.step(p, U, oracle.cfl_dt(p, U))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(p, U, oracle.cfl_dt(p, U))
    el = time.perf_counter() - t0
    value = zones * args.steps / el
    line = {
        "impl": "reference",
        "metric": "zone-updates/s (cells x steps / s) of the unsplit CTU step",
        "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded initial conditions)",
        "config": {"workload": wname, "nx": pr.nx, "ny": pr.ny, "gamma": pr.gamma, "cfl": pr.cfl,
                   "precision": "fp64", "step": "oracle dt + oracle CTU step (CPU)"},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="kh1024")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
