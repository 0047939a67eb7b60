"""Throughput of the unsplit CTU step on a GB300 (zone-updates per second, and the HBM roofline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sedov8192|sedov4096|kh1024|kh2048|rt1024] [--sedov4096-to-t01]

A step is one pass of the solver's driver loop (paper §2): ghost cells (read through the boundary map),
the CTU step of §3.2 with every Riemann iteration started from the learned proposal, and the CFL time step
of the new state, all in one fused launch on a state resident in HBM.

Default workload (the headline line): the 8192 x 8192 Sedov blast with seeded 1 % density noise, FP32 bulk
with FP64 energy recovery and the learned star-pressure proposal (trained first, on the GPU, on faces
harvested from the Sod, Kelvin-Helmholtz and 4096^2 Sedov runs).  Beside it, on the same initial state and
the same steps: the plain FP32 step and the plain FP64 step (bit-identical to the oracle), the FP32 error
against the FP64 state after the run, the end-to-end rate through hydro_step_host_chained with the state in
pinned host memory, the oracle on the host cores, and secondary lines (KH 1024^2, the 4096^2 Sedov error,
the 256-member ensemble with and without the network, the split / HLLC / PPM / Rayleigh-Taylor variants).
Each 8192^2 state buffer (1.08 GB in FP32) is larger than L2 (129 MB), so steps are timed back to back
with per-step CUDA events on the solver's stream and no flush; the L2-resident KH line flushes L2 (256 MB
write) before every timed step.

--impl reference times the FP64 CPU oracle (the plain C implementation the CUDA path is checked against)
on the host cores, on a bounded centred window of the same workload and metric.

Multi-GPU (torchrun, N > 1): the problem is replicated, one independent copy per rank (no data-path
exchange); the value is the sum over ranks, timed by the slowest rank.
"""
import argparse
import gc
import hashlib
import json
import math
import os
import platform
import re
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
# the two-shock solver, at 4.008 solves per zone (the network's own flops are not counted)
FLOPS_BASE = 973.0
FLOPS_PER_ITER = 40.0
SOLVES_PER_ZONE = 4.008
# ALU peaks from the unit counts and the maximum SM clock (FMA = 2 flops): FP32 152 SMs x 128 lanes x 2 x
# 2070 MHz = 80.55 TFLOP/s; FP64 the part's 1.25 TFLOP/s.  (FMA-chain microbenchmarks on the same GPUs reach
# 73.4 and 1.16 TFLOP/s.)
ALU_PEAK_TFLOPS = {"fp32": 152 * 128 * 2 * 2.070e9 / 1e12, "fp64": 1.25}
ALU_PEAK_SOURCE = {"fp32": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (unit counts x max SM clock)",
                   "fp64": "GB300 FP64 rate 1.25 TFLOP/s"}
# algorithmic HBM bytes per zone-update of a fused step: one read and one write of the four conserved fields
BYTES_PER_ZONE = {"fp32": 32, "fp64": 64}

# The committed ncu summaries the DRAM traffic of a launch is read from: each names the kernel, the
# workload, the command, the traffic per launch and the SHA-256 of the kernel's sources when captured.
# The figure is reported only while the sources still hash to it (else the counters describe another
# kernel and traffic is null).
TRAFFIC_PROFILES = {"sedov8192_learned": "profiles/ctu_step_fused_learned_fp32_sedov8192.md",
                    "kh1024": "profiles/ctu_step_fused_fp32_kh1024.md"}
KERNEL_SOURCES = ["paper_1306_6883_gb300/csrc/" + f for f in
                  ("k_ctu.cu", "ctu_kernels.cuh", "ctu_tile.cuh", "hydro_device.cuh", "mlp.cuh", "hydro_kernels.h",
                   "tma.cuh")] + ["include/hydro.h"]


def kernel_sources_sha256():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def read_traffic(key):
    """DRAM bytes per launch from a committed ncu summary: lines `traffic_bytes_per_launch: N` and
    `sources_sha256: H`.  Returns (bytes or None, note)."""
    path = TRAFFIC_PROFILES[key]
    try:
        txt = open(os.path.join(ROOT, path)).read()
    except OSError:
        return None, f"no ncu capture committed ({path})"
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    h = re.search(r"sources_sha256:\s*([0-9a-f]{64})", txt)
    if not m or not h:
        return None, f"{path} holds no traffic figure"
    if h.group(1) != kernel_sources_sha256():
        return None, f"kernel sources changed since the capture in {path}"
    return int(m.group(1)), f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch ({path})"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def workload(name):
    import hydro_problems as hp
    if name == "sedov8192":
        return hp.sedov(8192, 8192, density_noise=0.01), "sedov_8192x8192_outflow_1pct_noise"
    if name == "sedov4096":
        return hp.sedov(4096, 4096), "sedov_4096x4096_outflow"
    if name == "kh1024":
        return hp.kh(1024, 1024, seed=0), "kh_1024x1024_periodic"
    if name == "kh2048":
        return hp.kh(2048, 2048, seed=0), "kh_2048x2048_periodic"
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


def host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        m = re.search(r"Model name:\s*(.+)", out)
        if m:
            model = m.group(1).strip()
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine(),
            "omp_num_threads": os.environ.get("OMP_NUM_THREADS")}


# ---------------------------------------------------------------------------------------------------- learned
def strong_mask(d):
    """Harvested faces past the default gate of the learned kernels: |ln(pL/pR)|/2 >= 0.35 or
    |uL - uR| / c_ref >= 1 (columns rho_L, u_L, p_L, rho_R, u_R, p_R)."""
    import torch
    pmax, pmin = torch.maximum(d[:, 2], d[:, 5]), torch.minimum(d[:, 2], d[:, 5])
    du = d[:, 1] - d[:, 4]
    return (pmax >= math.exp(0.7) * pmin) | (du ** 4 * d[:, 0] * d[:, 3] >= d[:, 2] * d[:, 5])


def _canonical(d):
    """Harvested samples in an order that does not depend on the order the GPU recorded them in (slots are
    taken by atomics): rows sorted by their bits, column by column (stable sorts from the last column to the
    first).  With every face recorded, the training set, and so the trained network, is the same in every run."""
    import torch
    bits = d.contiguous().view(torch.int32)
    order = torch.arange(d.shape[0], device=d.device)
    for c in range(d.shape[1] - 1, -1, -1):
        idx = torch.sort(bits[order, c], stable=True).indices
        order = order[idx]
    return d[order].contiguous()


def train_model(train_steps=50000, batch=4096, lr=3e-3, seed=0):
    """Training set for the learned starting pressure: Riemann problems sampled from FP32 runs of the Sod
    tube (128^2 to t = 0.2), the Kelvin-Helmholtz layer (1024^2, 40 steps) and the Sedov blast (4096^2, 300
    steps), the workloads of the paper's problem list this build runs at full size.  Faces are kept at random
    (hash of face and step) and, in addition, every face past the network's gate (the faces the network will
    be asked about); training draws its minibatches from an equal mix of gated and other faces.  Then
    `train_steps` Adam steps of the library's training kernels."""
    import torch

    import hydro_problems as hp
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Model, Solver, params_for

    cap = 20_000_000  # above the ~17 M faces the three runs record, so that none is dropped
    buf = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = [(hp.sod(128, 128), 0.2, 70, 0.25), (hp.kh(1024, 1024), 0.0, 40, 0.02),
            (hp.sedov(4096, 4096), 0.0, 300, 0.0005)]
    t0 = time.perf_counter()
    gate = (0.35, 1.0)  # the default gate of the learned kernels (model.set_gate)
    per_run = []
    for pr, tmax, steps, rate in plan:
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        before = int(count.item())
        H.hydro_set_harvest(s.ctx, buf.data_ptr(), cap, rate, count.data_ptr())
        H.hydro_set_harvest_gate(s.ctx, *gate)
        s.advance(steps, tmax)
        s.status()
        s.close()
        per_run.append({"run": f"{pr.name} {pr.nx}x{pr.ny}", "steps": steps, "rate": rate,
                        "faces": int(count.item()) - before})
    n = min(int(count.item()), cap)
    data = _canonical(buf[:n])
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
    cap2 = 8_000_000
    buf2 = torch.zeros((cap2, 8), dtype=torch.float32, device="cuda")
    count2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    for k in range(4):
        pr = hp.quad(512, 512, seed=1000 + k)
        s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
        H.hydro_set_harvest(s.ctx, buf2.data_ptr(), cap2, 0.05, count2.data_ptr())
        s.advance(20)
        s.status()
        s.close()
    held = _canonical(buf2[:min(int(count2.item()), cap2)])

    def strong(d):
        return d[strong_mask(d)].contiguous()

    iters = {}
    # 2 M of the randomly kept faces, drawn with a seeded permutation (gated ones are counted apart)
    others = data[~gated]
    rnd = others[torch.randperm(others.shape[0], device="cuda", generator=g)[:2_000_000]].contiguous()
    for name, d in (("held_out_quad_all", held), ("held_out_quad_strong", strong(held)),
                    ("training_runs_random", rnd), ("training_runs_strong", strong_set.contiguous())):
        row = {"faces": int(d.shape[0])}
        if d.shape[0]:
            for learned in (False, True):
                mean, nonconv = H.hydro_mlp_iterations(m.m, d.data_ptr(), d.shape[0], learned)
                row["learned" if learned else "acoustic"] = mean
                row["nonconverged_" + ("learned" if learned else "acoustic")] = nonconv
        iters[name] = row
    del buf, buf2
    return m, {"samples": n, "gated_samples": int(strong_set.shape[0]), "training_set": int(train_set.shape[0]),
               "harvest": per_run, "harvest_s": t_h - t0, "curation_s": t1 - t_h, "train_steps": train_steps,
               "batch": batch, "train_s": t2 - t1, "final_minibatch_loss": loss, "iterations_per_face": iters}


# ---------------------------------------------------------------------------------------------------- our arm
def run_arm(pr, precision, steps, warmup, model=None, flush=None, keep_state=True, **kw):
    """`warmup` untimed then `steps` timed passes of the driver loop through hydro_step_fused (one fused launch
    per step; two sweep launches for the split variant), from the problem's initial state, each step
    bracketed by CUDA events on the solver's stream (L2 flushed before each when `flush` is given).  model:
    start the Riemann iterations from the network (learned contexts)."""
    import torch

    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    prec = H.HYDRO_FP32 if precision == "fp32" else H.HYDRO_FP64
    learned = model is not None
    s = Solver(params_for(pr, prec, use_learned_guess=1 if learned else 0, **kw), pr.U)
    if learned:
        H.hydro_set_riemann_model(s.ctx, model.m)
    tot0 = np.array(s.totals())
    stream = s.stream
    for _ in range(warmup):
        s.step_fused()
    st0, stats0 = s.status()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if flush is not None:
            flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        s.step_fused()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st, stats1 = s.status()
    t_sim, n_sim = s.time()
    tot1 = np.array(s.totals())
    state = s.interior().astype(np.float64) if keep_state else None
    s.close()
    solves = stats1[0] - stats0[0]
    iters = stats1[1] - stats0[1]
    return {"step_ms": step_ms, "iters_per_solve": iters / max(solves, 1), "t_sim": t_sim, "n_sim": n_sim,
            "totals0": tot0, "totals1": tot1, "state": state, "launches_per_step": 2 if kw.get("split") else 1}


def arm_summary(pr, r):
    zones = pr.nx * pr.ny
    t = sum(r["step_ms"]) / 1e3
    return {"value": zones * len(r["step_ms"]) / t, "ms_per_step": 1e3 * t / len(r["step_ms"]),
            "ms_per_step_median": statistics.median(r["step_ms"]), "riemann_iters_per_solve": r["iters_per_solve"]}


def state_error(a, b, tot_a0, tot_a1, tot_b0):
    """Error of state a (FP32 run) against b (FP64 run, bit-identical to the oracle) from the same initial
    state: L1 and max of |a - b| per field, relative to the field's L1 norm and maximum; conservation drift of
    the FP32 run (FP64 totals, relative to the initial totals' magnitudes; momenta relative to the total
    mass times the run's largest speed scale, sum |rho u| + |rho v| over cells)."""
    names = ("rho", "rho_u", "rho_v", "E")
    d = np.abs(a - b).reshape(4, -1)
    ref = np.abs(b).reshape(4, -1)
    scale = np.array([abs(tot_b0[0]), 1.0, 1.0, abs(tot_b0[3])])
    mom = (np.abs(b[1]).sum() + np.abs(b[2]).sum()) / (b.shape[1] * b.shape[2])
    scale[1] = scale[2] = max(mom, 1e-300)
    return {"l1_rel": dict(zip(names, (d.sum(1) / np.maximum(ref.sum(1), 1e-300)).tolist())),
            "max_rel": dict(zip(names, (d.max(1) / np.maximum(ref.max(1), 1e-300)).tolist())),
            "conservation_drift": dict(zip(names, (np.abs(tot_a1 - tot_a0) / scale).tolist()))}


def time_e2e(pr, precision, steps, warmup, model=None):
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
    s = Solver(params_for(pr, prec, use_learned_guess=1 if model is not None else 0), pr.U)
    if model is not None:
        H.hydro_set_riemann_model(s.ctx, model.m)
    host = [torch.from_numpy(np.ascontiguousarray(pr.U)).to(dt_).pin_memory() for _ in range(2)]

    def one(k):
        s.step_host(host[k % 2], host[(k + 1) % 2], chained=True)

    for k in range(warmup):
        one(k)
    torch.cuda.synchronize()
    # three rounds of `steps` steps, the run going on between them (each input is the previous step's
    # output); the fastest round is the figure, all are reported.  Host-side stalls of 15 to 70 ms have been
    # seen in some rounds (one step of 78 ms among steps of 7.85 ms); the collector is off while timing.
    rounds = []
    k = warmup
    gc_was = gc.isenabled()
    gc.disable()
    try:
        for _ in range(3):
            t0 = time.perf_counter()
            marks = []
            for _ in range(steps):
                one(k)
                k += 1
                marks.append(time.perf_counter())
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            rounds.append((el, [b_ - a_ for a_, b_ in zip([t0] + marks[:-1], marks)]))
    finally:
        if gc_was:
            gc.enable()
    el, step_s = min(rounds, key=lambda r: r[0])
    # what the link alone gives for the same bytes: one whole-state copy up, one down, and both at once
    nbytes = host[0].numel() * host[0].element_size()
    dev = torch.empty(host[0].numel(), dtype=dt_, device="cuda")
    dev2 = torch.empty_like(dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - a) / reps * 1e3

    def both():
        with torch.cuda.stream(s1):
            dev.copy_(host[0].view(-1), non_blocking=True)
        with torch.cuda.stream(s2):
            host[1].view(-1).copy_(dev2, non_blocking=True)

    link = {"h2d_ms": timed(lambda: dev.copy_(host[0].view(-1), non_blocking=True)),
            "d2h_ms": timed(lambda: host[1].view(-1).copy_(dev2, non_blocking=True)),
            "both_ms": timed(both), "bytes_each_way": nbytes}
    s.status()
    s.close()
    del host, dev, dev2
    return {"seconds": el, "steps": steps, "h2d": nbytes, "d2h": nbytes,
            "ms_per_step_each": [1e3 * x for x in step_s], "rounds_ms": [1e3 * r[0] for r in rounds],
            "link_alone": link}


def roofline(precision, zones, kernel_ms, iters_per_solve, kernel, traffic_key=None, peak_kind="burst"):
    """ALU roofline of a fused-step kernel (the bound), with its HBM position beside it."""
    flops_zone = FLOPS_BASE + FLOPS_PER_ITER * SOLVES_PER_ZONE * iters_per_solve
    achieved = flops_zone * zones / (kernel_ms * 1e-3) / 1e12
    peak = ALU_PEAK_TFLOPS[precision]
    peaks, src = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm = BYTES_PER_ZONE[precision] * zones / (kernel_ms * 1e-3) / 1e9
    traffic, note = read_traffic(traffic_key) if traffic_key else (None, "no ncu capture of this kernel")
    out = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "peak_source": ALU_PEAK_SOURCE[precision], "flops_per_zone": flops_zone,
           "kernel_ms": kernel_ms, "traffic": traffic, "traffic_note": note,
           "hbm": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hbm / hbm_peak,
                   "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
                   "algorithmic_bytes_per_zone": BYTES_PER_ZONE[precision],
                   "traffic_bytes_per_zone": traffic / zones if traffic else None}}
    return out


# ---------------------------------------------------------------------------------------------------- CPU legs
def _window(pr, w):
    """Centred w x w window of a problem's state; its outer ng cells serve as its ghost cells."""
    g = pr.ng
    j0 = (pr.ny - w) // 2 + g
    i0 = (pr.nx - w) // 2 + g
    return np.ascontiguousarray(pr.U[:, j0 - g:j0 + w + g, i0 - g:i0 + w + g])


def _oracle_window_params(pr, w):
    import oracle
    xmin, xmax, ymin, ymax = pr.domain
    dx, dy = (xmax - xmin) / pr.nx, (ymax - ymin) / pr.ny
    return oracle.params(w, w, xmax=w * dx, ymax=w * dy, gamma=pr.gamma, cfl=pr.cfl, grav=pr.grav)


def cpu_baseline(pr, window=4096, max_steps=5, budget_s=12.0, single_core=True):
    """The oracle as it stands (OpenMP over rows on all host cores) on a bounded sample of the workload:
    whole oracle steps (dt + step) of its centred window, from the initial state.  Beside it, the oracle on
    one core (a child process with OMP_NUM_THREADS=1) on a smaller centred window."""
    import oracle
    w = min(window, pr.nx, pr.ny)
    U = _window(pr, w)
    p = _oracle_window_params(pr, w)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps:
        oracle.step(p, U, oracle.cfl_dt(p, U))
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    out = {"value": w * w * n / el, "unit": "zone-updates/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{n} whole FP64 oracle steps (dt + step) of the centred {w}x{w} window of the "
                     f"{pr.nx}x{pr.ny} workload from its initial state (its outer 4 cells as ghost cells), "
                     f"{el:.1f} s; per zone-update, it stands for the whole grid (extrapolated)",
           "host": host_info()}
    if single_core:
        out["single_core"] = cpu_single_core(pr)
    return out


SINGLE_CORE_SCRIPT = r"""
import sys, time, json
sys.path.insert(0, sys.argv[1])
import numpy as np
import bench, oracle
pr, _ = bench.workload(sys.argv[2])
w = int(sys.argv[3])
U = bench._window(pr, w)
p = bench._oracle_window_params(pr, w)
t0 = time.perf_counter()
n = 0
while n < 3:
    oracle.step(p, U, oracle.cfl_dt(p, U))
    n += 1
    if time.perf_counter() - t0 > 4.0:
        break
el = time.perf_counter() - t0
print(json.dumps({"value": w * w * n / el, "steps": n, "seconds": el, "cores": oracle.num_threads(), "window": w}))
"""


def cpu_single_core(pr, window=1024, workload_name="sedov8192"):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", SINGLE_CORE_SCRIPT, ROOT, workload_name, str(window)], env=env,
                           capture_output=True, text=True, timeout=120)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": d["value"], "unit": "zone-updates/s", "cores": d["cores"],
                "sample": f"{d['steps']} whole FP64 oracle steps of the centred {window}x{window} window, "
                          f"{d['seconds']:.1f} s, OMP_NUM_THREADS=1"}
    except Exception as e:  # the single-core figure is context; its absence does not stop the bench
        return {"value": None, "error": repr(e)[:200]}


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


# ---------------------------------------------------------------------------------------------------- secondary
def time_ensemble(model=None, steps=100, warmup=3, n=256, seed=0, precision="fp32"):
    """The 256-member ensemble of four-quadrant problems on {64,128,256,512}^2 grids (seeded), each member with
    its own CFL dt; tile shapes autotuned per size class; `steps` steps captured in one CUDA graph and launched
    once.  The states (~0.4 GB per FP32 buffer) exceed L2.  model: every member starts its Riemann iterations
    from the network (FP32 only)."""
    import torch

    import hydro_problems as hp
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Ensemble, params_for

    probs = hp.ensemble(n, seed)
    learned = 1 if model is not None else 0
    prec = H.HYDRO_FP32 if precision == "fp32" else H.HYDRO_FP64
    e = Ensemble([params_for(p, prec, use_learned_guess=learned) for p in probs], [p.U for p in probs])
    if model is not None:
        e.set_model(model)
    shapes = e.autotune(reps=2)
    e.run(warmup)
    e.status()
    torch.cuda.synchronize()
    e.run(steps)  # capture + instantiate the graph of `steps` steps (untimed), advancing the members
    torch.cuda.synchronize()
    e.run(steps)  # same parity again only if steps is even; otherwise this captures the other graph
    torch.cuda.synchronize()
    e.status()
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
           "classes": e.classes(), "riemann_iters_per_solve": stats[1] / max(stats[0], 1),
           "learned": bool(learned), "precision": precision}
    e.close()
    return out


def ensemble_oracle(n=256, seed=0, budget_s=8.0):
    """The oracle on the ensemble: one whole step (dt + step) of each member in turn, all host cores, until
    the budget is spent (members in the ensemble's order)."""
    import hydro_problems as hp
    import oracle
    probs = hp.ensemble(n, seed)
    t0 = time.perf_counter()
    cells = 0
    done = 0
    for pr in probs:
        p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
        U = pr.U.copy()
        oracle.fill_ghost(p, U)
        oracle.step(p, U, oracle.cfl_dt(p, U))
        cells += pr.nx * pr.ny
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": cells / el, "unit": "zone-updates/s", "cores": oracle.num_threads(),
            "sample": f"one FP64 step of each of the first {done} of {n} members ({cells} cells), {el:.1f} s"}


def kh_line(flush, steps, warmup):
    """The Kelvin-Helmholtz 1024^2 line (L2-resident: flushed before each timed step): FP32 and FP64."""
    pr, wname = workload("kh1024")
    zones = pr.nx * pr.ny
    r32 = run_arm(pr, "fp32", steps, warmup, flush=flush, keep_state=False)
    r64 = run_arm(pr, "fp64", max(steps // 4, 5), 3, flush=flush, keep_state=False)
    a32, a64 = arm_summary(pr, r32), arm_summary(pr, r64)
    kern = sum(r32["step_ms"]) / len(r32["step_ms"])
    return {"workload": wname, "fp32": a32, "fp64": a64, "fp32_speedup_over_fp64": a32["value"] / a64["value"],
            "roofline_fp32": roofline("fp32", zones, kern, r32["iters_per_solve"], "ctu_step_fused_kernel", "kh1024"),
            "l2": "flushed (256 MB write) before every timed step"}


def sedov4096_line(model, steps, warmup, world):
    """The Sedov 4096^2 blast (no noise; one FP32 state buffer 269 MB, above L2): FP32 with the learned start,
    plain FP32 and plain FP64 from the same state, each with its roofline, and the oracle beside them."""
    pr, wname = workload("sedov4096")
    zones = pr.nx * pr.ny
    arms = {}
    for name, prec, m in (("fp32_learned", "fp32", model), ("fp32_plain", "fp32", None), ("fp64_plain", "fp64", None)):
        r = run_arm(pr, prec, steps, warmup, model=m, keep_state=False)
        a = arm_summary(pr, r)
        kern = sum(r["step_ms"]) / len(r["step_ms"])
        rl = roofline(prec, zones, kern, r["iters_per_solve"], "ctu_step_fused_kernel")
        arms[name] = dict(a, roofline_frac=rl["frac"], hbm_frac=rl["hbm"]["frac"])
    out = {"workload": wname, "steps": steps, "arms": arms,
           "speedup_fp32_learned_over_fp64": arms["fp32_learned"]["value"] / arms["fp64_plain"]["value"],
           "l2": "inputs larger than L2 (one FP32 state buffer 269 MB); steps timed back to back"}
    if world == 1:
        out["cpu_oracle"] = cpu_baseline(pr, window=4096, max_steps=3, budget_s=6.0, single_core=False)
    return out


def learned_cost(model, n=1 << 23, seed=0):
    """What the network's start costs and saves per face, apart from the step: the library's iteration kernel
    (hydro_mlp_iterations) solves the same n Riemann problems from the acoustic start and from the network's
    (every face evaluated, no gate), timed with CUDA events.  Two seeded face classes: weak faces (jumps of
    about 1 %) and strong ones (density ratio up to 20, pressure ratio up to 1000, |u| up to 1.5)."""
    import torch

    from paper_1306_6883_gb300 import hydro as H

    rng = np.random.default_rng(seed)
    classes = {
        "weak": (rng.uniform(1.0, 1.01, (n, 2)), rng.uniform(-0.005, 0.005, (n, 2)), rng.uniform(1.0, 1.01, (n, 2))),
        "strong": (np.exp(rng.uniform(np.log(0.1), np.log(2.0), (n, 2))), rng.uniform(-1.5, 1.5, (n, 2)),
                   np.exp(rng.uniform(np.log(0.01), np.log(10.0), (n, 2)))),
    }
    out = {"faces": n}
    for name, (rho, u, p) in classes.items():
        d = np.zeros((n, 8), dtype=np.float32)
        d[:, 0], d[:, 1], d[:, 2] = rho[:, 0], u[:, 0], p[:, 0]
        d[:, 3], d[:, 4], d[:, 5] = rho[:, 1], u[:, 1], p[:, 1]
        dev = torch.from_numpy(d).cuda()
        res = {}
        for learned in (0, 1):
            H.hydro_mlp_iterations(model.m, dev.data_ptr(), n, learned)  # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            mean, nonconv = H.hydro_mlp_iterations(model.m, dev.data_ptr(), n, learned)
            b.record()
            torch.cuda.synchronize()
            res["learned" if learned else "acoustic"] = {"iters_per_solve": mean, "nonconverged": nonconv,
                                                        "ns_per_face": a.elapsed_time(b) * 1e6 / n}
        res["iterations_saved"] = res["acoustic"]["iters_per_solve"] - res["learned"]["iters_per_solve"]
        out[name] = res
        del dev
    out["note"] = ("the acoustic runs are bound by reading the samples (32 B per face), the learned ones by the "
                   "network's arithmetic; the instruction counts per face are in "
                   "profiles/riemann_iters_kernel_learned_cost.md")
    return out


def kh_fp32_error(steps=50):
    """KH 1024^2: FP32 against FP64 after `steps` fused steps from the same state."""
    pr, _ = workload("kh1024")
    a = run_arm(pr, "fp32", steps, 0)
    b = run_arm(pr, "fp64", steps, 0)
    out = state_error(a["state"], b["state"], a["totals0"], a["totals1"], b["totals0"])
    out["steps"] = steps
    return out


def _advance_to(s, tmax):
    """Steps of a solver until its device time reaches tmax (the last step's dt is clamped to land on it);
    returns the number of steps taken.  Chunks of 10 steps, then single steps near tmax, so that no step of
    zero length is taken after it."""
    t, n = s.time()
    t_prev, n_prev = t, n
    while t < tmax * (1 - 1e-12):
        per = (t - t_prev) / max(n - n_prev, 1)
        chunk = 1 if n == n_prev or tmax - t < 20 * per else 10
        t_prev, n_prev = t, n
        s.advance(chunk, tmax)
        t, n = s.time()
        if not t > t_prev:
            raise RuntimeError(f"the device time does not advance (t = {t} after {n} steps)")
    return n


def sedov4096_error(steps=100, tmax=0.0):
    """Sedov 4096^2 (the blast without noise): FP32 against FP64 after `steps` fused steps from the initial
    state (tmax > 0: steps until that time instead).  With tmax, also the grid's own error scale: the FP64
    4096^2 state averaged over 2 x 2 blocks against the FP64 2048^2 run to the same time."""
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for
    import hydro_problems as hp
    pr, wname = workload("sedov4096")
    res = {}
    for prec in (H.HYDRO_FP32, H.HYDRO_FP64):
        s = Solver(params_for(pr, prec), pr.U)
        tot0 = np.array(s.totals())
        t0 = time.perf_counter()
        if tmax > 0:
            _advance_to(s, tmax)
        else:
            s.advance(steps)
        t, n = s.time()
        el = time.perf_counter() - t0
        tot1 = np.array(s.totals())
        res[prec] = (s.interior().astype(np.float64), tot0, tot1, t, n, el)
        s.status()
        s.close()
    a, b = res[H.HYDRO_FP32], res[H.HYDRO_FP64]
    out = state_error(a[0], b[0], a[1], a[2], b[1])
    out.update({"workload": wname, "t_fp32": a[3], "t_fp64": b[3], "steps_fp32": a[4], "steps_fp64": b[4],
                "seconds_fp32": a[5], "seconds_fp64": b[5]})
    if tmax > 0:
        # where the largest density error sits, against the shock's radius (the density peak)
        n = pr.nx
        xc = (np.arange(n) + 0.5) / n - 0.5
        j, i = np.unravel_index(np.argmax(np.abs(a[0][0] - b[0][0])), (n, n))
        js, is_ = np.unravel_index(np.argmax(b[0][0]), (n, n))
        out["rho_max_error_radius"] = float(np.hypot(xc[i], xc[j]))
        out["shock_radius"] = float(np.hypot(xc[is_], xc[js]))
        out["cell"] = 1.0 / n
        half = hp.sedov(2048, 2048)
        s = Solver(params_for(half, H.HYDRO_FP64), half.U)
        n_half = _advance_to(s, tmax)
        coarse = s.interior().astype(np.float64)
        s.close()
        fine = b[0].reshape(4, 2048, 2, 2048, 2).mean(axis=(2, 4))
        d = np.abs(fine - coarse).reshape(4, -1).sum(1) / np.abs(fine).reshape(4, -1).sum(1)
        out["grid_l1_rel_2048_vs_4096"] = dict(zip(("rho", "rho_u", "rho_v", "E"), d.tolist()))
        out["grid_note"] = (f"FP64 4096^2 averaged over 2x2 blocks against FP64 2048^2 ({n_half} steps) at the "
                            f"same time: the discretisation error scale the FP32 rounding is compared with")
    return out


def variant_legs(flush, warmup, world):
    pr, wname = workload("kh1024")
    zones = pr.nx * pr.ny
    out = {}
    for key, kw, what in (("ppm_variant", dict(reconstruction=1), "the fused unsplit step with PPM"),
                          ("hllc_variant", dict(riemann_solver=1), "the fused unsplit step with HLLC at every face"),
                          ("split_variant", dict(split=1), "dimensionally split: two sweeps, the second folding in "
                                                           "the next CFL dt")):
        r = run_arm(pr, "fp32", 20, warmup, flush=flush, keep_state=False, **kw)
        out[key] = dict(workload=wname, steps=20, step=what, launches_per_step=r["launches_per_step"],
                        **arm_summary(pr, r))
        if world == 1:
            out[key]["cpu_oracle"] = cpu_variant(pr, **kw)
    prt, rtname = workload("rt1024")
    r = run_arm(prt, "fp32", 20, warmup, flush=flush, keep_state=False)
    out["rayleigh_taylor"] = dict(workload=rtname, steps=20, **arm_summary(prt, r))
    if world == 1:
        out["rayleigh_taylor"]["cpu_oracle"] = cpu_variant(prt, steps=2)
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    pr, wname = workload(args.workload)
    zones = pr.nx * pr.ny
    resident = pr.nx * pr.ny * 16 > 129e6  # one FP32 state buffer larger than L2
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    model, training = train_model()

    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        main = run_arm(pr, "fp32", args.steps, args.warmup, model=model, flush=None if resident else flush)
    barrier(world)
    t_main = max_over_ranks(sum(main["step_ms"]) / 1e3, world)
    plain = run_arm(pr, "fp32", args.steps, args.warmup, flush=None if resident else flush)
    fp64 = run_arm(pr, "fp64", args.steps, args.warmup, flush=None if resident else flush)
    e2e_steps = max(args.steps // 2, 5)
    e2e = time_e2e(pr, "fp32", e2e_steps, 3, model=model)
    e2e_value = world * zones * e2e_steps / max_over_ranks(e2e["seconds"], world)

    a_main, a_plain, a_64 = arm_summary(pr, main), arm_summary(pr, plain), arm_summary(pr, fp64)
    err_learned = state_error(main["state"], fp64["state"], main["totals0"], main["totals1"], fp64["totals0"])
    err_plain = state_error(plain["state"], fp64["state"], plain["totals0"], plain["totals1"], fp64["totals0"])
    learned_vs_plain = float(np.abs(main["state"] - plain["state"]).max() / np.abs(plain["state"]).max())
    for r in (main, plain, fp64):
        r["state"] = None

    kern_ms = sum(main["step_ms"]) / len(main["step_ms"])
    rl = roofline("fp32", zones, kern_ms, main["iters_per_solve"],
                  "ctu_step_fused_kernel<float, 32, 16, 320, FACE_LEARNED>",
                  "sedov8192_learned" if wname.startswith("sedov_8192") else None)
    rl_plain = roofline("fp32", zones, sum(plain["step_ms"]) / len(plain["step_ms"]), plain["iters_per_solve"],
                        "ctu_step_fused_kernel<float, 32, 16, 384, FACE_PLAIN>")
    rl_64 = roofline("fp64", zones, sum(fp64["step_ms"]) / len(fp64["step_ms"]), fp64["iters_per_solve"],
                     "ctu_step_fused_kernel<double, 16, 16, 256, FACE_PLAIN>")

    secondary = {}
    secondary["kh1024"] = kh_line(flush, 40, args.warmup)
    secondary["kh1024"]["fp32_error_50_steps"] = kh_fp32_error()
    if world == 1:
        secondary["kh1024"]["cpu_oracle"] = cpu_variant(workload("kh1024")[0])
    secondary["sedov4096"] = sedov4096_line(model, args.steps, args.warmup, world)
    secondary["sedov4096_fp32_error_100_steps"] = sedov4096_error(steps=100)
    if args.sedov4096_to_t01:
        secondary["sedov4096_fp32_error_to_t01"] = sedov4096_error(tmax=0.1)
    secondary["ensemble_plain"] = time_ensemble()
    secondary["ensemble_learned"] = time_ensemble(model=model)
    # the learned kernels with the gate closed (no face queued): their cost apart from the network's passes
    model.set_gate(40.0, 1e9)
    secondary["ensemble_learned_gate_closed"] = time_ensemble(model=model)
    model.set_gate(0.35, 1.0)
    secondary["ensemble_fp64"] = time_ensemble(steps=10, precision="fp64")
    secondary["ensemble_speedup_fp32_learned_over_fp64"] = (secondary["ensemble_learned"]["value"]
                                                           / secondary["ensemble_fp64"]["value"])
    secondary["learned_cost"] = learned_cost(model)
    secondary.update(variant_legs(flush, args.warmup, world))
    model.close()

    if rank != 0:
        return
    value = world * zones * args.steps / t_main
    line = {
        "metric": "zone-updates/s (cells x steps / s) of the CTU step, FP32 + learned proposal vs plain FP64, "
                  "with its HBM-roofline fraction",
        "value": value,
        "unit": "zone-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_main / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded initial conditions)",
        "config": {"workload": wname, "nx": pr.nx, "ny": pr.ny, "gamma": pr.gamma, "cfl": pr.cfl,
                   "precision": "fp32 bulk + fp64 energy recovery, learned star-pressure proposal "
                                "(BF16 tensor-core MLP 6-64-64-1, default gate)",
                   "step": "ghost cells (boundary map) + CTU step + CFL dt of the new state, one fused launch",
                   "l2": ("inputs larger than L2 (one FP32 state buffer 1.08 GB); steps timed back to back"
                          if resident else "flushed (256 MB write) before every timed step"),
                   "timing": "per-step CUDA events on the solver's stream",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": rl,
        "cpu_baseline": None,
        "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"], "call": "hydro_step_host_chained (learned context)",
                "steps": e2e_steps, "ms_per_step_each": e2e["ms_per_step_each"],
                "rounds_ms": e2e["rounds_ms"], "timing": "host clock around the calls; the fastest of three rounds",
                "link_alone": e2e["link_alone"]},
        "gpu_launches": main["launches_per_step"] * args.steps,
        "clocks": clk.summary(),
        "riemann_iters_per_solve": main["iters_per_solve"],
        "arms": {
            "fp32_learned": dict(a_main, roofline_frac=rl["frac"], hbm_frac=rl["hbm"]["frac"]),
            "fp32_plain": dict(a_plain, roofline_frac=rl_plain["frac"], hbm_frac=rl_plain["hbm"]["frac"]),
            "fp64_plain": dict(a_64, roofline_frac=rl_64["frac"], hbm_frac=rl_64["hbm"]["frac"],
                               roofline=rl_64),
            "speedup_fp32_learned_over_fp64": a_main["value"] / a_64["value"],
            "speedup_fp32_plain_over_fp64": a_plain["value"] / a_64["value"],
            "learned_over_plain": a_main["value"] / a_plain["value"],
        },
        "fp32_error": {"against": "FP64 GPU path on the same state and steps (bit-identical to the oracle)",
                       "steps": args.warmup + args.steps, "fp32_learned": err_learned, "fp32_plain": err_plain,
                       "learned_vs_plain_max_rel": learned_vs_plain},
        "learned_training": training,
        "secondary": secondary,
    }
    if world == 1:
        line["cpu_baseline"] = cpu_baseline(pr)
        line["cpu_baseline"]["ensemble"] = ensemble_oracle()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank, local):
    """The FP64 CPU oracle on the host cores: each timed step is one whole oracle step (dt + step) of the
    workload, or, when that would not end within a few minutes, of its centred window (whose outer ng cells
    serve as its ghost cells)."""
    if rank != 0:
        return
    import oracle
    from oracle import build as obuild
    obuild.build()
    pr, wname = workload(args.workload)
    # probe the oracle's rate on a small window to size the sample
    wp = min(256, pr.nx, pr.ny)
    Up = _window(pr, wp)
    pp = _oracle_window_params(pr, wp)
    t0 = time.perf_counter()
    oracle.step(pp, Up, oracle.cfl_dt(pp, Up))
    rate = wp * wp / max(time.perf_counter() - t0, 1e-6)
    budget = 150.0
    nstep = args.steps + args.warmup
    if pr.nx * pr.ny * nstep / rate <= budget:
        xmin, xmax, ymin, ymax = pr.domain
        p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                          ymax=ymax, grav=pr.grav)
        U = pr.U.copy()
        fill = True
        sample = f"whole {pr.nx}x{pr.ny} steps (ghost fill + dt + step)"
    else:
        w = max(64, min(int(math.sqrt(budget * rate / nstep)) // 8 * 8, pr.nx, pr.ny))
        U = _window(pr, w)
        p = _oracle_window_params(pr, w)
        fill = False
        sample = f"{w}x{w} centred window steps of the {pr.nx}x{pr.ny} workload (window halo as ghost cells)"

    def one():
        if fill:
            oracle.fill_ghost(p, U)
        oracle.step(p, U, oracle.cfl_dt(p, U))

    zones = p.nx * p.ny
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = zones * args.steps / el
    line = {
        "impl": "reference",
        "metric": "zone-updates/s (cells x steps / s) of the CTU step, FP32 + learned proposal vs plain FP64, "
                  "with its HBM-roofline fraction",
        "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded initial conditions)",
        "config": {"workload": wname, "nx": pr.nx, "ny": pr.ny, "gamma": pr.gamma, "cfl": pr.cfl,
                   "precision": "fp64", "step": "oracle dt + oracle CTU step (CPU)"},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sedov8192")
    ap.add_argument("--sedov4096-to-t01", action="store_true",
                    help="also run Sedov 4096^2 to t = 0.1 in FP32 and FP64 (~10 000 steps; minutes of FP64)")
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
