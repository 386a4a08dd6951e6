"""Benchmark: Sternheimer solves/s and chi0bar applications/s at 1e-8 residual on one GB300.

Workload (the medium configuration): cubic cell L = 20 bohr, FFT grid 64^3, plane-wave cutoff
|G|^2 <= 25 bohr^-2 (16,879 plane waves, 8,440 stored at Gamma), 32 Gaussian-well atoms with s and
p Kleinman-Bylander projectors (128 projectors), 64 occupied orbitals (computed by the library),
128 orthonormal seeded perturbations. One step is one pass of the whole hot path over that block:
wdf_pdep_davidson with one iteration, i.e. v^1/2, dV in real space, right-hand sides, the
64 x 128 = 8,192 Sternheimer solves to ||b - A x|| <= 1e-8 ||b||, the density response, v^1/2 and
the Rayleigh-Ritz step of PDEP (subspace matrix, FP64 eigensolve, Ritz residuals).

Timing: W warm-up steps, then K steps bracketed by barriers and device synchronisation, CUDA events
on the library's stream; L2 is flushed (256 MiB write) before every step and the step's working
set (~10 GB) exceeds L2 anyway. The e2e figure repeats the step through the same C ABI with host
buffers (host-to-device copy of the perturbations and device-to-host copy of the eigenpairs
inside the timed region). Multi-GPU: the path shards by perturbation blocks with no exchange, so
each rank runs its own block (weak scaling) and rank 0 reports the total.

--impl reference times the FP64 CPU oracle instead (a bounded sample of the same workload).
"""

from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "medium"
NPERT = 128
NEIG = 64
METRIC = "sternheimer_solves_per_s_at_1e-8"
# the workload both arms report in config.workload (the reference arm times a bounded sample of it)
WORKLOAD_DESC = ("medium: L=20 bohr, 64^3 grid, |G|^2<=25, 8440 stored PWs, 32 atoms (128 KB projectors), "
                 "64 occupied, 128 perturbations per GPU, PDEP 64 eigenpairs, one Davidson iteration per step")
# kernel class timed for the roofline, per precision: (class, bound). The per-plane FFT kernel
# keeps its data on chip (its HBM traffic is the column buffer only): its limit is arithmetic.
ROOFLINE_KERNEL = {"mixed_df": ("plane_vloc:32", "alu"), "mixed": ("plane_vloc:32", "alu"), "fp64": ("plane_vloc:64", "alu")}
# arithmetic peaks: FP32 from unit counts and clock (152 SMs x 128 lanes x 2 flop x 2.07 GHz);
# FP64 from a measured FMA loop on this GPU (the FP64 unit count is not published)
ALU_PEAK_TFLOPS = {"mixed_df": 152 * 128 * 2 * 2.07e9 / 1e12, "mixed": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 1.19}
ALU_PEAK_SOURCE = {"mixed_df": "FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                   "mixed": "FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                   "fp64": "FP64: measured FMA loop on GB300, 1.19 TFLOP/s"}


# DRAM bytes per (pair, z plane) unit of the FP32 V_loc plane kernel on the medium system, per
# kernel variant (the one chosen at setup, wdf_plane_variant), from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum over the units of the captured launch; see
# profiles/); traffic grows in proportion to the units launched. A variant without a capture of
# its current code reports null.
PLANE64_DRAM_BYTES_PER_UNIT = {
    1: (210.873088e6 + 167.385088e6) / 32768,  # k_plane_reg<64>: 32,768 units
    5: (210.877440e6 + 149.595648e6) / 32768,  # k_plane_pipe<15>: 32,768 units
}


def plane_flops(system, npair: int) -> float:
    """FFT flops (5 n log2 n per complex line) of one V_loc plane launch over npair pairs.

    Per pair and z plane: n2 inverse transforms of the occupied n1 columns, n1 inverse transforms
    of every row, the real V_loc product, and the same transforms forward.
    """
    import math

    n1, n2, n3 = system.grid
    full = np.concatenate([system.miller, -system.miller[1:]])
    nx = len({int(a) % n1 for a in full[:, 0]})
    line = lambda n: 5.0 * n * math.log2(n)  # noqa: E731
    per_plane = 2.0 * (nx * line(n2) + n2 * line(n1)) + 2.0 * n1 * n2
    return per_plane * n3 * npair
UNIT = "solves/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1862.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(system_name: str, nsolve_target: int = 64):
    """Time the FP64 oracle on one perturbation (all occupied orbitals) of the workload."""
    from oracle import dfpt, hamiltonian

    s = synth.make_system(system_name)
    H = hamiltonian.Hamiltonian(s)
    t0 = time.time()
    w, psi = H.ground_state(s.nocc, tol=1e-6)
    t_gs = time.time() - t0
    R = dfpt.Response(H, w, psi)
    phi = synth.make_perturbations(s, 1, 0)
    return s, R, phi, t_gs


def rank_block_seed(rank: int) -> int:
    """Seed of the perturbation block a rank owns (blocks are independent: no exchange)."""
    return 1000 + rank


def reduce_step_times(times, device=None):
    """Max over ranks of each per-step time (the slowest rank sets the job's pace)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(world: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample, one perturbation per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s, R, phi, t_gs = oracle_sample(WORKLOAD)
    times = []
    nsolve = s.nocc
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        o = R.apply(phi, tol=1e-8)
        dt = time.time() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = nsolve / (ms * 1e-3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "precision": "fp64 (CPU oracle)", "cg_tol": 1e-8,
                   "sample": "1 perturbation (all occupied orbitals) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle",
                         "sample": f"1 perturbation x {nsolve} occupied orbitals = {nsolve} Sternheimer solves per step (FP64 numpy/scipy oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cg_iters_per_solve": float(np.mean(o["iters"])),
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2607_14025_gb300 import build as wbuild
    from paper_2607_14025_gb300 import wdf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        wbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    s = synth.make_system(WORKLOAD)
    # each rank applies chi0bar to its own seeded perturbation block (weak scaling)
    phi_h = synth.make_perturbations(s, NPERT, rank_block_seed(rank))
    t_setup = time.perf_counter()
    ctx = wdf.Context(s, precision=args.precision, cg_tol=1e-8, stream=stream.cuda_stream, device=local,
                      max_batch=args.max_batch)
    t_setup = time.perf_counter() - t_setup
    eps, _ = ctx.orbitals()
    def train_learned():
        # train on other seeds of the same system family (the benchmarked system is seed 0)
        t_tr = time.perf_counter()
        fam = [wdf.Context(synth.make_system(dataclasses.replace(synth.spec(WORKLOAD), seed=k)), precision=args.precision, cg_tol=1e-8,
                           stream=stream.cuda_stream, device=local) for k in range(1, args.train_systems + 1)]
        model, ts = wdf.train_preconditioner(fam, npert=args.train_npert, steps=args.train_steps, seed=12345)
        for c in fam:
            c.close()
        ctx.set_model(model)
        return {"systems": f"{WORKLOAD} family, seeds 1..{args.train_systems} (benchmarked system: seed 0)",
                "perturbations_per_system": args.train_npert, "samples": ts.nsamples, "adam_steps": ts.steps,
                "loss_first": ts.loss_first, "loss_last": ts.loss_last, "train_ms": ts.ms,
                "wall_s_incl_ground_states": time.perf_counter() - t_tr}

    train_info = train_learned() if args.precond == "learned" else None
    phi_d = torch.from_numpy(phi_h).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(phi):
        try:
            return ctx.pdep(NEIG, phi, maxiter=1, tol=1e-8)
        except wdf.NotConverged as e:  # one Davidson iteration never converges all 64 pairs
            return e.result

    if args.profile_step:
        # one warm step, then exactly one step inside cudaProfilerStart/Stop (for ncu
        # --profile-from-start off); prints a short summary and exits
        with torch.cuda.stream(stream):
            step(phi_d)
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.start()
            lam, vec, st = step(phi_d)
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": True, "npert": NPERT, "precision": args.precision, "stats": st.as_dict()}))
        ctx.close()
        return

    # dominant kernel of the step, timed live with CUDA events on its stream
    target, bound = ROOFLINE_KERNEL[args.precision]
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step(phi_d)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        clk = Clocks(local)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stats = []
        ctx.profile_kernel(target)
        nl0 = wdf.launch_count()
        for i in range(args.steps):
            flush.fill_(1.0)
            ev[i][0].record(stream)
            lam, vec, st = step(phi_d)
            ev[i][1].record(stream)
            stats.append(st.as_dict())
        torch.cuda.synchronize(dev)
        clocks = clk.stop()
        launches = (wdf.launch_count() - nl0) / args.steps
        k_launches, k_ms = ctx.profile_read()
        k_blocks = ctx.profile_units()  # (pair, z plane) units of the timed plane launches
        variant = ctx.plane_variant(32 if args.precision != "fp64" else 64)  # plane kernel chosen at setup
        ctx.profile_kernel(None)
        ms_dev = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        # end to end through the C ABI with host buffers
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lam_h, vec_h, st_h = step(phi_h)
        torch.cuda.synchronize(dev)
        ms_e2e = 1e3 * (time.perf_counter() - t0) / args.steps
    learned_line = None
    if args.precond == "tpa" and args.with_learned and world == 1:
        # the same step with the learned preconditioner (trained here, not timed), same protocol
        info = train_learned()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                flush.fill_(1.0)
                step(phi_d)
            torch.cuda.synchronize(dev)
            evl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for i in range(args.steps):
                flush.fill_(1.0)
                evl[i][0].record(stream)
                _, _, stl = step(phi_d)
                evl[i][1].record(stream)
            torch.cuda.synchronize(dev)
        ms_l = sum(a.elapsed_time(b) for a, b in evl) / args.steps
        dl = stl.as_dict()
        learned_line = {"value": job_throughput(world, dl["nsolve"], ms_l), "unit": UNIT, "ms_per_step": ms_l,
                        "cg_iters_per_solve": dl["cg_iters"] / max(1, dl["nsolve"]), "cg_iters_max": dl["cg_iters_max"],
                        "max_residual": dl["max_residual"], "fallbacks_per_step": dl["fallbacks"], "training": info}
    ms_dev, ms_e2e = reduce_step_times([ms_dev, ms_e2e], device=dev)
    nsolve = stats[-1]["nsolve"]
    iters = stats[-1]["cg_iters"] / max(1, nsolve)
    value = job_throughput(world, nsolve, ms_dev)
    e2e = job_throughput(world, nsolve, ms_e2e)
    ctx.close()
    if rank != 0:
        return
    hbm, bf16, src = peaks()
    # algorithmic flops of the dominant kernel over its timed launches (FFT convention: 5 n log2 n
    # per complex line): per (pair, z plane) unit, times the units launched (compaction shrinks
    # the later launches, so the per-launch work varies)
    per_plane_flops = plane_flops(s, 1) / s.grid[2]
    total_flops = per_plane_flops * k_blocks
    avg_ms = k_ms / max(1, k_launches)
    per_launch_flops = total_flops / max(1, k_launches)
    achieved = total_flops / (k_ms * 1e-3) / 1e12 if k_launches else None
    alu_peak = ALU_PEAK_TFLOPS[args.precision]
    # DRAM traffic per launch from the ncu capture (FP32 64^3 kernel only), and the algorithmic
    # bytes: the column-buffer slice read and written (8 B per disk column and z) + V_loc plane
    blocks_per_launch = k_blocks / max(1, k_launches)
    full = np.concatenate([s.miller, -s.miller[1:]])
    ndisk = len({(int(a), int(b)) for a, b, _ in full})
    alg_bytes = blocks_per_launch * 2 * ndisk * 8
    per_unit = PLANE64_DRAM_BYTES_PER_UNIT.get(variant) if args.precision != "fp64" and tuple(s.grid) == (64, 64, 64) else None
    traffic = per_unit * blocks_per_launch if per_unit else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_dev, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "mixed_df": "f32+df64+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "precision": args.precision, "precond": args.precond, "cg_tol": 1e-8,
                   "l2": "flushed (256 MiB write) before each step; working set > L2",
                   "parallelism": f"perturbation blocks x{world}"},
        "chi0_applies_per_s": job_throughput(world, NPERT, ms_dev),
        "cg_iters_per_solve": iters,
        "cg_iters_max": stats[-1]["cg_iters_max"],
        "max_residual": stats[-1]["max_residual"],
        "fallbacks_per_step": stats[-1]["fallbacks"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": NPERT * s.npw_h * 16,
                "d2h_bytes_per_step": NEIG * s.npw_h * 16 + NEIG * 8},
        "gpu_launches": int(round(launches)),
        "roofline": {"kernel": target, "variant": variant, "bound": bound, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": (achieved / alu_peak) if achieved else None, "traffic": traffic,
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launches_per_step": k_launches / args.steps, "ms_per_launch": avg_ms,
                     "share_of_step": k_ms / args.steps / ms_dev, "algorithmic_flops_per_launch": per_launch_flops,
                     "flops_per_pair_plane": per_plane_flops, "pair_planes_per_step": k_blocks / args.steps,
                     "peak_source": ALU_PEAK_SOURCE[args.precision]},
        "clocks": clocks,
        "peaks_source": src,
        "setup_s": t_setup,
        "eps_homo": float(eps[-1]),
    }
    if train_info:
        line["learned_preconditioner"] = train_info
    if learned_line:
        line["learned_preconditioner"] = learned_line
    if args.cpu_baseline:
        sys_o, R, phi1, t_gs = oracle_sample(WORKLOAD)
        t0 = time.time()
        o = R.apply(phi1, tol=1e-8)
        dt = time.time() - t0
        line["cpu_baseline"] = {"value": sys_o.nocc / dt, "unit": UNIT, "cores": cores(), "kind": "oracle",
                                "sample": f"1 perturbation x {sys_o.nocc} occupied = {sys_o.nocc} Sternheimer solves at 1e-8 "
                                          f"(ground state by the oracle's iterative eigensolver, {t_gs:.0f} s, not timed)"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batching(args):
    """The batching workload: 16 seeded systems of uneven size (grids 32^3-80^3, 10-148 occupied
    orbitals) with their perturbation blocks in one wdf_apply_chi0_multi call per step, against
    the same applies one system after another. Host buffers: the timings are end to end."""
    import torch

    from paper_2607_14025_gb300 import build as wbuild
    from paper_2607_14025_gb300 import wdf

    torch.cuda.set_device(0)
    wbuild.build()
    specs = synth.batch_family(args.batch_systems, seed=0)
    t0 = time.perf_counter()
    systems = [synth.make_system(sp) for sp in specs]
    ctxs = [wdf.Context(s, precision=args.precision, cg_tol=1e-8) for s in systems]
    t_setup = time.perf_counter() - t0
    phis = [synth.make_perturbations(s, args.batch_npert, 500 + k) for k, s in enumerate(systems)]
    nsolve = sum(args.batch_npert * s.nocc for s in systems)

    def multi():
        try:
            return wdf.apply_chi0_multi(ctxs, phis)[1]
        except wdf.NotConverged as e:
            return e.result[1]

    for _ in range(args.warmup):
        multi()
    clk = Clocks(0)
    clk.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = multi()
    ms_multi = 1e3 * (time.perf_counter() - t0) / args.steps
    clocks = clk.stop()
    t0 = time.perf_counter()
    for c, p in zip(ctxs, phis):
        try:
            c.apply_chi0(p)
        except wdf.NotConverged:
            pass
    ms_seq = 1e3 * (time.perf_counter() - t0)
    for c in ctxs:
        c.close()
    value = nsolve / (ms_multi * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_multi, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "mixed_df": "f32+df64+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": f"batching: {len(specs)} systems, grids " + ",".join(str(sp.grid[0]) for sp in specs)
                               + f"; {args.batch_npert} perturbations each; {nsolve} solves per step",
                   "precision": args.precision, "cg_tol": 1e-8, "timing": "host clock around the multi-system call (host buffers)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": sum(p.nbytes for p in phis),
                "d2h_bytes_per_step": sum(p.nbytes for p in phis)},
        "sequential": {"value": nsolve / (ms_seq * 1e-3), "ms_per_step": ms_seq},
        "multi_over_sequential": ms_seq / ms_multi,
        "cg_iters_per_solve": sum(x.cg_iters for x in st) / max(1, sum(x.nsolve for x in st)),
        "max_residual": max(x.max_residual for x in st), "setup_s": t_setup, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["wdf", "reference"], default="wdf")
    ap.add_argument("--precision", choices=["mixed_df", "mixed", "fp64"], default="mixed_df")
    ap.add_argument("--max-batch", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-step", action="store_true", help="one warm step, then one step between "
                    "cudaProfilerStart/Stop for ncu --profile-from-start off; no timing line")
    ap.add_argument("--npert", type=int, default=128, help="perturbations per block (default 128)")
    ap.add_argument("--precond", choices=["tpa", "learned"], default="tpa",
                    help="learned: train the MLP preconditioner on other seeds of the family first (not timed)")
    ap.add_argument("--no-learned", dest="with_learned", action="store_false",
                    help="skip the extra timing of the learned preconditioner after the TPA headline")
    ap.add_argument("--workload", choices=["medium", "batching"], default="medium",
                    help="batching: the uneven multi-system workload (its own line; medium is the headline)")
    ap.add_argument("--batch-systems", type=int, default=16)
    ap.add_argument("--batch-npert", type=int, default=64)
    ap.add_argument("--train-systems", type=int, default=4)
    ap.add_argument("--train-npert", type=int, default=8)
    ap.add_argument("--train-steps", type=int, default=600)
    args = ap.parse_args()
    global NPERT, NEIG
    NPERT = args.npert
    NEIG = min(NEIG, NPERT)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batching":
        run_batching(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
