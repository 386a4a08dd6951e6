"""Benchmark: Sternheimer solves/s and chi0bar applications/s at 1e-8 residual on one GB300.

Workload (the precision configuration, the largest that fits one GPU): cubic cell L = 28 bohr,
FFT grid 96^3, plane-wave cutoff |G|^2 <= 25 bohr^-2 (46,297 plane waves, 23,149 stored at
Gamma), 128 Gaussian-well atoms with s and p Kleinman-Bylander projectors (512 projectors), 256
occupied orbitals (computed by the library), a block of 512 orthonormal seeded perturbations.
The block is applied in 8 chunks of 64 (a whole block of 512 x 256 solves would need ~800 GB of
CG workspace); one step is one pass of the whole hot path over one chunk: wdf_pdep_davidson for
64 eigenpairs with one iteration, i.e. v^1/2, dV in real space, right-hand sides, the
64 x 256 = 16,384 Sternheimer solves to ||b - A x|| <= 1e-8 ||b||, the density response, v^1/2
and the Rayleigh-Ritz step of PDEP (subspace matrix, FP64 eigensolve, Ritz residuals). Steps
cycle through the chunks, so 8 steps cover the 512-perturbation block.

The inner CG uses the learned preconditioner (the MLP scale on TPA, with TPA as the fallback of a
stalling solve), trained before the timed region on converged solves of 8 seeded systems of the
96^3 learned family (the same grid and basis with 16 orbitals). Beside it, in the same line: the
same steps with TPA alone, the plain FP64 GPU form on a sample of the same block (the metric's
"vs FP64 GPU"), the medium configuration (64^3, 64 orbitals, 128 perturbations per step, TPA) as a
secondary figure, and the FP64 CPU oracle on a bounded sample (cpu_baseline).

Timing: W warm-up steps, then K steps bracketed by barriers and device synchronisation, CUDA events
on the library's stream; L2 is flushed (256 MiB write) before every step and the step's working
set (~100 GB) exceeds L2 anyway. The e2e figure repeats the steps through the same C ABI with
host buffers (host-to-device copy of the perturbations and device-to-host copy of the eigenpairs
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

METRIC = "sternheimer_solves_per_s_at_1e-8"
UNIT = "solves/s"


@dataclasses.dataclass(frozen=True)
class Workload:
    system: str      # synth spec
    nblock: int      # perturbations of the block per GPU
    chunk: int       # perturbations per step (one Davidson iteration of PDEP on them)
    neig: int        # PDEP eigenpairs
    desc: str        # config.workload of the JSON line
    oracle_system: str  # system the CPU oracle is timed on
    oracle_nv: int   # Sternheimer solves (orbitals of one perturbation) per oracle sample


WORKLOADS = {
    "precision": Workload(
        "precision", 512, 64, 64,
        "precision: L=28 bohr, 96^3 grid, |G|^2<=25, 23149 stored PWs, 128 atoms (512 KB projectors), 256 occupied, "
        "512 perturbations per GPU applied in 8 chunks of 64; one step = one chunk: PDEP 64 eigenpairs, one Davidson "
        "iteration (16384 solves)",
        "precision_reduced", 8),
    # small case of the precision workload for profiler captures: the same 96^3 grid and 23,149-wave
    # layout (so the same kernels and per-unit work) with 8 atoms and 16 orbitals
    "precision_small": Workload(
        "precision_reduced", 32, 32, 16,
        "precision_small: L=28 bohr, 96^3 grid, |G|^2<=25, 23149 stored PWs, 8 atoms (32 KB projectors), 16 occupied, "
        "32 perturbations per step, PDEP 16 eigenpairs, one Davidson iteration per step (512 solves)",
        "precision_reduced", 8),
    "medium": Workload(
        "medium", 128, 128, 64,
        "medium: L=20 bohr, 64^3 grid, |G|^2<=25, 8440 stored PWs, 32 atoms (128 KB projectors), 64 occupied, "
        "128 perturbations per GPU, PDEP 64 eigenpairs, one Davidson iteration per step",
        "medium", 64),
}

# kernel class timed for the roofline, per precision: (class, bound). The per-plane FFT kernel
# keeps its data on chip (its HBM traffic is the column buffer only): its limit is arithmetic.
ROOFLINE_KERNEL = {"mixed_df": ("plane_vloc:32", "alu"), "mixed": ("plane_vloc:32", "alu"), "fp64": ("plane_vloc:64", "alu")}
# arithmetic peaks: FP32 from unit counts and clock (152 SMs x 128 lanes x 2 flop x 2.07 GHz);
# FP64 from a measured FMA loop on this GPU (the FP64 unit count is not published)
ALU_PEAK_TFLOPS = {"mixed_df": 152 * 128 * 2 * 2.07e9 / 1e12, "mixed": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 1.19}
ALU_PEAK_SOURCE = {"mixed_df": "FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                   "mixed": "FP32: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)",
                   "fp64": "FP64: measured FMA loop on GB300, 1.19 TFLOP/s"}


# DRAM bytes per (pair, z plane) unit of the FP32 V_loc plane kernel, per (grid, kernel variant
# chosen at setup), from one ncu capture each on a small case of the same system
# (dram__bytes_read.sum + dram__bytes_write.sum over the units of the captured launch; see
# profiles/); traffic grows in proportion to the units launched. A variant without a capture of
# its current code reports null.
PLANE_DRAM_BYTES_PER_UNIT = {
    (64, 1): (210.873088e6 + 167.385088e6) / 32768,  # k_plane_reg<64>: 32,768 units
    (64, 5): (210.877440e6 + 149.595648e6) / 32768,  # k_plane_pipe<15>: 32,768 units
    (96, 7): (311.997440e6 + 249.979648e6) / 24576,  # k_plane_pipe2<96, 22>: 24,576 units
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


class OracleSample:
    """The FP64 CPU oracle on a bounded sample of a workload: its own ground state (not timed),
    then, per timed sample, one perturbation's right-hand sides for the first ``nv`` occupied
    orbitals (Q over all of them), their Sternheimer solves to 1e-8 and their density."""

    def __init__(self, wl: Workload):
        from oracle import dfpt, hamiltonian

        self.wl = wl
        self.s = synth.make_system(wl.oracle_system)
        H = hamiltonian.Hamiltonian(self.s)
        t0 = time.time()
        w, psi = H.ground_state(self.s.nocc, tol=1e-8)
        self.t_gs = time.time() - t0
        self.R = dfpt.Response(H, w, psi)
        self.nv = min(wl.oracle_nv, self.s.nocc)
        self.x = self.R.vhalf_times(synth.make_perturbations(self.s, 1, 0))

    def run(self):
        """One sample; returns (seconds, solves, mean CG iterations)."""
        vidx = np.arange(self.nv)
        pidx = np.zeros(self.nv, dtype=np.int64)
        t0 = time.time()
        b = self.R.rhs(self.x[pidx], vidx)
        d, iters, _ = self.R.sternheimer(b, vidx, tol=1e-8)
        self.R.density(d, vidx, 1, pidx)
        return time.time() - t0, self.nv, float(np.mean(iters))

    def describe(self) -> str:
        s = self.s
        same = self.wl.oracle_system == self.wl.system
        what = (f"1 perturbation x {self.nv} of {s.nocc} occupied orbitals (Q over all {s.nocc}) = {self.nv} Sternheimer "
                f"solves at 1e-8 with their right-hand sides and density, FP64 numpy/scipy oracle")
        if same:
            return what + f" (oracle ground state {self.t_gs:.0f} s, not timed)"
        return (what + f", on {s.spec.name}: the workload's {s.grid[0]}^3 grid and {s.npw_h}-wave basis with "
                f"{s.spec.natom} atoms and {s.nocc} orbitals, since the oracle's ground state of the full system would take "
                f"hours; its solves project on {s.nocc} instead of 256 orbitals and {s.nproj} instead of 512 projectors, so "
                f"the rate overstates the oracle on the full system (ground state {self.t_gs:.0f} s, not timed)")


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
    """Reference arm: the FP64 CPU oracle on a bounded sample of the workload, one sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS.get(args.workload, WORKLOADS["medium"])
    o = OracleSample(wl)
    times, its = [], []
    for i in range(args.warmup + args.steps):
        dt, nsolve, it = o.run()
        if i >= args.warmup:
            times.append(dt)
            its.append(it)
    ms = 1e3 * sum(times) / len(times)
    value = o.nv / (ms * 1e-3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.desc, "precision": "fp64 (CPU oracle)", "cg_tol": 1e-8,
                   "sample": f"{o.nv} solves per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle", "sample": o.describe()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cg_iters_per_solve": float(np.mean(its)),
    }
    print(json.dumps(line), flush=True)


def roofline_line(s, precision, variant, k_launches, k_ms, k_blocks, steps, ms_dev):
    """The dominant kernel's roofline from its live CUDA-event timing inside the timed region."""
    target, bound = ROOFLINE_KERNEL[precision]
    # algorithmic flops of the kernel over its timed launches (FFT convention: 5 n log2 n per
    # complex line): per (pair, z plane) unit, times the units launched (compaction shrinks the
    # later launches, so the per-launch work varies)
    per_plane_flops = plane_flops(s, 1) / s.grid[2]
    total_flops = per_plane_flops * k_blocks
    avg_ms = k_ms / max(1, k_launches)
    achieved = total_flops / (k_ms * 1e-3) / 1e12 if k_launches else None
    alu_peak = ALU_PEAK_TFLOPS[precision]
    # algorithmic bytes: the column-buffer slice read and written (8 B per disk column and z)
    blocks_per_launch = k_blocks / max(1, k_launches)
    full = np.concatenate([s.miller, -s.miller[1:]])
    ndisk = len({(int(a), int(b)) for a, b, _ in full})
    alg_bytes = blocks_per_launch * 2 * ndisk * 8
    per_unit = PLANE_DRAM_BYTES_PER_UNIT.get((s.grid[0], variant)) if precision != "fp64" else None
    return {"kernel": target, "variant": variant, "bound": bound, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": (achieved / alu_peak) if achieved else None, "traffic": per_unit * blocks_per_launch if per_unit else None,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)", "algorithmic_bytes_per_launch": alg_bytes,
            "launches_per_step": k_launches / steps, "ms_per_launch": avg_ms, "share_of_step": k_ms / steps / ms_dev,
            "algorithmic_flops_per_launch": total_flops / max(1, k_launches), "flops_per_pair_plane": per_plane_flops,
            "pair_planes_per_step": k_blocks / steps, "peak_source": ALU_PEAK_SOURCE[precision]}


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
    wl = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    s = synth.make_system(wl.system)
    # each rank applies chi0bar to its own seeded perturbation block (weak scaling)
    phi_h = synth.make_perturbations(s, wl.nblock, rank_block_seed(rank))
    nch = wl.nblock // wl.chunk
    t_setup = time.perf_counter()
    ctx = wdf.Context(s, precision=args.precision, cg_tol=1e-8, stream=stream.cuda_stream, device=local,
                      max_batch=args.max_batch)
    t_setup = time.perf_counter() - t_setup
    eps, psi = ctx.orbitals()

    def train_learned():
        # train on other seeds of the system's family (the benchmarked system is seed 0); for the
        # precision workload on the learned-preconditioner family at 96^3 (the same grid and basis
        # with 16 orbitals), whose ground states take a second each instead of ~50 s
        t_tr = time.perf_counter()
        if wl.system == "precision":
            specs = [synth.learned_family(k, 96) for k in range(1, args.train_systems + 1)]
            fam_desc = f"learned_family 96^3 (8 atoms, 16 orbitals), seeds 1..{args.train_systems}"
        else:
            specs = [dataclasses.replace(synth.spec(wl.system), seed=k) for k in range(1, args.train_systems + 1)]
            fam_desc = f"{wl.system} family, seeds 1..{args.train_systems} (benchmarked system: seed 0)"
        fam = [wdf.Context(synth.make_system(sp), precision=args.precision, cg_tol=1e-8, stream=stream.cuda_stream, device=local)
               for sp in specs]
        model, ts = wdf.train_preconditioner(fam, npert=args.train_npert, steps=args.train_steps, seed=12345)
        for c in fam:
            c.close()
        ctx.set_model(model)
        return {"systems": fam_desc, "perturbations_per_system": args.train_npert, "samples": ts.nsamples, "adam_steps": ts.steps,
                "loss_first": ts.loss_first, "loss_last": ts.loss_last, "train_ms": ts.ms,
                "wall_s_incl_ground_states": time.perf_counter() - t_tr}

    train_info = train_learned() if args.precond == "learned" else None
    phi_d = torch.from_numpy(phi_h).to(dev)
    chunks_d = [phi_d[k * wl.chunk:(k + 1) * wl.chunk] for k in range(nch)]
    chunks_h = [np.ascontiguousarray(phi_h[k * wl.chunk:(k + 1) * wl.chunk]) for k in range(nch)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(phi):
        try:
            return ctx.pdep(wl.neig, phi, maxiter=1, tol=1e-8)
        except wdf.NotConverged as e:  # one Davidson iteration never converges every pair
            return e.result

    if args.profile_step:
        # one warm step, then exactly one step inside cudaProfilerStart/Stop (for ncu
        # --profile-from-start off); prints a short summary and exits
        with torch.cuda.stream(stream):
            step(chunks_d[0])
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.start()
            lam, vec, st = step(chunks_d[0])
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": True, "workload": args.workload, "chunk": wl.chunk, "precision": args.precision,
                          "stats": st.as_dict()}))
        ctx.close()
        return

    # dominant kernel of the step, timed live with CUDA events on its stream
    target, bound = ROOFLINE_KERNEL[args.precision]
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            flush.fill_(1.0)
            step(chunks_d[i % nch])
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
            lam, vec, st = step(chunks_d[i % nch])
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
        # end to end through the C ABI with host buffers: one pass over the block's chunks
        n_e2e = max(1, min(args.steps, nch))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(n_e2e):
            lam_h, vec_h, st_h = step(chunks_h[i % nch])
        torch.cuda.synchronize(dev)
        ms_e2e = 1e3 * (time.perf_counter() - t0) / n_e2e
    other_line = None
    if args.with_other and world == 1:
        # the same steps with the other preconditioner (the learned one trained here, not timed),
        # same protocol, one pass over the block's chunks
        if args.precond == "tpa":
            info = train_learned()
        else:
            ctx.set_model(None)
            info = None
        nl = max(1, min(args.steps, nch))
        with torch.cuda.stream(stream):
            for i in range(args.warmup):
                flush.fill_(1.0)
                step(chunks_d[i % nch])
            torch.cuda.synchronize(dev)
            evl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
            for i in range(nl):
                flush.fill_(1.0)
                evl[i][0].record(stream)
                _, _, stl = step(chunks_d[i % nch])
                evl[i][1].record(stream)
            torch.cuda.synchronize(dev)
        ms_l = sum(a.elapsed_time(b) for a, b in evl) / nl
        dl = stl.as_dict()
        other_line = {"value": job_throughput(world, dl["nsolve"], ms_l), "unit": UNIT, "ms_per_step": ms_l, "steps": nl,
                      "cg_iters_per_solve": dl["cg_iters"] / max(1, dl["nsolve"]), "cg_iters_max": dl["cg_iters_max"],
                      "max_residual": dl["max_residual"], "fallbacks_per_step": dl["fallbacks"]}
        if info:
            other_line["training"] = info
    ctx.close()
    fp64_line = None
    if args.fp64_npert > 0:
        # the plain FP64 GPU form on a sample of the same block (same orbitals, same CG tolerance)
        with wdf.Context(s, psi=psi, eps=eps, precision="fp64", cg_tol=1e-8, stream=stream.cuda_stream, device=local) as c64:
            sample = chunks_d[0][: args.fp64_npert]
            with torch.cuda.stream(stream):
                c64.apply_chi0(sample)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 2
                e0.record(stream)
                for _ in range(reps):
                    _, _, st64 = c64.apply_chi0(sample)
                e1.record(stream)
                torch.cuda.synchronize(dev)
            ms64 = e0.elapsed_time(e1) / reps
            d64 = st64.as_dict()
        fp64_line = {"value": job_throughput(world, d64["nsolve"], ms64), "unit": UNIT, "ms_per_call": ms64,
                     "sample": f"{args.fp64_npert} perturbations x {s.nocc} orbitals = {d64['nsolve']} solves of the same block, "
                               "chi0bar applications (S1-S8) in plain FP64 on the GPU, cg_tol 1e-8, CUDA events, 1 warm-up + 2 timed",
                     "cg_iters_per_solve": d64["cg_iters"] / max(1, d64["nsolve"]), "max_residual": d64["max_residual"]}
    ms_dev, ms_e2e = reduce_step_times([ms_dev, ms_e2e], device=dev)
    nsolve = stats[-1]["nsolve"]
    iters = stats[-1]["cg_iters"] / max(1, nsolve)
    value = job_throughput(world, nsolve, ms_dev)
    e2e = job_throughput(world, nsolve, ms_e2e)
    secondary = None
    if args.secondary and wl.system != "medium" and world == 1:
        secondary = run_secondary_medium(args, stream, dev, flush)
    if rank != 0:
        return
    hbm, bf16, src = peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_dev, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "mixed_df": "f32+df64+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": wl.desc, "precision": args.precision, "precond": args.precond, "cg_tol": 1e-8,
                   "l2": "flushed (256 MiB write) before each step; working set > L2",
                   "parallelism": f"perturbation blocks x{world}"},
        "chi0_applies_per_s": job_throughput(world, wl.chunk, ms_dev),
        "cg_iters_per_solve": iters,
        "cg_iters_max": stats[-1]["cg_iters_max"],
        "max_residual": stats[-1]["max_residual"],
        "fallbacks_per_step": stats[-1]["fallbacks"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": wl.chunk * s.npw_h * 16,
                "d2h_bytes_per_step": wl.neig * s.npw_h * 16 + wl.neig * 8, "steps": n_e2e},
        "gpu_launches": int(round(launches)),
        "roofline": roofline_line(s, args.precision, variant, k_launches, k_ms, k_blocks, args.steps, ms_dev),
        "clocks": clocks,
        "peaks_source": src,
        "setup_s": t_setup,
        "eps_homo": float(eps[-1]),
    }
    if fp64_line:
        line["fp64_gpu"] = fp64_line
        line["mixed_over_fp64_gpu"] = value / fp64_line["value"]
    if secondary:
        line["medium"] = secondary
    if train_info:
        line["learned_preconditioner"] = {"training": train_info, "fallbacks_per_step": stats[-1]["fallbacks"]}
    if other_line:
        line["learned_preconditioner" if args.precond == "tpa" else "tpa_preconditioner"] = other_line
    if args.cpu_baseline:
        o = OracleSample(wl)
        dt, nv, it = o.run()
        line["cpu_baseline"] = {"value": nv / dt, "unit": UNIT, "cores": cores(), "kind": "oracle", "sample": o.describe()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_secondary_medium(args, stream, dev, flush):
    """The medium configuration with the same step (PDEP, one Davidson iteration over 128
    perturbations), a few steps, as a secondary figure of the line."""
    import torch

    from paper_2607_14025_gb300 import wdf

    wl = WORKLOADS["medium"]
    s = synth.make_system(wl.system)
    phi = torch.from_numpy(synth.make_perturbations(s, wl.nblock, rank_block_seed(0))).to(dev)
    with wdf.Context(s, precision=args.precision, cg_tol=1e-8, stream=stream.cuda_stream, device=dev.index) as c:
        def step():
            try:
                return c.pdep(wl.neig, phi, maxiter=1, tol=1e-8)
            except wdf.NotConverged as e:
                return e.result

        with torch.cuda.stream(stream):
            for _ in range(2):
                flush.fill_(1.0)
                step()
            n = 5
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
            for i in range(n):
                flush.fill_(1.0)
                ev[i][0].record(stream)
                _, _, st = step()
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev) / n
    d = st.as_dict()
    return {"workload": wl.desc, "value": d["nsolve"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": n, "warmup": 2,
            "cg_iters_per_solve": d["cg_iters"] / max(1, d["nsolve"]), "max_residual": d["max_residual"]}


def run_learned(args):
    """The learned-preconditioner protocol: a model trained on converged solves of 32 seeded
    systems of the family (96^3 and 108^3 grids alternating, L = 28 n / 96 bohr, |G|^2 <= 25, the
    reduced precision system's atom density) is applied to 8 held-out seeds; each held-out system
    applies chi0bar to a block of perturbations to 1e-8 with TPA and with the learned scale.
    Reports CG iterations per solve, wall time (CUDA events, one warm-up apply each) and the TPA
    fallbacks."""
    import torch

    from paper_2607_14025_gb300 import build as wbuild
    from paper_2607_14025_gb300 import wdf

    torch.cuda.set_device(0)
    wbuild.build()
    grids = (96, 108)  # 128^3 planes exceed the shared-memory tile of the FP64 plane kernel
    t0 = time.perf_counter()
    train = [wdf.Context(synth.make_system(synth.learned_family(k, grids[k % 2])), precision=args.precision, cg_tol=1e-8)
             for k in range(args.learned_train)]
    t_gs = time.perf_counter() - t0
    model, ts = wdf.train_preconditioner(train, npert=args.train_npert, steps=args.train_steps, seed=12345)
    for c in train:
        c.close()
    rows = []
    tot = {"tpa": [0, 0.0, 0], "learned": [0, 0.0, 0]}  # solves, ms, iterations
    fallbacks = 0
    for k in range(args.learned_train, args.learned_train + args.learned_test):
        s = synth.make_system(synth.learned_family(k, grids[k % 2]))
        phi = torch.from_numpy(synth.make_perturbations(s, args.learned_npert, 700 + k)).cuda()
        row = {"seed": k, "grid": s.grid[0], "nocc": s.nocc, "npw_h": s.npw_h}
        with wdf.Context(s, precision=args.precision, cg_tol=1e-8) as c:
            for name in ("tpa", "learned"):
                c.set_model(model if name == "learned" else None)
                c.apply_chi0(phi)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                _, _, st = c.apply_chi0(phi)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                d = st.as_dict()
                row[name] = {"cg_iters_per_solve": d["cg_iters"] / d["nsolve"], "ms": ms, "max_residual": d["max_residual"],
                             "fallbacks": d["fallbacks"]}
                tot[name][0] += d["nsolve"]
                tot[name][1] += ms
                tot[name][2] += d["cg_iters"]
                if name == "learned":
                    fallbacks += d["fallbacks"]
        rows.append(row)
    value = tot["learned"][0] / (tot["learned"][1] * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": tot["learned"][1], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "mixed_df": "f32+df64+f64", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": f"learned: train seeds 0..{args.learned_train - 1}, held-out seeds {args.learned_train}.."
                               f"{args.learned_train + args.learned_test - 1}, grids 96^3/108^3 alternating, "
                               f"{args.learned_npert} perturbations per held-out system, cg_tol 1e-8",
                   "precision": args.precision},
        "tpa": {"value": tot["tpa"][0] / (tot["tpa"][1] * 1e-3), "unit": UNIT, "ms": tot["tpa"][1],
                "cg_iters_per_solve": tot["tpa"][2] / tot["tpa"][0]},
        "learned": {"value": value, "unit": UNIT, "ms": tot["learned"][1], "cg_iters_per_solve": tot["learned"][2] / tot["learned"][0],
                    "fallbacks": fallbacks},
        "iteration_gain": tot["tpa"][2] / max(1, tot["learned"][2]),
        "time_gain": tot["tpa"][1] / tot["learned"][1],
        "training": {"systems": args.learned_train, "samples": ts.nsamples, "adam_steps": ts.steps, "loss_first": ts.loss_first,
                     "loss_last": ts.loss_last, "train_ms": ts.ms, "ground_states_s": t_gs},
        "systems": rows,
    }
    print(json.dumps(line), flush=True)


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
    ap.add_argument("--precond", choices=["tpa", "learned"], default="learned",
                    help="learned (default): train the MLP preconditioner on seeded systems of the family first (not "
                         "timed; for the precision workload on the 96^3 learned family), TPA as fallback; tpa: TPA alone")
    ap.add_argument("--no-other-precond", dest="with_other", action="store_false",
                    help="skip the extra timing of the other preconditioner (TPA when the headline is learned)")
    ap.add_argument("--workload", choices=["precision", "precision_small", "medium", "batching", "learned"], default="precision",
                    help="precision (the headline: 96^3, 256 orbitals, 512 perturbations in chunks of 64); precision_small "
                         "(its 96^3 layout with 16 orbitals, for small-case profiler captures); medium "
                         "(64^3, 64 orbitals, 128 perturbations); batching: the uneven multi-system workload (its own line)")
    ap.add_argument("--npert", type=int, default=0,
                    help="perturbations per step (default: the workload's chunk, 64 for precision, 128 for medium); "
                         "the block keeps its number of chunks")
    ap.add_argument("--fp64-npert", type=int, default=2,
                    help="perturbations of the block timed in the plain FP64 GPU form (0: skip)")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the secondary medium-configuration figure")
    ap.add_argument("--learned-train", type=int, default=32, help="learned workload: training seeds")
    ap.add_argument("--learned-test", type=int, default=8, help="learned workload: held-out seeds")
    ap.add_argument("--learned-npert", type=int, default=32, help="learned workload: perturbations per held-out system")
    ap.add_argument("--batch-systems", type=int, default=16)
    ap.add_argument("--batch-npert", type=int, default=64)
    ap.add_argument("--train-systems", type=int, default=8)
    ap.add_argument("--train-npert", type=int, default=8)
    ap.add_argument("--train-steps", type=int, default=600)
    args = ap.parse_args()
    if args.npert > 0:
        for k, wl in list(WORKLOADS.items()):
            nch = wl.nblock // wl.chunk
            WORKLOADS[k] = dataclasses.replace(wl, chunk=args.npert, nblock=args.npert * nch, neig=min(wl.neig, args.npert),
                                               desc=wl.desc + f" [--npert {args.npert}: {args.npert} perturbations per step]")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batching":
        run_batching(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
