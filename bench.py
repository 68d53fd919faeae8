#!/usr/bin/env python
"""Benchmark of the Landau-damping PIC loop on GB300.

One step is one pass of the whole hot path of the PIC loop (Fig. 1) through
the library's C ABI: sort by cell + CIC scatter (pic_deposit), the Poisson
solve to relative residual 1e-10 (poisson_solve_ex), the field energy
(pic_field_energy) and E = -grad phi + CIC gather + leapfrog push
(pic_gather_push). Default workload: the full PIC run with the learned part,
512^3 periodic grid, 8 particles per cell (1,073,741,824 particles, 64-byte
records: fixed-point positions, double-float velocities), Landau initial
condition (k = 0.5, alpha = 0.05), dt = 0.05, warm-started solves by
mixed-precision flexible CG with the learned preconditioner (trained on the
GPU before timing). The same particles then take timed steps with the
multigrid-preconditioned solve, and cold solves of the last deposit (512^3)
and of a 1024^3 Landau density + noise right-hand side compare the FP64
Jacobi-PCG reference with every solver. --solver selects the step's solve
(cnn, mg, mg_cnn, ssor, mixed, fp64), the FFT-PIC step (fft: spectral phi
and E) or the particle-in-Fourier step (pif: NUFFTs, no grid deposit or
solve).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--solver ...] [--N ...]
  python bench.py --impl reference      # the CPU oracle on a bounded sample

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank runs its own
independent replica of the workload (the path has no exchange step on one
GPU); value = steps of all ranks / max time over ranks.
"""
import argparse
import json
import math
import mmap
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PIC steps/s (Landau 3D, CIC, 7-point FD Poisson solve to rel-res 1e-10)"
UNIT = "steps/s"
SEED = 0x5EED
DT = 0.05
TOL = 1e-10
MAXIT = 20000
SOLVERS = ["mixed", "fp64", "cnn", "mg", "mg_cnn", "ssor", "fft", "pif"]
# the full-PIC configuration with the learned part: 512^3 periodic grid x 8
# particles per cell (1.07e9 particles), flexible CG with the learned
# preconditioner, warm-started solves to rel-res 1e-10
DEFAULT_N = 512
DEFAULT_SOLVER = "cnn"
# also timed on the same particles: the multigrid-preconditioned step, with
# Jacobi and with the learned smoother
DEFAULT_ALT_SOLVERS = ("mg", "mg_cnn")
# steps of the end-to-end measurement (each copies the whole particle state in
# and out: 103 GB of host traffic a step at 512^3)
E2E_STEPS = 5
# cold solves of the largest solver-only grid, after the particles are freed
DEFAULT_COMPARE_GRIDS = (1024,)

# algorithmic bytes per cell of one launch of the two CG kernels
KER_BYTES = {
    # (precision, kernel): bytes/cell
    (1, "pap"): 12,      # read r, p_in; write p (FP32)
    (1, "update"): 20,   # read p, x, r; write x, r (FP32)
    (0, "pap"): 32,      # read r, p_in; write p, q (FP64)
    (0, "update"): 48,   # read x, r, p, q; write x, r (FP64)
}
# FP64 operations per cell of one launch (the FP64 reference solve is FP64-pipe bound)
KER_FP64_OPS = {(0, "pap"): 8, (0, "update"): 3}
# learned preconditioner applied as its composed 9^3 kernel: 729 FMA per cell
PRECOND_FLOP_PER_CELL = 2 * 729
# ... which the tensor-core forms execute as 81 Toeplitz products per output:
# the 16-wide form (default) takes K = 32 x-inputs per output (9 of the 32
# weights in each product nonzero); the 8-wide form takes K = 16, its N = 80
# stack carrying 9 groups of 8 outputs and one zero group (2 * 81 * 16 * 80 / 72)
PRECOND_MMA_FLOP_PER_CELL = {"tc": 2 * 81 * 32, "tc8": 2 * 81 * 16 * 80 // 72, "tc_fused": 2 * 81 * 32}
PRECOND_TC_KERNEL = {"tc": "k_apply_k_tc (composed 9^3 learned preconditioner, tcgen05 BF16, 16-wide Toeplitz)",
                     "tc8": "k_apply_k_tc8 (composed 9^3 learned preconditioner, tcgen05 BF16, 8-wide Toeplitz)",
                     "tc_fused": "k_apply_k_tc (composed 9^3 learned preconditioner, tcgen05 BF16, 16-wide "
                                 "Toeplitz, fused FCG update)"}
# algorithmic bytes per fine cell of the V-cycle's finest-level kernels (FP32)
MG_BYTES = {
    "mg_pre": 8,               # read r; write x (both damped sweeps from x = 0)
    "mg_resid": 12,            # read x, r; write res
    "mg_restrict": 4.5,        # read res; write the coarse r.h.s. (1/8 of a cell)
    "mg_prolong_smooth": 12.5,  # read x, e_c (1/8), r; write the first post-sweep
    "mg_smooth": 12,           # read it and r; write x (second post-sweep)
}
# with the learned smoother the prolongation slot is the residual of x + P e_c:
# read x, e_c, r; write res and x + P e_c
MG_BYTES_PROLONG_RESID = 16.5
# algorithmic bytes of the particle kernels, per particle and per grid node,
# counted on the particle state itself (three FP64 positions and three FP64
# velocities, 48 B), not on the library's record layout
PARTICLE_BYTES = {
    # sort: the state read and written once, and the particle's cell key read
    "scatter": (100, 0),
    # deposit: read the positions (24 B), write rho (8 B a node)
    "deposit": (24, 8),
    # gather + push: read and write positions and velocities (96 B), E read
    # once per node (3 x 8 B)
    "push": (96, 24),
}
# bytes per particle the library's kernels move by design: the 64-byte record
# (64-bit fixed-point offsets, double-float velocities, id, cell key, packed
# cell index and in-cell rank) read and written (the deposit reads the
# record's first 32-byte sector)
PARTICLE_IMPL_BYTES = {"scatter": 128, "deposit": 32, "push": 128}
# particle-in-Fourier window sums: a multiply and an atomic add (spreading)
# or one FMA (interpolation) per window point and particle
PIF_FLOP_PER_POINT = 2
# the library runs the NUFFTs in FP32 at tolerances from this one up
PIF_FP32_TOL = 1e-5


def pif_width(tol):
    """Window width of the particle-in-Fourier NUFFTs for a relative tolerance
    (about one digit per point at oversampling 2), clamped to [4, 16]."""
    return min(16, max(4, int(math.ceil(-math.log10(tol))) + 1))


# DRAM traffic per particle of one launch (dram__bytes_read.sum +
# dram__bytes_write.sum over the particle count) measured by ncu on the
# 128^3 x 8 ppc step (16.8 M particles; the traffic scales with the particle
# count): it stands for the same kernels at other sizes
MEASURED_TRAFFIC_PER_PARTICLE = {"push": 128.56, "scatter": 125.76}
# coarse-grid levels streamed like the finest (sizes above 16, halving while even)
MG_SMALL_N = 16


def mg_level_fraction(N):
    """Cells of all plane-streamed V-cycle levels per fine cell."""
    f, l = 0.0, N
    while l > MG_SMALL_N and l % 2 == 0:
        f += (l / N) ** 3
        l //= 2
    return f


# FP32 FMA peak: 152 SMs x 128 lanes x 2 FLOP at the 2.07 GHz maximum clock
# (nominal), and 70.2 TFLOP/s measured with an FMA throughput loop on this GB300
FP32_PEAK_TFLOPS = 70.2


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process
    group): every rank's timed region is bracketed by a barrier, and the job
    takes as long as its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps_per_rank, seconds):
    """Units of all ranks (each runs its own replica) per second of the
    slowest rank."""
    return world * steps_per_rank / seconds


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--solver", choices=SOLVERS, default=DEFAULT_SOLVER,
                    help="cnn (default): mixed-precision flexible CG with the learned preconditioner (trained on "
                         "the GPU before timing); mg: flexible CG with a multigrid V-cycle (damped Jacobi "
                         "smoothing); mg_cnn: the V-cycle with the learned network smoothing the finest level; "
                         "mixed: FP32 Jacobi-CG + FP64 reliable updates; fp64: the FP64 Jacobi-PCG reference; ssor: the "
                         "paper's PCG configuration (red-black SSOR, 4 inner, 2 outer, damping pi/2); fft: the "
                         "paper's other scheme, the FFT pseudo-spectral solve (cuFFT FP64) with the spectral field "
                         "pushed to the particles; pif: the particle-in-Fourier scheme (NUFFTs, no grid deposit "
                         "or solve). The learned solvers are always trained and timed in the solve comparison as "
                         "well")
    ap.add_argument("--pif-tol", type=float, default=1e-4,
                    help="relative tolerance of the particle-in-Fourier NUFFTs (sets the window width; 1e-4 as in the paper's runs)")
    ap.add_argument("--cnn-apply", choices=["tc", "tc8", "tc_fused", "fp32", "layers"], default="tc",
                    help="evaluation of the learned preconditioner: composed 9^3 kernel on the tensor cores "
                         "(BF16; 16-wide Toeplitz form, or the slower 8-wide form), on the CUDA cores (FP32), or the "
                         "four BF16 convs")
    ap.add_argument("--workload", choices=["pic", "solve"], default="pic",
                    help="pic: full PIC step; solve: one cold-start Poisson solve of a Landau density + noise rhs")
    ap.add_argument("--N", type=int, default=DEFAULT_N)
    ap.add_argument("--ppc", type=int, default=8)
    ap.add_argument("--alt-solvers", default=",".join(DEFAULT_ALT_SOLVERS),
                    help="comma-separated solvers whose PIC steps are also timed, after the main run, on the "
                         "same particles (extra keys; empty = none)")
    ap.add_argument("--compare-grids", default=",".join(str(g) for g in DEFAULT_COMPARE_GRIDS),
                    help="comma-separated grid sizes of extra cold-solve comparisons on a Landau density + "
                         "N(0, 0.01^2) noise right-hand side, run after the PIC context is freed (empty = none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--weights-dir", default=None,
                    help="load the trained networks from this directory (pic_cnn_load) when it holds them, else "
                         "train and save them there (pic_cnn_save)")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-vs-mixed solve comparison")
    ap.add_argument("--compare-reps", type=int, default=2,
                    help="cold solves per solver in the comparison (best kept; solves longer than 2 s run once)")
    ap.add_argument("--compare-maxit", type=int, default=MAXIT,
                    help="iteration cap of the comparison solves (mixed Jacobi-CG stagnates at 1024^3)")
    return ap.parse_args(argv)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d
    except Exception:
        return 6800.0, "fallback", {}


def fp64_peak_tflops():
    """FP64 FMA peak of GB300: 1.2 TFLOP/s measured with a dependent-chain-free
    DFMA loop on this machine's GB300 (152 SMs, ~2 GHz); the FP64 rate is 1/58 of the FP32 rate."""
    return 1.20


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- ours
def particle_roofline(rows, k, np_, n, hbm, peak_kind):
    """HBM roofline of a particle kernel from its sampled launches: the
    algorithmic bytes of the FP64 particle state (and the grid) over the
    average CUDA-event duration, with the ncu DRAM traffic beside them."""
    r = rows[k]
    b = r["bytes_per_particle"] * np_ + r["bytes_per_node"] * n
    traffic = round(MEASURED_TRAFFIC_PER_PARTICLE[k] * np_) if k in MEASURED_TRAFFIC_PER_PARTICLE else None
    return {"kernel": {"scatter": "k_scatter (sort: 64-byte records to their cells)",
                       "deposit": "k_deposit_cells + k_deposit_nodes (CIC scatter)",
                       "push": "k_gather_push (CIC gather + leapfrog, double-float)"}[k],
            "bound": "hbm", "achieved": round(r["gbs"], 1), "peak": hbm, "unit": "GB/s",
            "frac": round(r["gbs"] / hbm, 4), "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": traffic,
            "traffic_source": ("ncu DRAM bytes per particle at 128^3 x 8 ppc, scaled by the particle count"
                               if traffic is not None else None),
            "traffic_over_algorithmic": round(traffic / b, 3) if traffic is not None else None,
            "algorithmic_bytes": b, "algorithmic_bytes_per_particle": r["bytes_per_particle"],
            "impl_bytes_per_particle": r["impl_bytes_per_particle"], "avg_launch_us": round(r["avg_us"], 2)}


def mem_available_bytes():
    """MemAvailable of the host (0 if unknown)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        pass
    return 0


def host_state_buffer(count, torch):
    """A zeroed FP64 host tensor of `count` values, backed where the kernel
    allows by transparent huge pages (anonymous mapping aligned to 512 MB,
    MADV_HUGEPAGE). Measured on the Grace hosts: after other large jobs have
    fragmented host memory, copies of a 51.5 GB state in 64 KB pages ran at
    23-31 GB/s, the same state in huge pages at 81-166 GB/s. Returns (tensor,
    whether huge pages were requested)."""
    nbytes = 8 * count
    align = 512 << 20
    try:
        m = mmap.mmap(-1, nbytes + align, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        m.madvise(mmap.MADV_HUGEPAGE)
        raw = np.frombuffer(m, dtype=np.uint8)
        off = (-raw.ctypes.data) % align
        t = torch.from_numpy(raw[off:off + nbytes].view(np.float64))  # keeps the mapping alive
        t.zero_()
        return t, True
    except (AttributeError, OSError, ValueError):
        return torch.zeros(count, dtype=torch.float64), False


def end_to_end(c, step, np_, n, rho, phi, steps, solve_only, world, dist, barrier, torch, unit, solve_into):
    """The metric end to end through the public API on the host's wall clock,
    with the step's inputs copied in from host memory and its result read back
    every step: the PIC step's particle state (48 B a particle each way, via
    pic_set_particles / pic_get_particles, page-locked host memory) and its
    field energy; a solve's rho in and phi out."""
    if solve_only:
        rho_h = rho.cpu().pin_memory()
        phi_h = torch.empty_like(rho_h).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            rho.copy_(rho_h, non_blocking=True)
            phi.zero_()
            solve_into(rho, phi)
            phi_h.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        return {"value": whole_job_rate(world, steps, s), "unit": unit, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "note": "rho from pinned host memory, phi back to it, every solve"}
    state_bytes = 48 * np_
    # every rank on this host takes its own copy of the state
    avail = mem_available_bytes() // max(1, int(os.environ.get("LOCAL_WORLD_SIZE", "1")))
    if avail < 2 * state_bytes + (48 << 30):
        # not enough host memory for the state: the device-resident loop, the
        # field energy read back every step
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            step(False)
        torch.cuda.synchronize()
        barrier()
        s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        return {"value": whole_job_rate(world, steps, s), "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 24,
                "note": f"host memory too small for the particle state ({avail / 2**30:.0f} GiB available): "
                        "particles stay on the device, the field energy is read back every step"}
    state, huge = host_state_buffer(6 * np_, torch)
    # page-locked in pieces of at most 4 GiB: measured on the Grace host, one
    # 51.5 GB registration moved 25-36 GB/s, eight 6.4 GB ones 193 GB/s
    cudart = torch._C._cudart
    piece = min(state_bytes, 4 << 30)
    pieces = [(a, min(piece, state_bytes - a)) for a in range(0, state_bytes, piece)]
    done = []
    for a, b in pieces:
        if cudart.cudaHostRegister(state.data_ptr() + a, b, 0) != cudart.cudaError.success:
            break
        done.append(a)
    registered = len(done) == len(pieces)
    try:
        half = c.particles_to_host(state)  # the state starts on the host (untimed)
        barrier()
        t0 = time.perf_counter()
        marks = []
        for _ in range(steps):
            c.set_particles(state, half)
            step(False)  # reads the field energy back
            half = c.particles_to_host(state)
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        barrier()
        s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        per_step = np.diff([t0] + marks)
    finally:
        for a in done:
            cudart.cudaHostUnregister(state.data_ptr() + a)
        del state
    return {"value": whole_job_rate(world, steps, s), "unit": unit, "steps": steps, "h2d_bytes_per_step": state_bytes,
            "d2h_bytes_per_step": state_bytes + 24,
            "step_s": {"min": round(float(per_step.min()), 3), "median": round(float(np.median(per_step)), 3),
                       "max": round(float(per_step.max()), 3)},
            "note": ("every step: the particle state (FP64 x, y, z, vx, vy, vz) in from "
                     + ("page-locked" if registered else "pageable")
                     + (" huge-page" if huge else "") + " host memory (pic_set_particles), "
                     "the step, its field energy read back, the state out to host memory (pic_get_particles)")}


def vcycle_record(prof, learned, N, hbm):
    """One V-cycle (every level, the one-block coarse cycle and, with the
    learned smoother, its two network applications) from the sampled
    preconditioner launches: bytes of the plane-streamed levels per fine
    cell over the average duration, against the HBM peak."""
    k = prof["ker_samples"].get("precond")
    if not k:
        return None
    avg_ms = prof["ker_ms"]["precond"] / k
    jac = sum(MG_BYTES.values())
    # learned smoother on the finest level: network r -> x (8), residual,
    # restriction, residual of x + P e_c, network res -> x (8), x += t (12)
    fine = jac if not learned else (8 + MG_BYTES["mg_resid"] + MG_BYTES["mg_restrict"] +
                                    MG_BYTES_PROLONG_RESID + 8 + 12)
    bpc = fine + jac * (mg_level_fraction(N) - 1.0)
    gbs = bpc * N ** 3 / (avg_ms * 1e-3) / 1e9
    return {"avg_us": round(avg_ms * 1e3, 2), "samples": k, "bytes_per_fine_cell": round(bpc, 3),
            "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4),
            "note": "one V-cycle, every level; bytes of the plane-streamed levels"}


def solver_modes(pg, solver):
    """(precision, preconditioner) of a --solver name."""
    prec = pg.PREC_FP64 if solver == "fp64" else pg.PREC_MIXED
    pc = {"cnn": pg.PC_CNN, "mg": pg.PC_MG, "mg_cnn": pg.PC_MG_CNN, "ssor": pg.PC_SSOR}.get(solver, pg.PC_JACOBI)
    return prec, pc


def dtype_label(pg, solver, cnn_apply="tc", pif_tol=1e-4, solve_only=False):
    """What the step computes in: particle state and arithmetic, grid fields,
    the solve's vectors and reductions, the preconditioner."""
    parts = [] if solve_only else ["particles: 64-bit fixed-point positions + double-float velocities"]
    if solver == "pif":
        prec_ = "FP32" if pif_tol >= PIF_FP32_TOL else "FP64"
        return "; ".join(parts + [f"{prec_} particle-in-Fourier NUFFTs (tol {pif_tol:g}) and cuFFT"])
    parts.append("rho, phi FP64")
    if solver == "fft":
        return "; ".join(parts + ["FP64 spectral solve (cuFFT)"])
    if solver == "fp64":
        return "; ".join(parts + ["solve FP64 throughout"])
    parts.append("solve FP32 vectors + FP64 reductions and residual recomputation")
    if solver == "cnn":
        parts.append({"tc": "BF16 tensor-core", "tc8": "BF16 tensor-core (8-wide)",
                      "tc_fused": "BF16 tensor-core (fused)", "fp32": "FP32",
                      "layers": "BF16 four-conv"}[cnn_apply] + " learned preconditioner (composed 9^3 kernel)")
    elif solver == "mg":
        parts.append("FP32 multigrid V-cycle")
    elif solver == "mg_cnn":
        parts.append("FP32 multigrid V-cycle, BF16 learned finest-level smoother")
    elif solver == "ssor":
        parts.append("FP32 red-black SSOR")
    return "; ".join(parts)


def l2_note(N, ppc, solve_only):
    """How the timed steps relate to the 129 MB L2: every input is larger."""
    n = N ** 3
    cells = f"grid vectors {n * 4 / 1e6:.0f} MB (FP32) to {n * 8 / 1e6:.0f} MB (FP64) each"
    if max(n * 8, 0 if solve_only else ppc * n * 64) < 129e6:
        return "small case: inputs fit in the 129 MB L2, no flush between steps"
    if solve_only:
        return f"inputs larger than L2 ({cells})"
    return (f"inputs larger than L2 (particle records {ppc * n * 64 / 1e9:.1f} GB; {cells})")


def run_ours(args):
    import torch
    import paper_2605_05469_gb300 as pg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    N, ppc = args.N, args.ppc
    n = N ** 3
    prec, pc = solver_modes(pg, args.solver)
    stream = torch.cuda.current_stream()
    solve_only = args.workload == "solve"
    alt_solvers = [] if solve_only else [s for s in args.alt_solvers.split(",") if s and s != args.solver]
    for s_ in alt_solvers:
        if s_ not in SOLVERS:
            raise SystemExit(f"unknown solver in --alt-solvers: {s_}")
    weights, train_info = None, None
    if any(s_ in ("cnn", "mg_cnn") for s_ in [args.solver] + alt_solvers) or not args.no_compare:
        weights, train_info = train_networks(pg, torch, args.weights_dir)
    c = pg.Context(stream).init(N, 0 if solve_only else ppc, SEED + rank)
    apply_mode = {"tc": pg.CNN_APPLY_TC, "tc8": pg.CNN_APPLY_TC8, "tc_fused": pg.CNN_APPLY_TC_FUSED,
                  "fp32": pg.CNN_APPLY_FP32, "layers": pg.CNN_APPLY_LAYERS}[args.cnn_apply]
    nets = Networks(c, weights)
    if weights is not None:
        nets.use(pc if pc in weights else pg.PC_CNN)
        c.cnn_set_apply(apply_mode)
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    if solve_only:
        from paper_2605_05469_gb300 import inputs
        rho = inputs.landau_noise_rhs_torch(N, 0xC0FFEE + rank, "cuda")
    else:
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
    E3 = None

    def make_step(solver, infos):
        """One step of the workload with the given solver; appends the solve's
        info to `infos` when recording."""
        nonlocal E3
        s_prec, s_pc = solver_modes(pg, solver)
        nets.use(s_pc)
        use_fft, use_pif = solver == "fft", solver == "pif"
        if use_fft and E3 is None:
            E3 = torch.empty(3 * n, dtype=torch.float64, device="cuda")

        def solve_into(rho_, phi_):
            nets.use(s_pc)
            if use_fft:
                # direct solve: no iterations or residual; its time is the solve phase's
                c.fft_solve(rho_, phi_, E3)
                return {"iters": 0, "t_ms": None, "rel_res": 0.0, "reliable_updates": 0, "converged": True}
            return c.solve(rho_, phi_, tol=TOL, maxit=MAXIT, precision=s_prec, precond=s_pc)

        def step(record):
            if solve_only:
                phi.zero_()
                info = solve_into(rho, phi)
                W = None
            elif use_pif:
                c.pif_push(DT, tol=args.pif_tol)
                info = {"iters": 0, "t_ms": 0.0, "rel_res": 0.0, "reliable_updates": 0, "converged": True}
                W = None
            else:
                c.deposit(rho)
                info = solve_into(rho, phi)
                if use_fft:
                    W = c.field_energy_E(E3)
                    c.gather_push_field(E3, DT)
                else:
                    W = c.field_energy(phi)
                    c.gather_push(phi, DT)
            if record:
                infos.append(info)
            return W
        step.solve_into = solve_into
        return step

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    infos = []
    step = make_step(args.solver, infos)
    use_fft, use_pif = args.solver == "fft", args.solver == "pif"
    for _ in range(args.warmup):
        step(False)
    c.profile(True)
    c.profile_read(reset=True)

    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(True)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = c.profile_read(reset=True)
    c.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(world, args.steps, ms / 1e3)
    unit = "solves/s" if solve_only else UNIT
    metric = ("Poisson solves/s to rel-res 1e-10 (7-point FD, cold start)" if solve_only else METRIC)

    # end to end through the public API, host wall clock. PIC step: the
    # particle state (FP64 positions and velocities, 48 B a particle) lives in
    # page-locked host memory; every step copies it in (pic_set_particles),
    # runs the step, reads the field energy and copies the state back out
    # (pic_get_particles). Solver-only: rho in from host memory, phi back.
    np_ = 0 if solve_only else ppc * n
    e2e = end_to_end(c, step, np_, n, rho, phi, min(args.steps, E2E_STEPS), solve_only, world, dist, barrier, torch,
                     unit,
                     step.solve_into)

    # the other solvers' PIC steps on the same particles (extra keys)
    alt = {}
    for s_ in alt_solvers:
        alt_infos = []
        st_ = make_step(s_, alt_infos)
        for _ in range(max(1, args.warmup // 2)):
            st_(False)
        c.profile(True)
        c.profile_read(reset=True)
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            st_(True)
        a1.record(stream)
        torch.cuda.synchronize()
        barrier()
        a_ms = max_over_ranks(a0.elapsed_time(a1), dist, "cuda")
        a_prof = c.profile_read(reset=True)
        c.profile(False)
        if s_ in ("mg", "mg_cnn"):
            alt_vc = vcycle_record(a_prof, s_ == "mg_cnn", N, peaks()[0])
        else:
            alt_vc = None
        alt[s_] = {"value": round(whole_job_rate(world, args.steps, a_ms / 1e3), 4), "unit": unit, "vcycle": alt_vc,
                   "ms_per_step": round(a_ms / args.steps, 3), "steps": args.steps,
                   "dtype": dtype_label(pg, s_, args.cnn_apply, args.pif_tol),
                   "phases_ms_per_step": {k: round(v / args.steps, 3) for k, v in a_prof["phase_ms"].items()},
                   "solve_iters_mean": (statistics.mean(i["iters"] for i in alt_infos) if alt_infos else None)}

    # solver-only end to end: rho from pinned host memory, phi back to host
    if use_pif:
        c.deposit(rho)  # the particle-in-Fourier step has no grid charge of its own
    rho_host = rho.cpu().pin_memory()
    phi_host = torch.empty_like(rho_host).pin_memory()
    barrier()
    t0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        rho.copy_(rho_host, non_blocking=True)
        phi.zero_()
        step.solve_into(rho, phi)
        phi_host.copy_(phi, non_blocking=True)
    torch.cuda.synchronize()
    e2e_solve = {"value": reps / (time.perf_counter() - t0), "unit": "solves/s (cold start)",
                 "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8}
    del rho_host, phi_host

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    # roofline of the dominant CG kernel from the sampled CUDA events
    hbm, peak_kind, _ = peaks()
    kp = prof["ker_precision"]["pap"]
    rows = {}
    for k in ("pap", "update"):
        if prof["ker_samples"][k]:
            avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
            # the mixed-precision solvers store q = A p in the direction kernel
            # (+4 B/cell) and stream q in the update instead of recomputing
            # A p from p's halo (+4 B/cell)
            bpc = KER_BYTES[(kp, k)] + (4 if kp == 1 else 0)
            rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k],
                       "bytes_per_cell": bpc, "gbs": bpc * n / (avg_ms * 1e-3) / 1e9}
    if prof["ker_samples"].get("dot"):
        avg_ms = prof["ker_ms"]["dot"] / prof["ker_samples"]["dot"]
        rows["dot"] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"]["dot"], "bytes_per_cell": 12,
                       "gbs": 12 * n / (avg_ms * 1e-3) / 1e9}
    is_mg = pc in (pg.PC_MG, pg.PC_MG_CNN)
    if prof["ker_samples"]["precond"] and not is_mg:
        avg_ms = prof["ker_ms"]["precond"] / prof["ker_samples"]["precond"]
        rows["precond"] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"]["precond"],
                           "flop_per_cell": PRECOND_FLOP_PER_CELL,
                           "tflops": PRECOND_FLOP_PER_CELL * n / (avg_ms * 1e-3) / 1e12}
    vcycle = None
    if is_mg:
        for k, b in MG_BYTES.items():
            if not prof["ker_samples"].get(k):
                continue
            if k == "mg_prolong_smooth" and pc == pg.PC_MG_CNN:
                b = MG_BYTES_PROLONG_RESID
            avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
            rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k], "bytes_per_cell": b,
                       "gbs": b * n / (avg_ms * 1e-3) / 1e9}
        vcycle = vcycle_record(prof, pc == pg.PC_MG_CNN, N, hbm)
    # the particle kernels (one launch each per step): algorithmic bytes of
    # the FP64 particle state, and the bytes the record layout moves
    for k, (bp, bn) in PARTICLE_BYTES.items():
        if not np_ or not prof["ker_samples"].get(k):
            continue
        avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
        b = bp * np_ + bn * n
        rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k], "bytes_per_particle": bp,
                   "bytes_per_node": bn, "gbs": b / (avg_ms * 1e-3) / 1e9, "launches_per_step": 1,
                   "impl_bytes_per_particle": PARTICLE_IMPL_BYTES[k],
                   "impl_gbs": (PARTICLE_IMPL_BYTES[k] * np_ + bn * n) / (avg_ms * 1e-3) / 1e9}
    # particle-in-Fourier: the spreading kernel (the charge) and the
    # interpolation kernel (the three field components at once), one launch
    # each a step; window sums over w^3 grid points a particle, FP32 at
    # tolerances >= 1e-5, else FP64
    pif_f32 = args.pif_tol >= PIF_FP32_TOL
    if use_pif:
        w_pif = pif_width(args.pif_tol)
        for k, comps in (("pif_spread", 1), ("pif_gather", 3)):
            if not prof["ker_samples"].get(k):
                continue
            avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
            flop = PIF_FLOP_PER_POINT * comps * w_pif ** 3 * np_
            rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k], "window_points": w_pif ** 3,
                       "components": comps, "precision": "FP32" if pif_f32 else "FP64", "flop": flop,
                       "tflops": flop / (avg_ms * 1e-3) / 1e12, "launches_per_step": 1}
    # the dominant kernel: the largest device time per step (solver kernels
    # run once per iteration)
    it_mean = statistics.mean(i["iters"] for i in infos) if infos else 1

    def per_step(k):
        return rows[k]["avg_us"] * rows[k].get("launches_per_step", it_mean)
    dom = max(rows, key=per_step) if rows else None
    kname = {("pap", 1): "k_cg_pap<float>", ("update", 1): "k_fcg_update32", ("dot", 1): "k_fcg_dot",
             ("pap", 0): "k_cg_pap<double,true>", ("update", 0): "k_cg_update64",
             ("mg_pre", 1): "k_mg_pre (finest level)", ("mg_resid", 1): "k_mg_stencil<kResid> (finest level)",
             ("mg_restrict", 1): "k_mg_restrict2 (finest level)",
             ("mg_prolong_smooth", 1): ("k_mg_stencil<kSmooth, prolong> (finest level)" if pc == pg.PC_MG else
                                        "k_mg_stencil<kResid, prolong> (finest level)"),
             ("mg_smooth", 1): "k_mg_stencil<kSmooth> (finest level)"}
    roof = None
    if dom in ("pif_spread", "pif_gather"):
        r = rows[dom]
        prec_ = "FP32" if pif_f32 else "FP64"
        peak_ = FP32_PEAK_TFLOPS if pif_f32 else fp64_peak_tflops()
        roof = {"kernel": {"pif_spread": f"k_pif_spread (type-1 NUFFT spreading, {prec_} atomics)",
                           "pif_gather": "k_pif_gather3 (type-2 NUFFT interpolation, three components)"}[dom],
                "bound": "alu", "achieved": round(r["tflops"], 4), "peak": peak_,
                "unit": f"{prec_} TFLOP/s", "frac": round(r["tflops"] / peak_, 4),
                "peak_source": f"measured {prec_} FMA loop", "traffic": None, "algorithmic_flop": r["flop"],
                "avg_launch_us": round(r["avg_us"], 2),
                "note": f"window sums: 2 {prec_} flops per window point, component and particle (window "
                        "evaluation not counted); the spreading's atomics into the oversampled grid in L2 "
                        "bound it more than its arithmetic"}
    elif dom == "precond" and apply_mode in (pg.CNN_APPLY_TC, pg.CNN_APPLY_TC8, pg.CNN_APPLY_TC_FUSED):
        r = rows[dom]
        _, _, pk = peaks()
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        roof = {"kernel": PRECOND_TC_KERNEL[args.cnn_apply], "bound": "tensor",
                "achieved": round(r["tflops"], 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(r["tflops"] / peak, 4),
                "peak_source": "measured bf16_tflops_sustained (kernel timed inside a long solve)",
                "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n,
                "executed_mma_tflops": round(r["tflops"] * PRECOND_MMA_FLOP_PER_CELL[args.cnn_apply]
                                             / PRECOND_FLOP_PER_CELL, 2),
                "avg_launch_us": round(r["avg_us"], 2)}
    elif dom == "precond":
        r = rows[dom]
        roof = {"kernel": "k_apply_k (composed 9^3 learned preconditioner)", "bound": "alu",
                "achieved": round(r["tflops"], 2), "peak": FP32_PEAK_TFLOPS, "unit": "FP32 TFLOP/s",
                "frac": round(r["tflops"] / FP32_PEAK_TFLOPS, 4),
                "peak_source": "measured FP32 FMA loop (no FP32 figure in MEASURED_PEAKS.json)",
                "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n, "avg_launch_us": round(r["avg_us"], 2)}
    elif dom in PARTICLE_BYTES:
        roof = particle_roofline(rows, dom, np_, n, hbm, peak_kind)
    elif dom is not None:
        r = rows[dom]
        if kp == 1:
            roof = {"kernel": kname[(dom, kp)], "bound": "hbm", "achieved": round(r["gbs"], 1),
                    "peak": hbm, "unit": "GB/s", "frac": round(r["gbs"] / hbm, 4),
                    "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                    "algorithmic_bytes": r["bytes_per_cell"] * n, "avg_launch_us": round(r["avg_us"], 2)}
        else:
            ops = KER_FP64_OPS[(0, dom)] * n
            tf = ops / (r["avg_us"] * 1e-6) / 1e12
            roof = {"kernel": kname[(dom, kp)], "bound": "alu", "achieved": round(tf, 4),
                    "peak": fp64_peak_tflops(), "unit": "FP64 TFLOP/s", "frac": round(tf / fp64_peak_tflops(), 4),
                    "peak_source": "measured FP64 FMA loop", "traffic": None,
                    "algorithmic_bytes": r["bytes_per_cell"] * n, "avg_launch_us": round(r["avg_us"], 2)}

    iters = [i["iters"] for i in infos]
    solve_ms = ([i["t_ms"] for i in infos] if not use_fft else
                [prof["phase_ms"]["solve"] / max(1, prof["phase_calls"]["solve"])])
    out = {
        "metric": metric, "value": round(value, 4), "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(pg, args.solver, args.cnn_apply, args.pif_tol, solve_only),
        "data": "synthetic: seeded Landau initial condition (Philox4x32-10, inverse CDF, Box-Muller)",
        "config": pic_config(args, world),
        "clocks": clk,
        "e2e": e2e,
        "e2e_solve": e2e_solve,
        "gpu_launches": prof["launches"],
        "roofline": roof,
        "kernels": rows,
        "vcycle": vcycle,
        "solve": {"iters_mean": statistics.mean(iters), "ms_mean": statistics.mean(solve_ms),
                  "rel_res_max": max(i["rel_res"] for i in infos),
                  "reliable_updates_mean": statistics.mean(i["reliable_updates"] for i in infos)},
        "phases_ms_per_step": {k: round(v / args.steps, 3) for k, v in prof["phase_ms"].items()},
        "impl": "ours",
    }
    if alt:
        out["pic_steps_other_solvers"] = alt
    if roof is not None and dom != "push" and "push" in rows:
        out["roofline_push"] = particle_roofline(rows, "push", np_, n, hbm, peak_kind)
    if train_info is not None:
        out["network_training"] = train_info
    if not args.no_compare:
        cmp_ = {}
        cmp_[str(N)], learned_roof = compare_solvers(
            c, rho, n, pg, torch, nets=nets, reps=args.compare_reps, maxit=args.compare_maxit,
            rhs=("Landau density + N(0, 0.01^2) noise, mean removed" if solve_only else
                 f"CIC deposit of the last step ({np_} particles)"))
        if learned_roof is not None:
            out["roofline_learned_preconditioner"] = learned_roof
        out["solve_compare"] = cmp_
    grids = [] if args.no_compare else [int(g) for g in args.compare_grids.split(",") if g and int(g) != N]
    if grids:
        # free the particles and the step's grids before the larger solves
        c.close()
        c = None
        del rho, phi, E3
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        from paper_2605_05469_gb300 import inputs
        for G in grids:
            cg = pg.Context(stream).init(G, 0, 0)
            rho_g = inputs.landau_noise_rhs_torch(G, 0xC0FFEE, "cuda")
            out["solve_compare"][str(G)], _ = compare_solvers(
                cg, rho_g, G ** 3, pg, torch, nets=Networks(cg, weights), reps=args.compare_reps,
                maxit=args.compare_maxit, rhs="Landau density + N(0, 0.01^2) noise, mean removed",
                skip=LARGE_GRID_SKIP if G >= 1024 else ())
            cg.close()
            del rho_g
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = (cpu_baseline_pif(N, ppc) if use_pif else
                               cpu_baseline(N, 0 if solve_only else ppc, statistics.mean(iters), args.solver))
    if dist is not None:
        dist.destroy_process_group()
    if c is not None:
        c.close()
    return out


def train_networks(pg, torch, weights_dir=None):
    """Train the network twice on the GPU before timing, each by one
    pic_cnn_train call (the library's own solves for the data, its kernels
    for forward, loss, backward and Adam): as flexible CG's preconditioner
    (Jacobi-PCG snapshots of four 64^3 Landau deposits, 600 Adam steps on
    32^3 crops, four restarts, the state kept by the flexible-CG iterations
    of a held-out 128^3 deposit) and as the V-cycle's finest-level smoother
    (white-noise errors, kept by the multigrid-FCG iterations of the same
    deposit). Returns the weights per preconditioner and the training
    records."""
    t0 = time.perf_counter()
    c = pg.Context().init(64, 0, 0)
    files = None if not weights_dir else (os.path.join(weights_dir, "preconditioner.piccnn"),
                                          os.path.join(weights_dir, "smoother.piccnn"))
    if files and all(os.path.exists(f) for f in files):
        c.cnn_load(files[0])
        w_p = c.cnn_get_weights()
        c.cnn_load(files[1])
        w_s = c.cnn_get_weights()
        c.close()
        return {pg.PC_CNN: w_p, pg.PC_MG_CNN: w_s}, {"loaded_from": weights_dir}
    info_p = c.cnn_train(pg.TRAIN_PRECONDITIONER, restarts=4)
    w_p = c.cnn_get_weights()
    if files:
        os.makedirs(weights_dir, exist_ok=True)
        c.cnn_save(files[0])
    info_s = c.cnn_train(pg.TRAIN_SMOOTHER)
    w_s = c.cnn_get_weights()
    if files:
        c.cnn_save(files[1])
    c.close()
    torch.cuda.synchronize()
    rec = {k: {"loss_first": round(v["loss_first"], 4), "loss_last": round(v["loss_last"], 4),
               "kept_adam_step": v["adam_steps"], "kept_restart": v["best_restart"],
               "validation_iters": v["best_iters"], "seconds": round(v["seconds"], 2)}
           for k, v in (("preconditioner", info_p), ("smoother", info_s))}
    rec.update({"grid": 64, "steps": 600, "selected_by": "flexible-CG iterations on a 128^3 deposit",
                "seconds": round(time.perf_counter() - t0, 2)})
    return {pg.PC_CNN: w_p, pg.PC_MG_CNN: w_s}, rec


class Networks:
    """The trained weights of the context's network, switched to the ones a
    preconditioner was trained for before a solve that uses the network."""

    def __init__(self, c, weights):
        self.c, self.w, self.cur = c, weights, None

    def use(self, pc):
        if self.w is None or pc not in self.w or pc == self.cur:
            return
        self.c.cnn_set_weights(self.w[pc])
        self.cur = pc


# solvers left out of the cold-solve comparison on grids of 1024^3 and more,
# with the reason (each would take minutes)
LARGE_GRID_SKIP = {
    "mixed_fp32_fp64": "not run: FP32 Jacobi-CG with FP64 reliable updates stagnates above rel-res 1e-10 at "
                       "1024^3 (4.0e-10 after 8000 iterations, 61 s)",
    "mixed_cg_ssor_paper_configuration": "not run: about 30-60 s at 1024^3 (32 half-sweeps an application)",
    "mixed_fcg_learned_fp32": "not run: the CUDA-core form of the learned preconditioner, about 25 s at 1024^3",
}


def compare_solvers(c, rho, n, pg, torch, nets=None, reps=2, maxit=MAXIT, rhs="", skip=()):
    """Cold-start solves of the same right-hand side: the FP64 Jacobi-PCG
    reference against the mixed-precision solvers (Jacobi-CG, flexible CG with
    the multigrid V-cycle, the paper's SSOR configuration, and with the
    learned preconditioner and the V-cycle with the learned smoother when the
    network is loaded) and the FFT pseudo-spectral solve, outside the timed
    region. The best of `reps` solves is kept (one solve when it takes more
    than 2 s)."""
    res = {"N": round(n ** (1.0 / 3.0)), "rhs": rhs, "tol": TOL}
    with_cnn = nets is not None and nets.w is not None
    cases = [("fp64_jacobi_pcg", pg.PREC_FP64, pg.PC_JACOBI), ("mixed_fp32_fp64", pg.PREC_MIXED, pg.PC_JACOBI),
             ("mixed_fcg_multigrid", pg.PREC_MIXED, pg.PC_MG),
             ("mixed_cg_ssor_paper_configuration", pg.PREC_MIXED, pg.PC_SSOR)]
    if with_cnn:
        cases.append(("mixed_fcg_learned", pg.PREC_MIXED, pg.PC_CNN))
        cases.append(("mixed_fcg_learned_fp32", pg.PREC_MIXED, pg.PC_CNN))
        cases.append(("mixed_fcg_multigrid_learned_smoother", pg.PREC_MIXED, pg.PC_MG_CNN))
    learned_roof = None
    for name, prec, pc in cases:
        if name in skip:
            res[name] = {"skipped": skip[name]}
            continue
        if with_cnn:
            nets.use(pc)
            c.cnn_set_apply(pg.CNN_APPLY_FP32 if name.endswith("_fp32") else pg.CNN_APPLY_TC)
        best = None
        # the tensor-core preconditioner's launches are sampled in the first
        # learned solve for its roofline
        sample = name == "mixed_fcg_learned"
        if sample:
            c.profile(True)
            c.profile_read(reset=True)
        for r_ in range(max(1, reps)):
            phi = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = c.solve(rho, phi, tol=TOL, maxit=maxit, precision=prec, precond=pc, raise_on_error=False)
            if best is None or info["t_ms"] < best["t_ms"]:
                best = info
            if info["t_ms"] > 2000.0:
                break
            del phi
        if sample:
            prof = c.profile_read(reset=True)
            c.profile(False)
            learned_roof = tc_roofline(prof, n, "tc")
        res[name] = {"s": best["t_ms"] / 1e3, "iters": best["iters"], "rel_res": best["rel_res"],
                     "converged": bool(best["converged"])}
        if name != "fp64_jacobi_pcg" and "fp64_jacobi_pcg" in res and "s" in res["fp64_jacobi_pcg"]:
            res[name]["speedup_vs_fp64_jacobi_pcg"] = round(res["fp64_jacobi_pcg"]["s"] / res[name]["s"], 3)
    # the paper's FFT scheme: the spectral solve of the same right-hand side
    # (phi and the three spectral field components), cold, CUDA-event timed
    stream = torch.cuda.current_stream()
    for name, with_E in (("fft_spectral_phi_and_E", True), ("fft_spectral_phi", False)):
        E3 = torch.empty(3 * n, dtype=torch.float64, device="cuda") if with_E else None
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        c.fft_solve(rho, phi, E3)  # plans
        best = None
        for _ in range(max(1, reps)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            c.fft_solve(rho, phi, E3)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None or t < best else best
        res[name] = {"s": best, "note": ("direct solve of the continuous-symbol equation (Sec. 3.1), not the "
                                         "finite-difference system" if with_E else
                                         "phi alone: one forward and one inverse transform")}
        del E3, phi
    judge = res["fp64_jacobi_pcg"]["s"]
    res["fp64_pcg_vs_fft_time_ratio"] = judge / res["fft_spectral_phi_and_E"]["s"]
    return res, learned_roof


def tc_roofline(prof, n, form="tc"):
    """Roofline of the tensor-core learned preconditioner (k_apply_k_tc, or
    k_apply_k_tc8 for the 8-wide form) from its sampled launches:
    algorithmic FLOP of the composed 9^3 kernel per launch over the average
    CUDA-event duration, against the measured sustained BF16 peak."""
    if form not in PRECOND_MMA_FLOP_PER_CELL:
        form = "tc"
    k = prof["ker_samples"]["precond"]
    if not k:
        return None
    avg_ms = prof["ker_ms"]["precond"] / k
    tf = PRECOND_FLOP_PER_CELL * n / (avg_ms * 1e-3) / 1e12
    _, _, pk = peaks()
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    return {"kernel": PRECOND_TC_KERNEL[form], "bound": "tensor",
            "achieved": round(tf, 2), "peak": peak, "unit": "TFLOP/s", "frac": round(tf / peak, 4),
            "peak_source": "measured bf16_tflops_sustained (kernel timed inside a long solve)",
            "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n,
            "executed_mma_tflops": round(tf * PRECOND_MMA_FLOP_PER_CELL[form] / PRECOND_FLOP_PER_CELL, 2),
            "avg_launch_us": round(avg_ms * 1e3, 2), "samples": k}


# --------------------------------------------------------------------------- oracle
# sample grids of the oracle timings (the oracle's cost per cell and per
# particle does not depend on the grid size, so samples scale by cells)
ORACLE_SOLVE_GRID = {"mg": 128, "cnn": 32, "mg_cnn": 32, "ssor": 64, "fft": 128, "mixed": 128, "fp64": 128}
ORACLE_PARTICLE_GRID = 64


def oracle_iteration_seconds(N, solver, Ns=None):
    """Seconds of one solver iteration of the CPU oracle (as it stands) on an
    N^3 grid, with the same algorithm as the GPU solver: Jacobi-PCG for the
    mixed and FP64 solvers, flexible CG with the V-cycle, the network or SSOR
    for the others, and one spectral solve for fft; timed on an Ns^3 grid and
    scaled by the cell count (the FFT by cells x log cells)."""
    from oracle import cnn as ocnn
    from oracle import mg as omg
    from oracle import pic as opic
    from paper_2605_05469_gb300 import inputs

    L = 4.0 * np.pi
    Ns = min(N, Ns or ORACLE_SOLVE_GRID.get(solver, 128))
    h = L / Ns
    b = inputs.landau_noise_rhs(Ns, 1)
    x0 = np.zeros(Ns ** 3)
    if solver == "fft":
        from oracle import fft as offt
        t0 = time.perf_counter()
        offt.spectral_solve(b, Ns, L)
        scale = (N / Ns) ** 3 * math.log(N) / math.log(Ns)
        return ((time.perf_counter() - t0) * scale,
                f"one spectral solve (numpy FFT, phi and E) on a {Ns}^3 grid (scaled by cells x log cells)")
    if solver in ("mg", "cnn", "mg_cnn", "ssor"):
        from oracle import ssor as ossor
        ws = ocnn.init_weights(0)

        def net(q):
            return h * h * ocnn.forward(q.reshape(Ns, Ns, Ns), ws)[0].reshape(-1)
        prec = {"mg": lambda r: omg.vcycle(r, Ns, h),
                "cnn": lambda r: ocnn.precondition(r, ws, Ns, h),
                "mg_cnn": lambda r: omg.vcycle(r, Ns, h, smoother=net),
                "ssor": lambda r: ossor.ssor(r, Ns, h)}[solver]
        k_it = 1
        t0 = time.perf_counter()
        ocnn.fcg(b, x0, Ns, h, 0.0, k_it, prec)   # k_it iterations + the initial preconditioning
        dt = (time.perf_counter() - t0) / (k_it + 1)
        what = {"mg": "flexible-CG iterations with the multigrid V-cycle",
                "cnn": "flexible-CG iterations with the network preconditioner",
                "mg_cnn": "flexible-CG iterations with the V-cycle and network smoother",
                "ssor": "CG iterations with the red-black SSOR preconditioner"}[solver]
    else:
        k_it = 3
        t0 = time.perf_counter()
        opic.pcg_jacobi(b, x0, Ns, h, 0.0, k_it)   # k_it iterations + the initial residual
        dt = (time.perf_counter() - t0) / (k_it + 1)
        what = "Jacobi-PCG iterations"
    scale = (N / Ns) ** 3
    desc = f"{k_it + 1} {what} on a {Ns}^3 grid" + (f" (scaled by cells x{scale:g})" if Ns != N else "")
    return dt * scale, desc


def cpu_sample(N, ppc, iters_per_solve, solver, Ns_solve=None, Ns_part=None):
    """Seconds of one step of the CPU oracle (numpy, FP64, as it stands) on
    one core, from a bounded sample: solver iterations of the same algorithm
    (scaled by cells and by the iterations per solve), and init-free
    deposit + gather + push + field energy of ppc particles per cell on an
    Ns_part^3 grid (scaled by cells: the oracle's particle work is linear in
    the particle count at fixed ppc). Returns (seconds, description)."""
    from oracle import pic as opic

    if solver == "pif":
        return cpu_sample_pif(N, ppc, Ns_solve or 16, Ns_part or 65536)
    t_cg, cg_desc = oracle_iteration_seconds(N, solver, Ns_solve)
    it = 1 if solver == "fft" else iters_per_solve
    if ppc == 0:
        return t_cg * it, f"{cg_desc}, scaled by {it:.0f} iterations/solve"
    Np_ = min(N, Ns_part or ORACLE_PARTICLE_GRID)
    L = 4.0 * np.pi
    ns = ppc * Np_ ** 3
    rng = np.random.default_rng(3)
    pos = rng.random((3, ns)) * L
    vel = rng.normal(size=(3, ns))
    phi = inputs_rhs(Np_)
    t0 = time.perf_counter()
    opic.deposit(pos, Np_, L)
    Ep = opic.gather(opic.gradient(phi, Np_, L / Np_), pos, Np_, L)
    opic.push(pos, vel, Ep, DT, L, kick=DT)
    opic.field_energy(phi, Np_, L / Np_)
    t_part = (time.perf_counter() - t0) * (N / Np_) ** 3
    return (t_cg * it + t_part,
            f"{cg_desc} (scaled by {it:.0f} iterations/solve); deposit + gather + push + field energy of "
            f"{ns} particles on a {Np_}^3 grid (scaled by cells x{(N / Np_) ** 3:g})")


def inputs_rhs(N):
    from paper_2605_05469_gb300 import inputs
    return inputs.landau_noise_rhs(N, 1)


_ORACLE_BARRIER = None


def _oracle_worker_init(barrier):
    global _ORACLE_BARRIER
    _ORACLE_BARRIER = barrier


def _oracle_worker_task(spec):
    _ORACLE_BARRIER.wait()   # all workers start their samples together
    return cpu_sample(*spec)


class OraclePool:
    """One single-threaded oracle process per host core (spawned, so it can
    start after CUDA is initialised). Each round runs the same sample on
    every process at once; the host's throughput is procs / the slowest
    process's scaled step time (the cores share memory bandwidth, which the
    concurrent run includes)."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        ctx = mp.get_context("spawn")
        self.barrier = ctx.Barrier(self.procs)
        self.pool = ctx.Pool(self.procs, initializer=_oracle_worker_init, initargs=(self.barrier,))

    def step_seconds(self, spec):
        res = self.pool.map(_oracle_worker_task, [spec] * self.procs, chunksize=1)
        return max(r[0] for r in res) / self.procs, res[0][1]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(N, ppc, iters_per_solve, solver="mixed", procs=None):
    """The CPU oracle (numpy, FP64, as it stands) on every host core: the
    bounded sample of cpu_sample run by one process per core at once."""
    pool = OraclePool(procs)
    try:
        step_s, desc = pool.step_seconds((N, ppc, iters_per_solve, solver))
    finally:
        pool.close()
    return {"value": 1.0 / step_s, "unit": "solves/s" if ppc == 0 else UNIT, "cores": pool.procs, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": f"per process: {desc}; {pool.procs} single-threaded processes at once, "
                      f"throughput = processes / slowest scaled step"}


def cpu_sample_pif(N, ppc, Ns=16, ns=65536):
    """Seconds of one particle-in-Fourier step of the CPU oracle on one core:
    its direct type-1/type-2 sums and push timed on ns particles with Ns^3
    modes, scaled to the step by particles x modes (the direct sums cost one
    term per particle and mode). Returns (seconds, description)."""
    from oracle import pic as opic
    from oracle import pif as opif

    L = 4.0 * np.pi
    rng = np.random.default_rng(3)
    pos = rng.random((3, ns)) * L
    vel = rng.normal(size=(3, ns))
    q = np.full(ns, -L ** 3 / ns)
    t0 = time.perf_counter()
    Er, _ = opif.field_at_particles(pos, q, Ns, L)
    t_field = time.perf_counter() - t0
    t0 = time.perf_counter()
    opic.push(pos, vel, Er, DT, L, kick=DT)
    t_push = time.perf_counter() - t0
    npart = ppc * N ** 3
    return (t_field * (npart / ns) * (N / Ns) ** 3 + t_push * (npart / ns),
            f"direct-sum field of {ns} particles on {Ns}^3 modes (scaled by particles x modes to {npart} x {N}^3) "
            f"and their push (scaled by particles)")


def cpu_baseline_pif(N, ppc, Ns=16, ns=65536, procs=None):
    """The particle-in-Fourier step of the CPU oracle on every host core (one
    process per core running the sample of cpu_sample_pif at once)."""
    pool = OraclePool(procs)
    try:
        step_s, desc = pool.step_seconds((N, ppc, 0, "pif", Ns, ns))
    finally:
        pool.close()
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "host_cpus": os.cpu_count(),
            "sample": f"per process: {desc}; {pool.procs} single-threaded processes at once, "
                      f"throughput = processes / slowest scaled step"}


def field_name(args):
    """How the step obtains its field when it is not the bench's Poisson solve
    (None for the solve)."""
    if args.solver == "fft":
        return "FFT pseudo-spectral solve with the spectral field"
    if args.solver == "pif":
        return f"particle-in-Fourier field ({args.N}^3 modes, NUFFT tol {args.pif_tol:g})"
    return None


def pic_config(args, world):
    """The `config` block of both arms' JSON lines."""
    solve_only = getattr(args, "workload", "pic") == "solve"
    N, ppc = args.N, args.ppc
    return {"workload": (f"Poisson solve, {N}^3 periodic grid, Landau density + N(0, 0.01^2) noise rhs, "
                         f"cold start, rel-res {TOL:g}") if solve_only else pic_workload(N, ppc, field_name(args)),
            "N": N, "ppc": 0 if solve_only else ppc, "particles": 0 if solve_only else ppc * N ** 3,
            "solver": args.solver, "tol": TOL, "dt": None if solve_only else DT, "warm_start": not solve_only,
            "parallelism": f"replicas x{world}", "l2": l2_note(N, ppc, solve_only)}


def pic_workload(N, ppc, field=None):
    """The name of the PIC-step workload (both arms): grid, particles, how the
    field is obtained (default: the Poisson solve to the bench tolerance)."""
    return (f"Landau PIC step, {N}^3 periodic grid x {ppc} ppc ({ppc * N ** 3} particles), "
            + (field or f"solve to rel-res {TOL:g}") + f", dt {DT}")


def oracle_iters_per_solve(N, ppc, solver):
    """Iterations of a warm-started solve of the PIC step for the CPU oracle:
    two steps of the oracle's loop on an N0^3 grid (deposit, cold solve,
    push, deposit, solve warm-started from the previous phi), the second
    solve's iterations with the step's algorithm, scaled to N^3 by the
    algorithm's growth: CG with a fixed-stencil preconditioner (Jacobi; the
    learned network, whose untrained oracle weights are exactly the Jacobi
    direction) like sqrt(kappa) ~ N, SSOR-CG like N^(1/2), multigrid FCG not
    at all. Returns (iterations, description)."""
    from oracle import cnn as ocnn
    from oracle import mg as omg
    from oracle import pic as opic
    from oracle import ssor as ossor
    if solver in ("fft", "pif"):
        return 1, "direct solve"
    N0 = min(N, 32)
    L = 4.0 * np.pi
    h = L / N0
    pos, vel = opic.init_particles(N0, ppc, SEED)
    jac = solver in ("mixed", "fp64", "cnn")

    def solve(b, x0):
        if jac:
            x, it, _, _ = opic.pcg_jacobi(b, x0, N0, h, TOL, MAXIT)
            return x, it
        prec = {"mg": lambda r: omg.vcycle(r, N0, h), "mg_cnn": lambda r: omg.vcycle(r, N0, h),
                "ssor": lambda r: ossor.ssor(r, N0, h)}[solver]
        out = ocnn.fcg(b, x0, N0, h, TOL, MAXIT, prec)
        return out[0], out[1]
    rho = opic.deposit(pos, N0, L)
    b = rho - rho.mean()
    phi, _ = solve(b, np.zeros(N0 ** 3))
    Ep = opic.gather(opic.gradient(phi, N0, h), pos, N0, L)
    pos, vel = opic.push(pos, vel, Ep, DT, L, kick=0.5 * DT)
    rho = opic.deposit(pos, N0, L)
    _, it0 = solve(rho - rho.mean(), phi)
    growth = {"ssor": (N / N0) ** 0.5, "mg": 1.0, "mg_cnn": 1.0}.get(solver, N / N0)
    what = "Jacobi-PCG" if jac else {"mg": "multigrid FCG", "mg_cnn": "multigrid FCG (Jacobi-smoothed)",
                                     "ssor": "SSOR-CG"}[solver]
    return (max(1.0, it0 * growth),
            f"{it0} iterations of a warm-started {what} solve at {N0}^3 x {ppc} ppc, scaled x{growth:g} to {N}^3")


def run_reference(args):
    """The CPU oracle, as it stands, on this arm's workload: every step is one
    round of the bounded sample of cpu_sample on one process per host core
    (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    N, ppc = args.N, args.ppc
    iters, it_desc = oracle_iters_per_solve(N, ppc, args.solver)
    # a small sample per step keeps the whole run within a few minutes
    spec = ((N, ppc, 0, "pif", 8, 16384) if args.solver == "pif" else
            (N, ppc, iters, args.solver, min(64, ORACLE_SOLVE_GRID.get(args.solver, 64)), 32))
    pool = OraclePool()
    t0 = time.perf_counter()
    try:
        for _ in range(max(0, args.warmup)):
            pool.step_seconds(spec)
        secs = []
        for _ in range(max(1, args.steps)):
            s_, desc = pool.step_seconds(spec)
            secs.append(s_)
    finally:
        pool.close()
    total = time.perf_counter() - t0
    value = float(f"{len(secs) / sum(secs):.6g}")
    cfg = pic_config(args, 1)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 / value, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (numpy)",
        "data": "synthetic: seeded Landau initial condition (Philox4x32-10, inverse CDF, Box-Muller)",
        "impl": "reference", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                         "host_cpus": os.cpu_count(),
                         "sample": f"per step and process: {desc}; iterations per solve: {it_desc}; "
                                   f"{pool.procs} single-threaded processes at once, throughput = processes / "
                                   f"slowest scaled step; {args.warmup} + {len(secs)} rounds in {total:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return out


def main():
    args = parse()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
