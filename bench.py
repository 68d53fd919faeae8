#!/usr/bin/env python
"""Benchmark of the Landau-damping PIC loop on GB300.

One step is one pass of the whole hot path of the PIC loop (Fig. 1) through
the library's C ABI: sort by cell + CIC scatter (pic_deposit), the Poisson
solve to relative residual 1e-10 (poisson_solve_ex), the field energy
(pic_field_energy) and E = -grad phi + CIC gather + leapfrog push
(pic_gather_push). Default workload: 256^3 periodic grid, 8 particles per cell
(134,217,728 particles, 64-byte records: fixed-point positions, double-float
velocities; 8.6 GB), Landau initial condition (k = 0.5, alpha = 0.05),
dt = 0.05, warm-started solves preconditioned by the multigrid V-cycle.
--solver selects the solve (mg, mg_cnn, cnn, ssor, mixed, fp64), the FFT-PIC
step (fft: spectral phi and E) or the particle-in-Fourier step (pif: NUFFTs,
no grid deposit or solve).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--solver ...]
  python bench.py --impl reference      # the CPU oracle on a bounded sample

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank runs its own
independent replica of the workload (the path has no exchange step on one
GPU); value = steps of all ranks / max time over ranks.
"""
import argparse
import json
import math
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
# ... which the tensor-core form executes as 81 Toeplitz products of K = 32
# x-inputs per output (9 of the 32 weights in each product are nonzero)
PRECOND_MMA_FLOP_PER_CELL = 2 * 81 * 32
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
# algorithmic bytes of the particle kernels: per particle, and per grid node
PARTICLE_BYTES = {
    # scatter: read and write the 64-byte record, read its key and rank, one
    # offset per particle (cached: counted once per cell)
    "scatter": (136, 4),
    # deposit: the record's first 32-byte sector (offsets), 8 corner sums per
    # cell written and read back (8 B each), the cell offsets, rho written
    "deposit": (32, 64 + 64 + 4 + 8),
    # push: read and write the 64-byte record, its key and rank; E (3 x 8 B) read
    # once per node
    "push": (136, 24),
}
# DRAM traffic per particle of one launch (dram__bytes_read.sum +
# dram__bytes_write.sum over the particle count) measured by ncu on the
# 128^3 x 8 ppc step (16.8 M particles; the traffic scales with the particle
# count): it stands for the same kernels at other sizes
# particle-in-Fourier window sums: a multiply and an atomic add (spreading)
# or one FMA (interpolation) per window point and particle
PIF_FLOP_PER_POINT = 2


def pif_width(tol):
    """Window width of the particle-in-Fourier NUFFTs for a relative tolerance
    (about one digit per point at oversampling 2), clamped to [4, 16]."""
    return min(16, max(4, int(math.ceil(-math.log10(tol))) + 1))


MEASURED_TRAFFIC_PER_PARTICLE = {"push": 136.70, "scatter": 133.72}
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
    ap.add_argument("--solver", choices=["mixed", "fp64", "cnn", "mg", "mg_cnn", "ssor", "fft", "pif"], default="mg",
                    help="mg (default, the fastest): mixed-precision flexible CG with a multigrid V-cycle (damped "
                         "Jacobi smoothing); cnn: flexible CG with the learned preconditioner (trained on the GPU "
                         "before timing); mg_cnn: the V-cycle with the learned network smoothing the finest level; "
                         "mixed: FP32 Jacobi-CG + FP64 reliable updates; fp64: the FP64 Jacobi-PCG reference; ssor: the "
                         "paper's PCG configuration (red-black SSOR, 4 inner, 2 outer, damping pi/2); fft: the "
                         "paper's other scheme, the FFT pseudo-spectral solve (cuFFT FP64) with the spectral field "
                         "pushed to the particles; pif: the particle-in-Fourier scheme (NUFFTs, no grid deposit "
                         "or solve). The learned solvers are always trained and timed in the solve comparison as "
                         "well")
    ap.add_argument("--pif-tol", type=float, default=1e-4,
                    help="relative tolerance of the particle-in-Fourier NUFFTs (sets the window width; 1e-4 as in the paper's runs)")
    ap.add_argument("--cnn-apply", choices=["tc", "tc_fused", "fp32", "layers"], default="tc",
                    help="evaluation of the learned preconditioner: composed 9^3 kernel on the tensor cores "
                         "(BF16), on the CUDA cores (FP32), or the four BF16 convs")
    ap.add_argument("--workload", choices=["pic", "solve"], default="pic",
                    help="pic: full PIC step; solve: one cold-start Poisson solve of a Landau density + noise rhs")
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--ppc", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-vs-mixed solve comparison")
    ap.add_argument("--compare-reps", type=int, default=2, help="cold solves per solver in the comparison (best kept)")
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
    prec = pg.PREC_FP64 if args.solver == "fp64" else pg.PREC_MIXED
    pc = {"cnn": pg.PC_CNN, "mg": pg.PC_MG, "mg_cnn": pg.PC_MG_CNN, "ssor": pg.PC_SSOR}.get(args.solver,
                                                                                          pg.PC_JACOBI)
    stream = torch.cuda.current_stream()
    solve_only = args.workload == "solve"
    weights, train_info = None, None
    if args.solver in ("cnn", "mg_cnn") or not args.no_compare:
        weights, train_info = train_preconditioner(pg, torch)
    c = pg.Context(stream).init(N, 0 if solve_only else ppc, SEED + rank)
    apply_mode = {"tc": pg.CNN_APPLY_TC, "tc_fused": pg.CNN_APPLY_TC_FUSED, "fp32": pg.CNN_APPLY_FP32,
                  "layers": pg.CNN_APPLY_LAYERS}[args.cnn_apply]
    if weights is not None and pc in (pg.PC_CNN, pg.PC_MG_CNN):
        c.cnn_set_weights(weights)
        c.cnn_set_apply(apply_mode)
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    if solve_only:
        from paper_2605_05469_gb300 import inputs
        rho = inputs.landau_noise_rhs_torch(N, 0xC0FFEE + rank, "cuda")
    else:
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
    infos = []

    use_fft = args.solver == "fft"
    use_pif = args.solver == "pif"
    E3 = torch.empty(3 * n, dtype=torch.float64, device="cuda") if use_fft else None

    def solve_into(rho_, phi_):
        if use_fft:
            # direct solve: no iterations or residual; its time is the solve phase's
            c.fft_solve(rho_, phi_, E3)
            return {"iters": 0, "t_ms": None, "rel_res": 0.0, "reliable_updates": 0, "converged": True}
        return c.solve(rho_, phi_, tol=TOL, maxit=MAXIT, precision=prec, precond=pc)

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

    for _ in range(args.warmup):
        step(False)
    c.profile(True)
    c.profile_read(reset=True)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

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

    # end to end through the public API, host wall clock: per step the host
    # reads back the step's result (field energy, 3 doubles) and the solver's
    # status; the particle state is device resident by design.
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(False)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": whole_job_rate(world, args.steps, e2e_s), "unit": unit, "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": 0 if solve_only else 24,
           "note": "wall clock through the Python binding; per step the field energy is read to host"}

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
        solve_into(rho, phi)
        phi_host.copy_(phi, non_blocking=True)
    torch.cuda.synchronize()
    e2e_solve = {"value": reps / (time.perf_counter() - t0), "unit": "solves/s (cold start)",
                 "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8}

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
        if prof["ker_samples"]["precond"]:
            # the whole cycle (all levels, the one-block coarse cycle, and with
            # the learned smoother its two network applications) for context
            avg_ms = prof["ker_ms"]["precond"] / prof["ker_samples"]["precond"]
            frac = mg_level_fraction(N)
            jac = sum(MG_BYTES.values())
            # learned smoother on the finest level: network r -> x (8), residual,
            # restriction, residual of x + P e_c, network res -> x (8), x += t (12)
            fine = jac if pc == pg.PC_MG else (8 + MG_BYTES["mg_resid"] + MG_BYTES["mg_restrict"] +
                                               MG_BYTES_PROLONG_RESID + 8 + 12)
            bpc = fine + jac * (frac - 1.0)
            vcycle = {"avg_us": round(avg_ms * 1e3, 2), "samples": prof["ker_samples"]["precond"],
                      "bytes_per_fine_cell": round(bpc, 3), "gbs": round(bpc * n / (avg_ms * 1e-3) / 1e9, 1),
                      "note": "one V-cycle, every level; bytes of the plane-streamed levels"}
    # the particle kernels (one launch each per step)
    np_ = 0 if solve_only else ppc * n
    for k, (bp, bn) in PARTICLE_BYTES.items():
        if not np_ or not prof["ker_samples"].get(k):
            continue
        avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
        b = bp * np_ + bn * n
        rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k], "bytes_per_particle": bp,
                   "bytes_per_node": bn, "gbs": b / (avg_ms * 1e-3) / 1e9, "launches_per_step": 1}
    # particle-in-Fourier: the spreading kernel (the charge) and the
    # interpolation kernel (the three field components at once), one launch
    # each a step; FP64 window sums over w^3 grid points a particle
    if use_pif:
        w_pif = pif_width(args.pif_tol)
        for k, comps in (("pif_spread", 1), ("pif_gather", 3)):
            if not prof["ker_samples"].get(k):
                continue
            avg_ms = prof["ker_ms"][k] / prof["ker_samples"][k]
            flop = PIF_FLOP_PER_POINT * comps * w_pif ** 3 * np_
            rows[k] = {"avg_us": avg_ms * 1e3, "samples": prof["ker_samples"][k], "window_points": w_pif ** 3,
                       "components": comps, "fp64_flop": flop, "tflops": flop / (avg_ms * 1e-3) / 1e12,
                       "launches_per_step": 1}
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
        roof = {"kernel": {"pif_spread": "k_pif_spread (type-1 NUFFT spreading, FP64 atomics)",
                           "pif_gather": "k_pif_gather3 (type-2 NUFFT interpolation, three components)"}[dom],
                "bound": "alu", "achieved": round(r["tflops"], 4), "peak": fp64_peak_tflops(),
                "unit": "FP64 TFLOP/s", "frac": round(r["tflops"] / fp64_peak_tflops(), 4),
                "peak_source": "measured FP64 FMA loop", "traffic": None, "algorithmic_flop": r["fp64_flop"],
                "avg_launch_us": round(r["avg_us"], 2),
                "note": "window sums: 2 FP64 flops per window point, component and particle (window "
                        "evaluation not counted)"}
    elif dom == "precond" and apply_mode in (pg.CNN_APPLY_TC, pg.CNN_APPLY_TC_FUSED):
        r = rows[dom]
        _, _, pk = peaks()
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        roof = {"kernel": "k_apply_k_tc (composed 9^3 learned preconditioner, tcgen05 BF16)", "bound": "tensor",
                "achieved": round(r["tflops"], 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(r["tflops"] / peak, 4),
                "peak_source": "measured bf16_tflops_sustained (kernel timed inside a long solve)",
                "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n,
                "executed_mma_tflops": round(r["tflops"] * PRECOND_MMA_FLOP_PER_CELL / PRECOND_FLOP_PER_CELL, 2),
                "avg_launch_us": round(r["avg_us"], 2)}
    elif dom == "precond":
        r = rows[dom]
        roof = {"kernel": "k_apply_k (composed 9^3 learned preconditioner)", "bound": "alu",
                "achieved": round(r["tflops"], 2), "peak": FP32_PEAK_TFLOPS, "unit": "FP32 TFLOP/s",
                "frac": round(r["tflops"] / FP32_PEAK_TFLOPS, 4),
                "peak_source": "measured FP32 FMA loop (no FP32 figure in MEASURED_PEAKS.json)",
                "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n, "avg_launch_us": round(r["avg_us"], 2)}
    elif dom in PARTICLE_BYTES:
        r = rows[dom]
        b = r["bytes_per_particle"] * np_ + r["bytes_per_node"] * n
        roof = {"kernel": {"scatter": "k_scatter (sort: 64-byte records to their cells)",
                           "deposit": "k_deposit_cells + k_deposit_nodes (CIC scatter)",
                           "push": "k_gather_push (CIC gather + leapfrog, double-float)"}[dom],
                "bound": "hbm", "achieved": round(r["gbs"], 1), "peak": hbm, "unit": "GB/s",
                "frac": round(r["gbs"] / hbm, 4), "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": (round(MEASURED_TRAFFIC_PER_PARTICLE[dom] * np_) if dom in MEASURED_TRAFFIC_PER_PARTICLE
                            else None),
                "traffic_source": ("ncu DRAM bytes per particle at 128^3 x 8 ppc, scaled by the particle count"
                                   if dom in MEASURED_TRAFFIC_PER_PARTICLE else None),
                "algorithmic_bytes": b, "avg_launch_us": round(r["avg_us"], 2),
                "note": "dominant kernel of the whole step (device time per step)"}
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
        "dtype": ("f64" if prec == pg.PREC_FP64 else
                  "f64 particles/grid; solve f32 vectors + f64 reductions" +
                  ((f"; {'bf16 tensor-core' if args.cnn_apply == 'tc' else args.cnn_apply} "
                    "9^3 learned preconditioner") if pc == pg.PC_CNN else "") +
                  ("; f32 multigrid V-cycle" if pc == pg.PC_MG and not use_fft else "") +
                  ("; FP64 spectral solve (cuFFT)" if use_fft else "") +
                  (f"; FP64 particle-in-Fourier NUFFTs (tol {args.pif_tol:g})" if use_pif else "") +
                  ("; f32 multigrid V-cycle, learned finest-level smoother" if pc == pg.PC_MG_CNN else "")),
        "data": "synthetic: seeded Landau initial condition (Philox4x32-10, inverse CDF, Box-Muller)",
        "config": {"workload": (f"Poisson solve, {N}^3 periodic grid, Landau density + N(0, 0.01^2) noise rhs, "
                                f"cold start, rel-res {TOL:g}") if solve_only else
                               pic_workload(N, ppc, field_name(args)),
                   "N": N, "ppc": ppc, "particles": ppc * n, "solver": args.solver, "tol": TOL, "dt": DT,
                   "warm_start": True, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (particle records 8.6 GB; solver vectors 4 x 67-134 MB per iteration)"},
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
    if train_info is not None:
        out["preconditioner_training"] = train_info
    if not args.no_compare:
        if weights is not None:
            c.cnn_set_weights(weights)
        out["solve_compare"], learned_roof = compare_solvers(c, rho, n, pg, torch, with_cnn=weights is not None,
                                                             reps=args.compare_reps, maxit=args.compare_maxit)
        if learned_roof is not None:
            out["roofline_learned_preconditioner"] = learned_roof
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = (cpu_baseline_pif(N, ppc) if use_pif else
                               cpu_baseline(N, 0 if solve_only else ppc, statistics.mean(iters), args.solver))
    if dist is not None:
        dist.destroy_process_group()
    c.close()
    return out


def train_preconditioner(pg, torch, N=64, steps=600, val_grid=128, val_every=100):
    """Train the learned preconditioner on the GPU before timing (the library's
    own kernels: Jacobi-PCG snapshots of four 64^3 Landau deposits, 600 Adam
    steps on 32^3 crops); the weights kept are those with the fewest
    flexible-CG iterations, scored every 100 steps on a held-out 128^3
    deposit (another seed)."""
    from paper_2605_05469_gb300 import train as T
    t0 = time.perf_counter()
    sets = T.landau_snapshot_sets(N, seeds=[11, 12, 13, 14])
    c = pg.Context().init(N, 0, 0)
    val = T.fcg_iterations(val_grid)
    losses = T.train(c, sets, steps, B=8, D=32, lr=2e-3, seed=0, validate=val, validate_every=val_every)
    w = c.cnn_get_weights()
    c.close()
    del sets, val
    torch.cuda.synchronize()
    return w, {"grid": N, "steps": steps, "loss_first": float(losses[:10].mean()),
               "loss_last": float(losses[-50:].mean()), "selected_by": f"FCG iterations on a {val_grid}^3 deposit",
               "seconds": round(time.perf_counter() - t0, 2)}


def compare_solvers(c, rho, n, pg, torch, with_cnn=False, reps=2, maxit=MAXIT):
    """Cold-start solves of the same right-hand side (the last deposit): the FP64
    Jacobi-PCG reference against the mixed-precision solvers (Jacobi-CG, flexible
    CG with the multigrid V-cycle, and with the learned preconditioner and the
    V-cycle with the learned smoother when the network is loaded), outside the
    timed region."""
    res = {}
    cases = [("fp64_jacobi_pcg", pg.PREC_FP64, pg.PC_JACOBI), ("mixed_fp32_fp64", pg.PREC_MIXED, pg.PC_JACOBI),
             ("mixed_fcg_multigrid", pg.PREC_MIXED, pg.PC_MG),
             ("mixed_cg_ssor_paper_configuration", pg.PREC_MIXED, pg.PC_SSOR)]
    if with_cnn:
        cases.append(("mixed_fcg_learned", pg.PREC_MIXED, pg.PC_CNN))
        cases.append(("mixed_fcg_learned_fp32", pg.PREC_MIXED, pg.PC_CNN))
        cases.append(("mixed_fcg_multigrid_learned_smoother", pg.PREC_MIXED, pg.PC_MG_CNN))
    learned_roof = None
    for name, prec, pc in cases:
        if with_cnn:
            c.cnn_set_apply(pg.CNN_APPLY_FP32 if name.endswith("_fp32") else pg.CNN_APPLY_TC)
        best = None
        # the tensor-core preconditioner's launches are sampled in the first
        # learned solve for its roofline
        sample = name == "mixed_fcg_learned"
        if sample:
            c.profile(True)
            c.profile_read(reset=True)
        for _ in range(max(1, reps)):
            phi = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = c.solve(rho, phi, tol=TOL, maxit=maxit, precision=prec, precond=pc, raise_on_error=False)
            if best is None or info["t_ms"] < best["t_ms"]:
                best = info
        if sample:
            prof = c.profile_read(reset=True)
            c.profile(False)
            learned_roof = tc_roofline(prof, n)
        res[name] = {"s": best["t_ms"] / 1e3, "iters": best["iters"], "rel_res": best["rel_res"],
                     "converged": bool(best["converged"])}
    # the paper's FFT scheme: the spectral solve of the same right-hand side
    # (phi and the three spectral field components), cold, CUDA-event timed
    E3 = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    c.fft_solve(rho, phi, E3)  # plans
    best = None
    for _ in range(max(1, reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0.record(stream)
        c.fft_solve(rho, phi, E3)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None or t < best else best
    res["fft_spectral_phi_and_E"] = {"s": best, "note": "direct solve of the continuous-symbol equation "
                                                        "(Sec. 3.1), not the finite-difference system"}
    best = None
    for _ in range(max(1, reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c.fft_solve(rho, phi)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None or t < best else best
    res["fft_spectral_phi"] = {"s": best, "note": "phi alone: one forward and one inverse transform"}
    del E3
    res["speedup_mixed_vs_fp64"] = res["fp64_jacobi_pcg"]["s"] / res["mixed_fp32_fp64"]["s"]
    res["fp64_pcg_vs_fft_time_ratio"] = res["fp64_jacobi_pcg"]["s"] / res["fft_spectral_phi_and_E"]["s"]
    res["speedup_multigrid_vs_fp64"] = res["fp64_jacobi_pcg"]["s"] / res["mixed_fcg_multigrid"]["s"]
    res["speedup_ssor_vs_fp64"] = res["fp64_jacobi_pcg"]["s"] / res["mixed_cg_ssor_paper_configuration"]["s"]
    if with_cnn:
        res["speedup_learned_vs_fp64"] = res["fp64_jacobi_pcg"]["s"] / res["mixed_fcg_learned"]["s"]
        res["speedup_learned_fp32_vs_fp64"] = res["fp64_jacobi_pcg"]["s"] / res["mixed_fcg_learned_fp32"]["s"]
        res["speedup_multigrid_learned_vs_fp64"] = (res["fp64_jacobi_pcg"]["s"] /
                                                     res["mixed_fcg_multigrid_learned_smoother"]["s"])
    return res, learned_roof


def tc_roofline(prof, n):
    """Roofline of the tensor-core learned preconditioner (k_apply_k_tc) from
    its sampled launches: algorithmic FLOP of the composed 9^3 kernel per
    launch over the average CUDA-event duration, against the measured
    sustained BF16 peak."""
    k = prof["ker_samples"]["precond"]
    if not k:
        return None
    avg_ms = prof["ker_ms"]["precond"] / k
    tf = PRECOND_FLOP_PER_CELL * n / (avg_ms * 1e-3) / 1e12
    _, _, pk = peaks()
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    return {"kernel": "k_apply_k_tc (composed 9^3 learned preconditioner, tcgen05 BF16)", "bound": "tensor",
            "achieved": round(tf, 2), "peak": peak, "unit": "TFLOP/s", "frac": round(tf / peak, 4),
            "peak_source": "measured bf16_tflops_sustained (kernel timed inside a long solve)",
            "traffic": None, "algorithmic_flop": PRECOND_FLOP_PER_CELL * n,
            "executed_mma_tflops": round(tf * PRECOND_MMA_FLOP_PER_CELL / PRECOND_FLOP_PER_CELL, 2),
            "avg_launch_us": round(avg_ms * 1e3, 2), "samples": k}


# --------------------------------------------------------------------------- oracle
def oracle_iteration_seconds(N, solver):
    """Seconds of one solver iteration of the CPU oracle (as it stands) on an
    N^3 grid, with the same algorithm as the GPU solver: Jacobi-PCG for the
    mixed and FP64 solvers (timed on the full grid), flexible CG with the
    V-cycle or with the network (timed on a smaller grid and scaled by the
    cell count, the oracle's cost being linear in it)."""
    from oracle import cnn as ocnn
    from oracle import mg as omg
    from oracle import pic as opic
    from paper_2605_05469_gb300 import inputs

    L = 4.0 * np.pi
    Ns = min(N, {"mg": 128, "cnn": 32, "mg_cnn": 32, "ssor": 64}.get(solver, N))
    h = L / Ns
    b = inputs.landau_noise_rhs(Ns, 1)
    x0 = np.zeros(Ns ** 3)
    if solver == "fft":
        from oracle import fft as offt
        h = L / N
        b = inputs.landau_noise_rhs(N, 1)
        t0 = time.perf_counter()
        offt.spectral_solve(b, N, L)
        return time.perf_counter() - t0, f"one spectral solve (numpy FFT, phi and E) on the full {N}^3 grid"
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


def cpu_baseline(N, ppc, iters_per_solve, solver="mixed", reference_iters=None, budget_s=20.0):
    """The CPU oracle (numpy, FP64, as it stands) timed on a bounded sample of
    the same step: solver iterations of the same algorithm as the GPU solve
    and the particle kernels on a subset of particles, scaled to one step."""
    from oracle import pic as opic

    L = 4.0 * np.pi
    h = L / N
    n = N ** 3
    t_cg, cg_desc = oracle_iteration_seconds(N, solver)
    it = reference_iters if reference_iters else iters_per_solve
    if solver == "fft":
        it = 1  # a direct solve
    if ppc == 0:
        step_s = t_cg * it
        return {"value": 1.0 / step_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "host_cpus": os.cpu_count(),
                "sample": f"{cg_desc}, scaled by {it:.0f} iterations/solve"}
    ns = min(ppc * n, 1 << 21)
    rng = np.random.default_rng(3)
    pos = rng.random((3, ns)) * L
    vel = rng.normal(size=(3, ns))
    phi = np.zeros(n)
    t0 = time.perf_counter()
    opic.deposit(pos, N, L)
    Ep = opic.gather(opic.gradient(phi, N, h), pos, N, L)
    opic.push(pos, vel, Ep, DT, L, kick=DT)
    t_part = (time.perf_counter() - t0) * (ppc * n / ns)
    t0 = time.perf_counter()
    opic.field_energy(phi, N, h)
    t_en = time.perf_counter() - t0
    step_s = t_cg * it + t_part + t_en
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": f"{cg_desc} (scaled by {it:.0f} iterations/solve), "
                      f"deposit+gather+push of {ns} of {ppc * n} particles (scaled linearly), one field energy"}


def cpu_baseline_pif(N, ppc, Ns=16, ns=65536):
    """The CPU oracle's particle-in-Fourier field (direct type-1/type-2 sums)
    and push timed on ns particles with Ns^3 modes, scaled to the step by
    particles x modes (the direct sums cost one term per particle and mode)."""
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
    step_s = t_field * (npart / ns) * (N / Ns) ** 3 + t_push * (npart / ns)
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": 1, "kind": "oracle", "host_cpus": os.cpu_count(),
            "sample": f"direct-sum field of {ns} particles on {Ns}^3 modes (scaled by particles x modes "
                      f"to {npart} x {N}^3) and their push (scaled by particles)"}


def field_name(args):
    """How the step obtains its field when it is not the bench's Poisson solve
    (None for the solve)."""
    if args.solver == "fft":
        return "FFT pseudo-spectral solve with the spectral field"
    if args.solver == "pif":
        return f"particle-in-Fourier field ({args.N}^3 modes, NUFFT tol {args.pif_tol:g})"
    return None


def pic_workload(N, ppc, field=None):
    """The name of the PIC-step workload (both arms): grid, particles, how the
    field is obtained (default: the Poisson solve to the bench tolerance)."""
    return (f"Landau PIC step, {N}^3 periodic grid x {ppc} ppc ({ppc * N ** 3} particles), "
            + (field or f"solve to rel-res {TOL:g}") + f", dt {DT}")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    N, ppc = args.N, args.ppc
    iters = None
    if args.solver not in ("fft", "pif"):
        # iterations per warm-started solve: the oracle's Jacobi-PCG on this
        # workload needs the same count as any exact-arithmetic CG; measured once
        # at 64^3 and scaled by N (CG iterations grow like sqrt(kappa) ~ N).
        from oracle import pic as opic
        N0 = 64
        pos, _ = opic.init_particles(N0, ppc, SEED)
        L = 4.0 * np.pi
        rho = opic.deposit(pos, N0, L)
        _, it0, _, _ = opic.pcg_jacobi(rho, np.zeros(N0 ** 3), N0, L / N0, TOL, MAXIT)
        iters = it0 * N / N0
    t0 = time.perf_counter()
    base = None
    for _ in range(max(1, args.steps)):
        if args.solver == "pif":
            base = cpu_baseline_pif(N, ppc)
        elif args.solver == "fft":
            base = cpu_baseline(N, ppc, 1, "fft")
        else:
            base = cpu_baseline(N, ppc, iters)
    total = time.perf_counter() - t0
    value = float(f"{base['value']:.6g}")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 / value, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Landau density + particles", "impl": "reference",
        "config": {"workload": pic_workload(N, ppc, field_name(args)), "solver": args.solver,
                   "N": N, "ppc": ppc, "iters_per_solve_est": iters},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": base["sample"] + f"; {args.steps} samples in {total:.1f} s"},
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
