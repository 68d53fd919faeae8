"""Host-side helpers of bench.py: the byte accounting of the V-cycle levels
and the particle kernels, and the whole-job rate (no GPU)."""
import bench


def test_vcycle_level_fraction():
    # streamed levels of a 256^3 grid: 256, 128, 64, 32 (16 and below run in one block)
    assert abs(bench.mg_level_fraction(256) - (1 + 1 / 8 + 1 / 64 + 1 / 512)) < 1e-15
    # 48 -> 24 streamed, 12 in one block
    assert abs(bench.mg_level_fraction(48) - (1 + 1 / 8)) < 1e-15
    assert bench.mg_level_fraction(16) == 0.0


def test_vcycle_bytes_per_cell():
    # pre 8, residual 12, restriction 4.5, prolongation + sweep 12.5, sweep 12
    assert sum(bench.MG_BYTES.values()) == 49.0


def test_particle_kernel_bytes():
    # record read and written (128 B), key and rank (8 B)
    assert bench.PARTICLE_BYTES["push"][0] == 136
    assert bench.PARTICLE_BYTES["scatter"][0] == 136
    for k in ("push", "scatter"):
        assert abs(bench.MEASURED_TRAFFIC_PER_PARTICLE[k] - 136) < 5


def test_whole_job_rate_and_ranks():
    assert bench.whole_job_rate(4, 10, 2.0) == 20.0
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_pif_window_width():
    # about one digit a window point at oversampling 2: w = ceil(-log10 tol) + 1 in [4, 16]
    assert bench.pif_width(1e-4) == 5
    assert bench.pif_width(1e-6) == 7
    assert bench.pif_width(1e-12) == 13
    assert bench.pif_width(1e-2) == 4
    assert bench.pif_width(1e-20) == 16
    # flops of the window sums: a multiply and an add per point, component and particle
    assert bench.PIF_FLOP_PER_POINT == 2


def test_pif_cpu_baseline_scales_by_particles_and_modes():
    # the direct sums cost one term per (particle, mode): the sampled rate of a
    # 2x larger grid (8x the modes, 8x the particles at the same ppc) is ~64x lower
    a = bench.cpu_baseline_pif(16, 1, Ns=8, ns=1024)
    b = bench.cpu_baseline_pif(32, 1, Ns=8, ns=1024)
    assert a["kind"] == "oracle" and a["unit"] == bench.UNIT
    assert 16 < a["value"] / b["value"] < 256
