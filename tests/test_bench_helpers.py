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
    # algorithmic: the FP64 state (x, y, z, vx, vy, vz: 48 B) read and written
    # by the push, positions read by the deposit, E read once per node
    assert bench.PARTICLE_BYTES["push"] == (96, 24)
    assert bench.PARTICLE_BYTES["deposit"] == (24, 8)
    # the library's record layout: 64-byte record (with its cell key and
    # in-cell rank) read and written
    assert bench.PARTICLE_IMPL_BYTES["push"] == 128
    assert bench.PARTICLE_IMPL_BYTES["scatter"] == 128
    for k in ("push", "scatter"):
        assert abs(bench.MEASURED_TRAFFIC_PER_PARTICLE[k] - 128) < 5


def test_particle_roofline_counts_algorithmic_bytes():
    # 256^3 x 8 ppc, push at 4991.4 us: 96 B a particle + 24 B a node
    n, np_ = 256 ** 3, 8 * 256 ** 3
    b = 96 * np_ + 24 * n
    rows = {"push": {"avg_us": 4991.4, "bytes_per_particle": 96, "bytes_per_node": 24,
                     "gbs": b / 4991.4e-6 / 1e9, "impl_bytes_per_particle": 128}}
    r = bench.particle_roofline(rows, "push", np_, n, 6787.2, "measured")
    assert r["algorithmic_bytes"] == b
    assert abs(r["frac"] - b / 4991.4e-6 / 1e9 / 6787.2) < 1e-4
    assert abs(r["frac"] - 0.392) < 0.002
    assert abs(r["traffic_over_algorithmic"] - bench.MEASURED_TRAFFIC_PER_PARTICLE["push"] * np_ / b) < 1e-3


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


def test_pif_cpu_sample_scales_by_particles_and_modes():
    # the direct sums cost one term per (particle, mode): the sampled time of a
    # 2x larger grid (8x the modes, 8x the particles at the same ppc) is ~64x higher
    a, _ = bench.cpu_sample_pif(16, 1, Ns=8, ns=1024)
    b, _ = bench.cpu_sample_pif(32, 1, Ns=8, ns=1024)
    assert 16 < b / a < 256


def test_cpu_baseline_uses_every_core():
    r = bench.cpu_baseline(16, 2, 5, "mixed", procs=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0
    assert "Jacobi-PCG" in r["sample"] and "2 single-threaded processes" in r["sample"]


def test_dtype_label_names_the_arithmetic():
    import types
    pg = types.SimpleNamespace()
    d = bench.dtype_label(pg, "cnn")
    assert "64-bit fixed-point positions + double-float velocities" in d
    assert "rho, phi FP64" in d and "FP32 vectors + FP64 reductions" in d and "BF16 tensor-core" in d
    assert "particles" not in bench.dtype_label(pg, "mg", solve_only=True)


def test_host_state_buffer_is_zeroed_and_sized():
    """The end-to-end particle state buffer (huge-page backed where the
    kernel allows): zeroed, FP64, the requested length, writable."""
    import torch
    t, _ = bench.host_state_buffer(3 * 1000003, torch)
    assert t.dtype == torch.float64 and t.numel() == 3 * 1000003
    assert float(t.abs().max()) == 0.0
    t[-1] = 2.5
    assert float(t.sum()) == 2.5
