"""GPU parity: every C-ABI call of the PIC loop against the CPU oracle on the
same seeded inputs, element by element, at sizes spanning several slabs and
the single-slab case, plus edge cases and full-size properties.

Tolerances (FP64 everywhere on these paths; differences come from rounding
order, FMA contraction and libm vs CUDA sin/cos/log at the ulp level):
  operator / gradient / energy: 1e-12 relative;
  initial particles: 1e-12 absolute (positions are O(L = 12.6));
  deposit: 1e-12 absolute on rho = O(1);
  solve: phi rel-L2 <= 1e-10 against the exact discrete solution at tol 1e-12;
  40-step loop: particles within 1e-10, field energy rel 1e-8 (the stated
  accuracy targets), with solves at tol 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pic as opic  # noqa: E402
from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

K = 0.5
L = 2.0 * np.pi / K


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def solver_ctx(pg, N):
    return pg.Context().init(N, 0, 0)


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("N", [8, 16, 24, 40, 64, 128])
def test_apply_laplacian_matches_oracle(pg, N):
    c = solver_ctx(pg, N)
    x = inputs.noise_field(N, N)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.apply_laplacian(dev(x), y)
    ref = opic.apply_A(x, N, L / N)
    got = host(y)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [256, 512, 1024])
def test_apply_laplacian_fourier_modes_full_size(pg, N):
    """A x for x a sum of three Fourier modes equals the sum of the modes times
    their closed-form eigenvalues (4/h^2) sum_d sin^2(pi m_d / N), at every
    cell; covers the 4-, 2- and 1-row slab geometries."""
    h = L / N
    c = solver_ctx(pg, N)
    i = torch.arange(N, device="cuda", dtype=torch.float64)
    modes = [((1, 0, 0), 1.0), ((0, 3, 2), 0.5), ((5, 1, N // 2), -0.25)]
    x = torch.zeros(N, N, N, dtype=torch.float64, device="cuda")
    ref = torch.zeros_like(x)
    for (mx, my, mz), a in modes:
        th = (2 * np.pi / N) * (mx * i[None, None, :] + my * i[None, :, None] + mz * i[:, None, None])
        v = a * torch.cos(th)
        x += v
        ref += opic.laplacian_eigenvalue((mx, my, mz), N, h) * v
        del th, v
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.apply_laplacian(x.reshape(-1), y)
    err = (y.reshape(N, N, N) - ref).abs().max().item()
    assert err <= 1e-10 * ref.abs().max().item()


# ------------------------------------------------------------------ solve
@pytest.mark.parametrize("N", [8, 16, 24, 32])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_exact_discrete_solution(pg, N, precision):
    c = solver_ctx(pg, N)
    h = L / N
    b = inputs.noise_field(N, 100 + N, mean=0.7)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    info = c.solve(dev(b), phi, tol=1e-12, maxit=5000, precision=precision)
    ref = opic.spectral_solve(b, N, h)
    got = host(phi)
    assert info["converged"] and info["rel_res"] <= 1e-12
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    assert abs(got.mean()) <= 1e-14 * np.abs(ref).max()
    if precision == 0:
        _, it, _, _ = opic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-12, 5000)
        assert abs(info["iters"] - it) <= 2


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_tolerance_1e10_landau_rhs(pg, precision):
    N = 64
    c = solver_ctx(pg, N)
    h = L / N
    b = inputs.landau_noise_rhs(N, 7)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    info = c.solve(dev(b), phi, tol=1e-10, maxit=5000, precision=precision)
    got = host(phi)
    bp = b - b.mean()
    r = bp - opic.apply_A(got, N, h)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(bp)
    ref, _, _, _ = opic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-13, 5000)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    if precision == 1:
        assert info["reliable_updates"] >= 1


def test_solve_edge_cases(pg):
    N = 16
    h = L / N
    c = solver_ctx(pg, N)
    b = inputs.noise_field(N, 5)
    exact = opic.spectral_solve(b, N, h)
    for prec in (0, 1):
        # zero right-hand side (constant rho): phi = 0 whatever the warm start
        phi = dev(np.ones(N ** 3))
        info = c.solve(dev(np.full(N ** 3, 3.0)), phi, precision=prec)
        assert info["converged"] and np.all(host(phi) == 0.0)
        # warm start at the solution: no iterations
        phi = dev(exact)
        info = c.solve(dev(b), phi, tol=1e-8, precision=prec)
        assert info["iters"] == 0 and info["converged"]
        # maxit too small: PIC_ENOCONV, info filled, phi holds the last iterate
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(dev(b), phi, tol=1e-12, maxit=3, precision=prec, raise_on_error=False)
        assert info["code"] == pg.PIC_ENOCONV and info["iters"] == 3 and not info["converged"]
        assert np.isfinite(host(phi)).all()
        # a NaN in rho: breakdown, no hang
        bad = b.copy()
        bad[17] = np.nan
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(dev(bad), phi, precision=prec, raise_on_error=False)
        assert info["code"] == pg.PIC_EBREAKDOWN


def test_solve_rejects_bad_arguments(pg):
    c = solver_ctx(pg, 16)
    rho = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        c.solve(rho, torch.zeros(15, dtype=torch.float64, device="cuda"))
    code, _ = pg.poisson_solve_ex(c.h, rho, rho.clone(), -1.0, 10, c.n)
    assert code == pg.PIC_EINVAL
    with pytest.raises(pg.PicError):
        pg.Context().init(12, 1, 0)  # N % 8 != 0


# ------------------------------------------------------------------ particles
@pytest.mark.parametrize("N,ppc,mode,vth,alpha", [(8, 3, 0, 1.0, 0.05), (16, 8, 0, 1.0, 0.05), (16, 8, 1, 1.0, 0.05),
                                                  (16, 4, 1, 1.7, 0.3), (8, 2, 0, 0.5, 0.3)])
def test_init_particles_match_oracle(pg, N, ppc, mode, vth, alpha):
    """Every particle against the oracle's: the paper's product density by
    inverse CDF (mode 0) and the sum density by rejection (mode 1, the same
    Philox trials; an accept decision is an FP64 comparison on both sides,
    so a cos that differs in its last bit could flip one only within
    ~1e-16 of the boundary), velocities scaled by v_th."""
    c = pg.Context().init(N, ppc, 0x5EED, alpha=alpha, vth=vth, init_mode=mode)
    got, half = c.particles()
    pos, vel = opic.init_particles(N, ppc, 0x5EED, alpha=alpha, vth=vth, mode=mode)
    assert not half
    assert np.max(np.abs(got[:3] - pos)) <= 1e-12
    assert np.max(np.abs(got[3:] - vel)) <= 1e-12 * vth


def test_init_rejects_bad_parameters(pg):
    c = pg.Context()
    for kw in ({"init_mode": 2}, {"init_mode": 1, "alpha": 0.4}, {"vth": -1.0}, {"vth": float("nan")},
               {"alpha": 1.0}):
        with pytest.raises(pg.PicError) as e:
            c.init(8, 1, 1, **kw)
        assert e.value.code == pg.PIC_EINVAL, kw
    c.init(8, 1, 1, vth=0.0)   # 0 selects v_th = 1
    got, _ = c.particles()
    ref_pos, ref_vel = opic.init_particles(8, 1, 1)
    assert np.max(np.abs(got[3:] - ref_vel)) <= 1e-12
    c.close()


@pytest.mark.parametrize("N,ppc", [(8, 8), (16, 8), (32, 2)])
def test_deposit_matches_oracle(pg, N, ppc):
    c = pg.Context().init(N, ppc, 11)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    pos, _ = opic.init_particles(N, ppc, 11)
    ref = opic.deposit(pos, N, L)
    got = host(rho)
    assert np.max(np.abs(got - ref)) <= 1e-12
    # charge conservation (Eq. 2): sum rho h^3 = 0 up to rounding
    assert abs(got.sum()) * (L / N) ** 3 <= 1e-9
    # deposit twice without a push: particles stay sorted, same result
    c.deposit(rho)
    assert np.max(np.abs(host(rho) - got)) <= 1e-13


def test_gradient_push_and_energy_match_oracle(pg):
    N, ppc = 16, 8
    h = L / N
    c = pg.Context().init(N, ppc, 3)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    c.solve(rho, phi, tol=1e-13)
    W = c.field_energy(phi)
    phi_h = host(phi)
    assert np.allclose(W, opic.field_energy(phi_h, N, h), rtol=1e-12, atol=0)
    c.gather_push(phi, 0.05)
    got, half = c.particles()
    assert half
    pos, vel = opic.init_particles(N, ppc, 3)
    Ep = opic.gather(opic.gradient(phi_h, N, h), pos, N, L)
    pos, vel = opic.push(pos, vel, Ep, 0.05, L, kick=0.025)
    d = np.abs(got[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-12
    assert np.max(np.abs(got[3:] - vel)) <= 1e-12
    # closing half-kick makes velocities synchronous again
    c.sync_velocity(phi, 0.05)
    got2, half2 = c.particles()
    assert not half2
    Ep2 = opic.gather(opic.gradient(phi_h, N, h), pos, N, L)
    assert np.max(np.abs(got2[3:] - opic.sync_velocity(vel, Ep2, 0.05))) <= 1e-12


def test_pic_loop_40_steps_32cubed(pg):
    """The small Landau case: 32^3, 8 ppc, dt = 0.05, 40 steps."""
    N, ppc, steps, dt = 32, 8, 40, 0.05
    h = L / N
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    W = []
    for n in range(steps):
        c.deposit(rho)
        c.solve(rho, phi, tol=1e-12, maxit=5000)
        W.append(c.field_energy(phi))
        c.gather_push(phi, dt)
    got, _ = c.particles()
    pos, vel, phi_o, en, _ = opic.pic_run(N, ppc, 0x5EED, steps, dt=dt, tol=1e-12)
    d = np.abs(got[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-10
    assert np.max(np.abs(got[3:] - vel)) <= 1e-10
    W = np.array(W)
    assert np.max(np.abs(W - en) / en) <= 1e-8
    assert np.linalg.norm(host(phi) - phi_o) <= 1e-9 * np.linalg.norm(phi_o)


# ------------------------------------------------------------------ full size
def test_full_size_step_properties_256cubed(pg):
    """One PIC step at 256^3 x 8 ppc (134M particles), the benchmark's launch
    configuration: charge conservation, the true FP64 residual of both solver
    precisions checked by the oracle's operator, and the field energy."""
    N, ppc = 256, 8
    h = L / N
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    rho_h = host(rho)
    assert abs(rho_h.sum()) * h ** 3 <= 1e-6 * L ** 3
    bp = rho_h - rho_h.mean()
    for prec in (0, 1):
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(rho, phi, tol=1e-10, maxit=5000, precision=prec)
        phi_h = host(phi)
        r = bp - opic.apply_A(phi_h, N, h)
        assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(bp), (prec, info)
        W = c.field_energy(phi)
        assert np.allclose(W, opic.field_energy(phi_h, N, h), rtol=1e-11)
    c.gather_push(phi, 0.05)
    c.deposit(rho)
    assert abs(host(rho).sum()) * h ** 3 <= 1e-6 * L ** 3


# ------------------------------------------------------- Landau damping on the GPU
def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return dict((r[0], float(r[1])) for r in rows)


@pytest.mark.parametrize("solver", ["fp64_judge", "mixed_mg"])
def test_landau_damping_rate_on_the_gpu_path(pg, solver):
    """Fig. 2's check on the GPU path (Sec. 2.1, 3D Landau damping): 32^3 x 8
    ppc, dt = 0.05, 190 steps (t = 9.5) through pic_deposit, the solve
    (poisson_solve, the FP64 Jacobi-PCG, or the mixed-precision multigrid
    FCG of the benchmark) and pic_gather_push. The amplitude of the three
    k = 0.5 Fourier modes of phi peaks every pi / omega_r; a log-linear fit of
    the peaks before t = 8.5 gives the damping rate, within 10 % of the
    dispersion relation's gamma = -0.1534, and the period within 10 %."""
    g = _golden("landau_linear.txt")
    N, ppc, dt, steps = 32, 8, 0.05, 190
    n = N ** 3
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    amp = []
    for _ in range(steps):
        c.deposit(rho)
        if solver == "fp64_judge":
            assert pg.poisson_solve(c.h, rho, phi, 1e-10, 5000, n) == pg.PIC_OK
        else:
            c.solve(rho, phi, tol=1e-10, maxit=200, precision=pg.PREC_MIXED, precond=pg.PC_MG)
        F = np.fft.fftn(host(phi).reshape(N, N, N))
        amp.append(abs(F[0, 0, 1]) + abs(F[0, 1, 0]) + abs(F[1, 0, 0]))
        c.gather_push(phi, dt)
    c.close()
    a = np.array(amp)
    t = np.arange(a.size) * dt
    pk = [i for i in range(1, a.size - 1) if a[i] > a[i - 1] and a[i] >= a[i + 1] and t[i] < 8.5]
    assert len(pk) >= 3
    gamma = np.polyfit(t[pk], np.log(a[pk]), 1)[0]
    assert abs(gamma - g["gamma"]) < 0.1 * abs(g["gamma"]), gamma
    period = np.mean(np.diff(t[pk]))
    assert abs(period - np.pi / g["omega_r"]) < 0.1 * np.pi / g["omega_r"], period
    print(f"\nGPU Landau damping ({solver}): gamma {gamma:.4f} (theory {g['gamma']}), "
          f"period {period:.3f} (theory {np.pi / g['omega_r']:.3f})")


def test_refine_max_caps_the_fp64_recomputations(pg):
    """pic_solve_opts.refine_max: the mixed solve stops with PIC_ENOCONV after
    that many FP64 residual recomputations (the last iterate returned, its
    true residual reported); 0 leaves it uncapped; negative is rejected."""
    N = 64
    c = solver_ctx(pg, N)
    b = dev(inputs.landau_noise_rhs(N, 2))
    phi = torch.zeros_like(b)
    free = c.solve(b, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED)
    assert free["converged"] and free["reliable_updates"] >= 3, free
    for cap in (1, 2):
        phi.zero_()
        info = c.solve(b, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, refine_max=cap,
                       raise_on_error=False)
        assert info["code"] == pg.PIC_ENOCONV and not info["converged"], info
        assert info["reliable_updates"] == cap, info
        assert 1e-10 < info["rel_res"] < 1.0, info
        assert torch.isfinite(phi).all()
    phi.zero_()
    info = c.solve(b, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, refine_max=-1, raise_on_error=False)
    assert info["code"] == pg.PIC_EINVAL
    c.close()


def test_reliable_delta_range(pg):
    """reliable_delta below 1e-4 (where the FP32 recursion runs out of
    precision before its first FP64 recomputation) and at or above 1 is
    rejected; 1e-4 converges."""
    N = 32
    c = solver_ctx(pg, N)
    b = dev(inputs.landau_noise_rhs(N, 4))
    phi = torch.zeros_like(b)
    for bad in (1e-5, 1.0, 2.0):
        info = c.solve(b, phi, tol=1e-10, maxit=2000, precision=pg.PREC_MIXED, reliable_delta=bad,
                       raise_on_error=False)
        assert info["code"] == pg.PIC_EINVAL, bad
    info = c.solve(b, phi.zero_(), tol=1e-10, maxit=2000, precision=pg.PREC_MIXED, precond=pg.PC_MG,
                   reliable_delta=1e-4)
    assert info["converged"] and info["rel_res"] <= 1e-10, info
    c.close()
