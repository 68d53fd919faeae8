"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (256^3 x 8 ppc, 134 217 728 particles, multigrid-preconditioned mixed
solve; particle-in-Fourier at 128^3 x 8 ppc), where the oracle cannot run the
whole problem:

* sampled particles: the oracle's CIC gather and leapfrog push of 4096
  particles, one by one, with the GPU's own potential, against the GPU push;
* properties that hold at any size: the deposit is neutral (mean zero); CIC
  deposit and gather with the central-difference field conserve the total
  momentum (the deposit is the gather's adjoint and the difference operator
  is antisymmetric and commutes with the Laplacian), up to the solve's
  residual; the particle-in-Fourier field conserves it to rounding (type 2 is
  the adjoint of type 1 and the multiplier -i k / |k|^2 is odd over the
  symmetric mode set).

The particle state stays on the device; only the sample and phi reach the
host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pic as opic  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def test_first_step_at_bench_size(pg):
    N, ppc, dt = 256, 8, 0.05
    n, npart = N ** 3, ppc * N ** 3
    h = L / N
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    assert abs(rho.mean().item()) <= 1e-12 * rho.abs().max().item()
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = c.solve(rho, phi, tol=1e-10, maxit=200, precision=pg.PREC_MIXED, precond=pg.PC_MG)
    assert info["converged"] and info["rel_res"] <= 1e-10
    before = torch.empty(6 * npart, dtype=torch.float64, device="cuda")
    assert not c.particles_into(before)
    c.gather_push(phi, dt)
    after = torch.empty_like(before)
    assert c.particles_into(after)
    # sampled particles against the oracle with the same potential
    idx = torch.from_numpy(np.random.default_rng(0).choice(npart, 4096, replace=False)).cuda()
    b6 = before.view(6, npart)[:, idx].cpu().numpy()
    a6 = after.view(6, npart)[:, idx].cpu().numpy()
    E = opic.gradient(phi.cpu().numpy(), N, h)
    Ep = opic.gather(E, b6[:3], N, L)
    pos, vel = opic.push(b6[:3], b6[3:], Ep, dt, L, kick=0.5 * dt)
    d = np.abs(a6[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-11
    assert np.max(np.abs(a6[3:] - vel)) <= 1e-11
    # total momentum: the kick moves it by -(dt / 2) sum_j E(x_j), zero up to the solve's residual
    dv = after.view(6, npart)[3:] - before.view(6, npart)[3:]
    net = dv.sum(dim=1).abs()
    scale = dv.abs().sum(dim=1)
    assert bool(torch.all(net <= 1e-7 * scale)), (net.tolist(), scale.tolist())


def test_particle_in_fourier_field_conserves_momentum_at_bench_size(pg):
    N, ppc = 128, 8
    npart = ppc * N ** 3
    c = pg.Context().init(N, ppc, 0x5EED)
    E = torch.empty(3 * npart, dtype=torch.float64, device="cuda")
    c.pif_field(E, tol=1e-4)
    E3 = E.view(3, npart)
    assert bool(torch.isfinite(E3).all())
    net = E3.sum(dim=1).abs()
    scale = E3.abs().sum(dim=1)
    assert bool(torch.all(scale > 0))
    assert bool(torch.all(net <= 1e-10 * scale)), (net.tolist(), scale.tolist())
