"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (512^3 x 8 ppc, 1 073 741 824 particles, and 256^3 x 8 ppc;
particle-in-Fourier at 128^3 x 8 ppc), where the oracle cannot run the whole
problem:

* sampled particles: the oracle's CIC gather and leapfrog push of 4096
  particles, one by one, with the GPU's own potential, against the GPU push;
* sampled nodes: the oracle's CIC deposit of every particle that reaches 4096
  sampled nodes, against the GPU's rho there (the deposit after a push, as in
  the timed steps);
* properties that hold at any size: the deposit is neutral (mean zero); CIC
  deposit and gather with the central-difference field conserve the total
  momentum (the deposit is the gather's adjoint and the difference operator
  is antisymmetric and commutes with the Laplacian), up to the solve's
  residual; the particle-in-Fourier field conserves it to rounding (type 2 is
  the adjoint of type 1 and the multiplier -i k / |k|^2 is odd over the
  symmetric mode set).

The particle state stays on the device; only the samples and phi reach the
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


def sample_rows(dev6, npart, idx):
    """Columns idx of the (6, npart) device state, on the host."""
    return dev6.view(6, npart)[:, idx].cpu().numpy()


def particles_near_nodes(pos3, N, h, nodes, chunk=1 << 26):
    """Positions (host, 3 x M) of every particle whose CIC cell has one of the
    given nodes as a corner; cells are taken with one cell of margin on each
    side, so rounding of the FP64 positions cannot drop a particle."""
    n = N ** 3
    mask = torch.zeros(n, dtype=torch.bool, device="cuda")
    nz, ny, nx = nodes // (N * N), (nodes // N) % N, nodes % N
    for dz in range(-2, 2):
        for dy in range(-2, 2):
            for dx in range(-2, 2):
                mask[((nx + dx) % N) + N * (((ny + dy) % N) + N * ((nz + dz) % N))] = True
    out = []
    npart = pos3.shape[1]
    for a in range(0, npart, chunk):
        p = pos3[:, a:a + chunk]
        cell = torch.clamp(torch.floor(p / h).long(), 0, N - 1)
        key = cell[0] + N * (cell[1] + N * cell[2])
        out.append(p[:, mask[key]].cpu())
    return torch.cat(out, dim=1).numpy()


@pytest.mark.parametrize("N", [256, 512])
def test_first_steps_at_bench_size(pg, N):
    """Two steps of the bench's loop at 8 ppc (256^3: 134 M particles; 512^3:
    1.07 G particles, the full-PIC configuration): the first deposit is
    neutral; 4096 sampled particles pushed by the oracle with the GPU's own
    potential match the GPU push; the total momentum is conserved up to the
    solve's residual; and the second deposit (sorted by the keys and ranks
    the push wrote) equals the oracle's deposit at 4096 sampled nodes, from
    every particle that reaches them."""
    ppc, dt = 8, 0.05
    n, npart = N ** 3, ppc * N ** 3
    h = L / N
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    assert abs(rho.mean().item()) <= 1e-12 * rho.abs().max().item()
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = c.solve(rho, phi, tol=1e-10, maxit=200, precision=pg.PREC_MIXED, precond=pg.PC_MG)
    assert info["converged"] and info["rel_res"] <= 1e-10
    idx = torch.from_numpy(np.random.default_rng(0).choice(npart, 4096, replace=False)).cuda()
    state = torch.empty(6 * npart, dtype=torch.float64, device="cuda")
    assert not c.particles_into(state)
    b6 = sample_rows(state, npart, idx)
    v_sum0 = state.view(6, npart)[3:].sum(dim=1)
    c.gather_push(phi, dt)
    assert c.particles_into(state)
    a6 = sample_rows(state, npart, idx)
    # sampled particles against the oracle with the same potential
    E = opic.gradient(phi.cpu().numpy(), N, h)
    Ep = opic.gather(E, b6[:3], N, L)
    pos, vel = opic.push(b6[:3], b6[3:], Ep, dt, L, kick=0.5 * dt)
    d = np.abs(a6[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-11
    assert np.max(np.abs(a6[3:] - vel)) <= 1e-11
    # total momentum: the kick moves it by -(dt / 2) sum_j E(x_j), zero up to
    # the solve's residual (scale: the sample's mean |dv| times the count)
    net = (state.view(6, npart)[3:].sum(dim=1) - v_sum0).abs().cpu().numpy()
    scale = np.abs(a6[3:] - b6[3:]).mean(axis=1) * npart
    assert np.all(net <= 1e-7 * scale), (net, scale)
    # the second deposit at sampled nodes against the oracle's
    c.deposit(rho)
    nodes = torch.from_numpy(np.random.default_rng(1).choice(n, 4096, replace=False)).cuda()
    got = rho[nodes].cpu().numpy() - 1.0   # the electrons' charge density
    near = particles_near_nodes(state.view(6, npart)[:3], N, h, nodes)
    del state
    q_p = -L ** 3 / npart
    ref = opic.deposit(near, N, L, q_p=q_p) - near.shape[1] / npart  # minus the subset's own background
    assert np.max(np.abs(got - ref[nodes.cpu().numpy()])) <= 1e-12
    c.close()
    del rho, phi
    torch.cuda.empty_cache()  # give the cached blocks back before the next full-size test


@pytest.mark.parametrize("tol,bound", [(1e-4, 1e-6), (1e-6, 1e-10)])
def test_particle_in_fourier_field_conserves_momentum_at_bench_size(pg, tol, bound):
    """The bench's tolerance 1e-4 runs the FP32 NUFFTs, whose rounding bounds
    the conservation at ~1e-7 relative; 1e-6 runs them in FP64."""
    N, ppc = 128, 8
    npart = ppc * N ** 3
    c = pg.Context().init(N, ppc, 0x5EED)
    E = torch.empty(3 * npart, dtype=torch.float64, device="cuda")
    c.pif_field(E, tol=tol)
    E3 = E.view(3, npart)
    assert bool(torch.isfinite(E3).all())
    net = E3.sum(dim=1).abs()
    scale = E3.abs().sum(dim=1)
    assert bool(torch.all(scale > 0))
    assert bool(torch.all(net <= bound * scale)), (net.tolist(), scale.tolist())
