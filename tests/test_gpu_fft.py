"""GPU parity of the FFT pseudo-spectral solve (Sec. 3.1) and of the FFT-PIC
step (spectral E pushed to the particles) against the CPU oracle
(oracle/fft.py with oracle/pic.py's particle kernels).

The GPU transforms are FP64 (cuFFT); phi and E agree with numpy's FP64 FFT to
rounding (1e-12 of the field's maximum)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fft as offt  # noqa: E402
from oracle import pic as opic  # noqa: E402
from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def host(t):
    return t.detach().cpu().numpy()


def max_rel(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("N", [8, 16, 24, 64])
def test_spectral_solve_matches_oracle(pg, N):
    rho = np.random.default_rng(N).normal(size=N ** 3) + 1.0
    c = pg.Context().init(N, 0, 0)
    rt = torch.from_numpy(rho).cuda()
    phi = torch.full((N ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    E = torch.full((3 * N ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    c.fft_solve(rt, phi, E)
    ref_phi, ref_E = offt.spectral_solve(rho, N, L)
    assert max_rel(host(phi), ref_phi) <= 1e-12
    assert max_rel(host(E).reshape(3, -1), ref_E) <= 1e-12
    assert np.array_equal(host(rt), rho), "rho must not be modified"
    # phi alone
    phi2 = torch.zeros_like(phi)
    c.fft_solve(rt, phi2)
    assert np.array_equal(host(phi2), host(phi))


def test_spectral_solve_256cubed(pg):
    """The full-size grid of the PIC benchmark, against numpy's FFT."""
    N = 256
    b = inputs.landau_noise_rhs(N, 5)
    c = pg.Context().init(N, 0, 0)
    phi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    E = torch.empty(3 * N ** 3, dtype=torch.float64, device="cuda")
    c.fft_solve(torch.from_numpy(b).cuda(), phi, E)
    ref_phi, ref_E = offt.spectral_solve(b, N, L)
    assert max_rel(host(phi), ref_phi) <= 1e-12
    assert max_rel(host(E).reshape(3, -1), ref_E) <= 1e-12


def test_push_and_energy_with_the_spectral_field(pg):
    N, ppc = 16, 8
    h = L / N
    c = pg.Context().init(N, ppc, 7)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    phi = torch.empty_like(rho)
    E = torch.empty(3 * N ** 3, dtype=torch.float64, device="cuda")
    c.fft_solve(rho, phi, E)
    Eh = host(E).reshape(3, -1)
    W = c.field_energy_E(E)
    assert np.allclose(W, h ** 3 * np.sum(Eh ** 2, axis=1), rtol=1e-12, atol=0)
    c.gather_push_field(E, 0.05)
    got, half = c.particles()
    assert half
    pos, vel = opic.init_particles(N, ppc, 7)
    Ep = opic.gather(Eh, pos, N, L)
    pos, vel = opic.push(pos, vel, Ep, 0.05, L, kick=0.025)
    d = np.abs(got[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-12
    assert np.max(np.abs(got[3:] - vel)) <= 1e-12
    c.sync_velocity_field(E, 0.05)
    got2, half2 = c.particles()
    assert not half2
    assert np.max(np.abs(got2[3:] - opic.sync_velocity(vel, opic.gather(Eh, pos, N, L), 0.05))) <= 1e-12


def test_fft_pic_loop_20_steps_32cubed(pg):
    """The FFT-PIC scheme (deposit, spectral phi and E, push with the spectral
    field) for 20 steps against the same loop in the oracle."""
    N, ppc, steps, dt = 32, 8, 20, 0.05
    h = L / N
    c = pg.Context().init(N, ppc, 0x5EED)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    phi = torch.empty_like(rho)
    E = torch.empty(3 * N ** 3, dtype=torch.float64, device="cuda")
    W = []
    for n in range(steps):
        c.deposit(rho)
        c.fft_solve(rho, phi, E)
        W.append(c.field_energy_E(E))
        c.gather_push_field(E, dt)
    got, _ = c.particles()
    pos, vel = opic.init_particles(N, ppc, 0x5EED)
    Wo = []
    for n in range(steps):
        r = opic.deposit(pos, N, L)
        _, Eo = offt.spectral_solve(r, N, L)
        Wo.append(h ** 3 * np.sum(Eo ** 2, axis=1))
        pos, vel = opic.push(pos, vel, opic.gather(Eo, pos, N, L), dt, L, kick=(0.5 * dt if n == 0 else dt))
    d = np.abs(got[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-10
    assert np.max(np.abs(got[3:] - vel)) <= 1e-10
    assert np.max(np.abs(np.array(W) - np.array(Wo)) / np.array(Wo)) <= 1e-8
