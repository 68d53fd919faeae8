"""GPU parity of the particle-in-Fourier scheme (Sec. 3.4, Appendix A)
against the CPU oracle's direct non-uniform DFT sums (oracle/pif.py): the
field at the particles, and a few leapfrog steps with it.

The GPU evaluates the sums by NUFFTs (window width from the tolerance, FP64
cuFFT); at tol = 1e-12 they match the direct sums to ~1e-12 of the field's
maximum (checked at 1e-9)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pic as opic  # noqa: E402
from oracle import pif as opif  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


@pytest.mark.parametrize("N,ppc", [(8, 1), (16, 1)])
def test_pif_field_matches_direct_sums(pg, N, ppc):
    c = pg.Context().init(N, ppc, 21)
    npart = ppc * N ** 3
    E = torch.full((3 * npart,), float("nan"), dtype=torch.float64, device="cuda")
    c.pif_field(E, tol=1e-12)
    pos, _ = opic.init_particles(N, ppc, 21)
    ref, imag = opif.field_at_particles(pos, np.full(npart, -L ** 3 / npart), N, L)
    got = E.cpu().numpy().reshape(3, -1)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(imag)) <= 1e-12 * np.max(np.abs(ref))


def test_pif_steps_match_the_oracle(pg):
    N, ppc, steps, dt = 8, 2, 5, 0.05
    npart = ppc * N ** 3
    c = pg.Context().init(N, ppc, 0x5EED)
    for _ in range(steps):
        c.pif_push(dt, tol=1e-12)
    got, half = c.particles()
    assert half
    pos, vel = opic.init_particles(N, ppc, 0x5EED)
    q = np.full(npart, -L ** 3 / npart)
    for n in range(steps):
        Ep, _ = opif.field_at_particles(pos, q, N, L)
        pos, vel = opic.push(pos, vel, Ep, dt, L, kick=(0.5 * dt if n == 0 else dt))
    d = np.abs(got[:3] - pos)
    assert np.max(np.minimum(d, L - d)) <= 1e-9
    assert np.max(np.abs(got[3:] - vel)) <= 1e-9
