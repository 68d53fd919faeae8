"""GPU parity of the particle-in-Fourier scheme (Sec. 3.4, Appendix A)
against the CPU oracle's direct non-uniform DFT sums (oracle/pif.py): the
field at the particles, and a few leapfrog steps with it.

The GPU evaluates the sums by NUFFTs (window width w = ceil(-log10 tol) + 1;
FP32 window sums and cuFFT at tol >= 1e-5, FP64 below); their error follows
the tolerance: about 1.0-1.3 tol of the
field's maximum for tol = 1e-4 (the tolerance of the paper's runs, w = 5),
1e-5, 1e-6 and 1e-12, so the bounds below are 5 tol, and 1e-9 where FP64 rounding
of the sums dominates (tol <= 1e-12; tol = 1e-15 takes the widest window,
w = 16, which spans the whole oversampled grid at N = 8)."""
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


@pytest.mark.parametrize("N,ppc,tol,bound", [(8, 1, 1e-12, 1e-9), (16, 1, 1e-12, 1e-9), (8, 1, 1e-15, 1e-9),
                                             (16, 2, 1e-4, 5e-4), (16, 2, 1e-5, 5e-5), (16, 1, 1e-6, 5e-6)])
def test_pif_field_matches_direct_sums(pg, N, ppc, tol, bound):
    c = pg.Context().init(N, ppc, 21)
    npart = ppc * N ** 3
    E = torch.full((3 * npart,), float("nan"), dtype=torch.float64, device="cuda")
    c.pif_field(E, tol=tol)
    pos, _ = opic.init_particles(N, ppc, 21)
    ref, imag = opif.field_at_particles(pos, np.full(npart, -L ** 3 / npart), N, L)
    got = E.cpu().numpy().reshape(3, -1)
    assert np.max(np.abs(got - ref)) <= bound * np.max(np.abs(ref))
    assert np.max(np.abs(imag)) <= 1e-12 * np.max(np.abs(ref))
    # a second evaluation finds the particles already in cell order (the
    # spreading's atomics add in another order: FP32 rounding at tol >= 1e-5)
    E2 = torch.full_like(E, float("nan"))
    c.pif_field(E2, tol=tol)
    rep = 1e-6 if tol >= 1e-5 else 1e-12
    assert torch.allclose(E2, E, rtol=0.0, atol=rep * float(np.max(np.abs(ref))))


def test_pif_field_at_sampled_particles_with_32cubed_modes(pg):
    """32^3 modes (a 64^3 oversampled grid: the window kernels over many
    blocks and cells), 32 768 particles: the field at 1024 sampled particles
    against the oracle's direct sums from every charge, at the paper's
    tolerance 1e-4 and at 1e-12."""
    N, ppc = 32, 1
    npart = ppc * N ** 3
    c = pg.Context().init(N, ppc, 21)
    pos, _ = opic.init_particles(N, ppc, 21)
    idx = np.random.default_rng(4).choice(npart, 1024, replace=False)
    ref, imag = opif.field_at(pos, np.full(npart, -L ** 3 / npart), N, L, pos[:, idx])
    assert np.max(np.abs(imag)) <= 1e-12 * np.max(np.abs(ref))
    for tol, bound in ((1e-4, 5e-4), (1e-12, 1e-9)):
        E = torch.full((3 * npart,), float("nan"), dtype=torch.float64, device="cuda")
        c.pif_field(E, tol=tol)
        got = E.view(3, npart)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= bound * np.max(np.abs(ref)), tol
    c.close()


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


def test_pif_rejects_bad_arguments(pg):
    # checked before any launch: a solver-only context has no particles, and
    # the tolerance and time step must be positive and finite
    c = pg.Context().init(8, 0, 0)
    with pytest.raises(pg.PicError) as e:
        c.pif_push(0.05, tol=1e-4)
    assert e.value.code == pg.PIC_ESTATE
    c = pg.Context().init(8, 1, 0)
    for tol, dt in ((0.0, 0.05), (float("nan"), 0.05), (1e-4, float("inf"))):
        with pytest.raises(pg.PicError) as e:
            c.pif_push(dt, tol=tol)
        assert e.value.code == pg.PIC_EINVAL
