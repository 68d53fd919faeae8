"""Pins of the oracle's multigrid V-cycle (oracle/mg.py) against closed forms
and invariants: the transfer operators' adjointness and action on constants
and Fourier modes, the Jacobi sweep's eigen-factor, symmetry and positivity
of the cycle, and grid-independent flexible-CG iteration counts."""
import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import mg
from oracle import pic
from paper_2605_05469_gb300 import inputs

L = 4.0 * np.pi


def test_restriction_is_prolongation_transpose_over_8():
    rng = np.random.default_rng(0)
    N = 8
    f = rng.normal(size=N ** 3)
    c = rng.normal(size=(N // 2) ** 3)
    lhs = mg.restrict_fw(f, N) @ c
    rhs = f @ mg.prolong_trilinear(c, N // 2) / 8.0
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


def test_transfers_keep_constants_and_prolongation_is_exact_on_coarse_nodes():
    N = 8
    assert np.allclose(mg.restrict_fw(np.full(N ** 3, 2.5), N), 2.5, rtol=0, atol=1e-14)
    assert np.allclose(mg.prolong_trilinear(np.full((N // 2) ** 3, -1.25), N // 2), -1.25, rtol=0, atol=1e-14)
    c = np.random.default_rng(1).normal(size=(N // 2) ** 3)
    fine = mg.prolong_trilinear(c, N // 2).reshape(N, N, N)
    assert np.array_equal(fine[::2, ::2, ::2].reshape(-1), c)
    # a fine node between two coarse nodes in x is their mean
    g = c.reshape(N // 2, N // 2, N // 2)
    assert np.allclose(fine[2, 4, 3], 0.5 * (g[1, 2, 1] + g[1, 2, 2]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", [1, 3, 6])
def test_restriction_of_a_fourier_mode(m):
    """Full weighting of cos(theta i) (theta = 2 pi m / N, along x) is
    cos^2(theta / 2) cos(theta 2 I) on the coarse nodes."""
    N = 16
    i = np.arange(N ** 3)
    x = i % N
    theta = 2 * np.pi * m / N
    f = np.cos(theta * x)
    got = mg.restrict_fw(f, N)
    I = np.arange((N // 2) ** 3) % (N // 2)
    ref = np.cos(theta / 2) ** 2 * np.cos(theta * 2 * I)
    assert np.allclose(got, ref, rtol=0, atol=1e-14)


def test_jacobi_sweep_damps_the_checkerboard_by_its_eigen_factor():
    """A on the checkerboard (-1)^(i+j+k) is 12/h^2, so one damped sweep on
    A x = 0 multiplies it by 1 - 2 omega = -5/7."""
    N = 8
    h = L / N
    i = np.arange(N ** 3)
    cb = (-1.0) ** ((i % N) + (i // N) % N + i // (N * N))
    got = mg.jacobi_sweeps(cb, np.zeros_like(cb), N, h, 1)
    assert np.allclose(got, (1 - 2 * mg.OMEGA) * cb, rtol=0, atol=1e-13)


def _network_smoother(N, h, ws):
    def s(res):
        y, _ = ocnn.forward(res.reshape(N, N, N), ws)
        return h * h * y.reshape(-1)
    return s


def _damped_jacobi_network(noise, seed):
    """Tied weights with N = omega/6 (channel 0 of G carries sqrt(omega/6) x
    through the centre taps), plus small seeded noise on the free layers."""
    rng = np.random.default_rng(seed)
    w1 = noise * rng.normal(size=(16, 1, 3, 3, 3))
    w2 = noise * rng.normal(size=(16, 16, 3, 3, 3))
    w1[0, 0, 1, 1, 1] += np.sqrt(mg.OMEGA / 6.0)
    w2[0, 0, 1, 1, 1] += 1.0
    return ocnn.tie(w1, w2)


@pytest.mark.parametrize("smoother", ["jacobi", "random_network", "damped_jacobi_network"])
def test_vcycle_is_symmetric_and_positive_definite(smoother):
    """Symmetric for any symmetric fine-level smoother (random tied network
    weights included); positive definite when the smoother converges (Jacobi,
    or a network near damped Jacobi)."""
    N = 16
    h = L / N
    rng = np.random.default_rng(2)
    a = rng.normal(size=N ** 3)
    b = rng.normal(size=N ** 3)
    a -= a.mean()
    b -= b.mean()
    sm = {"jacobi": None, "random_network": _network_smoother(N, h, ocnn.init_weights(3)),
          "damped_jacobi_network": _network_smoother(N, h, _damped_jacobi_network(1e-3, 4))}[smoother]
    Va = mg.vcycle(a, N, h, smoother=sm)
    Vb = mg.vcycle(b, N, h, smoother=sm)
    assert abs(Va @ b - a @ Vb) <= 1e-12 * np.linalg.norm(Va) * np.linalg.norm(b)
    if smoother != "random_network":
        assert Va @ a > 0.0 and Vb @ b > 0.0


def test_vcycle_inverts_a_smooth_mode_nearly():
    """On the lowest Fourier mode one cycle applied to A u returns u up to the
    cycle's contraction (0.13 here: the coarse-grid corrections are exact for
    the mode, the trilinear interpolation on the coarser grids, where it is no
    longer smooth, is not); a mis-scaled transfer or coarse right-hand side
    would be off by factors."""
    N = 32
    h = L / N
    i = np.arange(N ** 3)
    u = np.cos(2 * np.pi * (i % N) / N)
    got = mg.vcycle(pic.apply_A(u, N, h), N, h)
    assert np.linalg.norm(got - u) <= 0.2 * np.linalg.norm(u)


def test_vcycle_fcg_iterations_do_not_grow_with_the_grid():
    its = {}
    for N in (16, 32, 64):
        h = L / N
        b = inputs.landau_noise_rhs(N, 5)
        x, it, rel, ok = ocnn.fcg(b, np.zeros(N ** 3), N, h, 1e-10, 200, lambda r: mg.vcycle(r, N, h))
        ref = pic.spectral_solve_fft(b, N, h)
        assert ok and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
        its[N] = it
    assert max(its.values()) <= 20, its
    assert its[64] <= its[16] + 4, its


@pytest.mark.parametrize("nu", [1, 3, 4])
def test_vcycle_with_nu_sweeps_is_symmetric_and_positive_definite(nu):
    """Equal numbers of damped-Jacobi sweeps before and after the coarse
    correction keep the cycle symmetric and positive definite for any count."""
    N = 16
    h = L / N
    rng = np.random.default_rng(nu)
    a = rng.normal(size=N ** 3)
    b = rng.normal(size=N ** 3)
    a -= a.mean()
    b -= b.mean()
    Va = mg.vcycle(a, N, h, nu, nu)
    Vb = mg.vcycle(b, N, h, nu, nu)
    assert abs(Va @ b - a @ Vb) <= 1e-12 * np.linalg.norm(Va) * np.linalg.norm(b)
    assert Va @ a > 0.0 and Vb @ b > 0.0


def test_more_smoothing_takes_fewer_fcg_iterations():
    """More sweeps per cycle make a stronger preconditioner: the FCG iteration
    count does not grow with nu (13, 9, 8, 7 for nu = 1..4 at 32^3), and every
    solve reaches the exact discrete solution."""
    N = 32
    h = L / N
    b = inputs.landau_noise_rhs(N, 1)
    ref = pic.spectral_solve_fft(b, N, h)
    its = []
    for nu in (1, 2, 3, 4):
        x, it, rel, ok = ocnn.fcg(b, np.zeros(N ** 3), N, h, 1e-10, 200, lambda r: mg.vcycle(r, N, h, nu, nu))
        assert ok and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
        its.append(it)
    assert all(its[k + 1] <= its[k] for k in range(3)), its
    assert its[3] < its[1], its
