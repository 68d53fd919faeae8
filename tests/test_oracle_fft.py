"""Pins of the oracle's FFT pseudo-spectral solve (oracle/fft.py, Sec. 3.1)
against closed forms: single Fourier modes, constants, the Nyquist reading,
a written-out DFT on tiny grids, and the exact ratio to the finite-difference
solution of one mode."""
import numpy as np
import pytest

from oracle import fft
from oracle import pic

L = 4.0 * np.pi


def grid(N):
    h = L / N
    i = np.arange(N) * h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (1, -3, 2), (3, 1, -1)])
def test_single_mode_closed_form(m):
    """rho = cos(k.x): phi = rho / |k|^2 and E = -grad phi = (k / |k|^2) sin(k.x)."""
    N = 16
    x, y, z = grid(N)
    k = 2.0 * np.pi * np.array(m, dtype=float) / L
    arg = k[0] * x + k[1] * y + k[2] * z
    k2 = float(k @ k)
    phi, E = fft.spectral_solve(np.cos(arg), N, L)
    assert np.allclose(phi, np.cos(arg) / k2, rtol=0, atol=1e-13)
    for d in range(3):
        assert np.allclose(E[d], k[d] / k2 * np.sin(arg), rtol=0, atol=1e-13)


def test_constant_density_has_no_field():
    phi, E = fft.spectral_solve(np.full(8 ** 3, 3.5), 8, L)
    assert np.max(np.abs(phi)) <= 1e-14 and np.max(np.abs(E)) <= 1e-14


def test_nyquist_mode_has_potential_but_no_field():
    """The checkerboard along x (m_x = N/2) keeps phi = rho / k_N^2; its x
    derivative is zero by the reading, its y and z derivatives are zero."""
    N = 8
    i = np.arange(N ** 3) % N
    rho = np.cos(np.pi * i)
    kN = 2.0 * np.pi * (N / 2) / L
    phi, E = fft.spectral_solve(rho, N, L)
    assert np.allclose(phi, rho / kN ** 2, rtol=0, atol=1e-14)
    assert np.max(np.abs(E)) <= 1e-14


@pytest.mark.parametrize("N", [4, 6])
def test_fft_form_matches_written_out_dft(N):
    rho = np.random.default_rng(N).normal(size=N ** 3)
    phi, E = fft.spectral_solve(rho, N, L)
    phi_b, E_b = fft.dft_solve_bruteforce(rho, N, L)
    assert np.allclose(phi, phi_b, rtol=0, atol=1e-12)
    assert np.allclose(E, E_b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m", [(1, 0, 0), (2, 3, 1)])
def test_ratio_to_finite_difference_solution(m):
    """For one mode the second-order finite-difference solution is the
    spectral one times k^2 / lambda with lambda = (4/h^2) sum_d sin^2(pi m_d / N)."""
    N = 16
    h = L / N
    x, y, z = grid(N)
    md = np.array(m, dtype=float)
    k = 2.0 * np.pi * md / L
    rho = np.cos(k[0] * x + k[1] * y + k[2] * z)
    lam = (4.0 / h ** 2) * np.sum(np.sin(np.pi * md / N) ** 2)
    phi, _ = fft.spectral_solve(rho, N, L)
    fd = pic.spectral_solve_fft(rho, N, h)
    assert np.allclose(fd, phi * (k @ k) / lam, rtol=0, atol=1e-13)
