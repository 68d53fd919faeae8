"""Pins of the oracle's red-black SSOR preconditioner (oracle/ssor.py, the
paper's PCG configuration of Sec. 4.1): the textbook matrix form of SOR with
the red-black ordering, exactness of a half-sweep, symmetry and positivity,
and the flexible-CG solve it preconditions."""
import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import pic
from oracle import ssor
from paper_2605_05469_gb300 import inputs

L = 4.0 * np.pi


def scaled_matrix(N):
    """h^2 A = 6 I - (sum of the 6 periodic neighbours) as a dense matrix."""
    h = L / N
    n = N ** 3
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = h * h * pic.apply_A(e, N, h)
    return A


def test_half_sweep_solves_its_colour_exactly():
    """With omega = 1 a red half-sweep leaves the red rows of (h^2 A) x = h^2 r satisfied."""
    N = 8
    h = L / N
    rng = np.random.default_rng(0)
    x = rng.normal(size=N ** 3)
    r = rng.normal(size=N ** 3)
    red = ssor.red_mask(N)
    y = ssor.half_sweep(x, h * h * r, N, 1.0, red)
    res = h * h * r - h * h * pic.apply_A(y, N, h)
    assert np.max(np.abs(res[red])) <= 1e-12 * np.max(np.abs(h * h * r))
    assert np.array_equal(y[~red], x[~red])


@pytest.mark.parametrize("omega,inner,outer", [(1.0, 1, 1), (np.pi / 2, 2, 2), (1.3, 4, 2)])
def test_matches_textbook_matrix_form(omega, inner, outer):
    """SOR in matrix form (Saad sec. 4.1) with the nodes ordered red first:
    forward  (D/w + L) x' = b - (U + (1 - 1/w) D) x,
    backward (D/w + U) x' = b - (L + (1 - 1/w) D) x,
    L and U the strictly lower and upper parts of h^2 A in that order."""
    N = 4
    h = L / N
    A = scaled_matrix(N)
    red = ssor.red_mask(N)
    perm = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    Lo = np.tril(Ap, -1)
    Up = np.triu(Ap, 1)
    r = np.random.default_rng(1).normal(size=N ** 3)
    b = (h * h * r)[perm]
    x = np.zeros_like(b)
    for _ in range(outer):
        for _ in range(inner):
            x = np.linalg.solve(D / omega + Lo, b - (Up + (1 - 1 / omega) * D) @ x)
        for _ in range(inner):
            x = np.linalg.solve(D / omega + Up, b - (Lo + (1 - 1 / omega) * D) @ x)
    ref = np.empty_like(x)
    ref[perm] = x
    got = ssor.ssor(r, N, h, omega, inner, outer)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_paper_configuration_is_symmetric_and_positive():
    N = 8
    h = L / N
    rng = np.random.default_rng(2)
    a = rng.normal(size=N ** 3)
    b = rng.normal(size=N ** 3)
    a -= a.mean()
    b -= b.mean()
    Ma = ssor.ssor(a, N, h)
    Mb = ssor.ssor(b, N, h)
    assert abs(Ma @ b - a @ Mb) <= 1e-12 * np.linalg.norm(Ma) * np.linalg.norm(b)
    assert Ma @ a > 0.0 and Mb @ b > 0.0


def test_preconditioned_cg_reaches_the_exact_solution():
    its = {}
    for N in (16, 32):
        h = L / N
        b = inputs.landau_noise_rhs(N, 9)
        x, it, rel, ok = ocnn.fcg(b, np.zeros(N ** 3), N, h, 1e-10, 500, lambda r: ssor.ssor(r, N, h))
        ref = pic.spectral_solve_fft(b, N, h)
        assert ok and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
        _, it_j, _, _ = pic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-10, 5000)
        its[N] = (it, it_j)
        assert it < it_j / 2, its
