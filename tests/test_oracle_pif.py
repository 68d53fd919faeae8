"""Pins of the oracle's particle-in-Fourier field (oracle/pif.py; Sec. 3.4,
Appendix A): the type-1 sum against numpy's FFT for particles on the grid
nodes, adjointness of the two transforms, the field of band-limited node
charges against the FFT pseudo-spectral oracle, a vanishing self-force and
the pairwise action-reaction symmetry (momentum conservation)."""
import numpy as np
import pytest

from oracle import fft as offt
from oracle import pif

L = 4.0 * np.pi


def node_positions(N):
    h = L / N
    i = np.arange(N) * h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)])


@pytest.mark.parametrize("N", [4, 6])
def test_type1_on_grid_nodes_is_the_fft(N):
    rho = np.random.default_rng(N).normal(size=N ** 3)
    got = pif.nudft_type1(node_positions(N), rho, N, L)
    F = np.fft.fftn(rho.reshape(N, N, N))          # F[mz, my, mx], FFT order
    m = pif.mode_numbers(N) % N
    ref = F[np.ix_(m, m, m)]
    assert np.allclose(got, ref, rtol=0, atol=1e-11)


def test_type2_is_the_adjoint_of_type1():
    N = 6
    rng = np.random.default_rng(1)
    pos = rng.random((3, 17)) * L
    q = rng.normal(size=17)
    g = rng.normal(size=(N, N, N)) + 1j * rng.normal(size=(N, N, N))
    lhs = np.vdot(pif.nudft_type1(pos, q, N, L), g)          # sum conj(type1) g
    rhs = np.vdot(q, pif.nudft_type2(g, pos, N, L))          # sum q type2(g)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_field_of_node_charges_matches_the_spectral_solve():
    """Charges rho_n h^3 on the nodes of a band-limited density give, at the
    nodes, the FFT pseudo-spectral field of rho (no Nyquist content, so the
    two mode readings agree)."""
    N = 8
    h = L / N
    x = node_positions(N)
    k1, k2 = 2 * np.pi / L, 4 * np.pi / L
    rho = 0.3 * np.cos(k1 * x[0]) + 0.2 * np.sin(k2 * x[1] + k1 * x[2]) + 0.1 * np.cos(k1 * (x[0] - x[1]))
    E, Eim = pif.field_at_particles(x, rho * h ** 3, N, L)
    _, ref = offt.spectral_solve(rho, N, L)
    assert np.allclose(E, ref, rtol=0, atol=1e-13)
    assert np.max(np.abs(Eim)) <= 1e-13


def test_no_self_force_and_action_reaction():
    N = 8
    rng = np.random.default_rng(2)
    p = rng.random((3, 2)) * L
    E1, _ = pif.field_at_particles(p[:, :1], np.array([1.0]), N, L)
    assert np.max(np.abs(E1)) <= 1e-14
    # field at particle a from a unit charge at b, and the reverse
    Eab, _ = pif.field_at_particles(p, np.array([0.0, 1.0]), N, L)
    Eba, _ = pif.field_at_particles(p, np.array([1.0, 0.0]), N, L)
    assert np.allclose(Eab[:, 0], -Eba[:, 1], rtol=0, atol=1e-14)
    assert np.max(np.abs(Eab[:, 0])) > 1e-3   # a real interaction, not zero
