"""Particle-in-Fourier (PIF) field, plain FP64 on the CPU by direct sums.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 3.4 and Appendix A: the charge of the particles is taken straight to
Fourier modes by a type-1 non-uniform discrete Fourier transform,
rho_hat(k) = sum_j q_j exp(-i k.x_j), Poisson's equation is solved mode by
mode and the field is evaluated at the particles by the type-2 transform,
E(x_j) = sum_k E_hat(k) exp(i k.x_j), over the mode set
K_N = (2 pi / L) {-N/2, ..., N/2 - 1}^3. This module writes both transforms
out as sums over every (particle, mode) pair (the definition; a NUFFT
approximates them), so it is for small N and few particles.

Readings where the paper is silent or at odds with itself:
* normalisation: the transforms as printed carry no factor; for the field of
  the charge density rho(x) = sum_j q_j delta(x - x_j) in a periodic box of
  volume L^3 the Fourier series needs 1/L^3, so
  E(x) = (1/L^3) sum_{k != 0} (-i k / |k|^2) rho_hat(k) exp(i k.x);
* sign: Eq. 2 (Laplacian phi = -rho, eps0 = 1) gives phi_hat = rho_hat / |k|^2;
  the Poisson line of Sec. 3.4 prints the opposite sign, Eq. 2 is followed;
* modes: the layer m_d = -N/2 has no partner +N/2 in K_N, so a sum over K_N
  of real data is not real off the grid nodes; the field uses the symmetric
  set |m_d| <= N/2 - 1 in every dimension (k = 0 excluded: the neutralising
  background removes it).
"""
import numpy as np


def mode_numbers(N):
    """The integer modes -N/2, ..., N/2 - 1 of K_N (N even)."""
    return np.arange(-N // 2, N // 2)


def _phases(x, m, L, sign):
    """exp(sign i 2 pi m x / L) for particles x (Np) and modes m: (Np, len(m))."""
    return np.exp(sign * 2j * np.pi * np.outer(x, m) / L)


def nudft_type1(pos, q, N, L):
    """rho_hat[mz, my, mx] = sum_j q_j exp(-i k.x_j) over K_N; pos (3, Np);
    the mode axes in the order of mode_numbers(N)."""
    m = mode_numbers(N)
    ex = _phases(pos[0], m, L, -1.0)
    ey = _phases(pos[1], m, L, -1.0)
    ez = _phases(pos[2], m, L, -1.0)
    return np.einsum("j,jc,jb,ja->abc", np.asarray(q, dtype=np.float64), ex, ey, ez)


def nudft_type2(fhat, pos, N, L):
    """f(x_j) = sum_k fhat[mz, my, mx] exp(i k.x_j) over K_N (complex)."""
    m = mode_numbers(N)
    ex = _phases(pos[0], m, L, 1.0)
    ey = _phases(pos[1], m, L, 1.0)
    ez = _phases(pos[2], m, L, 1.0)
    return np.einsum("abc,jc,jb,ja->j", fhat, ex, ey, ez)


def field_at_particles(pos, q, N, L):
    """E (3, Np) at the particles from the charges q at pos (the readings
    above): (1/L^3) sum over the symmetric nonzero modes of
    -i k / |k|^2 rho_hat(k) exp(i k.x_j); returned real (the imaginary part is
    zero to rounding over the symmetric mode set)."""
    return field_at(pos, q, N, L, pos)


def field_at(pos, q, N, L, at):
    """The field of the charges q at pos (as in field_at_particles) evaluated
    at the points `at` (3, M): type 1 over every charge, type 2 at `at` only."""
    m = mode_numbers(N)
    rho_hat = nudft_type1(pos, q, N, L)
    k = 2.0 * np.pi * m / L
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    keep = (np.abs(m) <= N // 2 - 1)
    sym = keep[:, None, None] & keep[None, :, None] & keep[None, None, :]
    sym &= k2 > 0
    inv = np.zeros_like(k2)
    inv[sym] = 1.0 / k2[sym]
    phi_hat = rho_hat * inv / L ** 3
    E = []
    for kd in (kx, ky, kz):
        E.append(nudft_type2(-1j * kd * phi_hat, at, N, L))
    E = np.stack(E)
    return E.real, E.imag
