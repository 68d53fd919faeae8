"""FFT pseudo-spectral periodic Poisson solve, plain FP64 on the CPU.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 3.1: with periodic boundaries, -Laplacian phi = rho (eps0 = 1, Eq. 2)
becomes k^2 phi_hat = rho_hat in Fourier space, so

    phi = F^-1( rho_hat / k^2 ),   E = -grad phi = F^-1( -i k rho_hat / k^2 ),

with the wave-vector k = 2 pi m / L of the integer mode m (numpy's FFT
order: m = 0, 1, ..., N/2 - 1, -N/2, ..., -1). Readings where the paper is
silent: the k = 0 mode of phi and E is zero (mean-zero potential; the
neutralising background removes the mean of rho); for even N the Nyquist
mode m_d = -N/2 of the derivative along d is zero in E_d (its multiplier
-i k_d has no partner of opposite sign on the grid, so a real field has no
consistent derivative there); phi keeps its Nyquist modes.
"""
import numpy as np


def mode_numbers(N):
    """Integer mode numbers m of an N-point FFT, in numpy's order."""
    return np.fft.fftfreq(N, d=1.0 / N)


def wave_vectors(N, L):
    """k_z, k_y, k_x broadcastable over an (N, N, N) array (x fastest)."""
    k = 2.0 * np.pi * mode_numbers(N) / L
    return k[:, None, None], k[None, :, None], k[None, None, :]


def spectral_solve(rho, N, L):
    """phi and E = (E_x, E_y, E_z) of the pseudo-spectral solve on an N^3
    node grid of a periodic box of side L; rho flat, x fastest."""
    r = np.asarray(rho, dtype=np.float64).reshape(N, N, N)
    rh = np.fft.fftn(r)
    kz, ky, kx = wave_vectors(N, L)
    k2 = kx * kx + ky * ky + kz * kz
    inv = np.zeros_like(k2)
    np.divide(1.0, k2, out=inv, where=k2 > 0)
    ph = rh * inv
    phi = np.real(np.fft.ifftn(ph)).reshape(-1)
    m = mode_numbers(N)
    nyq = (m == -N / 2) if N % 2 == 0 else np.zeros(N, dtype=bool)
    E = []
    for axis, kd in ((2, kx), (1, ky), (0, kz)):   # x, y, z
        kk = kd.copy()
        shape = [1, 1, 1]
        shape[axis] = N
        kk = np.where(nyq.reshape(shape), 0.0, kk)
        E.append(np.real(np.fft.ifftn(-1j * kk * ph)).reshape(-1))
    return phi, np.stack(E)


def dft_solve_bruteforce(rho, N, L):
    """The same solve with the Fourier transforms written out as sums over
    every node and mode (tiny N only): an independent check of the FFT
    form's conventions (mode order, signs, normalisation)."""
    r = np.asarray(rho, dtype=np.float64).reshape(N, N, N)
    idx = np.arange(N)
    m = mode_numbers(N)
    W = np.exp(-2j * np.pi * np.outer(m, idx) / N)        # W[m, i] = exp(-2 pi i m i / N)
    rh = np.einsum("ai,bj,ck,kji->cba", W, W, W, r)        # rh[mz, my, mx]
    k = 2.0 * np.pi * m / L
    phi = np.zeros((N, N, N))
    E = np.zeros((3, N, N, N))
    nyq = m == -N / 2
    for a in range(N):          # mode index along z
        for b in range(N):      # y
            for c in range(N):  # x
                k2 = k[a] ** 2 + k[b] ** 2 + k[c] ** 2
                if k2 == 0.0:
                    continue
                ph = rh[a, b, c] / k2
                # e^{+i k.x} at every node (z, y, x)
                wave = np.exp(2j * np.pi * (m[a] * idx[:, None, None] + m[b] * idx[None, :, None]
                                            + m[c] * idx[None, None, :]) / N) / N ** 3
                phi += np.real(ph * wave)
                for d, (kd, isn) in enumerate(((k[c], nyq[c]), (k[b], nyq[b]), (k[a], nyq[a]))):
                    if not isn:
                        E[d] += np.real(-1j * kd * ph * wave)
    return phi.reshape(-1), E.reshape(3, -1)
