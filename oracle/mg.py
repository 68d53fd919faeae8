"""Geometric multigrid V-cycle as a preconditioner, plain FP64 on the CPU.

Test infrastructure only (see ``oracle/__init__.py``).

The paper's conclusion (Sec. 5) sets its PCG solver beside the multigrid
solvers of a cited comparison and names better preconditioning as future
work (Secs. 4.3, 5); it prints no multigrid algorithm. This module defines the V-cycle the GPU library
offers, from the textbook geometric multigrid for the periodic 7-point
Laplacian (Trottenberg, Oosterlee & Schueller, "Multigrid", 2001, ch. 2-4):

* levels l = 0, 1, ...: N_l = N / 2^l nodes per dimension, h_l = 2^l h, the
  same operator A_l = (6 I - sum of the 6 periodic neighbours) / h_l^2;
* restriction R: full weighting, coarse node I takes fine node 2I and its
  26 neighbours with weights prod_d w(o_d), w(0) = 1/2, w(+-1) = 1/4;
* prolongation P: trilinear interpolation, fine node 2I + o (o_d in {0, 1})
  is the mean of the coarse nodes I + s, s_d in {0, o_d}; R = P^T / 8;
* smoother: damped Jacobi x <- x + omega h_l^2/6 (r - A_l x), omega = 6/7
  (the smoothing-optimal damping of the 3-D 7-point Laplacian), nu1 sweeps
  before and nu2 after the coarse-grid correction, starting from x = 0; on
  the finest level the learned preconditioner may replace it,
  x <- x + S(r - A_0 x) with S symmetric;
* coarsest level (N_l <= coarsest, or N_l odd): ``coarse_sweeps`` damped
  Jacobi sweeps from x = 0.

With the same smoother before and after (nu1 = nu2) and a fixed number of
coarsest sweeps the cycle is a fixed linear operator, symmetric in the
Euclidean inner product; with convergent smoothers it is positive definite on
the mean-zero subspace, so it serves as the preconditioner of (flexible) CG.
"""
import numpy as np

from . import pic

OMEGA = 6.0 / 7.0


def _roll3(g, sz, sy, sx):
    return np.roll(np.roll(np.roll(g, sz, axis=0), sy, axis=1), sx, axis=2)


def restrict_fw(f, N):
    """Full weighting of the N^3 field f onto the (N/2)^3 grid (periodic)."""
    g = f.reshape(N, N, N)
    w1 = {-1: 0.25, 0: 0.5, 1: 0.25}
    acc = np.zeros_like(g)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                # value at fine node i + o, placed at i
                acc += w1[oz] * w1[oy] * w1[ox] * _roll3(g, -oz, -oy, -ox)
    return acc[::2, ::2, ::2].reshape(-1).copy()


def prolong_trilinear(c, Nc):
    """Trilinear interpolation of the Nc^3 field c onto the (2 Nc)^3 grid."""
    g = c.reshape(Nc, Nc, Nc)
    N = 2 * Nc
    out = np.empty((N, N, N))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                acc = np.zeros_like(g)
                cnt = 0
                for sz in range(oz + 1):
                    for sy in range(oy + 1):
                        for sx in range(ox + 1):
                            acc += _roll3(g, -sz, -sy, -sx)
                            cnt += 1
                out[oz::2, oy::2, ox::2] = acc / cnt
    return out.reshape(-1)


def jacobi_sweeps(x, r, N, h, k, omega=OMEGA):
    """k damped Jacobi sweeps on A x = r."""
    for _ in range(k):
        x = x + (omega * h * h / 6.0) * (r - pic.apply_A(x, N, h))
    return x


def vcycle(r, N, h, nu1=2, nu2=2, coarsest=4, coarse_sweeps=40, smoother=None, level=0):
    """z = V(r) on level `level` of the hierarchy (grid N^3, spacing h).

    ``smoother`` (finest level only): a symmetric map res -> correction used
    once before and once after the coarse-grid correction instead of the
    Jacobi sweeps.
    """
    if N <= coarsest or N % 2:
        return jacobi_sweeps(np.zeros_like(r), r, N, h, coarse_sweeps)
    fine_s = smoother if level == 0 else None
    if fine_s is not None:
        x = fine_s(r)
    else:
        x = jacobi_sweeps(np.zeros_like(r), r, N, h, nu1)
    res = r - pic.apply_A(x, N, h)
    ec = vcycle(restrict_fw(res, N), N // 2, 2.0 * h, nu1, nu2, coarsest, coarse_sweeps, None, level + 1)
    x = x + prolong_trilinear(ec, N // 2)
    if fine_s is not None:
        x = x + fine_s(r - pic.apply_A(x, N, h))
    else:
        x = jacobi_sweeps(x, r, N, h, nu2)
    return x
