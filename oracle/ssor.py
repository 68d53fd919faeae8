"""Red-black SSOR preconditioner, plain FP64 on the CPU.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 4.1 configures the paper's PCG with SSOR: 4 inner and 2 outer
iterations, damping pi/2. The paper does not define the two kinds of
iteration further; this module fixes the reading the GPU library
implements (textbook SOR, e.g. Saad, "Iterative Methods for Sparse Linear
Systems", 2nd ed., sec. 4.1, with the red-black ordering of sec. 12.4):

* nodes are red when i + j + k is even, black otherwise (N even, so every
  7-point neighbour of a red node is black and vice versa);
* a forward SOR sweep with damping omega updates every red node, then every
  black node: x_i <- (1 - omega) x_i + omega (r_i + sum of the 6 neighbours) / 6
  in the scaled units of (h^2 A) x = h^2 r (the diagonal of h^2 A is 6);
  with this ordering each half-sweep solves its triangular part exactly;
* a backward sweep updates black, then red;
* the preconditioner z = M(r) starts from x = 0 and repeats ``outer`` times:
  ``inner`` forward sweeps, then ``inner`` backward sweeps.

Each block of backward sweeps is the adjoint of the forward block before it,
so M is symmetric; for 0 < omega < 2 it is positive definite on the
mean-zero space and serves as the preconditioner of (flexible) CG.
"""
import numpy as np

OMEGA = np.pi / 2
INNER = 4
OUTER = 2


def red_mask(N):
    i = np.arange(N)
    return ((i[:, None, None] + i[None, :, None] + i[None, None, :]) % 2 == 0).reshape(-1)


def _neighbour_sum(x, N):
    g = x.reshape(N, N, N)
    s = np.zeros_like(g)
    for axis in range(3):
        s += np.roll(g, 1, axis=axis) + np.roll(g, -1, axis=axis)
    return s.reshape(-1)


def half_sweep(x, rh, N, omega, colour_mask):
    """SOR update of the nodes in colour_mask (rh = h^2 r, scaled units)."""
    new = (1.0 - omega) * x + omega * (rh + _neighbour_sum(x, N)) / 6.0
    return np.where(colour_mask, new, x)


def ssor(r, N, h, omega=OMEGA, inner=INNER, outer=OUTER):
    """z = M(r) for A = (6 I - sum of neighbours) / h^2 (r, z flat, x fastest)."""
    rh = h * h * np.asarray(r, dtype=np.float64)
    red = red_mask(N)
    black = ~red
    x = np.zeros_like(rh)
    for _ in range(outer):
        for _ in range(inner):
            x = half_sweep(x, rh, N, omega, red)
            x = half_sweep(x, rh, N, omega, black)
        for _ in range(inner):
            x = half_sweep(x, rh, N, omega, black)
            x = half_sweep(x, rh, N, omega, red)
    return x
