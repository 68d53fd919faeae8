"""Training of the learned preconditioner: one call into the library.

pic_cnn_train generates the (residual, error) pairs with the library's own
solves (Jacobi-PCG snapshots of seeded Landau deposits for the
preconditioner, white-noise errors for the multigrid smoother), draws the
crops from a seeded Philox stream, runs the forward, loss, backward and Adam
kernels, and keeps the weights with the fewest flexible-CG iterations on a
held-out solve. Python only passes the options. ``init_weights`` builds the
network's Jacobi start on the host, for tests that need a fixed network.
"""
import numpy as np

from . import CNN_WEIGHTS, TRAIN_PRECONDITIONER, TRAIN_SMOOTHER

CHANNELS = (1, 16, 16, 16, 1)


def _adjoint(w, cout, cin):
    """w[o][c][t] -> adj[c][o][26 - t] (flattened)."""
    w = w.reshape(cout, cin, 27)
    return np.ascontiguousarray(np.transpose(w, (1, 0, 2))[:, :, ::-1]).reshape(-1)


def init_weights(seed, noise=0.02):
    """The Jacobi start plus small seeded noise (numpy): channel 0 of G carries
    r / sqrt(6) through the centre taps, so N = G^T G = 1/6 (the Jacobi
    direction of the scaled operator); layers 3-4 are the adjoints of layers
    2-1, in the library's order w[out][in][tz][ty][tx]."""
    rng = np.random.default_rng(seed)
    w1 = noise * rng.normal(0.0, np.sqrt(2.0 / 27.0), size=16 * 27)
    w2 = noise * rng.normal(0.0, np.sqrt(2.0 / (27.0 * 16)), size=16 * 16 * 27)
    w1[0 * 27 + 13] += 1.0 / np.sqrt(6.0)
    w2[(0 * 16 + 0) * 27 + 13] += 1.0
    w = np.concatenate([w1, w2, _adjoint(w2, 16, 16), _adjoint(w1, 16, 1)]).astype(np.float32)
    assert w.size == CNN_WEIGHTS
    return w


def train_preconditioner(ctx, **opts):
    """The network as flexible CG's preconditioner (pic_cnn_train with
    PIC_TRAIN_PRECONDITIONER; defaults: 64^3 snapshots of four deposits, 600
    Adam steps on 8 crops of 32^3, lr 2e-3, scored every 100 steps on a
    128^3 deposit). Returns the training info."""
    return ctx.cnn_train(TRAIN_PRECONDITIONER, **opts)


def train_smoother(ctx, **opts):
    """The network as the V-cycle's finest-level smoother (pic_cnn_train with
    PIC_TRAIN_SMOOTHER: white-noise errors, scored by multigrid FCG)."""
    return ctx.cnn_train(TRAIN_SMOOTHER, **opts)
