"""Learned preconditioner and flexible CG, plain FP64 on the CPU.

Test infrastructure only (see ``oracle/__init__.py``).

The paper solves the Poisson system with preconditioned CG (Sec. 3.2) and
lists its preconditioners; it has no learned one. This module defines the
learned variant the GPU library offers, from standard published methods:

* conv3d: 3x3x3 cross-correlation with periodic wrap, weights
  w[c_out, c_in, tz, ty, tx], tap offset (tz-1, ty-1, tx-1):
      y[o, p] = sum_{c, t} w[o, c, t] * x[c, p + t - 1].
  Backward (data): gx[c, p] = sum_{o, t} w[o, c, t] * gy[o, p - t + 1].
  Backward (weights): gw[o, c, t] = sum_p gy[o, p] * x[c, p + t - 1].
* network N: conv(1->16), act, conv(16->16), act, conv(16->16), act,
  conv(16->1); no biases (14 688 weights); act = leaky ReLU with negative
  slope 1/8. N is positively homogeneous: N(c x) = c N(x) for c > 0.
* preconditioner P(r) = h^2 * s * N(r / s) - mean, s = RMS(r).
* training loss on a crop (periodic convs; only outputs at least 4 cells
  from every crop face are scored, where periodic and valid convolutions
  agree):  L = sum_in (N(r/s) - e/(s h^2))^2 / sum_in (e/(s h^2))^2.
* Adam: Kingma & Ba, ICLR 2015, with bias correction.
* FCG: flexible CG of Golub & Ye (SIAM J. Sci. Comput. 21, 1999) with the
  Polak-Ribiere-type beta = r_{k+1}.(z_{k+1} - z_k) / (r_k.z_k).
  Descent guard: when the preconditioned residual is not a descent
  direction (r.z <= 0 or not finite), that iteration uses the Jacobi
  direction z = (h^2/6) r instead; Jacobi-PCG is the fallback.
"""
import numpy as np

from . import pic

LEAK = 0.125
CHANNELS = (1, 16, 16, 16, 1)


def act(z):
    return np.where(z > 0.0, z, LEAK * z)


def act_grad(z):
    return np.where(z > 0.0, 1.0, LEAK)


def _shift(x, t):
    """x[..., p + t] with periodic wrap, t = (tz, ty, tx) offsets in {-1, 0, 1}."""
    return np.roll(x, shift=(-t[0], -t[1], -t[2]), axis=(-3, -2, -1))


TAPS = [(tz, ty, tx) for tz in (-1, 0, 1) for ty in (-1, 0, 1) for tx in (-1, 0, 1)]


def conv3d(x, w):
    """x[c_in, Z, Y, X], w[c_out, c_in, 3, 3, 3] -> y[c_out, Z, Y, X] (periodic)."""
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for t in TAPS:
        wt = w[:, :, t[0] + 1, t[1] + 1, t[2] + 1]
        y += np.einsum("oc,czyx->ozyx", wt, _shift(x, t))
    return y


def conv3d_bwd_data(gy, w):
    """Gradient w.r.t. the input of ``conv3d``: the adjoint map."""
    gx = np.zeros((w.shape[1],) + gy.shape[1:])
    for t in TAPS:
        wt = w[:, :, t[0] + 1, t[1] + 1, t[2] + 1]
        gx += np.einsum("oc,ozyx->czyx", wt, _shift(gy, (-t[0], -t[1], -t[2])))
    return gx


def conv3d_bwd_weight(x, gy):
    """Gradient w.r.t. the weights of ``conv3d``."""
    gw = np.zeros((gy.shape[0], x.shape[0], 3, 3, 3))
    for t in TAPS:
        gw[:, :, t[0] + 1, t[1] + 1, t[2] + 1] = np.einsum("ozyx,czyx->oc", gy, _shift(x, t))
    return gw


def init_weights(seed):
    """He-style random init (normal, std sqrt(2 / fan_in)) from a seeded generator."""
    rng = np.random.default_rng(seed)
    ws = []
    for i in range(4):
        cin, cout = CHANNELS[i], CHANNELS[i + 1]
        ws.append(rng.normal(0.0, np.sqrt(2.0 / (27 * cin)), size=(cout, cin, 3, 3, 3)))
    return ws


def forward(x, ws):
    """N(x) for x[Z, Y, X]; returns (y[Z, Y, X], cache for ``backward``)."""
    a = x[None]
    cache = [a]
    for i, w in enumerate(ws):
        z = conv3d(a, w)
        if i < 3:
            cache.append(z)
            a = act(z)
            cache.append(a)
        else:
            a = z
    return a[0], cache


def backward(gy, ws, cache):
    """Weight gradients of sum(gy * N(x)) given the forward cache."""
    g = gy[None]
    grads = [None] * 4
    for i in (3, 2, 1, 0):
        a_in = cache[2 * i]
        grads[i] = conv3d_bwd_weight(a_in, g)
        if i > 0:
            g = conv3d_bwd_data(g, ws[i]) * act_grad(cache[2 * i - 1])
    return grads


def interior_mask(shape, border=4):
    m = np.zeros(shape, dtype=bool)
    m[border:shape[0] - border, border:shape[1] - border, border:shape[2] - border] = True
    return m


def loss_and_grads(ws, r_crops, e_crops, h):
    """Mean over crops of the relative interior loss, and its weight gradients."""
    B = len(r_crops)
    total = 0.0
    gsum = [np.zeros_like(w) for w in ws]
    for r, e in zip(r_crops, e_crops):
        s = np.sqrt(np.mean(r * r))
        x = r / s
        t = e / (s * h * h)
        y, cache = forward(x, ws)
        m = interior_mask(r.shape)
        den = np.sum(t[m] ** 2)
        d = np.where(m, y - t, 0.0)
        total += np.sum(d * d) / den
        gy = 2.0 * d / den / B
        for acc, g in zip(gsum, backward(gy, ws, cache)):
            acc += g
    return total / B, gsum


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), t >= 1 the step number. In place."""
    for p, g, mi, vi in zip(params, grads, m, v):
        mi *= b1
        mi += (1.0 - b1) * g
        vi *= b2
        vi += (1.0 - b2) * g * g
        mhat = mi / (1.0 - b1 ** t)
        vhat = vi / (1.0 - b2 ** t)
        p -= lr * mhat / (np.sqrt(vhat) + eps)


def precondition(r, ws, N, h):
    """z = P(r) = h^2 s N(r/s) - mean, s = RMS(r)."""
    s = np.sqrt(np.mean(r * r))
    if s == 0.0:
        return np.zeros_like(r)
    y, _ = forward((r / s).reshape(N, N, N), ws)
    z = (h * h * s) * y.reshape(-1)
    return z - z.mean()


def fcg(b, x0, N, h, tol, maxit, prec):
    """Flexible CG (Golub & Ye 1999) on A x = b - mean(b) with z = prec(r).

    Stops when ||r||_2 <= tol ||b||_2 on the recursive residual. Returns
    (x with mean zero, iters, rel_res, converged flag).
    """
    b = b - b.mean()
    x = x0 - x0.mean()
    bnorm = np.sqrt(b @ b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    jacobi = h * h / 6.0
    fallbacks = 0

    def guarded(r):
        nonlocal fallbacks
        z = prec(r)
        rz = r @ z
        if not (np.isfinite(rz) and rz > 0.0):
            fallbacks += 1
            z = jacobi * r
        return z

    r = b - pic.apply_A(x, N, h)
    z = guarded(r)
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.sqrt(r @ r) / bnorm
    while rel > tol and it < maxit:
        q = pic.apply_A(p, N, h)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z_new = guarded(r)
        beta = (r @ (z_new - z)) / rz
        rz = r @ z_new
        p = z_new + beta * p
        z = z_new
        it += 1
        rel = np.sqrt(r @ r) / bnorm
    fcg.last_fallbacks = fallbacks
    return x - x.mean(), it, rel, rel <= tol
