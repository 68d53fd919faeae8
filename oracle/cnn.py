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
* network N = G^T G with G = conv(16->16) o conv(1->16): four 3x3x3 convs
  1 -> 16 -> 16 -> 16 -> 1, no biases, identity activations, where layers 3
  and 4 are the adjoints of layers 2 and 1 (channels transposed, taps
  flipped): w3 = adj(w2), w4 = adj(w1). N is then linear, symmetric and
  positive semi-definite for any weights, a learned factorised sparse
  approximate inverse (Kolotilina & Yeremin 1993) with 9^3 support;
  14 688 weights of which 7 344 (w1, w2) are free.
* preconditioner P(r) = h^2 * s * N(r / s) - mean, s = RMS(r).
* training loss on a crop, the sum of the error in the energy (A-) norm and
  the residual norm, each relative to the target's:
    L = E(d) / E(t) + |A_I d|^2 / |A_I t|^2,  d = N(r/s) - t, t = e/(s h^2),
  with E(d) = sum over grid edges inside the valid interior R4 (cells at
  least 4 from every crop face, where periodic and valid convolutions agree)
  of the squared difference across the edge (d^T A d restricted to R4, up to
  h^2), and A_I d = 6 d_i - sum_nb d_j on the cells of R5 (at least 5 from
  every face, so the stencil stays in R4). Per Fourier mode k of the residual
  the two terms weight |r_k|^2 |1 - lambda_k p_k|^2 by 1/lambda_k and by 1:
  the first fixes the low-frequency gain (CG's condition number), the second
  keeps lambda_k p_k close to 1 (and positive) at high frequencies.
* Adam: Kingma & Ba, ICLR 2015, with bias correction.
* FCG: flexible CG with one retained direction, FCG(1) of Notay (SIAM J.
  Sci. Comput. 22, 2000): the new direction is z_{k+1} made A-conjugate to
  the previous one, beta = -(z_{k+1}.A p_k) / (p_k.A p_k), which keeps the
  local optimality for any (nonlinear, nonsymmetric) preconditioner; for a
  fixed SPD preconditioner it equals the PCG (Polak-Ribiere) beta.
  Descent guard: when the preconditioned residual is not a descent
  direction (r.z <= 0 or not finite), that iteration uses the Jacobi
  direction z = (h^2/6) r instead; Jacobi-PCG is the fallback.
"""
import numpy as np

from . import pic

CHANNELS = (1, 16, 16, 16, 1)


def adjoint(w):
    """Weights of the adjoint conv: w[o][c][tz][ty][tx] -> w[c][o][2-tz][2-ty][2-tx]."""
    return np.ascontiguousarray(np.transpose(w, (1, 0, 2, 3, 4))[:, :, ::-1, ::-1, ::-1])


def tie(w1, w2):
    """The four layers of N = G^T G from the free weights w1, w2."""
    return [w1, w2, adjoint(w2), adjoint(w1)]


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
    """Random free weights (normal, std sqrt(2 / fan_in)), tied into 4 layers."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, np.sqrt(2.0 / 27.0), size=(16, 1, 3, 3, 3))
    w2 = rng.normal(0.0, np.sqrt(2.0 / (27.0 * 16)), size=(16, 16, 3, 3, 3))
    return tie(w1, w2)


def forward(x, ws):
    """N(x) for x[Z, Y, X]; returns (y[Z, Y, X], cache for ``backward``)."""
    a = x[None]
    cache = [a]
    for w in ws:
        a = conv3d(a, w)
        cache.append(a)
    return a[0], cache


def backward(gy, ws, cache):
    """Gradients of sum(gy * N(x)) with respect to each of the 4 layers'
    weights, as if they were independent (see ``tied_grads``)."""
    g = gy[None]
    grads = [None] * 4
    for i in (3, 2, 1, 0):
        grads[i] = conv3d_bwd_weight(cache[i], g)
        if i > 0:
            g = conv3d_bwd_data(g, ws[i])
    return grads


def tied_grads(grads):
    """Gradients of the tied network: g1 + adj(g4) and g2 + adj(g3) for the
    free weights, repeated through the adjoint for layers 3 and 4."""
    g1 = grads[0] + adjoint(grads[3])
    g2 = grads[1] + adjoint(grads[2])
    return tie(g1, g2)


def interior_mask(shape, border=4):
    m = np.zeros(shape, dtype=bool)
    m[border:shape[0] - border, border:shape[1] - border, border:shape[2] - border] = True
    return m


def interior_energy(d, mask):
    """E(d) = sum of (d_i - d_j)^2 over neighbour pairs (i, j) along the three
    axes with both cells inside ``mask`` (no wrap)."""
    E = 0.0
    for ax in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[ax] = slice(0, -1)
        b[ax] = slice(1, None)
        both = mask[tuple(a)] & mask[tuple(b)]
        diff = d[tuple(a)] - d[tuple(b)]
        E += np.sum(np.where(both, diff * diff, 0.0))
    return E


def interior_energy_grad(d, mask):
    """dE/dd: 2 sum over the in-mask neighbours j of i of (d_i - d_j)."""
    g = np.zeros_like(d)
    for ax in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[ax] = slice(0, -1)
        b[ax] = slice(1, None)
        both = mask[tuple(a)] & mask[tuple(b)]
        diff = np.where(both, d[tuple(a)] - d[tuple(b)], 0.0)
        g[tuple(a)] += 2.0 * diff
        g[tuple(b)] -= 2.0 * diff
    return g


def interior_stencil(d, mask5):
    """q = 6 d_i - sum of the 6 neighbours d_j (no wrap) on the cells of
    ``mask5``, zero elsewhere (the caller keeps mask5 one cell inside the
    crop so the neighbours exist)."""
    q = 6.0 * d
    for ax in range(3):
        q = q - np.roll(d, 1, axis=ax) - np.roll(d, -1, axis=ax)
    return np.where(mask5, q, 0.0)


def interior_stencil_adjoint(q):
    """Transpose of ``interior_stencil`` applied to q (q zero outside mask5):
    g_i = 6 q_i - sum of the 6 neighbours q_j."""
    g = 6.0 * q
    for ax in range(3):
        g = g - np.roll(q, 1, axis=ax) - np.roll(q, -1, axis=ax)
    return g


def loss_and_grads(ws, r_crops, e_crops, h):
    """Mean over crops of the energy-norm plus residual-norm loss, and its
    gradients with respect to the tied weights (4 layers, layers 3-4 the
    adjoints of the gradients of the free layers 2-1)."""
    B = len(r_crops)
    total = 0.0
    gsum = [np.zeros_like(w) for w in ws]
    for r, e in zip(r_crops, e_crops):
        s = np.sqrt(np.mean(r * r))
        x = r / s
        t = e / (s * h * h)
        y, cache = forward(x, ws)
        m4 = interior_mask(r.shape, border=4)
        m5 = interior_mask(r.shape, border=5)
        den_e = interior_energy(t, m4)
        qt = interior_stencil(t, m5)
        den_r = np.sum(qt * qt)
        d = y - t
        q = interior_stencil(d, m5)
        total += interior_energy(d, m4) / den_e + np.sum(q * q) / den_r
        gy = (interior_energy_grad(d, m4) / den_e + 2.0 * interior_stencil_adjoint(q) / den_r) / B
        for acc, g in zip(gsum, tied_grads(backward(gy, ws, cache))):
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
    """Flexible CG, FCG(1) (Notay 2000), on A x = b - mean(b) with z = prec(r).

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
        pq = p @ q
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = guarded(r)
        beta = -(z @ q) / pq
        rz = r @ z
        p = z + beta * p
        it += 1
        rel = np.sqrt(r @ r) / bnorm
    fcg.last_fallbacks = fallbacks
    return x - x.mean(), it, rel, rel <= tol
