"""Pins of the learned-preconditioner oracle (oracle/cnn.py): a library
convolution, brute-force loops, the adjoint identity, the symmetry and
positive semi-definiteness of N = G^T G, central finite differences,
Adam's closed-form first step, and FCG reducing to PCG.
"""
import numpy as np
import pytest
import torch

from oracle import cnn, pic

L = 4.0 * np.pi


def test_conv3d_matches_torch_circular():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6, 7))
    w = rng.normal(size=(4, 3, 3, 3, 3))
    xt = torch.nn.functional.pad(torch.from_numpy(x)[None], (1, 1, 1, 1, 1, 1), mode="circular")
    ref = torch.nn.functional.conv3d(xt, torch.from_numpy(w))[0].numpy()
    assert np.allclose(cnn.conv3d(x, w), ref, atol=1e-12)


def test_conv3d_brute_force_loop():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 4, 4))
    w = rng.normal(size=(2, 2, 3, 3, 3))
    ref = np.zeros((2, 4, 4, 4))
    for o in range(2):
        for z in range(4):
            for y in range(4):
                for xx in range(4):
                    s = 0.0
                    for c in range(2):
                        for tz in range(3):
                            for ty in range(3):
                                for tx in range(3):
                                    s += w[o, c, tz, ty, tx] * x[c, (z + tz - 1) % 4, (y + ty - 1) % 4, (xx + tx - 1) % 4]
                    ref[o, z, y, xx] = s
    assert np.allclose(cnn.conv3d(x, w), ref, atol=1e-12)


def test_conv3d_single_tap_is_a_shift():
    x = np.random.default_rng(2).normal(size=(1, 4, 5, 6))
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 2, 1, 0] = 1.0   # offset (+1, 0, -1)
    y = cnn.conv3d(x, w)
    assert np.array_equal(y[0], np.roll(x[0], shift=(-1, 0, 1), axis=(0, 1, 2)))


def test_bwd_data_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3, 4, 5, 6))
    gy = rng.normal(size=(2, 4, 5, 6))
    w = rng.normal(size=(2, 3, 3, 3, 3))
    lhs = np.sum(cnn.conv3d(x, w) * gy)
    rhs = np.sum(x * cnn.conv3d_bwd_data(gy, w))
    assert np.isclose(lhs, rhs, rtol=1e-12)


def test_bwd_weight_finite_differences():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 4, 4, 5))
    gy = rng.normal(size=(3, 4, 4, 5))
    w = rng.normal(size=(3, 2, 3, 3, 3))
    gw = cnn.conv3d_bwd_weight(x, gy)
    eps = 1e-6
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 0, 2, 2, 2), (0, 1, 1, 1, 1)]:
        wp = w.copy(); wp[idx] += eps
        wm = w.copy(); wm[idx] -= eps
        fd = (np.sum(cnn.conv3d(x, wp) * gy) - np.sum(cnn.conv3d(x, wm) * gy)) / (2 * eps)
        assert np.isclose(gw[idx], fd, rtol=1e-7, atol=1e-8)


def test_network_backward_finite_differences():
    rng = np.random.default_rng(5)
    ws = cnn.init_weights(11)
    x = rng.normal(size=(6, 6, 6))
    gy = rng.normal(size=(6, 6, 6))
    y, cache = cnn.forward(x, ws)
    grads = cnn.backward(gy, ws, cache)
    eps = 1e-6
    for layer, idx in [(0, (3, 0, 1, 1, 2)), (1, (5, 7, 0, 2, 1)), (2, (15, 15, 2, 2, 2)), (3, (0, 9, 1, 0, 1))]:
        wp = [w.copy() for w in ws]; wp[layer][idx] += eps
        wm = [w.copy() for w in ws]; wm[layer][idx] -= eps
        fd = (np.sum(cnn.forward(x, wp)[0] * gy) - np.sum(cnn.forward(x, wm)[0] * gy)) / (2 * eps)
        assert np.isclose(grads[layer][idx], fd, rtol=1e-6, atol=1e-9)


def test_network_weight_count_linearity_and_symmetry():
    ws = cnn.init_weights(0)
    assert sum(w.size for w in ws) == 14688
    assert np.array_equal(ws[2], cnn.adjoint(ws[1])) and np.array_equal(ws[3], cnn.adjoint(ws[0]))
    rng = np.random.default_rng(6)
    x, y = rng.normal(size=(5, 5, 5)), rng.normal(size=(5, 5, 5))
    Nx, Ny = cnn.forward(x, ws)[0], cnn.forward(y, ws)[0]
    # linear
    assert np.allclose(cnn.forward(3.0 * x - 2.0 * y, ws)[0], 3.0 * Nx - 2.0 * Ny, atol=1e-10)
    # self-adjoint and positive semi-definite: N = G^T G
    assert np.isclose(np.sum(Nx * y), np.sum(x * Ny), rtol=1e-12)
    assert np.sum(Nx * x) >= 0.0
    G = lambda v: cnn.conv3d(cnn.conv3d(v[None], ws[0]), ws[1])
    assert np.isclose(np.sum(Nx * x), np.sum(G(x) ** 2), rtol=1e-12)


def test_adjoint_weights_give_the_adjoint_conv():
    rng = np.random.default_rng(7)
    w = rng.normal(size=(4, 3, 3, 3, 3))
    x, gy = rng.normal(size=(3, 5, 4, 6)), rng.normal(size=(4, 5, 4, 6))
    assert np.allclose(cnn.conv3d(gy, cnn.adjoint(w)), cnn.conv3d_bwd_data(gy, w), atol=1e-12)


def test_loss_gradient_finite_differences():
    # gradients with respect to the free weights w1, w2 of the tied network
    rng = np.random.default_rng(7)
    ws = cnn.init_weights(3)
    r = [rng.normal(size=(12, 12, 12)) for _ in range(2)]
    e = [rng.normal(size=(12, 12, 12)) for _ in range(2)]
    h = 0.3
    loss, grads = cnn.loss_and_grads(ws, r, e, h)
    assert np.array_equal(grads[2], cnn.adjoint(grads[1])) and np.array_equal(grads[3], cnn.adjoint(grads[0]))
    eps = 1e-6
    for layer, idx in [(0, (1, 0, 0, 1, 2)), (0, (9, 0, 2, 2, 2)), (1, (4, 9, 1, 1, 0)), (1, (0, 3, 2, 1, 1))]:
        def loss_at(delta):
            free = [ws[0].copy(), ws[1].copy()]
            free[layer][idx] += delta
            return cnn.loss_and_grads(cnn.tie(*free), r, e, h)[0]
        fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
        assert np.isclose(grads[layer][idx], fd, rtol=1e-6, atol=1e-10)


def test_interior_stencil_closed_forms():
    # a linear field has zero 7-point stencil; a quadratic x^2 gives -2
    m5 = cnn.interior_mask((12, 12, 12), border=5)
    x = np.broadcast_to(np.arange(12.0)[None, None, :], (12, 12, 12)).copy()
    assert np.all(cnn.interior_stencil(3.0 * x + 1.0, m5) == 0.0)
    q = cnn.interior_stencil(x * x, m5)
    assert np.all(q[m5] == -2.0) and np.all(q[~m5] == 0.0)
    # the adjoint: <A_I d, q> = <d, A_I^T q> for q supported on the mask
    rng = np.random.default_rng(0)
    d = rng.normal(size=(12, 12, 12))
    qq = np.where(m5, rng.normal(size=(12, 12, 12)), 0.0)
    assert np.isclose(np.sum(cnn.interior_stencil(d, m5) * qq), np.sum(d * cnn.interior_stencil_adjoint(qq)))


def test_interior_energy_closed_forms():
    # d = x index on a 10^3 crop; the valid interior is cells 4..5 along each
    # axis, so it holds one x-edge per (y, z) row, 2 x 2 rows, each differing
    # by 1, and no y- or z-edge with a difference
    m = cnn.interior_mask((10, 10, 10))
    d = np.broadcast_to(np.arange(10.0)[None, None, :], (10, 10, 10)).copy()
    assert cnn.interior_energy(d, m) == 4.0
    assert cnn.interior_energy(np.full((10, 10, 10), 3.0), m) == 0.0
    full = np.ones((6, 6, 6), dtype=bool)
    v = np.random.default_rng(0).normal(size=(6, 6, 6))
    # E is quadratic: E(v) = v . grad / 2
    assert np.isclose(cnn.interior_energy(v, full), 0.5 * np.sum(v * cnn.interior_energy_grad(v, full)))


def test_energy_below_target_gives_descent_direction():
    # on a periodic grid, E(z - e) < E(e) implies r.z > 0 with r = A e
    rng = np.random.default_rng(3)
    N, h = 8, 0.5
    e = rng.normal(size=N ** 3)
    r = pic.apply_A(e, N, h)
    for _ in range(20):
        z = e + 0.9 * rng.uniform() * np.linalg.norm(e) * rng.normal(size=N ** 3) / np.sqrt(N ** 3)
        d = z - e
        if d @ pic.apply_A(d, N, h) < e @ r:
            assert r @ z > 0


def test_residual_loss_ignores_constant_offsets():
    # a constant offset of the prediction (null space of the stencil) costs nothing
    m5 = cnn.interior_mask((12, 12, 12), border=5)
    t = np.random.default_rng(1).normal(size=(12, 12, 12))
    assert np.allclose(cnn.interior_stencil(t + 2.5, m5), cnn.interior_stencil(t, m5), atol=1e-12)


def test_loss_ignores_crop_border():
    rng = np.random.default_rng(8)
    ws = cnn.init_weights(3)
    r = rng.normal(size=(12, 12, 12))
    e = rng.normal(size=(12, 12, 12))
    l0, _ = cnn.loss_and_grads(ws, [r], [e], 1.0)
    e2 = e.copy(); e2[0:4, :, :] += 5.0; e2[:, 8:, :] -= 2.0     # within 4 cells of a face only
    l1, _ = cnn.loss_and_grads(ws, [r], [e2], 1.0)
    assert l0 == l1
    # an input change 4 cells from the face moves interior outputs only through the
    # receptive field; a change on the face itself (distance 0) must not reach them
    # through wrap-around
    r2 = r.copy(); r2[:, :, 0] += 1.0
    y1, _ = cnn.forward(r, ws)
    y2, _ = cnn.forward(r2, ws)
    m = cnn.interior_mask(r.shape)
    assert np.array_equal((y1 != y2) & m & (np.arange(12)[None, None, :] >= 5), np.zeros_like(m))


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -1e-3, 0.0])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    cnn.adam_step(p, g, m, v, 1, lr=0.01)
    # m_hat = g, v_hat = g^2  =>  step = lr * g / (|g| + eps)
    ref = np.array([1.0, -2.0, 0.5]) - 0.01 * np.array([0.3, -1e-3, 0.0]) / (np.abs([0.3, -1e-3, 0.0]) + 1e-8)
    assert np.allclose(p[0], ref, atol=1e-15)


def test_fcg_with_jacobi_equals_pcg():
    N = 8
    h = L / N
    b = np.random.default_rng(9).normal(size=N ** 3)
    x1, it1, rel1, _ = pic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-12, 500)
    x2, it2, rel2, _ = cnn.fcg(b, np.zeros(N ** 3), N, h, 1e-12, 500, lambda r: r * (h * h / 6.0))
    assert it1 == it2
    assert np.allclose(x1, x2, atol=1e-12 * np.abs(x1).max())


def test_fcg_nonlinear_preconditioner_converges():
    N = 8
    h = L / N
    b = np.random.default_rng(10).normal(size=N ** 3)
    prec = lambda r: (h * h / 6.0) * r * (1.0 + 0.3 * np.tanh(r / (np.abs(r).max() + 1e-300)))
    x, it, rel, ok = cnn.fcg(b, np.zeros(N ** 3), N, h, 1e-11, 500, prec)
    assert ok
    ref = pic.spectral_solve(b, N, h)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_cnn_preconditioner_fcg_reaches_tolerance():
    N = 8
    h = L / N
    b = np.random.default_rng(12).normal(size=N ** 3)
    ws = cnn.init_weights(5)
    x, it, rel, ok = cnn.fcg(b, np.zeros(N ** 3), N, h, 1e-10, 2000, lambda r: cnn.precondition(r, ws, N, h))
    assert ok
    ref = pic.spectral_solve(b, N, h)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
