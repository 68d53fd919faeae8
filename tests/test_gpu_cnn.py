"""GPU parity of the learned preconditioner against the CPU oracle
(oracle/cnn.py).

Single convolutions (tensor cores, BF16 operands, FP32 accumulation) are
compared with the oracle's FP64 direct-loop convolution of the same
BF16-rounded inputs and weights: only the accumulation order differs, so the
tolerance is 1e-5 relative. The full network stores BF16 activations between
layers, so forward values and the loss are compared at BF16 tolerance (2e-2
relative), and weight gradients by direction (cosine >= 0.995) and magnitude
(1e-1 relative L2): they are sums over all cells of products whose signs
cancel, which magnifies the BF16 rounding of the data gradients. The FP32
test mode of the training passes pins every weight gradient element by element
(1e-2 of its value plus 1e-4 of the layer's largest). Adam is compared exactly
on the GPU's own gradients.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn  # noqa: E402
from oracle import pic as opic  # noqa: E402
from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rounded_weights(seed, scale=1.0):
    ws = [bf16_round(w * scale) for w in ocnn.init_weights(seed)]
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    return ws, flat


def ctx_with_weights(pg, flat, N=16):
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    return c


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("D", [16, 32])
def test_conv_raw_layers_match_oracle(pg, D):
    ws, flat = rounded_weights(1)
    c = ctx_with_weights(pg, flat)
    B = 2
    rng = np.random.default_rng(D)
    x1 = bf16_round(rng.normal(size=(B, D, D, D)))                  # one channel
    x16 = bf16_round(rng.normal(size=(B, D, D, D, 16)))             # channels last
    t1 = torch.from_numpy(x1.astype(np.float32)).cuda().reshape(-1)
    t16 = torch.from_numpy(x16.astype(np.float32)).to(torch.bfloat16).cuda().reshape(-1)
    out = torch.empty(B * D ** 3 * 16, dtype=torch.float32, device="cuda")
    cases = {
        0: (t1, lambda b: ocnn.conv3d(x1[b][None], ws[0])),
        1: (t16, lambda b: ocnn.conv3d(np.moveaxis(x16[b], -1, 0), ws[1])),
        2: (t16, lambda b: ocnn.conv3d(np.moveaxis(x16[b], -1, 0), ws[2])),
        3: (t16, lambda b: ocnn.conv3d(np.moveaxis(x16[b], -1, 0), ws[3])),
        4: (t1, lambda b: ocnn.conv3d_bwd_data(x1[b][None], ws[3])),
        5: (t16, lambda b: ocnn.conv3d_bwd_data(np.moveaxis(x16[b], -1, 0), ws[2])),
        6: (t16, lambda b: ocnn.conv3d_bwd_data(np.moveaxis(x16[b], -1, 0), ws[1])),
    }
    for which, (tin, ref_fn) in cases.items():
        out.fill_(float("nan"))
        c.cnn_conv_raw(which, tin, out, B, D)
        got = np.moveaxis(out.cpu().numpy().reshape(B, D, D, D, 16), -1, 1).astype(np.float64)
        for b in range(B):
            ref = ref_fn(b)
            nch = ref.shape[0]
            assert rel(got[b, :nch], ref) <= 1e-5, (which, b, rel(got[b, :nch], ref))
            if nch < 16:
                assert np.all(got[b, nch:] == 0.0), which


@pytest.mark.parametrize("N,mode,tol", [(32, "fp32", 1e-5), (64, "fp32", 1e-5), (64, "tc", 1e-5),
                                        (64, "layers", 2e-2), (48, "tc", 2e-2)])
def test_preconditioner_apply_matches_oracle(pg, N, mode, tol):
    """z = N r on the periodic grid against the oracle's FP64 four-layer
    network: the composed 9^3 kernel on the CUDA cores to FP32 accuracy (also
    what the tensor-core mode runs on grids that are not a multiple of 128),
    the four BF16 convs (what N = 48, not a multiple of 32, runs in every mode)
    to BF16 accuracy."""
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    ws32 = [w.astype(np.float32).astype(np.float64) for w in ws]
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    c.cnn_set_apply({"tc": pg.CNN_APPLY_TC, "fp32": pg.CNN_APPLY_FP32, "layers": pg.CNN_APPLY_LAYERS}[mode])
    r = inputs.noise_field(N, 3)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z = torch.empty_like(rt)
    c.cnn_apply(rt, z)
    ref, _ = ocnn.forward(r.astype(np.float32).astype(np.float64).reshape(N, N, N), ws32)
    assert rel(z.cpu().numpy().astype(np.float64), ref.reshape(-1)) <= tol


def oracle_sampled_apply(r, N, ws, points):
    """The oracle network at sampled cells: N r at p depends on r within
    distance 4 (four 3x3x3 layers), so the oracle's forward pass on the 9^3
    periodic crop centred at p gives the exact value at the crop's centre."""
    g = r.reshape(N, N, N)
    out = []
    for (pz, py, px) in points:
        idx = [(c + np.arange(-4, 5)) % N for c in (pz, py, px)]
        crop = g[np.ix_(*idx)]
        y, _ = ocnn.forward(crop, ws)
        out.append(y[4, 4, 4])
    return np.array(out)


@pytest.mark.parametrize("N", [128, 256, 384])
@pytest.mark.parametrize("mode", ["tc", "tc8"])
def test_tensor_core_preconditioner_matches_oracle_sampled(pg, N, mode):
    """The composed 9^3 kernel on the tensor cores (BF16 r and K, FP32
    accumulation in TMEM; the 16-wide default and the 8-wide form) against the
    oracle's FP64 network at 200 sampled cells (BF16 tolerance), and against
    the FP32 CUDA-core evaluation of the same composed kernel at every cell.
    The sample includes the grid's corners and faces, where the periodic wrap
    and the edges of the 8 x 128 and 16 x 128 column blocks are exercised."""
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    ws32 = [w.astype(np.float32).astype(np.float64) for w in ws]
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    r = inputs.noise_field(N, 4)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z_tc = torch.full_like(rt, float("nan"))
    z_32 = torch.full_like(rt, float("nan"))
    c.cnn_set_apply(pg.CNN_APPLY_TC if mode == "tc" else pg.CNN_APPLY_TC8)
    c.cnn_apply(rt, z_tc)
    c.cnn_set_apply(pg.CNN_APPLY_FP32)
    c.cnn_apply(rt, z_32)
    zt = z_tc.cpu().numpy().astype(np.float64)
    z3 = z_32.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(zt))
    assert rel(zt, z3) <= 1e-2
    rng = np.random.default_rng(N)
    pts = [tuple(p) for p in rng.integers(0, N, size=(180, 3))]
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 15), (N - 1, 0, 16), (5, 127, 0), (6, 128 % N, N - 1),
            (N // 2, N - 1, N // 2), (3, 4, N - 16), (N - 4, 124, 31), (1, 1, N - 1), (N - 1, 129 % N, 0),
            (7, N - 5, 8), (N // 3, 63, 47), (2, N - 2, N - 2), (N - 2, 2, 2), (9, 120, 112), (11, 135 % N, 113),
            (0, 64, 0), (N - 1, 191 % N, N - 1), (17, 255 % N, 240 % N)]
    ref = oracle_sampled_apply(r.astype(np.float32).astype(np.float64), N, ws32, pts)
    got = np.array([zt.reshape(N, N, N)[p] for p in pts])
    assert rel(got, ref) <= 1e-2


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("N", [128, 256, 384])
def test_tensor_core_preconditioner_exact_in_bf16(pg, N):
    """Both tensor-core forms compute z = K * r exactly for the BF16-rounded
    r and K, up to FP32 accumulation: the composed kernel K is read back as
    the FP32 CUDA-core path's response to a unit impulse, both operands are
    rounded to BF16 on the host, and z at 300 sampled cells is the FP64 sum
    over the 729 taps. The bound is 1e-5 of the sum of |products| at each cell
    (a wrong, missing or shifted tap moves z by a whole product). 8-wide and
    16-wide forms agree to FP32 rounding at every cell. At 128^3 the CTAs' unit
    ranges end inside columns every ~13 planes, so every truncated group list
    at the ends of a run (and the split zero-led pairs) is exercised."""
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    ctr = N // 2
    delta = torch.zeros(N ** 3, dtype=torch.float32, device="cuda")
    delta[(ctr * N + ctr) * N + ctr] = 1.0
    resp = torch.empty_like(delta)
    c.cnn_set_apply(pg.CNN_APPLY_FP32)
    c.cnn_apply(delta, resp)
    Kr = resp.cpu().numpy().reshape(N, N, N)[ctr - 4:ctr + 5, ctr - 4:ctr + 5, ctr - 4:ctr + 5]
    Kb = bf16_round(Kr)  # Kb[e + 4] = response at offset e; z = Kb (convolution) r
    r = inputs.noise_field(N, 6).astype(np.float32)
    rb = bf16_round(r).reshape(N, N, N)
    rt = torch.from_numpy(r).cuda()
    out = {}
    for mode in (pg.CNN_APPLY_TC, pg.CNN_APPLY_TC8):
        z = torch.full_like(rt, float("nan"))
        c.cnn_set_apply(mode)
        c.cnn_apply(rt, z)
        out[mode] = z.cpu().numpy().astype(np.float64).reshape(N, N, N)
        assert np.all(np.isfinite(out[mode])), mode
    rng = np.random.default_rng(N + 1)
    pts = [tuple(p) for p in rng.integers(0, N, size=(260, 3))]
    for x in (0, 7, 8, 15, 16, N - 9, N - 8, N - 1):  # column edges in x, both widths
        for y in (0, 127, 128 % N, N - 1):
            pts.append((int(rng.integers(0, N)), y, x))
    e = np.arange(-4, 5)
    for p in pts:
        idx = [(p[a] - e) % N for a in range(3)]
        win = rb[np.ix_(*idx)]
        prod = Kb * win
        ref, bound = prod.sum(), np.abs(prod).sum()
        for mode, z in out.items():
            assert abs(z[p] - ref) <= 1e-5 * bound + 1e-30, (mode, p, z[p], ref, bound)
    assert rel(out[pg.CNN_APPLY_TC].reshape(-1), out[pg.CNN_APPLY_TC8].reshape(-1)) <= 1e-6


def test_network_forward_loss_and_gradients_match_oracle(pg):
    N, D, B = 32, 16, 2
    h = L / N
    ws, flat = rounded_weights(2)
    c = ctx_with_weights(pg, flat, N)
    r = inputs.noise_field(N, 5)
    a = inputs.noise_field(N, 6)
    b = inputs.noise_field(N, 7)
    origins = np.array([[0, 3, 5], [20, 31, 9]], dtype=np.int32)
    x = torch.empty(B * D ** 3, dtype=torch.float32, device="cuda")
    t = torch.empty_like(x)
    c.cnn_make_batch(torch.from_numpy(r).cuda(), torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                     origins, D, x, t, h * h)
    # oracle crops (periodic) of r and e = a - b
    def crop(f, o):
        g = f.reshape(N, N, N)
        iz = (o[2] + np.arange(D)) % N
        iy = (o[1] + np.arange(D)) % N
        ix = (o[0] + np.arange(D)) % N
        return g[np.ix_(iz, iy, ix)]
    r_cr = [crop(r, o) for o in origins]
    e_cr = [crop(a - b, o) for o in origins]
    xs = x.cpu().numpy().reshape(B, D, D, D)
    ts = t.cpu().numpy().reshape(B, D, D, D)
    for i in range(B):
        s = np.sqrt(np.mean(r_cr[i] ** 2))
        assert rel(xs[i], r_cr[i] / s) <= 1e-6
        assert rel(ts[i], e_cr[i] / (s * h * h)) <= 1e-6
    y = torch.empty_like(x)
    c.cnn_forward(x, y, B, D)
    ys = y.cpu().numpy().reshape(B, D, D, D)
    for i in range(B):
        ref, _ = ocnn.forward(r_cr[i] / np.sqrt(np.mean(r_cr[i] ** 2)), ws)
        assert rel(ys[i], ref) <= 2e-2
    gy = torch.empty_like(x)
    loss = c.cnn_loss(y, t, B, D, gy)
    ref_loss, ref_grads = ocnn.loss_and_grads(ws, r_cr, e_cr, h)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    c.cnn_backward(gy, B, D)
    g = c.cnn_get_grads()
    off = 0
    report = []
    for layer, rg in enumerate(ref_grads):
        gl = g[off:off + rg.size].reshape(rg.shape).astype(np.float64)
        off += rg.size
        cos = np.sum(gl * rg) / (np.linalg.norm(gl) * np.linalg.norm(rg))
        report.append((layer, rel(gl, rg), cos))
    # BF16 activations and data gradients, then a sum over all cells with
    # cancelling signs: the direction is pinned tightly, the magnitude loosely
    for layer, r_err, cos in report:
        assert cos >= 0.995 and r_err <= 0.1, report


def test_network_gradients_fp32_mode_match_oracle_elementwise(pg):
    """The training passes in the FP32 test mode (every convolution on the
    CUDA cores in FP32): the forward values, the loss and every weight
    gradient (which carries the whole chain of data gradients) against the
    oracle's FP64 network on the same crops, element by element. Bound per
    weight: 1e-2 of its own value plus 1e-4 of the layer's largest gradient
    (a gradient is a sum over 8192 cells whose terms can cancel to far below
    their magnitudes, where FP32 accumulation of ~5e-6 of the sum of |terms|
    dominates)."""
    N, D, B = 32, 16, 2
    h = L / N
    ws, flat = rounded_weights(2)
    c = ctx_with_weights(pg, flat, N)
    c.cnn_set_train_precision(pg.CNN_TRAIN_FP32)
    r = inputs.noise_field(N, 5)
    a = inputs.noise_field(N, 6)
    b = inputs.noise_field(N, 7)
    origins = np.array([[0, 3, 5], [20, 31, 9]], dtype=np.int32)
    x = torch.empty(B * D ** 3, dtype=torch.float32, device="cuda")
    t = torch.empty_like(x)
    c.cnn_make_batch(torch.from_numpy(r).cuda(), torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                     origins, D, x, t, h * h)

    def crop(f, o):
        g = f.reshape(N, N, N)
        return g[np.ix_((o[2] + np.arange(D)) % N, (o[1] + np.arange(D)) % N, (o[0] + np.arange(D)) % N)]
    r_cr = [crop(r, o) for o in origins]
    e_cr = [crop(a - b, o) for o in origins]
    y = torch.empty_like(x)
    c.cnn_forward(x, y, B, D)
    ys = y.cpu().numpy().reshape(B, D, D, D)
    for i in range(B):
        ref, _ = ocnn.forward(r_cr[i] / np.sqrt(np.mean(r_cr[i] ** 2)), ws)
        assert np.max(np.abs(ys[i] - ref)) <= 1e-5 * np.max(np.abs(ref))
    gy = torch.empty_like(x)
    loss = c.cnn_loss(y, t, B, D, gy)
    ref_loss, ref_grads = ocnn.loss_and_grads(ws, r_cr, e_cr, h)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    c.cnn_backward(gy, B, D)
    g = c.cnn_get_grads()
    off = 0
    for layer, rg in enumerate(ref_grads):
        gl = g[off:off + rg.size].reshape(rg.shape).astype(np.float64)
        off += rg.size
        err = np.abs(gl - rg)
        bound = 1e-2 * np.abs(rg) + 1e-4 * np.max(np.abs(rg))
        assert np.all(err <= bound), (layer, float(np.max(err / bound)), float(np.median(err / np.abs(rg))))
    # a backward pass in the other mode needs its own forward pass
    c.cnn_set_train_precision(pg.CNN_TRAIN_BF16)
    with pytest.raises(pg.PicError) as ex:
        c.cnn_backward(gy, B, D)
    assert ex.value.code == pg.PIC_ESTATE
    c.close()


def test_adam_matches_oracle_on_gpu_gradients(pg):
    ws, flat = rounded_weights(3)
    c = ctx_with_weights(pg, flat, 16)
    D, B = 16, 1
    x = torch.from_numpy(inputs.noise_field(D, 1).astype(np.float32)).cuda()
    y = torch.empty_like(x)
    c.cnn_forward(x, y, B, D)
    c.cnn_backward(torch.ones_like(y), B, D)
    g = c.cnn_get_grads().astype(np.float64)
    c.cnn_adam(1e-3)
    got = c.cnn_get_weights().astype(np.float64)
    p = [flat.astype(np.float64)]
    m = [np.zeros_like(p[0])]
    v = [np.zeros_like(p[0])]
    ocnn.adam_step(p, [g], m, v, 1, lr=1e-3)
    assert np.max(np.abs(got - p[0])) <= 1e-6
    assert np.all(c.cnn_get_grads() == 0.0)


@pytest.mark.parametrize("N", [32, 64])
def test_fcg_cnn_solve_reaches_true_residual(pg, N):
    """Flexible CG with the network (random weights: the descent guard keeps
    it convergent) reaches the same true FP64 relative residual 1e-10 as the
    Jacobi-PCG reference."""
    h = L / N
    _, flat = rounded_weights(4)
    c = ctx_with_weights(pg, flat, N)
    b = inputs.landau_noise_rhs(N, 11)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    info = c.solve(torch.from_numpy(b).cuda(), phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED,
                   precond=pg.PC_CNN)
    got = phi.cpu().numpy()
    bp = b - b.mean()
    assert np.linalg.norm(bp - opic.apply_A(got, N, h)) <= 1.05e-10 * np.linalg.norm(bp), info
    ref, _, _, _ = opic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-13, 5000)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_fused_fcg_step_matches_the_unfused_one(pg):
    """On a 128^3 grid the tensor-core preconditioner runs with the CG update
    and the direction's dots fused into it (and recomputes z after each
    reliable update), or alone with the update and the dots in their own
    kernels (the default form). Each must reach the true FP64 relative residual 1e-10
    (checked with the oracle's operator) in about as many iterations as the
    unfused sequence with the FP32 evaluation of the same composed kernel, and
    its solution must agree with that one to the solve tolerance."""
    N = 128
    h = L / N
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    c = ctx_with_weights(pg, flat, N)
    b = inputs.landau_noise_rhs(N, 12)
    bt = torch.from_numpy(b).cuda()
    res = {}
    modes = {"tc_fused": pg.CNN_APPLY_TC_FUSED, "tc": pg.CNN_APPLY_TC, "fp32": pg.CNN_APPLY_FP32}
    for mode, code in modes.items():
        c.cnn_set_apply(code)
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(bt, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, precond=pg.PC_CNN)
        got = phi.cpu().numpy()
        bp = b - b.mean()
        assert np.linalg.norm(bp - opic.apply_A(got, N, h)) <= 1.05e-10 * np.linalg.norm(bp), (mode, info)
        res[mode] = (info, got)
    f32 = res["fp32"][0]
    for mode in ("tc_fused", "tc"):
        tc = res[mode][0]
        assert tc["reliable_updates"] > 0, (mode, tc)
        assert abs(tc["iters"] - f32["iters"]) <= 0.15 * f32["iters"] + 3, (mode, tc, f32)
        a, r = res[mode][1], res["fp32"][1]
        assert np.linalg.norm(a - r) <= 1e-8 * np.linalg.norm(r), mode


def jacobi_network_weights():
    """Weights for which N(x) = x / 6: channel 0 of G carries x / sqrt(6)
    through the centre taps, so N = G^T G = 1/6, the Jacobi direction r / 6
    of the scaled operator."""
    w1 = np.zeros((16, 1, 3, 3, 3)); w2 = np.zeros((16, 16, 3, 3, 3))
    w1[0, 0, 1, 1, 1] = 1.0 / np.sqrt(6.0)
    w2[0, 0, 1, 1, 1] = 1.0
    return np.concatenate([w.reshape(-1) for w in ocnn.tie(w1, w2)]).astype(np.float32)


@pytest.mark.parametrize("N", [64, 128])
def test_fcg_with_jacobi_network_takes_the_jacobi_iterations(pg, N):
    """The whole inference + flexible-CG chain with a network that computes
    the Jacobi direction must converge like mixed Jacobi-CG, up to the cost of
    the BF16 rounding of its activations (an inexact preconditioner, which
    flexible CG tolerates with a few more iterations). N = 128 runs the
    tensor-core form with the CG update fused into it."""
    c = pg.Context().init(N, 0, 0)
    if N % 128 == 0:
        c.cnn_set_apply(pg.CNN_APPLY_TC_FUSED)
    c.cnn_set_weights(jacobi_network_weights())
    b = torch.from_numpy(inputs.landau_noise_rhs(N, 11)).cuda()
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    ref = c.solve(b, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED)
    phi.zero_()
    got = c.solve(b, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, precond=pg.PC_CNN)
    assert got["fallbacks"] == 0, got
    assert got["iters"] <= 1.25 * ref["iters"], (got, ref)


def test_cnn_requires_weights_and_mixed_precision(pg):
    c = pg.Context().init(16, 0, 0)
    rho = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rho)
    code, _ = pg.poisson_solve_ex(c.h, rho, phi, 1e-10, 10, c.n, pg.PREC_MIXED, pg.PC_CNN)
    assert code == pg.PIC_ESTATE
    code, _ = pg.poisson_solve_ex(c.h, rho, phi, 1e-10, 10, c.n, pg.PREC_FP64, pg.PC_CNN)
    assert code == pg.PIC_EINVAL


def test_trained_preconditioner_gain(pg, capsys):
    """What the trained network gains over the method without it.

    The network is trained on the GPU by pic_cnn_train (600 Adam steps on
    32^3 crops of (residual, error) pairs from Jacobi-PCG snapshots of four
    64^3 Landau deposits, forward/backward by the library's kernels, the
    weights scored on a held-out 128^3 deposit), then flexible CG with it
    solves other held-out Landau deposits at 64^3 and 128^3 to the true
    relative residual 1e-10. Asserted: the loss falls, convergence, no
    descent-guard fallback, and at least 2x fewer iterations than
    mixed-precision Jacobi-CG; reported: iterations and device time of both
    and of the FP64 reference solve."""
    c = pg.Context().init(64, 0, 0)
    info = c.cnn_train(pg.TRAIN_PRECONDITIONER)
    assert info["loss_last"] < 0.7 * info["loss_first"], info
    assert 0 < info["best_iters"] < 2001 and info["adam_steps"] <= 600, info
    w = c.cnn_get_weights()
    report = {}
    for N in (64, 128):
        ce = pg.Context().init(N, 8, 99)
        rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        ce.deposit(rho)
        ce.cnn_set_weights(w)
        res = {}
        for name, prec, pc in (("fp64_jacobi", pg.PREC_FP64, pg.PC_JACOBI),
                               ("mixed_jacobi", pg.PREC_MIXED, pg.PC_JACOBI),
                               ("mixed_fcg_cnn", pg.PREC_MIXED, pg.PC_CNN)):
            best = None
            for _ in range(2):
                phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
                r = ce.solve(rho, phi, tol=1e-10, maxit=20000, precision=prec, precond=pc)
                best = r if best is None or r["t_ms"] < best["t_ms"] else best
            res[name] = best
        cnn, jac = res["mixed_fcg_cnn"], res["mixed_jacobi"]
        assert cnn["converged"] and cnn["rel_res"] <= 1e-10 and cnn["fallbacks"] == 0, cnn
        assert cnn["iters"] * 2 <= jac["iters"], (cnn, jac)
        report[N] = {k: (v["iters"], round(v["t_ms"], 2)) for k, v in res.items()}
        ce.close()
    c.close()
    with capsys.disabled():
        print("\npreconditioner gain (iterations, device ms):", report, "training:", info)