"""Training of the learned preconditioner on the GPU.

Data are (residual, error) pairs that the method's own Jacobi-PCG solves
generate (Sec. 3.2 solver, Sec. 2.1 Landau densities): for a right-hand side
rho the library solves to a tight tolerance for phi*, then reruns CG from zero
for k iterations to get the iterate phi_k, and pic_residual gives
r_k = b - A phi_k; the target is e_k = phi* - phi_k. Training draws random
periodic crops of (r_k, e_k), runs the network forward, the interior loss,
the backward pass and Adam, all as library kernels. Python only sequences the
calls and draws the seeded random crop origins.
"""
import numpy as np

from . import CNN_WEIGHTS, PC_CNN, PC_JACOBI, PREC_FP64, PREC_MIXED, Context

CHANNELS = (1, 16, 16, 16, 1)
SNAPSHOT_ITERS = (1, 2, 4, 8, 16, 32, 64, 128)


def _adjoint(w, cout, cin):
    """w[o][c][t] -> adj[c][o][26 - t] (flattened)."""
    w = w.reshape(cout, cin, 27)
    return np.ascontiguousarray(np.transpose(w, (1, 0, 2))[:, :, ::-1]).reshape(-1)


def init_weights(seed, noise=0.02):
    """Start from the Jacobi preconditioner plus small seeded noise: channel 0
    of G carries r / sqrt(6) through the centre taps, so N = G^T G = 1/6
    (the Jacobi direction of the scaled operator); layers 3-4 are the
    adjoints of layers 2-1, in the library's order w[out][in][tz][ty][tx]."""
    rng = np.random.default_rng(seed)
    w1 = noise * rng.normal(0.0, np.sqrt(2.0 / 27.0), size=16 * 27)
    w2 = noise * rng.normal(0.0, np.sqrt(2.0 / (27.0 * 16)), size=16 * 16 * 27)
    w1[0 * 27 + 13] += 1.0 / np.sqrt(6.0)
    w2[(0 * 16 + 0) * 27 + 13] += 1.0
    w = np.concatenate([w1, w2, _adjoint(w2, 16, 16), _adjoint(w1, 16, 1)]).astype(np.float32)
    assert w.size == CNN_WEIGHTS
    return w


def snapshots(ctx, rho, iters=SNAPSHOT_ITERS, tol_star=1e-12):
    """phi* and the CG iterates / residuals after k iterations, k in iters."""
    import torch
    n = ctx.n
    phi_star = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.solve(rho, phi_star, tol=tol_star, maxit=50 * ctx.N + 1000, precision=PREC_FP64)
    out = []
    for k in iters:
        xk = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.solve(rho, xk, tol=1e-300, maxit=k, precision=PREC_FP64, raise_on_error=False)
        rk = torch.empty_like(xk)
        ctx.residual(rho, xk, rk)
        out.append((rk, xk))
    return phi_star, out


def landau_snapshot_sets(N, seeds, ppc=8, iters=SNAPSHOT_ITERS):
    """Snapshot sets from the CIC deposits of Landau initial conditions."""
    import torch
    sets = []
    for seed in seeds:
        c = Context().init(N, ppc, seed)
        rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        c.deposit(rho)
        phi_star, snaps = snapshots(c, rho, iters)
        sets.append((rho, phi_star, snaps))
        c.close()
    return sets


def train(ctx, sets, steps, B=8, D=32, lr=2e-3, seed=0, weights=None, log_every=0, lr_final=None,
          validate=None, validate_every=0):
    """Adam on random crops of the snapshot sets; returns the loss history.

    ``ctx`` must be a context on the snapshots' grid (N^3); it holds the
    network. ``weights`` (14 688 FP32) initialises it, else the Jacobi start.
    With ``lr_final`` the step size follows a cosine from ``lr`` down to it.
    With ``validate`` (weights -> cost, e.g. flexible-CG iterations on a
    held-out right-hand side) the weights are scored every
    ``validate_every`` steps and at the end, and the best scored weights are
    loaded into ``ctx`` when training ends (the loss is only a proxy for
    the iteration count).
    """
    import torch
    N = ctx.N
    h2 = (ctx.L / N) ** 2
    ctx.cnn_set_weights(init_weights(seed) if weights is None else weights)
    rng = np.random.default_rng(seed + 1)
    m = B * D ** 3
    x = torch.empty(m, dtype=torch.float32, device="cuda")
    t = torch.empty_like(x)
    y = torch.empty_like(x)
    gy = torch.empty_like(x)
    losses = []
    best = None

    def score():
        nonlocal best
        w = ctx.cnn_get_weights()
        cost = validate(w)
        if best is None or cost < best[0]:
            best = (cost, w)

    for step in range(steps):
        rho, phi_star, snaps = sets[rng.integers(len(sets))]
        rk, xk = snaps[rng.integers(len(snaps))]
        origins = rng.integers(0, N, size=(B, 3)).astype(np.int32)
        ctx.cnn_make_batch(rk, phi_star, xk, origins, D, x, t, h2)
        ctx.cnn_forward(x, y, B, D)
        losses.append(ctx.cnn_loss(y, t, B, D, gy))
        ctx.cnn_backward(gy, B, D)
        step_lr = lr
        if lr_final is not None and steps > 1:
            step_lr = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * step / (steps - 1)))
        ctx.cnn_adam(step_lr)
        if log_every and (step + 1) % log_every == 0:
            print(f"step {step + 1}: loss {np.mean(losses[-log_every:]):.4f}", flush=True)
        if validate is not None and validate_every and (step + 1) % validate_every == 0 and step + 1 < steps:
            score()
    if validate is not None:
        score()
        ctx.cnn_set_weights(best[1])
    return np.array(losses)


def fcg_iterations(N=128, seed=21, tol=1e-10, maxit=2000):
    """Validation cost for ``train``: flexible-CG iterations of a solve of
    the CIC deposit of a seeded N^3 x 8 ppc Landau initial condition with
    the given weights (a held-out right-hand side: other seed and grid than
    the training snapshots)."""
    import torch
    c = Context().init(N, 8, seed)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")

    def cost(w):
        c.cnn_set_weights(w)
        phi.zero_()
        info = c.solve(rho, phi, tol=tol, maxit=maxit, precision=PREC_MIXED, precond=PC_CNN, raise_on_error=False)
        return info["iters"] if info["converged"] else maxit + 1
    return cost


def compare_preconditioners(ctx, rho, tol=1e-10, maxit=20000):
    """Cold-start solves of rho with FCG + network and with mixed Jacobi-CG
    (and the FP64 reference solve): iterations, device time, true relative residual."""
    import torch
    res = {}
    for name, prec, pc in (("fp64_jacobi", PREC_FP64, PC_JACOBI), ("mixed_jacobi", PREC_MIXED, PC_JACOBI),
                           ("mixed_fcg_cnn", PREC_MIXED, PC_CNN)):
        best = None
        for _ in range(2):
            phi = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
            info = ctx.solve(rho, phi, tol=tol, maxit=maxit, precision=prec, precond=pc)
            if best is None or info["t_ms"] < best["t_ms"]:
                best = info
        res[name] = best
    return res
