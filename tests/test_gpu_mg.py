"""GPU parity of the multigrid V-cycle preconditioner against the CPU oracle
(oracle/mg.py), and multigrid-preconditioned flexible-CG solves against the
exact discrete solution.

The GPU cycle works in the solver's scaled units (input r^ = h^2 r, the same
output); it runs in FP32, so one cycle matches the oracle's FP64 cycle to
FP32 accuracy (1e-5 relative). With the learned smoother on the finest level
the network runs as its composed kernel: FP32 on the CUDA cores for grids that
are not a multiple of 128 (compared here), BF16 on the tensor cores otherwise
(covered by the solve tests).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn  # noqa: E402
from oracle import mg  # noqa: E402
from oracle import pic as opic  # noqa: E402
from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("N", [8, 16, 32, 40, 48, 64, 72, 96, 128, 256])
def test_vcycle_matches_oracle(pg, N):
    """16^3 and below run entirely in the one-block kernel; 32^3, 64^3 and
    96^3 add plane-streamed full-grid levels (whole-plane blocks at 32^3,
    slabs with halo rows above); 48^3 coarsens 48 -> 24 -> 12 -> 6 -> 3 (odd
    coarsest); 40^3 has a 20^3 streamed level; 72^3 coarsens to 36^3 and then
    18^3, a size not a multiple of 4, which takes the per-cell kernels; 128^3
    and 256^3 have levels that take the z-marching kernels."""
    h = L / N
    r = np.random.default_rng(N).normal(size=N ** 3)
    r -= r.mean()
    c = pg.Context().init(N, 0, 0)
    rt = torch.from_numpy((h * h * r).astype(np.float32)).cuda()
    z = torch.full_like(rt, float("nan"))
    c.mg_apply(rt, z)
    ref = mg.vcycle(r, N, h)
    assert rel(z.cpu().numpy().astype(np.float64), ref) <= 1e-5


def test_vcycle_with_learned_smoother_matches_oracle(pg):
    N = 64
    h = L / N
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    ws32 = [w.astype(np.float32).astype(np.float64) for w in ws]
    r = np.random.default_rng(3).normal(size=N ** 3)
    r -= r.mean()
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    rt = torch.from_numpy((h * h * r).astype(np.float32)).cuda()
    z = torch.full_like(rt, float("nan"))
    c.mg_apply(rt, z, learned=True)

    def smoother(res):
        y, _ = ocnn.forward(res.reshape(N, N, N), ws32)
        return h * h * y.reshape(-1)
    ref = mg.vcycle(r, N, h, smoother=smoother)
    assert rel(z.cpu().numpy().astype(np.float64), ref) <= 1e-5


@pytest.mark.parametrize("N", [64, 128, 256])
def test_mg_fcg_reaches_the_exact_solution(pg, N, capsys):
    """Flexible CG with the V-cycle (Jacobi smoothing, and the learned
    smoother with the network's damped-Jacobi start) reaches rel-res 1e-10
    on the true FP64 residual and the exact discrete solution to 1e-9, in a
    number of iterations that does not grow with the grid."""
    from paper_2605_05469_gb300 import train as T
    h = L / N
    b = inputs.landau_noise_rhs(N, 7)
    exact = opic.spectral_solve_fft(b, N, h)
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(T.init_weights(0))
    its = {}
    for name, pc in (("mg", pg.PC_MG), ("mg_cnn", pg.PC_MG_CNN)):
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(torch.from_numpy(b).cuda(), phi, tol=1e-10, maxit=200, precision=pg.PREC_MIXED, precond=pc)
        assert info["converged"] and info["rel_res"] <= 1e-10, (name, info)
        assert rel(phi.cpu().numpy(), exact) <= 1e-9, name
        its[name] = info["iters"]
    with capsys.disabled():
        print(f"\nMG-FCG iterations at {N}^3: {its}")
    assert max(its.values()) <= 25, its


def test_mg_requires_mixed_precision_and_weights_for_the_learned_smoother(pg):
    c = pg.Context().init(32, 0, 0)
    rho = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rho)
    with pytest.raises(RuntimeError):
        c.solve(rho, phi, tol=1e-10, maxit=10, precision=pg.PREC_FP64, precond=pg.PC_MG)
    with pytest.raises(RuntimeError):
        c.solve(rho, phi, tol=1e-10, maxit=10, precision=pg.PREC_MIXED, precond=pg.PC_MG_CNN)
