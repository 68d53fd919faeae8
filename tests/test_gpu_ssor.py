"""GPU parity of the red-black SSOR preconditioner (the paper's PCG
configuration, Sec. 4.1) against the CPU oracle (oracle/ssor.py), and
SSOR-preconditioned flexible-CG solves against the exact discrete solution.

The GPU preconditioner works in FP32 on the scaled system (input r^ = h^2 r),
so one application matches the oracle's FP64 one to FP32 accuracy over its
32 half-sweeps (1e-5 relative)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn  # noqa: E402
from oracle import pic as opic  # noqa: E402
from oracle import ssor  # noqa: E402
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


@pytest.mark.parametrize("N", [8, 16, 24, 40, 64, 128])
def test_ssor_matches_oracle(pg, N):
    """128^3 takes the z-marching half-sweeps."""
    h = L / N
    r = np.random.default_rng(N).normal(size=N ** 3)
    c = pg.Context().init(N, 0, 0)
    rt = torch.from_numpy((h * h * r).astype(np.float32)).cuda()
    z = torch.full_like(rt, float("nan"))
    c.ssor_apply(rt, z)
    ref = ssor.ssor(r, N, h)
    assert rel(z.cpu().numpy().astype(np.float64), ref) <= 1e-5
    # r is not modified
    assert np.array_equal(rt.cpu().numpy(), (h * h * r).astype(np.float32))


@pytest.mark.parametrize("N", [64, 128])
def test_ssor_fcg_reaches_the_exact_solution(pg, N, capsys):
    h = L / N
    b = inputs.landau_noise_rhs(N, 9)
    exact = opic.spectral_solve_fft(b, N, h)
    c = pg.Context().init(N, 0, 0)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    info = c.solve(torch.from_numpy(b).cuda(), phi, tol=1e-10, maxit=1000, precision=pg.PREC_MIXED,
                   precond=pg.PC_SSOR)
    assert info["converged"] and info["rel_res"] <= 1e-10, info
    assert rel(phi.cpu().numpy(), exact) <= 1e-9
    with capsys.disabled():
        print(f"\nSSOR-FCG iterations at {N}^3: {info['iters']}")
    if N == 64:
        # the oracle's flexible CG with its FP64 SSOR on the same right-hand side
        _, it, _, _ = ocnn.fcg(b, np.zeros(N ** 3), N, h, 1e-10, 500, lambda r: ssor.ssor(r, N, h))
        assert abs(info["iters"] - it) <= max(2, it // 5), (info["iters"], it)


def test_ssor_requires_mixed_precision(pg):
    c = pg.Context().init(32, 0, 0)
    rho = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rho)
    with pytest.raises(RuntimeError):
        c.solve(rho, phi, tol=1e-10, maxit=10, precision=pg.PREC_FP64, precond=pg.PC_SSOR)
