"""Solution error of the three solvers against the exact discrete solution at
the benchmark's sizes (256^3 and 512^3), per solver at its tolerance.

The exact solution of A phi = b - mean(b) comes from the oracle's FFT form of
the spectral solve (pinned in test_oracle_pic.py against the brute-force DFT,
the operator and single Fourier modes); the right-hand side is the seeded
Landau density + N(0, 0.01^2) noise of the solver-only workloads. The solvers
stop at ||b - A phi|| <= 1e-10 ||b|| (the FP64 reference solve on its recursive
residual, the mixed-precision solvers on the true FP64 residual), which bounds
the relative error by 1e-10 ||b|| / (lambda_min ||phi||); the measured errors
are asserted below the 1e-9 target.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pic as opic  # noqa: E402
from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


@pytest.mark.parametrize("N", [256, 512])
def test_solver_errors_against_exact_solution(pg, N, capsys):
    h = L / N
    b = inputs.landau_noise_rhs(N, 3)
    exact = opic.spectral_solve_fft(b, N, h)
    enorm = np.linalg.norm(exact)
    # the learned preconditioner, trained as the benchmark trains it
    c = pg.Context().init(N, 0, 0)
    c.cnn_train(pg.TRAIN_PRECONDITIONER)
    bt = torch.from_numpy(b).cuda()
    errs = {}
    for name, prec, pc in (("fp64_jacobi", pg.PREC_FP64, pg.PC_JACOBI), ("mixed_jacobi", pg.PREC_MIXED, pg.PC_JACOBI),
                           ("mixed_fcg_learned", pg.PREC_MIXED, pg.PC_CNN)):
        phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
        info = c.solve(bt, phi, tol=1e-10, maxit=20000, precision=prec, precond=pc)
        got = phi.cpu().numpy()
        errs[name] = (np.linalg.norm(got - exact) / enorm, info["iters"], info["rel_res"])
    with capsys.disabled():
        print(f"\nrel-L2 error vs exact discrete solution at {N}^3, tol 1e-10:",
              {k: (f"{e:.2e}", it) for k, (e, it, _) in errs.items()})
    for name, (e, it, rr) in errs.items():
        assert rr <= 1e-10, (name, rr)
        assert e <= 1e-9, (name, e)
