"""Failure detection without a GPU fault: every failure is made on the host
or by a device wait that runs out on purpose (no copy in flight), and the
library must report it through its return codes while the process and the
GPU stay usable.

* Bounded waits: the library's mbarrier wait (the one the streaming solver
  kernels and the tensor-core preconditioner use) run out in the self-test
  entry point with a 20 us budget and no producer: PIC_ETIMEOUT, recorded by
  the context (its next solve fails too); a fresh context works.
* The learned preconditioner's descent guard: all-zero weights give z = 0,
  so (r, z) = 0 in every iteration and flexible CG must take the Jacobi
  direction every time, converging like Jacobi-CG.
* Non-finite input to the push: a non-finite dt is rejected on the host; an
  infinite or NaN potential leaves the particles it reaches unchanged (in
  the box, finite), and the next synchronising call reports PIC_EBREAKDOWN.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_05469_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def test_bounded_wait_runs_out_and_is_reported(pg):
    c = pg.Context().init(16, 0, 0)
    assert c.selftest_bounded_wait(1_000_000, True) == pg.PIC_OK
    assert c.selftest_bounded_wait(0, False) == pg.PIC_EINVAL
    assert c.selftest_bounded_wait(3_000_000_000, False) == pg.PIC_EINVAL
    assert c.selftest_bounded_wait(20_000, False) == pg.PIC_ETIMEOUT
    # the context keeps the expired wait recorded
    rho = torch.from_numpy(inputs.landau_noise_rhs(16, 1)).cuda()
    phi = torch.zeros_like(rho)
    info = c.solve(rho, phi, tol=1e-10, maxit=500, raise_on_error=False)
    assert info["code"] == pg.PIC_ETIMEOUT
    c.close()
    # a fresh context solves normally
    c2 = pg.Context().init(16, 0, 0)
    info = c2.solve(rho, phi.zero_(), tol=1e-10, maxit=500)
    assert info["converged"]
    c2.close()


@pytest.mark.parametrize("N", [64, 128])
def test_zero_weights_take_the_jacobi_direction_every_iteration(pg, N):
    """64^3: the FP32 composed kernel; 128^3: the tensor-core kernel."""
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(np.zeros(pg.CNN_WEIGHTS, dtype=np.float32))
    rho = torch.from_numpy(inputs.landau_noise_rhs(N, 3)).cuda()
    phi = torch.zeros_like(rho)
    info = c.solve(rho, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, precond=pg.PC_CNN)
    assert info["converged"] and info["rel_res"] <= 1e-10
    assert info["iters"] <= info["fallbacks"] <= info["iters"] + 1, info
    jac = c.solve(rho, phi.zero_(), tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, precond=pg.PC_JACOBI)
    assert abs(info["iters"] - jac["iters"]) <= 0.1 * jac["iters"], (info["iters"], jac["iters"])
    c.close()


@pytest.mark.parametrize("bad", [np.inf, -np.inf, np.nan])
def test_non_finite_potential_in_the_push_is_reported(pg, bad):
    N, ppc = 16, 2
    n = N ** 3
    c = pg.Context().init(N, ppc, 5)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    phi = torch.zeros_like(rho)
    c.solve(rho, phi, tol=1e-10, maxit=500)
    with pytest.raises(pg.PicError) as e:
        c.gather_push(phi, float("inf"))
    assert e.value.code == pg.PIC_EINVAL
    with pytest.raises(pg.PicError) as e:
        c.gather_push(phi, float("nan"))
    assert e.value.code == pg.PIC_EINVAL
    before, _ = c.particles()
    bad_phi = phi.clone()
    bad_phi[n // 2 + N // 2 + 3] = bad
    c.gather_push(bad_phi, 0.05)       # enqueued; the fault is found on the device
    with pytest.raises(pg.PicError) as e:
        c.field_energy(phi)
    assert e.value.code == pg.PIC_EBREAKDOWN
    after, _ = c.particles()
    assert np.all(np.isfinite(after))
    assert np.all((after[:3] >= 0.0) & (after[:3] < L))
    # the particles next to the bad node kept their state; the others moved
    moved = np.any(after != before, axis=0)
    assert 0 < np.count_nonzero(~moved) < after.shape[1] // 4
    assert np.count_nonzero(moved) > after.shape[1] // 2
    c.close()
    c2 = pg.Context().init(N, ppc, 5)
    c2.deposit(rho)
    c2.solve(rho, phi.zero_(), tol=1e-10, maxit=500)
    c2.gather_push(phi, 0.05)
    assert np.all(np.isfinite(c2.field_energy(phi)))
    c2.close()
