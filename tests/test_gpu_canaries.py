"""Guard-band canaries around every caller-owned output buffer (the bounds
check that stands in for compute-sanitizer, which this pool does not offer).

Each output is a view into a larger allocation with 4096-byte guard bands
before and after it, filled with a sentinel bit pattern; after the call the
bands must be unchanged, so a write outside the buffer fails the test
instead of corrupting memory silently. The 4096-byte offset keeps the views
as aligned as a fresh allocation. Sizes are ones the parity tests cover,
including grids that are not a multiple of the kernels' tiles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_05469_gb300 import inputs  # noqa: E402
from oracle import cnn as ocnn  # noqa: E402

pytestmark = pytest.mark.gpu

L = 4.0 * np.pi
GUARD_BYTES = 4096
SENTINEL = {torch.float64: -7.25e300, torch.float32: -3.125e37}


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


class Guarded:
    """A device buffer of n elements between two sentinel-filled guard bands."""

    def __init__(self, n, dtype, fill=0.0):
        self.g = GUARD_BYTES // torch.tensor([], dtype=dtype).element_size()
        self.n = n
        self.buf = torch.full((self.g + n + self.g,), SENTINEL[dtype], dtype=dtype, device="cuda")
        self.sentinel = self.buf[:1].clone()
        self.view = self.buf[self.g:self.g + n]
        self.view.fill_(fill)

    def intact(self):
        torch.cuda.synchronize()
        head = self.buf[:self.g]
        tail = self.buf[self.g + self.n:]
        return bool(torch.all(head == self.sentinel)) and bool(torch.all(tail == self.sentinel))


def test_deposit_and_particle_field_outputs(pg):
    N, ppc = 32, 2
    c = pg.Context().init(N, ppc, 7)
    rho = Guarded(N ** 3, torch.float64)
    c.deposit(rho.view)
    assert rho.intact()
    c.close()
    N, ppc = 16, 1
    c = pg.Context().init(N, ppc, 21)
    E = Guarded(3 * ppc * N ** 3, torch.float64)
    c.pif_field(E.view, tol=1e-4)
    assert E.intact()
    c.close()


@pytest.mark.parametrize("N,solver", [(24, "fp64"), (24, "mixed"), (64, "mg"), (64, "ssor")])
def test_solve_output(pg, N, solver):
    precision = pg.PREC_FP64 if solver == "fp64" else pg.PREC_MIXED
    precond = {"mg": pg.PC_MG, "ssor": pg.PC_SSOR}.get(solver, pg.PC_JACOBI)
    c = pg.Context().init(N, 0, 0)
    b = torch.from_numpy(inputs.noise_field(N, 5, mean=0.7)).cuda()
    phi = Guarded(N ** 3, torch.float64)
    info = c.solve(b, phi.view, tol=1e-10, maxit=5000, precision=precision, precond=precond)
    assert info["converged"]
    assert phi.intact()


def test_spectral_solve_outputs(pg):
    N = 24
    c = pg.Context().init(N, 0, 0)
    rho = torch.from_numpy(np.random.default_rng(4).normal(size=N ** 3)).cuda()
    phi = Guarded(N ** 3, torch.float64)
    E = Guarded(3 * N ** 3, torch.float64)
    c.fft_solve(rho, phi.view, E.view)
    assert phi.intact() and E.intact()


@pytest.mark.parametrize("N", [40, 128])
def test_operator_and_preconditioner_outputs(pg, N):
    h = L / N
    c = pg.Context().init(N, 0, 0)
    x = torch.from_numpy(np.random.default_rng(N).normal(size=N ** 3)).cuda()
    y = Guarded(N ** 3, torch.float64)
    c.apply_laplacian(x, y.view)
    assert y.intact()
    r = torch.from_numpy((h * h * np.random.default_rng(N + 1).normal(size=N ** 3)).astype(np.float32)).cuda()
    z = Guarded(N ** 3, torch.float32)
    c.mg_apply(r, z.view)
    assert z.intact()
    z = Guarded(N ** 3, torch.float32)
    c.ssor_apply(r, z.view)
    assert z.intact()


@pytest.mark.parametrize("N,mode", [(32, "fp32"), (128, "tc")])
def test_learned_preconditioner_output(pg, N, mode):
    ws = ocnn.init_weights(9)
    flat = np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)
    c = pg.Context().init(N, 0, 0)
    c.cnn_set_weights(flat)
    c.cnn_set_apply(pg.CNN_APPLY_TC if mode == "tc" else pg.CNN_APPLY_FP32)
    r = torch.from_numpy(inputs.noise_field(N, 3).astype(np.float32)).cuda()
    z = Guarded(N ** 3, torch.float32)
    c.cnn_apply(r, z.view)
    assert z.intact()
