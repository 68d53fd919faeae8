"""Pins of the CPU oracle (oracle/pic.py, oracle/philox.py) against facts fixed
independently of it: published known-answer vectors, closed forms of the
discrete operators, invariants of CIC, exact leapfrog trajectories, a library
FFT, brute-force loops on tiny inputs, and the linear Landau damping rate.
"""
import os

import numpy as np
import pytest

from oracle import philox, pic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
K = 0.5
L = 2.0 * np.pi / K


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in _read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniforms_open_interval_and_moments():
    U = philox.particle_uniforms(np.arange(200_000, dtype=np.uint64), 0x5EED)
    assert U.min() > 0.0 and U.max() < 1.0
    n = U.shape[2]
    for j in range(4):
        for s in range(2):
            assert abs(U[j, s].mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    # distinct calls are distinct streams
    assert abs(np.corrcoef(U[0, 0], U[2, 0])[0, 1]) < 5 / np.sqrt(n)


def test_box_muller_moments():
    U = philox.particle_uniforms(np.arange(200_000, dtype=np.uint64), 7)
    g1, g2 = philox.box_muller(U[2, 0], U[2, 1])
    n = g1.size
    for g in (g1, g2):
        assert abs(g.mean()) < 5 / np.sqrt(n)
        assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert abs(np.mean(g ** 4) - 3.0) < 0.1


# ---------------------------------------------------------------- S0 init
def test_inverse_cdf_solves_cdf_equation():
    u = np.linspace(1e-9, 1 - 1e-9, 10001)
    x = pic.inverse_cdf(u, L, 0.05, K)
    F = (x + (0.05 / K) * np.sin(K * x)) / L
    assert np.max(np.abs(F - u)) < 1e-14
    assert np.all(np.diff(x) > 0) and x.min() >= 0.0 and x.max() < L


def test_inverse_cdf_alpha_zero_is_uniform():
    u = np.random.default_rng(1).random(1000)
    assert np.allclose(pic.inverse_cdf(u, L, 0.0, K), u * L, rtol=0, atol=1e-15)


def test_init_marginal_cosine_moment():
    # E[cos(k x)] under (1 + a cos kx)/L on [0, L) equals a/2.
    pos, vel = pic.init_particles(16, 8, 0x5EED)
    n = pos.shape[1]
    for d in range(3):
        assert abs(np.mean(np.cos(K * pos[d])) - 0.025) < 5 * np.sqrt(0.5 / n)
        assert abs(vel[d].mean()) < 5 / np.sqrt(n)
        assert abs(vel[d].var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert pos.min() >= 0.0 and pos.max() < L


# ---------------------------------------------------------------- S2 deposit
def test_deposit_charge_conservation_and_mean():
    N = 8
    rng = np.random.default_rng(3)
    pos = rng.random((3, 5000)) * L
    rho = pic.deposit(pos, N, L)
    h = L / N
    # sum of electron charge on the grid equals sum_p q_p = -L^3
    assert np.isclose(np.sum(rho - 1.0) * h ** 3, -L ** 3, rtol=1e-13)
    assert abs(rho.mean()) < 1e-13


def test_deposit_node_and_centre_special_cases():
    N = 8
    h = L / N
    # one particle exactly on node (2, 3, 4): everything there
    pos = np.array([[2 * h], [3 * h], [4 * h]])
    rho = pic.deposit(pos, N, L, q_p=1.0)
    e = rho + 1.0 / L ** 3  # remove the background -q_p*Np/L^3
    idx = 2 + N * (3 + N * 4)
    assert np.isclose(e[idx], 1.0 / h ** 3, rtol=1e-12)
    assert np.allclose(np.delete(e, idx), 0.0, atol=1e-12 / h ** 3)
    # one particle at the centre of cell (7, 7, 7): 1/8 on each corner, with wrap
    pos = np.array([[7.5 * h], [7.5 * h], [7.5 * h]])
    e = pic.deposit(pos, N, L, q_p=1.0) + 1.0 / L ** 3
    for i in (7, 0):
        for j in (7, 0):
            for k in (7, 0):
                assert np.isclose(e[i + N * (j + N * k)], 0.125 / h ** 3, rtol=1e-12)
    assert np.isclose(e.sum(), 1.0 / h ** 3, rtol=1e-12)


def test_deposit_uniform_lattice_is_neutral():
    N = 6
    h = L / N
    g = (np.arange(2 * N) + 0.5) * (h / 2)   # 2 particles per cell per dimension
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    rho = pic.deposit(pos, N, L)
    assert np.max(np.abs(rho)) < 1e-13


def test_deposit_brute_force_loop():
    N = 4
    h = L / N
    rng = np.random.default_rng(5)
    pos = rng.random((3, 7)) * L
    q = -(L ** 3) / 7
    ref = np.full(N ** 3, 1.0)
    for p in range(7):
        c = [int(np.floor(pos[d, p] / h)) for d in range(3)]
        f = [pos[d, p] / h - c[d] for d in range(3)]
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                    idx = (c[0] + dx) % N + N * ((c[1] + dy) % N + N * ((c[2] + dz) % N))
                    ref[idx] += q * w / h ** 3
    assert np.allclose(pic.deposit(pos, N, L), ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- S3/S4 solve
def _mode(N, m):
    i = np.arange(N)
    Kz, Jy, Ix = np.meshgrid(i, i, i, indexing="ij")
    return np.cos(2 * np.pi * (m[0] * Ix + m[1] * Jy + m[2] * Kz) / N).ravel()


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (3, 1, 5)])
def test_operator_eigenmode_closed_form(m):
    N = 8
    h = L / N
    b = _mode(N, m)
    lam = pic.laplacian_eigenvalue(m, N, h)
    assert np.allclose(pic.apply_A(b, N, h), lam * b, rtol=0, atol=1e-12 * lam)
    phi = pic.spectral_solve(b, N, h)
    assert np.allclose(phi, b / lam, rtol=0, atol=1e-13)


def test_operator_axes_not_transposed():
    # a mode along x only: the operator must see the x-stride (stride 1)
    N = 8
    h = L / N
    i = np.arange(N ** 3)
    b = np.cos(2 * np.pi * (i % N) / N)
    lam = pic.laplacian_eigenvalue((1, 0, 0), N, h)
    assert np.allclose(pic.apply_A(b, N, h), lam * b, atol=1e-12 * lam)


def test_spectral_solve_matches_numpy_fft():
    N = 12
    h = L / N
    b = np.random.default_rng(2).normal(size=N ** 3)
    m = np.arange(N)
    s2 = np.sin(np.pi * m / N) ** 2
    lam = (4 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    lam[0, 0, 0] = 1.0
    B = np.fft.fftn((b - b.mean()).reshape(N, N, N)) / lam
    B[0, 0, 0] = 0.0
    ref = np.fft.ifftn(B).real.ravel()
    assert np.allclose(pic.spectral_solve(b, N, h), ref, atol=1e-14 * np.abs(ref).max())


def test_fft_spectral_solve_matches_the_brute_force_dft_and_the_operator():
    """spectral_solve_fft (numpy FFT) against the brute-force DFT form at 16^3
    (independent transform), against the operator itself at 64^3 (A phi =
    b - mean(b), mean(phi) = 0), and on a single Fourier mode, where the exact
    solution is the mode divided by its closed-form eigenvalue."""
    N = 16
    h = L / N
    b = np.random.default_rng(7).normal(size=N ** 3) + 1.5
    ref = pic.spectral_solve(b, N, h)
    assert np.allclose(pic.spectral_solve_fft(b, N, h), ref, atol=1e-13 * np.abs(ref).max())
    N = 64
    h = L / N
    b = np.random.default_rng(8).normal(size=N ** 3)
    phi = pic.spectral_solve_fft(b, N, h)
    bp = b - b.mean()
    assert np.linalg.norm(pic.apply_A(phi, N, h) - bp) <= 1e-12 * np.linalg.norm(bp)
    assert abs(phi.mean()) <= 1e-15 * np.abs(phi).max()
    i = np.arange(N ** 3)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    mode = np.cos(2 * np.pi * (3 * x + 5 * z) / N)
    lam = pic.laplacian_eigenvalue((3, 0, 5), N, h)
    assert np.allclose(pic.spectral_solve_fft(mode, N, h), mode / lam, atol=1e-13 / lam)


@pytest.mark.parametrize("N", [8, 16, 12])
def test_pcg_matches_exact_discrete_solution(N):
    h = L / N
    b = np.random.default_rng(N).normal(size=N ** 3) + 3.0   # nonzero mean is projected out
    x, it, rel, ok = pic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-14, 2000)
    ref = pic.spectral_solve(b, N, h)
    assert ok and rel <= 1e-14
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(x.mean()) < 1e-15 * np.abs(ref).max()
    # true residual of the mean-projected system
    r = (b - b.mean()) - pic.apply_A(x, N, h)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b - b.mean())


def test_pcg_warm_start_and_zero_rhs():
    N = 8
    h = L / N
    b = np.random.default_rng(0).normal(size=N ** 3)
    ref = pic.spectral_solve(b, N, h)
    x, it, rel, ok = pic.pcg_jacobi(b, ref, N, h, 1e-10, 100)
    assert ok and it == 0
    x, it, rel, ok = pic.pcg_jacobi(np.full(N ** 3, 2.5), np.zeros(N ** 3), N, h, 1e-10, 100)
    assert ok and it == 0 and np.all(x == 0.0)


def test_pcg_reports_non_convergence():
    N = 16
    h = L / N
    b = np.random.default_rng(0).normal(size=N ** 3)
    x, it, rel, ok = pic.pcg_jacobi(b, np.zeros(N ** 3), N, h, 1e-12, 5)
    assert not ok and it == 5 and rel > 1e-12


# ---------------------------------------------------------------- S5 gradient
@pytest.mark.parametrize("m", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 3, 1)])
def test_gradient_closed_form(m):
    N = 8
    h = L / N
    i = np.arange(N)
    Kz, Jy, Ix = np.meshgrid(i, i, i, indexing="ij")
    theta = (2 * np.pi / N) * (m[0] * Ix + m[1] * Jy + m[2] * Kz)
    E = pic.gradient(np.cos(theta).ravel(), N, h)
    for d in range(3):
        ref = (np.sin(2 * np.pi * m[d] / N) / h) * np.sin(theta).ravel()
        assert np.allclose(E[d], ref, atol=1e-13)


def test_field_energy_single_mode():
    N = 8
    h = L / N
    i = np.arange(N ** 3)
    theta = 2 * np.pi * (i % N) / N
    W = pic.field_energy(np.cos(theta), N, h)
    # sum over the grid of sin^2 = N^3 / 2
    ref = h ** 3 * (np.sin(2 * np.pi / N) / h) ** 2 * N ** 3 / 2
    assert np.isclose(W[0], ref, rtol=1e-13) and abs(W[1]) < 1e-25 and abs(W[2]) < 1e-25


# ---------------------------------------------------------------- S6 gather/push
def test_gather_constant_and_linear_fields():
    N = 8
    h = L / N
    rng = np.random.default_rng(4)
    pos = (1.0 + 4.0 * rng.random((3, 200))) * h     # inside cells 1..4: no wrap
    E = np.ones((3, N ** 3)) * np.array([[1.5], [-2.0], [0.25]])
    assert np.allclose(pic.gather(E, pos, N, L), E[:, :200], atol=1e-14)
    i = np.arange(N ** 3)
    xs = np.stack([(i % N) * h, ((i // N) % N) * h, (i // N ** 2) * h])
    lin = 0.3 + 0.7 * xs[0] - 0.2 * xs[1] + 0.1 * xs[2]
    Ep = pic.gather(np.stack([lin, 2 * lin, -lin]), pos, N, L)
    ref = 0.3 + 0.7 * pos[0] - 0.2 * pos[1] + 0.1 * pos[2]
    assert np.allclose(Ep[0], ref, atol=1e-13) and np.allclose(Ep[1], 2 * ref, atol=1e-13)


def test_wrap_edge_cases():
    x = np.array([L, -1e-300, L + 0.5, -0.5, 0.0, L * (1 - 1e-16)])
    w = pic.wrap(x, L)
    assert np.all(w >= 0.0) and np.all(w < L)
    assert w[0] == 0.0 and w[1] == 0.0
    assert np.isclose(w[2], 0.5) and np.isclose(w[3], L - 0.5)


def test_free_streaming_is_exact():
    rng = np.random.default_rng(8)
    pos = rng.random((3, 50)) * L
    vel = rng.normal(size=(3, 50))
    x, v = pos.copy(), vel.copy()
    for n in range(10):
        x, v = pic.push(x, v, np.zeros_like(x), 0.05, L, kick=0.025 if n == 0 else 0.05)
    assert np.array_equal(v, vel)
    ref = np.mod(pos + 0.5 * vel, L)
    d = np.abs(x - ref)
    assert np.all(np.minimum(d, L - d) < 1e-12)


def test_constant_field_parabola():
    # KDK with constant force is exact: x(t) = x0 + v0 t + a t^2 / 2, a = (q/m) E.
    pos = np.full((3, 1), 3.0)
    vel = np.array([[0.1], [-0.2], [0.05]])
    Ep = np.array([[0.4], [0.1], [-0.3]])
    a = pic.QM * Ep
    dt, n = 0.05, 20
    x, v = pos.copy(), vel.copy()
    for s in range(n):
        x, v = pic.push(x, v, Ep, dt, 1e9, kick=0.5 * dt if s == 0 else dt)
    v = pic.sync_velocity(v, Ep, dt)
    t = n * dt
    assert np.allclose(x, pos + vel * t + 0.5 * a * t * t, atol=1e-13)
    assert np.allclose(v, vel + a * t, atol=1e-14)


# ---------------------------------------------------------------- the paper's cases
def test_paper_case_sizes_are_8_ppc():
    for nx, ny, nz, npart in _read_golden("paper_cases.txt"):
        assert 8 * int(nx) * int(ny) * int(nz) == int(npart)


# ---------------------------------------------------------------- full loop
def test_landau_dispersion_root():
    from scipy.special import wofz
    g = dict((r[0], float(r[1])) for r in _read_golden("landau_linear.txt"))
    k = g["k"]

    def D(w):
        z = w / (np.sqrt(2.0) * k)
        return 1.0 + (1.0 + z * 1j * np.sqrt(np.pi) * wofz(z)) / k ** 2

    w = 1.4 - 0.15j
    for _ in range(60):
        d = 1e-7
        w = w - D(w) * d / (D(w + d) - D(w))
    assert abs(w.real - g["omega_r"]) < g["abs_tol"] and abs(w.imag - g["gamma"]) < g["abs_tol"]


@pytest.mark.slow
def test_landau_damping_rate_32cubed():
    """Fig. 2's check: the field oscillation damps at the analytic rate.

    32^3 grid, 8 ppc, dt = 0.05, 190 steps (t = 9.5). The amplitude of the
    three k = 0.5 Fourier modes of phi has peaks spaced pi/omega_r apart; a
    log-linear fit of the peaks before t = 8.5 gives the damping rate.
    """
    g = dict((r[0], float(r[1])) for r in _read_golden("landau_linear.txt"))
    N = 32
    amp = []

    def rec(n, pos, vel, phi):
        F = np.fft.fftn(phi.reshape(N, N, N))
        amp.append(abs(F[0, 0, 1]) + abs(F[0, 1, 0]) + abs(F[1, 0, 0]))

    pic.pic_run(N, 8, 0x5EED, 190, tol=1e-6, record=rec)
    a = np.array(amp)
    t = np.arange(a.size) * 0.05
    pk = [i for i in range(1, a.size - 1) if a[i] > a[i - 1] and a[i] >= a[i + 1] and t[i] < 8.5]
    assert len(pk) >= 3
    gamma = np.polyfit(t[pk], np.log(a[pk]), 1)[0]
    assert abs(gamma - g["gamma"]) < 0.1 * abs(g["gamma"])
    period = np.mean(np.diff(t[pk]))
    assert abs(period - np.pi / g["omega_r"]) < 0.1 * np.pi / g["omega_r"]


# ------------------------------------------------------ the sum-form initial density
def test_sum_form_density_moments():
    """Reading 1's sum form f ~ 1 + alpha sum_d cos(k x_d) against the product
    form prod_d (1 + alpha cos(k x_d)), by their moments over the box (alpha
    0.3 to resolve them with 2^18 particles): both have E[cos k x_d] = alpha/2;
    the sum form's E[cos k x cos k y] is 0, the product form's alpha^2/4;
    every position lies in [0, L). Tolerances are five standard errors."""
    N, ppc, alpha, k = 32, 8, 0.3, 0.5
    L = 2.0 * np.pi / k
    Np = ppc * N ** 3
    se = 1.0 / np.sqrt(Np)
    for mode, cc in ((1, 0.0), (0, alpha ** 2 / 4)):
        pos, vel = pic.init_particles(N, ppc, 0x5EED, alpha=alpha, k=k, mode=mode)
        assert np.all((pos >= 0.0) & (pos < L))
        c = np.cos(k * pos)
        for d in range(3):
            assert abs(c[d].mean() - alpha / 2) < 5 * 0.75 * se, (mode, d, c[d].mean())
        for a, b in ((0, 1), (1, 2), (0, 2)):
            assert abs((c[a] * c[b]).mean() - cc) < 5 * 0.6 * se, (mode, a, b, (c[a] * c[b]).mean())


def test_thermal_velocity_scales_the_maxwellian():
    pos1, vel1 = pic.init_particles(8, 8, 7)
    pos2, vel2 = pic.init_particles(8, 8, 7, vth=2.5)
    assert np.array_equal(pos1, pos2)
    assert np.array_equal(vel2, 2.5 * vel1)
    assert abs(vel2.std() - 2.5) < 0.05
