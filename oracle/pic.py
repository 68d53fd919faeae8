"""Plain FP64 CPU restatement of the PIC loop for Landau damping.

Test infrastructure only (see ``oracle/__init__.py``). Every function follows
the paper's statement of the problem; the numbered "readings" below are the
places where the paper is silent and a choice had to be made.

Units and conventions (Sec. 2, Eqs. 1-4): electrons with q/m = -1, eps0 = 1,
mean electron density 1, so the neutralising ion background is rho_i = +1.
Uniform periodic node grid x_i = i*h, h = L/N, i = 0..N-1 (reading: node
centred), linear index i + N*(j + N*k) (x fastest). Each macro-particle
carries charge q_p = -L^3/Np.

Readings of the paper used here
  R1 initial density is the paper's product form (Sec. 2.1); the sum form
     1 + alpha sum_d cos(k x_d) (mode 1) is sampled by rejection.
  R2 CIC cell of a particle is floor(x/h); weights are the trilinear
     (cloud-in-cell) weights to the 8 nodes of that cell.
  R3 the Poisson operator is the 2nd-order central FD Laplacian (Sec. 3.2),
     here written as A = -Delta_h so that A phi = rho is SPD on mean-zero
     vectors; the right-hand side is projected to mean zero and the solution
     is returned with mean zero (the periodic null space is the constants).
  R4 Jacobi-PCG stops when ||r_k||_2 <= tol * ||b||_2, r_k the CG residual.
  R5 E = -grad(phi) by 2nd-order central differences at nodes.
  R6 leapfrog is kick-drift-kick; the two half-kicks that meet at a step
     boundary are applied as one full kick (see ``push``).
  R7 field energy W_d = h^3 * sum_i E_{d,i}^2 (no factor 1/2).
"""
import numpy as np

from . import philox

QM = -1.0  # electron charge-to-mass ratio in plasma units


# ----------------------------------------------------------------------------
# S0: initial condition (Sec. 2.1, Landau damping)
# ----------------------------------------------------------------------------
def inverse_cdf(u, L, alpha, k, newton_steps=12):
    """x in [0, L) with F(x) = u, F(x) = (x + (alpha/k) sin(k x)) / L.

    F is the CDF of the 1-D marginal (1 + alpha cos(k x)) / L of the paper's
    separable initial density (Sec. 2.1). Newton's method from x0 = u L;
    F is strictly increasing for alpha < 1, so the iteration converges.
    """
    x = u * L
    for _ in range(newton_steps):
        f = (x + (alpha / k) * np.sin(k * x)) / L - u
        fp = (1.0 + alpha * np.cos(k * x)) / L
        x = x - f / fp
    return x


# trials of the rejection sampling of the sum-form density (init_mode 1)
SUM_FORM_TRIALS = 32


def sum_form_positions(p, seed, L, alpha, k, trials=SUM_FORM_TRIALS):
    """Positions drawn from the sum-form density (1 + alpha sum_d cos(k x_d))/L^3
    by rejection from the uniform density on [0, L)^3 (reading 1's sum form).

    Trial t of particle p uses Philox calls 4 + 2t -> (u_x, u_y) and
    5 + 2t -> (u_z, u_accept) of the particle's stream; the proposal
    x = u L is accepted when u_accept (1 + 3 alpha) <= 1 + alpha sum cos(k x_d)
    (the density's maximum over the box is 1 + 3 alpha). The first accepted
    trial is kept; if none of the trials is accepted (probability below
    (3 alpha / (1 + 3 alpha))^trials) the last proposal is kept.
    """
    p = np.asarray(p, dtype=np.uint64)
    pos = np.empty((3, p.size))
    done = np.zeros(p.size, dtype=bool)
    for t in range(trials):
        U = philox.particle_uniforms_calls(p, seed, (4 + 2 * t, 5 + 2 * t))
        prop = np.stack([U[0, 0], U[0, 1], U[1, 0]]) * L
        dens = 1.0 + alpha * np.cos(k * prop).sum(axis=0)
        acc = U[1, 1] * (1.0 + 3.0 * alpha) <= dens
        take = ~done & (acc | (t == trials - 1))
        pos[:, take] = prop[:, take]
        done |= take
        if done.all():
            break
    return pos


def init_particles(N, ppc, seed, alpha=0.05, k=0.5, vth=1.0, mode=0):
    """Particles of the Landau initial condition (Sec. 2.1).

    mode 0 (the paper's product form): f(x, v, 0) = (2 pi)^(-3/2) exp(-|v|^2/2)
    prod_d (1 + alpha cos(k x_d)) on [0, L]^3, L = 2 pi / k; positions by the
    per-dimension inverse CDF of the separable density. mode 1 (the sum form
    1 + alpha sum_d cos(k x_d)): positions by rejection (sum_form_positions).
    Velocities: Box-Muller normals times v_th. Particle p draws from the
    Philox stream described in ``oracle/philox.py``. Returns
    (pos[3, Np], vel[3, Np]) as FP64 arrays.
    """
    L = 2.0 * np.pi / k
    Np = ppc * N ** 3
    p = np.arange(Np, dtype=np.uint64)
    U = philox.particle_uniforms(p, seed)
    pos = np.empty((3, Np))
    if mode == 1:
        pos[:] = sum_form_positions(p, seed, L, alpha, k)
    else:
        pos[0] = inverse_cdf(U[0, 0], L, alpha, k)
        pos[1] = inverse_cdf(U[0, 1], L, alpha, k)
        pos[2] = inverse_cdf(U[1, 0], L, alpha, k)
    vel = np.empty((3, Np))
    vel[0], vel[1] = philox.box_muller(U[2, 0], U[2, 1])
    vel[2], _ = philox.box_muller(U[3, 0], U[3, 1])
    return pos, vth * vel


# ----------------------------------------------------------------------------
# S2: CIC scatter (Sec. 2 and Fig. 1, "scatter"; rho = rho_e + rho_i, Eq. 2)
# ----------------------------------------------------------------------------
def cic_cell_and_weights(pos, N, L):
    """Cell index (3, Np) and the fractional offsets (3, Np) of each particle."""
    h = L / N
    s = pos / h
    cell = np.floor(s).astype(np.int64)
    cell = np.minimum(cell, N - 1)       # x < L always; guards round-up to N
    frac = s - cell
    return cell, frac


def deposit(pos, N, L, q_p=None):
    """rho at nodes: +1 (ion background) + sum_p q_p W(x_i - x_p) / h^3.

    W is the cloud-in-cell (trilinear) weight. Particles are accumulated
    in index order (np.bincount runs sequentially). With equal charges
    q_p = -L^3/Np, the background is exactly -sum_p q_p / L^3 = +1.
    """
    Np = pos.shape[1]
    h = L / N
    if q_p is None:
        q_p = -(L ** 3) / Np
    cell, f = cic_cell_and_weights(pos, N, L)
    rho = np.zeros(N ** 3)
    for dz in (0, 1):
        wz = f[2] if dz else 1.0 - f[2]
        kz = (cell[2] + dz) % N
        for dy in (0, 1):
            wy = f[1] if dy else 1.0 - f[1]
            jy = (cell[1] + dy) % N
            for dx in (0, 1):
                wx = f[0] if dx else 1.0 - f[0]
                ix = (cell[0] + dx) % N
                idx = ix + N * (jy + N * kz)
                rho += np.bincount(idx, weights=wx * wy * wz, minlength=N ** 3)
    rho *= q_p / h ** 3
    rho += -q_p * Np / L ** 3
    return rho


# ----------------------------------------------------------------------------
# S3: the operator A = -Delta_h (Sec. 3.2, 2nd-order central differences)
# ----------------------------------------------------------------------------
def apply_A(phi, N, h):
    """(A phi)_i = (6 phi_i - sum of the 6 periodic neighbours) / h^2."""
    g = phi.reshape(N, N, N)   # [k][j][i]
    out = 6.0 * g
    for ax in range(3):
        out = out - np.roll(g, 1, axis=ax) - np.roll(g, -1, axis=ax)
    return (out / h ** 2).reshape(-1)


def laplacian_eigenvalue(m, N, h):
    """Eigenvalue of A for Fourier mode m = (mx, my, mz): (4/h^2) sum sin^2(pi m_d / N)."""
    return (4.0 / h ** 2) * sum(np.sin(np.pi * md / N) ** 2 for md in m)


# ----------------------------------------------------------------------------
# S4: Jacobi-preconditioned CG (Sec. 3.2); warm start (Sec. 4.1)
# ----------------------------------------------------------------------------
def pcg_jacobi(b, x0, N, h, tol, maxit):
    """Textbook Jacobi-PCG (Hestenes-Stiefel) on A x = b - mean(b).

    Preconditioner M = diag(A) = 6/h^2 (Sec. 3.2 lists Jacobi). x0 is the
    warm start (Sec. 4.1: previous step's solution). Stops when
    ||r||_2 <= tol ||b||_2 (reading R4). Returns (x with mean zero, iters,
    rel_res of the recursive residual, converged flag).
    """
    b = b - b.mean()
    x = x0 - x0.mean()
    dinv = h ** 2 / 6.0
    bnorm = np.sqrt(b @ b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    r = b - apply_A(x, N, h)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.sqrt(r @ r) / bnorm
    while rel > tol and it < maxit:
        q = apply_A(p, N, h)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        rel = np.sqrt(r @ r) / bnorm
    return x - x.mean(), it, rel, rel <= tol


def dft_matrix(N, sign):
    n = np.arange(N)
    return np.exp(sign * 2j * np.pi * np.outer(n, n) / N)


def spectral_solve(b, N, h):
    """Exact discrete solution of A phi = b - mean(b), mean(phi) = 0.

    Brute force: the separable 3-D DFT written out as three multiplications
    by the N x N DFT matrix (O(N^4)), division by the eigenvalue
    lambda_m = (4/h^2) sum_d sin^2(pi m_d/N), zero mode set to 0, and the
    inverse DFT. Meant for N <= 32.
    """
    g = (b - b.mean()).reshape(N, N, N).astype(np.complex128)
    F = dft_matrix(N, -1.0)
    Fi = dft_matrix(N, +1.0) / N
    g = np.einsum("ai,kji->kja", F, g)
    g = np.einsum("aj,kji->kai", F, g)
    g = np.einsum("ak,kji->aji", F, g)
    m = np.arange(N)
    s2 = np.sin(np.pi * m / N) ** 2
    lam = (4.0 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    lam[0, 0, 0] = 1.0
    g = g / lam
    g[0, 0, 0] = 0.0
    g = np.einsum("ai,kji->kja", Fi, g)
    g = np.einsum("aj,kji->kai", Fi, g)
    g = np.einsum("ak,kji->aji", Fi, g)
    return g.real.reshape(-1)


def spectral_solve_fft(b, N, h):
    """The same exact discrete solution as spectral_solve, with the 3-D DFT
    done by numpy's FFT (a library primitive) so that it reaches 256^3:
    phi_hat(m) = b_hat(m) / lambda_m, lambda_m = (4/h^2) sum_d sin^2(pi m_d/N),
    zero mode set to 0 (mean(phi) = 0)."""
    g = np.fft.fftn((b - b.mean()).reshape(N, N, N))
    m = np.arange(N)
    s2 = np.sin(np.pi * m / N) ** 2
    lam = (4.0 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    lam[0, 0, 0] = 1.0
    g /= lam
    g[0, 0, 0] = 0.0
    return np.fft.ifftn(g).real.reshape(-1)


# ----------------------------------------------------------------------------
# S5: E = -grad(phi) (Eq. 2), central differences (reading R5)
# ----------------------------------------------------------------------------
def gradient(phi, N, h):
    """E[d] at nodes, d = x, y, z: -(phi_{i+e_d} - phi_{i-e_d}) / (2h)."""
    g = phi.reshape(N, N, N)
    E = np.empty((3, N ** 3))
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        E[d] = (-(np.roll(g, -1, axis=ax) - np.roll(g, 1, axis=ax)) / (2.0 * h)).reshape(-1)
    return E


# ----------------------------------------------------------------------------
# S6: CIC gather (Fig. 1, "gather") and leapfrog push (Eqs. 3-4)
# ----------------------------------------------------------------------------
def gather(E, pos, N, L):
    """E at particles: sum over the 8 nodes of the CIC cell of weight * E_node."""
    cell, f = cic_cell_and_weights(pos, N, L)
    Ep = np.zeros((3, pos.shape[1]))
    for dz in (0, 1):
        wz = f[2] if dz else 1.0 - f[2]
        kz = (cell[2] + dz) % N
        for dy in (0, 1):
            wy = f[1] if dy else 1.0 - f[1]
            jy = (cell[1] + dy) % N
            for dx in (0, 1):
                wx = f[0] if dx else 1.0 - f[0]
                ix = (cell[0] + dx) % N
                idx = ix + N * (jy + N * kz)
                Ep += (wx * wy * wz) * E[:, idx]
    return Ep


def wrap(x, L):
    """Periodic wrap into [0, L): x >= L -> x - L, x < 0 -> x + L, result L -> 0."""
    x = np.where(x >= L, x - L, x)
    x = np.where(x < 0.0, x + L, x)
    return np.where(x >= L, 0.0, x)


def push(pos, vel, Ep, dt, L, kick):
    """One leapfrog step with the force of Eq. 4 (E_ext = 0, B_ext = 0).

    Kick-drift-kick with the two half-kicks that meet at a step boundary
    merged into one full kick (reading R6): v <- v + (q/m) * kick * E(x),
    then x <- wrap(x + dt v). ``kick`` is dt/2 on the first step (velocities
    synchronous with positions) and dt afterwards (velocities half a step
    behind). ``sync_velocity`` applies the closing half-kick.
    """
    vel = vel + QM * kick * Ep
    pos = wrap(pos + dt * vel, L)
    return pos, vel


def sync_velocity(vel, Ep, dt):
    """Closing half-kick v^n = v^(n-1/2) + (q/m)(dt/2) E^n(x^n)."""
    return vel + QM * 0.5 * dt * Ep


# ----------------------------------------------------------------------------
# S7: field energy (Fig. 2 diagnostic)
# ----------------------------------------------------------------------------
def field_energy(phi, N, h):
    """(W_x, W_y, W_z), W_d = h^3 sum_i E_{d,i}^2 (reading R7)."""
    E = gradient(phi, N, h)
    return h ** 3 * np.sum(E * E, axis=1)


# ----------------------------------------------------------------------------
# The PIC loop (Fig. 1): scatter -> solve -> gather -> push
# ----------------------------------------------------------------------------
def pic_run(N, ppc, seed, steps, dt=0.05, tol=1e-10, maxit=5000, alpha=0.05, k=0.5,
            record=None):
    """Run ``steps`` PIC steps from the Landau initial condition.

    Each step: deposit rho(x^n), solve A phi^n = rho (warm start from the
    previous phi), then kick with E^n = -grad phi^n and drift. Returns
    (pos, vel, phi, energies[steps, 3], iters[steps]); ``energies[n]`` is the
    field energy at time n*dt (before the n-th push). ``record`` (callable)
    receives (n, pos, vel, phi) after each solve when given.
    """
    L = 2.0 * np.pi / k
    h = L / N
    pos, vel = init_particles(N, ppc, seed, alpha, k)
    phi = np.zeros(N ** 3)
    energies = np.zeros((steps, 3))
    iters = np.zeros(steps, dtype=np.int64)
    for n in range(steps):
        rho = deposit(pos, N, L)
        phi, it, _, _ = pcg_jacobi(rho, phi, N, h, tol, maxit)
        iters[n] = it
        energies[n] = field_energy(phi, N, h)
        if record is not None:
            record(n, pos, vel, phi)
        Ep = gather(gradient(phi, N, h), pos, N, L)
        pos, vel = push(pos, vel, Ep, dt, L, kick=(0.5 * dt if n == 0 else dt))
    return pos, vel, phi, energies, iters
