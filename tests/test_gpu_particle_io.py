"""pic_set_particles / pic_get_particles: the particle state in and out of the
context through the C ABI, from and to device and host memory (the host path
converts and copies in chunks of 2^24 particles), against the oracle's push
of the same caller-given state.

Tolerances: velocities that came out of the context round-trip exactly
(double-float -> FP64 -> double-float), others keep 48 significant bits;
positions within 1e-15 L (the fixed-point offset keeps 53 bits of a cell);
one push of a caller-given state matches the oracle's to 1e-12 (the
particle parity tolerance of the PIC tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pic as opic  # noqa: E402

pytestmark = pytest.mark.gpu

K = 0.5
L = 2.0 * np.pi / K


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def test_round_trip_host_and_device(pg):
    N, ppc = 16, 2
    c = pg.Context().init(N, ppc, 7)
    np_ = c.num_particles
    ref, half0 = c.particles()
    # device -> device
    d = torch.from_numpy(ref.reshape(-1).copy()).cuda()
    c.set_particles(d, half0)
    got, half = c.particles()
    assert half == half0
    assert np.max(np.abs(got[:3] - ref[:3])) <= 1e-15 * L
    assert np.array_equal(got[3:], ref[3:])
    # host (pageable and pinned) -> host
    for pin in (False, True):
        h = torch.from_numpy(ref.reshape(-1).copy())
        if pin:
            h = h.pin_memory()
        c.set_particles(h, True)
        out = torch.empty(6 * np_, dtype=torch.float64)
        assert c.particles_to_host(out) is True
        o = out.numpy().reshape(6, np_)
        assert np.max(np.abs(o[:3] - ref[:3])) <= 1e-15 * L
        assert np.array_equal(o[3:], ref[3:])
    c.close()


def test_caller_state_is_wrapped_and_pushed_like_the_oracle(pg):
    """Positions anywhere on the real line are wrapped into [0, L); one push
    with a solved field then matches the oracle's push of the same state."""
    N, ppc = 16, 2
    c = pg.Context().init(N, ppc, 3)
    np_ = c.num_particles
    rng = np.random.default_rng(5)
    pos = rng.uniform(-3 * L, 4 * L, size=(3, np_))
    vel = rng.normal(size=(3, np_))
    c.set_particles(np.concatenate([pos, vel]), False)
    got, half = c.particles()
    assert half is False
    wrapped = np.mod(pos, L)  # the periodic image in [0, L)
    d = np.abs(got[:3] - wrapped)
    d = np.minimum(d, L - d)  # a wrapped value may land on either side of 0 == L
    assert np.max(d) <= 1e-12
    # velocities are kept as double-float pairs (two 24-bit significands)
    assert np.max(np.abs(got[3:] - vel) / np.maximum(np.abs(vel), 1e-300)) <= 2.0 ** -46
    # deposit, solve, push from this state against the oracle
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    rho_ref = opic.deposit(got[:3], N, L)
    torch.cuda.synchronize()
    assert np.max(np.abs(rho.cpu().numpy() - rho_ref)) <= 1e-12
    phi = torch.zeros_like(rho)
    c.solve(rho, phi, tol=1e-13, maxit=2000)
    dt = 0.05
    c.gather_push(phi, dt)
    p1, _ = c.particles()
    h = L / N
    Ep = opic.gather(opic.gradient(phi.cpu().numpy(), N, h), got[:3], N, L)
    xr, vr = opic.push(got[:3], got[3:], Ep, dt, L, kick=0.5 * dt)
    dx = np.abs(p1[:3] - xr)
    dx = np.minimum(dx, L - dx)
    assert np.max(dx) <= 1e-12 and np.max(np.abs(p1[3:] - vr)) <= 1e-12
    c.close()


def test_non_finite_state_is_rejected(pg):
    N, ppc = 8, 1
    c = pg.Context().init(N, ppc, 1)
    np_ = c.num_particles
    s = np.zeros((6, np_))
    s[4, 3] = np.nan
    with pytest.raises(pg.PicError) as e:
        c.set_particles(s, False)
    assert e.value.code == pg.PIC_EINVAL
    s[4, 3] = np.inf
    with pytest.raises(pg.PicError):
        c.set_particles(torch.from_numpy(s.reshape(-1)).cuda(), False)
    s[4, 3] = 0.0
    c.set_particles(s, False)  # accepted again
    c.close()


def test_host_round_trip_spans_several_chunks(pg):
    """128^3 x 20 ppc = 41.9 M particles: three 2^24-particle chunks, the last
    one ragged, in both directions, and the deposit of the state set from
    the host."""
    N, ppc = 128, 20
    c = pg.Context().init(N, ppc, 11)
    np_ = c.num_particles
    assert np_ > 2 * (1 << 24)
    rho0 = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho0)
    dev = torch.empty(6 * np_, dtype=torch.float64, device="cuda")
    c.particles_into(dev)
    host = torch.empty(6 * np_, dtype=torch.float64).pin_memory()
    c.particles_to_host(host)
    torch.cuda.synchronize()
    assert torch.equal(host.cuda(), dev)
    # permute the particles on the host, set, read back on the device
    perm = torch.from_numpy(np.random.default_rng(2).permutation(np_))
    hs = host.view(6, np_)[:, perm].contiguous().view(-1)
    c.set_particles(hs, True)
    c.particles_into(dev)
    torch.cuda.synchronize()
    back = dev.cpu().view(6, np_)
    assert torch.equal(back[3:], hs.view(6, np_)[3:])
    assert (back[:3] - hs.view(6, np_)[:3]).abs().max().item() <= 1e-15 * L
    # the cells counted while the chunks were converted sort the permuted
    # state: its deposit is the original state's (summation order aside)
    rho1 = torch.empty_like(rho0)
    c.deposit(rho1)
    assert (rho1 - rho0).abs().max().item() <= 1e-12
    c.close()
