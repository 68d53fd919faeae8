"""Host model of the tensor-core preconditioner's TMEM ring (no GPU).

k_apply_k_tc (16-wide Toeplitz groups) and k_apply_k_tc8 (8-wide, with a
zero group) accumulate each output plane's nine dz contributions, one per
input plane, in a ring of TMEM slots, and hand a finished plane to the
epilogue while the issuer runs ahead. This model restates, in Python, the
kernels' work order (whole columns dealt round-robin over the CTAs, the rest
split contiguously), their group lists per input plane, the ring and shadow
slot arithmetic and the issuer's wait on the epilogue of the plane
SLOT_REUSE_LAG planes back, and checks for every CTA of several launches:
  * every MMA writes inside the allocated columns and has a legal N;
  * every output plane receives each dz = 0..8 exactly once (primary plus
    shadow slot);
  * no MMA writes a slot whose previous output may still be read by the
    epilogue (reuse only after that output's epilogue completed), and the
    8-wide form's zero group never lands on a slot being read;
  * every (column, plane) unit is produced by exactly one CTA.
"""
import pytest


def work_runs(N, G, b, bx):
    """The runs (column, pa, pb) of CTA b: whole columns b, b + G, ... then
    its contiguous share of the leftover columns' units."""
    C = (N // bx) * (N // 128)
    R = C // G
    for k in range(R):
        yield b + k * G, 0, N
    tcol0 = R * G
    TU = (C - tcol0) * N
    tb, te = TU * b // G, TU * (b + 1) // G
    u = tb
    while u < te:
        col, pa = tcol0 + u // N, u % N
        pb = min(N, pa + (te - u))
        yield col, pa, pb
        u += pb - pa


def mma_sets16(dz_lo, dz_hi, s_lo):
    """16-wide form: one group list per input plane, slots from s_lo."""
    return [(s_lo, list(range(dz_lo, dz_hi + 1)))]


def mma_sets8(dz_lo, dz_hi, s_lo):
    """8-wide form: groups at physical slots from s_lo + 1; an odd count
    padded by a zero group in front (dz_lo == 0) or split into a
    [zero, dz_lo] pair and an even rest."""
    ng = dz_hi - dz_lo + 1
    p_lo = s_lo + 1
    if ng % 2 == 0:
        return [(p_lo, list(range(dz_lo, dz_hi + 1)))]
    if dz_lo == 0:
        return [(p_lo - 1, [None] + list(range(0, dz_hi + 1)))]
    sets = [(p_lo - 1, [None, dz_lo])]
    if ng > 1:
        sets.append((p_lo + 1, list(range(dz_lo + 1, dz_hi + 1))))
    return sets


FORMS = {
    # bx, ring slots T, physical slots, lag, group width in columns, max N, sets, primary/shadow
    "tc16": dict(bx=16, T=24, phys=32, lag=24 - 8, width=16, nmax=144, sets=mma_sets16,
                 primary=lambda s: s, shadow=lambda s, T: s + T),
    "tc8": dict(bx=8, T=55, phys=64, lag=55 - 9, width=8, nmax=80, sets=mma_sets8,
                primary=lambda s: s + 1, shadow=lambda s, T: s + T + 1),
}


def check(form, N, G):
    f = FORMS[form]
    T, PHYS, LAG, bx = f["T"], f["phys"], f["lag"], f["bx"]
    ring = lambda v: (T - v % T) % T  # noqa: E731
    seen = set()
    for b in range(G):
        runs = list(work_runs(N, G, b, bx))
        # epilogue index (input-plane counter) at which each output completes
        epi, j, vbase = {}, 0, 0
        for col, pa, pb in runs:
            for z in range(pa - 4, pb + 4):
                if z - 4 >= pa:
                    epi[vbase + z - 4 - pa] = j
                    assert (col, z - 4) not in seen
                    seen.add((col, z - 4))
                j += 1
            vbase += pb - pa
        owner = [None] * PHYS
        content = [dict() for _ in range(PHYS)]
        j, vbase = 0, 0
        for col, pa, pb in runs:
            for z in range(pa - 4, pb + 4):
                dz_lo, dz_hi = max(0, z + 4 - (pb - 1)), min(8, z + 4 - pa)
                s_lo = ring(vbase + z + 4 - dz_lo - pa)
                for p0, groups in f["sets"](dz_lo, dz_hi, s_lo):
                    n = f["width"] * len(groups)
                    assert n % 16 == 0 and 16 <= n <= f["nmax"], (form, n)
                    assert 0 <= p0 and p0 + len(groups) <= PHYS
                    for k, g in enumerate(groups):
                        X = p0 + k
                        o = owner[X]
                        if g is None:  # zero group: adds A x 0 to a live or finished slot
                            assert o is None or not (j - LAG < epi[o] < j), (form, N, G, b, j)
                            continue
                        u = vbase + z + 4 - g - pa
                        s = ring(u)
                        assert X == f["primary"](s) or (X == f["shadow"](s, T) and f["shadow"](s, T) < PHYS)
                        if o is not None and o != u:
                            assert epi[o] <= j - LAG, (form, N, G, b, j)
                        owner[X] = u
                        content[X].setdefault(u, []).append(g)
                if z - 4 >= pa:  # the epilogue of output plane z - 4
                    u = vbase + z - 4 - pa
                    s = ring(u)
                    got = content[f["primary"](s)].pop(u, [])
                    if f["shadow"](s, T) < PHYS:
                        got += content[f["shadow"](s, T)].pop(u, [])
                    assert sorted(got) == list(range(9)), (form, N, G, b, u, sorted(got))
                j += 1
            vbase += pb - pa
    assert len(seen) == (N // bx) * (N // 128) * N


@pytest.mark.parametrize("form", ["tc16", "tc8"])
@pytest.mark.parametrize("N,G", [(128, 152), (128, 7), (256, 152), (256, 1), (384, 152), (512, 152), (512, 148),
                                 (512, 37)])
def test_tensor_core_ring_is_safe_and_complete(form, N, G):
    check(form, N, G)
