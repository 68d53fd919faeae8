"""pic_field_energy_noalloc: the field-energy entry point for callers that
cannot allocate device memory (a host that owns a fixed device-memory budget,
or a stepping loop that must not call cudaMalloc/cudaFree because they can
synchronise the device). It takes no context and keeps its reduction scratch
in a fixed file-scope device array, so it is checked here against the
context's pic_field_energy on consecutive calls that share that scratch.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_field_energy_matches_context_entry_point():
    import paper_2605_05469_gb300 as pg
    from paper_2605_05469_gb300 import inputs

    k = 0.5
    for N, seeds in ((64, (1, 2)), (32, (3,))):
        ctx = pg.Context().init(N, 0, 0)
        for seed in seeds:  # consecutive calls share (and must clear) the scratch
            phi = torch.from_numpy(inputs.noise_field(N, seed)).cuda()
            ref = ctx.field_energy(phi)
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            assert pg.pic_field_energy_noalloc(phi, N, k, out) == pg.PIC_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (N, seed, got, ref)
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import paper_2605_05469_gb300 as pg

    phi = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    f = pg.lib().pic_field_energy_noalloc
    p, o = ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr())
    assert f(p, 2048, 0.5, o, None) == pg.PIC_EINVAL
    assert f(p, 12, 0.5, o, None) == pg.PIC_EINVAL
    assert f(None, 8, 0.5, o, None) == pg.PIC_EINVAL
