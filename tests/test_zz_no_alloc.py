"""The allocation-free far-field entry point against the regular one (GPU).

pstd_cross_section_noalloc serves callers that cannot allocate device memory while
running; its result must equal pstd_cross_section's on the same grid state, within the
FP64 tolerance the parity tests use, on two calls in a row (the second call reuses the
shared scratch array, which still holds the first call's contents).
"""
import math

import numpy as np
import pytest

from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu


def test_noalloc_cross_section_matches_the_regular_entry_point():
    import torch
    spec = inputs.GridSpec(n=(24, 32, 48), d=(0.25, 0.3, 0.2), dt=0.002, abc_cells=(4, 5, 6), tfsf_lo=(9, 12, 17),
                           tfsf_hi=(15, 20, 31), taper_cells=2, huygens_lo=(7, 9, 14), huygens_hi=(17, 23, 34))
    rng = np.random.default_rng(9)
    V = np.zeros(spec.shape)
    c = spec.core_box()
    V[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = rng.uniform(
        -3, 3, (c[2][1] - c[2][0] + 1, c[1][1] - c[1][0] + 1, c[0][1] - c[0][0] + 1))
    k = 2 * math.pi
    th = np.deg2rad(np.linspace(0.5, 179.5, 181))
    ph = np.deg2rad(np.linspace(0.0, 360.0, 181))
    with pstd.Grid(spec, precision=pstd.F64) as g:
        g.set_potential(V)
        g.set_incidence(0, (0.3, -0.5, 0.81), k, 0.05)
        g.huygens_dft(0, [k * k / 2], 20, 40)
        g.step(60)
        ds_ref, f_ref = g.cross_section(0, 0, th, ph)
        th_d = torch.from_numpy(th).cuda()
        ph_d = torch.from_numpy(ph).cuda()
        for _ in range(2):
            ds = torch.full((len(th),), -1.0, dtype=torch.float64, device="cuda")
            fa = torch.zeros(len(th), dtype=torch.complex128, device="cuda")
            g.cross_section_noalloc(0, 0, th_d, ph_d, ds, fa)
            torch.cuda.synchronize()
            ds_h, fa_h = ds.cpu().numpy(), fa.cpu().numpy()
            assert np.linalg.norm(fa_h - f_ref) / np.linalg.norm(f_ref) < 1e-10
            assert np.linalg.norm(ds_h - ds_ref) / np.linalg.norm(ds_ref) < 1e-10
        with pytest.raises(pstd.PstdError) as e:
            big = torch.zeros((1 << 20) + 1, dtype=torch.float64, device="cuda")
            g.cross_section_noalloc(0, 0, big, big, big, None)
        assert e.value.code == "EINVAL"
