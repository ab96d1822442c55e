"""The allocation-free far-field entry point against the regular one (GPU).

pstd_cross_section_noalloc serves callers that cannot allocate device memory while
running (a fully reserved memory budget, or a loop that cannot afford an allocation or
the synchronisation a free implies).  Its result must equal pstd_cross_section's on the
same grid state, within the tolerance the parity tests use for each precision, on two
calls in a row (the second call reuses the shared scratch array, which still holds the
first call's contents).  Both branches of the far-field launch are covered: few
directions (faces split over CTAs, six partial sums per direction) and many (faces summed
in the CTA).  This file is collected last, so a stopping run has already run every other
test when it reaches it.
"""
import math

import numpy as np
import pytest

from paper_2403_04053_gb300 import inputs, pstd

pytestmark = pytest.mark.gpu

K = 2 * math.pi


def _spec():
    return inputs.GridSpec(n=(24, 32, 48), d=(0.25, 0.3, 0.2), dt=0.002, abc_cells=(4, 5, 6), tfsf_lo=(9, 12, 17),
                           tfsf_hi=(15, 20, 31), taper_cells=2, huygens_lo=(7, 9, 14), huygens_hi=(17, 23, 34))


def _V(spec):
    rng = np.random.default_rng(9)
    V = np.zeros(spec.shape)
    c = spec.core_box()
    V[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = rng.uniform(
        -3, 3, (c[2][1] - c[2][0] + 1, c[1][1] - c[1][0] + 1, c[0][1] - c[0][0] + 1))
    return V


def _run(g, spec):
    g.set_potential(_V(spec))
    g.set_incidence(0, (0.3, -0.5, 0.81), K, 0.05)
    g.huygens_dft(0, [K * K / 2], 20, 40)
    g.step(60)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [(pstd.F64, 1e-10), (pstd.F32, 1e-5)])
# 200000 directions exceed six partial sums a direction in the 16 MiB scratch, so there the
# allocation-free call sums the faces in each CTA while the regular call splits them
@pytest.mark.parametrize("M", [181, 20000, 200000])
def test_noalloc_cross_section_matches_the_regular_entry_point(prec, tol, M):
    import torch
    spec = _spec()
    rng = np.random.default_rng(M)
    th = np.arccos(rng.uniform(-1.0, 1.0, M))
    ph = rng.uniform(0.0, 2 * math.pi, M)
    with pstd.Grid(spec, precision=prec) as g:
        _run(g, spec)
        ds_ref, f_ref = g.cross_section(0, 0, th, ph)
        th_d = torch.from_numpy(th).cuda()
        ph_d = torch.from_numpy(ph).cuda()
        for _ in range(2):
            ds = torch.full((M,), -1.0, dtype=torch.float64, device="cuda")
            fa = torch.zeros(M, dtype=torch.complex128, device="cuda")
            g.cross_section_noalloc(0, 0, th_d, ph_d, ds, fa)
            torch.cuda.synchronize()
            assert _rel(fa.cpu().numpy(), f_ref) < tol
            assert _rel(ds.cpu().numpy(), ds_ref) < tol
        # without the amplitude: dsigma/dOmega alone
        ds = torch.full((M,), -1.0, dtype=torch.float64, device="cuda")
        g.cross_section_noalloc(0, 0, th_d, ph_d, ds, None)
        torch.cuda.synchronize()
        assert _rel(ds.cpu().numpy(), ds_ref) < tol


def test_noalloc_rejects_bad_calls():
    import torch
    spec = _spec()
    th = torch.linspace(0.1, 3.0, 16, dtype=torch.float64, device="cuda")
    ph = torch.zeros(16, dtype=torch.float64, device="cuda")
    ds = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pstd.Grid(spec, precision=pstd.F64) as g:
        _run(g, spec)
        # the window has completed, but no regular transform has set up the surface records
        with pytest.raises(pstd.PstdError) as e:
            g.cross_section_noalloc(0, 0, th, ph, ds, None)
        assert e.value.code == "ESTATE"
        g.cross_section(0, 0, [0.3], [0.1])
        # more directions than the scratch array holds
        big = torch.zeros((1 << 20) + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(pstd.PstdError) as e:
            g.cross_section_noalloc(0, 0, big, big, big, None)
        assert e.value.code == "EINVAL"
        # host memory, a wrong dtype or a short output never reaches the library
        for args in ((th.cpu(), ph, ds), (th.float(), ph, ds), (th, ph, ds[:8])):
            with pytest.raises(ValueError):
                g.cross_section_noalloc(0, 0, *args, None)
        # the C entry point itself refuses a host pointer, before any launch
        host = np.zeros(16)
        st = g.lib.pstd_cross_section_noalloc(g.h, 0, 0, host.ctypes.data, ph.data_ptr(), 16, ds.data_ptr(), None)
        assert pstd.STATUS.get(st) == "EINVAL"
        # and the grid still works afterwards
        g.cross_section_noalloc(0, 0, th, ph, ds, None)
        torch.cuda.synchronize()
        ref, _ = g.cross_section(0, 0, th.cpu().numpy(), ph.cpu().numpy())
        assert _rel(ds.cpu().numpy(), ref) < 1e-10
