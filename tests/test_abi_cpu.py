"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/pstd.h declares, and rejects bad descriptors before touching a device."""
import math
import os
import re

import pytest

from paper_2403_04053_gb300 import inputs, pstd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pstd.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pstd.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pstd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pstd_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) == len(pstd._SIGS)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(pstd._SIGS)


def _spec(**kw):
    base = dict(n=(48, 48, 48), d=(0.25,) * 3, dt=0.004)
    base.update(kw)
    return inputs.GridSpec(**base)


def test_unstable_time_step_is_rejected(lib):
    """dt = 0.005 at dx = 0.25 exceeds Eq. PSTDstability: PSTD_EUNSTABLE from pstd_create_grid."""
    with pytest.raises(pstd.PstdError) as e:
        pstd.Grid(_spec(dt=0.005), stream=None)
    assert e.value.code == "EUNSTABLE"


@pytest.mark.parametrize("kw", [dict(n=(48, 48, 50)), dict(huygens_lo=(15, 11, 11)), dict(abc_cells=(12, 8, 8)),
                                dict(taper_cells=0), dict(tfsf_hi=(34, 34, 40))])
def test_bad_geometry_is_rejected(lib, kw):
    with pytest.raises(pstd.PstdError) as e:
        pstd.Grid(_spec(**kw), stream=None)
    assert e.value.code == "EINVAL"


def test_stability_bound_matches_the_formula(lib):
    assert pstd.stability_dt_max(_spec(), 0.3 * 2 * math.pi ** 2) == pytest.approx(0.0041188, rel=1e-4)


def test_binding_fails_loudly_without_the_library(tmp_path):
    # the product path has no fallback: a missing library is an ImportError, not a CPU path
    from paper_2403_04053_gb300 import pstd
    with pytest.raises(ImportError):
        pstd.load_library(str(tmp_path / "libpstd.so"))
