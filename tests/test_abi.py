"""The C ABI library builds, loads and exports every function include/pic.h
declares; argument errors come back as status codes (no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09605_gb300 import build, pic
    build.build()
    return pic.lib()


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2411_09605_gb300 import pic
    names = _declared("pic.h")
    assert names, "no declarations found"
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(pic.EXPORTS)


def test_version_string(lib):
    from paper_2411_09605_gb300 import pic
    assert "sm_103a" in pic.pic_version()


def test_debug_bounds_probe_unsupported_in_normal_build(lib):
    """The index checks exist only in the PIC_DEBUG_BOUNDS build; the normal
    library says so without touching the device."""
    import ctypes as C
    if os.environ.get("PIC_DEBUG_BOUNDS") == "1":
        pytest.skip("the debug-bounds library is loaded")
    flagged = C.c_int(7)
    assert lib.pic_debug_bounds(3, 10, C.byref(flagged)) == -7
    assert flagged.value == -1
    assert b"PIC_DEBUG_BOUNDS" in lib.pic_last_error()
    assert lib.pic_debug_bounds(3, 10, None) == -1
    assert "debug-bounds" not in lib.pic_version().decode()


def test_argument_errors_are_status_codes(lib):
    from paper_2411_09605_gb300 import pic
    x = np.array([0.5])
    v = np.array([0.1])
    sp = [dict(q=-1.0, m=1.0, x=x, v=v, w=None, w0=1.0)]
    bad = [
        pic.make_config(64, 1.0, 0.1, order=3),
        pic.make_config(64, 1.0, -0.1),
        pic.make_config(2, 1.0, 0.1),
        pic.make_config(64, 1.0, 0.1, scheme=3),
        pic.make_config(64, 1.0, 0.1, dim_x=2),
        # spectral solvers: a power of two in [4, 1024] nodes, dim_v = 2, c > 0
        pic.make_config(48, 1.0, 0.1, solver=pic.PIC_SOLVER_PSATD, dim_v=2),
        pic.make_config(2048, 1.0, 0.1, solver=pic.PIC_SOLVER_CN_SPECTRAL, dim_v=2),
        pic.make_config(2, 1.0, 0.1, solver=pic.PIC_SOLVER_CN_SPECTRAL, dim_v=2),
        pic.make_config(64, 1.0, 0.1, solver=pic.PIC_SOLVER_PSATD, dim_v=1),
        pic.make_config(64, 1.0, 0.1, solver=pic.PIC_SOLVER_PSATD, dim_v=2, c=0.0),
        pic.make_config(64, 1.0, 0.1, solver=5, dim_v=2),
        # standard comparator: 1D1V, a power of two in [4, 4096], 0..8 filter passes
        pic.make_config(48, 1.0, 0.1, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG),
        pic.make_config(8192, 1.0, 0.1, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG),
        pic.make_config(64, 1.0, 0.1, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG, binomial_passes=9),
        pic.make_config(64, 1.0, 0.1, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG, dim_v=2),
    ]
    for cfg in bad:
        with pytest.raises(pic.PicError) as ei:
            pic.pic_init(cfg, sp)
        assert ei.value.code == -1
    with pytest.raises(pic.PicError) as ei:
        pic.pic_init(pic.make_config(64, 1.0, 0.1), [])
    assert ei.value.code == -1
    with pytest.raises(pic.PicError) as ei:   # the mixed forms run one species
        pic.pic_init(pic.make_config(64, 1.0, 0.1, precision=pic.PIC_PREC_MIXED,
                                     solver=pic.PIC_SOLVER_PSATD, dim_v=2), sp * 2)
    assert ei.value.code == -7
    with pytest.raises(pic.PicError) as ei:   # no filtering in the Yee solver
        pic.pic_init(pic.make_config(64, 1.0, 0.1, binomial_passes=1,
                                     precision=pic.PIC_PREC_MIXED,
                                     solver=pic.PIC_SOLVER_YEE_LEAPFROG, dim_x=2, dim_v=3,
                                     ny=64, Ly=1.0), sp)
    assert ei.value.code == -7
    with pytest.raises(pic.PicError) as ei:
        pic.pic_init(pic.make_config(64, 1.0, 0.1, binomial_passes=9), sp)
    assert ei.value.code == -1
    for kw in ({"sort_period": 4},          # sorting: mixed forms of the Ampere and Yee solvers
               {"sort_period": 4, "solver": pic.PIC_SOLVER_YEE_LEAPFROG, "dim_x": 2, "dim_v": 3,
                "ny": 64, "Ly": 1.0},
               {"sort_period": 4, "solver": pic.PIC_SOLVER_PSATD, "dim_v": 2,
                "precision": pic.PIC_PREC_MIXED},
               {"charge_conserving": 1}):                           # Yee solver only
        with pytest.raises(pic.PicError) as ei:
            pic.pic_init(pic.make_config(64, 1.0, 0.1, **kw), sp)
        assert ei.value.code == -7
    for kw in ({"sort_period": -1}, {"charge_conserving": 2}):
        with pytest.raises(pic.PicError) as ei:
            pic.pic_init(pic.make_config(64, 1.0, 0.1, **kw), sp)
        assert ei.value.code == -1
    with pytest.raises(pic.PicError) as ei:   # its field follows from the charge
        pic.pic_init(pic.make_config(64, 1.0, 0.1, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG), sp,
                     np.zeros(64))
    assert ei.value.code == -1
    assert lib.pic_step(None, 1, None, None) == -1
    lib.pic_free(None)  # no-op


def test_batch_argument_errors_are_status_codes(lib):
    import ctypes as C
    from paper_2411_09605_gb300 import pic
    x = np.array([0.5])
    v = np.array([0.1])
    sp = [dict(q=-1.0, m=1.0, x=x, v=v, w=None, w0=1.0)]
    # not batchable: FP64 form, sorted markers, the filter, more than 512 nodes, mixed schemes
    for cfgs in ([pic.make_config(64, 1.0, 0.1)],
                 [pic.make_config(64, 1.0, 0.1, precision=pic.PIC_PREC_MIXED, sort_period=4)],
                 [pic.make_config(64, 1.0, 0.1, precision=pic.PIC_PREC_MIXED, binomial_passes=1)],
                 [pic.make_config(1024, 1.0, 0.1, precision=pic.PIC_PREC_MIXED)],
                 [pic.make_config(64, 1.0, 0.1, precision=pic.PIC_PREC_MIXED),
                  pic.make_config(64, 1.0, 0.1, scheme=pic.PIC_SCHEME_ESEC1,
                                  precision=pic.PIC_PREC_MIXED)]):
        with pytest.raises(pic.PicError) as ei:
            pic.pic_batch_init(cfgs, sp * len(cfgs))
        assert ei.value.code == -7
    assert lib.pic_batch_init(None, None, 1, C.byref(C.c_void_p())) == -1
    assert lib.pic_batch_step(None, 1) == -1
    lib.pic_batch_free(None)  # no-op


def test_every_entry_point_has_argument_types():
    """ctypes passes undeclared integer arguments as 32-bit ints, which would cut
    the 64-bit handle pointers."""
    from paper_2411_09605_gb300 import pic
    L = pic.lib()
    for name in pic.EXPORTS:
        if name not in ("pic_last_error", "pic_version"):
            assert getattr(L, name).argtypes is not None, name
