"""The C-ABI library: builds for sm_103a, loads without a GPU, exports every symbol of include/hgm.h,
and its host-side argument checks answer without touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_00581_gb300 import build, hgm
    build.build()
    return hgm.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hgm_create_model", "hgm_create_scene", "hgm_match", "hgm_match_batch", "hgm_destroy",
                     "hgm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1505_00581_gb300 import hgm
    assert set(declared_functions()) == set(hgm.SIGNATURES)


def test_default_params_are_the_papers(lib):
    from paper_1505_00581_gb300 import hgm
    p = hgm.default_params()
    assert (p.lambda1, p.lambda2, p.lambda3, p.T) == pytest.approx((0.6, 0.2, 5.0, 10))
    assert p.offset_lo == -2 ** 31 and p.offset_hi == 2 ** 31 - 1


def test_host_side_validation_needs_no_gpu(lib):
    from paper_1505_00581_gb300 import hgm
    h = ctypes.c_void_p()
    xy = np.zeros((2, 2), np.float32)
    t = np.zeros(2, np.int32)
    f = np.zeros((2, 4), np.float32)
    rc = lib.hgm_create_model(xy.ctypes.data, t.ctypes.data, f.ctypes.data, 2, 4, None, ctypes.byref(h))
    assert rc == hgm.HGM_EINVAL and not h.value
    assert b"M >= 3" in lib.hgm_last_error()
    rc = lib.hgm_create_model(xy.ctypes.data, t.ctypes.data, f.ctypes.data, 3, 0, None, ctypes.byref(h))
    assert rc == hgm.HGM_EINVAL
    rc = lib.hgm_create_scene(None, None, None, -1, 4, 0, None, ctypes.byref(h))
    assert rc == hgm.HGM_EINVAL
    lib.hgm_destroy(None)
    # an unknown handle type is ignored rather than freed
    junk = (ctypes.c_uint32 * 4)(1, 2, 3, 4)
    lib.hgm_destroy(ctypes.cast(junk, ctypes.c_void_p))


def test_params_validation(lib):
    from paper_1505_00581_gb300 import hgm
    n, f = ctypes.c_int32(), ctypes.c_int32()
    for over, code in ((dict(K=0), hgm.HGM_EINVAL), (dict(K=256), hgm.HGM_EINVAL), (dict(K=100), hgm.HGM_EUNSUPPORTED),
                       (dict(window=-1), hgm.HGM_EINVAL), (dict(lambda1=-1.0), hgm.HGM_EINVAL),
                       (dict(precision=7), hgm.HGM_EUNSUPPORTED), (dict(offset_lo=5, offset_hi=4), hgm.HGM_EINVAL)):
        p = hgm.default_params(**over)
        rc = lib.hgm_offsets(None, None, ctypes.byref(p), ctypes.byref(n), ctypes.byref(f))
        assert rc == code, over
    p = hgm.default_params()
    assert lib.hgm_offsets(None, None, ctypes.byref(p), ctypes.byref(n), ctypes.byref(f)) == hgm.HGM_EINVAL


def test_validation_of_the_wider_forms(lib):
    """Argument checks of the chains, whole-block, streaming, dummy and refinement options answer on the
    host, before any device work."""
    from paper_1505_00581_gb300 import hgm
    p = hgm.default_params(dummy_cost=float("nan"))
    n, f = ctypes.c_int32(), ctypes.c_int32()
    assert lib.hgm_offsets(None, None, ctypes.byref(p), ctypes.byref(n), ctypes.byref(f)) == hgm.HGM_EINVAL
    assert b"dummy_cost" in lib.hgm_last_error()
    nil = (ctypes.c_void_p * 1)(None)
    for over in (dict(precision=1), dict(dummy_cost=1.0)):
        p = hgm.default_params(**over)
        assert lib.hgm_match_block(nil, 1, nil, 1, ctypes.byref(p), None, None, None) == hgm.HGM_EUNSUPPORTED
        h = ctypes.c_void_p()
        assert lib.hgm_stream_create(nil, 1, ctypes.byref(p), 60, 100, None, ctypes.byref(h)) == hgm.HGM_EUNSUPPORTED
        assert not h.value
    p = hgm.default_params()
    h = ctypes.c_void_p()
    assert lib.hgm_stream_create(nil, 1, ctypes.byref(p), 0, 100, None, ctypes.byref(h)) == hgm.HGM_EINVAL
    assert lib.hgm_stream_create(nil, 1, ctypes.byref(p), 60, 0, None, ctypes.byref(h)) == hgm.HGM_EINVAL
    e = np.zeros(4, np.float32)
    assert lib.hgm_match_chains(None, None, ctypes.byref(p), 3, None, None, None, e.ctypes.data, None) == hgm.HGM_EINVAL
    assert lib.hgm_match_chains_batch(nil, 1, nil, 1, ctypes.byref(p), 0, None, e.ctypes.data, None) == hgm.HGM_EINVAL
    assert lib.hgm_debug_timeout(0, None, None) == hgm.HGM_EINVAL
    junk = (ctypes.c_uint32 * 4)(1, 2, 3, 4)
    assert lib.hgm_stream_match(ctypes.cast(junk, ctypes.c_void_p), None, None, None, 0, None, None, None) \
        == hgm.HGM_EINVAL
