"""The C-ABI library builds, loads and exports every function that
include/bdis.h declares; argument checks run on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = []
    for hp in HEADERS:
        text = open(hp).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(bdis_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_03133_gb300 import build
    build.build()
    from paper_2205_03133_gb300 import _binding
    return _binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/*.h but not exported"


def test_binding_covers_the_header():
    from paper_2205_03133_gb300 import _binding
    bound = {n for n, _, _ in _binding.EXPORTS}
    assert set(_declared_functions()) == bound


def test_struct_sizes_match_header(lib):
    from paper_2205_03133_gb300 import _binding as B
    assert C.sizeof(B.bdis_patch_record) == 64
    p = B.bdis_params()
    lib.bdis_default_params(C.byref(p))
    assert (p.patch, p.stride, p.levels, p.iters) == (8, 4, 3, 8)
    assert p.sigma_s == 4.0 and p.window_step == 0.5 and p.pdf_iters == 10


def test_host_side_argument_checks(lib):
    import paper_2205_03133_gb300 as bd
    with pytest.raises(bd.BdisError):
        bd.BDIS(patch=3)
    with pytest.raises(bd.BdisError):
        bd.BDIS(stride=9)
    with pytest.raises(bd.BdisError):
        bd.BDIS(levels=9)
    m = bd.BDIS(patch=12, stride=6, levels=4)
    B = bd.B
    # null pointers
    st = lib.bdis_match(m._h, None, None, 640, 480, 640, None, None, None, None)
    assert st == B.BDIS_EINVAL
    # too small for the pyramid: coarsest level below the patch size
    st = lib.bdis_match(m._h, 16, 16, 80, 60, 80, 16, None, 16, None)
    assert st == B.BDIS_EINVAL and b"too small" in lib.bdis_last_error(m._h)
    # pitch below width
    st = lib.bdis_match(m._h, 16, 16, 640, 480, 600, 16, None, 16, None)
    assert st == B.BDIS_EINVAL
    assert lib.bdis_strerror(B.BDIS_EUNSUPPORTED) == b"unsupported"
    # level views before any call
    v = B.bdis_level_view()
    assert lib.bdis_level_view_get(m._h, 0, 0, C.byref(v)) == B.BDIS_EINVAL
    # option ranges
    for opt, good, bad in ((B.OPT_BULK_COPY, (0, 1, 2, 3), (-1, 4)),
                           (B.OPT_SEARCH_PASSES, (0, 1, 2, 3, 4), (-1, 5)),
                           (B.OPT_FUSE_TILE, (0, 1, 2, 3), (-1, 4))):
        for val in good:
            assert lib.bdis_set_option(m._h, opt, val) == B.BDIS_OK, (opt, val)
        for val in bad:
            assert lib.bdis_set_option(m._h, opt, val) == B.BDIS_EINVAL, (opt, val)


def test_mode_parameter_checks(lib):
    import paper_2205_03133_gb300 as bd
    for bad in (dict(weight_mode=2), dict(finest_level=3), dict(finest_level=-1), dict(fast_exp=2)):
        with pytest.raises(bd.BdisError):
            bd.BDIS(levels=3, **bad)
    m = bd.BDIS(levels=6, patch=10, stride=4, finest_level=1, weight_mode="dis", fast_exp=1)
    p = bd.B.bdis_params()
    assert lib.bdis_get_params(m._h, C.byref(p)) == 0
    assert (p.finest_level, p.weight_mode, p.fast_exp) == (1, 1, 1)
    d = bd.default_params()
    assert (d.finest_level, d.weight_mode, d.fast_exp) == (0, 0, 0)


def test_depth_argument_checks(lib):
    from paper_2205_03133_gb300 import _binding as B
    # rejected before any CUDA call
    assert lib.bdis_depth(16, None, 10, C.c_float(0.0), 16, None, None) == B.BDIS_EINVAL
    assert lib.bdis_depth(16, None, 10, C.c_float(float("nan")), 16, None, None) == B.BDIS_EINVAL
    assert lib.bdis_depth(16, None, -1, C.c_float(1.0), 16, None, None) == B.BDIS_EINVAL
    assert lib.bdis_depth(None, None, 10, C.c_float(1.0), 16, None, None) == B.BDIS_EINVAL
    assert lib.bdis_depth(16, 16, 10, C.c_float(1.0), 16, None, None) == B.BDIS_EINVAL
    assert lib.bdis_depth(None, None, 0, C.c_float(1.0), None, None, None) == B.BDIS_OK


def test_empty_and_oversize_inputs_rejected(lib):
    import paper_2205_03133_gb300 as bd
    B = bd.B
    m = bd.BDIS(patch=8, stride=4, levels=2)
    for (w, h, pitch) in ((0, 48, 64), (64, 0, 64), (-5, 48, 64), (40000, 48, 40000),
                          (64, 40000, 64), (64, 48, 0)):
        st = lib.bdis_match(m._h, 16, 16, w, h, pitch, 16, None, 16, None)
        assert st == B.BDIS_EINVAL, (w, h, pitch)
    # an empty batch
    assert lib.bdis_match_batched(m._h, 0, None, None) == B.BDIS_EINVAL
    pairs = (B.bdis_pair * 1)()
    assert lib.bdis_match_batched(m._h, 0, pairs, None) == B.BDIS_EINVAL
    assert lib.bdis_match_batched(m._h, -1, pairs, None) == B.BDIS_EINVAL
    # the extreme patch geometries are accepted
    for kw in (dict(patch=4, stride=1), dict(patch=16, stride=16), dict(patch=16, stride=1)):
        bd.BDIS(levels=1, **kw).close()
