"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments on the host before any CUDA work."""
import ctypes

import pytest

from paper_2301_09710_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    from paper_2301_09710_gb300.build import build
    build()
    return _lib.load()


def test_exports_every_header_symbol(lib):
    names = _lib.header_symbols()
    assert {"spect_plan_create", "spect_forward", "spect_back", "spect_em_step", "spect_plan_destroy",
            "spect_last_error"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def _create(lib, nx=8, ny=8, nz=4, nview=3, px=3, pz=3, nvp=1, psf=16, fx=None, fz=None, dy=1.0, flags=0,
            out=True):
    h = ctypes.c_void_p()
    return lib.spect_plan_create(ctypes.byref(h) if out else None, nx, ny, nz, nview, None, ctypes.c_float(dy),
                                 psf, fx, fz, px, pz, nvp, None, flags, None)


@pytest.mark.parametrize("kw,msg", [
    (dict(ny=9), "nx must equal ny"),
    (dict(nx=1, ny=1), "nx must be in"),
    (dict(nz=0), "nz must be"),
    (dict(nview=0), "nview must be"),
    (dict(px=4), "odd"),
    (dict(pz=129), "odd"),
    (dict(nvp=2), "nview_psf"),
    (dict(psf=None), "no PSF"),
    (dict(psf=None, fx=16), "both psf_fx and psf_fz"),
    (dict(dy=-1.0), "dy"),
    (dict(flags=1 << 7), "flag"),
    (dict(psf=20), "aligned"),
    (dict(out=False), "out is NULL"),
])
def test_plan_create_rejects_on_host(lib, kw, msg):
    st = _create(lib, **kw)
    assert st == 1, (st, _lib.last_error())
    assert msg in _lib.last_error()


def test_calls_reject_null_plan_and_pointers(lib):
    assert lib.spect_forward(None, 16, 16, None) == 1
    assert "plan is NULL" in _lib.last_error()
    assert lib.spect_back(None, 16, 16, None) == 1
    assert lib.spect_em_step(None, 16, 16, None, 1, None) == 1
    assert lib.spect_plan_info(None, None, None, None, None) == 1
    assert lib.spect_plan_destroy(None) == 0


def test_binding_raises_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="missing"):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "nope.so"))
        finally:
            _lib._lib = None
