"""CPU-side checks of the C ABI: the library loads, exports every entry point
that include/*.h declares, and rejects bad descriptors before touching CUDA."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hyb_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2510_11174_gb300 import build, _abi
    build.build()
    return _abi.load()


def test_header_declares_the_entry_points():
    d = _declared()
    for n in ("hyb_init_grid", "hyb_load_species", "hyb_step", "hyb_diagnostics"):
        assert n in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_prototypes_cover_the_header():
    from paper_2510_11174_gb300 import _abi
    assert _declared() <= set(_abi.PROTOTYPES)


def _desc(**kw):
    from paper_2510_11174_gb300 import _abi
    d = _abi.hyb_grid_desc()
    d.nx, d.ny, d.nz = 16, 16, 16
    d.dx = d.dy = d.dz = 0.4
    d.cfl_frac = 0.95
    d.tile = 8
    for k, v in kw.items():
        if k == "bc":
            for a in range(3):
                d.bc[a] = v[a]
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw", [dict(nx=12), dict(tile=6), dict(dx=0.0), dict(cfl_frac=1.2),
                                dict(dt=1.0), dict(bc=(1, 0, 0), nx=0), dict(laser_kind=1, x_src=99),
                                dict(laser_kind=1, x_src=2, pol=3, tau_fwhm=1.0, w0_spot=1.0),
                                dict(laser_kind=7)])
def test_invalid_descriptors_rejected_without_a_device(lib, kw):
    from paper_2510_11174_gb300 import _abi
    d = _desc(**kw)
    h = C.c_void_p()
    assert lib.hyb_init_grid(C.byref(d), C.byref(h)) == _abi.HYB_EINVAL
    assert h.value is None
    assert len(lib.hyb_last_error()) > 0


def test_null_arguments_rejected(lib):
    from paper_2510_11174_gb300 import _abi
    h = C.c_void_p()
    assert lib.hyb_init_grid(None, C.byref(h)) == _abi.HYB_EINVAL
    assert lib.hyb_step(None, 1) == _abi.HYB_EINVAL
    assert lib.hyb_diagnostics(None, None) == _abi.HYB_EINVAL
