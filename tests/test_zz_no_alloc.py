"""The allocation-free field-energy entry point (hyb_field_energy_noalloc).

It serves callers that cannot call cudaMalloc (code that must not synchronise
the device mid-loop, code whose device memory belongs to another allocator,
code with a fixed memory budget): its scratch is a fixed static device array.
This test calls it through the C ABI twice in a row, on two different field
sets (the second smaller, so stale partial sums of the first call would show),
and checks each result against the energies hyb_diagnostics reports for the
same fields.  It is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C
import math

import numpy as np
import pytest

from _util import require_gpu

pytestmark = pytest.mark.gpu


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    E = rng.standard_normal((3,) + shape).astype(np.float32)
    B = (0.5 * rng.standard_normal((3,) + shape)).astype(np.float32)
    return E, B


def test_noalloc_field_energy_matches_diagnostics_twice():
    P = require_gpu()
    import torch
    from paper_2510_11174_gb300 import _abi

    lib = _abi.load()
    dx = 2 * math.pi / 16
    for (nz, ny, nx), seed in (((32, 32, 32), 1), ((8, 16, 16), 2)):
        E, B = _fields((nz, ny, nx), seed)
        sim = P.Simulation(nx, ny, nz, dx)
        sim.set_fields(E, B)
        ref = sim.diagnostics()
        sim.close()
        Ed = torch.from_numpy(E).cuda()
        Bd = torch.from_numpy(B).cuda()
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        code = lib.hyb_field_energy_noalloc(Ed.data_ptr(), Bd.data_ptr(), nx * ny * nz, dx, dx, dx,
                                            out.data_ptr(), stream.cuda_stream)
        assert code == _abi.HYB_OK, lib.hyb_last_error()
        stream.synchronize()
        w_e, w_b = out.cpu().tolist()
        assert w_e == pytest.approx(ref["w_e"], rel=1e-12)
        assert w_b == pytest.approx(ref["w_b"], rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    P = require_gpu()
    import torch
    from paper_2510_11174_gb300 import _abi

    lib = _abi.load()
    x = torch.zeros(3, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    too_big = 22369621 + 1
    assert lib.hyb_field_energy_noalloc(x.data_ptr(), x.data_ptr(), too_big, 1.0, 1.0, 1.0, out.data_ptr(),
                                        None) == _abi.HYB_EINVAL
    assert b"HYB_NOALLOC_MAX_CELLS" in lib.hyb_last_error()
