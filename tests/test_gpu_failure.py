"""Failure detection through the C ABI (paper, Methodology: the run's stability
is checked, values are clamped and unstable steps are skipped).  Every failure
here is made on the host side or by a bounded wait that gives up; none of them
faults the GPU, and the context stays usable afterwards:

* non-finite fields loaded with hyb_set_fields -> HYB_ENAN from the next
  synchronising call -> hyb_step refuses with HYB_ESTATE -> hyb_clear_status
  and finite fields bring the context back;
* a tile too small for the particles that migrate into it, with tile growth
  off -> HYB_EOVERFLOW, the particles that did not fit are dropped;
* the bounded mbarrier wait of the tensor-core pipelines, run on a barrier
  nothing completes -> HYB_ETIMEOUT.
"""
import math

import numpy as np
import pytest

from _util import require_gpu

pytestmark = pytest.mark.gpu


def _plasma_sim(P, n=16, tile=4):
    from paper_2510_11174_gb300 import inputs
    inp = inputs.periodic_plasma(n=n, ppc=1, seed=11)
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], tile=tile)
    for sp in inp["species"]:
        sim.load_species(**sp)
    sim.set_fields(inp["E"], inp["B"])
    return sim, inp


def test_nan_fields_latch_enan_then_estate_then_recover():
    P = require_gpu()
    from paper_2510_11174_gb300._abi import HybError, HYB_ENAN, HYB_ESTATE
    sim, inp = _plasma_sim(P)
    sim.step(2)
    assert sim.diagnostics()["status"] == 0
    E = inp["E"].copy()
    E[1, 3, 4, 5] = np.nan
    sim.set_fields(E, inp["B"])
    with pytest.raises(HybError) as ei:
        sim.diagnostics()
    assert ei.value.code == HYB_ENAN
    with pytest.raises(HybError) as ei:
        sim.step(1)
    assert ei.value.code == HYB_ESTATE
    sim.clear_status()
    sim.set_fields(inp["E"], inp["B"])
    sim.step(2)
    d = sim.diagnostics()
    assert d["status"] == 0 and math.isfinite(d["w_e"])
    sim.close()


def test_tile_overflow_without_growth_latches_eoverflow_and_drops():
    P = require_gpu()
    from paper_2510_11174_gb300._abi import HybError, HYB_EOVERFLOW, HYB_ESTATE
    dx = 2 * math.pi / 16
    sim = P.Simulation(16, 16, 16, dx, cfl_frac=0.95, tile=4)
    sim.set_auto_grow(False)
    # tile 0 (x in [0, 4)) and tile 1 (x in [4, 8)) each hold 32 particles, their
    # capacity; tile 0's particles sit next to the boundary moving at v ~ c in +x,
    # so one step moves all of them into tile 1, which has room for none
    rng = np.random.default_rng(3)
    n = 32
    f32 = lambda a: np.asarray(a, np.float32)
    x = np.concatenate([np.full(n, 3.9), np.full(n, 5.5)])
    y = rng.uniform(0.2, 3.8, 2 * n)
    z = rng.uniform(0.2, 3.8, 2 * n)
    ux = np.concatenate([np.full(n, 20.0), np.zeros(n)])
    sid = sim.load_species(q=-1.0, m=1.0, x=f32(x), y=f32(y), z=f32(z), ux=f32(ux), uy=f32(np.zeros(2 * n)),
                           uz=f32(np.zeros(2 * n)), w=f32(np.full(2 * n, 1e-3)), tile_capacity=32)
    assert sim.diagnostics()["tile_capacity"][sid] == 32
    sim.step(1)
    with pytest.raises(HybError) as ei:
        sim.diagnostics()
    assert ei.value.code == HYB_EOVERFLOW
    d = sim.diagnostics(raise_on_status=False)
    assert d["status"] == HYB_EOVERFLOW
    assert d["count"][sid] == 32            # tile 1 kept its capacity, the rest was dropped
    with pytest.raises(HybError) as ei:
        sim.step(1)
    assert ei.value.code == HYB_ESTATE
    sim.clear_status()
    sim.step(1)
    assert sim.diagnostics()["status"] == 0
    sim.close()


def test_bounded_wait_gives_up_with_etimeout():
    P = require_gpu()
    from paper_2510_11174_gb300._abi import HybError, HYB_ETIMEOUT, HYB_EINVAL
    sim, _ = _plasma_sim(P, n=8)
    with pytest.raises(HybError) as ei:
        sim.selftest_wait_timeout(0)
    assert ei.value.code == HYB_EINVAL
    sim.selftest_wait_timeout(4096)
    with pytest.raises(HybError) as ei:
        sim.diagnostics()
    assert ei.value.code == HYB_ETIMEOUT
    sim.clear_status()
    sim.step(3)
    assert sim.diagnostics()["status"] == 0
    sim.close()
