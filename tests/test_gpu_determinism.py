"""Bitwise reproducibility (paper, Methodology: stored code, parameters and
fixed random streams make every run repeatable).  The current deposition
accumulates in 64-bit fixed point, so J does not depend on the order in which
particles sit in their tiles or warps run; random events use counter-based
Philox streams keyed by particle id and step.  Two runs of the same input
therefore give the same fields and the same particles bit for bit, although
the slot order of particles inside tiles may differ."""
import numpy as np
import pytest

from _util import by_id, make_pair

pytestmark = pytest.mark.gpu


def _run(inp, steps, tile=8, laser=None):
    sim, _ = make_pair(inp, laser=laser, tile=tile, with_oracle=False)
    sim.step(steps)
    E, B, J = sim.get_fields()
    parts = [by_id(sim.get_species(s, with_zq=False)) for s in range(len(inp["species"]))]
    d = sim.diagnostics()
    sim.close()
    return E, B, J, parts, d


def _same(a, b):
    Ea, Ba, Ja, pa, da = a
    Eb, Bb, Jb, pb, db = b
    assert np.array_equal(Ea.view(np.uint32), Eb.view(np.uint32))
    assert np.array_equal(Ba.view(np.uint32), Bb.view(np.uint32))
    assert np.array_equal(Ja.view(np.uint32), Jb.view(np.uint32))
    for x, y in zip(pa, pb):
        assert np.array_equal(x["ids"], y["ids"])
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            assert np.array_equal(x[k].view(np.uint32), y[k].view(np.uint32)), k
    assert da["count"] == db["count"]


def test_periodic_plasma_runs_twice_bit_for_bit():
    from paper_2510_11174_gb300 import inputs
    inp = inputs.periodic_plasma(n=32, ppc=8, seed=6, a0=2.0, temperature_keV=10.0)
    _same(_run(inp, 30), _run(inp, 30))


def _hybrid_sim(P, inp):
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"])
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=inp["ppc"], to_species=[0, 1], policy="default")
    return sim


def _hybrid_inp():
    from paper_2510_11174_gb300 import inputs
    inp = inputs.ramp_slab(nx=64, ny=32, nz=32, vacuum_lambda=0.25, slab_lambda=0.5, a0=6.0, tile_capacity=16384,
                           ppc=4)
    inp["laser"].update(t_peak=6.0, tau_fwhm=6.0, w0_spot=6.0)
    return inp


def _advance(sim, steps, every=10):
    """Steps with a physics-criterion classification (and conversions) every `every` steps."""
    for _ in range(steps):
        if sim.diagnostics()["step"] % every == 0:
            sim.classify()
        sim.step(1)


def _snapshot(sim, nsp, nfl):
    E, B, J = sim.get_fields()
    parts = [by_id(sim.get_species(s)) for s in range(nsp)]
    fl = [sim.get_fluid(f) for f in range(nfl)]
    mask, rho_bg = sim.get_regime()
    return E, B, J, parts, fl, mask, rho_bg


def _same_snapshot(a, b):
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    for x, y in zip(a[3], b[3]):
        assert np.array_equal(x["ids"], y["ids"])
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            assert np.array_equal(x[k].view(np.uint32), y[k].view(np.uint32)), k
    for x, y in zip(a[4], b[4]):
        for k in ("n", "ux", "uy", "uz"):
            assert np.array_equal(x[k].view(np.uint32), y[k].view(np.uint32)), k
    assert np.array_equal(a[5], b[5])
    assert np.array_equal(a[6].view(np.uint32), b[6].view(np.uint32))


def test_hybrid_with_conversions_runs_twice_bit_for_bit():
    """Fluid <-> particle conversions (criterion, dilation, CIC moments, residual
    charge) repeat bit for bit as well."""
    from _util import require_gpu
    P = require_gpu()
    inp = _hybrid_inp()
    snaps = []
    for _ in range(2):
        sim = _hybrid_sim(P, inp)
        _advance(sim, 35)
        snaps.append(_snapshot(sim, 2, 2))
        assert sum(sim.diagnostics()["count"]) > 0
        sim.close()
    _same_snapshot(snaps[0], snaps[1])


def test_checkpoint_restore_continues_bit_for_bit():
    """25 steps, save, restore into a fresh context, 25 more steps (with
    classifications at steps 0, 10, 20, 30, 40) equals 50 uninterrupted steps."""
    from _util import require_gpu
    from paper_2510_11174_gb300._abi import HybError, HYB_EINVAL
    P = require_gpu()
    inp = _hybrid_inp()
    ref = _hybrid_sim(P, inp)
    _advance(ref, 50)
    want = _snapshot(ref, 2, 2)
    dref = ref.diagnostics()
    ref.close()

    a = _hybrid_sim(P, inp)
    _advance(a, 25)
    image = a.get_state()
    a.close()
    b = _hybrid_sim(P, inp)
    b.set_state(image)
    assert b.diagnostics()["step"] == 25
    _advance(b, 25)
    _same_snapshot(_snapshot(b, 2, 2), want)
    d = b.diagnostics()
    assert d["count"] == dref["count"] and d["step"] == dref["step"] == 50
    assert d["w_e"] == dref["w_e"] and d["w_b"] == dref["w_b"]
    b.close()
    # an image does not go into a context of another grid
    from paper_2510_11174_gb300 import inputs
    other = inputs.ramp_slab(nx=32, ny=32, nz=32, vacuum_lambda=0.25, slab_lambda=0.5, a0=6.0, ppc=4)
    c = _hybrid_sim(P, other)
    with pytest.raises(HybError) as ei:
        c.set_state(image)
    assert ei.value.code == HYB_EINVAL
    c.close()


def test_periodic_plasma_checkpoint_50_plus_50_is_100():
    from paper_2510_11174_gb300 import inputs
    inp = inputs.periodic_plasma(n=32, ppc=8, seed=6, a0=2.0, temperature_keV=10.0)
    want = _run(inp, 100)
    sim, _ = make_pair(inp, with_oracle=False)
    sim.step(50)
    image = sim.get_state()
    sim.close()
    sim2, _ = make_pair(inp, with_oracle=False)
    sim2.set_state(image)
    sim2.step(50)
    E, B, J = sim2.get_fields()
    parts = [by_id(sim2.get_species(s)) for s in range(2)]
    got = (E, B, J, parts, sim2.diagnostics())
    sim2.close()
    _same(got, want)
