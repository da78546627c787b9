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
