"""The quadratic (TSC) particle shape on the GPU against the oracle: one step
of a warm plasma in a plane wave (per-particle momentum within 1e-5, current
within 1e-5), 100 steps of fields within 1e-4, the discrete Gauss law held with
the same shape's charge density, and the descriptors it rejects."""
import numpy as np
import pytest

import oracle
import oracle.sim
from _util import by_id, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _pair(inp, order=2):
    P = require_gpu()
    import oracle.sim as S
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], shape_order=order, tile=4)
    orc = S.OracleSim(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], shape_order=order)
    for sp in inp["species"]:
        sim.load_species(**sp)
        orc.load_species(**sp)
    sim.set_fields(inp["E"], inp["B"])
    orc.set_fields(inp["E"], inp["B"])
    return sim, orc


def _plasma(n=16, ppc=4, seed=3):
    from paper_2510_11174_gb300 import inputs
    return inputs.periodic_plasma(n=n, ppc=ppc, seed=seed, a0=2.0, temperature_keV=20.0)


def test_one_step_matches_oracle():
    sim, orc = _pair(_plasma())
    sim.step(1)
    orc.step(1)
    for sid in range(2):
        g = by_id(sim.get_species(sid))
        o = orc.species[sid]
        k = np.argsort(o.ids)
        ug = np.stack([g["ux"], g["uy"], g["uz"]]).astype(np.float64)
        uo = np.stack([o.ux[k], o.uy[k], o.uz[k]])
        rel = np.linalg.norm(ug - uo, axis=0) / np.linalg.norm(uo, axis=0)
        assert rel.max() <= 1e-5, rel.max()
    E, B, J = sim.get_fields()
    assert rel_l2(J, orc.J) <= 1e-5, rel_l2(J, orc.J)
    sim.close()


def test_100_steps_fields_match_oracle():
    sim, orc = _pair(_plasma(n=16, ppc=4, seed=5))
    for _ in range(4):
        sim.step(25)
        orc.step(25)
    E, B, _ = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4, rel_l2(E, orc.E)
    assert rel_l2(B, orc.B) <= 1e-4, rel_l2(B, orc.B)
    sim.close()


def test_gauss_law_held_over_100_steps():
    """div E - rho, rho the quadratic shape's charge density, keeps its
    initial value.  The bound has the charge term of the linear-shape check
    and the FP32 rounding of E (each step rounds every component, and div E
    takes differences of them over dx), kept small by a weak wave."""
    inp = _plasma(n=16, ppc=4, seed=5)
    inp["E"] *= 0.1
    inp["B"] *= 0.1
    sim, _ = _pair(inp)
    g = oracle.sim.OracleSim(16, 16, 16, inp["grid"]["dx"], shape_order=2).g

    def residual():
        r = np.zeros(g.shape)
        for (q, m), s in zip(((-1.0, 1.0), (1.0, 1836.15267343)), range(2)):
            p = sim.get_species(s)
            oracle.charge_density(g, oracle.Particles(q, m, p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"],
                                                      p["w"]), r)
        scale = float(np.max(np.abs(r)))
        return oracle.div_e(g, sim.get_fields()[0].astype(np.float64)) - r, scale

    r0, scale = residual()
    sim.step(100)
    r1, _ = residual()
    emax = float(np.abs(sim.get_fields()[0]).max())
    err = float(np.max(np.abs(r1 - r0)))
    assert err <= 1e-5 * scale + 1e-6 * emax / g.dx, (err, scale, emax)
    sim.close()


def test_quadratic_shape_descriptor_checks():
    P = require_gpu()
    from paper_2510_11174_gb300._abi import HybError, HYB_EINVAL
    with pytest.raises(HybError) as ei:
        P.Simulation(16, 16, 16, 0.4, bc=(1, 0, 0), shape_order=2)
    assert ei.value.code == HYB_EINVAL
    with pytest.raises(HybError) as ei:
        P.Simulation(16, 16, 16, 0.4, shape_order=3)
    assert ei.value.code == HYB_EINVAL
