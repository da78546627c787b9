"""The quadratic (TSC) particle shape on the GPU against the oracle: one step
of a warm plasma in a plane wave (per-particle momentum within 1e-5, current
within 1e-5), 100 steps of fields within 1e-4, the discrete Gauss law held with
the same shape's charge density, and the descriptors it rejects."""
import numpy as np
import pytest

import oracle
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


def test_100_steps_fields_and_gauss_law():
    inp = _plasma(n=16, ppc=4, seed=5)
    sim, orc = _pair(inp)
    g = orc.g

    def rho(parts):
        r = np.zeros(g.shape)
        for (q, m), p in zip(((-1.0, 1.0), (1.0, 1836.15267343)), parts):
            oracle.charge_density(g, oracle.Particles(q, m, p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"],
                                                      p["w"]), r)
        return r

    E0 = sim.get_fields()[0]
    r0 = oracle.div_e(g, E0.astype(np.float64)) - rho([sim.get_species(s) for s in range(2)])
    for _ in range(4):
        sim.step(25)
        orc.step(25)
    E, B, _ = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4, rel_l2(E, orc.E)
    assert rel_l2(B, orc.B) <= 1e-4, rel_l2(B, orc.B)
    r1 = oracle.div_e(g, E.astype(np.float64)) - rho([sim.get_species(s) for s in range(2)])
    scale = np.max(np.abs(rho([sim.get_species(0)])))
    assert np.max(np.abs(r1 - r0)) <= 1e-5 * scale, (np.max(np.abs(r1 - r0)), scale)
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
