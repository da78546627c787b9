"""GPU cold relativistic fluid against the oracle: fluid + Maxwell over many
steps, the discrete Gauss law held by the face currents, and fluid coexisting
with particles (the hybrid configuration)."""
import math

import numpy as np
import pytest

import oracle
from _util import make_pair, rel_l2

pytestmark = pytest.mark.gpu


def _smooth(shape, rng, amp, base=0.0):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.full(shape, base)
    for _ in range(3):
        k = rng.integers(0, 3, 3)
        f += amp * rng.normal() * np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + rng.uniform(0, 6))
    return f.astype(np.float32)


def _fluid_case(bc=(0, 0, 0), seed=1, with_particles=False):
    rng = np.random.default_rng(seed)
    shape = (8, 16, 16)
    n = np.abs(_smooth(shape, rng, 0.05, 0.5)).astype(np.float32)
    u = [_smooth(shape, rng, 0.1) for _ in range(3)]
    E = np.stack([_smooth(shape, rng, 0.02) for _ in range(3)])
    B = np.stack([_smooth(shape, rng, 0.02) for _ in range(3)])
    inp = dict(grid=dict(nx=16, ny=16, nz=8, dx=0.35, bc=bc), E=E, B=B, species=[])
    if with_particles:
        m = 4000
        pos = lambda hi: np.minimum(rng.uniform(0, hi, m).astype(np.float32), np.float32(hi - 1e-3))
        inp["species"] = [dict(q=1.0, m=1836.15267343, x=pos(16), y=pos(16), z=pos(8),
                               ux=(0.01 * rng.standard_normal(m)).astype(np.float32),
                               uy=(0.01 * rng.standard_normal(m)).astype(np.float32),
                               uz=(0.01 * rng.standard_normal(m)).astype(np.float32),
                               w=np.full(m, 0.5 * 16 * 16 * 8 * 0.35 ** 3 / m, np.float32))]
    return inp, dict(q=-1.0, m=1.0, n=n, ux=u[0], uy=u[1], uz=u[2])


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0)])
def test_fluid_matches_oracle_over_50_steps(bc):
    inp, fl = _fluid_case(bc=bc)
    sim, orc = make_pair(inp)
    sim.load_fluid(**fl)
    orc.load_fluid(**fl)
    for _ in range(2):
        sim.step(25)
        orc.step(25)
    gf = sim.get_fluid(0)
    of = orc.fluids[0]
    assert rel_l2(gf["n"], of.n) <= 1e-5
    assert rel_l2(np.stack([gf["ux"], gf["uy"], gf["uz"]]), of.u) <= 1e-4
    E, B, J = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4 and rel_l2(B, orc.B) <= 1e-4
    d, od = sim.diagnostics(), orc.diagnostics()
    assert d["w_fluid"][0] == pytest.approx(od["w_fluid"][0], rel=1e-4)
    assert d["n_fluid"][0] == pytest.approx(float(of.n.sum()) * 0.35 ** 3, rel=1e-6)


def test_fluid_gauss_law_in_fp32():
    inp, fl = _fluid_case()
    sim, _ = make_pair(inp, with_oracle=False)
    sim.load_fluid(**fl)
    g = oracle.Grid.make(16, 16, 8, 0.35, 0.35, 0.35, 0.1)
    r0 = oracle.div_e(g, inp["E"].astype(np.float64)) + fl["n"]
    sim.step(40)
    E, _, _ = sim.get_fields()
    n1 = sim.get_fluid(0)["n"].astype(np.float64)
    r1 = oracle.div_e(g, E.astype(np.float64)) + n1
    assert np.max(np.abs(r1 - r0)) <= 1e-5 * np.max(np.abs(fl["n"]))


def test_fluid_and_particles_together():
    inp, fl = _fluid_case(with_particles=True, seed=4)
    sim, orc = make_pair(inp)
    sim.load_fluid(**fl)
    orc.load_fluid(**fl)
    sim.step(30)
    orc.step(30)
    E, B, J = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4
    assert rel_l2(sim.get_fluid(0)["n"], orc.fluids[0].n) <= 1e-5


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 0)])
def test_warm_electron_and_positron_fluids_match_oracle(bc):
    """A warm pair plasma (adiabatic pressure, Gamma = 5/3 and 3) against the
    oracle over 50 steps: densities, velocities and the fields they drive."""
    inp, fl = _fluid_case(bc=bc, seed=3)
    rng = np.random.default_rng(8)
    pos = dict(q=1.0, m=1.0, n=np.abs(_smooth((8, 16, 16), rng, 0.05, 0.4)).astype(np.float32),
               temperature_keV=20.0, gamma_ad=3.0, n_ref=0.4)
    fl.update(temperature_keV=5.0, gamma_ad=5.0 / 3.0, n_ref=0.5)
    sim, orc = make_pair(inp)
    for f in (fl, pos):
        sim.load_fluid(**f)
        orc.load_fluid(**f)
    for _ in range(2):
        sim.step(25)
        orc.step(25)
    for k in range(2):
        gf = sim.get_fluid(k)
        of = orc.fluids[k]
        assert rel_l2(gf["n"], of.n) <= 1e-5, k
        assert rel_l2(np.stack([gf["ux"], gf["uy"], gf["uz"]]), of.u) <= 1e-4, k
    E, B, J = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4 and rel_l2(B, orc.B) <= 1e-4
