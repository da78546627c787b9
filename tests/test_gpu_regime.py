"""GPU regime switching against the oracle: the physics criterion mask, the
fluid -> particle conversion (same Philox positions and ids), the particle ->
fluid deposit, and the Gauss-law invariant kept by the residual background
charge across conversions."""
import math

import numpy as np
import pytest

import oracle
from _util import by_id, make_pair, rel_l2

pytestmark = pytest.mark.gpu

NX, NY, NZ, DX = 16, 16, 8, 0.3


def _setup(seed=1):
    rng = np.random.default_rng(seed)
    shape = (NZ, NY, NX)
    E = (0.05 * rng.standard_normal((3,) + shape)).astype(np.float32)
    E[1, 2:5, 3:7, 4:9] = 2.5  # a relativistic-field pocket
    B = np.zeros_like(E)
    n = (0.3 + 0.05 * rng.random(shape)).astype(np.float32)
    n[6, 12, 12] = 2.0          # a density spike
    u = (0.02 * rng.standard_normal((3,) + shape)).astype(np.float32)
    m = 3000
    pos = lambda hi: np.minimum(rng.uniform(0, hi, m).astype(np.float32), np.float32(hi - 1e-3))
    electrons = dict(q=-1.0, m=1.0, x=pos(NX), y=pos(NY), z=pos(NZ),
                     ux=(0.05 * rng.standard_normal(m)).astype(np.float32),
                     uy=(0.05 * rng.standard_normal(m)).astype(np.float32),
                     uz=(0.05 * rng.standard_normal(m)).astype(np.float32),
                     w=np.full(m, 1e-4, np.float32), tile_capacity=8192)
    inp = dict(grid=dict(nx=NX, ny=NY, nz=NZ, dx=DX), E=E, B=B, species=[electrons])
    return inp, dict(q=-1.0, m=1.0, n=n, ux=u[0], uy=u[1], uz=u[2])


def _gauss(g, E, species_list, fluids, rho_bg):
    rho = np.zeros(g.shape)
    for sp in species_list:
        oracle.charge_density(g, sp, rho)
    for q, n in fluids:
        rho += q * n.astype(np.float64)
    return oracle.div_e(g, E.astype(np.float64)) - rho - rho_bg.astype(np.float64)


@pytest.mark.parametrize("quiet", [False, True])
def test_physics_criterion_and_conversions_match_oracle(quiet):
    inp, fl = _setup()
    sim, _ = make_pair(inp, with_oracle=False)
    sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=4, to_species=[0], quiet=quiet)
    g = oracle.Grid.make(NX, NY, NZ, DX, DX, DX, 0.1)
    sp0 = sim.get_species(0)
    before = _gauss(g, inp["E"], [oracle.Particles(-1, 1, sp0["x"], sp0["y"], sp0["z"], sp0["ux"], sp0["uy"], sp0["uz"],
                                                   sp0["w"])], [(-1.0, fl["n"])], np.zeros(g.shape))
    sim.classify()
    mask, rho_bg = sim.get_regime()
    # the oracle's criterion on the same state (electron density: fluid + CIC of the particles)
    ne = fl["n"].astype(np.float64) + oracle.charge_density(
        g, oracle.Particles(1, 1, sp0["x"], sp0["y"], sp0["z"], sp0["ux"], sp0["uy"], sp0["uz"], sp0["w"]))
    om = oracle.regime_criterion(g, inp["E"].astype(np.float64), inp["B"].astype(np.float64), ne,
                                 fluid_u=np.stack([fl["ux"], fl["uy"], fl["uz"]]).astype(np.float64), dilate=1)
    assert np.count_nonzero(mask != om) <= 2, np.count_nonzero(mask != om)
    assert 0 < mask.mean() < 1
    # conversions with the GPU's mask in the oracle
    ofl = oracle.Fluid(-1.0, 1.0, fl["n"], np.stack([fl["ux"], fl["uy"], fl["uz"]]))
    orho = np.zeros(g.shape)
    new = oracle.fluid_to_particles(g, mask, ofl, 4, 1, 0, 0, orho, quiet=quiet)
    osp = oracle.Particles(-1, 1, sp0["x"], sp0["y"], sp0["z"], sp0["ux"], sp0["uy"], sp0["uz"], sp0["w"],
                           ids=sp0["ids"])
    osp.append(new)
    oracle.particles_to_fluid(g, mask, osp, ofl)
    gsp = by_id(sim.get_species(0))
    assert np.array_equal(gsp["ids"], np.sort(osp.ids))
    o = np.argsort(osp.ids)
    for k in ("x", "y", "z", "ux", "w"):
        assert np.allclose(gsp[k], getattr(osp, k)[o], rtol=1e-6, atol=1e-6), k
    gf = sim.get_fluid(0)
    assert rel_l2(gf["n"], ofl.n) <= 1e-5
    assert rel_l2(rho_bg, orho) <= 1e-5
    # Gauss's law with the residual background charge is unchanged by the conversions
    after = _gauss(g, inp["E"], [oracle.Particles(-1, 1, gsp["x"], gsp["y"], gsp["z"], gsp["ux"], gsp["uy"],
                                                  gsp["uz"], gsp["w"])], [(-1.0, gf["n"])], rho_bg)
    assert np.max(np.abs(after - before)) <= 1e-5 * np.max(np.abs(fl["n"]))


def test_hybrid_steps_after_classification_keep_gauss_law():
    inp, fl = _setup(seed=2)
    sim, _ = make_pair(inp, with_oracle=False)
    sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=4, to_species=[0])
    g = oracle.Grid.make(NX, NY, NZ, DX, DX, DX, 0.1)
    sim.classify()
    def gauss():
        E, _, _ = sim.get_fields()
        s = sim.get_species(0)
        mask, rho_bg = sim.get_regime()
        return _gauss(g, E, [oracle.Particles(-1, 1, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"])],
                      [(-1.0, sim.get_fluid(0)["n"])], rho_bg)
    r0 = gauss()
    for _ in range(3):
        sim.step(5)
        sim.classify()
    assert np.max(np.abs(gauss() - r0)) <= 2e-5 * np.max(np.abs(fl["n"]))


def _mask_with(policy, model_seed=None, seed=3):
    from paper_2510_11174_gb300.model import Classifier
    inp, fl = _setup(seed=seed)
    sim, _ = make_pair(inp, with_oracle=False)
    sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=2, to_species=[0], policy=policy)
    model = None
    if model_seed is not None:
        model = Classifier(dropout=0.2, mc_passes=4, seed=model_seed)
        w, b = model.get_layer(3)
        model.set_layer(3, w, np.full_like(b, -1.0))
    sim.classify(model)
    mask, _ = sim.get_regime()
    return mask


def test_union_policy_is_the_union_of_classifier_and_criterion():
    # dilation commutes with the union, so the three masks of the same state obey
    # union = criterion | classifier exactly
    phys = _mask_with("default")
    cls = _mask_with("default", model_seed=5)
    uni = _mask_with("union", model_seed=5)
    assert 0 < cls.mean() < 1 and 0 < phys.mean() < 1
    assert np.array_equal(uni, phys | cls)


def test_all_kinetic_policy_converts_every_fluid_node_and_drops_the_fluid_phase():
    inp, fl = _setup(seed=4)
    sim, _ = make_pair(inp, with_oracle=False)
    sim.load_fluid(**fl)
    sim.step(1)
    launches_hybrid = sim.diagnostics()["launches_per_step"]
    n0 = sim.diagnostics()["count"][0]
    sim.set_regime(dilate=0, ppc=3, to_species=[0], policy="all_kinetic")
    g = oracle.Grid.make(NX, NY, NZ, DX, DX, DX, 0.1)
    sp0 = sim.get_species(0)
    E0, _, _ = sim.get_fields()
    fl0 = sim.get_fluid(0)["n"]
    before = _gauss(g, E0, [oracle.Particles(-1, 1, sp0["x"], sp0["y"], sp0["z"], sp0["ux"], sp0["uy"], sp0["uz"],
                                             sp0["w"])], [(-1.0, fl0)], np.zeros(g.shape))
    sim.classify()
    mask, rho_bg = sim.get_regime()
    assert mask.all()
    assert np.all(sim.get_fluid(0)["n"] == 0.0)
    d = sim.diagnostics()
    assert d["count"][0] == n0 + 3 * np.count_nonzero(fl0 > 0)
    sp1 = sim.get_species(0)
    after = _gauss(g, E0, [oracle.Particles(-1, 1, sp1["x"], sp1["y"], sp1["z"], sp1["ux"], sp1["uy"], sp1["uz"],
                                            sp1["w"])], [(-1.0, sim.get_fluid(0)["n"])], rho_bg)
    assert np.max(np.abs(after - before)) <= 1e-5 * np.max(np.abs(fl["n"]))
    sim.step(2)
    d = sim.diagnostics()
    assert d["status"] == 0
    assert d["launches_per_step"] == launches_hybrid - 2
    # every node still holds particles of its own dual cell only: ids unique
    ids = sim.get_species(0)["ids"]
    assert len(np.unique(ids)) == len(ids)
