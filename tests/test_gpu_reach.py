"""Classification restricted to the nodes near matter (hyb_regime_desc.reach).

The classifier then runs only on the x-range within reach + dilate nodes of an
x-plane holding matter and reports p_mean = p_std = 0 elsewhere.  With the
next classification at most reach - 1 steps away, matter cannot reach a node
whose decision was not computed, so the run must be the same, bit for bit, as
the run that classifies every node: fields, fluids, particles (ids and
momenta), the conversions' background charge.  Inside the range the MC
statistics equal the whole-grid ones exactly (the layers compute the same
outputs from the same inputs)."""
import numpy as np
import pytest

from _util import by_id, require_gpu, seeded_classifier

pytestmark = pytest.mark.gpu

EVERY = 5          # steps between classifications
REACH = EVERY + 1  # nodes: fluid moves at most one node per step, particles less, plus their CIC node


def _workload():
    from paper_2510_11174_gb300 import inputs
    # vacuum in x = 0..15, ramp 16..31, slab 32..39, vacuum 40..63
    inp = inputs.ramp_slab(nx=64, ny=16, nz=16, vacuum_lambda=1.0, slab_lambda=0.5, a0=8.0, tile_capacity=16384,
                           ppc=2)
    inp["laser"]["t_peak"] = 6.0
    inp["laser"]["tau_fwhm"] = 6.0
    inp["laser"]["w0_spot"] = 6.0
    return inp


def _sim(P, inp, reach):
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"])
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=inp["ppc"], to_species=[0, 1], policy="union", reach=reach)
    return sim


def _matter_range(sim, inp, R):
    """[lo, hi) of the x-planes within R of a plane holding matter (a fluid above
    its floor, or a particle in a cell of the plane)."""
    nx = inp["grid"]["nx"]
    hold = np.zeros(nx, dtype=bool)
    for f, fl in enumerate(inp["fluids"]):
        hold |= (sim.get_fluid(f)["n"] > fl["n_floor"]).any(axis=(0, 1))
    for s in range(len(inp["species"])):
        x = sim.get_species(s)["x"]
        if x.size:
            hold[np.clip(np.floor(x).astype(np.int64), 0, nx - 1)] = True
    planes = np.nonzero(hold)[0]
    return max(0, planes.min() - R), min(nx, planes.max() + 1 + R)


def test_reach_restricted_classification_repeats_the_whole_grid_run():
    P = require_gpu()
    import torch
    inp = _workload()
    g = inp["grid"]
    model, _ = seeded_classifier(P, 9, out_bias=-2.0, dropout=0.2, mc_passes=4)
    full, near = _sim(P, inp, 0), _sim(P, inp, REACH)
    cells = g["nx"] * g["ny"] * g["nz"]
    restricted = 0
    for cycle in range(4):
        lo, hi = _matter_range(near, inp, REACH + 1)
        restricted += lo > 0 or hi < g["nx"]
        outs = []
        for sim in (full, near):
            pm = torch.empty(cells, dtype=torch.float32, device="cuda")
            ps = torch.empty(cells, dtype=torch.float32, device="cuda")
            sim.classify(model, p_mean=pm, p_std=ps)
            torch.cuda.synchronize()
            shape = (g["nz"], g["ny"], g["nx"])
            outs.append((pm.cpu().numpy().reshape(shape), ps.cpu().numpy().reshape(shape)))
        (pm_f, ps_f), (pm_n, ps_n) = outs
        # inside the range the statistics are the whole grid's; outside they are zero
        assert np.array_equal(pm_n[:, :, lo:hi], pm_f[:, :, lo:hi]), cycle
        assert np.array_equal(ps_n[:, :, lo:hi], ps_f[:, :, lo:hi]), cycle
        assert not pm_n[:, :, :lo].any() and not pm_n[:, :, hi:].any(), cycle
        assert not ps_n[:, :, :lo].any() and not ps_n[:, :, hi:].any(), cycle
        assert pm_f[:, :, :lo].any() or pm_f[:, :, hi:].any() or (lo == 0 and hi == g["nx"])
        full.step(EVERY)
        near.step(EVERY)
        # the same run: fields, fluids, particles, background charge
        for a, b in zip(full.get_fields(), near.get_fields()):
            assert np.array_equal(a, b), cycle
        for f in range(2):
            fa, fb = full.get_fluid(f), near.get_fluid(f)
            for k in fa:
                assert np.array_equal(fa[k], fb[k]), (cycle, f, k)
        for s in range(2):
            sa, sb = by_id(full.get_species(s)), by_id(near.get_species(s))
            for k in sa:
                assert np.array_equal(sa[k], sb[k]), (cycle, s, k)
        assert np.array_equal(full.get_regime()[1], near.get_regime()[1]), cycle
    assert restricted >= 3  # the workload keeps vacuum on both sides of the matter
    d = near.diagnostics()
    assert d["status"] == 0
    assert sum(d["count"]) > 0  # conversions happened
    full.close()
    near.close()
    model.close()


def test_reach_without_matter_classifies_nothing():
    """No fluid above its floor and no particle: nothing to classify, the
    statistics are zero everywhere, and a negative reach is rejected."""
    P = require_gpu()
    import torch
    inp = _workload()
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"])
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**dict(fl, n=np.zeros_like(fl["n"])))
    with pytest.raises(Exception):
        sim.set_regime(dilate=1, ppc=inp["ppc"], to_species=[0, 1], policy="union", reach=-1)
    sim.set_regime(dilate=1, ppc=inp["ppc"], to_species=[0, 1], policy="union", reach=REACH)
    model, _ = seeded_classifier(P, 9, out_bias=-2.0, dropout=0.2, mc_passes=4)
    cells = g["nx"] * g["ny"] * g["nz"]
    pm = torch.full((cells,), 7.0, dtype=torch.float32, device="cuda")
    ps = torch.full((cells,), 7.0, dtype=torch.float32, device="cuda")
    sim.classify(model, p_mean=pm, p_std=ps)
    torch.cuda.synchronize()
    assert not pm.any().item() and not ps.any().item()
    d = sim.diagnostics()
    assert d["classified_cells"] == 0 and d["status"] == 0
    sim.close()
    model.close()


def test_reach_on_a_periodic_axis_keeps_every_plane_when_the_range_wraps():
    """A periodic box with fluid near x = 0: the range near matter would wrap
    round, so the classifier runs on every plane and its statistics equal the
    whole grid's everywhere."""
    P = require_gpu()
    import torch
    nx, ny, nz, dx = 64, 16, 16, 0.3
    n = np.zeros((nz, ny, nx), np.float32)
    n[:, :, 1:4] = 0.5
    rng = np.random.default_rng(8)
    E = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    B = (0.3 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
    model, _ = seeded_classifier(P, 9, out_bias=-2.0, dropout=0.2, mc_passes=4)
    outs = []
    for reach in (0, REACH):
        sim = P.Simulation(nx, ny, nz, dx, cfl_frac=0.95, bc=(0, 0, 0))
        sim.load_fluid(q=-1.0, m=1.0, n=n, n_floor=1e-10)
        sim.set_fields(E, B)
        sim.set_regime(dilate=1, ppc=2, to_species=[], policy="default", reach=reach)
        pm = torch.empty(nx * ny * nz, dtype=torch.float32, device="cuda")
        sim.classify(model, p_mean=pm)
        torch.cuda.synchronize()
        outs.append(pm.cpu().numpy())
        assert sim.diagnostics()["classified_cells"] == nx * ny * nz
        sim.close()
    assert np.array_equal(outs[0], outs[1])
    model.close()


def test_fluid_range_lapses_after_reach_steps():
    """A classification with reach 3 restricts the fluid update for 3 steps
    only: stepping 12 steps past it (the restriction lifted after 3) repeats
    the run without a reach bit for bit."""
    P = require_gpu()
    inp = _workload()
    model, _ = seeded_classifier(P, 9, out_bias=-2.0, dropout=0.2, mc_passes=4)
    runs = []
    for reach in (0, 3):
        sim = _sim(P, inp, reach)
        sim.classify(model)
        sim.step(4)                 # a step since the fluids were loaded: the next range is taken
        sim.classify(model)
        d = sim.diagnostics()
        g = inp["grid"]
        assert (d["fluid_cells"] < g["nx"] * g["ny"] * g["nz"]) == (reach > 0) and d["status"] == 0
        sim.step(12)
        runs.append((sim.get_fields(), [sim.get_fluid(f) for f in range(2)],
                     [by_id(sim.get_species(s)) for s in range(2)], sim.diagnostics()))
        sim.close()
    (fa, la, pa, da), (fb, lb, pb, db) = runs
    assert db["fluid_cells"] == da["fluid_cells"] == inp["grid"]["nx"] * inp["grid"]["ny"] * inp["grid"]["nz"]
    for a, b in zip(fa, fb):
        assert np.array_equal(a, b)
    for f in range(2):
        for k in la[f]:
            assert np.array_equal(la[f][k], lb[f][k]), (f, k)
    for s in range(2):
        for k in pa[s]:
            assert np.array_equal(pa[s][k], pb[s][k]), (s, k)
    model.close()
