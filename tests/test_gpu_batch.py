"""Batches of independent runs (hyb_batch_*): contexts of uneven sizes and
kinds advanced as one graph match the same contexts advanced one by one (the
shared-memory current atomics leave round-off differences only), and work on
a context's own stream stays ordered around the batch."""
import numpy as np
import pytest

from paper_2510_11174_gb300 import inputs
from _util import make_pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _hybrid(P, seed):
    inp = inputs.ramp_slab(nx=32, ny=16, nz=16, vacuum_lambda=0.25, slab_lambda=0.5, a0=3.0, seed=seed,
                           tile_capacity=8192, ppc=4)
    inp["laser"].update(t_peak=6.0, tau_fwhm=6.0, w0_spot=6.0)
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"], laser=inp["laser"])
    for sp in inp["species"]:
        sim.load_species(**sp)
    for fl in inp["fluids"]:
        sim.load_fluid(**fl)
    sim.set_regime(dilate=1, ppc=inp["ppc"], to_species=[0, 1])
    sim.classify()
    return sim


def _runs(P):
    sims = [make_pair(inputs.periodic_plasma(n=n, ppc=4, seed=s), with_oracle=False)[0]
            for n, s in ((16, 1), (24, 2), (32, 3))]
    sims.append(_hybrid(P, 4))
    return sims


def _state(sim):
    E, B, _ = sim.get_fields()
    return np.concatenate([E.ravel(), B.ravel()]), sim.diagnostics()["count"]


def test_batch_matches_individual_runs():
    P = require_gpu()
    batched, alone = _runs(P), _runs(P)
    b = P.Batch(batched)
    for _ in range(3):
        b.step(7)
        batched[3].classify()
        for s in alone[:3]:
            s.step(7)
        alone[3].step(7)
        alone[3].classify()
    for sb, sa in zip(batched, alone):
        fb, cb = _state(sb)
        fa, ca = _state(sa)
        assert cb == ca
        assert rel_l2(fb, fa) <= 1e-5, rel_l2(fb, fa)
        assert sb.diagnostics()["step"] == 21
    # a context keeps stepping on its own after the batch
    batched[0].step(2)
    alone[0].step(2)
    assert rel_l2(_state(batched[0])[0], _state(alone[0])[0]) <= 1e-5
    b.close()


def test_batch_rejects_duplicates():
    P = require_gpu()
    sims = _runs(P)[:2]
    with pytest.raises(P.HybError):
        P.Batch([sims[0], sims[0]])
