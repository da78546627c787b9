"""The Vay and Higuera-Cary pushers on the GPU against the oracle's: one
step of relativistic particles in strong random fields (per-particle
momentum within 1e-5), and the relativistic E x B drift held for 100 steps
(a force-free particle keeps its momentum), which Boris does not hold."""
import math

import numpy as np
import pytest

from _util import by_id, make_pair

pytestmark = pytest.mark.gpu


def _strong_case(pusher, n=16, count=3000, seed=4):
    rng = np.random.default_rng(seed)
    f32 = lambda a: np.asarray(a, np.float32)
    pos = lambda: f32(np.minimum(rng.uniform(0, n, count), n - 1e-3))
    sp = dict(q=-1.0, m=1.0, x=pos(), y=pos(), z=pos(), ux=f32(rng.normal(0, 20, count)),
              uy=f32(rng.normal(0, 20, count)), uz=f32(rng.normal(0, 20, count)),
              w=f32(np.full(count, 1e-4)), pusher=pusher)
    E = f32(30.0 * rng.standard_normal((3, n, n, n)))
    B = f32(30.0 * rng.standard_normal((3, n, n, n)))
    return dict(grid=dict(nx=n, ny=n, nz=n, dx=2 * math.pi / 16), species=[sp], E=E, B=B)


@pytest.mark.parametrize("pusher", ["vay", "higuera_cary", "boris"])
def test_one_step_momentum_matches_oracle(pusher):
    inp = _strong_case(pusher)
    sim, orc = make_pair(inp)
    sim.step(1)
    orc.step(1)
    g = by_id(sim.get_species(0))
    o = orc.species[0]
    k = np.argsort(o.ids)
    ug = np.stack([g["ux"], g["uy"], g["uz"]]).astype(np.float64)
    uo = np.stack([o.ux[k], o.uy[k], o.uz[k]])
    rel = np.linalg.norm(ug - uo, axis=0) / np.linalg.norm(uo, axis=0)
    assert rel.max() <= 1e-5, rel.max()
    sim.close()


def test_relativistic_exb_drift_is_held_by_vay_and_higuera_cary():
    n, B0, vd = 16, 40.0, 0.95
    g = 1.0 / math.sqrt(1.0 - vd * vd)
    E = np.zeros((3, n, n, n), np.float32)
    B = np.zeros_like(E)
    E[1] = vd * B0
    B[2] = B0
    rng = np.random.default_rng(1)
    count = 512
    f32 = lambda a: np.asarray(a, np.float32)
    drift = {}
    for pusher in ("vay", "higuera_cary", "boris"):
        sp = dict(q=-1.0, m=1.0, x=f32(rng.uniform(0, n - 1e-3, count)), y=f32(rng.uniform(0, n - 1e-3, count)),
                  z=f32(rng.uniform(0, n - 1e-3, count)), ux=f32(np.full(count, g * vd)), uy=f32(np.zeros(count)),
                  uz=f32(np.zeros(count)), w=f32(np.zeros(count)), pusher=pusher)
        sim, _ = make_pair(dict(grid=dict(nx=n, ny=n, nz=n, dx=2 * math.pi / 16), species=[sp], E=E, B=B),
                           with_oracle=False)
        sim.step(100)
        s = sim.get_species(0)
        drift[pusher] = float(np.max(np.abs(np.stack([s["ux"] - g * vd, s["uy"], s["uz"]]))) / g)
        sim.close()
    assert drift["vay"] < 1e-4 and drift["higuera_cary"] < 1e-4, drift
    assert drift["boris"] > 1e-2, drift
