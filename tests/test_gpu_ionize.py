"""GPU field ionization against the oracle: the FP64-built rate table against
the direct formula, and the Monte Carlo events on shared Philox streams
(per-event mismatch <= 1e-4, counts within 3 sigma)."""
import math

import numpy as np
import pytest

import oracle
from _util import by_id, make_pair, rel_l2

pytestmark = pytest.mark.gpu

CARBON_IP = [11.260, 24.383, 47.888, 64.494, 392.09, 489.99]
CARBON_L = [1, 1, 0, 0, 0, 0]
M_C = 12 * 1836.15267343


def _carbon_case(n_ions=20000, Ey=0.0085, seed=3, n=16, zq0=0.0):
    rng = np.random.default_rng(seed)
    f32 = lambda v: np.asarray(v, np.float32)
    pos = lambda: np.minimum(rng.uniform(0, n, n_ions).astype(np.float32), np.float32(n - 1e-3))
    ions = dict(q=1.0, m=M_C, x=pos(), y=pos(), z=pos(), ux=f32(np.zeros(n_ions)), uy=f32(np.zeros(n_ions)),
                uz=f32(np.zeros(n_ions)), w=f32(np.full(n_ions, 1e-3)), zq=f32(np.full(n_ions, zq0)),
                ionize=dict(zmax=6, ip_eV=CARBON_IP, l=CARBON_L, into=0), tile_capacity=4096)
    e0 = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    electrons = dict(q=-1.0, m=1.0, tile_capacity=6 * 4096, **e0)
    E = np.zeros((3, n, n, n), np.float32)
    E[1] = Ey
    B = np.zeros_like(E)
    return dict(grid=dict(nx=n, ny=n, nz=n, dx=2 * math.pi / 20), species=[electrons, ions], E=E, B=B)


def test_rate_table_matches_direct_formula():
    sim, _ = make_pair(_carbon_case(n_ions=64), with_oracle=False)
    w0_au, er, dt_au = oracle.atomic_units(0.8e-6, sim.desc.dt if sim.desc.dt > 0 else 0.95 * (2 * math.pi / 20) / math.sqrt(3))
    F = np.geomspace(1e-3, 50.0, 3000).astype(np.float32)
    worst = 0.0
    for Z in range(6):
        w_gpu = sim.eval_rate_table(0, 1, Z, F).astype(np.float64)
        Ip = CARBON_IP[Z] / oracle.HARTREE_EV
        w_ref = np.array([oracle.ionization_rate(float(f), Ip, Z + 1, CARBON_L[Z], w0_au) for f in F])
        sel = w_ref * dt_au > 1e-8
        rel = np.abs(w_gpu[sel] - w_ref[sel]) / w_ref[sel]
        worst = max(worst, rel.max())
    assert worst <= 1e-5, worst


def test_one_step_events_match_oracle():
    inp = _carbon_case()
    sim, orc = make_pair(inp)
    sim.step(1)
    orc.step(1)
    gi = by_id(sim.get_species(1, with_zq=True))
    o = np.argsort(orc.species[1].ids)
    zq_o = orc.species[1].zq[o]
    mism = np.count_nonzero(gi["zq"] != zq_o)
    assert mism <= max(1, 1e-4 * len(zq_o)), mism
    # binomial law of the events
    w0_au, er, dt_au = oracle.atomic_units(0.8e-6, orc.g.dt)
    P = -math.expm1(-oracle.ionization_rate(0.0085 * er, CARBON_IP[0] / oracle.HARTREE_EV, 1, 1, w0_au) * dt_au)
    n = len(zq_o)
    k = int(np.count_nonzero(gi["zq"] == 1))
    assert 0.02 < P < 0.98
    assert abs(k - n * P) <= 3 * math.sqrt(n * P * (1 - P))
    # spawned electrons: same ids, positions and momenta as the oracle's
    ge = by_id(sim.get_species(0))
    oe = orc.species[0]
    oo = np.argsort(oe.ids)
    common = np.intersect1d(ge["ids"], oe.ids)
    assert len(common) >= len(oe.ids) - mism
    d = sim.diagnostics()
    assert d["n_ionize"] == k
    assert d["w_ionize"] == pytest.approx(orc.w_ionize * k / max(1, orc.n_ionize), rel=1e-9)


def test_multi_step_ionization_parity():
    inp = _carbon_case(Ey=0.02, n_ions=20000)
    sim, orc = make_pair(inp)
    for _ in range(3):
        sim.step(4)
        orc.step(4)
    gi = by_id(sim.get_species(1, with_zq=True))
    o = np.argsort(orc.species[1].ids)
    mism = np.count_nonzero(gi["zq"] != orc.species[1].zq[o])
    assert mism <= max(2, 1e-4 * len(o)), mism
    assert np.mean(gi["zq"]) > 1.0  # several levels per ion over the run
    d, od = sim.diagnostics(), orc.diagnostics()
    assert abs(d["n_ionize"] - od["n_ionize"]) <= mism
    assert abs(d["count"][0] - od["count"][0]) <= mism
    assert d["w_ionize"] == pytest.approx(od["w_ionize"], rel=1e-3)
    E, B, J = sim.get_fields()
    assert rel_l2(E, orc.E) <= 1e-4


def test_fully_ionized_and_neutral_edge_cases():
    inp = _carbon_case(n_ions=500, zq0=6.0)
    sim, orc = make_pair(inp)
    sim.step(2)
    orc.step(2)
    assert sim.diagnostics()["n_ionize"] == 0 == orc.n_ionize
