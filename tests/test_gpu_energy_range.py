"""The FP64 energy diagnostics over twelve decades of momentum (Methodology:
total energy from the kinetic parts, checked during the steps).

The library forms each particle's term w (gamma - 1) (w |k| for photons) in
double-float arithmetic on the FP32 units and sums the block partials in
FP64; here electrons and photons with |u| log-uniform in [1e-6, 1e6] are
loaded as FP32 and the diagnostics at step 0 are compared with the oracle's
FP64 sum over the same FP32 values (and, for photons, the FP64 sum of
w |k|), to the same 1e-12 relative bound as the step's energy checks.
"""
import numpy as np
import pytest

import oracle
from _util import require_gpu

pytestmark = pytest.mark.gpu


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _particles(rng, n, nx):
    pos = [_f32(rng.uniform(0.0, nx - 1.0, n)) for _ in range(3)]
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = _f32(d * (10.0 ** rng.uniform(-6.0, 6.0, n))[:, None])
    w = _f32(rng.uniform(0.1, 2.0, n))
    return pos, u, w


def test_kinetic_energy_over_twelve_decades_of_momentum():
    P = require_gpu()
    rng = np.random.default_rng(12)
    n, nx = 200_000, 32
    sim = P.Simulation(nx, nx, nx, 0.3)
    (xe, ye, ze), ue, we = _particles(rng, n, nx)
    sim.load_species(q=-1.0, m=1.0, x=xe, y=ye, z=ze, ux=_f32(ue[:, 0]), uy=_f32(ue[:, 1]), uz=_f32(ue[:, 2]),
                     w=we, tile_capacity=8192)
    (xp, yp, zp), up, wp = _particles(rng, n, nx)
    sim.load_species(q=0.0, m=0.0, kind=1, x=xp, y=yp, z=zp, ux=_f32(up[:, 0]), uy=_f32(up[:, 1]),
                     uz=_f32(up[:, 2]), w=wp, tile_capacity=8192)
    d = sim.diagnostics()
    sim.close()
    assert d["count"][0] == n and d["count"][1] == n
    ref_e = oracle.energy_particles(oracle.Particles(-1.0, 1.0, xe, ye, ze, ue[:, 0], ue[:, 1], ue[:, 2], we))
    u64 = up.astype(np.float64)
    ref_p = float(np.sum(wp.astype(np.float64) * np.sqrt(np.sum(u64 * u64, axis=1))))
    assert d["w_kin"][0] == pytest.approx(ref_e, rel=1e-12)
    assert d["w_kin"][1] == pytest.approx(ref_p, rel=1e-12)
