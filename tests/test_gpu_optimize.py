"""The laser-parameter search on the GPU: the tile autotuner times both tile
edges, and differential evolution over (a0, tau, spot) advances each
population as one batch of hybrid runs and moves toward the target energy
of a reference pulse (Introduction; closing paragraph of the Results)."""
import numpy as np
import pytest

from _util import require_gpu

pytestmark = pytest.mark.gpu


def test_laser_scan_differential_evolution_reaches_toward_the_target():
    require_gpu()
    from paper_2510_11174_gb300.optimize import LaserScan
    scan = LaserScan(nx=32, ny=16, nz=16, ppc=4, steps=120, autotune=True)
    assert scan.tile in (4, 8) and set(scan.tile_times) == {4, 8}
    assert all(v > 0 for v in scan.tile_times.values())
    # the target is the energy a reference pulse deposits
    ref = scan.energies(np.array([[12.0, 6.0, 1.5]]))[0]
    assert ref > 0
    scan.target = ref
    res = scan.optimize(lo=(2.0, 3.0, 0.75), hi=(30.0, 10.0, 3.0), pop=6, generations=3, seed=2)
    h = res["history"]
    assert all(b <= a for a, b in zip(h, h[1:]))
    assert res["f"] < 0.5 and res["f"] <= h[0]
    assert scan.evaluations == 1 + 6 * 4
    # the same parameters give the same energy (each run is deterministic)
    again = scan.energies(res["x"][None])[0]
    assert abs(again - ref) / ref == pytest.approx(res["f"], rel=1e-6, abs=1e-9)
