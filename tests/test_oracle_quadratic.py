"""Pins of the oracle's quadratic (TSC) particle shape and its Esirkepov
deposition: the shape is a partition of unity with zero first moment and
second moment 1/4 (the quadratic B-spline), the deposited current satisfies
the discrete continuity equation with the same shape's charge density to
round-off, and a particle's total current is q w dx / dt along its motion."""
import numpy as np
import pytest

import oracle


def _tsc(d):
    return np.array([oracle.lib().orc_tsc(float(v)) for v in np.atleast_1d(d)])


def test_tsc_moments():
    for p in np.random.default_rng(1).uniform(-3, 3, 50):
        m = np.floor(p + 0.5)
        nodes = m + np.arange(-2, 3)
        w = _tsc(p - nodes)
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        assert (w * (nodes - p)).sum() == pytest.approx(0.0, abs=1e-15)
        assert (w * (nodes - p) ** 2).sum() == pytest.approx(0.25, abs=1e-14)
        assert w[0] == 0.0 and w[4] == 0.0


@pytest.mark.parametrize("order", [1, 2])
def test_quadratic_esirkepov_keeps_discrete_continuity(order):
    g = oracle.Grid.make(12, 10, 8, 0.4, 0.4, 0.4, 0.2, bc=(0, 0, 0), order=order)
    rng = np.random.default_rng(4)
    n = 400
    sp = oracle.Particles(-1.0, 1.0, rng.uniform(0, 12, n), rng.uniform(0, 10, n), rng.uniform(0, 8, n),
                          *(2.0 * rng.standard_normal((3, n))), rng.uniform(0.5, 1.5, n))
    rho0 = oracle.charge_density(g, sp)
    E, B, J = oracle.zeros_field(g), oracle.zeros_field(g), oracle.zeros_field(g)
    oracle.push_deposit(g, E, B, J, sp)
    rho1 = oracle.charge_density(g, sp)
    # div J at the nodes (J_a at i + 1/2 along a, backward differences)
    div = np.zeros(g.shape)
    for a, d in enumerate((g.dx, g.dy, g.dz)):
        div += (J[a] - np.roll(J[a], 1, axis=2 - a)) / d
    assert np.max(np.abs((rho1 - rho0) / g.dt + div)) < 1e-12 * np.max(np.abs(rho0))


def test_quadratic_single_particle_total_current():
    g = oracle.Grid.make(8, 8, 8, 0.5, 0.5, 0.5, 0.25, bc=(0, 0, 0), order=2)
    for x0, u in (((3.3, 4.6, 2.1), (0.6, 0.0, 0.0)), ((3.9, 4.45, 2.55), (1.5, -0.9, 2.0))):
        sp = oracle.Particles(1.0, 1.0, [x0[0]], [x0[1]], [x0[2]], [u[0]], [u[1]], [u[2]], [0.7])
        J = oracle.zeros_field(g)
        oracle.push_deposit(g, oracle.zeros_field(g), oracle.zeros_field(g), J, sp)
        dV = 0.5 ** 3
        for a, p in enumerate((sp.x, sp.y, sp.z)):
            moved = (p[0] - x0[a]) * 0.5
            assert J[a].sum() * dV == pytest.approx(0.7 * moved / 0.25, rel=1e-12)
