"""Pins of the oracle's cold relativistic fluid: exact discrete continuity
(Gauss's law invariant with the deposited face currents), particle-number
conservation, the exact impulse of a uniform field, and the linear Langmuir
oscillation at the plasma frequency w_p^2 = n (normalised units)."""
import math

import numpy as np
import pytest

import oracle


def _grid(nx=16, ny=8, nz=8, d=0.3, bc=(0, 0, 0)):
    dt = 0.9 / math.sqrt(3 / d ** 2)
    return oracle.Grid.make(nx, ny, nz, d, d, d, dt, bc=bc)


def _step(g, E, B, fluids):
    J = oracle.zeros_field(g)
    for fl in fluids:
        oracle.fluid_step(g, E, B, J, fl)
    oracle.fdtd_b_half(g, E, B)
    oracle.fdtd_e(g, E, B, J)
    oracle.fdtd_b_half(g, E, B)


def test_fluid_gauss_law_invariant_and_number_conservation():
    g = _grid()
    rng = np.random.default_rng(1)
    n = 0.5 + 0.3 * rng.random(g.shape)
    u = 0.2 * rng.standard_normal((3,) + g.shape)
    fl = oracle.Fluid(-1.0, 1.0, n, u)
    E = 0.05 * rng.standard_normal((3,) + g.shape)
    B = 0.05 * rng.standard_normal((3,) + g.shape)
    r0 = oracle.div_e(g, E) - fl.q * fl.n
    tot0 = fl.n.sum()
    for _ in range(20):
        _step(g, E, B, [fl])
    assert np.all(fl.n > 0)
    assert fl.n.sum() == pytest.approx(tot0, rel=1e-13)
    assert np.max(np.abs(oracle.div_e(g, E) - fl.q * fl.n - r0)) < 1e-12 * np.max(np.abs(r0))


def test_uniform_field_gives_exact_impulse():
    g = _grid()
    fl = oracle.Fluid(-1.0, 1.0, np.full(g.shape, 0.3))
    E = oracle.zeros_field(g)
    B = oracle.zeros_field(g)
    E[1][:] = 0.02
    J = oracle.zeros_field(g)
    for k in range(1, 6):
        oracle.fluid_step(g, E, B, J, fl)
        assert np.allclose(fl.u[1], -0.02 * k * g.dt, rtol=0, atol=1e-15)
        assert np.allclose(fl.n, 0.3, rtol=0, atol=1e-15)


def test_langmuir_oscillation_at_plasma_frequency():
    """Small density perturbation of an electron fluid over an immobile ion
    background: the field oscillates at w_p = sqrt(n0) (resolution-limited)."""
    nx, d = 64, 0.25
    g = oracle.Grid.make(nx, 4, 4, d, d, d, 0.05)
    n0, eps = 0.5, 1e-3
    x = np.arange(nx) * d
    k = 2 * math.pi / (nx * d)
    ne = n0 * (1 + eps * np.cos(k * x))
    el = oracle.Fluid(-1.0, 1.0, np.broadcast_to(ne, g.shape))
    ion = oracle.Fluid(1.0, 1e12, np.full(g.shape, n0))
    E = oracle.zeros_field(g)
    B = oracle.zeros_field(g)
    rho = n0 - ne
    Ex = np.cumsum(rho) * d
    Ex -= Ex.mean()
    E[0][:] = Ex[None, None, :]
    probe = []
    nsteps = 1600
    for _ in range(nsteps):
        _step(g, E, B, [el, ion])
        probe.append(E[0][0, 0, nx // 4])
    probe = np.array(probe)
    # zero crossings give the period
    s = np.sign(probe)
    cross = np.nonzero(s[1:] != s[:-1])[0]
    period = 2 * (cross[-1] - cross[0]) / (len(cross) - 1) * g.dt
    wp = math.sqrt(n0)
    assert period == pytest.approx(2 * math.pi / wp, rel=1e-2)
