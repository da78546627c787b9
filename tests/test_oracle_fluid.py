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


def _warm_run(g, fl, steps, node):
    E, B = oracle.zeros_field(g), oracle.zeros_field(g)
    trace = []
    for _ in range(steps):
        J = oracle.zeros_field(g)
        oracle.fluid_step(g, E, B, J, fl)
        trace.append(fl.n[node])
    return np.array(trace)


@pytest.mark.parametrize("T_keV,gam", [(10.0, 5.0 / 3.0), (40.0, 3.0)])
def test_warm_fluid_sound_wave_has_the_discrete_leapfrog_frequency(T_keV, gam):
    """A small standing sound wave in a neutral warm fluid: linearised, the
    scheme is a leapfrog with the central pressure difference, so
    sin(w dt / 2) = (dt / 2) c_s sin(k d) / d with c_s^2 = gamma K n0^(gamma-1) / m."""
    nx, d, dt = 32, 0.4, 0.2
    g = oracle.Grid.make(nx, 4, 4, d, d, d, dt, bc=(0, 0, 0))
    k = 2 * np.pi / (nx * d)
    x = np.arange(nx) * d
    n0, eps = 1.0, 1e-5
    n = np.broadcast_to(n0 * (1 + eps * np.cos(k * x))[None, None, :], g.shape).copy()
    K = (T_keV / 510.99895)
    fl = oracle.Fluid(0.0, 1.0, n, K=K, gamma_ad=gam)
    cs = np.sqrt(gam * K * n0 ** (gam - 1.0) / 1.0)
    w = 2.0 / dt * np.arcsin(0.5 * dt * cs * np.sin(k * d) / d)
    period = 2 * np.pi / w
    tr = _warm_run(g, fl, int(2.2 * period / dt), (1, 1, 0)) - n0
    # zero crossings of the density at x = 0 (it starts at +eps, a cosine)
    s = np.sign(tr)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    t_cross = [(i + 1 + tr[i] / (tr[i] - tr[i + 1])) * dt for i in idx]   # step n holds the state after n + 1 steps
    measured = 2.0 * (t_cross[2] - t_cross[0]) / 2.0
    assert measured == pytest.approx(period, rel=2e-3), (measured, period)


def test_warm_fluid_conserves_momentum_and_keeps_a_uniform_state():
    g = oracle.Grid.make(16, 12, 8, 0.3, 0.3, 0.3, 0.1, bc=(0, 0, 0))
    rng = np.random.default_rng(4)
    fl = oracle.Fluid(0.0, 1.0, 0.5 + rng.random(g.shape), 0.05 * rng.standard_normal((3,) + g.shape), K=0.02,
                      gamma_ad=5.0 / 3.0)
    dV = 0.3 ** 3
    mom0 = (fl.n * fl.u).sum(axis=(1, 2, 3)) * dV
    E, B = oracle.zeros_field(g), oracle.zeros_field(g)
    for _ in range(5):
        oracle.fluid_step(g, E, B, oracle.zeros_field(g), fl)
    mom1 = (fl.n * fl.u).sum(axis=(1, 2, 3)) * dV
    assert np.allclose(mom1, mom0, rtol=0, atol=1e-12 * np.abs(fl.n).sum() * dV)
    # a uniform warm fluid at rest stays so, walls included (the wall reflects the pressure)
    for bc in ((0, 0, 0), (1, 1, 1)):
        g = oracle.Grid.make(8, 8, 8, 0.3, 0.3, 0.3, 0.1, bc=bc)
        fl = oracle.Fluid(-1.0, 1.0, np.full(g.shape, 0.7), K=0.05, gamma_ad=5.0 / 3.0)
        oracle.fluid_step(g, oracle.zeros_field(g), oracle.zeros_field(g), oracle.zeros_field(g), fl)
        assert np.all(fl.u == 0.0) and np.all(fl.n == 0.7)
