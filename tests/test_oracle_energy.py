"""Pins of the oracle's FP64 energy sums (Methodology: total energy from the
electromagnetic and kinetic parts, checked during the steps) against values
that do not come from the oracle: exact discrete identities of a sampled
plane wave, momenta whose Lorentz factors are exact rationals (Pythagorean
triples), and the non- and ultra-relativistic series of gamma - 1.
"""
import math

import numpy as np
import pytest

import oracle


def _grid(nx, ny, nz, dx, dy, dz):
    return oracle.Grid.make(nx, ny, nz, dx, dy, dz, 0.1)


def _field(shape, fx, fy, fz):
    F = np.zeros((3,) + shape)
    F[0], F[1], F[2] = fx, fy, fz
    return F


def test_field_energy_of_a_sampled_plane_wave_over_whole_periods():
    # sum over N equally spaced samples of sin^2 and cos^2 over whole periods
    # is exactly N / 2 (discrete orthogonality), whatever the phase
    nx, ny, nz, dx, dy, dz = 24, 3, 2, 0.3, 0.5, 0.7
    g = _grid(nx, ny, nz, dx, dy, dz)
    x = np.arange(nx) * dx
    k = 2.0 * math.pi * 3 / (nx * dx)                      # three periods
    shape = (nz, ny, nx)
    ey = np.broadcast_to(np.sin(k * x + 0.4), shape)
    bz = np.broadcast_to(np.cos(k * x + 0.4), shape)
    E = _field(shape, 0.0, 2.0 * ey, 0.0)
    B = _field(shape, 0.0, 0.0, 2.0 * bz)
    we, wb = oracle.energy_fields(g, E, B)
    volume = nx * ny * nz * dx * dy * dz
    # (1/2) sum |E|^2 dV = (1/2) 4 (N / 2) dV = volume for amplitude 2
    assert we == pytest.approx(volume, rel=1e-13)
    assert wb == pytest.approx(volume, rel=1e-13)


def test_field_energy_of_uniform_fields():
    g = _grid(4, 3, 5, 0.25, 0.5, 2.0)
    shape = (5, 3, 4)
    E = _field(shape, 1.0, -2.0, 3.0)
    B = _field(shape, 0.5, 0.0, -1.0)
    we, wb = oracle.energy_fields(g, E, B)
    assert we == 0.5 * 14.0 * 60 * 0.25        # |E|^2 = 14, V = 60 cells x 0.25
    assert wb == 0.5 * 1.25 * 60 * 0.25


def _species(m, u, w):
    u = np.asarray(u, dtype=np.float64)
    n = len(u)
    z = np.zeros(n)
    return oracle.Particles(-1.0, m, z, z, z, u[:, 0], u[:, 1], u[:, 2], np.asarray(w, dtype=np.float64))


def test_kinetic_energy_with_rational_lorentz_factors():
    # |u| = a/b from Pythagorean triples (a, b, c): gamma = c/b exactly
    cases = [((3, 4, 5), (1, 0, 0)), ((4, 3, 5), (0, 1, 0)), ((12, 5, 13), (0, 0, 1)),
             ((5, 12, 13), (0.6, 0.8, 0.0)), ((8, 15, 17), (0.0, 0.6, -0.8)), ((20, 21, 29), (-1, 0, 0))]
    u, w, expect = [], [], 0.0
    for i, ((a, b, c), d) in enumerate(cases):
        d = np.asarray(d, dtype=np.float64)
        u.append(d / np.linalg.norm(d) * a / b)
        w.append(0.5 + i)
        expect += (0.5 + i) * (c - b) / b          # w (gamma - 1)
    for m in (1.0, 1836.15267343):
        assert oracle.energy_particles(_species(m, u, w)) == pytest.approx(m * expect, rel=1e-14)


def test_kinetic_energy_limits():
    rng = np.random.default_rng(4)
    d = rng.standard_normal((1000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w = rng.uniform(0.1, 2.0, 1000)
    # non-relativistic: gamma - 1 = u^2/2 - u^4/8 + u^6/16 - ...
    s = 1e-3
    expect = np.sum(w * (s ** 2 / 2 - s ** 4 / 8))
    assert oracle.energy_particles(_species(1.0, d * s, w)) == pytest.approx(expect, rel=1e-12)
    # ultra-relativistic: gamma - 1 = u - 1 + 1/(2u) - 1/(8u^3) + ...
    s = 1e6
    expect = np.sum(w * (s - 1 + 1 / (2 * s)))
    assert oracle.energy_particles(_species(1.0, d * s, w)) == pytest.approx(expect, rel=1e-14)
