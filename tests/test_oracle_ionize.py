"""Pins of the oracle's ionization rates and Monte Carlo against closed forms
(Landau-Lifshitz static tunnelling rate of hydrogen and hydrogen-like ions),
the textbook Keldysh relation gamma = sqrt(Ip / 2 Up), the construction of
the blend (continuity at gamma = 1.5, pure limits) and the binomial law of
the per-step events."""
import math

import numpy as np
import pytest

import oracle

LAMBDA = 0.8e-6


@pytest.mark.parametrize("F", [0.01, 0.03, 0.1, 0.3, 1.0])
def test_adk_reduces_to_hydrogen_static_rate(F):
    # Ip = 1/2, n* = 1, l = m = 0: w = (4/F) exp(-2/(3F)) atomic units
    assert oracle.adk_rate(F, 0.5, 1, 0, 0) == pytest.approx(4 / F * math.exp(-2 / (3 * F)), rel=1e-14)


@pytest.mark.parametrize("Z", [2, 3, 6])
def test_adk_hydrogen_like_scaling(Z):
    for F in (0.5 * Z ** 3 / 10, Z ** 3 / 10):
        want = 4 * Z ** 5 / F * math.exp(-2 * Z ** 3 / (3 * F))
        assert oracle.adk_rate(F, Z * Z / 2, Z, 0, 0) == pytest.approx(want, rel=1e-13)


def test_keldysh_matches_ponderomotive_form():
    # hydrogen, 800 nm, I = 1e14 W/cm^2: gamma = sqrt(Ip / (2 Up)), Up = 9.337e-14 I lambda_um^2 eV
    w0_au, _, _ = oracle.atomic_units(LAMBDA, 0.1)
    I = 1e18  # W/m^2
    E = math.sqrt(2 * I / (299792458.0 * 8.8541878128e-12))
    F = E / oracle.E_ATOMIC
    Up = 9.3373e-14 * 1e14 * 0.64
    assert oracle.keldysh(F, 0.5, w0_au) == pytest.approx(math.sqrt(13.598 / (2 * Up)), rel=2e-3)


CARBON = [(11.260, 1), (24.383, 1), (47.888, 0), (64.494, 0), (392.09, 0), (489.99, 0)]


@pytest.mark.parametrize("Z0", range(6))
def test_blend_continuous_at_gamma_1p5_and_pure_in_the_limits(Z0):
    w0_au, _, _ = oracle.atomic_units(LAMBDA, 0.1)
    Ip = CARBON[Z0][0] / oracle.HARTREE_EV
    l = CARBON[Z0][1]
    Fs = w0_au * math.sqrt(2 * Ip) / 1.5
    assert oracle.keldysh(Fs, Ip, w0_au) == pytest.approx(1.5, rel=1e-14)
    assert oracle.mpi_rate(Fs, Ip, Z0 + 1, l, w0_au) == pytest.approx(oracle.adk_rate(Fs, Ip, Z0 + 1, l, 0), rel=1e-12)
    assert oracle.ionization_rate(Fs, Ip, Z0 + 1, l, w0_au) == pytest.approx(
        oracle.adk_rate(Fs, Ip, Z0 + 1, l, 0), rel=1e-12)
    # weak field (gamma >= 3): multiphoton; strong field (gamma <= 0.5): ADK
    for F in (Fs / 2, Fs / 4):
        assert oracle.ionization_rate(F, Ip, Z0 + 1, l, w0_au) == pytest.approx(
            oracle.mpi_rate(F, Ip, Z0 + 1, l, w0_au), rel=1e-5)
    for F in (3 * Fs, 6 * Fs):
        assert oracle.ionization_rate(F, Ip, Z0 + 1, l, w0_au) == pytest.approx(
            oracle.adk_rate(F, Ip, Z0 + 1, l, 0), rel=2e-3)
    # multiphoton order K = ceil(Ip / w0): doubling F multiplies the rate by 4^K
    K = math.ceil(Ip / w0_au)
    r = math.log(oracle.mpi_rate(Fs, Ip, Z0 + 1, l, w0_au) / oracle.mpi_rate(0.99 * Fs, Ip, Z0 + 1, l, w0_au))
    assert r == pytest.approx(-2 * K * math.log(0.99), rel=1e-9)


def test_blend_monotone_in_field():
    """Increasing from deep multiphoton up to the maximum of the ADK formula
    (which peaks at F = 2 (2Ip)^{3/2} / (3 (2n* - 1)), far above the barrier-
    suppression field Ip^2 / 4Z where the formula stops being physical)."""
    w0_au, _, _ = oracle.atomic_units(LAMBDA, 0.1)
    for Z0, (Ip_eV, l) in enumerate(CARBON[:4]):
        Ip = Ip_eV / oracle.HARTREE_EV
        Fs = w0_au * math.sqrt(2 * Ip) / 1.5
        ns = (Z0 + 1) / math.sqrt(2 * Ip)
        Fpk = 2 * (2 * Ip) ** 1.5 / (3 * (2 * ns - 1))
        Fg = np.geomspace(Fs / 20, 0.9 * Fpk, 400)
        w = np.array([oracle.ionization_rate(F, Ip, 1, l, w0_au) for F in Fg])
        assert np.all(np.diff(w) > 0)


def _ion_set(n, zq=0.0):
    rng = np.random.default_rng(0)
    ions = oracle.Particles(1.0, 12 * 1836.15267343, rng.uniform(0, 8, n), rng.uniform(0, 8, n),
                            rng.uniform(0, 8, n), np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, 0.01),
                            zq=np.full(n, zq))
    return ions


def test_ionization_events_binomial_and_energy_tally():
    n = 40000
    ions = _ion_set(n)
    # a uniform field tuned so that P ~ 0.2 for neutral hydrogen-like carbon level 0
    dt = 0.2
    w0_au, er, dt_au = oracle.atomic_units(LAMBDA, dt)
    Ip = CARBON[0][0] / oracle.HARTREE_EV
    F = 0.06
    P = -math.expm1(-oracle.ionization_rate(F, Ip, 1, 1, w0_au) * dt_au)
    assert 0.05 < P < 0.6
    ions.eb = np.zeros((n, 6))
    ions.eb[:, 1] = F / er
    e, en = oracle.ionize(ions, 6, [c[0] for c in CARBON], [c[1] for c in CARBON], LAMBDA, dt, 7, 1, 3)
    k = e.n
    assert abs(k - n * P) <= 3 * math.sqrt(n * P * (1 - P))
    assert np.count_nonzero(ions.zq == 1) == k
    assert en == pytest.approx(k * 0.01 * CARBON[0][0] / 510998.95, rel=1e-12)
    # the new electrons sit on their parents with the parents' momentum and weight
    parent = (e.ids & np.uint64((1 << 63) - 1)) >> np.uint64(3)
    assert np.all((e.ids >> np.uint64(63)) == 1) and np.all((e.ids & np.uint64(7)) == 1)
    assert np.array_equal(e.x, ions.x[parent.astype(np.int64)])
    assert np.all(e.w == 0.01)


def test_ionization_uses_the_documented_philox_stream():
    n = 64
    ions = _ion_set(n)
    ions.eb = np.zeros((n, 6))
    w0_au, er, dt_au = oracle.atomic_units(LAMBDA, 0.2)
    F = 0.045
    ions.eb[:, 1] = F / er
    Ip = CARBON[0][0] / oracle.HARTREE_EV
    P = -math.expm1(-oracle.ionization_rate(F, Ip, 1, 1, w0_au) * dt_au)
    zq0 = ions.zq.copy()
    oracle.ionize(ions, 6, [c[0] for c in CARBON], [c[1] for c in CARBON], LAMBDA, 0.2, 11, 2, 5)
    for p in range(n):
        r = oracle.philox([p, 0, 5, 1], [11, 2])
        assert (oracle.u01(r[0]) < P) == (ions.zq[p] == zq0[p] + 1)


def test_fully_ionized_ions_do_not_ionize():
    n = 100
    ions = _ion_set(n, zq=6.0)
    ions.eb = np.zeros((n, 6))
    ions.eb[:, 0] = 1e3
    e, en = oracle.ionize(ions, 6, [c[0] for c in CARBON], [c[1] for c in CARBON], LAMBDA, 0.2, 1, 1, 0)
    assert e.n == 0 and en == 0.0
