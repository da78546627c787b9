"""Pins of the oracle's Airy functions and LCFA QED rates against library
routines (scipy), published asymptotic expansions (classical radiated power
with its first quantum correction, classical photon number, small-chi pair
rate with its first correction) and exact properties of the Monte Carlo
(energy balance per event, binomial event counts, spectrum inversion)."""
import math

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.special")
si = pytest.importorskip("scipy.integrate")


def test_airy_matches_scipy():
    for z in np.concatenate([[0.0, 1e-12, 1e-6], np.geomspace(1e-3, 40, 120)]):
        a = sp.airy(z)
        assert oracle.airy_ai(z) == pytest.approx(a[0], rel=1e-13)
        assert oracle.airy_aip(z) == pytest.approx(a[1], rel=1e-13)


def test_bessel_k_matches_scipy():
    for nu in (1 / 3, 2 / 3):
        for x in np.geomspace(1e-8, 60, 60):
            assert oracle.bessel_k(nu, x) == pytest.approx(sp.kv(nu, x), rel=1e-13)


@pytest.mark.parametrize("z", [0.0, 0.1, 1.0, 3.0, 8.0])
def test_airy_integral_matches_quadrature(z):
    q = si.quad(lambda t: sp.airy(t)[0], z, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert oracle.airy_int(z) == pytest.approx(q, rel=1e-12)
    if z == 0.0:
        assert oracle.airy_int(0.0) == pytest.approx(1 / 3, rel=1e-14)


@pytest.mark.parametrize("chi", [1e-5, 1e-4])
def test_radiated_power_classical_limit_with_first_quantum_correction(chi):
    # P / P_classical = 1 - (55 sqrt3 / 16) chi + O(chi^2), P_classical = (2/3) alpha m^2 c^4 chi^2 / hbar
    g = oracle.qed_power(chi) / (2 / 3 * chi ** 2)
    assert g == pytest.approx(1 - 55 * math.sqrt(3) / 16 * chi, abs=60 * chi ** 2)


def test_photon_number_classical_limit():
    # classical synchrotron photon rate: h(chi) -> 5 chi / (2 sqrt 3)
    assert oracle.qed_h(1e-6) / 1e-6 == pytest.approx(5 / (2 * math.sqrt(3)), rel=1e-5)


@pytest.mark.parametrize("chi", [0.005, 0.01, 0.02])
def test_pair_rate_small_chi_asymptote(chi):
    # T(chi) ~ (3 sqrt3 / (16 sqrt2)) chi exp(-8/(3 chi)) (1 - 11 chi / 64 + O(chi^2))
    a = 3 * math.sqrt(3) / (16 * math.sqrt(2)) * chi * math.exp(-8 / (3 * chi))
    assert oracle.qed_T(chi) / a == pytest.approx(1 - 11 * chi / 64, abs=3 * chi ** 2)


def test_pair_spectrum_symmetric_and_integrates():
    for chi in (0.3, 3.0, 1000.0):
        for xi in (0.05, 0.2, 0.4):
            assert oracle.qed_pair_density(chi, xi) == pytest.approx(oracle.qed_pair_density(chi, 1 - xi), rel=1e-12)
        # the spectrum reaches down to xi ~ 1/chi: give the adaptive rule those break points
        pts = [p for p in (0.25 / chi, 1 / chi, 4 / chi) if p < 0.5] or None
        q = 2 * si.quad(lambda x: oracle.qed_pair_density(chi, x), 0, 0.5, epsabs=0, epsrel=1e-11, limit=500,
                        points=pts)[0]
        assert oracle.qed_T(chi) == pytest.approx(q, rel=1e-9)


def test_emission_spectrum_integrates_and_inverts():
    for chi in (0.01, 1.0, 20.0):
        q = si.quad(lambda x: oracle.qed_em_density(chi, x), 0, 1, epsabs=0, epsrel=1e-10, limit=400,
                    points=[min(chi, 0.5)])[0]
        h = oracle.qed_h(chi)
        assert h == pytest.approx(q, rel=1e-7)
        for r in (0.05, 0.5, 0.95):
            xi = oracle.qed_em_sample(chi, r)
            cdf = si.quad(lambda x: oracle.qed_em_density(chi, x), 0, xi, epsabs=0, epsrel=1e-10, limit=400)[0]
            assert cdf / h == pytest.approx(r, abs=2e-7)


def test_chi_of_a_particle_in_a_transverse_field():
    # ultra-relativistic electron along x in E_y: chi = kappa (gamma E - u B...) ; for B = 0, chi = kappa gamma E
    k = oracle.qed_kappa(0.8e-6)
    u = np.array([1000.0, 0, 0])
    g = math.sqrt(1 + u @ u)
    assert oracle.chi_param(k, [0, 5.0, 0], [0, 0, 0], u) == pytest.approx(k * g * 5.0, rel=1e-12)
    # a plane wave co-moving with the particle (E_y = B_z) nearly cancels: chi = kappa E (gamma - u_x)
    assert oracle.chi_param(k, [0, 5.0, 0], [0, 0, 5.0], u) == pytest.approx(k * 5.0 * (g - 1000.0), rel=1e-9)
    # photon: chi_g = kappa eps E for k perpendicular to E, B = 0
    assert oracle.chi_param(k, [0, 3.0, 0], [0, 0, 0], [50.0, 0, 0], photon=True) == pytest.approx(k * 150, rel=1e-12)


def _leptons(n, gamma, seed=0):
    rng = np.random.default_rng(seed)
    u = math.sqrt(gamma ** 2 - 1)
    s = oracle.Particles(-1.0, 1.0, rng.uniform(0, 8, n), rng.uniform(0, 8, n), rng.uniform(0, 8, n),
                         np.full(n, u), np.zeros(n), np.zeros(n), np.full(n, 0.01))
    return s


def test_emission_events_binomial_and_energy_balance():
    n, gamma, E = 800, 2000.0, 300.0
    s = _leptons(n, gamma)
    k = oracle.qed_kappa(0.8e-6)
    s.eb = np.zeros((n, 6))
    s.eb[:, 1] = E
    s.tau = oracle.qed_tau0(s.ids, 5, 0)
    dt = 0.1
    chi = oracle.chi_param(k, [0, E, 0], [0, 0, 0], [s.ux[0], 0, 0])
    W = oracle.ALPHA / k * oracle.qed_h(chi) / gamma
    P = -math.expm1(-W * dt)
    assert 0.05 < P < 0.95
    e_before = oracle.energy_particles(s)
    ph, lost, events = oracle.qed_emit(s, k, dt, 2.0, 5, 0, 7)
    assert abs(events - n * P) <= 3 * math.sqrt(n * P * (1 - P))
    e_after = oracle.energy_particles(s)
    e_photons = np.sum(ph.w * np.sqrt(ph.ux ** 2 + ph.uy ** 2 + ph.uz ** 2))
    assert e_before - e_after == pytest.approx(e_photons + lost, rel=1e-12)
    # photons fly along the parent's momentum, the new optical depths are positive
    assert np.all(ph.uy == 0) and np.all(ph.ux > 0) and np.all(ph.tau > 0)
    assert np.all(s.tau > 0)


def test_pair_events_conserve_momentum_along_k():
    n, eps, E = 150, 4000.0, 400.0
    rng = np.random.default_rng(3)
    ph = oracle.Particles(0.0, 0.0, rng.uniform(0, 8, n), rng.uniform(0, 8, n), rng.uniform(0, 8, n),
                          np.full(n, eps), np.zeros(n), np.zeros(n), np.full(n, 0.01))
    k = oracle.qed_kappa(0.8e-6)
    ph.eb = np.zeros((n, 6))
    ph.eb[:, 1] = E
    ph.tau = oracle.qed_tau0(ph.ids, 5, 2)
    chi = oracle.chi_param(k, [0, E, 0], [0, 0, 0], [eps, 0, 0], photon=True)
    W = oracle.ALPHA / k * oracle.qed_T(chi) / eps
    P = -math.expm1(-W * 1.0)
    assert 0.05 < P < 0.95
    el, po, deficit, events = oracle.qed_pairs(ph, k, 1.0, 5, 2, 4)
    assert abs(events - n * P) <= 3 * math.sqrt(n * P * (1 - P))
    assert ph.n == n - events and el.n == po.n == events
    ge = np.sqrt(1 + el.ux ** 2) + np.sqrt(1 + po.ux ** 2)
    assert np.allclose(ge, eps, rtol=1e-12)
    assert deficit == 0.0
