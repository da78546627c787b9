"""Pins of the oracle's relativistic pushers -- Boris, Vay (2008) and
Higuera-Cary (2017) -- against what the equations of motion fix exactly:
a pure electric field adds 2 h E (h = q dt / 2m), a pure magnetic field
rotates u without changing |u|, a field along the motion accelerates it
without turning it, and a particle moving at the drift velocity E x B / B^2
(E perpendicular to B, |E| < |B|) feels no force, which Vay and Higuera-Cary
reproduce to round-off and Boris does not for a relativistic drift."""
import numpy as np
import pytest

import oracle

PUSHERS = ("boris", "vay", "higuera_cary")


@pytest.mark.parametrize("pusher", PUSHERS)
def test_pure_electric_field_adds_two_h_e(pusher):
    e = np.array([0.3, -0.2, 0.5])
    u = np.array([1.0, 2.0, -3.0])
    assert np.allclose(oracle.boris(0.4, e, np.zeros(3), u, pusher=pusher), u + 0.8 * e, rtol=0, atol=1e-14)


@pytest.mark.parametrize("pusher", PUSHERS)
def test_pure_magnetic_field_keeps_the_momentum_magnitude(pusher):
    b = np.array([0.4, -1.0, 3.0])
    u = np.array([5.0, 2.0, 1.0])
    n0 = np.linalg.norm(u)
    u_par = u @ b / np.linalg.norm(b)
    for _ in range(1000):
        u = oracle.boris(0.2, np.zeros(3), b, u, pusher=pusher)
    assert abs(np.linalg.norm(u) / n0 - 1) < 1e-12
    assert abs(u @ b / np.linalg.norm(b) - u_par) < 1e-11   # the component along B is untouched


@pytest.mark.parametrize("pusher", PUSHERS)
def test_field_along_the_motion_accelerates_without_turning(pusher):
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    u = 4.0 * d
    for _ in range(50):
        u = oracle.boris(0.1, 0.7 * d, 2.5 * d, u, pusher=pusher)
    assert np.allclose(u, (4.0 + 50 * 2 * 0.1 * 0.7) * d, rtol=1e-13, atol=0)


@pytest.mark.parametrize("vd", [0.3, 0.9, 0.99])
def test_exb_drift_is_force_free_for_vay_and_higuera_cary(vd):
    B0 = 4.0
    e = np.array([0.0, vd * B0, 0.0])
    b = np.array([0.0, 0.0, B0])
    g = 1.0 / np.sqrt(1.0 - vd * vd)
    u0 = np.array([g * vd, 0.0, 0.0])      # v = E x B / B^2 along +x
    for pusher in ("vay", "higuera_cary"):
        u = u0.copy()
        for _ in range(200):
            u = oracle.boris(0.3, e, b, u, pusher=pusher)
        assert np.max(np.abs(u - u0)) < 1e-12 * g, pusher
    u = u0.copy()
    for _ in range(200):
        u = oracle.boris(0.3, e, b, u, pusher="boris")
    if vd >= 0.9:
        assert np.max(np.abs(u - u0)) > 1e-2 * g   # Boris does not hold the relativistic drift
