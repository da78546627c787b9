"""Differential evolution (DE/rand/1/bin) on functions with known minima, and
its determinism; the laser-parameter search itself runs on the GPU
(test_gpu_optimize.py)."""
import numpy as np
import pytest

from paper_2510_11174_gb300.optimize import a0_from_intensity, de_minimize, intensity_w_cm2


def _batch(f):
    return lambda X: np.array([f(x) for x in X])


def test_de_finds_the_minimum_of_a_shifted_sphere():
    c = np.array([0.3, -1.2, 2.0])
    r = de_minimize(_batch(lambda x: float(np.sum((x - c) ** 2))), [-5] * 3, [5] * 3, pop=20, generations=150,
                    seed=3)
    assert np.allclose(r["x"], c, atol=1e-4) and r["f"] < 1e-8


def test_de_finds_the_rosenbrock_valley_minimum():
    rosen = lambda x: float(100.0 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2)
    r = de_minimize(_batch(rosen), [-2, -1], [2, 3], pop=24, generations=300, seed=5)
    assert np.allclose(r["x"], [1.0, 1.0], atol=1e-3)


def test_de_keeps_the_box_and_never_gets_worse():
    seen = []
    f = _batch(lambda x: float(np.abs(x).sum()))
    r = de_minimize(f, [1.0, 2.0], [3.0, 5.0], pop=8, generations=60, seed=1,
                    callback=lambda g, X, fx: seen.append(X.copy()))
    for X in seen:
        assert np.all(X >= [1.0, 2.0]) and np.all(X <= [3.0, 5.0])
    h = r["history"]
    assert all(b <= a for a, b in zip(h, h[1:]))
    assert r["x"] == pytest.approx([1.0, 2.0], abs=0.05)   # the corner minimum of |x|_1 on the box


def test_de_is_deterministic_for_a_seed():
    f = _batch(lambda x: float(np.sin(3 * x[0]) + (x[1] - 0.5) ** 2))
    a = de_minimize(f, [-2, -2], [2, 2], pop=10, generations=8, seed=11)
    b = de_minimize(f, [-2, -2], [2, 2], pop=10, generations=8, seed=11)
    assert np.array_equal(a["pop_x"], b["pop_x"]) and a["history"] == b["history"]


def test_intensity_relation_round_trip():
    assert intensity_w_cm2(1.0, 0.8) == pytest.approx(2.14e18, rel=1e-2)
    assert a0_from_intensity(intensity_w_cm2(7.3)) == pytest.approx(7.3, rel=1e-12)
