"""Pins for oracle.gauss: Gaussian partials by the Hermite recurrence.

Pinned against (a) the textbook probabilists' Hermite polynomials in 1-D,
(b) symbolic differentiation of the Gaussian density (sympy), (c) Isserlis'
pairing formula at the origin, (d) the heat equation by finite differences.
"""
import math

import numpy as np
import pytest

from oracle import gauss


def _spd(rng, d):
    A = rng.standard_normal((d, d))
    return A @ A.T + 0.5 * np.eye(d)


@pytest.mark.parametrize("k", range(0, 9))
def test_1d_matches_probabilists_hermite(k):
    from numpy.polynomial import hermite_e as He
    s2 = 0.37
    x = np.linspace(-2.5, 2.5, 41)
    got = gauss.gauss_deriv(x[:, None], np.array([[s2]]), (k,))
    s = math.sqrt(s2)
    coef = np.zeros(k + 1)
    coef[k] = 1.0
    phi = np.exp(-0.5 * x * x / s2) / math.sqrt(2 * math.pi * s2)
    want = (-1.0) ** k * s ** (-k) * He.hermeval(x / s, coef) * phi
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d,rmax", [(2, 6), (3, 4)])
def test_matches_symbolic_derivative(d, rmax):
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(11 + d)
    S = _spd(rng, d)
    xs = sp.symbols(f"x0:{d}")
    Lam = sp.Matrix(np.linalg.inv(S).tolist())
    xv = sp.Matrix(xs)
    phi = (2 * sp.pi) ** sp.Rational(-d, 2) / sp.sqrt(sp.Float(np.linalg.det(S), 30)) * \
        sp.exp(-(xv.T * Lam * xv)[0, 0] / 2)
    pts = rng.standard_normal((3, d)) * 0.7
    for r in range(0, rmax + 1):
        for alpha in gauss.multi_indices(d, r):
            expr = phi
            for k, m in enumerate(alpha):
                if m:
                    expr = sp.diff(expr, xs[k], m)
            f = sp.lambdify(xs, expr, "math")
            want = np.array([f(*p) for p in pts])
            got = gauss.gauss_deriv(pts, S, alpha)
            np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_value_at_origin_is_isserlis(d):
    rng = np.random.default_rng(d)
    S = _spd(rng, d)
    for r in (0, 2, 4, 6):
        for alpha in gauss.multi_indices(d, r):
            got = float(gauss.gauss_deriv(np.zeros((1, d)), S, alpha)[0])
            want = gauss.pairings_value_at_zero(S, alpha)
            assert got == pytest.approx(want, rel=1e-11, abs=1e-13)
    # odd orders vanish at the origin
    for alpha in gauss.multi_indices(d, 3):
        assert abs(float(gauss.gauss_deriv(np.zeros((1, d)), S, alpha)[0])) < 1e-14


def test_heat_equation_by_finite_differences():
    rng = np.random.default_rng(5)
    d = 3
    S = _spd(rng, d)
    x = rng.standard_normal((4, d)) * 0.8
    h = 1e-6
    for a in range(d):
        for b in range(a, d):
            E = np.zeros((d, d))
            E[a, b] = E[b, a] = 1.0
            fd = (gauss.gauss_density(x, S + h * E) - gauss.gauss_density(x, S - h * E)) / (2 * h)
            tie = 1.0 if a == b else 2.0
            al = [0] * d
            al[a] += 1
            al[b] += 1
            an = tie * 0.5 * gauss.gauss_deriv(x, S, tuple(al))
            np.testing.assert_allclose(fd, an, rtol=1e-6, atol=1e-9)


def test_kronecker_positions():
    d, r = 3, 3
    al = gauss.kron_alphas(d, r)
    assert len(al) == d ** r
    # position (i1, i2, i3) with i1 slowest
    assert al[0 * 9 + 1 * 3 + 2] == (1, 1, 1)
    assert al[2 * 9 + 2 * 3 + 0] == (1, 0, 2)
    assert len(gauss.multi_indices(4, 4)) == 35
