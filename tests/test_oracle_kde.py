"""Pins of the oracle's grid estimate and mixture ISE (Eqs. 1, 37) against
facts fixed by the mathematics: the estimate integrates to one (Riemann
sum over a grid that holds the sample and its kernel mass), equals a direct
sum over the nodes for a single point on a node, the ISE is non-negative,
int f^2 matches quadrature, and the binned ISE approaches the exact one as
the grid is refined (second-order binning error)."""
import numpy as np
import pytest

from oracle import binning, functionals as F, kde, rules


def _mixture():
    w = np.array([0.6, 0.4])
    mu = np.array([[-0.5, 0.0], [0.8, 0.5]])
    S = np.array([[[0.3, 0.1], [0.1, 0.2]], [[0.2, -0.05], [-0.05, 0.4]]])
    return w, mu, S


def _sample(n, seed):
    rng = np.random.default_rng(seed)
    w, mu, S = _mixture()
    lab = rng.choice(2, n, p=w)
    X = np.array([rng.multivariate_normal(mu[l], S[l]) for l in lab])
    return X


def test_grid_estimate_integrates_to_one_and_single_point():
    X = _sample(300, 1)
    H = np.array([[0.05, 0.01], [0.01, 0.04]])
    lo, hi = X.min(0) - 1.5, X.max(0) + 1.5
    M = [70, 64]
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    L = rules.support_L(rules.lambda_max(H), delta, M)
    f = kde.kde_grid(c, X.shape[0], H, delta, L)
    assert float(np.sum(f)) * float(np.prod(delta)) == pytest.approx(1.0, abs=2e-3)
    # one point on a node: f(g) = K_H(x_g - x_point) within the support
    c1 = np.zeros(M)
    c1[30, 31] = 1.0
    f1 = kde.kde_grid(c1, 1, H, delta, L)
    from oracle.gauss import gauss_density
    g = np.array([33, 29])
    x = (g - np.array([30, 31])) * delta
    assert f1[33, 29] == pytest.approx(float(gauss_density(x[None, :], H)[0]), rel=1e-12)
    assert f1[30 + L[0] + 1, 31] == 0.0      # outside the truncated stencil
    # the stencil reaches |l_k| = L_k inclusive (Eq. 26's support)
    xL = np.array([L[0], -L[1]]) * delta
    assert f1[30 + L[0], 31 - L[1]] == pytest.approx(float(gauss_density(xL[None, :], H)[0]), rel=1e-12)
    # n^-1 sum_g c_g f_hat(g) is Eq. 25's binned double sum of K_H
    got = float(np.sum(c * f)) / X.shape[0]
    want = F.binned_direct(c, X.shape[0], [(1.0, H, (0, 0))], delta, L)
    assert got == pytest.approx(want, rel=1e-12)


def test_mixture_square_integral_matches_quadrature():
    w, mu, S = _mixture()
    from oracle.gauss import gauss_density
    xs = np.linspace(-5, 5, 401)
    h = xs[1] - xs[0]
    G = np.stack(np.meshgrid(xs, xs, indexing="ij"), axis=-1).reshape(-1, 2)
    f = sum(wm * gauss_density(G - m[None, :], Sm) for wm, m, Sm in zip(w, mu, S))
    assert kde.mixture_sq_integral(w, mu, S) == pytest.approx(float(np.sum(f * f)) * h * h, rel=1e-6)


def test_ise_nonnegative_and_binning_converges():
    X = _sample(400, 2)
    w, mu, S = _mixture()
    H = np.array([[0.06, 0.01], [0.01, 0.05]])
    exact = kde.ise_mixture_exact(X, H, w, mu, S)
    assert exact > 0.0
    lo, hi = X.min(0) - 2.0, X.max(0) + 2.0
    errs = []
    for m in (40, 80, 160):
        M = [m, m]
        c = binning.bin_linear(X, lo, hi, M)
        delta = rules.bin_width(lo, hi, M)
        L2 = [mm - 1 for mm in M]
        b = kde.ise_mixture_binned(c, X.shape[0], lo, delta, H, w, mu, S, L2)
        assert b > 0.0
        errs.append(abs(b - exact))
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5   # about 4x per halving of delta


def test_exact_ise_matches_quadrature_of_the_squared_error():
    """Eq. 37 straight from its definition: int (f_hat - f)^2 by a Riemann
    sum on a fine grid, with f_hat and f evaluated pointwise (no Gaussian
    convolution identities)."""
    X = _sample(20, 5)
    w, mu, S = _mixture()
    H = np.array([[0.08, 0.02], [0.02, 0.06]])
    from oracle.gauss import gauss_density
    h = 0.02
    xs = np.arange(-4.5, 4.5, h)
    G = np.stack(np.meshgrid(xs, xs, indexing="ij"), axis=-1).reshape(-1, 2)
    fhat = sum(gauss_density(G - x[None, :], H) for x in X) / X.shape[0]
    f = sum(wm * gauss_density(G - m[None, :], Sm) for wm, m, Sm in zip(w, mu, S))
    quad = float(np.sum((fhat - f) ** 2)) * h * h
    assert kde.ise_mixture_exact(X, H, w, mu, S) == pytest.approx(quad, rel=1e-6)
