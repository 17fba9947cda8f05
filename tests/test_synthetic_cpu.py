"""The seeded input recipe (CPU): draws repeat bit for bit from their seeds,
and each generator produces what its recipe states — mixture moments,
rotations and spectra, the normal-scale rule, grid ranges that hold the data,
candidate bandwidths inside their eigenvalue band, and the workload shapes
(grid sizes, padded sizes, candidate counts, the uneven batch's grid rule)."""
import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic as syn


def test_draws_repeat_from_their_seeds():
    a = syn.mixture_2d_large(n=5000)
    b = syn.mixture_2d_large(n=5000)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.H, b.H) and np.array_equal(a.G, b.G)
    c = syn.mixture_2d_large(n=5000, seed=3)
    assert not np.array_equal(a.X, c.X)
    u1 = syn.batched_uneven(n_datasets=3, n_range=(500, 800))
    u2 = syn.batched_uneven(n_datasets=3, n_range=(500, 800))
    assert all(np.array_equal(x.X, y.X) for x, y in zip(u1, u2))


def test_mixture_moments_match_the_recipe():
    rng = np.random.default_rng(1)
    w = [0.7, 0.3]
    mus = [[-1.0, 2.0], [3.0, 0.5]]
    sig = [np.array([[0.5, 0.2], [0.2, 0.3]]), np.array([[1.0, -0.4], [-0.4, 0.8]])]
    n = 400_000
    X = syn.sample_mixture(rng, n, w, mus, sig)
    mean = sum(wk * np.asarray(m) for wk, m in zip(w, mus))
    second = sum(wk * (S + np.outer(m, m)) for wk, m, S in zip(w, mus, sig))
    cov = second - np.outer(mean, mean)
    np.testing.assert_allclose(X.mean(0), mean, atol=0.01)
    np.testing.assert_allclose(np.cov(X, rowvar=False), cov, atol=0.02)


def test_rotations_and_spectra():
    rng = np.random.default_rng(2)
    for d in (1, 2, 3, 4):
        Q = syn.random_rotation(rng, d)
        np.testing.assert_allclose(Q.T @ Q, np.eye(d), atol=1e-13)
        lam = rng.uniform(0.1, 2.0, size=d)
        S = syn.random_spd(rng, d, lam)
        np.testing.assert_allclose(S, S.T, atol=1e-14)
        np.testing.assert_allclose(np.linalg.eigvalsh(S), np.sort(lam), rtol=1e-12)


def test_normal_scale_reduces_to_the_1d_rule():
    """d = 1: H = h^2 with the textbook normal-reference bandwidth
    h = (4 / (3 n))^{1/5} sigma."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5000, 1)) * 1.7
    h = (4.0 / (3.0 * 5000)) ** 0.2 * np.std(x, ddof=1)
    assert syn.normal_scale(x)[0, 0] == pytest.approx(h * h, rel=1e-12)
    # d = 2: the same power law in n and a multiple of the sample covariance
    X = rng.standard_normal((3000, 2)) @ np.array([[1.0, 0.5], [0.0, 0.8]])
    H = syn.normal_scale(X)
    np.testing.assert_allclose(H, (4.0 / 4.0) ** (2.0 / 6.0) * 3000 ** (-1.0 / 3.0) * np.cov(X, rowvar=False),
                               rtol=1e-12)


def test_grid_range_holds_the_data_with_three_bandwidths():
    w = syn.small_case(n=500, d=3, M=20)
    s = 3.0 * np.sqrt(np.diag(w.extra["H_NS"]))
    np.testing.assert_allclose(w.lo, w.X.min(0) - s, rtol=0, atol=0)
    np.testing.assert_allclose(w.hi, w.X.max(0) + s, rtol=0, atol=0)
    assert np.all(w.X >= w.lo) and np.all(w.X <= w.hi)


def test_candidates_lie_in_their_eigenvalue_band():
    rng = np.random.default_rng(4)
    H0 = np.array([[0.3, 0.1, 0.0], [0.1, 0.2, 0.05], [0.0, 0.05, 0.4]])
    Hs = syn.candidates_around(rng, H0, 200)
    R = np.linalg.cholesky(H0)
    Ri = np.linalg.inv(R)
    for H in Hs:
        np.testing.assert_array_equal(H, H.T)
        ev = np.linalg.eigvalsh(Ri @ H @ Ri.T)
        assert ev[0] >= 0.25 * (1 - 1e-12) and ev[-1] <= 4.0 * (1 + 1e-12)


def test_workload_shapes():
    w2 = syn.mixture_2d_large()
    assert w2.X.shape == (100_000, 2) and w2.M == [256, 256] and w2.H.shape == (16, 2, 2)
    assert np.array_equal(w2.G, w2.extra["H_NS"])
    w4 = syn.mixture_4d(n=20_000)
    assert w4.M == [48] * 4 and w4.P == [96] * 4 and w4.H.shape == (8, 4, 4)
    p = syn.plain_mixture_2d()
    assert p.X.shape == (1000, 2) and p.M == [100, 100]
    np.testing.assert_array_equal(p.H[0], [[0.10, 0.05], [0.05, 0.20]])
    s = syn.paper_speed_shape(n=2000)
    np.testing.assert_allclose(s.H[0], 2000 ** (-1.0 / 3.0) * np.eye(2))
    for u in syn.batched_uneven(n_datasets=40, n_range=(1e3, 1e5)):
        assert 1000 <= u.n <= 100_000
        assert u.M == [64 if u.n < 5000 else (128 if u.n < 30000 else 256)] * 2
        assert u.H.shape == (16, 2, 2)
