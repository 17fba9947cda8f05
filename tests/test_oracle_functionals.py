"""Pins for oracle.binning, oracle.functionals and oracle.selectors.

Every pin compares the oracle with something other than itself: closed
forms (n = 1, 2), brute-force scalar loops, invariants that hold exactly,
an independent formulation (tent functions for linear binning, the Parseval
sum for the binned functional), finite differences for gradients and the
convergence order of the binning error.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import binning, functionals as F, gauss, rules, selectors as S


def _spd(rng, d, scale=1.0):
    A = rng.standard_normal((d, d))
    return scale * (A @ A.T / d + 0.3 * np.eye(d))


def _mix(rng, n, d):
    X = rng.standard_normal((n, d))
    X[: n // 2] += 1.5
    return X


# ---------------------------------------------------------------- binning

@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_linear_binning_matches_tent_functions(d):
    """c_j = sum_i prod_k max(0, 1 - |t_ik - j_k|): the multilinear weights
    written as hat functions, an independent formulation."""
    rng = np.random.default_rng(d)
    M = [5, 4, 6, 3][:d]
    lo = -np.ones(d)
    hi = np.array([1.0, 2.0, 1.5, 0.5][:d])
    X = lo + rng.uniform(0, 1, size=(30, d)) * (hi - lo)
    X[0] = hi  # upper corner
    X[1] = lo
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    want = np.zeros(M)
    for i in range(X.shape[0]):
        t = (X[i] - lo) / delta
        for j in itertools.product(*[range(m) for m in M]):
            want[j] += math.prod(max(0.0, 1.0 - abs(t[k] - j[k])) for k in range(d))
    np.testing.assert_allclose(c, want, rtol=1e-13, atol=1e-13)


def test_binning_invariants():
    rng = np.random.default_rng(3)
    d, M = 2, [17, 23]
    X = _mix(rng, 500, d)
    lo, hi = X.min(0) - 0.1, X.max(0) + 0.1
    c = binning.bin_linear(X, lo, hi, M)
    assert c.sum() == pytest.approx(500.0, rel=1e-14)
    g = binning.grid_points(lo, hi, M)
    # multilinear weights reproduce linear functions: sum c_j g_j = sum X_i
    assert float(np.sum(c.sum(1) * g[0])) == pytest.approx(X[:, 0].sum(), rel=1e-12)
    assert float(np.sum(c.sum(0) * g[1])) == pytest.approx(X[:, 1].sum(), rel=1e-12)
    cs = binning.bin_simple(X, lo, hi, M)
    assert cs.dtype == np.int64 and int(cs.sum()) == 500
    # nodes bin onto themselves
    nodes = np.array([[g[0][3], g[1][7]], [g[0][16], g[1][0]]])
    cn = binning.bin_linear(nodes, lo, hi, M)
    assert cn[3, 7] == pytest.approx(1.0, abs=1e-12) and cn[16, 0] == pytest.approx(1.0, abs=1e-12)
    assert cn.sum() == pytest.approx(2.0, abs=1e-12)
    # simple binning: ties at half a bin round up
    half = np.array([[lo[0] + 2.5 * (hi[0] - lo[0]) / 16, g[1][4]]])
    assert binning.bin_simple(half, lo, hi, M)[3, 4] == 1


def test_upper_edge_rounding_stays_inside():
    """A point exactly at hi is inside even when (hi - lo)/delta rounds to
    just above M - 1; it lands on the last node with weight 1."""
    lo, hi, M = -0.920732229392339, 0.11341865083372567, 120
    assert (hi - lo) / ((hi - lo) / (M - 1)) > M - 1      # the rounding case
    X = np.array([[hi], [lo]])
    c = binning.bin_linear(X, [lo], [hi], [M])
    # the clamp puts t on M - 1 exactly: weight 1 on the last node, 0 on the one before
    assert c[-1] == 1.0 and c[-2] == 0.0 and c[0] == 1.0 and c.sum() == 2.0
    cs = binning.bin_simple(X, [lo], [hi], [M])
    assert cs[-1] == 1 and cs[0] == 1


def test_outside_points():
    X = np.array([[0.5, 0.5], [1.5, 0.5]])
    with pytest.raises(binning.OutsideGrid):
        binning.bin_linear(X, [0, 0], [1, 1], [4, 4])
    c = binning.bin_linear(X, [0, 0], [1, 1], [4, 4], policy="drop")
    assert c.sum() == pytest.approx(1.0)


# ---------------------------------------------------------------- direct sums

def test_direct_brute_force_scalar_loop():
    rng = np.random.default_rng(1)
    d, n = 2, 25
    X = rng.standard_normal((n, d))
    H = _spd(rng, d, 0.3)
    Hi = np.linalg.inv(H)
    nrm = 1.0 / (2 * math.pi * math.sqrt(np.linalg.det(H)))
    tot = 0.0
    for i in range(n):
        for j in range(n):
            u = X[i] - X[j]
            tot += nrm * math.exp(-0.5 * u @ Hi @ u)
    got = F.direct_sum(X, [(1.0, H, (0, 0))], block=7)
    assert got == pytest.approx(tot / n ** 2, rel=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_psi_closed_forms_n1_n2(d):
    rng = np.random.default_rng(20 + d)
    H = _spd(rng, d, 0.5)
    X1 = rng.standard_normal((1, d))
    for alpha in gauss.multi_indices(d, 4):
        got = F.direct_sum(X1, [(1.0, H, alpha)])
        assert got == pytest.approx(gauss.pairings_value_at_zero(H, alpha), rel=1e-12)
    X2 = rng.standard_normal((2, d))
    for alpha in gauss.multi_indices(d, 2):
        got = F.direct_sum(X2, [(1.0, H, alpha)])
        want = 0.5 * gauss.pairings_value_at_zero(H, alpha) + \
            0.5 * float(gauss.gauss_deriv((X2[0] - X2[1])[None], H, alpha)[0])
        assert got == pytest.approx(want, rel=1e-12)


def test_psi_invariants_scaling_rotation():
    rng = np.random.default_rng(9)
    d, n = 2, 40
    X = _mix(rng, n, d)
    H = _spd(rng, d, 0.4)
    ev = lambda X_: (lambda terms: F.direct_sum(X_, terms))
    # scaling: psi_alpha(c^2 H; c X) = c^{-d-|alpha|} psi_alpha(H; X)
    c = 1.7
    for r in (0, 2, 4):
        a = S.psi_vector(ev(X), H, r)
        b = S.psi_vector(ev(c * X), c * c * H, r)
        np.testing.assert_allclose(b, c ** (-d - r) * a, rtol=1e-11, atol=1e-15)
    # rotation: psi_r(R H R^T; X R^T) = R^{(x)r} psi_r(H; X)
    th = 0.61
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    for r in (2, 4):
        a = S.psi_vector(ev(X), H, r)
        b = S.psi_vector(ev(X @ R.T), R @ H @ R.T, r)
        Rk = R
        for _ in range(r - 1):
            Rk = np.kron(Rk, R)
        np.testing.assert_allclose(b, Rk @ a, rtol=1e-10, atol=1e-12)


def test_psi2_is_vec_hessian():
    """D^{(x)2} f = vec(Hessian f) (Sec. 5)."""
    rng = np.random.default_rng(4)
    d, n = 3, 12
    X = rng.standard_normal((n, d))
    H = _spd(rng, d, 0.5)
    v = S.psi_vector(lambda t: F.direct_sum(X, t), H, 2)
    Hess = np.zeros((d, d))
    for a in range(d):
        for b in range(d):
            al = [0] * d
            al[a] += 1
            al[b] += 1
            Hess[a, b] = F.direct_sum(X, [(1.0, H, tuple(al))])
    np.testing.assert_allclose(v, Hess.reshape(-1, order="F"), rtol=1e-13)


# ---------------------------------------------------------------- binned sums

def _binned_case(d, M, n=300, seed=0):
    rng = np.random.default_rng(seed)
    X = _mix(rng, n, d)
    lo, hi = X.min(0) - 0.2, X.max(0) + 0.2
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    return X, c, delta


@pytest.mark.parametrize("d,M,L", [(1, [40], [9]), (2, [20, 17], [6, 9]), (3, [9, 8, 10], [3, 4, 2])])
def test_fft_steps_equal_binned_double_sum(d, M, L):
    X, c, delta = _binned_case(d, M)
    rng = np.random.default_rng(d)
    H = _spd(rng, d, 0.2)
    for terms in (S.lscv_T_terms(H), [(1.0, H, tuple([2] + [0] * (d - 1)))]):
        ref = F.binned_direct(c, 300, terms, delta, L)
        for P in (rules.P_paper(M, L), rules.P_minimal(M, L)):
            got = F.binned_fft(c, 300, terms, delta, L, P)
            assert got == pytest.approx(ref, rel=1e-11, abs=1e-15)


def test_untruncated_layout_of_eqs_19_to_23():
    """With no truncation (L_k = M_k - 1, Eq. 17) and the padded size of
    Eq. 21 (2^ceil(log2(3 M_k - 1))), the printed layout holds as it stands:
    Eq. 23's extraction of M_k outputs from index 2 M_k - 2 (0-based)
    reproduces the binned double sum."""
    X, c, delta = _binned_case(2, [12, 10])
    H = _spd(np.random.default_rng(3), 2, 0.4)
    M = [12, 10]
    L = [m - 1 for m in M]
    assert rules.P_paper_full(M) == [64, 32]
    for terms in (S.lscv_T_terms(H), [(1.0, H, (1, 1))]):
        ref = F.binned_direct(c, 300, terms, delta, L)
        for P in (rules.P_paper_full(M), rules.P_paper(M, L), rules.P_minimal(M, L)):
            assert F.binned_fft(c, 300, terms, delta, L, P) == pytest.approx(ref, rel=1e-11, abs=1e-15)


def _parseval(c, n, terms, delta, L, P):
    """n^-2 P_tot^-1 sum_w |C_w|^2 K_w with k wrapped to j mod P: the
    frequency-domain form of Eq. 25 (discrete Parseval)."""
    d = c.ndim
    czp = np.zeros(P)
    czp[tuple(slice(0, m) for m in c.shape)] = c
    k = F.lag_kernel(terms, delta, L)
    kzp = np.zeros(P)
    for j in itertools.product(*[range(-l, l + 1) for l in L]):
        kzp[tuple(jj % p for jj, p in zip(j, P))] += k[tuple(jj + l for jj, l in zip(j, L))]
    C = np.fft.fftn(czp)
    K = np.fft.fftn(kzp)
    return float(np.sum(np.abs(C) ** 2 * K.real)) / np.prod(P) / n ** 2


def test_parseval_form_and_aliasing():
    rng = np.random.default_rng(5)
    c = rng.uniform(0.0, 3.0, size=(16, 14))     # mass up to the grid edges
    delta = np.array([0.11, 0.13])
    H = _spd(np.random.default_rng(8), 2, 0.5)
    L = [8, 7]
    terms = S.lscv_T_terms(H)
    ref = F.binned_direct(c, 300, terms, delta, L)
    for P in ([24, 21], [25, 24], [32, 32]):
        assert _parseval(c, 300, terms, delta, L, P) == pytest.approx(ref, rel=1e-11)
    # one short of M + L aliases
    bad = _parseval(c, 300, terms, delta, L, [23, 20])
    assert abs(bad - ref) > 1e-4 * abs(ref)


@pytest.mark.parametrize("d,M", [(1, [23]), (2, [9, 7]), (3, [5, 6, 4])])
def test_autocorrelation_pins(d, M):
    """a_0 = sum c^2; the half box with its weights covers every lag once,
    so over the whole lag range sum_full a_j = (sum c)^2; a brute-force
    double loop over cell pairs gives the same a_j; the half-box form
    n^-2 sum_half w_j k_j a_j is Eq. 25 (binned_direct)."""
    rng = np.random.default_rng(40 + d)
    c = rng.uniform(0.0, 2.0, size=M)
    A = [m - 1 for m in M]
    a = F.autocorr(c, A)
    w = F.half_box_weights(A)
    zero = tuple(A[k] for k in range(d - 1, 0, -1)) + (0,)
    assert a[zero] == pytest.approx(float(np.sum(c * c)), rel=1e-14)
    assert float(np.sum(w * a)) == pytest.approx(float(np.sum(c)) ** 2, rel=1e-13)
    # brute force over pairs of cells (i, i'), lag j = i' - i, on a few lags
    cells = list(np.ndindex(*M))
    for jj in [(1,) + (0,) * (d - 1), tuple([0] + [-1] * (d - 1)) if d > 1 else (2,), tuple(A)]:
        want = sum(c[i] * c[i2] for i in cells for i2 in cells
                   if all(i2[k] - i[k] == jj[k] for k in range(d)))
        idx = tuple(jj[k] + A[k] for k in range(d - 1, 0, -1)) + (jj[0],)
        assert a[idx] == pytest.approx(want, rel=1e-13, abs=1e-13)
    # the engine's formula: half box, weights, lag kernel
    delta = np.full(d, 0.3)
    H = _spd(np.random.default_rng(7), d, 0.3)
    L = [min(3, m - 1) for m in M]
    terms = S.lscv_T_terms(H)
    k = F.lag_kernel(terms, delta, L)      # full box, index j_k + L_k
    aL = F.autocorr(c, L)
    wL = F.half_box_weights(L)
    tot = 0.0
    for idx in np.ndindex(*aL.shape):
        j = [idx[-1]] + [idx[d - 1 - q] - L[q] for q in range(1, d)]
        tot += wL[idx] * aL[idx] * k[tuple(j[q] + L[q] for q in range(d))]
    assert tot / 300.0 ** 2 == pytest.approx(F.binned_direct(c, 300, terms, delta, L), rel=1e-12)


@pytest.mark.parametrize("d,M", [(1, [13]), (2, [9, 12]), (3, [5, 6, 4])])
def test_fft_autocorrelation_and_lag_sums(d, M):
    """The FFT autocorrelation equals the direct lag overlaps on every lag of
    the half box, and the lag-first sum equals Eq. 25's double sum; the
    absolute functional equals the double sum of |k|."""
    X, c, delta = _binned_case(d, M, n=250, seed=40 + d)
    a = F.autocorr_fft(c)
    A = [m - 1 for m in M]
    ref = F.autocorr(c, A)
    for idx in np.ndindex(*ref.shape):
        j = [idx[-1]] + [idx[d - 1 - k] - A[k] for k in range(1, d)]
        got = a[tuple(jj % a.shape[k] for k, jj in enumerate(j))]
        assert got == pytest.approx(ref[idx], rel=1e-12, abs=1e-9 * ref.max())
    rng = np.random.default_rng(d)
    H = _spd(rng, d, 0.5)
    L = [min(m - 1, 3 + k) for k, m in enumerate(M)]
    terms = [(1.0, H, (0,) * d), (-0.7, 2.0 * H, tuple([2] + [0] * (d - 1)))]
    v, s_abs = F.lag_sums(a, 250, terms, delta, L)
    assert v == pytest.approx(F.binned_direct(c, 250, terms, delta, L), rel=1e-11)
    k = F.lag_kernel(terms, delta, L)
    want = 0.0
    for j in itertools.product(*[range(-l, l + 1) for l in L]):
        want += abs(k[tuple(jj + l for jj, l in zip(j, L))]) * F._overlap(c, j)
    assert s_abs == pytest.approx(want / 250.0 ** 2, rel=1e-11)


def test_binned_equals_direct_on_nodes():
    """All points on nodes and L = M - 1: binned sum = direct sum."""
    rng = np.random.default_rng(2)
    M = [11, 9]
    lo, hi = np.array([-1.0, -2.0]), np.array([1.5, 1.0])
    g = binning.grid_points(lo, hi, M)
    idx = rng.integers(0, 9, size=(50, 2))
    X = np.stack([g[0][idx[:, 0]], g[1][idx[:, 1]]], axis=1)
    c = binning.bin_linear(X, lo, hi, M)
    H = _spd(rng, 2, 0.3)
    delta = rules.bin_width(lo, hi, M)
    for terms in (S.lscv_T_terms(H), [(1.0, H, (2, 2))]):
        a = F.binned_direct(c, 50, terms, delta, [10, 8])
        b = F.direct_sum(X, terms)
        assert a == pytest.approx(b, rel=1e-11)


def test_binning_error_is_second_order():
    """Binned-vs-direct error falls about 4x when the grid spacing halves."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((400, 2))
    H = np.array([[0.3, 0.1], [0.1, 0.4]])
    terms = S.lscv_T_terms(H)
    ref = F.direct_sum(X, terms)
    lo, hi = X.min(0) - 0.5, X.max(0) + 0.5
    errs = []
    for m in (21, 41, 81):
        M = [m, m]
        c = binning.bin_linear(X, lo, hi, M)
        delta = rules.bin_width(lo, hi, M)
        errs.append(abs(F.binned_fft(c, 400, terms, delta, [m - 1, m - 1], [2 * m, 2 * m]) - ref))
    for e1, e2 in zip(errs, errs[1:]):
        assert 2.5 < e1 / e2 < 6.0


def test_riemann_sum_of_T_is_minus_one():
    H = np.array([[0.2, 0.07], [0.07, 0.15]])
    delta = [0.02, 0.02]
    L = [300, 300]
    k = F.lag_kernel(S.lscv_T_terms(H), delta, L)
    assert float(np.prod(delta) * k.sum()) == pytest.approx(-1.0, abs=1e-9)


def test_mirrored_lag_layout_fails_for_full_H():
    """Wand's reshaping uses k_{|j_1|,|j_2|}: exact for diagonal H, wrong for
    off-diagonal H (Sec. 2, the corrupted estimate)."""
    X, c, delta = _binned_case(2, [18, 18], seed=3)
    L = [10, 10]

    def mirrored(terms):
        k = F.lag_kernel(terms, delta, L)
        tot = 0.0
        for j in itertools.product(range(-L[0], L[0] + 1), range(-L[1], L[1] + 1)):
            tot += k[abs(j[0]) + L[0], abs(j[1]) + L[1]] * F._overlap(c, j)
        return tot / 300 ** 2

    Hd = np.diag([0.2, 0.3])
    assert mirrored(S.lscv_T_terms(Hd)) == pytest.approx(F.binned_direct(c, 300, S.lscv_T_terms(Hd), delta, L), rel=1e-12)
    Hf = np.array([[0.2, 0.15], [0.15, 0.3]])
    a = mirrored(S.lscv_T_terms(Hf))
    b = F.binned_direct(c, 300, S.lscv_T_terms(Hf), delta, L)
    assert abs(a - b) > 1e-3 * abs(b)
    # the correct functional is invariant under (H_12, x_2) -> (-H_12, -x_2)
    Hm = Hf * np.array([[1, -1], [-1, 1]])
    Xm = X * np.array([1.0, -1.0])
    assert F.direct_sum(Xm, S.lscv_T_terms(Hm)) == pytest.approx(F.direct_sum(X, S.lscv_T_terms(Hf)), rel=1e-12)


def test_normal_population_limit():
    """For X ~ N(0, Sigma): E psi_alpha = n^-1 d^alpha phi_H(0) +
    (1 - n^-1) d^alpha phi_{H + 2 Sigma}(0); Monte Carlo with a CLT tolerance
    (5 standard errors, Var ~ 4 Var_i(row mean) / n for a V-statistic)."""
    rng = np.random.default_rng(31)
    d, n = 2, 1500
    Sig = np.array([[1.0, 0.4], [0.4, 0.7]])
    H = np.array([[0.2, 0.05], [0.05, 0.15]])
    X = rng.standard_normal((n, d)) @ np.linalg.cholesky(Sig).T
    diff = X[:, None, :] - X[None, :, :]
    for alpha in [(0, 0), (2, 0), (1, 1)]:
        got = F.direct_sum(X, [(1.0, H, alpha)])
        rows = gauss.gauss_deriv(diff, H, alpha).mean(axis=1)
        se = math.sqrt(4.0 * rows.var() / n)
        want = gauss.pairings_value_at_zero(H, alpha) / n + \
            (1 - 1 / n) * gauss.pairings_value_at_zero(H + 2 * Sig, alpha)
        assert abs(got - want) < 5.0 * se
        assert se < 0.2 * abs(want)


# ---------------------------------------------------------------- selectors

def _ev_binned(c, n, delta, L):
    return lambda terms: F.binned_direct(c, n, terms, delta, L)


@pytest.mark.parametrize("exact", [False, True])
def test_lscv_gradient_by_finite_differences(exact):
    X, c, delta = _binned_case(2, [20, 20], n=200, seed=4)
    L = [8, 8]
    ev = _ev_binned(c, 200, delta, L)
    H = np.array([[0.35, 0.12], [0.12, 0.25]])
    _, g = S.lscv(ev, H, 200, exact_loo=exact, grad=True)
    h = 1e-5
    for a, b in itertools.product(range(2), repeat=2):   # every entry, both triangles
        E = np.zeros((2, 2))
        E[a, b] = E[b, a] = 1.0
        fd = (S.lscv(ev, H + h * E, 200, exact) - S.lscv(ev, H - h * E, 200, exact)) / (2 * h)
        assert g[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_scv_and_pi_gradients_by_finite_differences():
    X, c, delta = _binned_case(2, [18, 18], n=200, seed=6)
    ev = _ev_binned(c, 200, delta, [10, 10])
    H = np.array([[0.3, -0.08], [-0.08, 0.22]])
    G = np.array([[0.2, 0.03], [0.03, 0.25]])
    _, g = S.scv(ev, H, G, 200, grad=True)
    psi4 = S.psi_vector(ev, G, 4)
    _, gp = S.pi_from_psi4(psi4, H, 200, grad=True)
    h = 1e-5
    for a, b in itertools.product(range(2), repeat=2):   # every entry, both triangles
        E = np.zeros((2, 2))
        E[a, b] = E[b, a] = 1.0
        fd = (S.scv(ev, H + h * E, G, 200) - S.scv(ev, H - h * E, G, 200)) / (2 * h)
        assert g[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        fdp = (S.pi_from_psi4(psi4, H + h * E, 200) - S.pi_from_psi4(psi4, H - h * E, 200)) / (2 * h)
        assert gp[a, b] == pytest.approx(fdp, rel=1e-6, abs=1e-9)


def test_pi_eta02_route_equals_psi4_contraction():
    rng = np.random.default_rng(8)
    X = _mix(rng, 60, 3)
    ev = lambda t: F.direct_sum(X, t)
    H = _spd(rng, 3, 0.2)
    G = _spd(rng, 3, 0.3)
    a = S.pi_from_psi4(S.psi_vector(ev, G, 4), H, 60)
    b = S.pi_eta(ev, H, G, 60)
    assert a == pytest.approx(b, rel=1e-11)


# ---------------------------------------------------------------- SCV and PI by quadrature
#
# Both readings (SCV and PI are named in Sec. 3; Sec. 5 defers their formulas)
# are pinned here to integrals of plain kernel estimates, evaluated by a
# Riemann sum on a uniform box.  For Gaussian integrands the uniform sum
# converges faster than any power of the step (its aliasing error is about
# exp(-2 pi^2 sd^2 / h^2)), so a step of a quarter of the narrowest standard
# deviation and a box reaching ten of the widest ones beyond the sample give
# the integral to rounding.  The densities and the Hessian below are written
# out from the normal density, without the oracle's Hermite recurrence.

def _normal_pdf_2d(P, mu, Sg):
    """phi_Sigma(P - mu) for an array of points P (..., 2)."""
    Sg = np.asarray(Sg, dtype=np.float64)
    Li = np.linalg.inv(Sg)
    y = P - mu
    q = np.einsum("...a,ab,...b->...", y, Li, y)
    return np.exp(-0.5 * q) / (2.0 * math.pi * math.sqrt(np.linalg.det(Sg)))


def _plain_kde(P, X, Sg):
    """f_hat_Sigma(P) = n^-1 sum_i phi_Sigma(P - X_i) (Eq. 1 with a Gaussian K_Sigma)."""
    return sum(_normal_pdf_2d(P, x, Sg) for x in X) / len(X)


def _quad_box(X, covs, pad=10.0, per_sd=4.0):
    """Nodes of a uniform box holding every kernel's mass around the sample,
    and the area of one cell."""
    sd_max = max(math.sqrt(np.linalg.eigvalsh(C).max()) for C in covs)
    sd_min = min(math.sqrt(np.linalg.eigvalsh(C).min()) for C in covs)
    lo, hi = X.min(0) - pad * sd_max, X.max(0) + pad * sd_max
    h = sd_min / per_sd
    axes = [np.arange(lo[k], hi[k] + h, h) for k in range(2)]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1), h * h


def _scv_pi_case():
    rng = np.random.default_rng(21)
    n = 30
    X = rng.standard_normal((n, 2))
    X[: n // 2] += [1.2, -0.4]
    H = np.array([[0.30, -0.09], [-0.09, 0.22]])
    G = np.array([[0.18, 0.05], [0.05, 0.26]])
    return X, H, G


def test_scv_is_integrated_squared_difference_of_estimates():
    """SCV(H) - n^-1 R(K_H) = int (f_hat_{H+G} - f_hat_G)^2: the smoothed
    bootstrap's integrated squared bias, K_H * f_hat_G - f_hat_G with the
    pilot estimate f_hat_G; K_H * f_hat_G = f_hat_{H+G} for Gaussians.  The
    double-sum reading convolves the Gaussians pairwise (2H + 2G, H + 2G,
    2G); here the integral is taken numerically."""
    X, H, G = _scv_pi_case()
    n = len(X)
    P, dA = _quad_box(X, [H + G, G])
    quad = float(np.sum((_plain_kde(P, X, H + G) - _plain_kde(P, X, G)) ** 2) * dA)
    got = S.scv(lambda t: F.direct_sum(X, t), H, G, n) - S.RK(H) / n
    assert got == pytest.approx(quad, rel=1e-10)
    # the n^-1 R(K_H) term is int K_H^2, also by quadrature
    Pk, dAk = _quad_box(np.zeros((1, 2)), [H])
    assert S.RK(H) == pytest.approx(float(np.sum(_normal_pdf_2d(Pk, 0.0, H) ** 2) * dAk), rel=1e-10)


def _trace_H_hessian_of_kde(P, X, H, Sg):
    """tr(H grad grad^T f_hat_Sigma)(P), with grad grad^T phi_Sigma(y) =
    (Lambda y y^T Lambda - Lambda) phi_Sigma(y), Lambda = Sigma^-1."""
    Li = np.linalg.inv(Sg)
    out = 0.0
    for x in X:
        z = (P - x) @ Li.T
        quad = np.einsum("...a,ab,...b->...", z, H, z)
        out = out + (quad - np.trace(H @ Li)) * _normal_pdf_2d(P, x, Sg)
    return out / len(X)


def test_pi_contraction_is_integrated_squared_hessian_trace():
    """(vec^T H)^{(x)2} psi_4(G) = int (tr(H grad grad^T f_hat_{G/2}))^2
    (integration by parts twice, and phi_{G/2} * phi_{G/2} = phi_G): the
    contraction the plug-in reading uses, from psi_4 of Eq. 13 and from the
    eta_{0,2} kernel of Eq. 30, against a numerical integral."""
    X, H, G = _scv_pi_case()
    n = len(X)
    P, dA = _quad_box(X, [G / 2.0])
    quad = float(np.sum(_trace_H_hessian_of_kde(P, X, H, G / 2.0) ** 2) * dA)
    ev = lambda t: F.direct_sum(X, t)
    T = S.psi_vector(ev, G, 4).reshape((2, 2, 2, 2))
    assert float(np.einsum("ab,ce,abce->", H, H, T)) == pytest.approx(quad, rel=1e-10)
    assert ev(S.eta02_terms(H, G)) == pytest.approx(quad, rel=1e-10)


def test_pi_is_the_small_bandwidth_limit_of_the_exact_bias():
    """The plug-in term is the leading order of the exact integrated squared
    bias: int (f_hat_{G/2 + tH} - f_hat_{G/2})^2 = t^2 (PI(H) - n^-1 R(K_H))
    + O(t^3) as t -> 0 (heat equation: phi_{S + tH} = exp(t/2 tr(H grad
    grad^T)) phi_S, whose second-order term squared carries 1/4).  This fixes
    the reading's factor 1/4, on both routes, without restating it: the
    bias is integrated numerically at t, t/2, t/4 and extrapolated to t = 0."""
    X, H, G = _scv_pi_case()
    n = len(X)
    Gh = G / 2.0
    P, dA = _quad_box(X, [Gh])
    f0 = _plain_kde(P, X, Gh)
    r = lambda t: float(np.sum((_plain_kde(P, X, Gh + t * H) - f0) ** 2) * dA) / t ** 2
    t = 0.01
    lim = (8.0 * r(t / 4) - 6.0 * r(t / 2) + r(t)) / 3.0   # removes the O(t) and O(t^2) terms
    ev = lambda tt: F.direct_sum(X, tt)
    want_psi4 = S.pi_from_psi4(S.psi_vector(ev, G, 4), H, n) - S.RK(H) / n
    want_eta = S.pi_eta(ev, H, G, n) - S.RK(H) / n
    assert want_psi4 == pytest.approx(lim, rel=1e-3)
    assert want_eta == pytest.approx(lim, rel=1e-3)


def test_scv_single_point_closed_form():
    H = np.array([[0.3, 0.1], [0.1, 0.2]])
    G = np.array([[0.15, 0.0], [0.0, 0.1]])
    X = np.array([[0.3, -0.2]])
    got = S.scv(lambda t: F.direct_sum(X, t), H, G, 1)
    phi0 = lambda Sg: 1.0 / (2 * math.pi * math.sqrt(np.linalg.det(Sg)))
    want = 1.0 / (4 * math.pi * math.sqrt(np.linalg.det(H))) + \
        phi0(2 * H + 2 * G) - 2 * phi0(H + 2 * G) + phi0(2 * G)
    assert got == pytest.approx(want, rel=1e-13)


def test_lscv_loo_forms_and_lscv_r0():
    rng = np.random.default_rng(13)
    X = _mix(rng, 80, 2)
    ev = lambda t: F.direct_sum(X, t)
    H = np.array([[0.25, 0.05], [0.05, 0.3]])
    n = 80
    # Eq. 8 evaluated literally with an explicit j != i loop
    Hi2, Hi = np.linalg.inv(2 * H), np.linalg.inv(H)
    p2 = 1 / (2 * math.pi * math.sqrt(np.linalg.det(2 * H)))
    p1 = 1 / (2 * math.pi * math.sqrt(np.linalg.det(H)))
    a = b = 0.0
    for i in range(n):
        for j in range(n):
            u = X[i] - X[j]
            a += p2 * math.exp(-0.5 * u @ Hi2 @ u)
            if i != j:
                b += p1 * math.exp(-0.5 * u @ Hi @ u)
    eq8 = a / n ** 2 - 2 * b / (n * (n - 1))
    assert S.lscv(ev, H, n, exact_loo=True) == pytest.approx(eq8, rel=1e-12)
    # Eq. 10 form differs from Eq. 8 by O(1/n)
    assert abs(S.lscv(ev, H, n) - eq8) < 5.0 / n * abs(eq8) + 1e-3
    # Eqs. 35-36 at r = 0 reduce to Eqs. 8 and 10
    assert S.lscv_r(ev, H, n, 0, exact_loo=True) == pytest.approx(eq8, rel=1e-12)
    assert S.lscv_r(ev, H, n, 0) == pytest.approx(S.lscv(ev, H, n), rel=1e-12)


def test_eta_r_is_iterated_laplacian():
    sp = pytest.importorskip("sympy")
    Sg = np.array([[0.5, 0.2], [0.2, 0.4]])
    x0, x1 = sp.symbols("x0 x1")
    Lam = sp.Matrix(np.linalg.inv(Sg).tolist())
    v = sp.Matrix([x0, x1])
    phi = 1 / (2 * sp.pi * sp.sqrt(sp.Float(np.linalg.det(Sg), 30))) * sp.exp(-(v.T * Lam * v)[0, 0] / 2)
    pt = np.array([[0.3, -0.4]])
    f = phi
    for r in (1, 2):
        f = sp.diff(f, x0, 2) + sp.diff(f, x1, 2)
        want = float(f.subs({x0: pt[0, 0], x1: pt[0, 1]}))
        got = float(gauss.kernel_eval(pt, S.eta_r_terms(Sg, r))[0])
        assert got == pytest.approx(want, rel=1e-10)


def test_eta_rs_reduces_to_eta02_and_eta_r():
    """Eq. 30 in general: r = 0, s = 2 gives eta_{0,2} (Eq. 30's special
    case used by the plug-in functional); A = I, s = 0 gives the iterated
    Laplacian eta_r (Eq. 31); swapping (A, r) with (B, s) permutes the
    Kronecker factors of a symmetric derivative tensor and changes
    nothing; and at a point the weights reproduce the brute-force
    contraction of the full Kronecker vectors."""
    rng = np.random.default_rng(12)
    for d in (2, 3):
        A = _spd(rng, d, 0.5)
        B = _spd(rng, d, 0.7)
        Sg = _spd(rng, d, 0.4)
        as_dict = lambda terms: {a: w for w, _, a in terms}
        e02 = as_dict(S.eta02_terms(B, Sg))
        g02 = as_dict(S.eta_rs_terms(A, B, Sg, 0, 2))
        assert e02.keys() == g02.keys() and all(abs(e02[k] - g02[k]) <= 1e-12 * abs(e02[k]) for k in e02)
        for m in (1, 2):
            er = as_dict(S.eta_r_terms(Sg, m))
            gr = as_dict(S.eta_rs_terms(np.eye(d), B, Sg, m, 0))
            assert er.keys() == gr.keys() and all(abs(er[k] - gr[k]) <= 1e-12 * abs(er[k]) for k in er)
        x = rng.standard_normal(d) * 0.3
        v1 = gauss.kernel_eval(x, S.eta_rs_terms(A, B, Sg, 1, 1))
        v2 = gauss.kernel_eval(x, S.eta_rs_terms(B, A, Sg, 1, 1))
        assert v1 == pytest.approx(v2, rel=1e-12)
        # brute force at x: sum over all index tuples of A_ab B_ce d_a d_b d_c d_e phi
        want = 0.0
        for a, b, c, e in itertools.product(range(d), repeat=4):
            al = [0] * d
            for i in (a, b, c, e):
                al[i] += 1
            want += A[a, b] * B[c, e] * float(gauss.gauss_deriv(x, Sg, tuple(al)))
        assert v1 == pytest.approx(want, rel=1e-10)


def test_lscv_r_is_cross_validation_of_the_derivative():
    """Eq. 35 is least-squares cross-validation of the r-th derivative
    estimate: up to the constant int |D^r f|^2 it is

        int |D^{(x)r} f_hat|^2 - 2 (-1)^r n^-1 sum_i Lap^r f_hat_{-i}(X_i),

    since int D^r f_hat . D^r f = (-1)^r int f Lap^r f_hat (integration by
    parts) and f_hat_{-i} leaves X_i out.  Both parts are computed here
    without the Hermite partials: the first by a Riemann sum of the squared
    gradient (r = 1, d = 2) or second derivative (r = 2, d = 1) written out
    by hand, the second by central finite differences of the leave-one-out
    density."""
    rng = np.random.default_rng(31)
    # r = 1, d = 2
    n = 30
    X = 0.6 * _mix(rng, n, 2)
    H = np.array([[0.2, 0.05], [0.05, 0.15]])
    Hi = np.linalg.inv(H)
    nrm = 1.0 / (2 * math.pi * math.sqrt(np.linalg.det(H)))

    def dens(x, pts):
        u = x[:, None, :] - pts[None, :, :]
        return nrm * np.exp(-0.5 * np.einsum("pqi,ij,pqj->pq", u, Hi, u))

    h = 0.05
    axes = [np.arange(X[:, k].min() - 3.0, X[:, k].max() + 3.0, h) for k in range(2)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 2)
    u = g[:, None, :] - X[None, :, :]
    grad = -np.einsum("ij,pqj->pi", Hi, u * dens(g, X)[:, :, None]) / n
    quad = float(np.sum(grad * grad)) * h * h
    e = 1e-3
    lap = 0.0
    for i in range(n):
        rest = np.delete(X, i, axis=0)
        f = lambda x: float(np.sum(dens(x[None, :], rest))) / (n - 1)
        for k in range(2):
            ek = np.eye(2)[k] * e
            lap += (f(X[i] + ek) - 2 * f(X[i]) + f(X[i] - ek)) / (e * e)
    want = quad + 2.0 * lap / n
    ev = lambda t: F.direct_sum(X, t)
    got = S.lscv_r(ev, H, n, 1, exact_loo=True)
    assert got == pytest.approx(want, rel=1e-6, abs=1e-6 * (abs(quad) + abs(2.0 * lap / n)))
    # r = 2, d = 1
    n = 25
    x1 = rng.standard_normal(n) * 0.8
    s2 = 0.1
    phi = lambda x: np.exp(-0.5 * x * x / s2) / math.sqrt(2 * math.pi * s2)
    xs = np.arange(x1.min() - 3.0, x1.max() + 3.0, 0.005)
    u = xs[:, None] - x1[None, :]
    f2 = np.sum((u * u / (s2 * s2) - 1.0 / s2) * phi(u), axis=1) / n
    quad = float(np.sum(f2 * f2)) * 0.005
    e = 5e-3
    d4 = 0.0
    for i in range(n):
        rest = np.delete(x1, i)
        f = lambda x: float(np.sum(phi(x - rest))) / (n - 1)
        xi = x1[i]
        d4 += (f(xi + 2 * e) - 4 * f(xi + e) + 6 * f(xi) - 4 * f(xi - e) + f(xi - 2 * e)) / e ** 4
    want = quad - 2.0 * d4 / n
    got = S.lscv_r(lambda t: F.direct_sum(x1[:, None], t), np.array([[s2]]), n, 2, exact_loo=True)
    assert got == pytest.approx(want, abs=1e-3 * (abs(quad) + abs(2.0 * d4 / n)))
