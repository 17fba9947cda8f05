"""Edge cases of the path against the oracle (Sec. 4's binned sums, Eqs. 8,
10-13, 25-27).

- The smallest samples: one point, and many points at one place.  Every
  functional is the oracle's binned double sum over the 2^d linear-binning
  weights of that place.  The normal-scale start of a selection has a zero
  covariance there and is refused (KDEFFT_ERR_NOT_SPD, or KDEFFT_ERR_ARG
  for a start below the grid's resolution); Eq. 8's
  leave-one-out form has no value for one point and is refused
  (KDEFFT_ERR_ARG).
- The largest padded size: a bandwidth wide enough that the support is the
  whole grid (L_k = M_k - 1) on a 2048-node axis needs P_k = 4096, the
  limit.  Values against the oracle there, in 1-D (both precisions) and with
  a second axis.
- The first sizes past it (2100 nodes with the whole grid as support; the
  paper's power-of-two padding, Eq. 27, of the 2048-node box) are refused
  with KDEFFT_ERR_UNSUPPORTED before any launch, and the dataset stays
  usable for narrower bandwidths.
- An empty sample is refused (KDEFFT_ERR_ARG).

Failures are made on the host (arguments the library refuses); nothing
faults or waits on the device.  Tolerances as in the parity tests: FP32
|got - ref| / max(|ref|, S/10) <= 1e-5 with S the magnitude of the summed
terms, FP64 1e-11 relative."""
import numpy as np
import pytest

from oracle import binning, functionals as F, gauss, rules, selectors as S

pytestmark = pytest.mark.gpu

ERR_ARG, ERR_NOT_SPD, ERR_UNSUPPORTED = 1, 2, 7
GRIDS = {1: [41], 2: [33, 29], 3: [15, 13, 11]}
PLACE = [0.3137, -0.2219, 0.1411]


@pytest.fixture(scope="module")
def ctx():
    from paper_1511_07482_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _bw(d, diag, off):
    return diag * np.eye(d) + off * (np.ones((d, d)) - np.eye(d))


def _err(got, ref, sabs):
    return abs(got - ref) / max(abs(ref), 0.1 * sabs)


def _launches(c):
    return c.profile_read()[1]


def _check_functionals(ds, X, lo, hi, M, H, G, tol, rs=(0, 2, 4)):
    """psi_r (every Kronecker entry), LSCV with its gradient and SCV with
    its gradient at H against the oracle's lag sums over the oracle's
    counts, each at the support the library reports (itself checked against
    Eq. 26)."""
    n, d = X.shape
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    a = F.autocorr_fft(c)

    def ev_at(L):
        return (lambda t: F.lag_sums(a, n, t, delta, L)[0]), (lambda t: F.lag_sums(a, n, t, delta, L)[1])

    for r in rs:
        got = ds.psi(H, r)[0]
        L, P = ds.plan(-1, H)
        assert list(L) == [max(1, x) for x in rules.support_L(rules.lambda_max(H), delta, M)]
        assert list(P) == rules.P_minimal(M, list(L))
        ev, ev_abs = ev_at(list(L))
        for pos, alpha in enumerate(gauss.kron_alphas(d, r)):
            t = [(1.0, H, alpha)]
            assert _err(got[pos], ev(t), ev_abs(t)) <= tol, (r, alpha, got[pos], ev(t))
    L, _ = ds.plan(0, H)
    ev, ev_abs = ev_at(list(L))
    v, g = ds.lscv(H, grad=True)
    rv, rg = S.lscv(ev, H, n, grad=True)
    sv, sg = S.abs_scales(ev_abs, "lscv", H, n)
    assert _err(v[0], rv, sv) <= tol, (v[0], rv)
    assert np.max(np.abs(g[0] - rg) / np.maximum(np.abs(rg), 0.1 * sg)) <= tol, (g[0], rg)
    L, _ = ds.plan(1, H, G)
    assert list(L) == [max(1, x) for x in rules.support_L(rules.lambda_max(2 * H + 2 * G), delta, M)]
    ev, ev_abs = ev_at(list(L))
    v, g = ds.scv(H, G, grad=True)
    rv, rg = S.scv(ev, H, G, n, grad=True)
    sv, sg = S.abs_scales(ev_abs, "scv", H, n, G)
    assert _err(v[0], rv, sv) <= tol, (v[0], rv)
    assert np.max(np.abs(g[0] - rg) / np.maximum(np.abs(rg), 0.1 * sg)) <= tol, (g[0], rg)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n", [1, 40])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_one_point_and_coincident_points(ctx, d, n, precision):
    from paper_1511_07482_gb300 import FP32, FP64, LSCV, SCV, KdefftError
    M = GRIDS[d]
    lo, hi = -np.ones(d), np.ones(d)
    X = np.tile(np.array(PLACE[:d]), (n, 1))
    H, G = _bw(d, 0.04, 0.01), _bw(d, 0.03, 0.0)
    ds = ctx.bin(X, lo, hi, M, precision=FP64 if precision == "fp64" else FP32)
    assert ds.info() == (n, d, 0)
    assert np.isclose(ds.counts().sum(), n, rtol=1e-6)
    _check_functionals(ds, X, lo, hi, M, H, G, 1e-11 if precision == "fp64" else 1e-5)
    # every point at one place.  One point: the normal-scale matrix (start and
    # pilot) is zero, not positive definite.  Coincident points: the one-pass
    # covariance leaves at most a rounding residue, so the normal-scale start
    # is not positive definite or lies far below the grid's resolution
    # (outside the search domain); a pilot of that size may still be SPD, so
    # only the start is checked there
    if n == 1:
        calls, codes = (lambda: ds.select_H(LSCV), lambda: ds.select_H(SCV, H0=H),
                        lambda: ds.select_H_many([LSCV, SCV])), (ERR_NOT_SPD,)
    else:
        calls, codes = (lambda: ds.select_H(LSCV),), (ERR_NOT_SPD, ERR_ARG)
    for call in calls:
        with pytest.raises(KdefftError) as e:
            call()
        assert e.value.code in codes
    # Eq. 8's leave-one-out sum: refused for one point, the oracle's value otherwise
    if n == 1:
        for call in (lambda: ctx.bin(X, lo, hi, M, exact_loo=1), lambda: ds.set_opts(exact_loo=1),
                     lambda: ctx.bin_many([X, X], [lo, lo], [hi, hi], [M, M], exact_loo=1)):
            with pytest.raises(KdefftError) as e:
                call()
            assert e.value.code == ERR_ARG
    else:
        ds.set_opts(exact_loo=1)
        c = binning.bin_linear(X, lo, hi, M)
        delta = rules.bin_width(lo, hi, M)
        L, _ = ds.plan(0, H)
        a = F.autocorr_fft(c)
        rv = S.lscv(lambda t: F.lag_sums(a, n, t, delta, list(L))[0], H, n, exact_loo=True)
        got = ds.lscv(H)[0]
        assert abs(got - rv) <= (1e-11 if precision == "fp64" else 1e-5) * abs(rv), (got, rv)
    ds.close()


def _wide_sample(rng, n, d):
    """A two-component normal mixture clipped to [-0.99, 0.99]^d."""
    half = n // 2
    X = np.vstack([rng.normal(-0.3, 0.2, size=(half, d)), rng.normal(0.35, 0.25, size=(n - half, d))])
    return np.clip(X, -0.99, 0.99)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_largest_padding_1d(ctx, precision):
    """M = 2048 and a support of the whole grid: P = 4096 (the limit) for
    psi_r, LSCV and SCV."""
    from paper_1511_07482_gb300 import FP32, FP64
    X = _wide_sample(np.random.default_rng(301), 20000, 1)
    lo, hi, M = np.array([-1.0]), np.array([1.0]), [2048]
    H, G = np.array([[0.36]]), np.array([[0.09]])
    ds = ctx.bin(X, lo, hi, M, precision=FP64 if precision == "fp64" else FP32)
    for method, Gx in ((-1, None), (0, None), (1, G)):
        L, P = ds.plan(method, H, Gx)
        assert list(L) == [2047] and list(P) == [4096]
    _check_functionals(ds, X, lo, hi, M, H, G, 1e-11 if precision == "fp64" else 1e-5)
    ds.close()


def test_largest_padding_2d(ctx):
    """M = [2048, 16] with the whole grid as support on both axes: P =
    [4096, 32]; a correlated H."""
    X = _wide_sample(np.random.default_rng(302), 30000, 2)
    lo, hi, M = -np.ones(2), np.ones(2), [2048, 16]
    H = np.array([[0.36, 0.012], [0.012, 0.02]])
    G = np.array([[0.09, 0.0], [0.0, 0.01]])
    ds = ctx.bin(X, lo, hi, M)
    L, P = ds.plan(0, H)
    assert list(L) == [2047, 15] and list(P) == [4096, 32]
    _check_functionals(ds, X, lo, hi, M, H, G, 1e-5, rs=(0, 4))
    ds.close()


def test_padding_past_the_limit_is_refused(ctx):
    from paper_1511_07482_gb300 import P_PAPER, KdefftError
    rng = np.random.default_rng(303)
    X = _wide_sample(rng, 5000, 1)
    lo, hi = np.array([-1.0]), np.array([1.0])
    wide, narrow = np.array([[0.36]]), np.array([[0.01]])
    cases = [(ctx.bin(X, lo, hi, [2100]), wide),                 # M + L = 4199: P would be 4320
             (ctx.bin(X, lo, hi, [2048], P_rule=P_PAPER), wide)]  # Eq. 27: P would be 8192
    for ds, H in cases:
        ctx.profile(0)   # clears the launch counter
        for call in (lambda: ds.plan(0, H), lambda: ds.lscv(H), lambda: ds.psi(H, 2),
                     lambda: ds.scv(H, np.array([[0.09]]))):
            with pytest.raises(KdefftError) as e:
                call()
            assert e.value.code == ERR_UNSUPPORTED
        assert _launches(ctx) == 0
    # the 2100-node dataset still evaluates a narrower bandwidth (L = 389,
    # P = 2500)
    ds = cases[0][0]
    M = [2100]
    L, P = ds.plan(0, narrow)
    assert list(L) == rules.support_L(rules.lambda_max(narrow), rules.bin_width(lo, hi, M), M)
    assert list(P) == [2500]
    _check_functionals(ds, X, lo, hi, M, narrow, np.array([[0.0025]]), 1e-5, rs=(0, 2))
    for ds, _ in cases:
        ds.close()


def test_empty_sample_is_refused(ctx):
    from paper_1511_07482_gb300 import KdefftError
    for d in (1, 2, 4):
        with pytest.raises(KdefftError) as e:
            ctx.bin(np.zeros((0, d)), -np.ones(d), np.ones(d), [8] * d)
        assert e.value.code == ERR_ARG
    with pytest.raises(KdefftError) as e:
        ctx.bin_many([np.zeros((0, 2)), np.zeros((10, 2))], [-np.ones(2)] * 2, [np.ones(2)] * 2, [[8, 8]] * 2)
    assert e.value.code == ERR_ARG
