"""eta_r V-statistics and LSCV_r on the device (Eqs. 31-32, 35-36): Q_r for
the total derivative orders of the paper's V-statistics experiment
(r = 0, 2, 4, 6, 8 on a bivariate normal sample) and in 1-D and 3-D, and
LSCV_r for density-derivative orders r <= 4, against the oracle's binned
sums of the same kernels (Eq. 25)."""
import numpy as np
import pytest

from oracle import binning, functionals as F, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["auto", "fft"])
def ctx(request):
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, Context
    c = Context(0)
    c.set_engine(ENGINE_AUTO if request.param == "auto" else ENGINE_FFT)
    yield c
    c.close()


def _abs_functional(c, n, terms, delta, L):
    k = np.abs(F.lag_kernel(terms, delta, L))
    a = F.autocorr(c, L)
    w = F.half_box_weights(L)
    d = len(L)
    tot = 0.0
    for idx in np.ndindex(*a.shape):
        j = [idx[-1]] + [idx[d - 1 - q] - L[q] for q in range(1, d)]
        tot += w[idx] * a[idx] * k[tuple(j[q] + L[q] for q in range(d))]
    return tot / float(n) ** 2


def _err(got, ref, Sabs):
    return abs(got - ref) / max(abs(ref), 0.1 * Sabs)


def _normal2(n, M, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 2))
    Hns = synthetic.normal_scale(X)
    lo, hi = synthetic.grid_range(X, Hns)
    return X, lo, hi, Hns


@pytest.mark.parametrize("r", [0, 2, 4, 6, 8])
def test_qr_bivariate_normal_all_orders(ctx, r):
    X, lo, hi, Hns = _normal2(4000, [50, 50], 91)
    M = [50, 50]
    ds = ctx.bin(X, lo, hi, M)
    Sig = [Hns, 2.0 * Hns, np.array([[0.08, 0.02], [0.02, 0.05]])]
    got = ds.qr(np.stack(Sig), r)
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    for g, Sg in zip(got, Sig):
        L = rules.support_L(rules.lambda_max(Sg), delta, M)
        terms = S.eta_r_terms(Sg, r // 2)
        ref = F.binned_direct(c, X.shape[0], terms, delta, L)
        Sa = _abs_functional(c, X.shape[0], terms, delta, L)
        assert _err(g, ref, Sa) <= 1e-5, (r, g, ref, Sa)
    ds.close()


@pytest.mark.parametrize("d,M,r", [(1, [80], 8), (3, [16, 14, 12], 6), (3, [16, 14, 12], 2)])
def test_qr_other_dimensions(ctx, d, M, r):
    w = synthetic.small_case(n=2000, d=d, M=M, seed=92 + d, n_candidates=1)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    Sg = w.extra["H_NS"]
    got = ds.qr(Sg, r)[0]
    c = binning.bin_linear(w.X, w.lo, w.hi, M)
    delta = rules.bin_width(w.lo, w.hi, M)
    L = rules.support_L(rules.lambda_max(Sg), delta, M)
    terms = S.eta_r_terms(Sg, r // 2)
    ref = F.binned_direct(c, w.n, terms, delta, L)
    assert _err(got, ref, _abs_functional(c, w.n, terms, delta, L)) <= 1e-5, (got, ref)
    ds.close()


@pytest.mark.parametrize("r", [0, 1, 2, 4])
def test_lscv_r_matches_oracle(ctx, r):
    X, lo, hi, Hns = _normal2(3000, [48, 48], 93)
    M = [48, 48]
    ds = ctx.bin(X, lo, hi, M)
    Hs = [Hns, 0.5 * Hns]
    got = ds.lscv_r(np.stack(Hs), r)
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    for g, H in zip(got, Hs):
        L, P = ds.plan(0, H)
        ev = lambda t: F.binned_direct(c, X.shape[0], t, delta, L)
        ref = S.lscv_r(ev, H, X.shape[0], r)
        terms = [(w, Sg, a) for w, Sg, a in S.eta_r_terms(2.0 * H, r)] + \
                [(-2.0 * w, Sg, a) for w, Sg, a in S.eta_r_terms(H, r)]
        Sa = _abs_functional(c, X.shape[0], terms, delta, L)
        assert _err(g, ref, Sa) <= 1e-5, (r, g, ref, Sa)
    if r == 0:   # LSCV_0 is LSCV (Eq. 10)
        np.testing.assert_allclose(got, ds.lscv(np.stack(Hs)), rtol=1e-6)
    ds.close()


def test_lscv_r_exact_leave_one_out():
    from paper_1511_07482_gb300 import Context
    X, lo, hi, Hns = _normal2(2000, [40, 40], 94)
    M = [40, 40]
    c0 = Context(0)
    ds = c0.bin(X, lo, hi, M, exact_loo=1)
    got = ds.lscv_r(Hns, 1)[0]
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    L, P = ds.plan(0, Hns)
    ref = S.lscv_r(lambda t: F.binned_direct(c, X.shape[0], t, delta, L), Hns, X.shape[0], 1, exact_loo=True)
    terms = [(w, Sg, a) for w, Sg, a in S.eta_r_terms(2.0 * Hns, 1)] + list(S.eta_r_terms(Hns, 1))
    Sa = _abs_functional(c, X.shape[0], terms, delta, L)
    assert _err(got, ref, Sa) <= 1e-5, (got, ref)
    with pytest.raises(Exception):
        ds.lscv_r(Hns, 5)          # order 10 is beyond the tables
    ds.close()
    c0.close()


@pytest.mark.parametrize("d,M,r,s", [(2, [56, 50], 1, 1), (2, [56, 50], 0, 3), (2, [56, 50], 2, 2), (3, [18, 16, 14], 1, 2)])
def test_eta_rs_matches_oracle(ctx, d, M, r, s):
    """Eqs. 29-30 for general (r, s) with full A, B; r = 0, s = 2 agrees with
    the plug-in functional's eta_{0,2} entry point."""
    w = synthetic.small_case(n=3000, d=d, M=M, seed=95 + d, n_candidates=2)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    A, B, Sg = w.H[0], w.H[1], w.extra["H_NS"]
    got = ds.eta_rs(Sg, r, s, A=A, B=B)[0]
    c = binning.bin_linear(w.X, w.lo, w.hi, M)
    delta = rules.bin_width(w.lo, w.hi, M)
    L = rules.support_L(rules.lambda_max(Sg), delta, M)
    terms = S.eta_rs_terms(A, B, Sg, r, s)
    ref = F.binned_direct(c, w.n, terms, delta, L)
    assert _err(got, ref, _abs_functional(c, w.n, terms, delta, L)) <= 1e-5, (got, ref)
    if (r, s) == (0, 3):
        e02 = ds.eta_rs(Sg, 0, 2, B=B)[0]
        assert e02 == pytest.approx(ds.eta02(B, Sg)[0], rel=1e-6)
    ds.close()
