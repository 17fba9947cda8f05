"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerance (FP32 mode): 1e-5 relative.  A functional whose exact value is
tiny compared with the magnitude of its summed terms (mixed partials of
near-symmetric data, the near-cancelling SCV and eta kernels) cannot be
resolved to that relative accuracy by any FP32 evaluation: the rounding of the
terms and their transform is bounded by about u D S (u = 6e-8, D ~ 20
radix stages), with S = n^-2 sum_i c_i sum_j c_{i-j} |k_j| the absolute
functional.  The relative error is therefore floored at S/10:
  err = |gpu - ref| / max(|ref|, S / 10) <= 1e-5,
i.e. plain relative error up to a cancellation ratio S/|ref| of 10 and
|gpu - ref| <= 1e-6 S beyond it; gradient entries likewise, each with the S
of its own kernel (plus the magnitude of its closed-form term).  FP64 mode:
1e-11 relative.  Integer counts: bit-exact.
"""
import itertools

import numpy as np
import pytest

from oracle import binning, functionals as F, gauss, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["auto", "fft", "multipass"])
def ctx(request):
    """auto: the lag-domain engine wherever the padding has no aliasing;
    fft: the FFT route (fused cluster kernel for d = 2); multipass: the
    pass-per-axis FFT kernels only."""
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, ENGINE_MULTIPASS, Context
    c = Context(0)
    c.set_engine({"auto": ENGINE_AUTO, "fft": ENGINE_FFT, "multipass": ENGINE_MULTIPASS}[request.param])
    yield c
    c.close()


def _abs_functional(c, n, terms, delta, L):
    k = np.abs(F.lag_kernel(terms, delta, L))
    tot = 0.0
    for j in itertools.product(*[range(-l, l + 1) for l in L]):
        tot += k[tuple(jj + l for jj, l in zip(j, L))] * F._overlap(c, j)
    return tot / float(n) ** 2


def _err(got, ref, Sabs):
    """|got - ref| relative to |ref|, floored at S/10: a value more than 10
    times smaller than the magnitude S of its summed terms is held to
    |got - ref| <= 1e-6 S, the FP32 rounding bound u D S of a transform of
    depth D ~ 20 stages (u = 6e-8)."""
    return abs(got - ref) / max(abs(ref), 0.1 * Sabs)


def _grad_ok(g, rg, c, n, delta, L, H, kind, G=None, tol=1e-5):
    """Per-entry gradient check with each entry's own absolute functional."""
    d = H.shape[0]
    Hinv = np.linalg.inv(H)
    for a in range(d):
        for b in range(a, d):
            if kind == "lscv":
                terms = S.lscv_grad_terms(H, a, b)
                extra = abs(2.0 / n * (1 if a == b else 2) * 0.5 * S.K0(H) * Hinv[a, b])
            else:
                terms = S.scv_grad_terms(H, G, a, b)
                extra = abs((1 if a == b else 2) * 0.5 * S.RK(H) * Hinv[a, b] / n)
            Sab = _abs_functional(c, n, terms, delta, L) + extra
            e = _err(g[a, b], rg[a, b], Sab)
            assert e <= tol, (a, b, g[a, b], rg[a, b], Sab, e)


def _case(d, M, n=300, seed=1):
    w = synthetic.small_case(n=n, d=d, M=M, seed=seed)
    return w


# ------------------------------------------------------------------ binning

@pytest.mark.parametrize("d,M", [(1, [37]), (2, [23, 17]), (3, [9, 11, 7]), (4, [5, 6, 4, 7])])
def test_simple_binning_bit_exact(ctx, d, M):
    from paper_1511_07482_gb300 import BIN_SIMPLE, DT_I32
    w = _case(d, M, n=2000, seed=d)
    X = w.X.copy()
    # points on the upper corner, the lower corner and at exact half-bin ties
    X[0] = w.hi
    X[1] = w.lo
    delta = rules.bin_width(w.lo, w.hi, M)
    X[2] = w.lo + 1.5 * delta
    ds = ctx.bin(X, w.lo, w.hi, M, binning=BIN_SIMPLE)
    got = ds.counts(DT_I32)
    want = binning.bin_simple(X, w.lo, w.hi, M)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("M", [[40, 40], [300, 280]])
def test_linear_binning_is_deterministic(ctx, M):
    """FP32 counts are accumulated in fixed point: two binnings of the same
    sample (shared-memory histogram for 40 x 40, global atomics for
    300 x 280) give the same bits, and so do the objective values and the
    selected bandwidth computed from them."""
    from paper_1511_07482_gb300 import LSCV
    w = _case(2, M, n=200000, seed=33)
    a = ctx.bin(w.X, w.lo, w.hi, M)
    b = ctx.bin(w.X, w.lo, w.hi, M)
    assert np.array_equal(a.counts(), b.counts())
    assert np.array_equal(a.lscv(w.H, grad=True)[1], b.lscv(w.H, grad=True)[1])
    a.close()
    b.close()
    if M[0] <= 64:
        # the search from two binnings of a smaller sample (its bandwidths
        # span several bins of this grid)
        v = _case(2, M, n=5000, seed=34)
        a = ctx.bin(v.X, v.lo, v.hi, M)
        b = ctx.bin(v.X, v.lo, v.hi, M)
        Ha, fa, _ = a.select_H(LSCV, n_starts=4)
        Hb, fb, _ = b.select_H(LSCV, n_starts=4)
        assert fa == fb and np.array_equal(Ha, Hb)
        a.close()
        b.close()


@pytest.mark.parametrize("d,M", [(1, [64]), (2, [100, 100]), (2, [300, 280]), (3, [20, 18, 16])])
def test_linear_binning(ctx, d, M):
    w = _case(d, M, n=5000, seed=10 + d)
    X = w.X.copy()
    X[0] = w.hi
    ds = ctx.bin(X, w.lo, w.hi, M)
    got = ds.counts()
    want = binning.bin_linear(X, w.lo, w.hi, M)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6)
    assert got.sum() == pytest.approx(5000, rel=1e-6)


def test_upper_edge_rounding(ctx):
    from paper_1511_07482_gb300 import BIN_SIMPLE, DT_I32
    lo, hi, M = -0.920732229392339, 0.11341865083372567, 120
    X = np.array([[hi], [lo], [0.5 * (lo + hi)]])
    got = ctx.bin(X, [lo], [hi], [M]).counts()
    np.testing.assert_allclose(got, binning.bin_linear(X, [lo], [hi], [M]), atol=1e-7)
    gi = ctx.bin(X, [lo], [hi], [M], binning=BIN_SIMPLE).counts(DT_I32)
    assert np.array_equal(gi, binning.bin_simple(X, [lo], [hi], [M]))


def test_outside_points(ctx):
    from paper_1511_07482_gb300 import KdefftError, OUTSIDE_DROP
    w = _case(2, [20, 20])
    X = np.vstack([w.X, [[w.hi[0] + 1.0, 0.0]]])
    with pytest.raises(KdefftError):
        ctx.bin(X, w.lo, w.hi, w.M)
    ds = ctx.bin(X, w.lo, w.hi, w.M, outside_policy=OUTSIDE_DROP)
    n, d, dropped = ds.info()
    assert (n, d, dropped) == (w.n + 1, 2, 1)


# ------------------------------------------------------------------ functionals

def _oracle_setup(w, ds, method, H, G=None):
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    L, P = ds.plan(method, H, G)
    return c, delta, L, P


@pytest.mark.parametrize("d,M,r", [(1, [60], 0), (1, [60], 4), (2, [40, 36], 0), (2, [40, 36], 2),
                                   (2, [40, 36], 4), (3, [14, 12, 16], 2), (3, [14, 12, 16], 4),
                                   (4, [8, 9, 7, 8], 2)])
def test_psi_r(ctx, d, M, r):
    w = _case(d, M, n=400, seed=20 + d)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    H = w.H[0]
    got = ds.psi(H, r)[0]
    c, delta, L, P = _oracle_setup(w, ds, -1, H)
    assert L == rules.support_L(rules.lambda_max(H), delta, M)
    assert P == rules.P_minimal(M, L)
    for pos, alpha in enumerate(gauss.kron_alphas(d, r)):
        terms = [(1.0, H, alpha)]
        ref = F.binned_direct(c, w.n, terms, delta, L)
        Sa = _abs_functional(c, w.n, terms, delta, L)
        assert _err(got[pos], ref, Sa) <= 1e-5, (alpha, got[pos], ref, Sa)


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("d,M", [(1, [50]), (2, [48, 44]), (3, [15, 14, 13])])
def test_lscv_value_and_gradient(ctx, d, M, exact):
    w = _case(d, M, n=500, seed=30 + d)
    ds = ctx.bin(w.X, w.lo, w.hi, M, exact_loo=int(exact))
    Hs = w.H
    val, g = ds.lscv(Hs, grad=True)
    for i, H in enumerate(Hs):
        c, delta, L, P = _oracle_setup(w, ds, 0, H)
        assert L == rules.support_L(rules.lambda_max(H), delta, M)
        ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
        rv, rg = S.lscv(ev, H, w.n, exact_loo=exact, grad=True)
        assert abs(val[i] - rv) <= 1e-5 * abs(rv), (val[i], rv)
        if not exact:
            _grad_ok(g[i], rg, c, w.n, delta, L, H, "lscv")
        else:
            assert np.max(np.abs(g[i] - rg)) <= 1e-5 * np.max(np.abs(rg)), (g[i], rg)


def test_lscv_fp64_mode(ctx):
    from paper_1511_07482_gb300 import FP64
    w = _case(2, [40, 40], n=500, seed=41)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M, precision=FP64)
    val, g = ds.lscv(w.H, grad=True)
    for i, H in enumerate(w.H):
        c, delta, L, P = _oracle_setup(w, ds, 0, H)
        ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
        rv, rg = S.lscv(ev, H, w.n, grad=True)
        assert abs(val[i] - rv) <= 1e-11 * abs(rv), (val[i], rv)
        assert np.max(np.abs(g[i] - rg)) <= 1e-11 * np.max(np.abs(rg))


@pytest.mark.parametrize("d,M", [(2, [40, 38]), (3, [14, 13, 12])])
def test_scv_value_and_gradient(ctx, d, M):
    w = _case(d, M, n=400, seed=50 + d)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    G = w.G
    val, g = ds.scv(w.H, G, grad=True)
    for i, H in enumerate(w.H):
        c, delta, L, P = _oracle_setup(w, ds, 1, H, G)
        assert L == rules.support_L(rules.lambda_max(2 * H + 2 * G), delta, M)
        ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
        rv, rg = S.scv(ev, H, G, w.n, grad=True)
        Sa = _abs_functional(c, w.n, S.scv_terms(H, G), delta, L)
        assert _err(val[i], rv, Sa) <= 1e-5, (val[i], rv)
        _grad_ok(g[i], rg, c, w.n, delta, L, H, "scv", G=G)


@pytest.mark.parametrize("d,M", [(2, [40, 38]), (3, [14, 13, 12])])
def test_pi_and_eta02(ctx, d, M):
    w = _case(d, M, n=400, seed=60 + d)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    G = w.G
    val, g = ds.pi(w.H, G, grad=True)
    eta = ds.eta02(w.H, G)
    c, delta, L, P = _oracle_setup(w, ds, 2, w.H[0], G)
    ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
    psi4 = S.psi_vector(ev, G, 4)
    for i, H in enumerate(w.H):
        rv, rg = S.pi_from_psi4(psi4, H, w.n, grad=True)
        assert abs(val[i] - rv) <= 1e-5 * abs(rv), (val[i], rv)
        assert np.max(np.abs(g[i] - rg)) <= 1e-5 * np.max(np.abs(rg))
        re = ev(S.eta02_terms(H, G))
        Sa = _abs_functional(c, w.n, S.eta02_terms(H, G), delta, L)
        assert _err(eta[i], re, Sa) <= 1e-5, (eta[i], re)


@pytest.mark.parametrize("rule,basis", [("paper", "auto"), ("paper_full", "full"), ("fixed", "auto")])
def test_padding_rules_and_full_support(ctx, rule, basis):
    from paper_1511_07482_gb300 import L_AUTO, L_FULL, P_FIXED, P_PAPER, P_PAPER_FULL
    w = _case(2, [30, 26], n=300, seed=70)
    kw = {"P_rule": {"paper": P_PAPER, "paper_full": P_PAPER_FULL, "fixed": P_FIXED}[rule],
          "L_basis": {"auto": L_AUTO, "full": L_FULL}[basis]}
    if rule == "fixed":
        kw["P_fixed"] = [90, 75]
    ds = ctx.bin(w.X, w.lo, w.hi, w.M, **kw)
    H = w.H[0]
    val = ds.lscv(H)[0]
    c, delta, L, P = _oracle_setup(w, ds, 0, H)
    if basis == "full":
        assert L == [29, 25]
    if rule == "paper":
        assert P == rules.P_paper(w.M, L)
    if rule == "paper_full":
        assert P == rules.P_paper_full(w.M)
    if rule == "fixed":
        assert P == [90, 75]
    ev = lambda t: F.binned_fft(c, w.n, t, delta, L, P)
    assert abs(val - S.lscv(ev, H, w.n)) <= 1e-5 * abs(S.lscv(ev, H, w.n))


def test_plain_config_psi4_and_lscv(ctx):
    """The plain 2-D configuration: n = 1000, 100 x 100 grid, fixed H."""
    w = synthetic.plain_mixture_2d()
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    H = w.H[0]
    psi4 = ds.psi(H, 4)[0]
    val = ds.lscv(H)[0]
    c, delta, L, P = _oracle_setup(w, ds, 0, H)
    assert L == rules.support_L(rules.lambda_max(H), delta, w.M)
    ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
    assert abs(val - S.lscv(ev, H, w.n)) <= 1e-5 * abs(S.lscv(ev, H, w.n))
    for pos, alpha in enumerate(gauss.kron_alphas(2, 4)):
        t = [(1.0, H, alpha)]
        ref = ev(t)
        assert _err(psi4[pos], ref, _abs_functional(c, w.n, t, delta, L)) <= 1e-5


def test_batch_matches_single(ctx):
    ws = synthetic.batched_uneven(n_datasets=5, n_candidates=3, n_range=(300, 3000))
    dss = [ctx.bin(w.X, w.lo, w.hi, w.M) for w in ws]
    val, g = ctx.batch_lscv(dss, [w.H for w in ws])
    k = 0
    for w, ds in zip(ws, dss):
        v1, g1 = ds.lscv(w.H, grad=True)
        np.testing.assert_allclose(val[k:k + len(w.H)], v1, rtol=1e-12)
        np.testing.assert_allclose(g[k:k + len(w.H)], g1, rtol=1e-12, atol=1e-300)
        k += len(w.H)


def _gauss_case(n=3000, seed=81):
    """A correlated bivariate Gaussian sample: its LSCV and SCV have one minimum."""
    rng = np.random.default_rng(seed)
    X = rng.multivariate_normal([0.0, 1.0], [[1.0, 0.5], [0.5, 2.0]], size=n)
    Hns = synthetic.normal_scale(X)
    lo, hi = synthetic.grid_range(X, Hns)
    return X, lo, hi, Hns


@pytest.mark.parametrize("method", ["lscv", "scv"])
def test_nelder_mead_parity_mode(ctx, method):
    """The paper's derivative-free search (Sec. 6: reflection 1, contraction
    0.5, expansion 2) on a Gaussian sample: the value returned is the
    objective at the H returned, the evaluation budget per start is kept, the
    end point is at least as good as the gradient search's from the same
    starts (the support L_k steps with H, Eq. 26, so the binned objective is
    piecewise smooth and a line search can stop at a step; the simplex does
    not), and a gradient search started there improves it by less than the
    FP32 value tolerance: a numerical minimum."""
    from paper_1511_07482_gb300 import LSCV, SCV
    X, lo, hi, Hns = _gauss_case()
    ds = ctx.bin(X, lo, hi, [80, 72])
    m = LSCV if method == "lscv" else SCV
    Hb, fb, _ = ds.select_H(m, G=Hns, n_starts=4, max_iter=100)
    Hn, fn, ne = ds.select_H(m, G=Hns, n_starts=4, max_iter=400, optimizer="nelder-mead")
    assert ne <= 4 * (400 + 3)
    v = ds.scv(Hn, Hns)[0] if m == SCV else ds.lscv(Hn)[0]
    assert v == pytest.approx(fn, rel=1e-6)
    assert fn <= fb + 1e-5 * abs(fb)
    assert fn == pytest.approx(fb, rel=5e-3)
    Hp, fp, _ = ds.select_H(m, H0=Hn, G=Hns, n_starts=1, max_iter=100)
    assert fp >= fn - 1e-5 * abs(fn)
    with pytest.raises(ValueError):
        ds.select_H(m, G=Hns, optimizer="simplex")
    ds.close()


@pytest.mark.parametrize("method", ["lscv", "scv"])
def test_device_resident_selection_matches_host_driven(method):
    """The device-resident search (one cluster per start) and the
    host-driven one (one batched launch per round) run the same algorithm on
    the same counts.  On a Gaussian sample, whose objective has one minimum,
    every start ends at the same point, so both return the same minimum.  On
    a mixture with several basins FP32 rounding may send a start into
    another basin, so there each engine is held to its own objective: the
    value it returns is the objective at the H it returns."""
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_HOST_SELECT, LSCV, SCV, Context
    X, lo, hi, Hns = _gauss_case()
    mix = _case(2, [80, 72], n=3000, seed=81)
    m = LSCV if method == "lscv" else SCV
    res = {}
    for eng in (ENGINE_AUTO, ENGINE_HOST_SELECT):
        c = Context(0)
        c.set_engine(eng)
        for name, (Xs, l, h, G) in {"gauss": (X, lo, hi, Hns), "mix": (mix.X, mix.lo, mix.hi, mix.G)}.items():
            ds = c.bin(Xs, l, h, [80, 72])
            H, f, ne = ds.select_H(m, G=G, n_starts=8, max_iter=60)
            v = ds.scv(H, G)[0] if m == SCV else ds.lscv(H)[0]
            assert v == pytest.approx(f, rel=1e-6), (name, eng)
            assert ne >= 8
            res[eng, name] = (H, f)
        c.close()
    fa, fh = res[ENGINE_AUTO, "gauss"][1], res[ENGINE_HOST_SELECT, "gauss"][1]
    # SCV iterates on its FP32 kernel, whose cancellation noise (the FP32
    # value tolerance, 1e-5) moves the end point on a flat minimum
    assert fa == pytest.approx(fh, rel=1e-6 if m == LSCV else 1e-5)
    np.testing.assert_allclose(res[ENGINE_AUTO, "gauss"][0], res[ENGINE_HOST_SELECT, "gauss"][0], rtol=2e-2)


def test_select_H_reaches_a_stationary_point(ctx):
    from paper_1511_07482_gb300 import LSCV
    w = _case(2, [60, 60], n=800, seed=80)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    H, f, ne = ds.select_H(LSCV, n_starts=4)
    assert ne > 4
    v, g = ds.lscv(H, grad=True)
    assert v[0] == pytest.approx(f, rel=1e-12)
    # parity of the objective at the returned H
    c, delta, L, P = _oracle_setup(w, ds, 0, H)
    ev = lambda t: F.binned_direct(c, w.n, t, delta, L)
    rv, rg = S.lscv(ev, H, w.n, grad=True)
    assert abs(v[0] - rv) <= 1e-5 * abs(rv)
    # not worse than the normal-scale start
    v0 = ds.lscv(synthetic.normal_scale(w.X))[0]
    assert f <= v0 + 1e-12
