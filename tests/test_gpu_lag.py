"""The lag-domain engine: the count autocorrelation against the oracle's
direct sums, its use by the default engine, and the engine's values against
the FFT route and the oracle on the paper's workload shapes (the parity
tests of test_gpu_parity run every functional through it as well)."""
import numpy as np
import pytest

from oracle import binning, functionals as F, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1511_07482_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("d,M,A", [(1, [90], [40]), (2, [40, 36], [12, 9]), (3, [14, 12, 10], [5, 4, 6])])
def test_autocorrelation_matches_oracle(ctx, d, M, A):
    """The autocorrelation of the counts against the oracle's direct lag sums
    over its own binning of the sample.  Simple binning gives the same
    integer counts on both sides and FP64 datasets the same counts to
    rounding, so there the transform is held to 1e-12 a_0.  FP32
    linear-binned counts are the library's fixed-point sums of FP32 corner
    weights rounded to FP32, within 3u |c| of the oracle's (u = 2^-24), so
    their autocorrelation is within 6u a_0 (Cauchy-Schwarz bounds every
    |a_j| by a_0)."""
    from paper_1511_07482_gb300 import BIN_LINEAR, BIN_SIMPLE, FP32, FP64
    w = synthetic.small_case(n=2500, d=d, M=M, seed=50 + d)
    for prec in (FP32, FP64):
        for rule in (BIN_LINEAR, BIN_SIMPLE):
            ds = ctx.bin(w.X, w.lo, w.hi, M, precision=prec, binning=rule)
            c = (binning.bin_simple if rule == BIN_SIMPLE else binning.bin_linear)(w.X, w.lo, w.hi, M)
            got = ds.autocorr(A)
            want = F.autocorr(c, A)
            a0 = float(np.sum(c * c))
            assert got.shape == want.shape
            tol = 6.0 * 2.0 ** -24 + 1e-12 if (prec == FP32 and rule == BIN_LINEAR) else 1e-12
            assert np.max(np.abs(got - want)) <= tol * a0, (prec, rule)
            if rule == BIN_SIMPLE:   # integer counts: integer autocorrelation
                assert np.max(np.abs(got - np.round(want))) <= 1e-9 * a0
            ds.close()
    for kw in ({}, {"binning": BIN_SIMPLE}):
        ds = ctx.bin(w.X, w.lo, w.hi, M, **kw)
        # a larger box later (the cached box grows) and a smaller one agree
        big = [min(m - 1, 2 * a) for m, a in zip(M, A)]
        gb = ds.autocorr(big)
        sl = tuple(slice(big[k] - A[k], big[k] + A[k] + 1) for k in range(d - 1, 0, -1)) + (slice(0, A[0] + 1),)
        np.testing.assert_array_equal(gb[sl], ds.autocorr(A))
        ds.close()


def test_default_engine_uses_the_lag_domain(ctx):
    w = synthetic.small_case(n=3000, d=2, M=[64, 60], seed=52, n_candidates=3)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    ctx.profile(1)
    v, g = ds.lscv(w.H, grad=True)
    stats, _, _, _ = ctx.profile_read()
    ctx.profile(0)
    assert "lag_f32" in stats and not any(k.startswith("fused2d") or k.startswith("final") for k in stats
                                         if not k.startswith("final_f64"))
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    for i, H in enumerate(w.H):
        L, P = ds.plan(0, H)
        rv, rg = S.lscv(lambda t: F.binned_direct(c, w.n, t, delta, L), H, w.n, grad=True)
        assert abs(v[i] - rv) <= 1e-5 * abs(rv)
        assert np.max(np.abs(g[i] - rg)) <= 1e-5 * np.max(np.abs(rg))
    ds.close()


@pytest.mark.parametrize("d,M,r", [(2, [72, 64], 4), (3, [24, 20, 22], 4), (4, [10, 9, 8, 9], 2)])
def test_lag_and_fft_engines_agree(d, M, r):
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, Context
    w = synthetic.small_case(n=4000, d=d, M=M, seed=53 + d, n_candidates=4)
    out = {}
    for eng in (ENGINE_AUTO, ENGINE_FFT):
        c = Context(0)
        c.set_engine(eng)
        ds = c.bin(w.X, w.lo, w.hi, M)
        out[eng] = (ds.psi(w.H, r), ds.lscv(w.H, grad=True), ds.scv(w.H, w.G, grad=True))
        ds.close()
        c.close()
    a, b = out[ENGINE_AUTO], out[ENGINE_FFT]
    assert np.max(np.abs(a[0] - b[0])) <= 2e-5 * np.max(np.abs(b[0]))
    for (va, ga), (vb, gb) in ((a[1], b[1]), (a[2], b[2])):
        np.testing.assert_allclose(va, vb, rtol=2e-5)
        assert np.max(np.abs(ga - gb)) <= 2e-5 * np.max(np.abs(gb))
