"""The FFT route (Sec. 4 steps 2-4: zero-padded transforms, Eqs. 19-24, and
the Parseval multiply-and-sum) at the full sizes of the benchmark
configurations, forced with ENGINE_FFT (for d = 2 the one-cluster-per-item
fused kernel) and ENGINE_MULTIPASS (the pass-per-axis kernels), against the
FP64 oracle element by element.

Every value is compared with the oracle's lag-first form of Eq. 25 (the
count autocorrelation by an FP64 FFT at twice the grid, then n^-2 sum k_j
a_j over the support box), which equals the paper's FFT steps whenever
P_k >= M_k + L_k (pinned on the CPU in test_oracle_functionals).  Tolerance
1e-5 relative to max(|ref|, S/10), S the magnitude of the summed terms of
that value or gradient entry.  The library's kernel counters confirm that
the transform kernels ran and the lag-domain kernels did not."""
import numpy as np
import pytest

from oracle import binning, functionals as F, gauss, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _err(got, ref, scale):
    return abs(got - ref) / max(abs(ref), 0.1 * scale)


@pytest.fixture(scope="module")
def c2():
    w = synthetic.mixture_2d_large()
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    return w, rules.bin_width(w.lo, w.hi, w.M), F.autocorr_fft(c)


def _kernels_ran(ctx):
    ks, _, _, _ = ctx.profile_read()
    return {k for k, v in ks.items() if v["launches"] > 0 and not k.startswith("host:")}


@pytest.mark.parametrize("engine", ["fft", "multipass"])
@pytest.mark.parametrize("P_rule", ["minimal", "paper"])
def test_c2_lscv_scv_psi4_on_the_fft_route(c2, engine, P_rule):
    """n = 1e5 three-component bivariate mixture on 256^2: LSCV and SCV
    values and gradients at four candidate bandwidths and psi_4 (every
    partial) at two, under both padding rules (the minimal 2^a 3^b 5^c size
    and Eq. 27's power of two)."""
    from paper_1511_07482_gb300 import ENGINE_FFT, ENGINE_MULTIPASS, P_MINIMAL, P_PAPER, Context
    w, delta, a = c2
    ctx = Context(0)
    try:
        ctx.set_engine(ENGINE_FFT if engine == "fft" else ENGINE_MULTIPASS)
        rule = P_MINIMAL if P_rule == "minimal" else P_PAPER
        ds = ctx.bin(w.X, w.lo, w.hi, w.M, P_rule=rule)
        Hs = w.H[:4]
        ctx.profile(1)
        v, g = ds.lscv(Hs, grad=True)
        vs, gs = ds.scv(Hs, w.G, grad=True)
        p4 = ds.psi(Hs[:2], 4)
        ran = _kernels_ran(ctx)
        ctx.profile(0)
        assert "lag_f32" not in ran and "lag_f64" not in ran, ran
        assert ("fused2d_f32" in ran) if engine == "fft" else ({"stage_a_f32", "final_f32"} <= ran), ran
        kal = gauss.kron_alphas(2, 4)
        for i, H in enumerate(Hs):
            for m, (val, grad) in ((0, (v[i], g[i])), (1, (vs[i], gs[i]))):
                L, P = ds.plan(m, H, w.G if m else None)
                B = H if m == 0 else 2 * H + 2 * w.G
                assert L == rules.support_L(rules.lambda_max(B), delta, w.M)
                want_P = rules.P_minimal(w.M, L) if P_rule == "minimal" else rules.P_paper(w.M, L)
                assert P == want_P, (P, want_P)
                ev = lambda t: F.lag_sums(a, w.n, t, delta, L)[0]
                ea = lambda t: F.lag_sums(a, w.n, t, delta, L)[1]
                if m == 0:
                    rv, rg = S.lscv(ev, H, w.n, grad=True)
                    sv, sg = S.abs_scales(ea, "lscv", H, w.n)
                else:
                    rv, rg = S.scv(ev, H, w.G, w.n, grad=True)
                    sv, sg = S.abs_scales(ea, "scv", H, w.n, w.G)
                assert _err(val, rv, sv) <= TOL, (i, m, val, rv)
                for x in range(2):
                    for y in range(2):
                        assert _err(grad[x, y], rg[x, y], sg[x, y]) <= TOL, (i, m, x, y, grad, rg)
            if i < 2:
                L, _ = ds.plan(-1, H)
                for pos, alpha in enumerate(kal):
                    ref, sa = F.lag_sums(a, w.n, [(1.0, H, alpha)], delta, L)
                    assert _err(p4[i, pos], ref, sa) <= TOL, (i, alpha, p4[i, pos], ref)
        ds.close()
    finally:
        ctx.close()


def test_c3_psi4_on_the_multipass_route():
    """n = 1e6 four-component trivariate mixture on 128^3: psi_4 (all 81
    Kronecker entries, 15 distinct partials) at sampled candidate bandwidths
    through the pass-per-axis transform kernels (stage A, the interior pass,
    the final pass with the spectral sum)."""
    from paper_1511_07482_gb300 import ENGINE_FFT, Context
    w = synthetic.mixture_3d()
    ctx = Context(0)
    try:
        ctx.set_engine(ENGINE_FFT)
        ds = ctx.bin(w.X, w.lo, w.hi, w.M)
        idx = [0, 77, 131, 255]
        ctx.profile(1)
        got = ds.psi(w.H[idx], 4)
        ran = _kernels_ran(ctx)
        ctx.profile(0)
        assert {"stage_a_f32", "mid_f32", "final_f32"} <= ran and "lag_f32" not in ran, ran
        c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
        delta = rules.bin_width(w.lo, w.hi, w.M)
        a = F.autocorr_fft(c)
        kal = gauss.kron_alphas(3, 4)
        for k, i in enumerate(idx):
            H = w.H[i]
            L, P = ds.plan(-1, H)
            assert L == rules.support_L(rules.lambda_max(H), delta, w.M)
            assert all(p >= m + l for p, m, l in zip(P, w.M, L))
            for alpha in sorted(set(kal)):
                ref, sa = F.lag_sums(a, w.n, [(1.0, H, alpha)], delta, L)
                pos = kal.index(alpha)
                assert _err(got[k, pos], ref, sa) <= TOL, (i, alpha, got[k, pos], ref)
        ds.close()
    finally:
        ctx.close()
