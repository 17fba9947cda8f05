"""The device-resident search's own evaluations against the oracle.

The minimiser of Eq. 9 (LSCV of Eq. 10 and SCV) runs on the device with
FP32 kernel values, FP32 per-thread and per-warp sums and FP32 bandwidth
algebra; it compares those values to choose its steps.  Here every
evaluation of a few starts at the benchmark configuration (n = 1e5
three-component bivariate mixture, 256^2 grid) is recorded by the search
kernel itself (value, the three gradient entries, the FP32 bandwidth and
the support it used) and recomputed by the FP64 oracle at that bandwidth
and support, element by element.  Tolerance: 1e-5 relative, normalised as
in every FP32 test (relative to max(|ref|, S/10), S the magnitude of the
summed terms of that value or gradient entry).  The support L the search
computed in FP32 must equal Eq. 26 in FP64 except where tau sqrt(lambda) /
delta_k lies within FP32 rounding of an integer."""
import math

import numpy as np
import pytest

from oracle import binning, functionals as F, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu

FIELDS = 12
TOL = 1e-5


def _oracle_errors(rec, c, n, delta, M, G, L_basis_widest=False):
    """Max errors of the recorded evaluations: (value, gradient, mismatched
    supports, rows) per criterion."""
    a = F.autocorr_fft(c)
    out = {0: [0.0, 0.0, 0, 0], 1: [0.0, 0.0, 0, 0]}
    for r in rec:
        method = int(r[2])
        H = np.array([[r[3], r[4]], [r[4], r[5]]])
        L = [int(r[6]), int(r[7])]
        ev = lambda t: F.lag_sums(a, n, t, delta, L)[0]
        ev_abs = lambda t: F.lag_sums(a, n, t, delta, L)[1]
        if method == 0:
            val, g = S.lscv(ev, H, n, grad=True)
            sv, sg = S.abs_scales(ev_abs, "lscv", H, n)
            B = 2.0 * H if L_basis_widest else H
        else:
            val, g = S.scv(ev, H, G, n, grad=True)
            sv, sg = S.abs_scales(ev_abs, "scv", H, n, G)
            B = 2.0 * H + 2.0 * G
        o = out[method]
        o[0] = max(o[0], abs(r[8] - val) / max(abs(val), 0.1 * sv))
        got_g = np.array([[r[9], r[10]], [r[10], r[11]]])
        o[1] = max(o[1], float(np.max(np.abs(got_g - g) / np.maximum(np.abs(g), 0.1 * sg))))
        want_L = rules.support_L(rules.lambda_max(B), delta, M)
        for k in range(2):
            if L[k] != max(1, want_L[k]):
                v = 3.7 * math.sqrt(rules.lambda_max(B)) / delta[k]
                if abs(v - round(v)) > 1e-5 * v:
                    o[2] += 1
        o[3] += 1
    return out


@pytest.mark.parametrize("engine", ["lag", "fft"])
def test_search_evaluations_match_oracle_at_benchmark_size(engine):
    import torch
    from paper_1511_07482_gb300 import LSCV, SCV, Context, ENGINE_FFT
    w = synthetic.mixture_2d_large()
    ctx = Context(0)
    try:
        if engine == "fft":
            ctx.set_engine(ENGINE_FFT)
        ds = ctx.bin(w.X, w.lo, w.hi, w.M)
        n_starts, cap = 3, 400

        def recorded(run, nst):
            rec = torch.full((nst * cap * FIELDS,), float("nan"), dtype=torch.float64, device="cuda:0")
            ctx.set_search_record(rec, cap)
            evals = run()
            ctx.set_search_record(None)
            R = rec.view(-1, FIELDS).cpu().numpy()
            R = R[np.isfinite(R[:, 0])]
            # every evaluation of every start is recorded (cap is above any
            # start's count); the reported count adds the end point's value
            assert len(R) == evals, (len(R), evals)
            return R

        if engine == "lag":   # both criteria in one launch, as the benchmark runs them
            R = recorded(lambda: sum(r[2] - 1 for r in ds.select_H_many([LSCV, SCV], G=w.G, n_starts=n_starts,
                                                                         max_iter=60)), 2 * n_starts)
        else:                 # the cluster FFT-route search, one criterion per launch
            R = np.concatenate([recorded(lambda m=m: ds.select_H(m, G=w.G, n_starts=n_starts, max_iter=60)[2] - 1,
                                         n_starts) for m in (LSCV, SCV)])
        assert set(R[:, 2].astype(int)) == {0, 1}
        c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
        delta = rules.bin_width(w.lo, w.hi, w.M)
        errs = _oracle_errors(R, c, w.n, delta, w.M, w.G)
        for m in (0, 1):
            ev, eg, bad_L, rows = errs[m]
            assert rows > 0
            assert bad_L == 0, (m, bad_L)
            assert ev <= TOL, (m, ev)
            assert eg <= TOL, (m, eg)
        ds.close()
    finally:
        ctx.close()


def test_search_record_rejects_small_or_host_buffers():
    import torch
    from paper_1511_07482_gb300 import Context, KdefftError, LSCV
    ctx = Context(0)
    try:
        small = torch.zeros(FIELDS * 3, dtype=torch.float64, device="cuda:0")
        with pytest.raises(KdefftError):
            ctx.set_search_record(small, 4)          # fewer than cap x 12 values
        host = torch.zeros(FIELDS * 8, dtype=torch.float64)
        with pytest.raises(TypeError):
            ctx.set_search_record(host, 4)
        # a search with more starts than the buffer holds fails before its launch
        w = synthetic.plain_mixture_2d(n=400, M=48)
        ds = ctx.bin(w.X, w.lo, w.hi, w.M)
        ctx.set_search_record(small, 1)              # room for 3 starts
        with pytest.raises(KdefftError):
            ds.select_H(LSCV, n_starts=4, max_iter=20)
        ctx.set_search_record(None)
        H, f, ne = ds.select_H(LSCV, n_starts=4, max_iter=20)
        assert np.isfinite(f)
        ds.close()
    finally:
        ctx.close()


@pytest.mark.parametrize("seed", [4, 5])
def test_search_evaluations_match_oracle_on_other_datasets(seed):
    """All 16 starts of both criteria, as the benchmark runs them, on two more
    draws of the benchmark's three-component mixture (other means and
    covariances): every recorded evaluation within the FP32 tolerance."""
    import torch
    from paper_1511_07482_gb300 import LSCV, SCV, Context
    w = synthetic.mixture_2d_large(seed=seed)
    ctx = Context(0)
    try:
        ds = ctx.bin(w.X, w.lo, w.hi, w.M)
        n_starts, cap = 16, 400
        rec = torch.full((2 * n_starts * cap * FIELDS,), float("nan"), dtype=torch.float64, device="cuda:0")
        ctx.set_search_record(rec, cap)
        res = ds.select_H_many([LSCV, SCV], G=w.G, n_starts=n_starts, max_iter=60)
        ctx.set_search_record(None)
        R = rec.view(-1, FIELDS).cpu().numpy()
        R = R[np.isfinite(R[:, 0])]
        assert len(R) == sum(r[2] - 1 for r in res)
        c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
        delta = rules.bin_width(w.lo, w.hi, w.M)
        errs = _oracle_errors(R, c, w.n, delta, w.M, w.G)
        for m in (0, 1):
            ev, eg, bad_L, rows = errs[m]
            assert rows > 0 and bad_L == 0, (m, rows, bad_L)
            assert ev <= TOL and eg <= TOL, (m, ev, eg)
        ds.close()
    finally:
        ctx.close()


def test_search_values_on_a_box_past_the_fast_quotient():
    """Lag boxes where a multiply-high quotient by L_0 + 1 is not exact: a
    1103 x 2048 grid whose support is the whole grid at every trial point
    (a pilot G wider than the grid), so each evaluation sums 1103 x 4095
    half-box points and index x 1103 reaches 2^32.  The search kernel takes
    its plain-division branch there; the values of the first recorded
    evaluations of two SCV starts against the oracle."""
    import torch
    from paper_1511_07482_gb300 import SCV, Context
    rng = np.random.default_rng(501)
    X = synthetic.random_mixture(rng, 40, 2, 2)
    lo, hi, M = X.min(0), X.max(0), [1103, 2048]
    G = (float(np.max(hi - lo)) / 3.7) ** 2 * np.eye(2)
    delta = rules.bin_width(lo, hi, M)
    ctx = Context(0)
    try:
        ds = ctx.bin(X, lo, hi, M)
        n_starts, cap = 2, 2
        rec = torch.full((n_starts * cap * FIELDS,), float("nan"), dtype=torch.float64, device="cuda:0")
        ctx.set_search_record(rec, cap)
        H, f, ne = ds.select_H(SCV, G=G, n_starts=n_starts, max_iter=20)
        ctx.set_search_record(None)
        assert np.isfinite(f) and ne > 1
        R = rec.view(-1, FIELDS).cpu().numpy()
        R = R[np.isfinite(R[:, 0])]
        assert len(R) >= 2
        a = F.autocorr_fft(binning.bin_linear(X, lo, hi, M))
        for r in R:
            L = [int(r[6]), int(r[7])]
            assert L == [M[0] - 1, M[1] - 1]
            n0, total = L[0] + 1, (L[0] + 1) * (2 * L[1] + 1)
            assert total * n0 >= 2 ** 32   # past the multiply-high quotient's exactness bound
            Hr = np.array([[r[3], r[4]], [r[4], r[5]]])
            sums = F.lag_sums(a, len(X), S.scv_terms(Hr, G), delta, L)   # (value, magnitude) of the double sum
            ref = S.scv(lambda t: sums[0], Hr, G, len(X))
            sv = sums[1] + S.RK(Hr) / len(X)   # the value's scale, as abs_scales defines it
            assert abs(r[8] - ref) / max(abs(ref), 0.1 * sv) <= TOL, (r[8], ref, sv)
        ds.close()
    finally:
        ctx.close()
