"""Selection over the constrained bandwidth classes of Sec. 3 (D: diagonal,
S: scalar h^2 I) on a correlated Gaussian sample: the result lies in its
class, the value returned at every class's end point is the oracle's value
there, no neighbouring class member is lower (SCV), and the classes nest (a
search over F started at the D end point, or over D started at the S end
point, never ends higher).  Also the paper's case against Wand's reshaping
(Sec. 2): on the plain mixture's data and grid, the GPU LSCV for correlated
bandwidths matches the correctly laid out binned sum, while the mirrored
layout k_{|j_1|,|j_2|} departs from it."""
import itertools

import numpy as np
import pytest

from oracle import binning, functionals as F, rules, selectors as S
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1511_07482_gb300 import Context
    rng = np.random.default_rng(71)
    X = rng.multivariate_normal([0.0, 0.0], [[1.0, 0.6], [0.6, 1.5]], size=4000)
    Hns = synthetic.normal_scale(X)
    lo, hi = synthetic.grid_range(X, Hns)
    c = Context(0)
    ds = c.bin(X, lo, hi, [80, 80])
    ds.oracle_case = (X, lo, hi, [80, 80])
    yield ds, Hns
    ds.close()
    c.close()


def _oracle_value(ds, H, G, method):
    """The objective at H by the FP64 oracle (its own binning, the support of
    Eq. 26, minimal padding) and the magnitude of its summed terms."""
    X, lo, hi, M = ds.oracle_case
    c = binning.bin_linear(X, lo, hi, M)
    delta = rules.bin_width(lo, hi, M)
    B = H if method == "lscv" else 2 * H + 2 * G
    L = [max(1, v) for v in rules.support_L(rules.lambda_max(B), delta, M)]
    a = F.autocorr_fft(c)
    ev = lambda t: F.lag_sums(a, X.shape[0], t, delta, L)[0]
    ea = lambda t: F.lag_sums(a, X.shape[0], t, delta, L)[1]
    if method == "lscv":
        return S.lscv(ev, H, X.shape[0]), S.abs_scales(ea, "lscv", H, X.shape[0])[0]
    return S.scv(ev, H, G, X.shape[0]), S.abs_scales(ea, "scv", H, X.shape[0], G)[0]


@pytest.mark.parametrize("method", ["lscv", "scv"])
def test_classes_nest_and_stay_in_class(setup, method):
    from paper_1511_07482_gb300 import LSCV, SCV
    ds, Hns = setup
    m = LSCV if method == "lscv" else SCV
    obj = (lambda H: ds.lscv(H)[0]) if m == LSCV else (lambda H: ds.scv(H, Hns)[0])
    res = {}
    for cls in ("full", "diag", "scalar"):
        H, f, ne = ds.select_H(m, G=Hns, n_starts=4, hclass=cls)
        assert f == pytest.approx(obj(H), rel=1e-6)
        ref, scale = _oracle_value(ds, H, Hns, method)
        assert abs(f - ref) <= 1e-5 * max(abs(ref), 0.1 * scale), (cls, f, ref)
        res[cls] = (H, f)
    Hd, fd = res["diag"]
    Hs, fs = res["scalar"]
    assert Hd[0, 1] == 0.0 and Hd[1, 0] == 0.0
    assert Hs[0, 1] == 0.0 and Hs[0, 0] == pytest.approx(Hs[1, 1], rel=1e-12)
    tol = 1e-5
    # nesting, in the form every descent method keeps: a search over the
    # larger class started at the smaller class's end point ends no higher
    _, fFd, _ = ds.select_H(m, H0=Hd, G=Hns, n_starts=1, hclass="full")
    _, fDs, _ = ds.select_H(m, H0=Hs, G=Hns, n_starts=1, hclass="diag")
    assert fFd <= fd + tol * abs(fd)
    assert fDs <= fs + tol * abs(fs)
    if m == SCV:
        # a minimum within D and S: scaling a diagonal entry by 0.9 / 1.1
        # does not go lower.  (Not asked of LSCV: under the paper's support
        # rule, L from lambda_max(H) (Eq. 26), phi_2H is cut at 2.6 of its
        # standard deviations, so the binned LSCV jumps where L_k steps and a
        # descent method can stop on the low side of a jump -- the
        # optimisation failures of binned LSCV that Sec. 6.1 reports.  SCV's
        # support comes from its widest covariance.)
        for k in range(2):
            for sc in (0.9, 1.1):
                Hp = Hd.copy()
                Hp[k, k] *= sc
                assert obj(Hp) >= fd - tol * abs(fd)
        for sc in (0.9, 1.1):
            assert obj(Hs * sc) >= fs - tol * abs(fs)


def test_class_search_with_nelder_mead_and_bad_class(setup):
    from paper_1511_07482_gb300 import LSCV
    ds, Hns = setup
    Hn, fn, _ = ds.select_H(LSCV, n_starts=2, hclass="diag", optimizer="nelder-mead", max_iter=300)
    assert Hn[0, 1] == 0.0
    # a numerical minimum within D: the gradient search from there gains less than the FP32 tolerance
    _, fq, _ = ds.select_H(LSCV, H0=Hn, n_starts=1, hclass="diag")
    assert fq >= fn - 1e-5 * abs(fn)
    with pytest.raises(ValueError):
        ds.select_H(LSCV, hclass="banded")


def test_wand_mirrored_layout_departs_for_correlated_bandwidths():
    """The plain mixture (n = 1000, 100 x 100 grid, data range +/- 3
    bandwidths) at H = [[0.10, 0.05], [0.05, 0.20]] with its correlation
    scaled: the GPU LSCV equals the binned double sum of Eq. 25 laid out over
    signed lags, and Wand's mirrored layout (kernel values at |j_1|, |j_2|
    only, Sec. 2) agrees with it for a diagonal H but not once H_12 != 0."""
    from paper_1511_07482_gb300 import Context
    w = synthetic.plain_mixture_2d()
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    H0 = np.array([[0.10, 0.05], [0.05, 0.20]])
    ctx = Context(0)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    dep = {}
    try:
        for rho_scale in (0.0, 0.5, 1.0, 1.5):
            H = H0.copy()
            H[0, 1] = H[1, 0] = H0[0, 1] * rho_scale
            L = rules.support_L(rules.lambda_max(H), delta, w.M)
            k = F.lag_kernel(S.lscv_T_terms(H), delta, L)
            right = mirrored = 0.0
            for j in itertools.product(range(-L[0], L[0] + 1), range(-L[1], L[1] + 1)):
                ov = F._overlap(c, j)
                right += k[j[0] + L[0], j[1] + L[1]] * ov
                mirrored += k[abs(j[0]) + L[0], abs(j[1]) + L[1]] * ov
            tail = 2.0 * S.K0(H) / w.n
            right, mirrored = right / w.n ** 2 + tail, mirrored / w.n ** 2 + tail
            got = ds.lscv(H)[0]
            assert abs(got - right) <= 1e-5 * abs(right), (rho_scale, got, right)
            dep[rho_scale] = abs(mirrored - right) / abs(right)
    finally:
        ds.close()
        ctx.close()
    print("Wand mirrored layout, relative departure of LSCV by H_12 scale:", dep)
    assert dep[0.0] < 1e-12
    assert all(dep[r] > 1e-3 for r in (0.5, 1.0, 1.5)), dep
