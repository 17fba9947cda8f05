"""Selection over the constrained bandwidth classes of Sec. 3 (D: diagonal,
S: scalar h^2 I) on a correlated Gaussian sample: the result lies in its
class, no neighbouring class member is lower (SCV), and the classes nest (a
search over F started at the D end point, or over D started at the S end
point, never ends higher)."""
import numpy as np
import pytest

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
    yield ds, Hns
    ds.close()
    c.close()


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
