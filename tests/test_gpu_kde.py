"""The grid estimate and the mixture ISE on the device (Eqs. 1, 37) against
the oracle's definitions, on the paper's kind of target: a bivariate normal
mixture sample, and 1-D / 3-D cases."""
import numpy as np
import pytest

from oracle import binning, kde, rules
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1511_07482_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("d,M", [(1, [120]), (2, [64, 58]), (3, [20, 18, 16])])
def test_grid_estimate_matches_oracle(ctx, d, M):
    w = synthetic.small_case(n=3000, d=d, M=M, seed=60 + d, n_candidates=2)
    ds = ctx.bin(w.X, w.lo, w.hi, M)
    for H in w.H:
        got = ds.kde_grid(H)
        c = binning.bin_linear(w.X, w.lo, w.hi, M)
        delta = rules.bin_width(w.lo, w.hi, M)
        L = rules.support_L(rules.lambda_max(H), delta, M)
        want = kde.kde_grid(c, w.n, H, delta, L)
        assert got.shape == want.shape
        assert np.max(np.abs(got - want)) <= 1e-6 * np.max(want)
    ds.close()


def test_mixture_ise_matches_oracle(ctx):
    w = synthetic.small_case(n=3000, d=2, M=[60, 56], seed=64, n_candidates=3)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    wt = np.array([0.5, 0.3, 0.2])
    mu = np.array([[-0.5, 0.1], [0.7, 0.6], [0.0, -0.8]])
    S = np.array([[[0.3, 0.1], [0.1, 0.2]], [[0.2, -0.05], [-0.05, 0.4]], [[0.5, 0.0], [0.0, 0.1]]])
    got = ds.ise_mixture(np.stack(w.H), wt, mu, S)
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    for g, H in zip(got, w.H):
        L2 = rules.support_L(rules.lambda_max(2.0 * H), delta, w.M)
        want = kde.ise_mixture_binned(c, w.n, np.asarray(w.lo), delta, H, wt, mu, S, L2)
        scale = kde.mixture_sq_integral(wt, mu, S)
        assert abs(g - want) <= 2e-6 * scale, (g, want)
        assert g > 0.0
    ds.close()
