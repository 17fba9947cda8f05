"""The support and padding rules the library applies (Eq. 26 with lambda_max
of the bandwidth, Q5's smallest 5-smooth padded size, Eqs. 21 and 27 for the
paper's rules) against the oracle's rules, over many random bandwidths of
every conditioning and several grids, through kdefft_plan.  The library
finds lambda_max by Jacobi rotations stopped at machine precision and the
next 5-smooth size from a table; the oracle uses numpy's eigenvalues and a
plain search, so a disagreement at an integer boundary of the support, or
an off-by-one in the table, shows here."""
import numpy as np
import pytest

from oracle import rules
from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _random_spd(rng, d, scale):
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    lam = scale * np.exp(rng.uniform(np.log(0.02), np.log(3.0), d))
    return (Q * lam) @ Q.T


@pytest.mark.parametrize("d,M", [(2, [256, 200]), (2, [97, 131]), (3, [64, 48, 80]), (4, [24, 20, 18, 30])])
def test_plan_matches_oracle_rules(d, M):
    from paper_1511_07482_gb300 import P_PAPER, Context
    rng = np.random.default_rng(300 + d)
    w = synthetic.small_case(n=500, d=d, M=M, seed=310 + d, n_candidates=1)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    c = Context(0)
    try:
        ds = c.bin(w.X, w.lo, w.hi, w.M)
        dsp = c.bin(w.X, w.lo, w.hi, w.M, P_rule=P_PAPER)
        span = float(np.max(np.asarray(w.hi) - np.asarray(w.lo)))
        checked = 0
        for k in range(150):
            H = _random_spd(rng, d, (span / 8.0) ** 2 * rng.uniform(0.01, 1.0))
            L_want = [max(1, v) for v in rules.support_L(rules.lambda_max(H), delta, w.M)]
            try:
                L, P = ds.plan(-1, H)
            except Exception:
                # a support whose padded size is beyond the library's limit
                assert max(rules.P_minimal(w.M, L_want)) > 4096
                continue
            assert L == L_want, (H, L, L_want)
            assert P == rules.P_minimal(w.M, L_want)
            try:
                Lp, Pp = dsp.plan(-1, H)
            except Exception:
                assert max(rules.P_paper(w.M, L_want)) > 4096
                continue
            assert Lp == L_want and Pp == rules.P_paper(w.M, L_want)
            checked += 1
        assert checked >= 100
        ds.close()
        dsp.close()
    finally:
        c.close()
