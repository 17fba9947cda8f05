"""Pins for oracle.rules against the paper's Tables 2 and 3 (Sec. 6.3)."""
import math
import os

import numpy as np
import pytest

from oracle import rules

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_table2_follows_from_table3_by_eq27():
    P = {(M, n): (p1, p2) for M, n, p1, p2 in _load("table2_P.txt")}
    L = {(n, M): (l1, l2) for n, M, l1, l2 in _load("table3_L.txt")}
    checked = 0
    for (n, M), (l1, l2) in L.items():
        if (M, n) in P:
            assert tuple(rules.P_paper([M, M], [l1, l2])) == P[(M, n)]
            checked += 1
    assert checked == 20


def test_table3_rows_fit_eq26_with_eq16():
    """Each (row, axis) of Table 3 must be ceil(c (M-1)) for one constant
    c = tau sqrt(lambda) / range (Eq. 26 with delta = range/(M-1), Eq. 16).
    The constant is recovered, then support_L must regenerate the row."""
    rows = {}
    for n, M, l1, l2 in _load("table3_L.txt"):
        rows.setdefault(n, []).append((M, l1, l2))
    for n, r in rows.items():
        for ax in (0, 1):
            lo, hi = -1.0, 1e9
            for M, l1, l2 in r:
                Lk = (l1, l2)[ax]
                lo = max(lo, (Lk - 1) / (M - 1))
                hi = min(hi, Lk / (M - 1))
            assert lo < hi, (n, ax)
            c = 0.5 * (lo + hi)
            rng_width = 10.0
            tau = 3.7
            lam = (c * rng_width / tau) ** 2
            for M, l1, l2 in r:
                delta = rules.bin_width([0.0], [rng_width], [M])
                got = rules.support_L(lam, delta, [M], tau)[0]
                assert got == (l1, l2)[ax], (n, M, ax)


def test_table3_rejects_range_over_M():
    """The same fit with delta = range/M fails on some rows: Table 3 does
    distinguish Eq. 16 from that plausible slip."""
    rows = {}
    for n, M, l1, l2 in _load("table3_L.txt"):
        rows.setdefault(n, []).append((M, l1, l2))
    bad = 0
    for n, r in rows.items():
        for ax in (0, 1):
            lo, hi = -1.0, 1e9
            for M, l1, l2 in r:
                Lk = (l1, l2)[ax]
                lo = max(lo, (Lk - 1) / M)
                hi = min(hi, Lk / M)
            bad += not (lo < hi)
    assert bad > 0


def test_P_rules_small_values():
    assert rules.P_paper_full([100]) == [512]          # 3*100-1 = 299
    assert rules.P_paper([100], [20]) == [256]         # 139
    assert rules.P_minimal([100], [20]) == [120]
    assert rules.P_minimal([256], [21]) == [288]
    assert rules.P_minimal([48], [47]) == [96]
    # bounds that are themselves powers of two or 5-smooth: Eqs. 21 and 27
    # round up only strictly above them, and the minimal rule stops at the
    # first smooth size at or above M + L (120 = M + L - 1 is one short)
    assert rules.P_paper([5], [2]) == [8]              # 5 + 4 - 1 = 8
    assert rules.P_paper([9], [12]) == [32]            # 9 + 24 - 1 = 32
    assert rules.P_paper_full([3]) == [8]              # 3*3-1 = 8
    assert rules.P_paper_full([11]) == [32]            # 3*11-1 = 32
    assert rules.P_minimal([100], [21]) == [125]       # 121..124 are not 5-smooth
    assert rules.support_L(1.0, [0.1], [10], 3.7) == [9]   # capped at M-1
    assert rules.support_L(0.04, [0.1], [100], 3.7) == [8]  # ceil(7.4)


def test_bin_width_eq16():
    np.testing.assert_allclose(rules.bin_width([0.0, -1.0], [1.0, 1.0], [11, 5]), [0.1, 0.5])


def test_lambda_max_closed_form_and_rayleigh_bound():
    """2 x 2: (tr + sqrt(tr^2 - 4 det)) / 2.  3 x 3: no Rayleigh quotient
    exceeds it, and the power iteration reaches it."""
    S2 = np.array([[0.3, 0.12], [0.12, 0.2]])
    tr, det = np.trace(S2), np.linalg.det(S2)
    assert rules.lambda_max(S2) == pytest.approx((tr + math.sqrt(tr * tr - 4 * det)) / 2, rel=1e-14)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3))
    S3 = A @ A.T + 0.2 * np.eye(3)
    lam = rules.lambda_max(S3)
    x = rng.standard_normal((1000, 3))
    q = np.einsum("pi,ij,pj->p", x, S3, x) / np.einsum("pi,pi->p", x, x)
    assert np.all(q <= lam * (1 + 1e-12))
    v = np.ones(3)
    for _ in range(500):
        v = S3 @ v
        v /= np.linalg.norm(v)
    assert float(v @ S3 @ v) == pytest.approx(lam, rel=1e-10)
