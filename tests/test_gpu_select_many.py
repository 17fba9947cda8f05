"""Several criteria selected on one dataset (kdefft_select_H_multi) and the
per-context block cache of dataset memory.

The two-criterion device search runs LSCV's and SCV's starts in one launch
against one autocorrelation box; each CTA's search depends only on its own
start and the box, so every result must be bit-identical to the one
select_H gives once the box is that large.  Criteria the device search does
not cover (PI; d = 3) take the host-driven path and must match it too."""
import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _mixture2d(n, seed, M):
    rng = np.random.default_rng(seed)
    X = synthetic.sample_mixture(rng, n, [0.6, 0.4], [[-1.0, 0.5], [1.2, -0.3]],
                                 [[[0.5, 0.2], [0.2, 0.4]], [[0.3, -0.1], [-0.1, 0.6]]])
    Hns = synthetic.normal_scale(X)
    lo, hi = synthetic.grid_range(X, Hns)
    return X, Hns, lo, hi, [M, M]


def test_two_criteria_in_one_launch_match_single_searches():
    from paper_1511_07482_gb300 import LSCV, SCV, Context
    X, Hns, lo, hi, M = _mixture2d(20000, 5, 128)
    c = Context(0)
    try:
        ds = c.bin(X, lo, hi, M)
        many = ds.select_H_many([LSCV, SCV], G=Hns, n_starts=6, max_iter=40)
        # the box is now sized for both; single searches reuse it
        for (Hm, fm, em), m in zip(many, (LSCV, SCV)):
            Hs, fs, es = ds.select_H(m, G=Hns, n_starts=6, max_iter=40)
            np.testing.assert_array_equal(Hm, Hs)
            assert fm == fs
            assert em == es
        # the order of the criteria does not matter
        rev = ds.select_H_many([SCV, LSCV], G=Hns, n_starts=6, max_iter=40)
        np.testing.assert_array_equal(rev[0][0], many[1][0])
        np.testing.assert_array_equal(rev[1][0], many[0][0])
        # a single-criterion list is select_H
        one = ds.select_H_many([LSCV], n_starts=6, max_iter=40)
        np.testing.assert_array_equal(one[0][0], many[0][0])
        # the value reported is the objective at the selected point
        H, f, _ = many[0]
        assert f == pytest.approx(ds.lscv(H)[0], rel=1e-12)
        ds.close()
    finally:
        c.close()


def test_uncovered_criteria_take_the_host_path():
    from paper_1511_07482_gb300 import LSCV, PI, SCV, Context
    c = Context(0)
    try:
        X, Hns, lo, hi, M = _mixture2d(3000, 9, 64)
        ds = c.bin(X, lo, hi, M)
        res = ds.select_H_many([PI, LSCV, SCV], G=Hns, n_starts=3, max_iter=30)
        Hp, fp, _ = ds.select_H(PI, G=Hns, n_starts=3, max_iter=30)
        np.testing.assert_array_equal(res[0][0], Hp)
        assert res[0][1] == fp
        ds.close()
        # d = 3: every criterion runs the host-driven search
        rng = np.random.default_rng(3)
        X3 = rng.multivariate_normal([0, 0, 0], [[1, 0.3, 0], [0.3, 1, 0.2], [0, 0.2, 1]], size=3000)
        H3 = synthetic.normal_scale(X3)
        lo3, hi3 = synthetic.grid_range(X3, H3)
        ds3 = c.bin(X3, lo3, hi3, [24, 24, 24])
        res3 = ds3.select_H_many([LSCV, SCV], G=H3, n_starts=2, max_iter=15)
        for (Hm, fm, _), m in zip(res3, (LSCV, SCV)):
            Hs, fs, _ = ds3.select_H(m, G=H3, n_starts=2, max_iter=15)
            np.testing.assert_array_equal(Hm, Hs)
            assert fm == fs
        ds3.close()
    finally:
        c.close()


def test_select_many_rejects_unknown_criteria():
    from paper_1511_07482_gb300 import LSCV, Context, KdefftError
    X, Hns, lo, hi, M = _mixture2d(1000, 1, 32)
    c = Context(0)
    try:
        ds = c.bin(X, lo, hi, M)
        with pytest.raises(KdefftError):
            ds.select_H_many([LSCV, 7])
        ds.close()
    finally:
        c.close()


def test_block_cache_reuses_dataset_memory_and_keeps_results():
    from paper_1511_07482_gb300 import Context
    X, Hns, lo, hi, M = _mixture2d(20000, 7, 128)
    Hs = np.stack([Hns * s for s in (0.5, 1.0, 2.0)])
    ref_ctx = Context(0)
    try:
        ds = ref_ctx.bin(X, lo, hi, M)
        ref, gref = ds.lscv(Hs, grad=True)
        ds.close()
    finally:
        ref_ctx.close()
    c = Context(0)
    try:
        st0 = c.memory_stats()
        for _ in range(3):
            ds = c.bin(X, lo, hi, M)
            v, g = ds.lscv(Hs, grad=True)
            ds.close()
            np.testing.assert_array_equal(v, ref)
            np.testing.assert_array_equal(g, gref)
        st = c.memory_stats()
        # the second and third datasets draw every block from the cache
        assert st["hits"] > st0["hits"]
        assert st["cached_bytes"] > 0
        misses_before = st["misses"]
        ds = c.bin(X, lo, hi, M)
        ds.lscv(Hs, grad=True)
        ds.close()
        assert c.memory_stats()["misses"] == misses_before
        c.trim()
        assert c.memory_stats()["cached_bytes"] == 0
    finally:
        c.close()
