"""Error behaviour of the C ABI: every invalid argument the header documents
fails with its code and leaves the context usable, bandwidth checks come
before any launch, and a batch with one poisoned dataset creates no dataset.
Failures are made on the host (bad arguments); nothing faults or waits on
the device."""
import ctypes as C

import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu

ERR_ARG, ERR_NOT_SPD, ERR_OUTSIDE = 1, 2, 3


@pytest.fixture(scope="module")
def setup():
    from paper_1511_07482_gb300 import Context
    rng = np.random.default_rng(90)
    X = rng.multivariate_normal([0.0, 0.5], [[1.0, 0.4], [0.4, 0.8]], size=3000)
    Hns = synthetic.normal_scale(X)
    lo, hi = synthetic.grid_range(X, Hns)
    c = Context(0)
    ds = c.bin(X, lo, hi, [64, 60])
    ref = ds.lscv(Hns, grad=True)
    yield c, ds, X, Hns, lo, hi, ref
    ds.close()
    c.close()


def _code(excinfo):
    return excinfo.value.code


def _launches(c):
    return c.profile_read()[1]


@pytest.mark.parametrize("bad,code", [
    ([[1.0, 2.0], [2.0, 1.0]], ERR_NOT_SPD),          # indefinite
    ([[0.0, 0.0], [0.0, 0.0]], ERR_NOT_SPD),          # singular
    ([[0.1, 0.02], [0.03, 0.1]], ERR_ARG),            # not symmetric
    ([[np.nan, 0.0], [0.0, 0.1]], ERR_ARG),           # non-finite
])
def test_bad_bandwidth_fails_before_any_launch(setup, bad, code):
    from paper_1511_07482_gb300 import KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    for call in (lambda: ds.lscv(np.array(bad)), lambda: ds.psi(np.array(bad), 2),
                 lambda: ds.scv(np.array(bad), Hns), lambda: ds.lscv(np.stack([Hns, np.array(bad)]))):
        c.profile(0)   # clears the launch counter
        with pytest.raises(KdefftError) as e:
            call()
        assert _code(e) == code
        assert _launches(c) == 0
    # the context and the dataset stay usable and give the same bits
    v, g = ds.lscv(Hns, grad=True)
    assert np.array_equal(v, ref[0]) and np.array_equal(g, ref[1])


def test_bad_pilot_and_start(setup):
    from paper_1511_07482_gb300 import SCV, KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    with pytest.raises(KdefftError) as e:
        ds.scv(Hns, np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert _code(e) == ERR_NOT_SPD
    with pytest.raises(KdefftError) as e:
        ds.select_H(SCV, H0=np.array([[1.0, 2.0], [2.0, 1.0]]), G=Hns)
    assert _code(e) == ERR_NOT_SPD
    assert np.array_equal(ds.lscv(Hns, grad=True)[0], ref[0])


@pytest.mark.parametrize("r", [1, 3, 12])
def test_bad_order(setup, r):
    from paper_1511_07482_gb300 import KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    with pytest.raises(KdefftError) as e:
        ds.psi(Hns, r)
    assert _code(e) == ERR_ARG


def test_bad_grids(setup):
    from paper_1511_07482_gb300 import KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    for lo_, hi_, M in ((lo, hi, [1, 60]), (hi, lo, [64, 60])):
        with pytest.raises(KdefftError) as e:
            c.bin(X, lo_, hi_, M)
        assert _code(e) == ERR_ARG
    X5 = np.zeros((10, 5))
    with pytest.raises(KdefftError) as e:
        c.bin(X5, np.zeros(5), np.ones(5), [4] * 5)
    assert _code(e) == ERR_ARG
    # a point outside the grid under the default policy: no dataset
    Xo = X.copy()
    Xo[7, 0] = hi[0] + 1.0
    with pytest.raises(KdefftError) as e:
        c.bin(Xo, lo, hi, [64, 60])
    assert _code(e) == ERR_OUTSIDE
    assert np.array_equal(ds.lscv(Hns, grad=True)[0], ref[0])


def test_poisoned_batch_creates_no_dataset(setup):
    from paper_1511_07482_gb300 import KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    ws = synthetic.batched_uneven(n_datasets=6, n_candidates=2, base_seed=91, n_range=(500, 2000))
    Xs = [w.X for w in ws]
    Ms = [list(w.M) for w in ws]
    Xs[3] = Xs[3].copy()
    Xs[3][0, 1] = ws[3].hi[1] + 5.0   # one point of one dataset outside its grid
    with pytest.raises(KdefftError) as e:
        c.bin_many(Xs, [w.lo for w in ws], [w.hi for w in ws], Ms)
    assert _code(e) == ERR_OUTSIDE
    # the clean batch still bins, and matches one-at-a-time binning
    Xs[3] = ws[3].X
    dss = c.bin_many(Xs, [w.lo for w in ws], [w.hi for w in ws], Ms)
    for w, dm in zip(ws, dss):
        d1 = c.bin(w.X, w.lo, w.hi, w.M)
        assert np.array_equal(dm.counts(), d1.counts())
        d1.close()
        dm.close()


def test_destroyed_handles_are_rejected():
    from paper_1511_07482_gb300 import Context, _lib
    lib = _lib.load()
    c = Context(0)
    w = synthetic.small_case(n=500, d=2, M=[20, 20], seed=92, n_candidates=1)
    ds = c.bin(w.X, w.lo, w.hi, w.M)
    h = C.c_void_p(ds.h.value)
    assert lib.kdefft_ds_destroy(h) == 0
    ds.h = None
    assert lib.kdefft_ds_destroy(h) == ERR_ARG      # a second destroy is an error, not a use after free
    hc = C.c_void_p(c.h.value)
    c.close()
    assert lib.kdefft_destroy(hc) == ERR_ARG
    assert lib.kdefft_destroy(None) == 0


def test_large_batch_failure_is_reported_exactly(setup):
    """A batch of thousands of bandwidths builds its requests on several host
    threads; one non-positive-definite bandwidth among them still fails with
    its code and message (the set is rebuilt serially to report it), before
    any launch, and the same batch without it gives the values of the
    smaller batches it is made of."""
    from paper_1511_07482_gb300 import KdefftError
    c, ds, X, Hns, lo, hi, ref = setup
    rng = np.random.default_rng(91)
    Hs = np.stack([Hns * s for s in rng.uniform(0.5, 2.0, 5000)])
    bad = Hs.copy()
    bad[3777] = np.array([[1.0, 2.0], [2.0, 1.0]]) * Hns[0, 0]
    c.profile(1)
    with pytest.raises(KdefftError) as e:
        ds.lscv(bad, grad=True)
    assert _code(e) == ERR_NOT_SPD
    assert "positive definite" in str(e.value)
    assert _launches(c) == 0
    c.profile(0)
    v, g = ds.lscv(Hs, grad=True)
    v1, g1 = ds.lscv(Hs[:1000], grad=True)
    v2, g2 = ds.lscv(Hs[4000:], grad=True)
    assert np.array_equal(v[:1000], v1) and np.array_equal(g[:1000], g1)
    assert np.array_equal(v[4000:], v2) and np.array_equal(g[4000:], g2)
