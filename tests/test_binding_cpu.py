"""Argument checks of the Python binding that run before any library call
(CPU): the C ABI reads d*d values through every matrix pointer and d values
through every per-axis pointer, so a short array must be refused on the host
rather than read past its end."""
import numpy as np
import pytest

from paper_1511_07482_gb300 import _lib
from paper_1511_07482_gb300._lib import Context, Dataset


def _ds(d=2, M=(8, 8)):
    return Dataset(None, None, d, list(M))


def _ctx():
    c = Context.__new__(Context)     # no device: only the host-side checks run
    c.h = None
    c._datasets = set()
    return c


@pytest.mark.parametrize("call", [
    lambda ds: ds.scv(np.eye(2), np.eye(1)),
    lambda ds: ds.pi(np.eye(2), [0.1, 0.2, 0.3]),
    lambda ds: ds.eta02(np.eye(2), np.eye(3)),
    lambda ds: ds.plan(0, np.eye(3)),
    lambda ds: ds.plan(1, np.eye(2), np.ones(3)),
    lambda ds: ds.kde_grid(np.ones(2)),
    lambda ds: ds.eta_rs(np.eye(2), 1, 1, A=np.eye(1)),
    lambda ds: ds.eta_rs(np.eye(2), 1, 1, B=np.zeros(5)),
    lambda ds: ds.select_H(0, H0=np.eye(3)),
    lambda ds: ds.select_H(1, G=np.eye(1)),
    lambda ds: ds.select_H_many([0, 1], G=np.ones(2)),
])
def test_short_matrices_are_refused(call):
    with pytest.raises(ValueError):
        call(_ds())


def test_sample_and_grid_arguments_are_checked():
    c = _ctx()
    X = np.zeros((10, 2))
    with pytest.raises(ValueError):
        c.bin(np.zeros(10), [0, 0], [1, 1], [8, 8])          # not n x d
    with pytest.raises(ValueError):
        c.bin(X, [0.0], [1.0, 1.0], [8, 8])                   # lo short
    with pytest.raises(ValueError):
        c.bin(X, [0.0, 0.0], [1.0, 1.0, 1.0], [8, 8])         # hi long
    with pytest.raises(ValueError):
        c.bin(X, [0.0, 0.0], [1.0, 1.0], [8])                 # M short
    with pytest.raises(ValueError):
        c.bin_many([X, np.zeros((5, 3))], [[0, 0], [0, 0]], [[1, 1], [1, 1]], [[8, 8], [8, 8]])


def test_well_shaped_arguments_pass_the_checks():
    a, _ = _lib._mat(np.eye(2)[None], 2, "G")         # a 1 x d x d stack of one is accepted
    assert a.size == 4
    assert _lib._opt_mat(None, 3, "G") == (None, None)
    v = _lib._vec([[1, 2, 3]], 3, "M", np.int64)
    assert v.dtype == np.int64 and v.shape == (3,)
    keep, p = _lib._ptr_of(np.zeros((4, 3)))
    assert keep.shape == (4, 3) and p == keep.ctypes.data != 0


def test_empty_batches_give_empty_results():
    """No bandwidths, no datasets: empty results of the documented shapes,
    without a library call (the C ABI itself refuses empty batches)."""
    ds = _ds(d=2)
    H0 = np.zeros((0, 2, 2))
    G = np.eye(2)
    assert ds.psi(H0, 4).shape == (0, 16)
    v, g = ds.lscv(H0, grad=True)
    assert v.shape == (0,) and g.shape == (0, 2, 2)
    assert ds.lscv(H0).shape == (0,)
    assert ds.scv(H0, G, grad=True)[1].shape == (0, 2, 2)
    assert ds.pi(H0, G).shape == (0,)
    assert ds.eta02(H0, G).shape == (0,)
    assert ds.qr(H0, 2).shape == (0,)
    assert ds.eta_rs(H0, 1, 1).shape == (0,)
    assert ds.lscv_r(H0, 1).shape == (0,)
    assert ds.ise_mixture(H0, [1.0], [[0.0, 0.0]], [np.eye(2)]).shape == (0,)
    c = _ctx()
    assert c.bin_many([], [], [], []) == []
    assert c.batch_lscv([], [], grad=False).shape == (0,)
    # the G check still runs on an empty batch
    with pytest.raises(ValueError):
        ds.scv(H0, np.eye(3))
