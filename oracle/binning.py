"""Binning of the sample onto the grid, Sec. 4 first step (oracle, FP64).

The paper refers linear binning to Wand (1994, Sec. 3) without printing the
weight rule; the reading used here is the standard multilinear one:

  t_k   = (x_k - g_{k1}) / delta_k          (delta_k from Eq. 16; FP64, the
                                             subtraction and the division are
                                             separate IEEE operations)
  l_k   = floor(t_k), f_k = t_k - l_k       (a point on the upper edge,
                                             t_k = M_k - 1, goes to cell
                                             M_k - 2 with f_k = 1)
  corner l + b (b in {0,1}^d) receives prod_k (f_k if b_k else 1 - f_k),
  the product taken in axis order k = 0..d-1.

Simple binning puts weight 1 on the nearest node, l_k = floor(t_k + 0.5)
(ties at half a bin round up).  A point lies inside the grid when
g_{k1} <= x_k <= g_{kM_k} on every axis (the grid range contains the data,
Sec. 4); rounding in delta_k can push t_k of a point at the upper end just
past M_k - 1, so t_k is clamped to M_k - 1.  A point outside: policy "error"
raises, policy "drop" skips it.

Counts are laid out row-major over (M_0, ..., M_{d-1}), last axis fastest.
"""
from __future__ import annotations

import itertools

import numpy as np

from .rules import bin_width


class OutsideGrid(ValueError):
    pass


def _coords(X, lo, hi, M):
    """t_k = (x_k - g_k1) / delta_k with delta_k of Eq. 16, clamped to M_k - 1
    (Sec. 4, first step; reading in the module header)."""
    X = np.asarray(X, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    delta = bin_width(lo, hi, M)
    t = (X - lo) / delta
    t = np.minimum(t, (np.asarray(M, dtype=np.int64) - 1).astype(np.float64))
    return t, delta


def _inside(X, lo, hi, policy):
    """g_k1 <= x_k <= g_kM_k on every axis (the grid range holds the data,
    Sec. 4); outside points raise under "error" and are skipped under "drop"."""
    X = np.asarray(X, dtype=np.float64)
    ok = np.all((X >= np.asarray(lo, dtype=np.float64)) & (X <= np.asarray(hi, dtype=np.float64)), axis=1)
    if not np.all(ok):
        if policy == "error":
            raise OutsideGrid(f"{int((~ok).sum())} points outside the grid")
    return ok


def bin_linear(X, lo, hi, M, policy: str = "error"):
    """Linear binning (Sec. 4, first step; multilinear weights as in the
    module header); returns FP64 counts of shape M."""
    M = [int(m) for m in M]
    t, _ = _coords(X, lo, hi, M)
    ok = _inside(X, lo, hi, policy)
    t = t[ok]
    l = np.floor(t)
    Mm1 = np.asarray(M, dtype=np.float64) - 1.0
    l = np.where(l >= Mm1, Mm1 - 1.0, l)
    f = t - l
    l = l.astype(np.int64)
    d = len(M)
    c = np.zeros(M, dtype=np.float64)
    for b in itertools.product((0, 1), repeat=d):
        w = np.ones(t.shape[0])
        for k in range(d):
            w = w * (f[:, k] if b[k] else (1.0 - f[:, k]))
        idx = tuple(l[:, k] + b[k] for k in range(d))
        np.add.at(c, idx, w)
    return c


def bin_simple(X, lo, hi, M, policy: str = "error"):
    """Simple (nearest-node) binning (Sec. 4, first step); returns int64
    counts of shape M."""
    M = [int(m) for m in M]
    t, _ = _coords(X, lo, hi, M)
    ok = _inside(X, lo, hi, policy)
    t = t[ok]
    l = np.floor(t + 0.5).astype(np.int64)
    c = np.zeros(M, dtype=np.int64)
    np.add.at(c, tuple(l[:, k] for k in range(len(M))), 1)
    return c


def grid_points(lo, hi, M):
    """The node coordinates g_{k j} = g_{k1} + (j-1) delta_k (Eq. 15-16)."""
    delta = bin_width(lo, hi, M)
    return [float(lo[k]) + delta[k] * np.arange(int(M[k])) for k in range(len(M))]
