"""Double sums of a kernel over the sample, direct and binned (oracle, FP64).

A "kernel" is a list of terms [(w_m, Sigma_m, alpha_m)] (see gauss.kernel_eval).

  direct_sum      n^-2 sum_i sum_j k(X_i - X_j), all pairs including i = j:
                  Eq. 12 (with k = T_H), Eq. 13 (k = a partial of K_H), the
                  degree-2 V-statistic of Eq. 29.  O(n^2).
  lag_kernel      k_j = k(delta_1 j_1, ..., delta_d j_d) on the lag box
                  [-L, L]^d: Eq. 18 / Eq. 34.
  binned_direct   the binned double sum with truncated lags, Eq. 25:
                  n^-2 sum_i c_i sum_{j in [-L,L]^d} c_{i-j} k_j  (c = 0 off
                  the grid).  The definition the GPU path must reproduce.
                  The finite double sum is evaluated lag by lag (outer sum
                  over j), an exact reordering.
  binned_fft      the paper's steps 3-4 with numpy's FFT in FP64: zero-pad
                  the counts and the lag kernel (layout of Eqs. 19-20: counts
                  at offset L_k, lag j at index j + L_k), C = F(c_zp),
                  K = F(k_zp), S = C K, s = F^{-1}(S) (Eq. 22), extract
                  s[2L : 2L + M] (Eq. 23; numpy's inverse already carries the
                  1 / prod P_k factor), multiply by the counts and sum
                  (Eq. 24).  Must equal binned_direct to rounding.
                  Eq. 23 is printed for the untruncated layout (P >= 3M - 1);
                  with truncated lags the extraction indices are read modulo
                  P, which is exact whenever P_k >= M_k + L_k (the circular
                  convolution then has no wrapped term at those indices).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .gauss import kernel_eval


def direct_sum(X, terms, block: int = 256) -> float:
    """n^-2 sum_i sum_j k(X_i - X_j) (Eqs. 12-13, 29)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    parts = []
    for s in range(0, n, block):
        diff = X[s:s + block, None, :] - X[None, :, :]
        parts.append(float(np.sum(kernel_eval(diff, terms))))
    return math.fsum(parts) / float(n) ** 2


def lag_kernel(terms, delta, L) -> np.ndarray:
    """k_j for j in [-L_0, L_0] x ... x [-L_{d-1}, L_{d-1}] (Eq. 18); array
    index j + L."""
    delta = np.asarray(delta, dtype=np.float64)
    axes = [delta[k] * np.arange(-L[k], L[k] + 1, dtype=np.float64) for k in range(len(L))]
    mesh = np.meshgrid(*axes, indexing="ij")
    x = np.stack(mesh, axis=-1)
    return kernel_eval(x, terms)


def _overlap(c: np.ndarray, j) -> float:
    """sum_i c_i c_{i-j} over the grid (c = 0 outside): the factor of k_j in
    Eq. 25's double sum."""
    sl_a, sl_b = [], []
    for k, jk in enumerate(j):
        Mk = c.shape[k]
        if abs(jk) >= Mk:
            return 0.0
        if jk >= 0:
            sl_a.append(slice(jk, Mk))
            sl_b.append(slice(0, Mk - jk))
        else:
            sl_a.append(slice(0, Mk + jk))
            sl_b.append(slice(-jk, Mk))
    return float(np.sum(c[tuple(sl_a)] * c[tuple(sl_b)]))


def binned_direct(c, n, terms, delta, L) -> float:
    """Eq. 25: n^-2 sum_i c_i sum_{|j_k| <= L_k} c_{i-j} k_j."""
    c = np.asarray(c, dtype=np.float64)
    k = lag_kernel(terms, delta, L)
    parts = []
    for j in itertools.product(*[range(-l, l + 1) for l in L]):
        kj = k[tuple(jj + l for jj, l in zip(j, L))]
        parts.append(kj * _overlap(c, j))
    return math.fsum(parts) / float(n) ** 2


def autocorr(c, A) -> np.ndarray:
    """a_j = sum_i c_i c_{i+j} (c = 0 off the grid): the factor that Eq. 25's
    double sum puts on k_j once the sum over the lag is taken first
    (binned_direct sums k_j times it).  Half box j_0 in [0, A_0], |j_k| <= A_k
    for k >= 1, array indexed [j_{d-1} + A_{d-1}]..[j_1 + A_1][j_0]; the
    other half follows from a_{-j} = a_j."""
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    shape = tuple(2 * A[k] + 1 for k in range(d - 1, 0, -1)) + (A[0] + 1,)
    out = np.zeros(shape)
    for idx in np.ndindex(*shape):
        j = [0] * d
        j[0] = idx[-1]
        for k in range(1, d):
            j[k] = idx[d - 1 - k] - A[k]
        out[idx] = _overlap(c, [-x for x in j])
    return out


def autocorr_fft(c):
    """a_j = sum_i c_i c_{i+j} for every lag |j_k| <= M_k - 1, by one FFT pair
    at P_k = 2 M_k (no wrapped term, since P_k >= 2 M_k - 1), FP64 on every
    host core (pocketfft through scipy.fft).  Lag j sits at index j mod P.
    The same numbers as `autocorr`; this is the route that reaches the
    full-size grids."""
    import scipy.fft as sf
    c = np.asarray(c, dtype=np.float64)
    P = [2 * m for m in c.shape]
    czp = np.zeros(P)
    czp[tuple(slice(0, m) for m in c.shape)] = c
    return sf.irfftn(np.abs(sf.rfftn(czp, workers=-1)) ** 2, s=P, workers=-1)


def lag_sums(a, n, terms, delta, L):
    """(n^-2 sum_{|j_k| <= L_k} k_j a_j, n^-2 sum |k_j| a_j) with a from
    `autocorr_fft`: Eq. 25 with the sum over the grid taken first, and the
    absolute functional of the same kernel (the magnitude of the summed
    terms)."""
    k = lag_kernel(terms, delta, L)
    idx = np.ix_(*[np.arange(-L[i], L[i] + 1) % a.shape[i] for i in range(len(L))])
    aj = a[idx]
    n2 = float(n) ** 2
    return float(np.sum(k * aj)) / n2, float(np.sum(np.abs(k) * aj)) / n2


def half_box_weights(A) -> np.ndarray:
    """w_j on the half box of `autocorr` (Eq. 25 summed over the lag): 2 where the first nonzero of
    (j_0, .., j_{d-1}) is positive, 1 at j = 0, 0 where it is negative, so
    that sum_half w_j f_j = sum_full f_j for every even f."""
    d = len(A)
    shape = tuple(2 * A[k] + 1 for k in range(d - 1, 0, -1)) + (A[0] + 1,)
    w = np.zeros(shape)
    for idx in np.ndindex(*shape):
        j = [idx[-1]] + [idx[d - 1 - k] - A[k] for k in range(1, d)]
        nz = [x for x in j if x != 0]
        w[idx] = 1.0 if not nz else (2.0 if nz[0] > 0 else 0.0)
    return w


def binned_fft(c, n, terms, delta, L, P) -> float:
    """Sec. 4 steps 2-4 with an FFT (Eqs. 19-24); requires P_k >= M_k + L_k."""
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    M = c.shape
    for k in range(d):
        if P[k] < M[k] + L[k]:
            raise ValueError("P_k must be at least M_k + L_k")
    k_lag = lag_kernel(terms, delta, L)
    c_zp = np.zeros(P)
    c_zp[tuple(slice(L[k], L[k] + M[k]) for k in range(d))] = c
    k_zp = np.zeros(P)
    k_zp[tuple(slice(0, 2 * L[k] + 1) for k in range(d))] = k_lag
    C = np.fft.fftn(c_zp)
    K = np.fft.fftn(k_zp)
    S = C * K
    s = np.fft.ifftn(S).real
    conv = s[np.ix_(*[(2 * L[k] + np.arange(M[k])) % P[k] for k in range(d)])]
    return float(np.sum(c * conv)) / float(n) ** 2
