"""Oracle (test infrastructure, CPU FP64): the binned kernel density estimate
on the grid (Eq. 1 with the sample replaced by its bin counts) and the
integrated squared error against a normal mixture (Eq. 37), both written out
from their definitions.  Imported only by the tests, the smoke check and the
benchmark's CPU baseline."""
from __future__ import annotations

import itertools

import numpy as np

from .gauss import gauss_density


def kde_grid(c, n, H, delta, L):
    """Eq. 1 with the sample replaced by its bin counts:
    f_hat(g) = n^-1 sum_{|l_k| <= L_k} c_{g - l} K_H(delta (.) l) at every
    grid node g (c = 0 off the grid): shifted copies of the counts weighted
    by the Gaussian at each lag."""
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    M = c.shape
    out = np.zeros(M)
    for l in itertools.product(*[range(-Lk, Lk + 1) for Lk in L]):
        x = np.asarray(delta, dtype=np.float64) * np.asarray(l, dtype=np.float64)
        k = float(gauss_density(x[None, :], np.asarray(H, dtype=np.float64))[0])
        dst = tuple(slice(max(0, lk), M[i] + min(0, lk)) for i, lk in enumerate(l))
        src = tuple(slice(max(0, -lk), M[i] - max(0, lk)) for i, lk in enumerate(l))
        out[dst] += k * c[src]
    return out / float(n)


def mixture_sq_integral(w, mu, S):
    """The int f^2 term of Eq. 37:
    int f^2 = sum_lm w_l w_m phi_{S_l + S_m}(mu_l - mu_m) for
    f = sum_m w_m phi_{S_m}(. - mu_m) (Gaussian convolution identity)."""
    K = len(w)
    tot = 0.0
    for a in range(K):
        for b in range(K):
            x = (np.asarray(mu[a]) - np.asarray(mu[b]))[None, :]
            tot += w[a] * w[b] * float(gauss_density(x, np.asarray(S[a]) + np.asarray(S[b]))[0])
    return tot


def ise_mixture_binned(c, n, lo, delta, H, w, mu, S, L2):
    """Eq. 37 for the binned estimate: int f_hat^2 (the binned double sum of
    phi_2H over the support L2), minus twice int f_hat f (the counts against
    the mixture smoothed by H), plus int f^2."""
    from .functionals import binned_direct
    c = np.asarray(c, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    d = c.ndim
    ff = binned_direct(c, n, [(1.0, 2.0 * H, (0,) * d)], delta, L2)
    grids = np.meshgrid(*[lo[k] + delta[k] * np.arange(c.shape[k]) for k in range(d)], indexing="ij")
    xg = np.stack([g.ravel() for g in grids], axis=1)
    fm = np.zeros(xg.shape[0])
    for wm, m, Sm in zip(w, mu, S):
        fm += wm * gauss_density(xg - np.asarray(m)[None, :], H + np.asarray(Sm))
    cross = float(np.sum(c.ravel() * fm)) / float(n)
    return ff - 2.0 * cross + mixture_sq_integral(w, mu, S)


def ise_mixture_exact(X, H, w, mu, S):
    """Eq. 37 for the unbinned estimate, in closed form:
    n^-2 sum_ij phi_2H(X_i - X_j) - 2 n^-1 sum_i sum_m w_m phi_{H+S_m}(X_i - mu_m)
    + int f^2."""
    X = np.asarray(X, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    n = X.shape[0]
    a = 0.0
    for i in range(n):
        a += float(np.sum(gauss_density(X - X[i][None, :], 2.0 * H)))
    b = 0.0
    for wm, m, Sm in zip(w, mu, S):
        b += wm * float(np.sum(gauss_density(X - np.asarray(m)[None, :], H + np.asarray(Sm))))
    return a / n ** 2 - 2.0 * b / n + mixture_sq_integral(w, mu, S)
