"""Gaussian density and its partial derivatives of any order (oracle, FP64).

Sec. 5 needs D^{(x)r} phi_Sigma(x), the vector of all r-th order partials of
the N(0, Sigma) density, and the scalar functionals eta_{r,s} (Eq. 30) built
from them.  The paper takes these from an external recursive routine and does
not print it; here the partials come from the multivariate Hermite
polynomials with covariance Lambda = Sigma^{-1}:

    d^alpha phi_Sigma(x) = (-1)^{|alpha|} He_alpha(z; Lambda) phi_Sigma(x),
    z = Lambda x,
    He_0 = 1,
    He_{alpha + e_i}(z) = z_i He_alpha(z) - sum_j alpha_j Lambda_ij He_{alpha - e_j}(z).

Derivation (first principles): d/dx_i phi = -z_i phi and dz_j/dx_i =
Lambda_ji; He_alpha is an Appell sequence in z, dHe_alpha/dz_j = alpha_j
He_{alpha-e_j}; differentiating (-1)^{|a|} He_a phi once more in x_i gives the
recurrence.  Pinned in tests against the textbook 1-D probabilists' Hermite
polynomials, against symbolic differentiation (sympy) and against Isserlis'
pairing formula at x = 0.

Multi-index conventions: alpha is a tuple of d non-negative ints.  Kronecker
order for D^{(x)r} (Sec. 5, the vec/Kronecker-power layout): entry
(i_1, ..., i_r), i_1 slowest, is d^{alpha(i)} with alpha(i)_k = #{m : i_m = k}.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def multi_indices(d: int, r: int):
    """All alpha in N^d with |alpha| = r, lexicographically descending: the
    unique entries of D^{(x)r} (Sec. 5)."""
    out = []
    for combo in itertools.combinations_with_replacement(range(d), r):
        a = [0] * d
        for k in combo:
            a[k] += 1
        out.append(tuple(a))
    return sorted(set(out), reverse=True)


def kron_alphas(d: int, r: int):
    """alpha(i) for every Kronecker position i of D^{(x)r}, i_1 slowest
    (Sec. 5's vec / Kronecker-power layout)."""
    out = []
    for idx in itertools.product(range(d), repeat=r):
        a = [0] * d
        for k in idx:
            a[k] += 1
        out.append(tuple(a))
    return out


def gauss_density(x: np.ndarray, Sigma: np.ndarray) -> np.ndarray:
    """phi_Sigma(x) = (2 pi)^{-d/2} |Sigma|^{-1/2} exp(-x^T Sigma^{-1} x / 2).

    This is K_H of Eq. 2 with K the standard normal density and H = Sigma.
    x has shape (..., d)."""
    x = np.asarray(x, dtype=np.float64)
    Sigma = np.asarray(Sigma, dtype=np.float64)
    d = Sigma.shape[0]
    Lam = np.linalg.inv(Sigma)
    q = np.einsum("...i,ij,...j->...", x, Lam, x)
    norm = (2.0 * math.pi) ** (-d / 2.0) / math.sqrt(np.linalg.det(Sigma))
    return norm * np.exp(-0.5 * q)


def hermite_table(z: np.ndarray, Lam: np.ndarray, R: int) -> dict:
    """He_alpha(z; Lambda) for every |alpha| <= R by the recurrence above,
    which gives the partials that Sec. 5 needs.

    z has shape (..., d).  Returns {alpha: array of shape z.shape[:-1]}."""
    d = Lam.shape[0]
    zero = tuple([0] * d)
    He = {zero: np.ones(z.shape[:-1])}
    for r in range(1, R + 1):
        for alpha in multi_indices(d, r):
            i = next(k for k in range(d) if alpha[k] > 0)
            beta = list(alpha)
            beta[i] -= 1
            beta = tuple(beta)
            val = z[..., i] * He[beta]
            for j in range(d):
                if beta[j] > 0:
                    bj = list(beta)
                    bj[j] -= 1
                    val = val - beta[j] * Lam[i, j] * He[tuple(bj)]
            He[alpha] = val
    return He


def gauss_derivs(x: np.ndarray, Sigma: np.ndarray, alphas) -> dict:
    """{alpha: d^alpha phi_Sigma(x)} for the requested multi-indices: the
    entries of D^{(x)r} phi_Sigma (Sec. 5)."""
    x = np.asarray(x, dtype=np.float64)
    Sigma = np.asarray(Sigma, dtype=np.float64)
    Lam = np.linalg.inv(Sigma)
    z = np.einsum("ij,...j->...i", Lam, x)
    phi = gauss_density(x, Sigma)
    alphas = [tuple(a) for a in alphas]
    R = max((sum(a) for a in alphas), default=0)
    He = hermite_table(z, Lam, R)
    return {a: ((-1.0) ** sum(a)) * He[a] * phi for a in alphas}


def gauss_deriv(x: np.ndarray, Sigma: np.ndarray, alpha) -> np.ndarray:
    """d^alpha phi_Sigma(x) for one multi-index (Sec. 5)."""
    return gauss_derivs(x, Sigma, [alpha])[tuple(alpha)]


def kernel_eval(x: np.ndarray, terms) -> np.ndarray:
    """A kernel that is a finite sum of Gaussian partials:

        k(x) = sum_m w_m d^{alpha_m} phi_{Sigma_m}(x),

    terms = [(w_m, Sigma_m, alpha_m), ...].  Every kernel in Secs. 4-5 has
    this form: T_H of Eq. 11 / Eq. 34, the eta_{r,s} of Eq. 30 (after the
    Kronecker contraction) and the gradient kernels."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[:-1])
    # group by covariance so that each Hermite table is built once
    groups: dict = {}
    for w, S, a in terms:
        key = tuple(np.asarray(S, dtype=np.float64).ravel())
        groups.setdefault(key, (np.asarray(S, dtype=np.float64), []))[1].append((w, tuple(a)))
    for _, (S, lst) in groups.items():
        D = gauss_derivs(x, S, [a for _, a in lst])
        for w, a in lst:
            out = out + w * D[a]
    return out


def pairings_value_at_zero(Sigma: np.ndarray, alpha) -> float:
    """Isserlis closed form of d^alpha phi_Sigma(0) (the value at the origin
    that the n = 1 case of Eq. 13 reduces to), independent of the
    recurrence: (-1)^{|alpha|/2} phi_Sigma(0) sum over perfect matchings of the
    multiset alpha of prod Lambda_ab; zero for odd |alpha|."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    Lam = np.linalg.inv(Sigma)
    labels = [k for k, m in enumerate(alpha) for _ in range(m)]
    r = len(labels)
    phi0 = gauss_density(np.zeros(Sigma.shape[0]), Sigma)
    if r % 2:
        return 0.0

    def matchings(items):
        if not items:
            yield []
            return
        a = items[0]
        for t in range(1, len(items)):
            rest = items[1:t] + items[t + 1:]
            for m in matchings(rest):
                yield [(a, items[t])] + m

    total = 0.0
    for m in matchings(labels):
        total += math.prod(Lam[a, b] for a, b in m)
    return ((-1.0) ** (r // 2)) * phi0 * total
