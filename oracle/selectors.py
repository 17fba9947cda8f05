"""Objective functions and functionals built on the double sums (oracle, FP64).

Every function takes an evaluator ``ev(terms) -> float`` that returns the
double sum n^-2 sum_i sum_j k(X_i - X_j) of a kernel given as terms
[(w, Sigma, alpha)]: either the direct sum (functionals.direct_sum, Eqs.
12-13) or the binned one (functionals.binned_direct / binned_fft, Eq. 25 and
Eqs. 19-24) with the caller's L and P.  This keeps each objective's algebra
in one place for both forms.

Gradient convention: the d x d symmetric matrix g with g_aa = dF/dH_aa and,
for a != b, g_ab = g_ba = dF/dh_ab where h_ab is the single free parameter
that sets both H_ab and H_ba (the derivative along E_ab + E_ba).  The
kernels use the heat equation of the Gaussian,

    d phi_Sigma / d Sigma_ab  (entries independent) = 1/2 d_a d_b phi_Sigma,

so under the tied convention off-diagonal entries carry a factor 2.
(Derivation: d log phi/dSigma = -Lambda/2 + Lambda x x^T Lambda / 2 and
grad grad^T phi = (Lambda x x^T Lambda - Lambda) phi.)  The gradient with L
held fixed is exactly the derivative of the binned sum of Eq. 25, since
k_j depends on H only through the kernel values.
"""
from __future__ import annotations

import math

import numpy as np

from .gauss import kron_alphas, multi_indices


def _e(d, *idx):
    """The multi-index with one count per listed axis (d_a d_b ... of Sec. 5)."""
    a = [0] * d
    for i in idx:
        a[i] += 1
    return tuple(a)


def _tie(a, b):
    """1 on the diagonal, 2 off it: the tied-entry gradient convention of the
    module header, one free parameter per entry pair of the unconstrained H
    (Sec. 3)."""
    return 1.0 if a == b else 2.0


def _det(S):
    """|S| (LAPACK via numpy), as in K_H(0) of Eq. 11."""
    return float(np.linalg.det(np.asarray(S, dtype=np.float64)))


def vech_pairs(d):
    """(a, b) with a <= b in row-major order: the free entries of the
    unconstrained H (Sec. 3)."""
    return [(a, b) for a in range(d) for b in range(a, d)]


# ---------------------------------------------------------------------------
# LSCV: Sec. 3 Eq. 8 (leave-one-out form) and Sec. 4 Eqs. 10-11 (n ~ n-1)

def lscv_T_terms(H):
    """T_H = K_H * K_H - 2 K_H = phi_{2H} - 2 phi_H (Eq. 11, Eq. 34)."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    z = _e(d)
    return [(1.0, 2.0 * H, z), (-2.0, H, z)]


def lscv_grad_terms(H, a, b, loo_factor: float = 1.0):
    """d T_H / dh_ab = s_ab (d_a d_b phi_{2H} - f d_a d_b phi_H), f = 1 for
    Eq. 10 and n/(n-1) for the leave-one-out form of Eq. 8."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    s = _tie(a, b)
    al = _e(d, a, b)
    return [(s, 2.0 * H, al), (-s * loo_factor, H, al)]


def K0(H) -> float:
    """K_H(0) = (2 pi)^{-d/2} |H|^{-1/2} (Eq. 11)."""
    d = np.asarray(H).shape[0]
    return (2.0 * math.pi) ** (-d / 2.0) / math.sqrt(_det(H))


def lscv(ev, H, n: int, exact_loo: bool = False, grad: bool = False):
    """LSCV(H).  exact_loo=False: Eq. 10, psi(H) + 2 n^-1 K_H(0) with psi of
    Eq. 12.  exact_loo=True: Eq. 8 with the j != i sum written as the full
    double sum minus its n diagonal terms K_H(0)."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    Hinv = np.linalg.inv(H)
    k0 = K0(H)
    if not exact_loo:
        val = ev(lscv_T_terms(H)) + 2.0 * k0 / n
        fac = 1.0
    else:
        z = _e(d)
        A = ev([(1.0, 2.0 * H, z)])
        B = ev([(1.0, H, z)])
        val = A - 2.0 * n / (n - 1.0) * B + 2.0 / (n - 1.0) * k0
        fac = n / (n - 1.0)
    if not grad:
        return val
    g = np.zeros((d, d))
    # d K_H(0) / dH (entries independent) = -K_H(0) H^{-1} / 2
    c0 = (2.0 / n) if not exact_loo else (2.0 / (n - 1.0))
    for a, b in vech_pairs(d):
        v = ev(lscv_grad_terms(H, a, b, fac)) + c0 * _tie(a, b) * (-0.5 * k0 * Hinv[a, b])
        g[a, b] = g[b, a] = v
    return val, g


# ---------------------------------------------------------------------------
# SCV: named in Sec. 3, formulas deferred by Sec. 5 to an external source.
# Reading (Gaussian kernel and pilot, V-statistic including i = j):
#   SCV(H) = n^-1 (4 pi)^{-d/2} |H|^{-1/2}
#            + n^-2 sum sum [phi_{2H+2G} - 2 phi_{H+2G} + phi_{2G}](X_i - X_j)

def scv_terms(H, G):
    """The kernel of the SCV double sum (reading in the comment above; SCV is
    named in Sec. 3): phi_{2H+2G} - 2 phi_{H+2G} + phi_{2G}."""
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    z = _e(H.shape[0])
    return [(1.0, 2.0 * H + 2.0 * G, z), (-2.0, H + 2.0 * G, z), (1.0, 2.0 * G, z)]


def scv_grad_terms(H, G, a, b):
    """d/dh_ab of the SCV kernel (SCV named in Sec. 3) by the heat equation:
    s_ab (d_a d_b phi_{2H+2G} - d_a d_b phi_{H+2G})."""
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    s = _tie(a, b)
    al = _e(H.shape[0], a, b)
    return [(s, 2.0 * H + 2.0 * G, al), (-s, H + 2.0 * G, al)]


def RK(H) -> float:
    """n-free roughness term (4 pi)^{-d/2} |H|^{-1/2} = int K_H^2, the K_H * K_H
    of Eq. 11 at 0."""
    d = np.asarray(H).shape[0]
    return (4.0 * math.pi) ** (-d / 2.0) / math.sqrt(_det(H))


def scv(ev, H, G, n: int, grad: bool = False):
    """SCV(H) (Sec. 3; the reading above) and, with grad, its gradient in the
    tied convention."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    r0 = RK(H)
    val = r0 / n + ev(scv_terms(H, G))
    if not grad:
        return val
    Hinv = np.linalg.inv(H)
    g = np.zeros((d, d))
    for a, b in vech_pairs(d):
        v = ev(scv_grad_terms(H, G, a, b)) + _tie(a, b) * (-0.5 * r0 * Hinv[a, b]) / n
        g[a, b] = g[b, a] = v
    return val, g


def abs_scales(ev_abs, method, H, n: int, G=None):
    """Magnitudes of the summed terms of an objective and of each gradient
    entry: the absolute functional n^-2 sum |k|(X_i - X_j) of its kernel
    (ev_abs) plus the magnitude of its closed-form term.  method: "lscv"
    (Eq. 10) or "scv" (the reading above).  A value much smaller than its
    scale is a difference of large terms, and its rounding error is bounded
    relative to the scale, not to the value."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    Hinv = np.linalg.inv(H)
    if method == "lscv":
        c0 = K0(H)
        sv = ev_abs(lscv_T_terms(H)) + 2.0 * c0 / n
        grad_terms = lambda a, b: lscv_grad_terms(H, a, b)
        closed = lambda a, b: 2.0 / n * _tie(a, b) * 0.5 * c0 * abs(Hinv[a, b])
    else:
        r0 = RK(H)
        sv = ev_abs(scv_terms(H, G)) + r0 / n
        grad_terms = lambda a, b: scv_grad_terms(H, G, a, b)
        closed = lambda a, b: _tie(a, b) * 0.5 * r0 * abs(Hinv[a, b]) / n
    sg = np.zeros((d, d))
    for a, b in vech_pairs(d):
        sg[a, b] = sg[b, a] = ev_abs(grad_terms(a, b)) + closed(a, b)
    return sv, sg


# ---------------------------------------------------------------------------
# psi_r (Eq. 13) and the eta functionals of Sec. 5 (Eqs. 29-32)

def psi_unique(ev, H, r):
    """{alpha: n^-2 sum sum d^alpha phi_H(X_i - X_j)} for |alpha| = r: the
    unique entries of psi_r of Eq. 13."""
    return {a: ev([(1.0, np.asarray(H, dtype=np.float64), a)])
            for a in multi_indices(np.asarray(H).shape[0], r)}


def psi_vector(ev, H, r):
    """psi_r(H) of Eq. 13 with K = Gaussian, as the length d^r vector in
    Kronecker order (Sec. 5: D^{(x)r}, vec stacking)."""
    d = np.asarray(H).shape[0]
    u = psi_unique(ev, H, r)
    return np.array([u[a] for a in kron_alphas(d, r)])


def eta02_terms(B, Sigma):
    """eta_{0,2}(x; B, Sigma) = (vec^T B)^{(x)2} D^{(x)4} phi_Sigma(x)
    (Eq. 30 with r = 0, s = 2): sum_{a,b,c,e} B_ab B_ce d_abce phi_Sigma,
    collected by multi-index."""
    B = np.asarray(B, dtype=np.float64)
    d = B.shape[0]
    w: dict = {}
    import itertools
    for a, b, c, e in itertools.product(range(d), repeat=4):
        al = _e(d, a, b, c, e)
        w[al] = w.get(al, 0.0) + B[a, b] * B[c, e]
    return [(wt, np.asarray(Sigma, dtype=np.float64), al) for al, wt in w.items() if wt != 0.0]


def eta_rs_terms(A, B, Sigma, r, s):
    """eta_{r,s}(x; A, B, Sigma) = {(vec^T A)^{(x)r} (x) (vec^T B)^{(x)s}}
    D^{(x)2r+2s} phi_Sigma(x) (Eq. 30): the Kronecker vector's entry at the
    index tuple (i_1, .., i_{2r+2s}) is prod_k A_{i_{2k-1} i_{2k}} (first r
    pairs) prod_k B_{..} (last s pairs), and the derivative entry is
    d_{i_1} .. d_{i_{2r+2s}} phi_Sigma; collected by multi-index."""
    import itertools
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    d = A.shape[0]
    w: dict = {}
    for idx in itertools.product(range(d), repeat=2 * (r + s)):
        c = 1.0
        for k in range(r):
            c *= A[idx[2 * k], idx[2 * k + 1]]
        for k in range(s):
            c *= B[idx[2 * r + 2 * k], idx[2 * r + 2 * k + 1]]
        if c == 0.0:
            continue
        al = [0] * d
        for i in idx:
            al[i] += 1
        al = tuple(al)
        w[al] = w.get(al, 0.0) + c
    return [(wt, np.asarray(Sigma, dtype=np.float64), al) for al, wt in w.items() if wt != 0.0]


def eta_r_terms(Sigma, r):
    """eta_r(x; Sigma) = (vec^T I)^{(x)r} D^{(x)2r} phi_Sigma = Laplacian^r
    phi_Sigma (Eq. 31) = sum_{|beta| = r} r!/beta! d^{2 beta} phi_Sigma."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    d = Sigma.shape[0]
    out = []
    for beta in multi_indices(d, r):
        coef = math.factorial(r) / math.prod(math.factorial(b) for b in beta)
        out.append((coef, Sigma, tuple(2 * b for b in beta)))
    return out


# ---------------------------------------------------------------------------
# Plug-in: named in Sec. 3, formulas deferred by Sec. 5 to an external source.
# Reading (AMISE with Gaussian kernel, mu_2(K) = 1):
#   PI(H) = n^-1 (4 pi)^{-d/2} |H|^{-1/2} + 1/4 (vec^T H)^{(x)2} psi_4(G)

def pi_from_psi4(psi4_kron, H, n: int, grad: bool = False):
    """PI(H) from psi_4(G) in Kronecker order (plug-in reading above; psi_4 of
    Eq. 13) and, with grad, its gradient in the tied convention."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    T = np.asarray(psi4_kron, dtype=np.float64).reshape((d, d, d, d))
    quad = float(np.einsum("ab,ce,abce->", H, H, T))
    r0 = RK(H)
    val = r0 / n + 0.25 * quad
    if not grad:
        return val
    Hinv = np.linalg.inv(H)
    half = 0.5 * np.einsum("ce,abce->ab", H, T)
    g = np.zeros((d, d))
    for a, b in vech_pairs(d):
        v = _tie(a, b) * (half[a, b] - 0.5 * r0 * Hinv[a, b] / n)
        g[a, b] = g[b, a] = v
    return val, g


def pi_eta(ev, H, G, n: int):
    """PI(H) through the per-H scalar kernel eta_{0,2}(x; H, G) (Eq. 29-30):
    one double sum instead of the d^4 psi_4 vector."""
    return RK(H) / n + 0.25 * ev(eta02_terms(H, G))


def lscv_r(ev, H, n: int, r: int, exact_loo: bool = False):
    """LSCV_r of Eq. 36 (exact_loo=False) or Eq. 35 (True), with eta_{r,0}
    = eta_r (Eq. 31, the I_d contraction).  Reading for the n ~ n-1 form: the
    added term is 2 n^-1 eta_r(0; H), which equals 2 n^-1 K_H(0) at r = 0."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    sgn = (-1.0) ** r
    from .gauss import kernel_eval
    e0 = float(kernel_eval(np.zeros(d), eta_r_terms(H, r)))
    if not exact_loo:
        terms = [(w, S, a) for w, S, a in eta_r_terms(2.0 * H, r)]
        terms += [(-2.0 * w, S, a) for w, S, a in eta_r_terms(H, r)]
        return sgn * (ev(terms) + 2.0 * e0 / n)
    A = ev(eta_r_terms(2.0 * H, r))
    B = ev(eta_r_terms(H, r))
    return sgn * (A - 2.0 / (n * (n - 1.0)) * (n * n * B - n * e0))
