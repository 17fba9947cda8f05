"""Seeded synthetic workloads (normal mixtures) shared by tests, bench and smoke.

This module only draws inputs: samples, grid ranges and candidate bandwidth
matrices.  It holds none of the method's arithmetic (no binning, no kernels,
no FFT, no objectives), so that the CUDA path and the CPU oracle receive
identical bytes without sharing code.

Recipe (all FP64, numpy default_rng(seed)):
  * labels  = rng.choice(K, n, p=w)
  * z       = rng.standard_normal((n, d))
  * X       = mu[label] + chol(Sigma[label]) z
  * random SPD Sigma = Q diag(lam) Q^T, Q from the QR factorisation of a
    standard normal matrix with the signs of R's diagonal folded into Q.
  * normal-scale bandwidth (a textbook rule of thumb, used as start point and
    as pilot placeholder): H_NS = (4/(d+2))^{2/(d+4)} n^{-2/(d+4)} S,
    S the sample covariance.
  * grid range: lo_k = min_i X_ik - 3 sqrt(H_kk), hi_k = max_i X_ik + 3 sqrt(H_kk).
  * candidate H around H_NS: H = R Q diag(exp(u)) Q^T R^T with H_NS = R R^T,
    u ~ U[log 1/4, log 4].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def random_rotation(rng, d):
    A = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def random_spd(rng, d, lam):
    Q = random_rotation(rng, d)
    return Q @ np.diag(np.asarray(lam, dtype=np.float64)) @ Q.T


def sample_mixture(rng, n, w, mus, sigmas):
    w = np.asarray(w, dtype=np.float64)
    K = len(w)
    d = len(mus[0])
    lab = rng.choice(K, n, p=w / w.sum())
    z = rng.standard_normal((n, d))
    X = np.empty((n, d))
    for k in range(K):
        m = lab == k
        C = np.linalg.cholesky(np.asarray(sigmas[k], dtype=np.float64))
        X[m] = np.asarray(mus[k], dtype=np.float64) + z[m] @ C.T
    return X


def normal_scale(X):
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    S = np.cov(X, rowvar=False).reshape(d, d)
    return (4.0 / (d + 2.0)) ** (2.0 / (d + 4.0)) * n ** (-2.0 / (d + 4.0)) * S


def grid_range(X, H, pad: float = 3.0):
    X = np.asarray(X, dtype=np.float64)
    s = pad * np.sqrt(np.diag(np.asarray(H, dtype=np.float64)))
    return X.min(axis=0) - s, X.max(axis=0) + s


def candidates_around(rng, H0, count, lo=0.25, hi=4.0):
    H0 = np.asarray(H0, dtype=np.float64)
    d = H0.shape[0]
    R = np.linalg.cholesky(H0)
    out = np.empty((count, d, d))
    for i in range(count):
        Q = random_rotation(rng, d)
        u = rng.uniform(np.log(lo), np.log(hi), size=d)
        A = Q @ np.diag(np.exp(u)) @ Q.T
        H = R @ A @ R.T
        out[i] = 0.5 * (H + H.T)
    return out


@dataclass
class Workload:
    name: str
    X: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    M: list
    H: np.ndarray                     # (nH, d, d) candidate bandwidths
    G: np.ndarray | None = None       # pilot for SCV / PI
    P: list | None = None             # fixed padded size, if the workload names one
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]


def plain_mixture_2d(n=1000, seed=0, M=100):
    """Equal mixture of N((-1,0), diag(.5,1)) and N((1,1), [[1,.7],[.7,1]]);
    the fixed H = [[.10,.05],[.05,.20]]; grid over the data range +/- 3
    bandwidths of that H."""
    rng = np.random.default_rng(seed)
    X = sample_mixture(rng, n, [0.5, 0.5], [[-1.0, 0.0], [1.0, 1.0]],
                       [np.diag([0.5, 1.0]), np.array([[1.0, 0.7], [0.7, 1.0]])])
    H = np.array([[0.10, 0.05], [0.05, 0.20]])
    lo, hi = grid_range(X, H)
    return Workload("plain-2d-n1000-M100", X, lo, hi, [M, M], H[None], G=None)


def random_mixture(rng, n, d, K, w=None, mean_box=2.0, eig=(0.1, 1.0), log_eig=False):
    if w is None:
        w = rng.dirichlet(np.ones(K))
    mus = rng.uniform(-mean_box, mean_box, size=(K, d))
    sig = []
    for _ in range(K):
        if log_eig:
            lam = np.exp(rng.uniform(np.log(eig[0]), np.log(eig[1]), size=d))
        else:
            lam = rng.uniform(eig[0], eig[1], size=d)
        sig.append(random_spd(rng, d, lam))
    return sample_mixture(rng, n, w, mus, sig)


def mixture_2d_large(n=100_000, seed=2, M=256, n_candidates=16):
    """3-component bivariate mixture, weights .5/.3/.2, means U[-2,2]^2,
    covariance eigenvalues U[0.1,1]; grid M^2 over the data range +/- 3
    normal-scale bandwidths."""
    rng = np.random.default_rng(seed)
    X = random_mixture(rng, n, 2, 3, w=np.array([0.5, 0.3, 0.2]))
    Hns = normal_scale(X)
    lo, hi = grid_range(X, Hns)
    Hc = candidates_around(np.random.default_rng(seed + 100), Hns, n_candidates)
    return Workload(f"mixture-2d-n{n}-M{M}", X, lo, hi, [M, M], Hc, G=Hns,
                    extra={"H_NS": Hns})


def mixture_3d(n=1_000_000, seed=3, M=128, n_candidates=256, seed_h=33):
    """4-component trivariate mixture, sd U[.3,1], correlations U[-.8,.8]
    (redrawn until SPD); 256 candidate H around H_NS."""
    rng = np.random.default_rng(seed)
    d, K = 3, 4
    mus = rng.uniform(-2.0, 2.0, size=(K, d))
    sig = []
    for _ in range(K):
        while True:
            sd = rng.uniform(0.3, 1.0, size=d)
            R = np.eye(d)
            for a in range(d):
                for b in range(a + 1, d):
                    R[a, b] = R[b, a] = rng.uniform(-0.8, 0.8)
            if np.linalg.eigvalsh(R)[0] > 1e-3:
                break
        sig.append(np.diag(sd) @ R @ np.diag(sd))
    X = sample_mixture(rng, n, np.full(K, 1.0 / K), mus, sig)
    Hns = normal_scale(X)
    lo, hi = grid_range(X, Hns)
    Hc = candidates_around(np.random.default_rng(seed_h), Hns, n_candidates)
    return Workload(f"mixture-3d-n{n}-M{M}", X, lo, hi, [M] * 3, Hc, G=Hns,
                    extra={"H_NS": Hns})


def batched_uneven(n_datasets=512, n_candidates=16, base_seed=4, n_range=(1e3, 1e5)):
    """Independent bivariate datasets: n log-uniform, 2-4 component mixtures
    with Dirichlet(1) weights; M = 64 (n < 5e3), 128 (n < 3e4), else 256."""
    out = []
    for i in range(n_datasets):
        rng = np.random.default_rng(base_seed + i)
        n = int(round(10 ** rng.uniform(np.log10(n_range[0]), np.log10(n_range[1]))))
        K = int(rng.integers(2, 5))
        X = random_mixture(rng, n, 2, K)
        M = 64 if n < 5000 else (128 if n < 30000 else 256)
        Hns = normal_scale(X)
        lo, hi = grid_range(X, Hns)
        Hc = candidates_around(rng, Hns, n_candidates)
        out.append(Workload(f"uneven-{i}", X, lo, hi, [M, M], Hc, G=Hns, extra={"H_NS": Hns}))
    return out


def mixture_4d(n=1_000_000, seed=5, M=48, P=96, n_candidates=8):
    """3-component 4-variate mixture, covariance eigenvalues log-U[1/20, 1]
    (condition number up to 20); grid 48^4 zero-padded to 96^4; pilot G =
    H_NS (placeholder)."""
    rng = np.random.default_rng(seed)
    X = random_mixture(rng, n, 4, 3, eig=(1.0 / 20.0, 1.0), log_eig=True)
    Hns = normal_scale(X)
    lo, hi = grid_range(X, Hns)
    Hc = candidates_around(np.random.default_rng(seed + 100), Hns, n_candidates)
    return Workload(f"mixture-4d-n{n}-M{M}-P{P}", X, lo, hi, [M] * 4, Hc, G=Hns, P=[P] * 4,
                    extra={"H_NS": Hns})


def paper_speed_shape(n=2000, M=100, seed=10):
    """The speed-study shape: N(0, I_2), H = n^{-1/3} I."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 2))
    H = n ** (-1.0 / 3.0) * np.eye(2)
    lo, hi = grid_range(X, H)
    return Workload(f"normal-2d-n{n}-M{M}", X, lo, hi, [M, M], H[None], G=H)


def small_case(n=200, d=2, M=24, seed=7, n_candidates=3):
    """A small mixture for quick parity checks."""
    rng = np.random.default_rng(seed)
    X = random_mixture(rng, n, d, 2)
    Hns = normal_scale(X)
    lo, hi = grid_range(X, Hns)
    Hc = candidates_around(np.random.default_rng(seed + 1), Hns, n_candidates)
    Ms = [int(m) for m in M] if hasattr(M, "__len__") else [int(M)] * d
    return Workload(f"small-{d}d-n{n}-M{'x'.join(map(str, Ms))}", X, lo, hi, Ms, Hc, G=Hns,
                    extra={"H_NS": Hns})
