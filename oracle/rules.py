"""Grid and padding rules of Sec. 4 (oracle, FP64, host arithmetic).

  bin_width    Eq. 16: delta_k = (g_{kM_k} - g_{k1}) / (M_k - 1).
  support_L    Eq. 26: L_k = min(M_k - 1, ceil(tau sqrt(lambda) / delta_k)),
               lambda the largest eigenvalue of the basis matrix (H in the
               paper; Sec. 4 suggests tau about 3.7).
  P_paper      Eq. 27: P_k = 2^ceil(log2(M_k + 2 L_k - 1)).
  P_paper_full Eq. 21: P_k = 2^ceil(log2(3 M_k - 1)).
  P_minimal    reading of the zero-padding layout of Eqs. 19-20: with the
               counts at offset L_k and lags -L_k..L_k, a circular
               convolution of length P_k reproduces every needed output of
               the linear one iff P_k >= M_k + L_k; the smallest
               2^a 3^b 5^c at or above that bound.

Pinned in tests by the paper's Tables 2 and 3 (Table 2's P values follow
from Table 3's L values through Eq. 27; Table 3's rows fit one constant
tau sqrt(lambda)/range per axis through Eqs. 16 and 26).
"""
from __future__ import annotations

import math

import numpy as np


def bin_width(lo, hi, M):
    """Eq. 16, elementwise over axes."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    M = np.asarray(M, dtype=np.int64)
    return (hi - lo) / (M - 1).astype(np.float64)


def lambda_max(S) -> float:
    """Largest eigenvalue of a symmetric matrix (LAPACK via numpy): the
    lambda of Eq. 26."""
    return float(np.linalg.eigvalsh(np.asarray(S, dtype=np.float64))[-1])


def support_L(lam: float, delta, M, tau: float = 3.7):
    """Eq. 26, one L_k per axis."""
    out = []
    for dk, Mk in zip(np.asarray(delta, dtype=np.float64), np.asarray(M, dtype=np.int64)):
        v = tau * math.sqrt(abs(lam)) / float(dk)
        out.append(int(min(int(Mk) - 1, math.ceil(v))))
    return out


def _next_pow2(x: int) -> int:
    """2^ceil(log2 x), the rounding of Eqs. 21 and 27."""
    p = 1
    while p < x:
        p *= 2
    return p


def P_paper(M, L):
    """Eq. 27."""
    return [_next_pow2(int(m) + 2 * int(l) - 1) for m, l in zip(M, L)]


def P_paper_full(M):
    """Eq. 21 (no truncation, L_k = M_k - 1 layout)."""
    return [_next_pow2(3 * int(m) - 1) for m in M]


def _is_smooth(x: int) -> bool:
    """x = 2^a 3^b 5^c: the lengths P_minimal allows (a reading of the
    zero-padding layout of Eqs. 19-20)."""
    for p in (2, 3, 5):
        while x % p == 0:
            x //= p
    return x == 1


def P_minimal(M, L):
    """Smallest 2^a 3^b 5^c >= M_k + L_k on each axis: the least padded size
    for which the layout of Eqs. 19-20 has no wrapped term at the outputs
    Eq. 23 extracts."""
    out = []
    for m, l in zip(M, L):
        x = int(m) + int(l)
        while not _is_smooth(x):
            x += 1
        out.append(x)
    return out
