"""Planted mistakes in the oracle must fail its pins (CPU only).

Each mutant below replaces one oracle function with a copy that carries one
plausible mistake: a dropped term or factor, a flipped sign, a wrong index,
a swapped operand or a wrong constant.  The whole battery of oracle pins
(every test in test_oracle_*.py) then runs against the mutated oracle, and
at least one pin must fail on a wrong value (an AssertionError, or the
oracle's OutsideGrid for a sample on its grid).  A mutant
that no pin catches marks a part of the oracle whose pins only restate it.

The mistakes are planted in this process only, with monkeypatch, and only in
the oracle; nothing here touches the CUDA library or a GPU."""
import importlib
import itertools
import math

import numpy as np
import pytest

from oracle import binning, functionals as F, gauss, kde, rules, selectors as S

PIN_MODULES = ("test_oracle_rules", "test_oracle_gauss", "test_oracle_functionals", "test_oracle_kde")
# the pins that take a second or more run last, so most mutants stop early
SLOW = ("symbolic", "normal_population", "binning_converges", "iterated_laplacian")


def _battery():
    pins = []
    for modname in PIN_MODULES:
        mod = importlib.import_module(modname)
        for name, fn in vars(mod).items():
            if not name.startswith("test_") or not callable(fn):
                continue
            marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
            if not marks:
                pins.append((f"{modname}::{name}", fn, {}))
                continue
            names = [a.strip() for a in marks[0].args[0].split(",")]
            for v in marks[0].args[1]:
                v = tuple(v) if len(names) > 1 else (v,)
                pins.append((f"{modname}::{name}{list(v)}", fn, dict(zip(names, v))))
    pins.sort(key=lambda p: any(s in p[0] for s in SLOW))
    return pins


def _first_failing_pin():
    """Runs the pins in order; returns the id of the first one that fails on a
    value (or on the oracle refusing a sample that lies on its grid), or
    None.  A pin that raises anything else is reported as such, so that a
    mutant which merely breaks the oracle's structure does not pass for one
    the pins catch."""
    for pid, fn, kw in _battery():
        try:
            fn(**kw)
        except (AssertionError, binning.OutsideGrid):
            return pid
        except pytest.skip.Exception:
            continue
        except Exception as e:  # noqa: BLE001 - reported, not swallowed
            raise RuntimeError(f"pin {pid} raised {type(e).__name__}: {e}") from e
    return None


# originals that some mutants wrap
_ORIG = {"eta_rs_terms": S.eta_rs_terms, "lscv_r": S.lscv_r, "kde_grid": kde.kde_grid,
         "pairings_value_at_zero": gauss.pairings_value_at_zero, "lscv_grad_terms": S.lscv_grad_terms}


def _patch(mp, fn, *targets):
    """Installs fn under the same name in every module that holds the
    original (a `from .x import f` in another oracle module keeps its own
    reference)."""
    for mod, name in targets:
        mp.setattr(mod, name, fn)


# ---------------------------------------------------------------- gauss

def _he_table(sign=-1.0, mult="beta"):
    """The Hermite recurrence of oracle.gauss with one of its pieces changed:
    sign of the contraction term, or its multiplicity (beta_j, alpha_j or 1)."""
    def table(z, Lam, R):
        d = Lam.shape[0]
        He = {tuple([0] * d): np.ones(z.shape[:-1])}
        for r in range(1, R + 1):
            for alpha in gauss.multi_indices(d, r):
                i = next(k for k in range(d) if alpha[k] > 0)
                beta = list(alpha)
                beta[i] -= 1
                beta = tuple(beta)
                val = z[..., i] * He[beta]
                for j in range(d):
                    if beta[j] > 0:
                        bj = list(beta)
                        bj[j] -= 1
                        m = {"beta": beta[j], "alpha": alpha[j], "one": 1.0}[mult]
                        val = val + sign * m * Lam[i, j] * He[tuple(bj)]
                He[alpha] = val
        return He
    return table


def _derivs(signed=True, whiten=True):
    def derivs(x, Sigma, alphas):
        x = np.asarray(x, dtype=np.float64)
        Sigma = np.asarray(Sigma, dtype=np.float64)
        Lam = np.linalg.inv(Sigma)
        z = np.einsum("ij,...j->...i", Lam, x) if whiten else x
        phi = gauss.gauss_density(x, Sigma)
        alphas = [tuple(a) for a in alphas]
        He = gauss.hermite_table(z, Lam, max((sum(a) for a in alphas), default=0))
        return {a: ((-1.0) ** sum(a) if signed else 1.0) * He[a] * phi for a in alphas}
    return derivs


def _density(expo=0.5, norm_pow=0.5):
    def density(x, Sigma):
        x = np.asarray(x, dtype=np.float64)
        Sigma = np.asarray(Sigma, dtype=np.float64)
        d = Sigma.shape[0]
        q = np.einsum("...i,ij,...j->...", x, np.linalg.inv(Sigma), x)
        return (2.0 * math.pi) ** (-d * norm_pow) / math.sqrt(np.linalg.det(Sigma)) * np.exp(-expo * q)
    return density


def _kernel_eval_unweighted(x, terms):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[:-1])
    for w, Sg, a in terms:
        out = out + gauss.gauss_derivs(x, Sg, [a])[tuple(a)]
    return out


def _pairings_unsigned(Sigma, alpha):
    r = sum(alpha)
    return (-1.0) ** (r // 2) * _ORIG["pairings_value_at_zero"](Sigma, alpha)


def _density_targets():
    return ((gauss, "gauss_density"), (kde, "gauss_density"))


def _kernel_targets():
    return ((gauss, "kernel_eval"), (F, "kernel_eval"))


# ---------------------------------------------------------------- binning and rules

def _bin_linear(swap=False, axis_flip=False):
    def bin_linear(X, lo, hi, M, policy="error"):
        M = [int(m) for m in M]
        t, _ = binning._coords(X, lo, hi, M)
        ok = binning._inside(X, lo, hi, policy)
        t = t[ok]
        l = np.floor(t)
        Mm1 = np.asarray(M, dtype=np.float64) - 1.0
        l = np.where(l >= Mm1, Mm1 - 1.0, l)
        f = t - l
        l = l.astype(np.int64)
        d = len(M)
        c = np.zeros(M)
        for b in itertools.product((0, 1), repeat=d):
            w = np.ones(t.shape[0])
            for k in range(d):
                take_f = (not b[k]) if swap else b[k]
                w = w * (f[:, k] if take_f else (1.0 - f[:, k]))
            idx = tuple(l[:, k] + b[d - 1 - k if axis_flip else k] for k in range(d))
            np.add.at(c, idx, w)
        return c
    return bin_linear


def _inside_lower_open(X, lo, hi, policy):
    """lo < x instead of lo <= x: a point on the lower edge counts as outside."""
    X = np.asarray(X, dtype=np.float64)
    ok = np.all((X > np.asarray(lo, dtype=np.float64)) & (X <= np.asarray(hi, dtype=np.float64)), axis=1)
    if not np.all(ok) and policy == "error":
        raise binning.OutsideGrid("outside")
    return ok


def _bin_simple_floor(X, lo, hi, M, policy="error"):
    M = [int(m) for m in M]
    t, _ = binning._coords(X, lo, hi, M)
    t = t[binning._inside(X, lo, hi, policy)]
    l = np.floor(t).astype(np.int64)
    c = np.zeros(M, dtype=np.int64)
    np.add.at(c, tuple(l[:, k] for k in range(len(M))), 1)
    return c


def _bin_width_over_M(lo, hi, M):
    return (np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)) / \
        np.asarray(M, dtype=np.float64)


def _support_L(rounding=math.ceil, root=True):
    def support_L(lam, delta, M, tau=3.7):
        out = []
        for dk, Mk in zip(np.asarray(delta, dtype=np.float64), np.asarray(M, dtype=np.int64)):
            s = math.sqrt(abs(lam)) if root else abs(lam)
            out.append(int(min(int(Mk) - 1, rounding(tau * s / float(dk)))))
        return out
    return support_L


def _lambda_min(S_):
    return float(np.linalg.eigvalsh(np.asarray(S_, dtype=np.float64))[0])


def _next_pow2_strict(x):
    p = 1
    while p <= x:
        p *= 2
    return p


def _is_7_smooth(x):
    for p in (2, 3, 5, 7):
        while x % p == 0:
            x //= p
    return x == 1


def _coords_unclamped(X, lo, hi, M):
    X = np.asarray(X, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    delta = rules.bin_width(lo, hi, M)
    return (X - lo) / delta, delta


def _P_paper_no_minus_one(M, L):
    return [rules._next_pow2(int(m) + 2 * int(l)) for m, l in zip(M, L)]


def _P_paper_full_3M(M):
    return [rules._next_pow2(3 * int(m)) for m in M]


def _P_minimal_short(M, L):
    out = []
    for m, l in zip(M, L):
        x = int(m) + int(l) - 1
        while not rules._is_smooth(x):
            x += 1
        out.append(x)
    return out


# ---------------------------------------------------------------- functionals

def _direct_sum_offdiag(X, terms, block=256):
    """The double sum over i != j only (a U-statistic, not Eq. 12's V-statistic)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    diff = X[:, None, :] - X[None, :, :]
    v = F.kernel_eval(diff, terms)
    return float(np.sum(v) - np.trace(v)) / float(n) ** 2


def _direct_sum_short_blocks(X, terms, block=256):
    """Block rows [s, s + block - 1): the last row of every block left out."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    parts = []
    for s0 in range(0, n, block):
        diff = X[s0:s0 + block - 1, None, :] - X[None, :, :]
        parts.append(float(np.sum(F.kernel_eval(diff, terms))))
    return math.fsum(parts) / float(n) ** 2


def _overlap_self(c, j):
    sl = []
    for k, jk in enumerate(j):
        Mk = c.shape[k]
        if abs(jk) >= Mk:
            return 0.0
        sl.append(slice(abs(jk), Mk))
    return float(np.sum(c[tuple(sl)] * c[tuple(sl)]))


def _lag_kernel_axes_swapped(terms, delta, L):
    delta = np.asarray(delta, dtype=np.float64)[::-1]
    axes = [delta[k] * np.arange(-L[k], L[k] + 1, dtype=np.float64) for k in range(len(L))]
    x = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    return F.kernel_eval(x, terms)


def _lag_kernel_uncentred(terms, delta, L):
    delta = np.asarray(delta, dtype=np.float64)
    axes = [delta[k] * np.arange(0, 2 * L[k] + 1, dtype=np.float64) for k in range(len(L))]
    x = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    return F.kernel_eval(x, terms)


def _binned_direct(norm_pow=2, inclusive=True):
    def binned_direct(c, n, terms, delta, L):
        c = np.asarray(c, dtype=np.float64)
        k = F.lag_kernel(terms, delta, L)
        parts = []
        for j in itertools.product(*[range(-l, l + 1 if inclusive else l) for l in L]):
            parts.append(k[tuple(jj + l for jj, l in zip(j, L))] * F._overlap(c, j))
        return math.fsum(parts) / float(n) ** norm_pow
    return binned_direct


def _binned_fft(count_offset=True, extract=2):
    def binned_fft(c, n, terms, delta, L, P):
        c = np.asarray(c, dtype=np.float64)
        d, M = c.ndim, c.shape
        if any(P[k] < M[k] + L[k] for k in range(d)):
            raise ValueError("P_k must be at least M_k + L_k")
        c_zp = np.zeros(P)
        c_zp[tuple(slice(L[k] if count_offset else 0, (L[k] if count_offset else 0) + M[k])
                   for k in range(d))] = c
        k_zp = np.zeros(P)
        k_zp[tuple(slice(0, 2 * L[k] + 1) for k in range(d))] = F.lag_kernel(terms, delta, L)
        s = np.fft.ifftn(np.fft.fftn(c_zp) * np.fft.fftn(k_zp)).real
        conv = s[np.ix_(*[(extract * L[k] + np.arange(M[k])) % P[k] for k in range(d)])]
        return float(np.sum(c * conv)) / float(n) ** 2
    return binned_fft


def _autocorr_axes_shifted(c, A):
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    shape = tuple(2 * A[k] + 1 for k in range(d - 1, 0, -1)) + (A[0] + 1,)
    out = np.zeros(shape)
    for idx in np.ndindex(*shape):
        j = [idx[-1]] + [idx[k - 1] - A[k] for k in range(1, d)]
        out[idx] = F._overlap(c, [-x for x in j])
    return out


def _half_box_weights(pos=2.0, first=True):
    def weights(A):
        d = len(A)
        shape = tuple(2 * A[k] + 1 for k in range(d - 1, 0, -1)) + (A[0] + 1,)
        w = np.zeros(shape)
        for idx in np.ndindex(*shape):
            j = [idx[-1]] + [idx[d - 1 - k] - A[k] for k in range(1, d)]
            nz = [x for x in j if x != 0]
            if not nz:
                w[idx] = 1.0
            else:
                w[idx] = pos if (nz[0] if first else nz[-1]) > 0 else 0.0
        return w
    return weights


# ---------------------------------------------------------------- selectors

def _vech_pairs_offdiag(d):
    return [(a, b) for a in range(d) for b in range(a + 1, d)] + [(a, a) for a in range(d)][:-1]


def _tie_swapped(a, b):
    return 2.0 if a == b else 1.0


def _psi_unique_2H(ev, H, r):
    return {a: ev([(1.0, 2.0 * np.asarray(H, dtype=np.float64), a)])
            for a in gauss.multi_indices(np.asarray(H).shape[0], r)}


def _T_terms(conv_scale=2.0, cross=-2.0):
    def terms(H):
        H = np.asarray(H, dtype=np.float64)
        z = (0,) * H.shape[0]
        return [(1.0, conv_scale * H, z), (cross, H, z)]
    return terms


def _lscv_grad_untied(H, a, b, loo_factor=1.0):
    H = np.asarray(H, dtype=np.float64)
    al = S._e(H.shape[0], a, b)
    return [(1.0, 2.0 * H, al), (-loo_factor, H, al)]


def _lscv_grad_no_loo(H, a, b, loo_factor=1.0):
    return _ORIG["lscv_grad_terms"](H, a, b, 1.0)


def _lscv_loo_const(k0_over):
    """Eq. 8 with the K_H(0) constant 2/k0_over(n) in place of 2/(n-1)."""
    def lscv(ev, H, n, exact_loo=False, grad=False):
        H = np.asarray(H, dtype=np.float64)
        z = S._e(H.shape[0])
        k0 = S.K0(H)
        if not exact_loo:
            val = ev(S.lscv_T_terms(H)) + 2.0 * k0 / n
        else:
            A = ev([(1.0, 2.0 * H, z)])
            B = ev([(1.0, H, z)])
            val = A - 2.0 * n / (n - 1.0) * B + 2.0 / k0_over(n) * k0
        assert not grad
        return val
    return lscv


def _const_pi(base):
    def const(H):
        d = np.asarray(H).shape[0]
        return (base * math.pi) ** (-d / 2.0) / math.sqrt(np.linalg.det(np.asarray(H, dtype=np.float64)))
    return const


def _scv_terms(mid=-2.0, last_G=2.0):
    def terms(H, G):
        H = np.asarray(H, dtype=np.float64)
        G = np.asarray(G, dtype=np.float64)
        z = S._e(H.shape[0])
        return [(1.0, 2.0 * H + 2.0 * G, z), (mid, H + 2.0 * G, z), (1.0, last_G * G, z)]
    return terms


def _scv_grad_sign(H, G, a, b):
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    s = S._tie(a, b)
    al = S._e(H.shape[0], a, b)
    return [(s, 2.0 * H + 2.0 * G, al), (s, H + 2.0 * G, al)]


def _scv_grad_rk_sign(ev, H, G, n, grad=False):
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    r0 = S.RK(H)
    val = r0 / n + ev(S.scv_terms(H, G))
    if not grad:
        return val
    Hinv = np.linalg.inv(H)
    g = np.zeros((d, d))
    for a, b in S.vech_pairs(d):
        g[a, b] = g[b, a] = ev(S.scv_grad_terms(H, G, a, b)) + S._tie(a, b) * (0.5 * r0 * Hinv[a, b]) / n
    return val, g


def _pi_eta_half(ev, H, G, n):
    return S.RK(H) / n + 0.5 * ev(S.eta02_terms(H, G))


def _scv_pilot_at_G_terms(H, G):
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    z = S._e(H.shape[0])
    return [(1.0, 2.0 * H + G, z), (-2.0, H + G, z), (1.0, G, z)]


def _scv_pilot_at_G_grad(H, G, a, b):
    H = np.asarray(H, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    s = S._tie(a, b)
    al = S._e(H.shape[0], a, b)
    return [(s, 2.0 * H + G, al), (-s, H + G, al)]


def _pi_from_psi4(quarter=0.25, half=0.5):
    def pi(psi4_kron, H, n, grad=False):
        H = np.asarray(H, dtype=np.float64)
        d = H.shape[0]
        T = np.asarray(psi4_kron, dtype=np.float64).reshape((d, d, d, d))
        r0 = S.RK(H)
        val = r0 / n + quarter * float(np.einsum("ab,ce,abce->", H, H, T))
        if not grad:
            return val
        Hinv = np.linalg.inv(H)
        hh = half * np.einsum("ce,abce->ab", H, T)
        g = np.zeros((d, d))
        for a, b in S.vech_pairs(d):
            g[a, b] = g[b, a] = S._tie(a, b) * (hh[a, b] - 0.5 * r0 * Hinv[a, b] / n)
        return val, g
    return pi


def _eta02_index_typo(B, Sigma):
    B = np.asarray(B, dtype=np.float64)
    d = B.shape[0]
    w = {}
    for a, b, c, e in itertools.product(range(d), repeat=4):
        al = S._e(d, a, b, c, e)
        w[al] = w.get(al, 0.0) + B[a, b] * B[a, e]
    return [(wt, np.asarray(Sigma, dtype=np.float64), al) for al, wt in w.items() if wt != 0.0]


def _eta_r_no_multinomial(Sigma, r):
    Sigma = np.asarray(Sigma, dtype=np.float64)
    return [(1.0, Sigma, tuple(2 * b for b in beta)) for beta in gauss.multi_indices(Sigma.shape[0], r)]


def _eta_rs_A_only(A, B, Sigma, r, s):
    return _ORIG["eta_rs_terms"](A, A, Sigma, r, s)


def _lscv_r_unsigned(ev, H, n, r, exact_loo=False):
    return (-1.0) ** r * _ORIG["lscv_r"](ev, H, n, r, exact_loo)


# ---------------------------------------------------------------- kde

def _kde_grid_n2(c, n, H, delta, L):
    return _ORIG["kde_grid"](c, n, H, delta, L) / float(n)


def _kde_grid_short_stencil(c, n, H, delta, L):
    c = np.asarray(c, dtype=np.float64)
    M = c.shape
    out = np.zeros(M)
    for l in itertools.product(*[range(-Lk + 1, Lk) for Lk in L]):
        x = np.asarray(delta, dtype=np.float64) * np.asarray(l, dtype=np.float64)
        k = float(gauss.gauss_density(x[None, :], np.asarray(H, dtype=np.float64))[0])
        dst = tuple(slice(max(0, lk), M[i] + min(0, lk)) for i, lk in enumerate(l))
        src = tuple(slice(max(0, -lk), M[i] - max(0, lk)) for i, lk in enumerate(l))
        out[dst] += k * c[src]
    return out / float(n)


def _mixture_sq_one_cov(w, mu, S_):
    tot = 0.0
    for a in range(len(w)):
        for b in range(len(w)):
            x = (np.asarray(mu[a]) - np.asarray(mu[b]))[None, :]
            tot += w[a] * w[b] * float(gauss.gauss_density(x, np.asarray(S_[a]))[0])
    return tot


def _ise_binned(cross_w=2.0, smooth_H=True):
    def ise(c, n, lo, delta, H, w, mu, S_, L2):
        c = np.asarray(c, dtype=np.float64)
        H = np.asarray(H, dtype=np.float64)
        d = c.ndim
        ff = F.binned_direct(c, n, [(1.0, 2.0 * H, (0,) * d)], delta, L2)
        grids = np.meshgrid(*[lo[k] + delta[k] * np.arange(c.shape[k]) for k in range(d)], indexing="ij")
        xg = np.stack([g.ravel() for g in grids], axis=1)
        fm = np.zeros(xg.shape[0])
        for wm, m, Sm in zip(w, mu, S_):
            fm += wm * gauss.gauss_density(xg - np.asarray(m)[None, :], (H if smooth_H else 0.0) + np.asarray(Sm))
        return ff - cross_w * float(np.sum(c.ravel() * fm)) / float(n) + kde.mixture_sq_integral(w, mu, S_)
    return ise


def _ise_exact(pair_scale=2.0, cross_H=1.0):
    def ise(X, H, w, mu, S_):
        return _ise_exact_scaled(X, H, w, mu, S_, pair_scale, cross_H)
    return ise


def _ise_exact_scaled(X, H, w, mu, S_, pair_scale, cross_H):
    X = np.asarray(X, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    n = X.shape[0]
    a = sum(float(np.sum(gauss.gauss_density(X - X[i][None, :], pair_scale * H))) for i in range(n))
    b = sum(wm * float(np.sum(gauss.gauss_density(X - np.asarray(m)[None, :], cross_H * H + np.asarray(Sm))))
            for wm, m, Sm in zip(w, mu, S_))
    return a / n ** 2 - 2.0 * b / n + kde.mixture_sq_integral(w, mu, S_)


# ---------------------------------------------------------------- the mutants

def _autocorr_fft(pad=0, power=2):
    """oracle.functionals.autocorr_fft with the padding 2 M_k - pad or the
    spectrum's modulus to another power."""
    def ac(c):
        import scipy.fft as sf
        c = np.asarray(c, dtype=np.float64)
        P = [2 * m - pad for m in c.shape]
        czp = np.zeros(P)
        czp[tuple(slice(0, m) for m in c.shape)] = c
        return sf.irfftn(np.abs(sf.rfftn(czp)) ** power, s=P)
    return ac


def _lag_sums(shrink=0, flip0=False, norm_pow=2, absolute=True):
    """oracle.functionals.lag_sums with one change: the lag box one short on
    every axis, the first axis' lag read with the wrong sign, n^-1 for n^-2,
    or the magnitude summed without |k|."""
    def ls(a, n, terms, delta, L):
        Ls = [max(0, l - shrink) for l in L]
        k = F.lag_kernel(terms, delta, Ls)
        ax = [np.arange(-Ls[i], Ls[i] + 1) for i in range(len(Ls))]
        if flip0:
            ax[0] = -ax[0][::-1] if len(ax) == 1 else ax[0][::-1]
        idx = np.ix_(*[ax[i] % a.shape[i] for i in range(len(Ls))])
        aj = a[idx]
        nn = float(n) ** norm_pow
        mag = np.abs(k) if absolute else k
        return float(np.sum(k * aj)) / nn, float(np.sum(mag * aj)) / nn
    return ls


MUTANTS = {
    # gauss: Hermite partials and the density (Sec. 5)
    "He recurrence: contraction term added": lambda mp: _patch(mp, _he_table(sign=+1.0), (gauss, "hermite_table")),
    "He recurrence: multiplicity dropped": lambda mp: _patch(mp, _he_table(mult="one"), (gauss, "hermite_table")),
    "He recurrence: alpha_j for beta_j": lambda mp: _patch(mp, _he_table(mult="alpha"), (gauss, "hermite_table")),
    "partials: sign (-1)^|alpha| dropped": lambda mp: _patch(mp, _derivs(signed=False), (gauss, "gauss_derivs")),
    "partials: Hermite argument x, not Sigma^-1 x": lambda mp: _patch(mp, _derivs(whiten=False), (gauss, "gauss_derivs")),
    "density: exponent without 1/2": lambda mp: _patch(mp, _density(expo=1.0), *_density_targets()),
    "density: (2 pi)^-d normalisation": lambda mp: _patch(mp, _density(norm_pow=1.0), *_density_targets()),
    "kernel: term weights dropped": lambda mp: _patch(mp, _kernel_eval_unweighted, *_kernel_targets()),
    "Isserlis: sign (-1)^(r/2) dropped": lambda mp: _patch(mp, _pairings_unsigned, (gauss, "pairings_value_at_zero")),
    # binning (Sec. 4) and the grid rules (Eqs. 16, 21, 26, 27)
    "linear binning: f and 1 - f swapped": lambda mp: _patch(mp, _bin_linear(swap=True), (binning, "bin_linear")),
    "linear binning: corner offsets on the reversed axis": lambda mp: _patch(mp, _bin_linear(axis_flip=True), (binning, "bin_linear")),
    "grid: a point on the lower edge is outside": lambda mp: _patch(mp, _inside_lower_open, (binning, "_inside")),
    "simple binning: floor, not nearest": lambda mp: _patch(mp, _bin_simple_floor, (binning, "bin_simple")),
    "Eq. 16: range / M": lambda mp: _patch(mp, _bin_width_over_M, (rules, "bin_width"), (binning, "bin_width")),
    "Eq. 26: floor for ceil": lambda mp: _patch(mp, _support_L(rounding=math.floor), (rules, "support_L")),
    "Eq. 26: lambda for sqrt(lambda)": lambda mp: _patch(mp, _support_L(root=False), (rules, "support_L")),
    "Eq. 26: smallest eigenvalue for the largest": lambda mp: _patch(mp, _lambda_min, (rules, "lambda_max")),
    "powers of two: next strictly above": lambda mp: _patch(mp, _next_pow2_strict, (rules, "_next_pow2")),
    "minimal P: 7 counted as a small prime": lambda mp: _patch(mp, _is_7_smooth, (rules, "_is_smooth")),
    "binning: upper-edge clamp left out": lambda mp: _patch(mp, _coords_unclamped, (binning, "_coords")),
    "Eq. 27: M + 2L for M + 2L - 1": lambda mp: _patch(mp, _P_paper_no_minus_one, (rules, "P_paper")),
    "Eq. 21: 3M for 3M - 1": lambda mp: _patch(mp, _P_paper_full_3M, (rules, "P_paper_full")),
    "minimal P: M + L - 1": lambda mp: _patch(mp, _P_minimal_short, (rules, "P_minimal")),
    # binned double sums (Eqs. 18-25) and the lag-domain form
    "direct sum: last row of each block left out": lambda mp: _patch(mp, _direct_sum_short_blocks, (F, "direct_sum")),
    "Eq. 12: i = j terms left out": lambda mp: _patch(mp, _direct_sum_offdiag, (F, "direct_sum")),
    "Eq. 25: a slice times itself": lambda mp: _patch(mp, _overlap_self, (F, "_overlap")),
    "Eq. 18: lag box not centred on 0": lambda mp: _patch(mp, _lag_kernel_uncentred, (F, "lag_kernel")),
    "Eq. 18: axis spacings swapped": lambda mp: _patch(mp, _lag_kernel_axes_swapped, (F, "lag_kernel")),
    "Eq. 25: n^-1 for n^-2": lambda mp: _patch(mp, _binned_direct(norm_pow=1), (F, "binned_direct")),
    "Eq. 25: lag +L_k left out": lambda mp: _patch(mp, _binned_direct(inclusive=False), (F, "binned_direct")),
    "Eq. 23: extraction at L": lambda mp: _patch(mp, _binned_fft(extract=1), (F, "binned_fft")),
    "Eq. 19: counts at offset 0": lambda mp: _patch(mp, _binned_fft(count_offset=False), (F, "binned_fft")),
    "autocorrelation: lag axes mismatched": lambda mp: _patch(mp, _autocorr_axes_shifted, (F, "autocorr")),
    "half box: weight 1 on the positive half": lambda mp: _patch(mp, _half_box_weights(pos=1.0), (F, "half_box_weights")),
    "half box: sign of the last nonzero lag": lambda mp: _patch(mp, _half_box_weights(first=False), (F, "half_box_weights")),
    "FFT autocorrelation: padding 2M - 2 (the largest lags wrap)": lambda mp: _patch(mp, _autocorr_fft(pad=2), (F, "autocorr_fft")),
    "FFT autocorrelation: |C| for |C|^2": lambda mp: _patch(mp, _autocorr_fft(power=1), (F, "autocorr_fft")),
    "lag sums: box one short on every axis": lambda mp: _patch(mp, _lag_sums(shrink=1), (F, "lag_sums")),
    "lag sums: first-axis lag read with the wrong sign": lambda mp: _patch(mp, _lag_sums(flip0=True), (F, "lag_sums")),
    "lag sums: n^-1 for n^-2": lambda mp: _patch(mp, _lag_sums(norm_pow=1), (F, "lag_sums")),
    "lag sums: magnitude without |k|": lambda mp: _patch(mp, _lag_sums(absolute=False), (F, "lag_sums")),
    # selectors (Eqs. 8, 10-11, 29-36; SCV and PI readings)
    "gradients: one diagonal entry left out": lambda mp: _patch(mp, _vech_pairs_offdiag, (S, "vech_pairs")),
    "gradients: factor 2 on the diagonal, not off it": lambda mp: _patch(mp, _tie_swapped, (S, "_tie")),
    "Eq. 13: psi at 2H": lambda mp: _patch(mp, _psi_unique_2H, (S, "psi_unique")),
    "Eq. 11: K_H * K_H as phi_H": lambda mp: _patch(mp, _T_terms(conv_scale=1.0), (S, "lscv_T_terms")),
    "Eq. 11: factor 2 on K_H dropped": lambda mp: _patch(mp, _T_terms(cross=-1.0), (S, "lscv_T_terms")),
    "LSCV gradient: off-diagonal factor 2 dropped": lambda mp: _patch(mp, _lscv_grad_untied, (S, "lscv_grad_terms")),
    "Eq. 8 gradient: n/(n - 1) dropped": lambda mp: _patch(mp, _lscv_grad_no_loo, (S, "lscv_grad_terms")),
    "Eq. 8: 2/n for 2/(n - 1) on K_H(0)": lambda mp: _patch(mp, _lscv_loo_const(lambda n: float(n)), (S, "lscv")),
    "K_H(0) with (4 pi)^-d/2": lambda mp: _patch(mp, _const_pi(4.0), (S, "K0")),
    "SCV: middle weight -1": lambda mp: _patch(mp, _scv_terms(mid=-1.0), (S, "scv_terms")),
    "SCV: phi_G for phi_2G": lambda mp: _patch(mp, _scv_terms(last_G=1.0), (S, "scv_terms")),
    "SCV gradient: middle sign flipped": lambda mp: _patch(mp, _scv_grad_sign, (S, "scv_grad_terms")),
    "SCV gradient: sign of the R(K) term": lambda mp: _patch(mp, _scv_grad_rk_sign, (S, "scv")),
    "PI by eta_02: 1/2 for 1/4": lambda mp: _patch(mp, _pi_eta_half, (S, "pi_eta")),
    "R(K) with (2 pi)^-d/2": lambda mp: _patch(mp, _const_pi(2.0), (S, "RK")),
    "PI: 1/2 for 1/4": lambda mp: _patch(mp, _pi_from_psi4(quarter=0.5), (S, "pi_from_psi4")),
    "PI gradient: factor 1/2 dropped": lambda mp: _patch(mp, _pi_from_psi4(half=1.0), (S, "pi_from_psi4")),
    # consistent misreadings: value and gradient (or both routes) carry the same slip
    "SCV: pilot convolutions at G, value and gradient together": lambda mp: (
        _patch(mp, _scv_pilot_at_G_terms, (S, "scv_terms")),
        _patch(mp, _scv_pilot_at_G_grad, (S, "scv_grad_terms"))),
    "PI: 1/2 for 1/4 on both routes (value and gradient)": lambda mp: (
        _patch(mp, _pi_from_psi4(quarter=0.5, half=1.0), (S, "pi_from_psi4")),
        _patch(mp, _pi_eta_half, (S, "pi_eta"))),
    "Eq. 30: B_ab B_ae for B_ab B_ce": lambda mp: _patch(mp, _eta02_index_typo, (S, "eta02_terms")),
    "Eq. 31: multinomial weights dropped": lambda mp: _patch(mp, _eta_r_no_multinomial, (S, "eta_r_terms")),
    "Eq. 30: A in place of B": lambda mp: _patch(mp, _eta_rs_A_only, (S, "eta_rs_terms")),
    "Eqs. 35-36: sign (-1)^r dropped": lambda mp: _patch(mp, _lscv_r_unsigned, (S, "lscv_r")),
    # grid estimate and ISE (Eqs. 1, 37)
    "grid estimate: n^-2 for n^-1": lambda mp: _patch(mp, _kde_grid_n2, (kde, "kde_grid")),
    "grid estimate: stencil stops short of L": lambda mp: _patch(mp, _kde_grid_short_stencil, (kde, "kde_grid")),
    "int f^2: one component's covariance": lambda mp: _patch(mp, _mixture_sq_one_cov, (kde, "mixture_sq_integral")),
    "binned ISE: cross term weight 1": lambda mp: _patch(mp, _ise_binned(cross_w=1.0), (kde, "ise_mixture_binned")),
    "binned ISE: mixture not smoothed by H": lambda mp: _patch(mp, _ise_binned(smooth_H=False), (kde, "ise_mixture_binned")),
    "exact ISE: phi_H for phi_2H": lambda mp: _patch(mp, _ise_exact(pair_scale=1.0), (kde, "ise_mixture_exact")),
    "exact ISE: mixture not smoothed by H": lambda mp: _patch(mp, _ise_exact(cross_H=0.0), (kde, "ise_mixture_exact")),
}


def test_unmutated_battery_passes():
    assert _first_failing_pin() is None


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    MUTANTS[name](monkeypatch)
    caught = _first_failing_pin()
    assert caught is not None, f"no oracle pin catches the planted mistake: {name}"
