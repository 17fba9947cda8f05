"""ctypes binding of the C ABI in include/kdefft.h (argument marshalling only).

Every computation runs in libkdefft.so on the GPU; if the library is missing
or no CUDA device is usable the calls raise: there is no CPU fallback.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); outputs
are returned as numpy arrays.  Every array's size is checked against d before
the library reads through its pointer; an empty batch (no bandwidths, no
datasets) returns empty results without a library call.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkdefft.so")

OK, ERR_ARG, ERR_NOT_SPD, ERR_OUTSIDE_GRID, ERR_CUDA, ERR_ALLOC, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
L_AUTO, L_PAPER, L_WIDEST, L_FULL = range(4)
P_MINIMAL, P_PAPER, P_PAPER_FULL, P_FIXED = range(4)
FP32, FP64 = 0, 1
BIN_LINEAR, BIN_SIMPLE = 0, 1
OUTSIDE_ERROR, OUTSIDE_DROP = 0, 1
LSCV, SCV, PI = 0, 1, 2
DT_F32, DT_F64, DT_I32 = 0, 1, 2

EXPORTS = [
    "kdefft_opts_default", "kdefft_create", "kdefft_destroy", "kdefft_bin", "kdefft_ds_destroy",
    "kdefft_ds_set_opts", "kdefft_ds_info", "kdefft_counts", "kdefft_plan", "kdefft_psi",
    "kdefft_lscv", "kdefft_scv", "kdefft_pi", "kdefft_eta02", "kdefft_select_H", "kdefft_select_H_nm",
    "kdefft_batch_lscv", "kdefft_profile", "kdefft_profile_read", "kdefft_strerror", "kdefft_last_error",
    "kdefft_lscv_noalloc", "kdefft_set_engine", "kdefft_set_autotune", "kdefft_set_graphs",
    "kdefft_runtime_stats", "kdefft_autocorr", "kdefft_qr", "kdefft_lscv_r", "kdefft_eta_rs",
    "kdefft_kde_grid", "kdefft_ise_mixture", "kdefft_select_H_class", "kdefft_bin_many",
    "kdefft_select_H_multi", "kdefft_memory_stats", "kdefft_trim", "kdefft_set_search_record",
    "kdefft_psi_grad", "kdefft_radix_plan",
]
ENGINE_AUTO, ENGINE_MULTIPASS, ENGINE_HOST_SELECT, ENGINE_FFT = 0, 1, 2, 3


class Opts(C.Structure):
    _fields_ = [("tau", C.c_double), ("L_basis", C.c_int), ("P_rule", C.c_int),
                ("P_fixed", C.c_int * 4), ("exact_loo", C.c_int), ("precision", C.c_int),
                ("binning", C.c_int), ("outside_policy", C.c_int)]


class KStat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


class KdefftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kdefft error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libkdefft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1511_07482_gb300.build.build()")
    lib = C.CDLL(path)
    P, D, I, I64 = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int64
    sig = {
        "kdefft_opts_default": (I, [C.POINTER(Opts)]),
        "kdefft_create": (I, [C.POINTER(C.c_void_p), I, P]),
        "kdefft_destroy": (I, [P]),
        "kdefft_bin": (I, [P, P, I64, I, P, P, P, C.POINTER(Opts), C.POINTER(C.c_void_p)]),
        "kdefft_ds_destroy": (I, [P]),
        "kdefft_ds_set_opts": (I, [P, C.POINTER(Opts)]),
        "kdefft_ds_info": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
        "kdefft_counts": (I, [P, P, I]),
        "kdefft_plan": (I, [P, I, P, P, P, P]),
        "kdefft_psi": (I, [P, P, I, I, P]),
        "kdefft_lscv": (I, [P, P, I, P, P]),
        "kdefft_scv": (I, [P, P, I, P, P, P]),
        "kdefft_pi": (I, [P, P, I, P, P, P]),
        "kdefft_eta02": (I, [P, P, I, P, P]),
        "kdefft_select_H": (I, [P, I, P, P, I, I, P, P, P]),
        "kdefft_select_H_nm": (I, [P, I, P, P, I, I, P, P, P]),
        "kdefft_batch_lscv": (I, [P, I, P, P, P, P, P]),
        "kdefft_profile": (I, [P, I]),
        "kdefft_profile_read": (I, [P, P, I, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]),
        "kdefft_lscv_noalloc": (I, [I, P, P, I64, P, P, C.c_double, P, P]),
        "kdefft_set_engine": (I, [P, I]),
        "kdefft_set_autotune": (I, [P, I]),
        "kdefft_autocorr": (I, [P, P, P]),
        "kdefft_qr": (I, [P, P, I, I, P]),
        "kdefft_lscv_r": (I, [P, P, I, I, P]),
        "kdefft_eta_rs": (I, [P, P, P, P, I, I, I, P]),
        "kdefft_kde_grid": (I, [P, P, P]),
        "kdefft_select_H_class": (I, [P, I, I, I, P, P, I, I, P, P, P]),
        "kdefft_bin_many": (I, [P, I, P, P, I, P, P, P, C.POINTER(Opts), P]),
        "kdefft_ise_mixture": (I, [P, P, I, I, P, P, P, P]),
        "kdefft_set_graphs": (I, [P, I]),
        "kdefft_runtime_stats": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "kdefft_memory_stats": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "kdefft_trim": (I, [P]),
        "kdefft_select_H_multi": (I, [P, I, P, P, P, I, I, P, P, P]),
        "kdefft_set_search_record": (I, [P, P, I64, I]),
        "kdefft_psi_grad": (I, [P, P, I, I, P, P]),
        "kdefft_radix_plan": (I, [I, I, P, C.POINTER(C.c_int)]),
        "kdefft_strerror": (C.c_char_p, [I]),
        "kdefft_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code):
    if code != OK:
        lib = load()
        raise KdefftError(code, (lib.kdefft_last_error() or b"").decode() or lib.kdefft_strerror(code).decode())


def _host_f64(a):
    """(contiguous FP64 copy or view, its address as an int: what a
    c_void_p argument takes, without building a ctypes object per call)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data


def _mat(a, d, what):
    """A d x d FP64 matrix argument: (host copy, pointer).  The library reads
    exactly d*d values through the pointer, so the size is checked here."""
    arr, p = _host_f64(a)
    if arr.size != d * d:
        raise ValueError(f"{what} must hold {d} x {d} values, got shape {arr.shape}")
    return arr, p


def _opt_mat(a, d, what):
    return _mat(a, d, what) if a is not None else (None, None)


def _vec(a, d, what, dtype=np.float64):
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype).ravel())
    if arr.size != d:
        raise ValueError(f"{what} must hold {d} values, got {arr.size}")
    return arr


def _ptr_of(x):
    """(keepalive, address) for an n x d sample: a numpy array or a torch
    tensor (host or CUDA)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64:
                raise TypeError("expected a float64 tensor")
            if x.dim() != 2:
                raise ValueError(f"the sample must be n x d, got shape {tuple(x.shape)}")
            x = x.contiguous()
            return x, x.data_ptr()
    except ImportError:
        pass
    arr, p = _host_f64(x)
    if arr.ndim != 2:
        raise ValueError(f"the sample must be n x d, got shape {arr.shape}")
    return arr, p


def lscv_noalloc(M, delta, n, counts, H, out, tau=3.7, stream=None):
    """LSCV(H) and gradient into `out` (a CUDA float64 tensor of 1 + d*d
    values) from device-resident FP32 counts, through the entry point that
    allocates nothing.  Asynchronous on `stream` (default: torch's current
    stream); the caller synchronises."""
    import torch
    d = len(M)
    M_a = _vec(M, d, "M", np.int64)
    dl = _vec(delta, d, "delta")
    pdl = dl.ctypes.data
    Ha, pH = _mat(H, d, "H")
    if not (isinstance(counts, torch.Tensor) and counts.is_cuda and counts.dtype == torch.float32):
        raise TypeError("counts must be a CUDA float32 tensor")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64):
        raise TypeError("out must be a CUDA float64 tensor")
    if not counts.is_contiguous() or counts.numel() != int(np.prod(M_a)):
        raise ValueError("counts must be a contiguous tensor of prod(M) values")
    if not out.is_contiguous() or out.numel() < 1 + d * d:
        raise ValueError(f"out must be a contiguous tensor of at least {1 + d * d} values")
    if stream is None:
        stream = torch.cuda.current_stream(out.device).cuda_stream
    _check(load().kdefft_lscv_noalloc(d, M_a.ctypes.data, pdl, int(n),
                                      C.c_void_p(counts.data_ptr()), pH, float(tau), C.c_void_p(stream),
                                      C.c_void_p(out.data_ptr())))


def radix_plan(P: int, max_radix: int = 32):
    """The radix schedule of the library's transforms of length P (no GPU
    needed)."""
    r = (C.c_int * 16)()
    n = C.c_int()
    _check(load().kdefft_radix_plan(int(P), int(max_radix), C.cast(r, C.c_void_p), C.byref(n)))
    return [int(r[i]) for i in range(n.value)]


_DEFAULT_OPTS = None


def _opts(**kw) -> Opts:
    """Options for a call: without fields one shared, never-modified
    instance of the defaults (the library only reads the options it is
    given), else a fresh default_opts(**kw)."""
    global _DEFAULT_OPTS
    if kw:
        return default_opts(**kw)
    if _DEFAULT_OPTS is None:
        _DEFAULT_OPTS = default_opts()
    return _DEFAULT_OPTS


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(load().kdefft_opts_default(C.byref(o)))
    for k, v in kw.items():
        if k == "P_fixed":
            for i, p in enumerate(v):
                o.P_fixed[i] = int(p)
        else:
            setattr(o, k, v)
    return o


class Context:
    """A kdefft context on one CUDA device and stream (a torch stream or a raw
    cudaStream_t handle; default: torch's current stream when torch is
    available, else the legacy default stream)."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        _check(lib.kdefft_create(C.byref(h), int(device), C.c_void_p(stream or 0)))
        self.h = h
        self.device = device
        self._datasets = weakref.WeakSet()

    def close(self):
        """Destroy the context and every dataset still open on it."""
        if self.h:
            for ds in list(self._datasets):
                ds.h = None          # freed by kdefft_destroy below
            load().kdefft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_engine(self, engine: int):
        """ENGINE_AUTO (fused cluster kernel for d = 2) or ENGINE_MULTIPASS."""
        _check(load().kdefft_set_engine(self.h, int(engine)))

    def set_autotune(self, on: bool = True):
        """Time the candidate engine / tile / radix configurations on the first
        batch of each shape and keep the fastest (kdefft_set_autotune)."""
        _check(load().kdefft_set_autotune(self.h, int(bool(on))))

    def set_graphs(self, on: bool = True):
        """Replay repeated batch launch sequences from CUDA graphs (default on)."""
        _check(load().kdefft_set_graphs(self.h, int(bool(on))))

    def set_search_record(self, rec=None, cap: int = 0):
        """Record the device-resident searches' own evaluations into `rec`, a
        CUDA float64 tensor of starts x cap x 12 values (None: stop
        recording).  The tensor is kept alive here while recording is on."""
        if rec is None:
            _check(load().kdefft_set_search_record(self.h, None, 0, 0))
            self._rec = None
            return
        import torch
        if not (isinstance(rec, torch.Tensor) and rec.is_cuda and rec.dtype == torch.float64
                and rec.is_contiguous()):
            raise TypeError("rec must be a contiguous CUDA float64 tensor")
        _check(load().kdefft_set_search_record(self.h, C.c_void_p(rec.data_ptr()), int(rec.numel()), int(cap)))
        self._rec = rec

    def runtime_stats(self):
        """{"shapes_tuned", "graphs_captured", "graph_replays"} since creation."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().kdefft_runtime_stats(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"shapes_tuned": a.value, "graphs_captured": b.value, "graph_replays": c.value}

    def memory_stats(self):
        """{"cached_bytes", "hits", "misses"} of the context's block cache."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().kdefft_memory_stats(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"cached_bytes": a.value, "hits": b.value, "misses": c.value}

    def trim(self):
        """Release the cached free device blocks."""
        _check(load().kdefft_trim(self.h))

    def profile(self, mode: int = 1):
        """1: reset counters and time every kernel with CUDA events; 2: keep
        timing without a reset; 0: reset and stop timing."""
        _check(load().kdefft_profile(self.h, int(mode)))

    def profile_read(self):
        """Per-kernel stats and counters: (dict name -> dict, launches, h2d, d2h)."""
        lib = load()
        arr = (KStat * 64)()
        cnt = C.c_int()
        la, hb, db = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.kdefft_profile_read(self.h, C.cast(arr, C.c_void_p), 64, C.byref(cnt), C.byref(la),
                                       C.byref(hb), C.byref(db)))
        ks = {}
        for i in range(min(cnt.value, 64)):
            k = arr[i]
            ks[k.name.decode()] = {"launches": k.launches, "ms": k.ms, "bytes": k.bytes, "flops": k.flops}
        return ks, la.value, hb.value, db.value

    def bin(self, X, lo, hi, M, **opts) -> "Dataset":
        """Sec. 4 step 1: bin the n x d FP64 sample onto the grid."""
        keep, px = _ptr_of(X)
        n, d = int(keep.shape[0]), int(keep.shape[1])
        lo_a = _vec(lo, d, "lo")
        hi_a = _vec(hi, d, "hi")
        plo, phi = lo_a.ctypes.data, hi_a.ctypes.data
        M_a = _vec(M, d, "M", np.int64)
        o = _opts(**opts)
        h = C.c_void_p()
        _check(load().kdefft_bin(self.h, px, n, d, plo, phi, M_a.ctypes.data, C.byref(o),
                                 C.byref(h)))
        ds = Dataset(self, h, d, [int(m) for m in M_a])
        self._datasets.add(ds)
        return ds

    def bin_many(self, Xs, los, his, Ms, **opts):
        """Bin many datasets of the same dimension in one call (a few
        batched launches): one Dataset per sample."""
        nds = len(Xs)
        if nds == 0:
            return []
        keep = [_ptr_of(X) for X in Xs]
        d = int(keep[0][0].shape[1])
        if any(int(k.shape[1]) != d for k, _ in keep):
            raise ValueError("every sample of a batch must have the same dimension d")
        ptrs = (C.c_void_p * nds)(*[p for _, p in keep])
        n = np.ascontiguousarray(np.array([int(k.shape[0]) for k, _ in keep], dtype=np.int64))
        lo = np.ascontiguousarray(np.asarray(los, dtype=np.float64).reshape(nds, d))
        hi = np.ascontiguousarray(np.asarray(his, dtype=np.float64).reshape(nds, d))
        M = np.ascontiguousarray(np.asarray(Ms, dtype=np.int64).reshape(nds, d))
        o = _opts(**opts)
        hs = (C.c_void_p * nds)()
        _check(load().kdefft_bin_many(self.h, nds, C.cast(ptrs, C.c_void_p), n.ctypes.data, d,
                                      lo.ctypes.data, hi.ctypes.data,
                                      M.ctypes.data, C.byref(o), C.cast(hs, C.c_void_p)))
        out = []
        for i in range(nds):
            ds = Dataset(self, C.c_void_p(hs[i]), d, [int(m) for m in M[i]])
            self._datasets.add(ds)
            out.append(ds)
        return out

    def batch_lscv(self, datasets, H_per_ds, grad=True):
        """LSCV (+ gradient) for many datasets in one batched launch sequence."""
        if len(datasets) == 0:
            return (np.zeros(0), np.zeros((0, 0, 0))) if grad else np.zeros(0)
        lib = load()
        d = datasets[0].d
        nh = np.array([len(h) for h in H_per_ds], dtype=np.int32)
        H = np.ascontiguousarray(np.concatenate([np.asarray(h, dtype=np.float64).reshape(-1, d, d)
                                                 for h in H_per_ds]))
        tot = int(nh.sum())
        val = np.zeros(tot)
        g = np.zeros((tot, d, d)) if grad else None
        arr = (C.c_void_p * len(datasets))(*[ds.h for ds in datasets])
        _check(lib.kdefft_batch_lscv(self.h, len(datasets), arr, nh.ctypes.data,
                                     H.ctypes.data, val.ctypes.data,
                                     g.ctypes.data if grad else None))
        return (val, g) if grad else val


class Dataset:
    def __init__(self, ctx, h, d, M):
        self.ctx, self.h, self.d, self.M = ctx, h, d, M

    def close(self):
        if self.h and self.ctx.h:
            load().kdefft_ds_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **opts):
        o = _opts(**opts)
        _check(load().kdefft_ds_set_opts(self.h, C.byref(o)))

    def info(self):
        n, d, dr = C.c_int64(), C.c_int(), C.c_int64()
        _check(load().kdefft_ds_info(self.h, C.byref(n), C.byref(d), C.byref(dr)))
        return n.value, d.value, dr.value

    def counts(self, dtype=DT_F64):
        np_t = {DT_F32: np.float32, DT_F64: np.float64, DT_I32: np.int32}[dtype]
        out = np.zeros(self.M, dtype=np_t)
        _check(load().kdefft_counts(self.h, out.ctypes.data, dtype))
        return out

    def plan(self, method, H, G=None):
        Ha, pH = _mat(H, self.d, "H")
        Ga, pG = _opt_mat(G, self.d, "G")
        L = np.zeros(self.d, dtype=np.int32)
        P = np.zeros(self.d, dtype=np.int32)
        _check(load().kdefft_plan(self.h, method, pH, pG, L.ctypes.data,
                                  P.ctypes.data))
        return [int(v) for v in L], [int(v) for v in P]

    def _Hs(self, H):
        H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1, self.d, self.d))
        return H, H.shape[0]

    def psi(self, H, r):
        """psi_r(H) (Eq. 13) as nH x d^r, Kronecker order."""
        H, nH = self._Hs(H)
        out = np.zeros((nH, self.d ** r))
        if nH == 0:
            return out
        _check(load().kdefft_psi(self.h, H.ctypes.data, nH, r, out.ctypes.data))
        return out

    def psi_grad(self, H, r, w):
        """sum_i w_i d psi_{r,i}(H) / dH per bandwidth (entries of H
        independent): nH x d x d, from psi_{r+2} through the library."""
        H, nH = self._Hs(H)
        wa = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        if wa.size != nH * self.d ** r:
            raise ValueError(f"w must hold {nH} x {self.d ** r} values, got {wa.size}")
        out = np.zeros((nH, self.d, self.d))
        if nH == 0:
            return out
        _check(load().kdefft_psi_grad(self.h, H.ctypes.data, nH, int(r),
                                      wa.ctypes.data, out.ctypes.data))
        return out

    def lscv(self, H, grad=False):
        H, nH = self._Hs(H)
        val = np.zeros(nH)
        g = np.zeros((nH, self.d, self.d)) if grad else None
        if nH == 0:
            return (val, g) if grad else val
        _check(load().kdefft_lscv(self.h, H.ctypes.data, nH, val.ctypes.data,
                                  g.ctypes.data if grad else None))
        return (val, g) if grad else val

    def scv(self, H, G, grad=False):
        H, nH = self._Hs(H)
        Ga, pG = _mat(G, self.d, "G")
        val = np.zeros(nH)
        g = np.zeros((nH, self.d, self.d)) if grad else None
        if nH == 0:
            return (val, g) if grad else val
        _check(load().kdefft_scv(self.h, H.ctypes.data, nH, pG, val.ctypes.data,
                                 g.ctypes.data if grad else None))
        return (val, g) if grad else val

    def pi(self, H, G, grad=False):
        H, nH = self._Hs(H)
        Ga, pG = _mat(G, self.d, "G")
        val = np.zeros(nH)
        g = np.zeros((nH, self.d, self.d)) if grad else None
        if nH == 0:
            return (val, g) if grad else val
        _check(load().kdefft_pi(self.h, H.ctypes.data, nH, pG, val.ctypes.data,
                                g.ctypes.data if grad else None))
        return (val, g) if grad else val

    def autocorr(self, A):
        """Count autocorrelation a_j = sum_i c_i c_{i+j} on the half box
        j_0 in [0, A_0], |j_k| <= A_k: array of shape (2 A_{d-1} + 1, ..,
        2 A_1 + 1, A_0 + 1), index j_k + A_k on the axes k >= 1."""
        A_a = np.ascontiguousarray(np.asarray(A, dtype=np.int32).reshape(self.d))
        shape = tuple(2 * int(a) + 1 for a in A_a[1:][::-1]) + (int(A_a[0]) + 1,)
        out = np.zeros(shape)
        _check(load().kdefft_autocorr(self.h, A_a.ctypes.data, out.ctypes.data))
        return out

    def qr(self, Sigma, r):
        """Q_r(Sigma) (Eq. 32), eta = Laplacian^{r/2} phi_Sigma; r = total
        derivative order (even).  One value per Sigma."""
        S, nS = self._Hs(Sigma)
        out = np.zeros(nS)
        if nS == 0:
            return out
        _check(load().kdefft_qr(self.h, S.ctypes.data, nS, int(r), out.ctypes.data))
        return out

    def eta_rs(self, Sigma, r, s, A=None, B=None):
        """n^-2 sum_ij eta_{r,s}(X_i - X_j; A, B, Sigma) (Eqs. 29-30) for each
        Sigma; A, B default to the identity."""
        S, nS = self._Hs(Sigma)
        Aa, pA = _opt_mat(A, self.d, "A")
        Ba, pB = _opt_mat(B, self.d, "B")
        out = np.zeros(nS)
        if nS == 0:
            return out
        _check(load().kdefft_eta_rs(self.h, pA, pB, S.ctypes.data, nS, int(r), int(s),
                                    out.ctypes.data))
        return out

    def kde_grid(self, H):
        """The binned kernel density estimate at every grid node (shape M)."""
        Ha, pH = _mat(H, self.d, "H")
        out = np.zeros(self.M)
        _check(load().kdefft_kde_grid(self.h, pH, out.ctypes.data))
        return out

    def ise_mixture(self, H, weights, means, covs):
        """ISE of the binned estimate at each H against the normal mixture
        sum_m w_m phi_{S_m}(. - mu_m) (closed form)."""
        H, nH = self._Hs(H)
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).ravel())
        mu = np.ascontiguousarray(np.asarray(means, dtype=np.float64).reshape(len(w), self.d))
        S = np.ascontiguousarray(np.asarray(covs, dtype=np.float64).reshape(len(w), self.d, self.d))
        out = np.zeros(nH)
        if nH == 0:
            return out
        _check(load().kdefft_ise_mixture(self.h, H.ctypes.data, nH, len(w),
                                         w.ctypes.data, mu.ctypes.data,
                                         S.ctypes.data, out.ctypes.data))
        return out

    def lscv_r(self, H, r):
        """LSCV_r(H) (Eq. 36, or Eq. 35 with exact_loo) for the r-th density
        derivative; values."""
        H, nH = self._Hs(H)
        out = np.zeros(nH)
        if nH == 0:
            return out
        _check(load().kdefft_lscv_r(self.h, H.ctypes.data, nH, int(r), out.ctypes.data))
        return out

    def eta02(self, H, G):
        H, nH = self._Hs(H)
        Ga, pG = _mat(G, self.d, "G")
        val = np.zeros(nH)
        if nH == 0:
            return val
        _check(load().kdefft_eta02(self.h, H.ctypes.data, nH, pG, val.ctypes.data))
        return val

    def select_H(self, method=LSCV, H0=None, G=None, n_starts=1, max_iter=None, optimizer="bfgs", hclass="full"):
        """Minimise the objective over H: optimizer "bfgs" (quasi-Newton on
        the exact gradients, max_iter iterations, default 100) or
        "nelder-mead" (the paper's derivative-free parity mode, max_iter
        objective evaluations per start, default 500); hclass "full" (the
        SPD matrices), "diag" or "scalar" (Sec. 3's constrained classes)."""
        if optimizer not in ("bfgs", "nelder-mead"):
            raise ValueError("optimizer must be 'bfgs' or 'nelder-mead'")
        classes = {"full": 0, "diag": 1, "scalar": 2}
        if hclass not in classes:
            raise ValueError("hclass must be 'full', 'diag' or 'scalar'")
        Ha, pH = _opt_mat(H0, self.d, "H0")
        Ga, pG = _opt_mat(G, self.d, "G")
        Hout = np.zeros((self.d, self.d))
        f = C.c_double()
        ne = C.c_int64()
        lib = load()
        if hclass == "full":
            fn = lib.kdefft_select_H if optimizer == "bfgs" else lib.kdefft_select_H_nm
            _check(fn(self.h, method, pH, pG, int(n_starts), int(max_iter or 0),
                      Hout.ctypes.data, C.byref(f), C.byref(ne)))
        else:
            _check(lib.kdefft_select_H_class(self.h, method, classes[hclass], 0 if optimizer == "bfgs" else 1, pH,
                                             pG, int(n_starts), int(max_iter or 0),
                                             Hout.ctypes.data, C.byref(f), C.byref(ne)))
        return Hout, f.value, ne.value

    def select_H_many(self, methods, H0=None, G=None, n_starts=1, max_iter=None):
        """select_H (quasi-Newton, full H) for several criteria on this
        dataset; two criteria the device search covers share one launch.
        Returns [(H, f, evals)] in the order of `methods`."""
        ms = np.ascontiguousarray(np.asarray(methods, dtype=np.int32))
        k = int(ms.size)
        Ha, pH = _opt_mat(H0, self.d, "H0")
        Ga, pG = _opt_mat(G, self.d, "G")
        Hout = np.zeros((k, self.d, self.d))
        f = np.zeros(k)
        ne = np.zeros(k, dtype=np.int64)
        _check(load().kdefft_select_H_multi(self.h, k, ms.ctypes.data, pH, pG, int(n_starts),
                                            int(max_iter or 0), Hout.ctypes.data,
                                            f.ctypes.data, ne.ctypes.data))
        return [(Hout[m], float(f[m]), int(ne[m])) for m in range(k)]
