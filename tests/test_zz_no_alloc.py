"""The entry point that allocates nothing (kdefft_lscv_noalloc).

Some callers cannot allocate device memory when they need an objective value
(a memory budget fixed up front, a call from inside another framework's
allocator, a latency-critical loop); kdefft_lscv_noalloc serves them from a
fixed scratch array in the library image.  This file checks, through the C
ABI, that two calls in a row agree with the regular entry point kdefft_lscv
within the tolerance of the other parity tests, and that the second call
leaves the device's free memory unchanged; that a sequence of calls with
different scratch layouts matches the FP64 oracle call by call; that a call
on a stream under capture is refused; and that host buffers are refused.
It is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,M", [(2, [64, 60]), (3, [20, 18, 16]), (1, [90])])
def test_noalloc_matches_lscv_on_two_calls(d, M):
    import torch

    from paper_1511_07482_gb300 import DT_F32, Context, _lib, synthetic

    w = synthetic.small_case(n=3000, d=d, M=M, seed=90 + d, n_candidates=2)
    ctx = Context(0)
    ds = ctx.bin(w.X, w.lo, w.hi, w.M)
    counts = torch.from_numpy(ds.counts(DT_F32).ravel()).cuda()
    delta = (np.asarray(w.hi) - np.asarray(w.lo)) / (np.asarray(w.M) - 1)
    outs = [torch.full((1 + d * d,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    refs = [ds.lscv(H, grad=True) for H in w.H]
    torch.cuda.synchronize()
    # first call: may perform the one-time set-up
    _lib.lscv_noalloc(w.M, delta, w.n, counts, w.H[0], outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # second call in a row, another bandwidth: no allocation
    _lib.lscv_noalloc(w.M, delta, w.n, counts, w.H[1], outs[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for (rv, rg), o in zip(refs, outs):
        got = o.cpu().numpy()
        assert abs(got[0] - rv[0]) <= 1e-5 * abs(rv[0]), (got[0], rv[0])
        g = got[1:].reshape(d, d)
        assert np.max(np.abs(g - rg[0])) <= 1e-5 * np.max(np.abs(rg[0])), (g, rg[0])
    ds.close()
    ctx.close()


def test_noalloc_rejects_host_output_and_oversize():
    import torch

    from paper_1511_07482_gb300 import KdefftError, _lib

    counts = torch.ones(16, dtype=torch.float32, device="cuda")
    out_host = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(TypeError):
        _lib.lscv_noalloc([4, 4], [0.1, 0.1], 16, counts, np.eye(2) * 0.01, out_host)
    # a grid whose spectrum and work buffers exceed the 32 MiB scratch
    big = torch.ones(4000 * 4000, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(KdefftError) as e:
        _lib.lscv_noalloc([4000, 4000], [1e-3, 1e-3], 100, big, np.eye(2) * 1e-4, out)
    assert e.value.code == _lib.ERR_UNSUPPORTED


def _oracle_lscv(w, H):
    """LSCV(H) of Eq. 10 and its gradient by the FP64 oracle on its own
    binning of the sample, with the support of Eq. 26 and the minimal
    no-alias padding, plus the magnitudes of the summed terms (the
    normalisation of every FP32 tolerance)."""
    from oracle import binning, functionals as F, rules, selectors as S
    c = binning.bin_linear(w.X, w.lo, w.hi, w.M)
    delta = rules.bin_width(w.lo, w.hi, w.M)
    L = [max(1, v) for v in rules.support_L(rules.lambda_max(H), delta, w.M)]
    P = rules.P_minimal(w.M, L)
    val, g = S.lscv(lambda t: F.binned_fft(c, w.n, t, delta, L, P), H, w.n, grad=True)
    a = F.autocorr_fft(c)
    sv, sg = S.abs_scales(lambda t: F.lag_sums(a, w.n, t, delta, L)[1], "lscv", H, w.n)
    return val, g, sv, sg


def test_noalloc_layout_sequence_matches_oracle():
    """Three calls in a row whose scratch layouts differ (d = 3 on the largest
    grid, then d = 2 on a smaller one, then d = 1): each result must match the
    oracle and the regular entry point, so no call reads what the previous
    one left in the shared scratch array."""
    import torch

    from paper_1511_07482_gb300 import DT_F32, Context, _lib, synthetic

    ctx = Context(0)
    try:
        for d, M in [(3, [30, 28, 26]), (2, [48, 44]), (1, [70])]:
            w = synthetic.small_case(n=2500, d=d, M=M, seed=120 + d, n_candidates=1)
            ds = ctx.bin(w.X, w.lo, w.hi, w.M)
            counts = torch.from_numpy(ds.counts(DT_F32).ravel()).cuda()
            delta = (np.asarray(w.hi) - np.asarray(w.lo)) / (np.asarray(w.M) - 1)
            H = w.H[0]
            out = torch.full((1 + d * d,), float("nan"), dtype=torch.float64, device="cuda")
            _lib.lscv_noalloc(w.M, delta, w.n, counts, H, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            rv, rg = ds.lscv(H, grad=True)
            val, g, sv, sg = _oracle_lscv(w, H)
            assert abs(got[0] - val) <= 1e-5 * max(abs(val), 0.1 * sv), (d, got[0], val)
            gg = got[1:].reshape(d, d)
            assert np.all(np.abs(gg - g) <= 1e-5 * np.maximum(np.abs(g), 0.1 * sg)), (d, gg, g)
            assert abs(got[0] - rv[0]) <= 1e-5 * max(abs(rv[0]), 0.1 * sv)
            ds.close()
    finally:
        ctx.close()


def test_noalloc_refuses_a_stream_under_capture():
    """The call's small tables come from host staging that the next call
    overwrites, so it refuses to run while its stream is being captured."""
    import torch

    from paper_1511_07482_gb300 import KdefftError, _lib

    counts = torch.ones(32 * 32, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        with pytest.raises(KdefftError) as e:
            _lib.lscv_noalloc([32, 32], [0.1, 0.1], 1024, counts, np.eye(2) * 0.05, out, stream=s.cuda_stream)
    assert e.value.code == _lib.ERR_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # outside a capture the same call runs
    _lib.lscv_noalloc([32, 32], [0.1, 0.1], 1024, counts, np.eye(2) * 0.05, out)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_c_abi_rejects_host_buffers():
    """Through the C ABI directly: an output or counts buffer in host memory
    is KDEFFT_ERR_ARG before anything runs."""
    import ctypes as C

    import torch

    from paper_1511_07482_gb300 import _lib

    lib = _lib.load()
    M = np.array([8, 8], dtype=np.int64)
    delta = np.array([0.1, 0.1])
    H = np.eye(2) * 0.05
    dev_counts = torch.ones(64, dtype=torch.float32, device="cuda")
    dev_out = torch.zeros(5, dtype=torch.float64, device="cuda")
    host_counts = np.ones(64, dtype=np.float32)
    host_out = np.zeros(5)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    r = lib.kdefft_lscv_noalloc(2, vp(M), vp(delta), 64, C.c_void_p(dev_counts.data_ptr()), vp(H), 3.7, None,
                                vp(host_out))
    assert r == _lib.ERR_ARG
    r = lib.kdefft_lscv_noalloc(2, vp(M), vp(delta), 64, vp(host_counts), vp(H), 3.7, None,
                                C.c_void_p(dev_out.data_ptr()))
    assert r == _lib.ERR_ARG
