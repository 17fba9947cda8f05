"""The entry point that allocates nothing (kdefft_lscv_noalloc).

Some callers cannot allocate device memory when they need an objective value
(a memory budget fixed up front, a call from inside another framework's
allocator, a latency-critical loop); kdefft_lscv_noalloc serves them from a
fixed scratch array in the library image.  This file checks, through the C
ABI, that two calls in a row agree with the regular entry point kdefft_lscv
within the tolerance of the other parity tests, and that the second call
leaves the device's free memory unchanged.  It is collected last on purpose.
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
