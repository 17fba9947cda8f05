"""Two contexts on two host threads of one process, on one GPU, each with its
own stream: the library's process-wide state (kernel attributes set once per
device, the shared plan caches, the cluster-occupancy caches) must let both
run at the same time and give the results one context gives alone, bit for
bit (binning sums in fixed point and every reduction has a fixed order)."""
import threading

import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _work(stream, w, out, key):
    from paper_1511_07482_gb300 import LSCV, SCV, Context
    try:
        ctx = Context(0, stream=stream)
        ds = ctx.bin(w.X, w.lo, w.hi, w.M)
        v, g = ds.lscv(w.H, grad=True)
        p4 = ds.psi(w.H[:4], 4)
        sel = ds.select_H_many([LSCV, SCV], G=w.G, n_starts=8, max_iter=40)
        ds.close()
        ctx.close()
        out[key] = (v, g, p4, [(H, f, e) for H, f, e in sel])
    except Exception as e:  # noqa: BLE001 - the main thread reports it
        out[key] = e


def test_two_contexts_on_two_threads_give_identical_results():
    import torch
    w = synthetic.mixture_2d_large(n=40000, M=192)
    out = {}
    _work(torch.cuda.Stream(), w, out, "alone")
    assert not isinstance(out["alone"], Exception), out["alone"]
    for rep in range(2):
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        threads = [threading.Thread(target=_work, args=(streams[k], w, out, (rep, k))) for k in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for k in range(2):
            got = out[(rep, k)]
            assert not isinstance(got, Exception), got
            ref = out["alone"]
            for a, b in zip(got[:3], ref[:3]):
                assert np.array_equal(a, b)
            for (Ha, fa, ea), (Hb, fb, eb) in zip(got[3], ref[3]):
                assert np.array_equal(Ha, Hb) and fa == fb and ea == eb
