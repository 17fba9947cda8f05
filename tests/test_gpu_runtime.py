"""Batch runtime: CUDA-graph replay of repeated launch sequences and the
autotuner.  Replayed batches give the same bits as direct launches (same
kernels, same inputs); tuned configurations agree with the default one
within the FP32 tolerance of the evaluation."""
import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _ctx(**kw):
    from paper_1511_07482_gb300 import Context
    c = Context(0)
    if "engine" in kw:
        c.set_engine(kw["engine"])
    if "graphs" in kw:
        c.set_graphs(kw["graphs"])
    if kw.get("autotune"):
        c.set_autotune(True)
    return c


@pytest.mark.parametrize("engine", ["auto", "fft", "multipass"])
def test_graph_replay_gives_the_direct_bits(engine):
    from paper_1511_07482_gb300 import ENGINE_AUTO, ENGINE_FFT, ENGINE_MULTIPASS
    eng = {"auto": ENGINE_AUTO, "fft": ENGINE_FFT, "multipass": ENGINE_MULTIPASS}[engine]
    w = synthetic.small_case(n=3000, d=2, M=[64, 60], seed=71, n_candidates=4)
    res = {}
    for g in (True, False):
        c = _ctx(engine=eng, graphs=g)
        ds = c.bin(w.X, w.lo, w.hi, w.M)
        outs = [ds.lscv(w.H, grad=True) for _ in range(3)]
        for v, gr in outs[1:]:
            assert np.array_equal(v, outs[0][0]) and np.array_equal(gr, outs[0][1])
        res[g] = (outs[0], c.runtime_stats())
        ds.close()
        c.close()
    assert np.array_equal(res[True][0][0], res[False][0][0])
    assert np.array_equal(res[True][0][1], res[False][0][1])
    st_on, st_off = res[True][1], res[False][1]
    assert st_on["graphs_captured"] >= 1 and st_on["graph_replays"] >= 2
    assert st_off["graphs_captured"] == 0 and st_off["graph_replays"] == 0


def test_selection_replay_gives_the_direct_bits():
    """The selection's launch sequence (table copies, count spectrum and
    autocorrelation passes, the device search and its copy back, then both
    end-point values) replays as CUDA graphs from the second step on, each
    step on a freshly binned dataset: the same bandwidths, values and
    evaluation counts as direct launches, step after step."""
    from paper_1511_07482_gb300 import LSCV, SCV
    w = synthetic.small_case(n=20000, d=2, M=[96, 90], seed=74, n_candidates=1)
    G = synthetic.normal_scale(w.X)
    res = {}
    for g in (True, False):
        c = _ctx(graphs=g)
        steps = []
        for _ in range(3):
            ds = c.bin(w.X, w.lo, w.hi, w.M)
            steps.append(ds.select_H_many([LSCV, SCV], G=G, n_starts=4, max_iter=30))
            ds.close()
        for st in steps[1:]:
            for (Ha, fa, ea), (Hb, fb, eb) in zip(st, steps[0]):
                assert np.array_equal(Ha, Hb) and fa == fb and ea == eb
        res[g] = (steps[0], c.runtime_stats())
        c.close()
    for (Ha, fa, ea), (Hb, fb, eb) in zip(res[True][0], res[False][0]):
        assert np.array_equal(Ha, Hb) and fa == fb and ea == eb
    assert res[True][1]["graph_replays"] >= 2
    assert res[False][1]["graphs_captured"] == 0


def test_graphs_are_recaptured_after_buffers_grow():
    """A captured graph copies through the context's staging buffers; once a
    larger batch has reallocated them, the small batch is captured again
    (never replayed against the old allocations) and gives the same bits."""
    w = synthetic.small_case(n=3000, d=2, M=[64, 60], seed=73, n_candidates=4)
    c = _ctx()
    ds = c.bin(w.X, w.lo, w.hi, w.M)
    small = [ds.lscv(w.H, grad=True) for _ in range(2)]
    st1 = c.runtime_stats()
    assert st1["graph_replays"] >= 1
    big = np.concatenate([w.H * s for s in (0.6, 0.8, 1.0, 1.25, 1.5, 2.0, 2.5, 3.0)] * 8)
    ds.lscv(big, grad=True)
    st2 = c.runtime_stats()
    again = ds.lscv(w.H, grad=True)
    st3 = c.runtime_stats()
    assert st3["graphs_captured"] == st2["graphs_captured"] + 1
    assert np.array_equal(again[0], small[0][0]) and np.array_equal(again[1], small[0][1])
    ds.close()
    c.close()


def test_graphs_are_bypassed_while_profiling():
    w = synthetic.small_case(n=2000, d=3, M=[20, 18, 16], seed=72, n_candidates=2)
    c = _ctx()
    ds = c.bin(w.X, w.lo, w.hi, w.M)
    a = ds.psi(w.H, 4)
    before = c.runtime_stats()
    c.profile(1)
    b = ds.psi(w.H, 4)
    stats, launches, _, _ = c.profile_read()
    c.profile(0)
    assert c.runtime_stats() == before
    assert launches >= 1 and any(k.startswith(("lag", "final")) for k in stats)
    assert np.array_equal(a, b)
    ds.close()
    c.close()


@pytest.mark.parametrize("d,M,r", [(2, [80, 72], 4), (3, [24, 20, 18], 4)])
def test_autotuned_batches_agree_with_default(d, M, r):
    """The tuner chooses among the FFT-route configurations (the lag-domain
    engine has no knobs), so both contexts take the FFT route."""
    from paper_1511_07482_gb300 import ENGINE_FFT
    w = synthetic.small_case(n=4000, d=d, M=M, seed=73 + d, n_candidates=6)
    ref_c = _ctx(engine=ENGINE_FFT)
    ref = ref_c.bin(w.X, w.lo, w.hi, w.M)
    want_psi = ref.psi(w.H, r)
    want_v, want_g = ref.lscv(w.H, grad=True)
    c = _ctx(engine=ENGINE_FFT, autotune=True)
    ds = c.bin(w.X, w.lo, w.hi, w.M)
    tuned = []
    for _ in range(2):
        got_psi = ds.psi(w.H, r)
        got_v, got_g = ds.lscv(w.H, grad=True)
        assert np.max(np.abs(got_psi - want_psi)) <= 1e-5 * np.max(np.abs(want_psi))
        np.testing.assert_allclose(got_v, want_v, rtol=1e-5)
        assert np.max(np.abs(got_g - want_g)) <= 1e-5 * np.max(np.abs(want_g))
        tuned.append(c.runtime_stats()["shapes_tuned"])
    # the psi batch and the LSCV batch are tuned on the first pass; the
    # second pass reuses both choices
    assert tuned[0] >= 2 and tuned[1] == tuned[0]
    for x in (ds, ref):
        x.close()
    c.close()
    ref_c.close()
