"""torch.autograd wrappers: the backward of psi_r, LSCV, SCV and PI against
central finite differences of the forward, on FP64 datasets (values to
~1e-12, so a step of 1e-5 relative resolves the derivative to ~1e-6), in the
full-matrix convention d f / d H_ab of f((H + H^T)/2).  The wrappers pass H
to the library as it is (which refuses an asymmetric H), so the finite
differences symmetrise each perturbed matrix themselves."""
import numpy as np
import pytest

from paper_1511_07482_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1511_07482_gb300 import FP64, Context
    w = synthetic.small_case(n=1500, d=2, M=[48, 44], seed=61, n_candidates=2)
    c = Context(0)
    ds = c.bin(w.X, w.lo, w.hi, w.M, precision=FP64)
    yield w, ds
    ds.close()
    c.close()


def _fd(f, H, h):
    d = H.shape[0]
    g = np.zeros((d, d))
    for a in range(d):
        for b in range(d):
            E = np.zeros((d, d))
            E[a, b] = h
            g[a, b] = (f(H + E) - f(H - E)) / (2 * h)
    return g


@pytest.mark.parametrize("kind", ["lscv", "scv", "pi"])
def test_objective_backward_matches_finite_differences(setup, kind):
    import torch

    from paper_1511_07482_gb300 import autograd as A
    w, ds = setup
    H0 = w.H[0]
    fn = {"lscv": lambda H: A.lscv(ds, H), "scv": lambda H: A.scv(ds, H, w.G), "pi": lambda H: A.pi(ds, H, w.G)}[kind]
    Ht = torch.tensor(H0, dtype=torch.float64, requires_grad=True)
    y = fn(Ht)
    y.backward()
    got = Ht.grad.numpy()
    h = 1e-5 * np.max(np.abs(H0))
    ref = _fd(lambda H: fn(torch.tensor(0.5 * (H + H.T))).item(), H0, h)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), (got, ref)
    # an asymmetric perturbation moves f like its symmetric part
    assert got[0, 1] == pytest.approx(got[1, 0], rel=1e-12)


def test_batched_objective_and_chain_rule(setup):
    import torch

    from paper_1511_07482_gb300 import autograd as A
    w, ds = setup
    Ht = torch.tensor(np.stack(w.H), dtype=torch.float64, requires_grad=True)
    y = A.lscv(ds, Ht)
    assert y.shape == (len(w.H),)
    (3.0 * y[0] - y[1]).backward()
    v, g = ds.lscv(np.stack(w.H), grad=True)
    half = np.where(np.eye(2, dtype=bool), 1.0, 0.5)
    np.testing.assert_allclose(Ht.grad.numpy()[0], 3.0 * g[0] * half, rtol=1e-12)
    np.testing.assert_allclose(Ht.grad.numpy()[1], -g[1] * half, rtol=1e-12)


def test_psi_grad_is_the_library_adjoint(setup):
    """kdefft_psi_grad through the C ABI: the contraction of psi_{r+2} with
    the weights, checked against central differences of psi_r itself, for a
    batch of two bandwidths; and the order limit."""
    from paper_1511_07482_gb300 import KdefftError
    w, ds = setup
    r = 2
    rng = np.random.default_rng(5)
    Hs = np.stack(w.H)
    wv = rng.standard_normal((len(Hs), 2 ** r))
    g = ds.psi_grad(Hs, r, wv)
    assert g.shape == (len(Hs), 2, 2)
    for k in range(len(Hs)):
        h = 1e-5 * np.max(np.abs(Hs[k]))
        ref = _fd(lambda H: float(ds.psi(0.5 * (H + H.T), r)[0] @ wv[k]), Hs[k], h)
        assert np.max(np.abs(g[k] - ref)) <= 1e-5 * np.max(np.abs(ref)), (g[k], ref)
    with pytest.raises(KdefftError):
        ds.psi_grad(Hs[:1], 8, np.ones(2 ** 8))       # needs psi_10


@pytest.mark.parametrize("r", [2, 4])
def test_psi_backward_uses_psi_r_plus_2(setup, r):
    import torch

    from paper_1511_07482_gb300 import autograd as A
    w, ds = setup
    H0 = w.H[1]
    rng = np.random.default_rng(r)
    wvec = rng.standard_normal(2 ** r)
    Ht = torch.tensor(H0, dtype=torch.float64, requires_grad=True)
    (A.psi(ds, Ht, r) * torch.from_numpy(wvec)).sum().backward()
    got = Ht.grad.numpy()
    h = 1e-5 * np.max(np.abs(H0))
    ref = _fd(lambda H: float(ds.psi(0.5 * (H + H.T), r)[0] @ wvec), H0, h)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), (got, ref)
