"""psi_r, LSCV, SCV and PI of a binned dataset as differentiable functions
of H for torch.autograd.

H is a float tensor of shape (d, d) or (nH, d, d) on any device; the
functions see its symmetric part (H + H^T)/2, so the gradient of an output
with respect to the full matrix is, entry by entry,

    d f / d H_ab = 1/2 (d f / d H_ab + d f / d H_ba)   of the symmetric form,

which for the Gaussian kernel follows from its heat equation
d phi_H / dH = 1/2 grad grad^T phi_H:
    d psi_alpha(H) / d H_ab = 1/2 psi_{alpha + e_a + e_b}(H),
so psi_r's backward evaluates psi_{r+2} at the same H (r <= 6), and the
objectives' backward takes the exact gradients the library returns with
their values (tied off-diagonal convention, halved off the diagonal here).

Every evaluation runs in the CUDA library through the C ABI; this module only
marshals tensors.
"""
import numpy as np
import torch

__all__ = ["psi", "lscv", "scv", "pi"]


def _batch(H):
    Hn = H.detach().to("cpu", torch.float64).numpy()
    single = Hn.ndim == 2
    Hb = Hn.reshape((-1,) + Hn.shape[-2:])
    return 0.5 * (Hb + np.swapaxes(Hb, 1, 2)), single


def _full_from_tied(g):
    g = np.array(g, dtype=np.float64, copy=True)
    d = g.shape[-1]
    g[..., ~np.eye(d, dtype=bool)] *= 0.5
    return g


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, ds, kind, G):
        Hs, single = _batch(H)
        if kind == "lscv":
            v, g = ds.lscv(Hs, grad=True)
        elif kind == "scv":
            v, g = ds.scv(Hs, G, grad=True)
        else:
            v, g = ds.pi(Hs, G, grad=True)
        ctx.single = single
        ctx.save_for_backward(torch.from_numpy(_full_from_tied(g)).to(H.device))
        out = torch.from_numpy(np.ascontiguousarray(v)).to(device=H.device, dtype=H.dtype)
        return out[0] if single else out

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        gH = grad_out.to(g.dtype).reshape(-1, 1, 1) * g
        if ctx.single:
            gH = gH[0]
        return gH.to(grad_out.dtype), None, None, None


class _Psi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, ds, r):
        Hs, single = _batch(H)
        out = ds.psi(Hs, r)
        ctx.ds, ctx.r, ctx.single = ds, r, single
        ctx.save_for_backward(H.detach())
        t = torch.from_numpy(out).to(device=H.device, dtype=H.dtype)
        return t[0] if single else t

    @staticmethod
    def backward(ctx, grad_out):
        (H,) = ctx.saved_tensors
        ds, r, d = ctx.ds, ctx.r, H.shape[-1]
        if r + 2 > 8:
            raise NotImplementedError("the gradient of psi_r needs psi_{r+2}, available for r <= 6")
        Hs, _ = _batch(H)
        p2 = ds.psi(Hs, r + 2).reshape(len(Hs), d ** r, d, d)
        go = grad_out.detach().to("cpu", torch.float64).numpy().reshape(len(Hs), d ** r)
        gH = 0.5 * np.einsum("ki,kiab->kab", go, p2)
        gH = torch.from_numpy(gH).to(device=H.device, dtype=grad_out.dtype)
        return (gH[0] if ctx.single else gH), None, None


def psi(ds, H, r):
    """psi_r(H) (Eq. 13) of dataset ds: shape (d^r,) or (nH, d^r), Kronecker order."""
    return _Psi.apply(H, ds, int(r))


def lscv(ds, H):
    """LSCV(H) (Eq. 10) of dataset ds: scalar or (nH,)."""
    return _Objective.apply(H, ds, "lscv", None)


def scv(ds, H, G):
    """SCV(H) with pilot G of dataset ds: scalar or (nH,)."""
    return _Objective.apply(H, ds, "scv", np.asarray(G, dtype=np.float64))


def pi(ds, H, G):
    """PI(H) with pilot G of dataset ds: scalar or (nH,)."""
    return _Objective.apply(H, ds, "pi", np.asarray(G, dtype=np.float64))
