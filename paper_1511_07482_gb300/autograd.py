"""psi_r, LSCV, SCV and PI of a binned dataset as differentiable functions
of H for torch.autograd.

H is a float tensor of shape (d, d) or (nH, d, d) on any device, symmetric
(the library checks it to 1e-12 relative).  Gradients are with respect to the
d^2 entries of H taken as independent.  psi_r's backward is the library's
adjoint (kdefft_psi_grad: psi_{r+2} by the Gaussian's heat equation, for
r + 2 within the order limit); the objectives' backward takes the exact
gradients the library returns with their values, whose off-diagonal entries
(derivatives along E_ab + E_ba) split evenly between H_ab and H_ba.

Every evaluation runs in the CUDA library through the C ABI; this module only
marshals tensors.
"""
import numpy as np
import torch

__all__ = ["psi", "lscv", "scv", "pi"]


def _batch(H):
    Hn = H.detach().to("cpu", torch.float64).numpy()
    single = Hn.ndim == 2
    return np.ascontiguousarray(Hn.reshape((-1,) + Hn.shape[-2:])), single


def _tied_share(d, device):
    """The library's off-diagonal gradient entries are derivatives along
    E_ab + E_ba; each of the two independent entries H_ab, H_ba carries half
    of it (1 on the diagonal, 1/2 off it)."""
    return torch.full((d, d), 0.5, dtype=torch.float64, device=device).fill_diagonal_(1.0)


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
        ctx.save_for_backward(torch.from_numpy(g).to(H.device))
        out = torch.from_numpy(np.ascontiguousarray(v)).to(device=H.device, dtype=H.dtype)
        return out[0] if single else out

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        gH = grad_out.to(g.dtype).reshape(-1, 1, 1) * (g * _tied_share(g.shape[-1], g.device))
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
        Hs, _ = _batch(H)
        go = grad_out.detach().to("cpu", torch.float64).numpy()
        gH = torch.from_numpy(ctx.ds.psi_grad(Hs, ctx.r, go)).to(device=H.device, dtype=grad_out.dtype)
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
