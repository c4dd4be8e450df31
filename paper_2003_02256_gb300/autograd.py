"""torch.autograd.Function over the adjoint misfit gradient of libmasw.

``MaswMisfit.apply(beta, h, batch, ce, kind, sigma)`` returns the misfit of
every model of ``batch`` (a ``masw.Batch``) at the refined roots C*, as a
function of the S speeds ``beta`` (sum(N_m + 1) values) and thicknesses
``h`` (sum(N_m)) with each layer's Poisson ratio and density held. The
forward pass uploads (beta, h) with masw_model_batch_update_beta_h and calls
masw_misfit_grad, which evaluates the curves and the exact gradient
d(misfit)/d(beta, h) in one go (implicit-function rule at C*); backward only
scales that gradient by the incoming gradient of each model's misfit.
"""
from __future__ import annotations

import numpy as np
import torch

from . import masw


class MaswMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, h, batch, ce, kind=masw.MISFIT_LSQ, sigma=2.0):
        if beta.dtype != torch.float64 or h.dtype != torch.float64:
            raise TypeError("beta and h must be float64")
        dev = beta.device
        b = beta.detach().contiguous()
        hh = h.detach().contiguous()
        masw.model_batch_update_beta_h(batch.handle, hh, b)
        ce_t = torch.as_tensor(ce, dtype=torch.float64, device=dev).contiguous()
        phi = torch.empty(batch.n_models, dtype=torch.float64, device=dev)
        gb = torch.empty_like(b)
        gh = torch.empty(max(hh.numel(), 1), dtype=torch.float64, device=dev)
        masw.misfit_grad(batch.handle, ce_t, kind, sigma, phi, gb, gh)
        nl = np.asarray(batch.models.n_layers, dtype=np.int64)
        rec_model = torch.as_tensor(np.repeat(np.arange(nl.size), nl + 1), device=dev)
        h_model = torch.as_tensor(np.repeat(np.arange(nl.size), nl), device=dev)
        ctx.save_for_backward(gb, gh[:hh.numel()], rec_model, h_model)
        return phi

    @staticmethod
    def backward(ctx, gphi):
        gb, gh, rec_model, h_model = ctx.saved_tensors
        return gphi[rec_model] * gb, gphi[h_model] * gh, None, None, None, None


def misfit(beta, h, batch, ce, kind=masw.MISFIT_LSQ, sigma=2.0):
    return MaswMisfit.apply(beta, h, batch, ce, kind, sigma)
