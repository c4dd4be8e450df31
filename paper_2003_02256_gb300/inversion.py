"""Inversion loops around the batched dispersion curves.

MASW fits a layered model to an observed curve C_e by repeatedly evaluating
theoretical curves (Section 1; Section 2.1: the misfit "behaves as a loss
function", minimised by exhaustive evaluation because there is no gradient).
Two loops run many independent inversions at once, one per model of a batch:

* ``gradient_inversion``: descent on log(beta), log(h) with Adam, driven by
  the exact adjoint gradient of the least-squares misfit at the refined roots
  (``MaswMisfit``);
* ``metropolis``: random-walk Metropolis sampling of the posterior
  exp(-Phi_lsq) over (beta, h), one chain per model, every step evaluated for
  all chains in one ``masw_misfit`` call.

Each layer keeps its Poisson ratio and density (alpha moves with beta).
"""
from __future__ import annotations

import numpy as np
import torch

from . import masw
from .autograd import misfit as misfit_fn


def gradient_inversion(batch, ce, iters: int = 50, lr: float = 0.02, sigma: float = 2.0,
                       h_min: float = 0.3, beta_min: float = 50.0):
    """Adam on (log beta, log h) of every model of ``batch`` (a masw.Batch).

    Returns (beta, h, history) with history[i] = per-model misfit before
    step i (numpy, float64)."""
    m = batch.models
    dev = "cuda"
    lb = torch.tensor(np.log(m.beta), device=dev, requires_grad=True)
    lh = torch.tensor(np.log(np.maximum(m.h, h_min)), device=dev, requires_grad=True)
    ce_t = torch.as_tensor(np.ascontiguousarray(ce), dtype=torch.float64, device=dev)
    opt = torch.optim.Adam([lb, lh], lr=lr)
    history = []
    for _ in range(iters):
        opt.zero_grad()
        phi = misfit_fn(torch.exp(lb), torch.exp(lh), batch, ce_t, masw.MISFIT_LSQ, sigma)
        history.append(phi.detach().cpu().numpy())
        phi.sum().backward()
        opt.step()
        with torch.no_grad():
            lb.clamp_(min=float(np.log(beta_min)))
            lh.clamp_(min=float(np.log(h_min)))
    return torch.exp(lb).detach(), torch.exp(lh).detach(), np.array(history)


def metropolis(batch, ce, steps: int = 200, step_frac: float = 0.02, sigma: float = 2.0,
               seed: int = 0, h_min: float = 0.3, beta_min: float = 50.0):
    """Random-walk Metropolis, one chain per model of ``batch``: each step
    perturbs every beta_i and h_i by N(0, step_frac^2) relative, evaluates all
    chains' misfits Phi = sum (C_t - C_e)^2 / (2 sigma^2) in one batched call
    and accepts with probability min(1, exp(Phi_old - Phi_new)).

    Returns (beta, h, phi, acceptance_rate) of the final states."""
    m = batch.models
    dev = "cuda"
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    nl = np.asarray(m.n_layers, dtype=np.int64)
    rec_model = torch.as_tensor(np.repeat(np.arange(nl.size), nl + 1), device=dev)
    h_model = torch.as_tensor(np.repeat(np.arange(nl.size), nl), device=dev)
    beta = torch.tensor(m.beta, dtype=torch.float64, device=dev)
    h = torch.tensor(np.maximum(m.h, h_min), dtype=torch.float64, device=dev)
    ce_t = torch.as_tensor(np.ascontiguousarray(ce), dtype=torch.float64, device=dev)
    phi = torch.empty(batch.n_models, dtype=torch.float64, device=dev)

    def evaluate(b, hh, out):
        masw.model_batch_update_beta_h(batch.handle, hh, b)
        masw.misfit(batch.handle, ce_t, masw.MISFIT_LSQ, sigma, out)
        return torch.nan_to_num(out, nan=float("inf"))

    cur = evaluate(beta, h, phi).clone()
    accepted = torch.zeros(batch.n_models, dtype=torch.float64, device=dev)
    new_phi = torch.empty_like(phi)
    for _ in range(steps):
        nb = beta * (1.0 + step_frac * torch.randn(beta.shape, generator=g, device=dev,
                                                   dtype=torch.float64))
        nh = h * (1.0 + step_frac * torch.randn(h.shape, generator=g, device=dev,
                                                dtype=torch.float64))
        nb = torch.clamp(nb, min=beta_min)
        nh = torch.clamp(nh, min=h_min)
        prop = evaluate(nb, nh, new_phi)
        u = torch.rand(batch.n_models, generator=g, device=dev, dtype=torch.float64)
        acc = torch.log(u) < (cur - prop)
        accepted += acc.double()
        beta = torch.where(acc[rec_model], nb, beta)
        h = torch.where(acc[h_model], nh, h)
        cur = torch.where(acc, prop, cur)
    # leave the batch holding the final states
    evaluate(beta, h, phi)
    return beta, h, cur, (accepted / steps).cpu().numpy()
