"""torch.autograd over the adjoint misfit gradient (differentiation workload).

Checks the backward pass per component (1e-5 relative, tests/gradcheck.py)
against the oracle's gradient of the same weighted misfit, and against
central finite differences of the forward pass itself (relative step 1e-4).
The forward's roots are refined to a relative bracket of 1e-13, which puts
up to ~1e-5 relative noise on single difference quotients, so that second
check is held to 1e-5 of the largest component. Also: a few gradient steps
lower the misfit of a perturbed model toward the true one.
"""
import numpy as np
import pytest

from gradcheck import assert_grad_close, root_grad_reference
from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import autograd, masw
    masw.load()
    return torch, masw, autograd


def _ce_from_oracle(oracle_lib, true, g):
    ht, at, bt, rt, lt = true.model(0)
    _, idx, _ = oracle_lib.dispersion(true.as_dict(), g.c0, g.dc, g.n_c)
    return np.array([oracle_lib.root(ht, at, bt, rt, l, g.c0, g.dc, g.n_c, int(i))
                     for l, i in zip(lt, idx)])


def test_backward_matches_finite_differences_of_forward(env, oracle_lib):
    torch, masw, autograd = env
    m, g, true = W.differentiation_batch(n_models=2, n_lambda=10)
    ce = np.tile(W.noisy_observation(_ce_from_oracle(oracle_lib, true, g), 2.0), m.n_models)
    with masw.Batch(m, g) as b:
        beta = torch.tensor(m.beta, device="cuda", requires_grad=True)
        h = torch.tensor(m.h, device="cuda", requires_grad=True)
        phi = autograd.misfit(beta, h, b, ce)
        w = torch.tensor([1.0, -0.5], dtype=torch.float64, device="cuda")
        (phi * w).sum().backward()
        gb, gh = beta.grad.cpu().numpy(), h.grad.cpu().numpy()

        def f(bv, hv):
            with torch.no_grad():
                p = autograd.misfit(torch.tensor(bv, device="cuda"), torch.tensor(hv, device="cuda"), b, ce)
            return float((p * w).sum())

        fd_b = np.zeros_like(gb)
        for i in range(m.beta.size):
            d = 1e-4 * m.beta[i]
            bp, bm = m.beta.copy(), m.beta.copy()
            bp[i] += d
            bm[i] -= d
            fd_b[i] = (f(bp, m.h) - f(bm, m.h)) / (2 * d)
        fd_h = np.zeros_like(gh)
        for i in range(m.h.size):
            d = 1e-4 * m.h[i]
            hp, hm = m.h.copy(), m.h.copy()
            hp[i] += d
            hm[i] -= d
            fd_h[i] = (f(m.beta, hp) - f(m.beta, hm)) / (2 * d)
        f(m.beta, m.h)  # the batch back on the unperturbed model
        _, idx, st = b.dispersion()
    fd = np.r_[fd_b, fd_h]
    got = np.r_[gb, gh]
    assert np.abs(got - fd).max() <= 1e-5 * np.abs(fd).max()
    # per component against the oracle's gradient of the same weighted misfit
    assert (st == 0).all()
    hoff, loff, woff = m.layer_offsets()
    ref_b = np.zeros_like(gb)
    ref_h = np.zeros_like(gh)
    for k in range(m.n_models):
        hk, ak, bk, rk, lam = m.model(k)
        N = hk.size
        for j in range(lam.size):
            it = woff[k] + j
            c = oracle_lib.root(hk, ak, bk, rk, lam[j], g.c0, g.dc, g.n_c, int(idx[it]))
            dc = root_grad_reference(oracle_lib, hk, ak, bk, rk, lam[j], g, idx[it])
            wgt = float(w[k]) * (c - ce[it]) / 4.0  # LSQ misfit, sigma = 2
            ref_b[loff[k]:loff[k + 1]] += wgt * dc[:N + 1]
            ref_h[hoff[k]:hoff[k + 1]] += wgt * dc[N + 1:]
    for k in range(m.n_models):
        assert_grad_close(np.r_[gb[loff[k]:loff[k + 1]], gh[hoff[k]:hoff[k + 1]]],
                          np.r_[ref_b[loff[k]:loff[k + 1]], ref_h[hoff[k]:hoff[k + 1]]], where=k)


def test_gradient_steps_reduce_the_misfit(env, oracle_lib):
    torch, masw, autograd = env
    m, g, true = W.differentiation_batch(n_models=1, n_lambda=30, spread=0.03)
    ce = _ce_from_oracle(oracle_lib, true, g)
    with masw.Batch(m, g) as b:
        beta = torch.tensor(m.beta, device="cuda", requires_grad=True)
        h = torch.tensor(m.h, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([{"params": [beta], "lr": 1.0}, {"params": [h], "lr": 0.02}])
        first = None
        for it in range(25):
            opt.zero_grad()
            phi = autograd.misfit(beta, h, b, ce, masw.MISFIT_LSQ, 2.0).sum()
            phi.backward()
            opt.step()
            with torch.no_grad():
                h.clamp_(min=0.3)
            first = float(phi.detach()) if first is None else first
        last = float(autograd.misfit(beta.detach(), h.detach(), b, ce).sum())
    assert last < 0.5 * first
