"""Inversion loops around the batched curves: adjoint-driven descent lowers
every model's misfit toward the noise-free observed curve of the true model,
and the batched Metropolis sampler accepts at a sane rate and moves chains
toward higher likelihood."""
import os

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "differentiation_true_roots.txt")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import inversion, masw
    masw.load()
    return masw, inversion


def test_gradient_inversion_lowers_every_misfit(env):
    masw, inversion = env
    m, g, _ = W.differentiation_batch(n_models=8, spread=0.05)
    ce = np.tile(np.loadtxt(GOLD)[:, 2], m.n_models)
    with masw.Batch(m, g) as b:
        beta, h, hist = inversion.gradient_inversion(b, ce, iters=40, lr=0.01)
    first, last = hist[0], hist[-1]
    assert np.isfinite(last).all()
    assert (last < 0.5 * first).mean() >= 0.75
    assert np.median(last / first) < 0.2


def test_metropolis_chains(env):
    masw, inversion = env
    m, g, _ = W.differentiation_batch(n_models=32, spread=0.03, seed=W.SEED + 40)
    ce = np.tile(np.loadtxt(GOLD)[:, 2], m.n_models)
    with masw.Batch(m, g) as b:
        phi0 = b.misfit(ce, kind=masw.MISFIT_LSQ, sigma=2.0)
        beta, h, phi, acc = inversion.metropolis(b, ce, steps=120, step_frac=0.01, seed=3)
        phi_check = b.misfit(ce, kind=masw.MISFIT_LSQ, sigma=2.0)
    phi = phi.cpu().numpy()
    assert np.allclose(phi, phi_check)  # the batch holds the final states
    assert 0.02 < acc.mean() < 0.95
    assert np.median(phi / phi0) < 0.8
