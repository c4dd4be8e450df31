"""Stored expected values under tests/golden/ (written by make_golden.py
from the oracle) stay reproducible, and the CUDA path matches them."""
import os

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "differentiation_true_roots.txt")


def load():
    a = np.loadtxt(GOLD)
    return a[:, 0], a[:, 1].astype(int), a[:, 2]


def test_fixture_reproduces_from_the_oracle(oracle_lib):
    lam, idx, roots = load()
    _, g, true = W.differentiation_batch(n_models=1)
    h, a, b, r, tl = true.model(0)
    # the stored wavelengths are the generator's (printed to 17 digits); a
    # platform's logspace may differ in the last bit
    assert np.allclose(tl, lam, rtol=4e-16, atol=0)
    _, o_idx, _ = oracle_lib.dispersion(true.as_dict(), g.c0, g.dc, g.n_c)
    assert np.array_equal(o_idx, idx)
    for j in range(0, lam.size, 15):
        assert oracle_lib.root(h, a, b, r, lam[j], g.c0, g.dc, g.n_c, int(idx[j])) == \
            pytest.approx(roots[j], rel=1e-13)


@pytest.mark.gpu
def test_cuda_roots_match_the_fixture():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import masw
    lam, idx, roots = load()
    _, g, true = W.differentiation_batch(n_models=1)
    with masw.Batch(true, g) as b:
        ct, gidx, st = b.dispersion()
        croot = b.roots()
    assert np.array_equal(gidx, idx)
    assert np.allclose(croot, roots, rtol=1e-9, atol=0)
