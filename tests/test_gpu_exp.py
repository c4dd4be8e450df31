"""The library's FP64 exponential (e^x, x <= 0) against exact values and
against CUDA's exp: within 1 ulp of the exact value on a sample checked with
60-digit mpmath, and within 2 ulp of CUDA's exp on a dense sweep of
[-708, 0]; 0 below -708."""
import math

import mpmath as mp
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def masw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import masw as M
    M.load()
    return M


def ulp_distance(a, b):
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    return np.abs(ia - ib)


def test_exp_against_cuda_on_a_dense_sweep(masw):
    rng = np.random.default_rng(5)
    x = np.concatenate([-np.linspace(0.0, 708.0, 400001), -rng.uniform(0.0, 40.0, 200000),
                        -rng.uniform(0.0, 1e-3, 10000), [-1e-300, -0.0]])
    y, yc = masw.exp_check(x)
    d = ulp_distance(y, yc)
    assert d.max() <= 2, (d.max(), x[np.argmax(d)])
    assert (y[x == 0.0] == 1.0).all()
    y2, _ = masw.exp_check(np.array([-708.5, -750.0, -1e4]))
    assert (y2 == 0.0).all()


def test_exp_within_one_ulp_of_exact(masw):
    rng = np.random.default_rng(6)
    x = -np.concatenate([rng.uniform(0, 708, 1500), rng.uniform(0, 2, 500)])
    y, _ = masw.exp_check(x)
    with mp.workdps(40):
        exact = np.array([float(mp.exp(mp.mpf(float(v)))) for v in x])
    assert ulp_distance(y, exact).max() <= 1
