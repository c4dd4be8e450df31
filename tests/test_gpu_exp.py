"""The library's FP64 exponential (e^x, x <= 0) against exact values and
against CUDA's exp: within 1 ulp of the exact value on a sample checked with
60-digit mpmath, and within 2 ulp of CUDA's exp on a dense sweep of
[-708, 0]; 0 below -708. Its sine and cosine on [0, 5 pi / 4] (the
clamped-layer count's range) the same way: within 2 ulp of the exact values,
within 3 ulp of CUDA's sincos."""
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


def test_sincos_within_two_ulp_of_exact(masw):
    rng = np.random.default_rng(7)
    hi = 5.0 * math.pi / 4.0
    x = np.concatenate([rng.uniform(0.0, hi, 1500), rng.uniform(0.0, 1e-3, 200),
                        math.pi / 2 + rng.uniform(-1e-6, 1e-6, 100),
                        math.pi + rng.uniform(-1e-6, 0.0, 100),
                        [0.0, 1e-300, math.pi / 4, math.pi / 2, 3 * math.pi / 4, math.pi,
                         np.nextafter(math.pi, 0.0)]])
    s, c, _, _ = masw.sincos_check(x)
    with mp.workdps(40):
        es = np.array([float(mp.sin(mp.mpf(float(v)))) for v in x])
        ec = np.array([float(mp.cos(mp.mpf(float(v)))) for v in x])
    ds, dc = ulp_distance(s, es), ulp_distance(c, ec)
    assert ds.max() <= 2, (ds.max(), x[np.argmax(ds)])
    assert dc.max() <= 2, (dc.max(), x[np.argmax(dc)])
    z = np.nonzero(x == 0.0)[0]
    assert (s[z] == 0.0).all() and (c[z] == 1.0).all()


def test_sincos_against_cuda_on_a_dense_sweep(masw):
    x = np.linspace(0.0, 5.0 * math.pi / 4.0, 400001)
    s, c, sc, cc = masw.sincos_check(x)
    ds, dc = ulp_distance(s, sc), ulp_distance(c, cc)
    assert ds.max() <= 3, (ds.max(), x[np.argmax(ds)])
    assert dc.max() <= 3, (dc.max(), x[np.argmax(dc)])
