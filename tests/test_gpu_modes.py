"""Wittrick-Williams counts on the GPU (masw_mode_count, the arithmetic of the
mode-count search) against the oracle, point by point: s = the number of
negative eigenvalues of the oracle's dense K (numpy's symmetric eigensolver)
and J0 = the sum over layers of the oracle's brute-force clamped-mode count
(each layer cut into pole-free sublayers, dense eigenvalues). Both sides
decide these integers in FP64; they must agree on >= 99.9 % of the points
(a point within rounding of a root or a pole may differ) and within one on
all."""
import math

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def masw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import masw as M
    M.load()
    return M


def sample_points(oracle_lib, m, g, n, seed, max_sub=120):
    """Random (item, c) with V[0] <= c < beta_halfspace, inside the oracle's
    domain, and the oracle's (s, J0) there."""
    rng = np.random.default_rng(seed)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    items, cs, s_ref, j_ref = [], [], [], []
    while len(items) < n:
        it = int(rng.integers(m.n_items))
        h, a, b, r, _ = m.model(item_model[it])
        k = 2.0 * math.pi / m.lam[it]
        if (len(h) and k * h.max() > oracle_lib.MAX_KH) or b[-1] <= g.c0:
            continue
        c = float(rng.uniform(g.c0, b[-1]))
        j0 = [oracle_lib.clamped_modes(k, c, h[i], a[i], b[i], r[i], max_sub) for i in range(len(h))]
        if min(j0, default=0) < 0:
            continue
        items.append(it)
        cs.append(c)
        s_ref.append(oracle_lib.negative_eigenvalues(h, a, b, r, k, c))
        j_ref.append(sum(j0))
    return (np.array(items, np.int32), np.array(cs), np.array(s_ref), np.array(j_ref))


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_mode_counts_match_the_oracle(masw, oracle_lib, which):
    if which == "uniform":
        m, g = W.uniform_batch(n_models=16, n_lambda=20)
    elif which == "ragged":
        m, g = W.ragged_batch(n_models=24, lambdas=(10, 20))
    else:
        m, g = W.extreme_batch(n_models=48, n_lambda=8, seed=W.SEED + 12)
    items, cs, s_ref, j_ref = sample_points(oracle_lib, m, g, 300, seed=21)
    with masw.Batch(m, g) as b:
        s, j0 = b.mode_count(items, cs)
    assert (s >= 0).all() and (j0 >= 0).all()
    same = (s == s_ref) & (j0 == j_ref)
    assert same.mean() >= 0.999, np.nonzero(~same)[0][:10]
    assert np.abs(s - s_ref).max() <= 1 and np.abs(j0 - j_ref).max() <= 1
    assert (j_ref > 0).sum() >= 60 and (s_ref > 0).sum() >= 60


def test_out_of_range_points_and_device_buffers(masw):
    torch = pytest.importorskip("torch")
    m, g = W.uniform_batch(n_models=2, n_lambda=3)
    with masw.Batch(m, g) as b:
        s, j0 = b.mode_count(np.array([0, 1, -1, 99], np.int32), np.array([-5.0, 1e6, 100.0, 100.0]))
        assert (s == -1).all() and (j0 == -1).all()
        items = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
        cs = torch.tensor([60.0, 120.0, 180.0], dtype=torch.float64, device="cuda")
        ds = torch.empty(3, dtype=torch.int32, device="cuda")
        dj = torch.empty(3, dtype=torch.int32, device="cuda")
        masw.mode_count(b.handle, items, cs, ds, dj)
        torch.cuda.synchronize()
        hs, hj = b.mode_count(items.cpu().numpy(), cs.cpu().numpy())
        assert np.array_equal(ds.cpu().numpy(), hs) and np.array_equal(dj.cpu().numpy(), hj)
