"""Higher modes (masw_dispersion_changes): Algorithm 1 carried past its first
sign change, each change labelled with the change in K's negative-eigenvalue
count. Parity with the oracle's continued scan (tests/test_oracle_changes.py
pins it): change indices equal on >= 99.9 % of (item, change) entries and
within one grid step on all, labels equal where the indices are; the first
change equals masw_dispersion's index exactly. The full-size samples include
root-pole pairs inside one grid interval (an FP32 screen loses those)."""
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


def oracle_changes(oracle_lib, models, grid, items, M):
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    idx = np.empty((len(items), M), dtype=np.int32)
    dl = np.empty((len(items), M), dtype=np.int32)
    for r, it in enumerate(items):
        h, a, b, rr, _ = models.model(item_model[it])
        _, idx[r], dl[r] = oracle_lib.scan_changes(h, a, b, rr, models.lam[it], grid.c0, grid.dc,
                                                   grid.n_c, M)
    return idx, dl


def assert_changes_parity(g_idx, g_st, g_dl, o_idx, o_dl, frac=0.999):
    o_st = np.where(o_idx >= 0, 0, 1)
    assert (g_st == o_st).mean() >= frac
    both = (g_idx >= 0) & (o_idx >= 0)
    d = np.abs(g_idx[both].astype(np.int64) - o_idx[both])
    assert d.max(initial=0) <= 1
    assert (d == 0).mean() >= frac if d.size else True
    same = both & (g_idx == o_idx)
    assert (g_dl[same] == o_dl[same]).all()
    assert (g_idx[g_st == 1] == -1).all() and (g_dl[g_st == 1] == 0).all()


def test_single_curve_changes_match_oracle(masw, oracle_lib):
    m, g = W.single_curve()
    M = 6
    with masw.Batch(m, g) as b:
        ct, idx, st, dl = b.changes(M)
        _, idx1, st1 = b.dispersion()
    o_idx, o_dl = oracle_changes(oracle_lib, m, g, range(m.n_items), M)
    assert np.array_equal(idx, o_idx) and np.array_equal(dl, o_dl)
    assert np.array_equal(idx[:, 0], np.where(st1 == 0, idx1, -1))
    found = idx >= 0
    assert np.allclose(ct[found], g.c0 + g.dc * idx[found]) and np.isnan(ct[~found]).all()
    assert (dl[:, 0][st[:, 0] == 0] == 1).all()  # the fundamental mode is a root
    assert (dl == -1).any() and (dl == 1).sum() > m.n_items  # poles and higher modes occur


@pytest.mark.parametrize("which", ["uniform", "ragged"])
def test_small_batches_match_oracle(masw, oracle_lib, which):
    if which == "uniform":
        m, g = W.uniform_batch(n_models=12, n_lambda=40)
    else:
        m, g = W.ragged_batch(n_models=16, lambdas=(20, 40))
    M = 4
    with masw.Batch(m, g) as b:
        _, idx, st, dl = b.changes(M)
    o_idx, o_dl = oracle_changes(oracle_lib, m, g, range(m.n_items), M)
    assert_changes_parity(idx, st, dl, o_idx, o_dl)


@pytest.mark.parametrize("which", ["uniform", "ragged"])
def test_full_size_first_change_and_sampled_oracle(masw, oracle_lib, which):
    m, g = W.uniform_batch() if which == "uniform" else W.ragged_batch()
    M = 3
    with masw.Batch(m, g) as b:
        _, idx, st, dl = b.changes(M)
        _, idx1, st1 = b.dispersion()
    assert np.array_equal(idx[:, 0], np.where(st1 == 0, idx1, -1))
    # changes are increasing, padded at the end
    valid = idx >= 0
    both = valid[:, 1:] & valid[:, :-1]
    assert (np.diff(idx, axis=1)[both] > 0).all()
    assert not (valid[:, 1:] & ~valid[:, :-1]).any()
    rng = np.random.default_rng(3)
    items = rng.choice(m.n_items, size=150, replace=False)
    o_idx, o_dl = oracle_changes(oracle_lib, m, g, items, M)
    assert_changes_parity(idx[items], st[items], dl[items], o_idx, o_dl)



def test_extreme_models_changes(masw, oracle_lib):
    """Models outside the paper's ranges (thin stiff layers, low-velocity
    layers, up to 30 layers): the first change is the batch scan's index and a
    sample of (item, change) entries matches the oracle's continued scan."""
    m, g = W.extreme_batch(n_models=128, seed=W.SEED + 9)
    M = 4
    with masw.Batch(m, g) as b:
        _, idx, st, dl = b.changes(M)
        _, idx1, st1 = b.dispersion()
    assert np.array_equal(idx[:, 0], np.where(st1 == 0, idx1, -1))
    assert set(np.unique(dl)) <= {-1, 0, 1}
    hmax = np.array([m.model(q)[0].max() for q in range(m.n_models)])
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    inside = np.nonzero(2 * np.pi / m.lam * hmax[item_model] <= oracle_lib.MAX_KH)[0]
    items = np.random.default_rng(9).choice(inside, size=120, replace=False)
    o_idx, o_dl = oracle_changes(oracle_lib, m, g, items, M)
    assert_changes_parity(idx[items], st[items], dl[items], o_idx, o_dl)

def test_edges_limits_and_device_outputs(masw, oracle_lib):
    torch = pytest.importorskip("torch")
    # grid above the fundamental root, a model with no scannable points, M = 1 and 15
    m = W.Models(np.array([1, 2, 1], np.int32), np.array([6.0, 3.0, 5.0, 2.0]),
                 np.array([400.0, 1700.0, 450.0, 700.0, 1800.0, 300.0, 320.0]),
                 np.array([150.0, 600.0, 170.0, 260.0, 650.0, 100.0, 120.0]),
                 np.full(7, 1900.0), np.array([4, 3, 2], np.int32),
                 np.array([2.0, 4.0, 8.0, 30.0, 3.0, 10.0, 25.0, 5.0, 9.0]))
    g = W.Grid(165.0, 0.5, 1000)
    for M in (1, 15):
        with masw.Batch(m, g) as b:
            _, idx, st, dl = b.changes(M)
            if M == 1:
                _, idx1, st1 = b.dispersion()
                assert np.array_equal(idx[:, 0], np.where(st1 == 0, idx1, -1))
        o_idx, o_dl = oracle_changes(oracle_lib, m, g, range(m.n_items), M)
        assert np.array_equal(idx, o_idx) and np.array_equal(dl, o_dl)
        assert (st[-2:] == 1).all()  # half-space below the grid start: nothing to scan
    with masw.Batch(m, g) as b:
        for bad in (0, masw.MAX_CHANGES + 1):
            with pytest.raises(masw.MaswError) as ei:
                b.changes(bad)
            assert ei.value.code == masw.EINVAL
        M = 5
        d_ct = torch.empty(m.n_items * M, dtype=torch.float64, device="cuda")
        d_idx = torch.empty(m.n_items * M, dtype=torch.int32, device="cuda")
        d_st = torch.empty_like(d_idx)
        d_dl = torch.empty_like(d_idx)
        masw.dispersion_changes(b.handle, M, d_ct, d_idx, d_st, d_dl)
        torch.cuda.synchronize()
        _, idx, st, dl = b.changes(M)
        assert np.array_equal(d_idx.cpu().numpy().reshape(-1, M), idx)
        assert np.array_equal(d_dl.cpu().numpy().reshape(-1, M), dl)


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_counting_search_equals_the_linear_fp64_scan(masw, which):
    """Plan precision 2 (search on the monotone mode count s + 2 J0) against
    precision 0 (FP64 sign and count at every grid point) item for item, all
    M entries and labels, at full size."""
    if which == "uniform":
        m, g = W.uniform_batch()
    elif which == "ragged":
        m, g = W.ragged_batch(n_models=2048)
    else:
        m, g = W.extreme_batch(seed=W.SEED + 11)
    M = 4
    with masw.Batch(m, g) as b:
        b.set_plan(precision=0)
        ref = b.changes(M)
        assert b.last_changes_linear() == -1
        b.set_plan(precision=2)
        got = b.changes(M)
        n_lin = b.last_changes_linear()
    for x, y in zip(got[1:], ref[1:]):
        bad = np.nonzero((x != y).any(axis=1))[0]
        assert bad.size == 0, (which, bad[:10], x[bad[:3]], y[bad[:3]])
    assert 0 <= n_lin <= max(2, m.n_items // 1000), n_lin
