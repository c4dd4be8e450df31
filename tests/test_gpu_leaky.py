"""Leaky continuation (masw_dispersion_leaky): Algorithm 1 over the whole
grid with the sign of Re det K (complex half-space block at and above its
shear speed). Parity with the oracle's whole-grid scan
(tests/test_oracle_leaky.py pins it) at the index bar of the batch path:
equal on >= 99.9 % of items, within one grid step on all, statuses equal;
items masw_dispersion resolves keep its result exactly."""
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


def oracle_leaky(oracle_lib, models, grid, items):
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    out = []
    for it in items:
        h, a, b, r, _ = models.model(item_model[it])
        out.append(oracle_lib.scan_leaky(h, a, b, r, models.lam[it], grid.c0, grid.dc, grid.n_c))
    return (np.array([o[1] for o in out]), np.array([o[2] for o in out]),
            np.array([o[0] for o in out]))


def assert_parity(g_idx, g_st, o_idx, o_st, frac=0.999):
    assert (g_st == o_st).all(), np.nonzero(g_st != o_st)
    ok = o_st == 0
    d = np.abs(g_idx[ok].astype(np.int64) - o_idx[ok])
    assert d.max(initial=0) <= 1, d.max()
    assert (d == 0).mean() >= frac if d.size else True
    assert (g_idx[~ok] == -1).all()


@pytest.mark.parametrize("which", ["uniform", "ragged"])
def test_small_batches_match_oracle_everywhere(masw, oracle_lib, which):
    if which == "uniform":
        m, g = W.leaky_batch(n_models=24, n_lambda=40)
    else:
        m, _ = W.ragged_batch(n_models=24, lambdas=(20, 40))
        g = W.Grid(500.0, 0.25, 3001)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.leaky()
        ct1, idx1, st1 = b.dispersion()
    o_ct, o_idx, o_st = oracle_leaky(oracle_lib, m, g, range(m.n_items))
    assert_parity(idx, st, o_idx, o_st)
    # items Algorithm 1 resolves below the half-space speed keep its result
    assert np.array_equal(idx[st1 == 0], idx1[st1 == 0])
    # and some are resolved only by the continuation
    assert ((st1 == 1) & (st == 0)).sum() >= 10
    found = st == 0
    assert np.allclose(ct[found], g.c0 + g.dc * idx[found], rtol=0, atol=1e-9)
    assert np.isnan(ct[~found]).all()


def test_full_size_sampled_against_oracle(masw, oracle_lib):
    m, g = W.leaky_batch()
    with masw.Batch(m, g) as b:
        ct, idx, st = b.leaky()
        _, idx1, st1 = b.dispersion()
    assert np.array_equal(idx[st1 == 0], idx1[st1 == 0])
    assert (st == 0).mean() > 0.99
    items = np.random.default_rng(12).choice(m.n_items, size=600, replace=False)
    _, o_idx, o_st = oracle_leaky(oracle_lib, m, g, items)
    assert_parity(idx[items], st[items], o_idx, o_st)


def test_grid_below_the_half_space_speed_is_algorithm_1(masw):
    m, g = W.uniform_batch(n_models=64)
    with masw.Batch(m, g) as b:
        assert all(np.array_equal(x, y) for x, y in zip(b.leaky()[1:], b.dispersion()[1:]))


def test_extreme_models_sampled_against_oracle(masw, oracle_lib):
    m, g = W.extreme_batch(n_models=128, seed=W.SEED + 10)
    g = W.Grid(200.0, 1.0, 3000)
    with masw.Batch(m, g) as b:
        _, idx, st = b.leaky()
    hmax = np.array([m.model(q)[0].max() for q in range(m.n_models)])
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    inside = np.nonzero(2 * np.pi / m.lam * hmax[item_model] <= oracle_lib.MAX_KH)[0]
    items = np.random.default_rng(13).choice(inside, size=300, replace=False)
    _, o_idx, o_st = oracle_leaky(oracle_lib, m, g, items)
    assert_parity(idx[items], st[items], o_idx, o_st)


def test_edges_and_device_outputs(masw, oracle_lib):
    torch = pytest.importorskip("torch")
    # a bare half-space (no change above its Rayleigh root), a model whose
    # half-space is slower than the grid start (all points complex), a
    # one-layer model; one-point grid tail
    m = W.Models(np.array([0, 1, 2], np.int32), np.array([5.0, 3.0, 6.0]),
                 np.array([520.0, 400.0, 700.0, 450.0, 900.0, 1500.0]),
                 np.array([300.0, 150.0, 260.0, 170.0, 380.0, 700.0]),
                 np.array([2000.0, 1800.0, 1900.0, 1800.0, 1900.0, 2100.0]),
                 np.array([3, 4, 5], np.int32),
                 np.array([5.0, 20.0, 80.0, 2.0, 6.0, 15.0, 40.0, 3.0, 9.0, 27.0, 81.0, 200.0]))
    for g in (W.Grid(100.0, 1.0, 1500), W.Grid(280.0, 0.5, 2001), W.Grid(100.0, 1.0, 2)):
        with masw.Batch(m, g) as b:
            ct, idx, st = b.leaky()
            o_ct, o_idx, o_st = oracle_leaky(oracle_lib, m, g, range(m.n_items))
            assert np.array_equal(idx, o_idx) and np.array_equal(st, o_st), (g, idx, o_idx)
            d_ct = torch.empty(m.n_items, dtype=torch.float64, device="cuda")
            d_idx = torch.empty(m.n_items, dtype=torch.int32, device="cuda")
            d_st = torch.empty_like(d_idx)
            masw.dispersion_leaky(b.handle, d_ct, d_idx, d_st)
            torch.cuda.synchronize()
            assert np.array_equal(d_idx.cpu().numpy(), idx)
            assert np.array_equal(d_st.cpu().numpy(), st)
    # the bare half-space finds its Rayleigh root and nothing above it
    g = W.Grid(300.0, 1.0, 1500)
    with masw.Batch(m.subset([0]), g) as b:
        _, idx, st = b.leaky()
    assert (st == 1).all()


def test_invalid_arguments_of_the_new_entry_points(masw):
    """Argument errors come back as MASW_EINVAL without touching the batch."""
    import ctypes
    m, g = W.uniform_batch(n_models=2, n_lambda=3)
    lib = masw.load()
    with masw.Batch(m, g) as b:
        h = ctypes.c_void_p(b.handle)
        assert lib.masw_dispersion_leaky(h, None, None, None, 7) == masw.EINVAL
        assert lib.masw_dispersion_leaky(None, None, None, None, 0) == masw.EINVAL
        assert lib.masw_mode_count(h, -1, None, None, None, None) == masw.EINVAL
        assert lib.masw_mode_count(h, 2, None, None, None, None) == masw.EINVAL
        assert lib.masw_mode_count(h, 0, None, None, None, None) == 0
        assert lib.masw_last_changes_linear(h, None) == masw.EINVAL
        n = ctypes.c_int32(99)
        assert lib.masw_last_changes_linear(h, ctypes.byref(n)) == 0 and n.value == -1
        ct, idx, st = b.leaky()  # still usable
        assert (st == 0).all()


def test_double_float_continuation_equals_the_fp64_one(masw, oracle_lib):
    """The default plan locates the continued change with the element and
    the Schur step in double-float (det_sign_leaky_dd), confirms it with the
    FP64 step at it and the two points below (det_sign_leaky_df) and scans
    the items it does not confirm again in FP64; plan precision 0 scans with
    the FP64 element and step (det_sign_leaky). On the full leaky batch they agree item for
    item but for sign decisions within rounding of zero: at most 0.01 % of
    items differ, and where they do, both lie within one grid step of the
    oracle's index (the test prints which of the two equals it)."""
    m, g = W.leaky_batch()
    with masw.Batch(m, g) as b:
        _, idx_dd, st_dd = b.leaky()
        b.set_plan(precision=0)
        _, idx64, st64 = b.leaky()
    assert np.array_equal(st_dd, st64)
    diff = np.nonzero(idx_dd != idx64)[0]
    print(f"{diff.size} of {m.n_items} items differ")
    assert diff.size <= 1e-4 * m.n_items
    if diff.size:
        _, o_idx, o_st = oracle_leaky(oracle_lib, m, g, diff)
        print("double-float / FP64 / oracle:", list(zip(idx_dd[diff], idx64[diff], o_idx)))
        assert (o_st == 0).all()
        assert (np.abs(idx_dd[diff] - o_idx) <= 1).all() and (np.abs(idx64[diff] - o_idx) <= 1).all()


def test_forced_rescan_gives_the_fp64_continuation(masw):
    """Test routing 3 sends every continued item, after its double-float scan
    and check, to the FP64 rescan: the results are the FP64 continuation's
    (plan precision 0), so the rescan path runs whatever the check finds."""
    m, g = W.leaky_batch(n_models=64, n_lambda=40)
    with masw.Batch(m, g) as b:
        b.set_plan(precision=0)
        ref = b.leaky()
        b.set_plan(precision=2)
        b.set_route(3)
        got = b.leaky()
        b.set_route(0)
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    assert (ref[2] == 0).mean() > 0.9
