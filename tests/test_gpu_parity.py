"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Bar (floating point decides an integer here): the GPU grid index of the
first sign change equals the oracle's on >= 99.9% of items and differs by at
most one grid step on all of them; per-item status is identical. Both sides
take the sign decision in FP64. Refined roots agree to 1e-9 relative; the
adjoint gradient agrees per component to 1e-5 relative with the oracle's
extrapolated central differences of its refined root (tests/gradcheck.py).
"""
import math

import numpy as np
import pytest

from gradcheck import assert_grad_close, root_grad_reference
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


def oracle_items(oracle_lib, models, grid, items):
    """Oracle scan of selected items, one by one."""
    hoff, loff, woff = models.layer_offsets()
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    out = []
    for it in items:
        m = item_model[it]
        h, a, b, r, _ = models.model(m)
        out.append(oracle_lib.scan(h, a, b, r, models.lam[it], grid.c0, grid.dc, grid.n_c))
    st = np.array([o[0] for o in out])
    ct = np.array([o[1] for o in out])
    idx = np.array([o[2] for o in out])
    return ct, idx, st


def oracle_domain(oracle_lib, models):
    """Items the oracle accepts: k h <= its MAX_KH in every layer (it uses the
    plain, unscaled hyperbolic functions)."""
    hmax = np.array([models.model(q)[0].max() for q in range(models.n_models)])
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    return np.nonzero(2 * np.pi / models.lam * hmax[item_model] <= oracle_lib.MAX_KH)[0]


def assert_index_parity(g_idx, g_st, o_idx, o_st, frac=0.999, explain=None):
    """The parity bar; with explain = (oracle_lib, models, grid, items) every
    index that differs is checked to lie where det K is within rounding of
    zero: at the grid point whose sign the two sides disagree on (the lower
    of the two indices), the oracle's ln|det K| is below both neighbours' by
    more than ln(1e6), i.e. the root is closer to that point than 1e-6 of a
    grid step."""
    assert (g_st == o_st).all(), np.nonzero(g_st != o_st)
    ok = o_st == 0
    d = np.abs(g_idx[ok].astype(np.int64) - o_idx[ok])
    assert d.max(initial=0) <= 1, d.max()
    assert (d == 0).mean() >= frac if d.size else True
    assert (g_idx[~ok] == -1).all()
    if explain is not None:
        oracle_lib, models, grid, items = explain
        item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
        items = np.arange(g_idx.size) if items is None else np.asarray(items)
        for j in np.nonzero(ok & (g_idx != o_idx))[0]:
            it = int(items[j])
            h, a, b, r, _ = models.model(item_model[it])
            k = 2.0 * math.pi / models.lam[it]
            p = int(min(g_idx[j], o_idx[j]))
            la = [oracle_lib.det(h, a, b, r, k, oracle_lib.grid_velocity(grid.c0, grid.dc, n))[1]
                  for n in (p - 1, p, p + 1)]
            assert la[1] < min(la[0], la[2]) - math.log(1e6), (it, p, la)


# ------------------------------------------------------------- full parity

def test_single_curve_matches_oracle_everywhere(masw, oracle_lib):
    m, g = W.single_curve()
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
    assert (st == o_st).all() and (idx == o_idx).all()
    assert np.array_equal(ct, o_ct)


def test_uniform_batch_small_matches_oracle(masw, oracle_lib):
    m, g = W.uniform_batch(n_models=24)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
    assert_index_parity(idx, st, o_idx, o_st, explain=(oracle_lib, m, g, None))
    same = idx == o_idx
    assert np.array_equal(ct[same & (st == 0)], o_ct[same & (st == 0)])


def test_ragged_batch_small_matches_oracle(masw, oracle_lib):
    m, g = W.ragged_batch(n_models=40)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
    assert_index_parity(idx, st, o_idx, o_st, explain=(oracle_lib, m, g, None))


def test_coarse_grid_with_ragged_tail(masw, oracle_lib):
    """A grid whose scan length is not a multiple of the 32-lane chunk."""
    m, _ = W.uniform_batch(n_models=12, n_layers=5, n_lambda=37, lam_max=90.0)
    g = W.Grid(61.3, 0.77, 1013)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        for precision in (0, 1, 2):
            for cpl in (1, 2, 4):
                b.set_plan(cpl=cpl, precision=precision)
                ct, idx, st = b.dispersion()
                assert_index_parity(idx, st, o_idx, o_st, explain=(oracle_lib, m, g, None))


# ------------------------------------------------- full-size workloads

def assert_on_grid(models, grid, ct, idx, st):
    """Properties that hold at any size: C_t is the grid velocity V[idx]."""
    found = st == 0
    assert found.mean() > 0.99
    k = (ct[found] - grid.c0) / grid.dc
    assert np.array_equal(np.round(k), idx[found])


def test_uniform_full_batch_matches_oracle_item_by_item(masw, oracle_lib):
    """Every one of the 204,800 items of the uniform batch (1024 models x 200
    wavelengths, the benchmark's launch) against the oracle's dense-LU scan
    (Algorithm 1, all host cores): >= 99.9 % identical indices, all within
    one grid step, every mismatch at a point where det K is within rounding
    of zero."""
    m, g = W.uniform_batch()
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    diff = int(np.sum((idx != o_idx) | (st != o_st)))
    print(f"uniform batch: {m.n_items} items, {diff} index mismatches against the oracle")
    assert_index_parity(idx, st, o_idx, o_st, explain=(oracle_lib, m, g, None))
    same = (idx == o_idx) & (st == 0)
    assert np.array_equal(ct[same], o_ct[same])
    assert_on_grid(m, g, ct, idx, st)


def test_ragged_batch_model_sample_matches_oracle(masw, oracle_lib):
    """The ragged batch (8192 models, 3..30 layers, 30..400 wavelengths) run
    whole on the GPU, as the benchmark launches it; every item of every
    tenth model (820 models, about 10 % of the items) against the oracle."""
    m, g = W.ragged_batch()
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
    sample = np.arange(0, m.n_models, 10)
    sub = m.subset(sample)
    _, _, woff = m.layer_offsets()
    items = np.concatenate([np.arange(woff[q], woff[q + 1]) for q in sample])
    o_ct, o_idx, o_st = oracle_lib.dispersion(sub.as_dict(), g.c0, g.dc, g.n_c)
    diff = int(np.sum((idx[items] != o_idx) | (st[items] != o_st)))
    print(f"ragged batch: {items.size} sampled items of {sample.size} models, {diff} index "
          "mismatches against the oracle")
    assert_index_parity(idx[items], st[items], o_idx, o_st, explain=(oracle_lib, m, g, items))
    assert_on_grid(m, g, ct, idx, st)


# --------------------------------------------------------- determinants

def test_block_recurrence_matches_dense_lu(masw, oracle_lib):
    m, g = W.ragged_batch(n_models=16)
    rng = np.random.default_rng(12)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    items = rng.integers(0, m.n_items, 3000)
    beta_hs = np.array([m.model(i)[2][-1] for i in range(m.n_models)])
    c = rng.uniform(50.0, beta_hs[item_model[items]] * 0.999)
    with masw.Batch(m, g) as b:
        sign, la = b.det_eval(items, c)
    o_sign = np.empty(items.size, dtype=int)
    o_la = np.empty(items.size)
    for t, (it, cc) in enumerate(zip(items, c)):
        h, a, bb, r, _ = m.model(item_model[it])
        o_sign[t], o_la[t] = oracle_lib.det(h, a, bb, r, 2 * np.pi / m.lam[it], cc)
    rel = np.abs(la - o_la) / np.maximum(1.0, np.abs(o_la))
    # ln|det| agrees closely; the sign agrees wherever |det| is not at rounding level
    assert np.median(rel) < 1e-12
    assert (sign == o_sign).mean() > 0.999


def test_half_space_rayleigh_and_exact_grid_hits(masw, oracle_lib):
    nu = 0.25
    beta = np.array([200.0])
    m = W.Models(np.array([0], np.int32), np.zeros(0), W.alpha_from_nu(beta, nu), beta,
                 np.array([2000.0]), np.array([6], np.int32),
                 np.array([0.5, 1.0, 7.0, 60.0, 150.0, 5000.0]))
    g = W.Grid(50.0, 0.25, 4601)
    cr = 200.0 * math.sqrt(2.0 - 2.0 / math.sqrt(3.0))
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
        croot = b.roots()
    assert (st == 0).all() and (idx == int(math.floor((cr - 50.0) / 0.25)) + 1).all()
    assert np.allclose(croot, cr, rtol=1e-11, atol=0)


def test_no_root_and_empty_models(masw, oracle_lib):
    m = W.Models(np.array([1, 1, 2], np.int32), np.array([3.0, 2.0, 1.0, 4.0]),
                 np.array([500.0, 900.0, 500.0, 900.0, 400.0, 600.0, 900.0]),
                 np.array([200.0, 380.0, 200.0, 380.0, 170.0, 250.0, 390.0]),
                 np.full(7, 1900.0), np.array([2, 0, 3], np.int32),
                 np.array([10.0, 30.0, 1.0, 5.0, 25.0]))
    # grid that stops below most roots -> NO_ROOT for some items
    g = W.Grid(50.0, 1.0, 150)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        for precision in (0, 1, 2):
            b.set_plan(precision=precision)
            ct, idx, st = b.dispersion()
            assert (st == o_st).all() and (idx == o_idx).all(), precision
            assert np.isnan(ct[st == 1]).all()
    assert (o_st == 1).any() and (o_st == 0).any()


def test_grid_starting_above_the_fundamental_root(masw, oracle_lib):
    """V[0] above the fundamental mode: det K already carries one negative
    eigenvalue there, and Algorithm 1 reports the next change (a higher
    mode) or none; the counting search hands such items to the linear
    screen."""
    m = W.Models(np.array([1, 2], np.int32), np.array([6.0, 3.0, 5.0]),
                 np.array([400.0, 1700.0, 450.0, 700.0, 1800.0]),
                 np.array([150.0, 600.0, 170.0, 260.0, 650.0]),
                 np.full(5, 1900.0), np.array([6, 5], np.int32),
                 np.array([2.0, 4.0, 8.0, 12.0, 20.0, 30.0, 3.0, 6.0, 10.0, 18.0, 25.0]))
    g = W.Grid(165.0, 0.5, 1000)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        for precision in (0, 1, 2):
            b.set_plan(precision=precision)
            ct, idx, st = b.dispersion()
            assert (st == o_st).all() and (idx == o_idx).all(), precision
        b.set_plan(precision=2)
        b.dispersion()
        assert b.last_scan_fallback() >= 1


def test_max_layers_model(masw, oracle_lib):
    """128 finite layers (a 258 x 258 stiffness matrix) at 200 wavelengths from
    1 to 150 m, under the counting plan and the FP64 scan: the full parity bar
    (every index equal to the oracle's)."""
    rng = np.random.default_rng(13)
    N = masw.MAX_LAYERS
    h = rng.uniform(0.2, 1.0, N)
    beta = np.cumsum(np.r_[120.0, rng.uniform(1.0, 4.0, N)])
    alpha = W.alpha_from_nu(beta, 0.3)
    rho = np.full(N + 1, 1900.0)
    lam = np.geomspace(1.0, 150.0, 200)
    m = W.Models(np.array([N], np.int32), h, alpha, beta, rho, np.array([lam.size], np.int32), lam)
    g = W.Grid(50.0, 0.5, 2000)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    with masw.Batch(m, g) as b:
        for precision in (2, 0):
            b.set_plan(precision=precision)
            ct, idx, st = b.dispersion()
            assert_index_parity(idx, st, o_idx, o_st, explain=(oracle_lib, m, g, None))
    assert (o_st == 0).all()


def test_invalid_inputs_are_rejected(masw):
    m, g = W.single_curve()
    bad = [dict(h=-m.h), dict(rho=np.zeros_like(m.rho)),
           dict(alpha=m.beta * 1.1), dict(lam=np.r_[np.nan, m.lam[1:]])]
    for kw in bad:
        mm = W.Models(m.n_layers, kw.get("h", m.h), kw.get("alpha", m.alpha), m.beta,
                      kw.get("rho", m.rho), m.n_lambda, kw.get("lam", m.lam))
        with pytest.raises(masw.MaswError) as ei:
            masw.Batch(mm, g)
        assert ei.value.code == masw.EINVAL
    with pytest.raises(masw.MaswError):
        masw.Batch(m, W.Grid(50.0, 0.0, 10))
    big = W.Models(np.array([masw.MAX_LAYERS + 1], np.int32), np.ones(masw.MAX_LAYERS + 1),
                   np.full(masw.MAX_LAYERS + 2, 900.0), np.full(masw.MAX_LAYERS + 2, 300.0),
                   np.full(masw.MAX_LAYERS + 2, 1900.0), np.array([1], np.int32), np.array([5.0]))
    with pytest.raises(masw.MaswError):
        masw.Batch(big, g)


# ------------------------------------------------------- plans and paths

@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("which", ["uniform", "ragged"])
def test_two_precision_scan_equals_the_fp64_scan_at_full_size(masw, which, precision):
    """The FP32 screen (linear, or the counting search) only locates the
    change; every reported index is an FP64 decision, so the plans agree
    with the FP64 scan item for item."""
    m, g = W.uniform_batch() if which == "uniform" else W.ragged_batch()
    with masw.Batch(m, g) as b:
        b.set_plan(precision=precision)
        ct1, idx1, st1 = b.dispersion()
        unresolved = b.last_scan_unresolved()
        fallback = b.last_scan_fallback()
        b.set_plan(precision=0)
        ct0, idx0, st0 = b.dispersion()
    assert np.array_equal(idx1, idx0) and np.array_equal(st1, st0)
    assert np.array_equal(ct1, ct0, equal_nan=True)
    assert 0 <= unresolved < 0.5 * m.n_items
    if precision == 2:
        assert 0 <= fallback < 0.5 * m.n_items
    else:
        assert fallback == -1


def test_split_search_with_shuffled_wavelengths_equals_the_fp64_scan(masw):
    """The second search pass starts from a guess on the line through its
    anchors' indices. With each model's wavelengths in random order the
    guesses miss by up to the whole range; the steps away from them and the
    bisection still give the FP64 scan's index, item for item."""
    import dataclasses

    m, g = W.ragged_batch(n_models=256, seed=91)
    rng = np.random.default_rng(5)
    woff = np.concatenate([[0], np.cumsum(m.n_lambda)])
    lam = m.lam.copy()
    for i in range(m.n_models):
        lam[woff[i]:woff[i + 1]] = rng.permutation(lam[woff[i]:woff[i + 1]])
    m = dataclasses.replace(m, lam=lam)
    with masw.Batch(m, g) as b:
        b.set_plan(precision=0)
        ct0, idx0, st0 = b.dispersion()
        for split in (1, 2):
            b.set_plan(precision=2, count_split=split)
            ct, idx, st = b.dispersion()
            assert np.array_equal(idx, idx0) and np.array_equal(st, st0), split
            assert np.array_equal(ct, ct0, equal_nan=True), split


def test_every_plan_and_the_plain_path_give_identical_indices(masw):
    m, g = W.ragged_batch(n_models=64, seed=77)
    with masw.Batch(m, g) as b:
        ref = b.dispersion()
        plain = b.dispersion(plain=True)
        assert np.array_equal(ref[0], plain[0], equal_nan=True)
        assert np.array_equal(ref[1], plain[1]) and np.array_equal(ref[2], plain[2])
        for plan in (dict(persistent=0), dict(ordered=0), dict(use_graph=0),
                     dict(stage_layers=0), dict(warps_per_block=2, blocks_per_sm=1),
                     dict(cpl=2), dict(cpl=4), dict(precision=0), dict(precision=0, cpl=2),
                     dict(precision=1, persistent=0), dict(precision=2),
                     dict(precision=2, use_graph=0), dict(precision=2, stage_layers=0),
                     dict(precision=2, count_split=1), dict(count_split=1, use_graph=1),
                     dict(count_split=1, count_block=64), dict(count_split=1, count_block=256),
                     dict(precision=2, warps_per_block=1, blocks_per_sm=1, count_split=0,
                          count_block=128),
                     dict(count_split=2, use_graph=0), dict(count_split=2, count_block=64),
                     dict(count_split=2, count_block=256, use_graph=1)):
            b.set_plan(**plan)
            got = b.dispersion()
            assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), plan
        tuned = b.autotune(reps=1)
        assert tuned.persistent in (0, 1)
        got = b.dispersion()
        assert np.array_equal(got[1], ref[1])


def test_scan_phase_timers(masw):
    """masw_last_scan_phases and masw_last_count_phases: the split counting
    plans time their search and certificate kernels separately, inside the
    first phase, and count_split 2 also its fallback chain on the second
    stream; fused, graph-replayed and per-model scans refuse."""
    m, g = W.ragged_batch(n_models=64, seed=77)
    with masw.Batch(m, g) as b:
        for split in (1, 2):
            b.set_plan(precision=2, count_split=split, use_graph=0)
            b.dispersion()
            ph = masw.last_scan_phases(b.handle)
            cp = masw.last_count_phases(b.handle)
            assert min(ph) >= 0.0 and min(cp[:2]) > 0.0
            assert cp[0] + cp[1] <= ph[0] * 1.001 + 1e-3
            if split == 1:
                assert cp[2] == 0.0
            else:
                assert cp[2] > 0.0  # the chain's kernels ran (with or without listed items)
        for plan, plain in ((dict(count_split=0), False), (dict(count_split=1, use_graph=1), False),
                            (dict(count_split=1, use_graph=0), True),
                            (dict(count_split=2, use_graph=1), False),
                            (dict(count_split=2, use_graph=0), True)):
            b.set_plan(**plan)
            b.dispersion(plain=plain)
            with pytest.raises(masw.MaswError):
                masw.last_count_phases(b.handle)
        with pytest.raises(masw.MaswError):
            masw.last_scan_phases(b.handle)


def test_graph_replay_after_update_gives_fresh_results(masw, oracle_lib):
    m1, g = W.uniform_batch(n_models=8, n_layers=6, n_lambda=20)
    m2, _ = W.uniform_batch(n_models=8, n_layers=6, n_lambda=20, seed=5)
    with masw.Batch(m1, g) as b:
        assert b.plan().use_graph == 1
        r1 = b.dispersion()
        b.update(m2.h, m2.alpha, m2.beta, m2.rho)
        r2 = b.dispersion()
    with masw.Batch(m2, g) as fresh:
        rf = fresh.dispersion()
    assert np.array_equal(r2[1], rf[1])
    assert not np.array_equal(r1[1], r2[1])


def test_update_validates_first_and_matches_a_fresh_batch(masw):
    """masw_model_batch_update builds the records on the device: an invalid
    update is refused and leaves the batch as it was; a valid one (host or
    device pointers) gives determinants identical to a fresh batch's."""
    import torch
    m1, g = W.ragged_batch(n_models=12, seed=21)
    m2, _ = W.ragged_batch(n_models=12, seed=21)
    m2 = W.Models(m2.n_layers, m2.h * 1.1, m2.alpha * 0.97, m2.beta * 0.97, m2.rho, m2.n_lambda,
                  m2.lam)
    rng = np.random.default_rng(4)
    items = rng.integers(0, m1.n_items, 64).astype(np.int32)
    cs = rng.uniform(60.0, 300.0, 64)
    with masw.Batch(m1, g) as b:
        before = b.dispersion()
        bad = [dict(h=-m1.h), dict(alpha=m1.beta * 1.1), dict(rho=np.where(np.arange(m1.rho.size) == 3,
                                                                             np.nan, m1.rho))]
        for kw in bad:
            with pytest.raises(masw.MaswError) as ei:
                b.update(kw.get("h", m1.h), kw.get("alpha", m1.alpha), m1.beta, kw.get("rho", m1.rho))
            assert ei.value.code == masw.EINVAL
            after = b.dispersion()
            assert np.array_equal(after[1], before[1]) and np.array_equal(after[2], before[2])
        for kw in bad:  # the same with device pointers (checked on the device)
            dbad = [torch.as_tensor(np.ascontiguousarray(x), device="cuda")
                    for x in (kw.get("h", m1.h), kw.get("alpha", m1.alpha), m1.beta,
                              kw.get("rho", m1.rho))]
            with pytest.raises(masw.MaswError) as ei:
                b.update(*dbad)
            assert ei.value.code == masw.EINVAL
            after = b.dispersion()
            assert np.array_equal(after[1], before[1]) and np.array_equal(after[2], before[2])
        b.update(m2.h, m2.alpha, m2.beta, m2.rho)
        s_host, l_host = b.det_eval(items, cs)
        r_host = b.dispersion()
        dev = [torch.as_tensor(x, device="cuda") for x in (m2.h, m2.alpha, m2.beta, m2.rho)]
        b.update(m1.h, m1.alpha, m1.beta, m1.rho)
        b.update(*dev)
        s_dev, l_dev = b.det_eval(items, cs)
    with masw.Batch(m2, g) as fresh:
        s_f, l_f = fresh.det_eval(items, cs)
        r_f = fresh.dispersion()
    assert np.array_equal(s_host, s_f) and np.array_equal(l_host, l_f)
    assert np.array_equal(s_dev, s_f) and np.array_equal(l_dev, l_f)
    assert np.array_equal(r_host[1], r_f[1]) and np.array_equal(r_host[2], r_f[2])


def test_device_pointer_inputs_and_outputs(masw):
    import torch
    m, g = W.ragged_batch(n_models=10, seed=8)
    with masw.Batch(m, g) as bh:
        ref = bh.dispersion()
    with masw.Batch(m, g, device=True) as bd:
        ct = torch.empty(bd.n_items, dtype=torch.float64, device="cuda")
        idx = torch.empty(bd.n_items, dtype=torch.int32, device="cuda")
        st = torch.empty(bd.n_items, dtype=torch.int32, device="cuda")
        masw.dispersion(bd.handle, ct, idx, st)
        torch.cuda.synchronize()
        assert np.array_equal(idx.cpu().numpy(), ref[1])
        assert np.array_equal(st.cpu().numpy(), ref[2])


# ------------------------------------------------------ roots, gradient

def test_refined_roots_match_oracle(masw, oracle_lib):
    m, g = W.ragged_batch(n_models=12, seed=21)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
        croot = b.roots()
    rng = np.random.default_rng(3)
    for it in rng.choice(m.n_items, 300, replace=False):
        h, a, bb, r, _ = m.model(item_model[it])
        o_st, _, o_idx = oracle_lib.scan(h, a, bb, r, m.lam[it], g.c0, g.dc, g.n_c)
        if o_st != 0 or o_idx != idx[it]:
            continue
        o_root = oracle_lib.root(h, a, bb, r, m.lam[it], g.c0, g.dc, g.n_c, o_idx)
        assert croot[it] == pytest.approx(o_root, rel=1e-9)
        assert g.c0 + (idx[it] - 1) * g.dc <= croot[it] <= g.c0 + idx[it] * g.dc


def test_adjoint_root_gradient_matches_finite_differences(masw, oracle_lib):
    """dC*/d(beta, h) of every item from the adjoint kernel against the
    oracle's extrapolated central differences, per component."""
    m, g, _ = W.differentiation_batch(n_models=6, n_lambda=12)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
        rows = b.root_grad()
    off = 0
    checked = 0
    for it in range(m.n_items):
        h, a, bb, r, _ = m.model(item_model[it])
        N = h.size
        row = rows[off:off + 2 * N + 1]
        off += 2 * N + 1
        if st[it] != 0:
            continue
        fd = root_grad_reference(oracle_lib, h, a, bb, r, m.lam[it], g, idx[it])
        if not np.isfinite(fd).all():
            continue
        assert_grad_close(row, fd, where=it)
        checked += 1
    assert checked >= m.n_items * 0.9


def test_misfit_matches_oracle(masw, oracle_lib):
    m, g = W.uniform_batch(n_models=6, n_lambda=30)
    o_ct, o_idx, o_st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    ce = W.noisy_observation(np.where(o_st == 0, o_ct, 300.0), sigma=5.0)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
        assert (idx == o_idx).all()
        mp = b.misfit(ce, kind=masw.MISFIT_PAPER)
        ml = b.misfit(ce, kind=masw.MISFIT_LSQ, sigma=2.0)
    for k in range(m.n_models):
        sl = slice(k * 30, (k + 1) * 30)
        assert mp[k] == pytest.approx(oracle_lib.misfit_paper(o_ct[sl], ce[sl]), rel=1e-12)
        assert ml[k] == pytest.approx(oracle_lib.misfit_lsq(o_ct[sl], ce[sl], 2.0), rel=1e-12)


def test_misfit_curves_returns_what_dispersion_and_misfit_return(masw):
    """masw_misfit_curves (one evaluation, curves and misfit copied out
    together) equals masw_dispersion + masw_misfit, with host buffers, device
    buffers and a mix of the two."""
    import torch
    m, g = W.ragged_batch(n_models=24, seed=9)
    ce = W.noisy_observation(np.full(m.n_items, 250.0), sigma=30.0)
    with masw.Batch(m, g) as b:
        ct0, idx0, st0 = b.dispersion()
        phi0 = b.misfit(ce, kind=masw.MISFIT_PAPER)
        phi, ct, idx, st = b.misfit_curves(ce, kind=masw.MISFIT_PAPER)
        assert np.array_equal(phi, phi0, equal_nan=True)
        assert np.array_equal(ct, ct0, equal_nan=True)
        assert np.array_equal(idx, idx0) and np.array_equal(st, st0)
        dev = dict(phi=torch.empty(m.n_models, dtype=torch.float64, device="cuda"),
                   ct=torch.empty(m.n_items, dtype=torch.float64, device="cuda"),
                   idx=torch.empty(m.n_items, dtype=torch.int32, device="cuda"),
                   st=torch.empty(m.n_items, dtype=torch.int32, device="cuda"))
        for ce_in in (torch.from_numpy(ce).cuda(), ce):
            for t in dev.values():
                t.fill_(-3)
            masw.misfit_curves(b.handle, ce_in, masw.MISFIT_PAPER, 2.0, dev["phi"], dev["ct"],
                               dev["idx"], dev["st"])
            torch.cuda.synchronize()
            assert np.array_equal(dev["phi"].cpu().numpy(), phi0, equal_nan=True)
            assert np.array_equal(dev["idx"].cpu().numpy(), idx0)
            assert np.array_equal(dev["st"].cpu().numpy(), st0)
        # host misfit, device curves, status not requested
        hphi = np.empty(m.n_models)
        masw.misfit_curves(b.handle, ce, masw.MISFIT_LSQ, 2.0, hphi, dev["ct"], dev["idx"], None)
        torch.cuda.synchronize()
        assert np.array_equal(hphi, b.misfit(ce, kind=masw.MISFIT_LSQ), equal_nan=True)
        assert np.array_equal(dev["idx"].cpu().numpy(), idx0)


@pytest.mark.parametrize("n_models,n_lambda", [(3, 10), (1, 150)])
def test_misfit_gradient_matches_oracle_finite_differences(masw, oracle_lib, n_models, n_lambda):
    """LSQ misfit and its gradient w.r.t. beta and h against the oracle, per
    component; (1, 150) is one model at the differentiation workload's shape
    (12 layers + half-space, 150 log-spaced wavelengths 1..150 m)."""
    m, g, true = W.differentiation_batch(n_models=n_models, n_lambda=n_lambda)
    ht, at, bt, rt, lt = true.model(0)
    _, t_idx, _ = oracle_lib.dispersion(true.as_dict(), g.c0, g.dc, g.n_c)
    ce0 = np.array([oracle_lib.root(ht, at, bt, rt, l, g.c0, g.dc, g.n_c, int(i))
                    for l, i in zip(lt, t_idx)])
    ce = np.tile(W.noisy_observation(ce0, 2.0), m.n_models)
    with masw.Batch(m, g) as b:
        ct, idx, st = b.dispersion()
        phi, gbeta, gh = b.misfit_grad(ce, kind=masw.MISFIT_LSQ, sigma=2.0)
    assert (st == 0).all()
    hoff, loff, woff = m.layer_offsets()
    for k in range(m.n_models):
        h, a, bb, r, lam = m.model(k)
        roots = np.array([oracle_lib.root(h, a, bb, r, lam[j], g.c0, g.dc, g.n_c,
                                          int(idx[woff[k] + j])) for j in range(lam.size)])
        res = roots - ce[woff[k]:woff[k + 1]]
        assert phi[k] == pytest.approx(0.5 * np.sum(res ** 2) / 4.0, rel=1e-8)
        ref = np.zeros(2 * h.size + 1)
        for j in range(lam.size):
            ref += res[j] / 4.0 * root_grad_reference(oracle_lib, h, a, bb, r, lam[j], g,
                                                      idx[woff[k] + j])
        got = np.r_[gbeta[loff[k]:loff[k + 1]], gh[hoff[k]:hoff[k + 1]]]
        assert_grad_close(got, ref, where=k)


def test_grid_finer_than_fp32_resolution(masw, oracle_lib):
    """Test velocities 1e-5 m/s apart near 188 m/s: FP32 cannot tell
    neighbouring grid points apart (its spacing there is ~1.5e-5), so the
    counting search only locates each change approximately; the FP64
    certificate, its walk and the FP64 re-scan still return the FP64 scan's
    index for every item, for both two-precision plans. 24 wavelengths of one
    model put their roots inside the 0.4 m/s window."""
    base, _ = W.uniform_batch(n_models=1, n_layers=4, n_lambda=2, lam_max=40.0, seed=31)
    h, a, b, r, _ = base.model(0)
    lam = np.linspace(10.0, 10.45, 24)
    m = W.Models(np.array([4], np.int32), h, a, b, r, np.array([24], np.int32), lam)
    g = W.Grid(188.40, 1e-5, 40000)
    out = {}
    for p in (0, 1, 2):
        with masw.Batch(m, g) as bt:
            bt.set_plan(precision=p)
            out[p] = bt.dispersion()
    for p in (1, 2):
        assert np.array_equal(out[p][1], out[0][1]), p
        assert np.array_equal(out[p][2], out[0][2]), p
    assert (out[0][2] == 0).all()
    # and the oracle agrees within the parity bar on a few of them
    for j in (0, 11, 23):
        st, _, idx = oracle_lib.scan(h, a, b, r, lam[j], g.c0, g.dc, g.n_c)
        assert st == 0 and abs(idx - out[0][1][j]) <= 1


@pytest.mark.parametrize("seed", [101, 102, W.SEED + 11])
def test_extreme_models_two_precision_equals_fp64_scan(masw, oracle_lib, seed):
    """Both two-precision plans against the pure FP64 scan, item for item, on
    models chosen to stress the counting search (tight pole-free bounds,
    low-velocity layers, thin stiff layers, large k h); a sample against the
    oracle at the parity bar."""
    m, g = W.extreme_batch(seed=seed)
    with masw.Batch(m, g) as bt:
        bt.set_plan(precision=0)
        ref = bt.dispersion()
        for p, split in ((1, 0), (2, 0), (2, 1), (2, 2)):
            bt.set_plan(precision=p, count_split=split)
            got = bt.dispersion()
            assert np.array_equal(got[1], ref[1]), (p, split, np.nonzero(got[1] != ref[1])[0][:10])
            assert np.array_equal(got[2], ref[2]), (p, split)
        fb = bt.last_scan_fallback()
    assert (ref[2] == 0).mean() > 0.5 and fb >= 0
    items = np.random.default_rng(seed).choice(oracle_domain(oracle_lib, m), size=48,
                                               replace=False)
    o_ct, o_idx, o_st = oracle_items(oracle_lib, m, g, items)
    assert_index_parity(ref[1][items], ref[2][items], o_idx, o_st,
                        explain=(oracle_lib, m, g, items))


@pytest.mark.parametrize("route", [1, 2, 3, 4])
def test_forced_routes_give_the_fp64_scan(masw, route):
    """masw_set_route sends every item through the paths ordinary inputs
    rarely reach: the linear FP32 scan from V[0] (1), the FP64 mode-count
    search after a failed check (2), the FP64 scan from V[0] (3), higher-mode
    events located off by -7..+3 points before their certificate (4). Every
    plan (the counting plan fused, split and with its second stream) still
    reports the pure FP64 scan's indices, on uniform, ragged and extreme
    models, and the higher modes match too."""
    cases = [W.uniform_batch(n_models=32, n_lambda=40), W.ragged_batch(n_models=48),
             W.extreme_batch(n_models=64, seed=W.SEED + 11)]
    for m, g in cases:
        with masw.Batch(m, g) as b:
            b.set_plan(precision=0)
            ref = b.dispersion()
            ref_ch = b.changes(3)
            b.set_route(route)
            # precision 2 in each form: fused, split search, split with the second stream
            for p, split in ((1, 0), (2, 0), (2, 1), (2, 2)):
                b.set_plan(precision=p, count_split=split)
                got = b.dispersion()
                assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), \
                    (route, p, split)
            ch = b.changes(3)
            assert all(np.array_equal(x, y) for x, y in zip(ch[1:], ref_ch[1:])), route
            if route == 3:
                assert b.last_changes_linear() == m.n_items - int(np.sum(ref[2] != 0))
            if route == 4:  # recovered by the FP64 steps and search, not the linear scan
                assert b.last_changes_linear() <= max(2, m.n_items // 1000)
            b.set_route(0)
    with masw.Batch(*W.uniform_batch(n_models=2, n_lambda=2)) as b:
        for bad in (-1, 5):
            with pytest.raises(masw.MaswError):
                b.set_route(bad)
