"""Continuous-batching server: each result is identical alone and in the mix
(and equal to the batch entry point and to the oracle), admission by slots
and bytes refuses with a status instead of failing, and the trace replay
returns sane latencies."""
import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import masw, serving
    masw.load()
    return masw, serving


def requests(n, seed=5):
    s = W.RandomWalkSampler(seed=seed, chain_len=8)
    return W.concat([s.next() for _ in range(n)])


def test_results_identical_alone_in_the_mix_and_batched(env, oracle_lib):
    masw, serving = env
    reqs = requests(60)
    grid = W.Grid(50.0, 0.25, 4601)
    with masw.Batch(reqs, grid) as b:
        ref_ct, ref_idx, ref_st = b.dispersion()
    # in the mix: fast Poisson arrivals, several ticks per request
    arr = W.poisson_arrivals(reqs.n_models, rate=2e4, seed=1)
    with serving.Server(grid, max_slots=32, chunks_per_tick=3) as srv:
        lat, ct, idx, st, stats = srv.run_trace(reqs, arr)
    assert np.array_equal(idx, ref_idx) and np.array_equal(st, ref_st)
    assert np.array_equal(ct, ref_ct, equal_nan=True)
    assert stats["ticks"] > 3 and stats["max_in_flight"] > 1
    assert (lat >= 0).all()
    # alone: one request at a time, ticked to completion
    hoff, loff, woff = reqs.layer_offsets()
    with serving.Server(grid, max_slots=1, chunks_per_tick=1) as srv:
        for q in range(0, reqs.n_models, 7):
            h, a, bb, r, lam = reqs.model(q)
            rid = srv.submit(h, a, bb, r, lam)
            out = None
            while out is None:
                srv.tick()
                out = srv.poll(rid, lam.size)
            assert np.array_equal(out[1], ref_idx[woff[q]:woff[q + 1]])
            assert np.array_equal(out[2], ref_st[woff[q]:woff[q + 1]])
    # a few requests against the oracle
    for q in (0, 13, 41):
        h, a, bb, r, lam = reqs.model(q)
        o_ct, o_idx, o_st = oracle_lib.dispersion(reqs.subset([q]).as_dict(), grid.c0, grid.dc,
                                                  grid.n_c)
        sl = slice(woff[q], woff[q + 1])
        assert np.array_equal(o_st, st[sl])
        d = np.abs(o_idx - idx[sl])
        assert d.max() <= 1 and (d == 0).mean() >= 0.99


def test_admission_refuses_past_the_caps_with_a_status(env):
    masw, serving = env
    reqs = requests(6, seed=9)
    grid = W.Grid(50.0, 0.25, 4601)
    h, a, b, r, lam = reqs.model(0)
    one = (len(a) * (64 + 32)) + lam.size * 40
    with serving.Server(grid, max_slots=4, mem_cap_bytes=int(one * 1.5)) as srv:
        rid = srv.submit(h, a, b, r, lam)
        h1, a1, b1, r1, l1 = reqs.model(1)
        with pytest.raises(masw.MaswError) as ei:
            srv.submit(h1, a1, b1, r1, l1)
        assert ei.value.code == masw.EADMIT
        while srv.poll(rid, lam.size) is None:
            srv.tick()
        srv.submit(h1, a1, b1, r1, l1)  # room again after the poll
    with serving.Server(grid, max_slots=2) as srv:
        srv.submit(*reqs.model(0))
        srv.submit(*reqs.model(1))
        with pytest.raises(masw.MaswError) as ei:
            srv.submit(*reqs.model(2))
        assert ei.value.code == masw.EADMIT
        st = srv.stats()
        assert st["in_flight"] == 2 and st["bytes_in_flight"] > 0


def test_invalid_requests_are_rejected(env):
    masw, serving = env
    grid = W.Grid(50.0, 0.25, 4601)
    with serving.Server(grid, max_slots=2, max_layers=4, max_lambda=10) as srv:
        ok = (np.ones(2), np.array([500.0, 600, 900]), np.array([200.0, 250, 400]),
              np.full(3, 1900.0), np.array([5.0, 10.0]))
        for bad in ((np.ones(5), np.full(6, 900.0), np.full(6, 300.0), np.full(6, 1900.0), ok[4]),
                    (ok[0], ok[1], ok[2], ok[3], np.arange(1.0, 12.0)),
                    (-ok[0], ok[1], ok[2], ok[3], ok[4])):
            with pytest.raises(masw.MaswError) as ei:
                srv.submit(*bad)
            assert ei.value.code == masw.EINVAL
        srv.submit(*ok)


def test_plain_per_request_mode_matches(env):
    masw, serving = env
    reqs = requests(12, seed=3)
    grid = W.Grid(50.0, 0.25, 4601)
    arr = W.poisson_arrivals(reqs.n_models, rate=1e4, seed=2)
    with serving.Server(grid, max_slots=32, chunks_per_tick=4) as a:
        la, ct_a, idx_a, st_a, _ = a.run_trace(reqs, arr)
    with serving.Server(grid, max_slots=1, chunks_per_tick=1 << 20) as p:
        lp, ct_p, idx_p, st_p, sp = p.run_trace(reqs, arr)
    assert np.array_equal(idx_a, idx_p) and np.array_equal(st_a, st_p)
    assert sp["max_in_flight"] == 1
    s = serving.latency_summary(la, arr, reqs.n_models)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_tick_profile_changes_nothing_and_accounts_for_every_tick(env):
    """masw_server_profile: with the profile on, results are those of the
    batch entry point, every tick is profiled, every part's time is finite
    and non-negative, and turning it off freezes the totals."""
    masw, serving = env
    reqs = requests(40, seed=11)
    grid = W.Grid(50.0, 0.25, 4601)
    with masw.Batch(reqs, grid) as b:
        _, ref_idx, ref_st = b.dispersion()
    arr = W.poisson_arrivals(reqs.n_models, rate=5e4, seed=4)
    with serving.Server(grid, max_slots=16, chunks_per_tick=2) as srv:
        zero = srv.profile(True)
        assert all(v == 0.0 for v in zero.values())
        _, _, idx, st, stats = srv.run_trace(reqs, arr)
        prof = srv.profile(False)
        assert srv.profile(False) == prof
    assert np.array_equal(idx, ref_idx) and np.array_equal(st, ref_st)
    assert prof["ticks"] == stats["ticks"]
    vals = np.array(list(prof.values()))
    assert np.isfinite(vals).all() and (vals >= 0).all()
    assert prof["count_kernel_ms"] > 0 and prof["host_admit_ms"] > 0


def test_fallback_items_match_the_batch_path(env):
    """Items whose change lies above the pole-free bound or below V[0] leave
    the counting search for the linear screen; served results still equal
    the batch entry point's, with the linear plan and the FP64 plan."""
    masw, serving = env
    m = W.Models(np.array([1, 2], np.int32), np.array([6.0, 3.0, 5.0]),
                 np.array([400.0, 1700.0, 450.0, 700.0, 1800.0]),
                 np.array([150.0, 600.0, 170.0, 260.0, 650.0]),
                 np.full(5, 1900.0), np.array([6, 5], np.int32),
                 np.array([2.0, 4.0, 8.0, 12.0, 20.0, 30.0, 3.0, 6.0, 10.0, 18.0, 25.0]))
    grid = W.Grid(165.0, 0.5, 1000)
    with masw.Batch(m, grid) as b:
        ref = b.dispersion()
        b.set_plan(precision=0)
        ref0 = b.dispersion()
        b.set_plan(precision=2)
        b.dispersion()
        assert b.last_scan_fallback() >= 1
    assert np.array_equal(ref[1], ref0[1]) and np.array_equal(ref[2], ref0[2])
    hoff, loff, woff = m.layer_offsets()
    with serving.Server(grid, max_slots=4, chunks_per_tick=1) as srv:
        ids = [srv.submit(*m.model(q)) for q in range(m.n_models)]
        outs = [None] * m.n_models
        for _ in range(200):
            srv.tick()
            for q in range(m.n_models):
                if outs[q] is None:
                    outs[q] = srv.poll(ids[q], int(m.n_lambda[q]))
            if all(o is not None for o in outs):
                break
    for q in range(m.n_models):
        sl = slice(woff[q], woff[q + 1])
        assert np.array_equal(outs[q][1], ref[1][sl]) and np.array_equal(outs[q][2], ref[2][sl])


@pytest.mark.parametrize("chunks", [1, 8])
def test_extreme_models_served_equal_the_fp64_scan(env, chunks):
    """The extreme-model batch whose fallback items include roots and poles one
    grid step apart (an FP32 screen loses such pairs): every served item
    equals the batch path's plain FP64 scan (trace replay, all requests at
    once, so every tick mixes counted, fallback and searched items)."""
    masw, serving = env
    m, g = W.extreme_batch(seed=W.SEED + 11)
    with masw.Batch(m, g) as b:
        b.set_plan(precision=0)
        _, ref_idx, ref_st = b.dispersion()
    with serving.Server(g, max_slots=m.n_models, max_lambda=int(m.n_lambda.max()),
                        chunks_per_tick=chunks) as srv:
        lat, ct, idx, st, stats = srv.run_trace(m, np.zeros(m.n_models), timeout_s=120.0)
    bad = np.nonzero((idx != ref_idx) | (st != ref_st))[0]
    assert bad.size == 0, (bad[:10], idx[bad[:5]], ref_idx[bad[:5]])
    assert stats["refused"] == 0 and np.isfinite(lat).all()


@pytest.mark.parametrize("route", [1, 2, 3])
def test_forced_routes_served_equal_the_fp64_scan(env, route):
    """masw_server_set_route sends every served item through the linear FP32
    screen from V[0] (1), then the failed check and the mode-count search
    (2), then the FP64 scan at one chunk per tick (3); the results stay the
    pure FP64 scan's."""
    masw, serving = env
    m, g = W.extreme_batch(n_models=48, seed=W.SEED + 11)
    with masw.Batch(m, g) as b:
        b.set_plan(precision=0)
        _, ref_idx, ref_st = b.dispersion()
    with serving.Server(g, max_slots=m.n_models, max_lambda=int(m.n_lambda.max()),
                        chunks_per_tick=4) as srv:
        srv.set_route(route)
        lat, ct, idx, st, stats = srv.run_trace(m, np.zeros(m.n_models), timeout_s=300.0)
    assert np.array_equal(idx, ref_idx) and np.array_equal(st, ref_st), route
    with serving.Server(g, max_slots=2) as srv:
        for bad in (-1, 4):
            with pytest.raises(masw.MaswError):
                srv.set_route(bad)
