"""Failures made on the host, never on the GPU: an injected device-allocation
failure at every allocation of batch creation is reported as MASW_ENOMEM and
leaks no device memory, and the batch made afterwards gives the usual
results; the server's bounded wait ends with MASW_ETIMEOUT and the server
still tears down cleanly."""
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
    return torch, masw, serving


def test_allocation_failures_are_reported_and_leak_nothing(env):
    torch, masw, _ = env
    m, g = W.uniform_batch(n_models=16, n_lambda=20)
    with masw.Batch(m, g) as b:
        ref = b.dispersion()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(48):
        masw.test_fail_alloc(k)
        try:
            b = masw.Batch(m, g)
        except masw.MaswError as e:
            assert e.code == masw.ENOMEM, (k, e.code)
            failed += 1
            continue
        finally:
            masw.test_fail_alloc(-1)
        b.close()  # the hook fired after creation (or not at all)
    torch.cuda.synchronize()
    assert failed >= 10  # creation makes that many allocations at least
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (8 << 20)
    with masw.Batch(m, g) as b:
        got = b.dispersion()
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


def test_server_bounded_wait_ends_with_a_status(env):
    _, masw, serving = env
    m, g = W.extreme_batch(n_models=64, seed=W.SEED + 11)
    srv = serving.Server(g, max_slots=8, max_lambda=int(m.n_lambda.max()), chunks_per_tick=1)
    srv.set_route(3)  # FP64 chunks, one per tick: the trace cannot finish in 1 ms
    with pytest.raises(masw.MaswError) as ei:
        srv.run_trace(m, np.zeros(m.n_models), timeout_s=1e-3)
    assert ei.value.code == masw.ETIMEOUT
    srv.close()
    with serving.Server(g, max_slots=64, max_lambda=int(m.n_lambda.max())) as ok:
        _, _, idx, st, stats = ok.run_trace(m, np.zeros(m.n_models), timeout_s=300.0)
    assert stats["refused"] == 0 and (st >= 0).all()
