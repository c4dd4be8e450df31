"""masw_dispersion_noalloc: the entry point for callers that cannot allocate.

Embedders whose GPU memory is handed out by someone else (a framework's
allocator, a fixed budget, a service that forbids allocation after start-up)
cannot use masw_model_batch_create, which allocates a device copy of the
batch. masw_dispersion_noalloc works from a fixed array inside the library
instead. These tests call it through the C ABI twice in a row and compare
each result with masw_dispersion on the same models (the scan and its
arithmetic are shared, so the indices must be identical), and check that
batches beyond the fixed limits are refused. The file is named to run last.
"""
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


def _arrays(models, device):
    import torch
    arrs = [np.ascontiguousarray(models.n_layers, dtype=np.int32),
            np.ascontiguousarray(models.h, dtype=np.float64),
            np.ascontiguousarray(models.alpha, dtype=np.float64),
            np.ascontiguousarray(models.beta, dtype=np.float64),
            np.ascontiguousarray(models.rho, dtype=np.float64),
            np.ascontiguousarray(models.n_lambda, dtype=np.int32),
            np.ascontiguousarray(models.lam, dtype=np.float64)]
    return [torch.from_numpy(a).cuda() for a in arrs] if device else arrs


def _noalloc(masw, models, grid, device):
    import torch
    n = models.n_items
    ct = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    idx = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    masw.dispersion_noalloc(*_arrays(models, device), (grid.c0, grid.dc, grid.n_c), ct, idx, st)
    torch.cuda.synchronize()
    return ct.cpu().numpy(), idx.cpu().numpy(), st.cpu().numpy()


def test_two_calls_in_a_row_match_the_batch_entry_point(masw):
    m1, g1 = W.ragged_batch(n_models=40, seed=101)
    m2, g2 = W.uniform_batch(n_models=48, n_layers=6, n_lambda=90, seed=202)
    assert m1.n_items <= masw.NOALLOC_MAX_ITEMS and m2.n_items <= masw.NOALLOC_MAX_ITEMS
    for models, grid, device in ((m1, g1, True), (m2, g2, False)):
        with masw.Batch(models, grid) as b:
            ref_ct, ref_idx, ref_st = b.dispersion()
        ct, idx, st = _noalloc(masw, models, grid, device)
        assert np.array_equal(st, ref_st)
        assert np.array_equal(idx, ref_idx)
        assert np.array_equal(ct, ref_ct, equal_nan=True)


def test_limits_are_refused_with_a_clear_error(masw):
    import torch
    too_many_models, g = W.uniform_batch(n_models=masw.NOALLOC_MAX_MODELS + 1, n_layers=1,
                                         n_lambda=1)
    too_many_items, _ = W.uniform_batch(n_models=2, n_layers=2,
                                        n_lambda=masw.NOALLOC_MAX_ITEMS // 2 + 1)
    out = [torch.empty(70000, dtype=t, device="cuda")
           for t in (torch.float64, torch.int32, torch.int32)]
    for m in (too_many_models, too_many_items):
        with pytest.raises(masw.MaswError) as ei:
            masw.dispersion_noalloc(*_arrays(m, False), (g.c0, g.dc, g.n_c), *out)
        assert ei.value.code == masw.ETOOBIG
        assert "MASW_NOALLOC_MAX" in str(ei.value)
