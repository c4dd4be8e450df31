"""masw_dispersion_noalloc: the entry point for callers that cannot allocate.

Embedders whose GPU memory is handed out by someone else (a framework's
allocator, a fixed budget, a service that forbids allocation after start-up)
cannot use masw_model_batch_create, which allocates a device copy of the
batch. masw_dispersion_noalloc works from a fixed array inside the library
instead. These tests call it through the C ABI twice in a row and compare
each result with masw_dispersion on the same models (the scan and its
arithmetic are shared, so the indices must be identical), and check that
batches beyond the fixed limits and inputs in the wrong memory space are
refused without touching the outputs. The file is named to run last.
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


def _sentinel_outputs(n):
    import torch
    return [torch.full((n,), -1.5, dtype=torch.float64, device="cuda"),
            torch.full((n,), -7, dtype=torch.int32, device="cuda"),
            torch.full((n,), -9, dtype=torch.int32, device="cuda")]


def _unchanged(out):
    import torch
    torch.cuda.synchronize()
    return ((out[0] == -1.5).all() and (out[1] == -7).all() and (out[2] == -9).all()).item()


def test_limits_are_refused_with_a_clear_error(masw):
    """Each of the three limits on its own (models; layer records, with the
    models and items under theirs; items) gives MASW_ETOOBIG and leaves the
    outputs untouched."""
    too_many_models, g = W.uniform_batch(n_models=masw.NOALLOC_MAX_MODELS + 1, n_layers=1,
                                         n_lambda=1)
    too_many_records, _ = W.uniform_batch(n_models=600, n_layers=30, n_lambda=1)
    too_many_items, _ = W.uniform_batch(n_models=2, n_layers=2,
                                        n_lambda=masw.NOALLOC_MAX_ITEMS // 2 + 1)
    assert too_many_records.n_models <= masw.NOALLOC_MAX_MODELS
    assert too_many_records.n_items <= masw.NOALLOC_MAX_ITEMS
    assert int(np.sum(too_many_records.n_layers + 1)) > masw.NOALLOC_MAX_RECORDS
    out = _sentinel_outputs(70000)
    for m in (too_many_models, too_many_records, too_many_items):
        with pytest.raises(masw.MaswError) as ei:
            masw.dispersion_noalloc(*_arrays(m, False), (g.c0, g.dc, g.n_c), *out)
        assert ei.value.code == masw.ETOOBIG
        assert "MASW_NOALLOC_MAX" in str(ei.value)
        assert _unchanged(out)


def test_mixed_memory_spaces_are_refused_before_any_launch(masw):
    """Model arrays whose memory space differs from the declared one (here a
    host thickness array in a call that declares device inputs, and device
    arrays in a call that declares host inputs) give MASW_EINVAL through the
    C ABI, with the outputs untouched; the Python binding refuses a mix of
    host and device arrays itself."""
    import ctypes
    m, g = W.ragged_batch(n_models=6, seed=303)
    host = _arrays(m, False)
    dev = _arrays(m, True)
    lib = masw.load()
    f = lib.masw_dispersion_noalloc
    f.argtypes = [ctypes.POINTER(masw.ModelsDesc), ctypes.POINTER(masw.GridDesc),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    grid = masw.GridDesc(g.c0, g.dc, g.n_c)
    out = _sentinel_outputs(m.n_items)
    mixed_dev = list(dev)
    mixed_dev[1] = host[1]  # h on the host, declared MASW_DEVICE
    for arrs, space in ((mixed_dev, masw.DEVICE), (dev, masw.HOST)):
        desc = masw.ModelsDesc(m.n_models, *(masw._ptr(a) for a in arrs), space)
        rc = f(ctypes.byref(desc), ctypes.byref(grid), masw._stream_handle(None),
               *(masw._ptr(o) for o in out))
        assert rc == masw.EINVAL
        assert _unchanged(out)
    with pytest.raises(ValueError):
        masw.dispersion_noalloc(*mixed_dev, (g.c0, g.dc, g.n_c), *out)
    # the same arrays, all in one space, are accepted
    masw.dispersion_noalloc(*dev, (g.c0, g.dc, g.n_c), *out)
    with masw.Batch(m, g) as b:
        _, ref_idx, ref_st = b.dispersion()
    assert np.array_equal(out[1].cpu().numpy(), ref_idx)
    assert np.array_equal(out[2].cpu().numpy(), ref_st)
