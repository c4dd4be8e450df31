"""The benchmark's CPU banded baseline (the paper's serial banded elimination
restated, Section 2.1 / Section 3.1) against the oracle's dense LU: the same
determinant sign at random points below the half-space speed, the same
Algorithm 1 index on small uniform, ragged and extreme batches, the bare
half-space, and the same domain errors."""
import math

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_banded_sign_is_the_dense_lu_sign(oracle_lib, which):
    m, g = {"uniform": lambda: W.uniform_batch(n_models=6, n_lambda=8),
            "ragged": lambda: W.ragged_batch(n_models=8, lambdas=(4, 8)),
            "extreme": lambda: W.extreme_batch(n_models=12, n_lambda=4, seed=W.SEED + 13)}[which]()
    rng = np.random.default_rng(51)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    checked = 0
    for it in range(m.n_items):
        h, a, b, r, _ = m.model(item_model[it])
        k = 2.0 * math.pi / m.lam[it]
        if len(h) and k * h.max() > oracle_lib.MAX_KH:
            continue
        for c in rng.uniform(g.c0, b[-1], 6):
            sd, la = oracle_lib.det(h, a, b, r, k, c)
            if not np.isfinite(la):
                continue
            assert oracle_lib.det_sign_banded(h, a, b, r, k, c) == sd, (which, it, c)
            checked += 1
    assert checked >= 100


def test_banded_scan_gives_algorithm_1_indices(oracle_lib):
    for m, g in (W.uniform_batch(n_models=8, n_lambda=20), W.ragged_batch(n_models=12, lambdas=(10, 20))):
        _, idx, st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
        _, idx2, st2 = oracle_lib.dispersion_banded(m.as_dict(), g.c0, g.dc, g.n_c)
        assert np.array_equal(st, st2)
        assert (idx == idx2).mean() >= 0.999 and np.abs(idx - idx2).max() <= 1


def test_bare_half_space_and_domain(oracle_lib):
    beta = 300.0
    h, a, b, r = np.zeros(0), W.alpha_from_nu(np.array([beta]), 0.25), np.array([beta]), \
        np.array([2000.0])
    assert oracle_lib.scan_banded(h, a, b, r, 10.0, 50.0, 0.5, 800)[1:] == \
        oracle_lib.scan(h, a, b, r, 10.0, 50.0, 0.5, 800)[1:]
    hh, aa, bb, rr = np.array([6.0]), np.array([500.0, 900.0]), np.array([200.0, 380.0]), \
        np.array([1800.0, 2000.0])
    assert oracle_lib.scan_banded(hh, aa, bb, rr, 0.1, 50.0, 1.0, 100)[0] == oracle_lib.EINVAL
