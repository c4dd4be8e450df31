"""CPU checks of the two facts the counting search (plan precision 2) rests
on, taken on the oracle's dense stiffness matrix with numpy's symmetric
eigensolver (brute force, independent of the CUDA path):

1. Pole-free bound: with both faces clamped, layer i has no mode below
   c_i = beta_i sqrt(1 + (pi / (k h_i))^2) (energy bound mu |grad u|^2 plus
   Poincare's inequality in depth), so the element stiffness K_e(k, c) stays
   finite for c < c_i.
2. Wittrick-Williams counting: below min(min_i c_i, beta_halfspace) the
   number of negative eigenvalues of the assembled K(k, c) is 0 at low c,
   non-decreasing in c, and first becomes nonzero exactly at Algorithm 1's
   first sign change of det K (Section 2.1).
"""
import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def pole_free_bound(h, beta, k):
    return min([beta[i] * np.sqrt(1.0 + (np.pi / (k * h[i])) ** 2) for i in range(len(h))]
               + [np.inf])


def negative_eigs(K):
    return int((np.linalg.eigvalsh(K) < 0.0).sum())


def test_layer_stiffness_is_finite_below_the_clamped_mode_bound(oracle_lib):
    rng = np.random.default_rng(31)
    for _ in range(120):
        beta = rng.uniform(80.0, 600.0)
        alpha = beta * rng.uniform(1.2, 3.0)
        h = rng.uniform(0.5, 10.0)
        k = 2.0 * np.pi / rng.uniform(0.5, 200.0)
        clb = beta * np.sqrt(1.0 + (np.pi / (k * h)) ** 2)
        scale = k * 1900.0 * beta ** 2
        cs = np.linspace(1.0, 0.999 * clb, 300)
        mx = max(np.abs(oracle_lib.layer_stiffness(k, c, h, alpha, beta, 1900.0)).max()
                 for c in cs) / scale
        assert mx < 1e5, (beta, alpha, h, k, mx)


def test_the_bound_is_nearly_tight(oracle_lib):
    """The bound is not vacuous: a thin layer's stiffness changes sign
    through a pole within 5% above c_lb (the clamped shear mode whose
    energy bound is almost attained)."""
    beta, alpha, h, k = 300.0, 600.0, 2.0, 2.0 * np.pi / 40.0
    clb = beta * np.sqrt(1.0 + (np.pi / (k * h)) ** 2)
    cs = np.linspace(clb, 1.05 * clb, 2000)
    d = np.array([oracle_lib.layer_stiffness(k, c, h, alpha, beta, 1900.0)[0, 0] for c in cs])
    flips = np.nonzero(np.sign(d[1:]) != np.sign(d[:-1]))[0]
    assert flips.size >= 1
    assert max(np.abs(d[flips])) / (k * 1900.0 * beta ** 2) > 1e3


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_negative_eigenvalue_count_is_monotone_and_marks_the_first_change(oracle_lib, which):
    rng = np.random.default_rng({"uniform": 32, "ragged": 33, "extreme": 34}[which])
    if which == "uniform":
        m, g = W.uniform_batch(n_models=16, n_lambda=10)
    elif which == "ragged":
        m, g = W.ragged_batch(n_models=24, lambdas=(8, 12))
    else:
        m, g = W.extreme_batch(n_models=40, n_lambda=12)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    checked = 0
    for it in rng.choice(m.n_items, 40 if which != "extreme" else 100, replace=False):
        h, a, b, r, _ = m.model(item_model[it])
        lam = m.lam[it]
        k = 2.0 * np.pi / lam
        st, _, idx = oracle_lib.scan(h, a, b, r, lam, g.c0, g.dc, g.n_c)
        nlim = oracle_lib.scan_limit(b[-1], g.c0, g.dc, g.n_c)
        cb = pole_free_bound(h, b, k)
        npf = min(nlim, int(np.sum(g.c0 + g.dc * np.arange(g.n_c) < cb)))
        if st != 0 or idx >= npf:
            continue  # the library scans these linearly
        pts = sorted(set([0, max(0, idx - 2), idx - 1, idx, npf - 1]
                         + list(rng.integers(0, npf, 10))))
        counts = [negative_eigs(oracle_lib.assemble(h, a, b, r, k, g.c0 + n * g.dc)) for n in pts]
        assert all(x <= y for x, y in zip(counts, counts[1:])), (it, pts, counts)
        assert counts[0] == 0 or pts[0] == idx
        assert counts[pts.index(idx - 1)] == 0 and counts[pts.index(idx)] % 2 == 1, (it, counts)
        assert next(p for p, s in zip(pts, counts) if s >= 1) == idx
        checked += 1
    assert checked >= 25
