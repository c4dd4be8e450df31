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


# ------------------------------------------------ clamped-layer mode count

def clamped_modes_halving(oracle_lib, k, c, h, alpha, beta, rho):
    """J0 of one layer (modes with both faces clamped below c) by halving the
    thickness: a clamped layer is two clamped halves joined at a free middle
    node whose stiffness K22(h/2) + K11(h/2) = diag(2a, 2d) (the half layer's
    diagonal entries), so by Wittrick-Williams J0(h) = 2 J0(h/2) + [a < 0] +
    [d < 0], down to the first thickness below which c is under the pole-free
    bound (J0 = 0 there)."""
    L = 0
    while beta * np.sqrt(1.0 + (np.pi * 2 ** L / (k * h)) ** 2) <= c:
        L += 1
    J = 0
    for j in range(L, 0, -1):
        K = oracle_lib.layer_stiffness(k, c, h / 2 ** j, alpha, beta, rho)
        J = 2 * J + int(K[0, 0] < 0) + int(K[1, 1] < 0)
    return J


def clamped_modes_dense(oracle_lib, k, c, h, alpha, beta, rho, m):
    """J0 by brute force: the layer cut into m equal sublayers, each under
    its pole-free bound, assembled over the m-1 interior nodes (faces
    clamped); the count of negative eigenvalues of that dense matrix."""
    Ke = oracle_lib.layer_stiffness(k, c, h / m, alpha, beta, rho)
    n = 2 * (m - 1)
    K = np.zeros((n, n))
    for i in range(m):
        for p in range(4):
            for q in range(4):
                a, b = i + p // 2, i + q // 2
                if 1 <= a <= m - 1 and 1 <= b <= m - 1:
                    K[2 * (a - 1) + p % 2, 2 * (b - 1) + q % 2] += Ke[p, q]
    return negative_eigs(K) if n else 0


def test_clamped_layer_mode_count_by_halving_matches_dense_subdivision(oracle_lib):
    rng = np.random.default_rng(35)
    nonzero = 0
    for _ in range(150):
        beta = rng.uniform(100.0, 600.0)
        alpha = beta * rng.uniform(1.3, 3.0)
        h = rng.uniform(0.5, 20.0)
        k = 2.0 * np.pi / rng.uniform(0.5, 100.0)
        c = beta * rng.uniform(0.5, 8.0)
        if k * h > 250.0:
            continue
        m = 2
        while beta * np.sqrt(1.0 + (np.pi * m / (k * h)) ** 2) <= c:
            m += 1
        J = clamped_modes_halving(oracle_lib, k, c, h, alpha, beta, 1900.0)
        assert J == clamped_modes_dense(oracle_lib, k, c, h, alpha, beta, 1900.0, m)
        assert J == clamped_modes_dense(oracle_lib, k, c, h, alpha, beta, 1900.0, m + 7)
        assert J == oracle_lib.clamped_modes(k, c, h, alpha, beta, 1900.0)
        nonzero += J > 0
    assert nonzero >= 60


def mode_counts(oracle_lib, h, a, b, r, k, c):
    """(s, J0): negative eigenvalues of K and clamped modes of all layers."""
    j0 = sum(clamped_modes_halving(oracle_lib, k, c, h[i], a[i], b[i], r[i])
             for i in range(len(h)))
    return negative_eigs(oracle_lib.assemble(h, a, b, r, k, c)), j0


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_mode_count_is_monotone_and_its_odd_jumps_are_the_sign_changes(oracle_lib, which):
    """Wittrick-Williams over the whole scan range: J = J0 + s (the number of
    modes of the layered structure below c) never decreases, so neither does
    T = J + J0 = s + 2 J0; T has the parity of s, so det K changes sign between
    two grid points exactly when T jumps by an odd amount there. Checked
    against the oracle's continued scan (all sign changes with their count
    changes) on every grid point of coarse grids."""
    if which == "uniform":
        m, _ = W.uniform_batch(n_models=4, n_lambda=5, seed=36)
    elif which == "ragged":
        m, _ = W.ragged_batch(n_models=6, lambdas=(3, 5), seed=37)
    else:
        m, _ = W.extreme_batch(n_models=8, n_lambda=4, seed=38)
    g = W.Grid(50.0, 4.0, 400)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    events = 0
    for it in range(m.n_items):
        h, a, b, r, _ = m.model(item_model[it])
        k = 2.0 * np.pi / m.lam[it]
        if len(h) and k * h.max() > 250.0:
            continue
        nlim = oracle_lib.scan_limit(b[-1], g.c0, g.dc, g.n_c)
        if nlim < 2:
            continue
        sc = [mode_counts(oracle_lib, h, a, b, r, k, g.c0 + n * g.dc) for n in range(nlim)]
        T = [s + 2 * j0 for s, j0 in sc]
        assert all(x <= y for x, y in zip(T, T[1:])), (which, it)
        odd = [n for n in range(1, nlim) if (T[n] - T[n - 1]) % 2 == 1]
        _, idx, delta = oracle_lib.scan_changes(h, a, b, r, m.lam[it], g.c0, g.dc, g.n_c, 15)
        found = [int(x) for x in idx if x >= 0]
        assert found == odd[:15], (which, it, found, odd[:15])
        for n, d in zip(found, delta):
            assert d == sc[n][0] - sc[n - 1][0]
        events += len(odd)
    assert events >= 20
