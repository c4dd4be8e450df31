"""Pins of the oracle's leaky continuation: Algorithm 1 over the whole grid,
test velocities at or above the half-space shear speed included, where the
half-space block is complex (the paper builds its stiffness matrices in
complex arithmetic, Section 3.3) and the sign is that of Re det K.

Independent routes:
- the complex half-space block against the eigenvectors of the P-SV
  motion-stress matrix for the outgoing branch (high-precision eigenvectors,
  not the closed form), and the other branch against its complex conjugate;
- a bare half-space against the textbook Rayleigh function: det K_hs =
  -(k mu)^2 R / (1 - r s) with R = (2 - q)^2 - 4 r s;
- the complex LU against numpy's determinant;
- below the half-space speed, the real oracle (pinned in test_oracle_pins);
- the scan against a brute-force sign sweep of numpy determinants.
"""
import cmath
import math

import mpmath as mp
import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads
from test_oracle_pins import A_dimensional

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def halfspace_K_branch(k, c, alpha, beta, rho, sign_im=1, dps=50):
    """Half-space stiffness from the eigenvectors of A with eigenvalues -k r
    and -k s, where r, s are the square roots of 1 - c^2/alpha^2 and
    1 - c^2/beta^2 whose imaginary part has the sign sign_im (real roots are
    the positive ones): -tau(0) = -E_t E_u^-1 u."""
    def root(x):
        w = cmath.sqrt(complex(x))
        return complex(w.real, sign_im * abs(w.imag))
    r = root(1 - c * c / (alpha * alpha))
    s = root(1 - c * c / (beta * beta))
    with mp.workdps(dps):
        kk, cc, aa, bb, rr = (mp.mpf(x) for x in (k, c, alpha, beta, rho))
        mu = rr * bb ** 2
        lam_l = rr * aa ** 2 - 2 * mu
        A = A_dimensional(kk, kk * cc, lam_l, mu, rr)
        ev, V = mp.eig(A)
        cols = []
        for w in (-k * r, -k * s):
            j = min(range(4), key=lambda i: abs(complex(ev[i]) - w))
            assert abs(complex(ev[j]) - w) <= 1e-12 * k
            cols.append(j)
        E = mp.matrix(4, 2)
        for j, col in enumerate(cols):
            for i in range(4):
                E[i, j] = V[i, col]
        Kh = -(E[2:4, 0:2] * mp.inverse(E[0:2, 0:2]))
        return np.array([[complex(Kh[i, j]) for j in range(2)] for i in range(2)])


def halfspace_cases(n, seed, lo, hi):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        beta = rng.uniform(100, 800)
        alpha = beta * rng.uniform(1.5, 3.0)
        rho = rng.uniform(1500, 2500)
        k = rng.uniform(0.01, 5.0)
        yield k, beta * rng.uniform(lo, hi), alpha, beta, rho


@pytest.mark.parametrize("lo,hi", [(1.001, 1.45), (1.01, 4.0)])
def test_complex_halfspace_matches_outgoing_eigenvectors(oracle_lib, lo, hi):
    """Between beta and alpha (r real, s imaginary) and above alpha (both
    imaginary): the continued closed form equals the eigenvector route on
    the principal branch, and the other branch gives its conjugate."""
    checked = 0
    for k, c, alpha, beta, rho in halfspace_cases(30, 41 if lo < 1.005 else 42, lo, hi):
        K = oracle_lib.halfspace_stiffness_complex(k, c, alpha, beta, rho)
        Ke = halfspace_K_branch(k, c, alpha, beta, rho, +1)
        Kc = halfspace_K_branch(k, c, alpha, beta, rho, -1)
        scale = np.abs(Ke).max()
        assert np.abs(K - Ke).max() <= 1e-10 * scale, (c / beta, c / alpha)
        assert np.abs(np.conj(K) - Kc).max() <= 1e-10 * scale
        assert np.abs(K.imag).max() > 1e-6 * scale  # complex indeed
        checked += c > alpha
    assert checked >= 1 if hi > 2 else True


def test_complex_halfspace_is_the_real_one_below_beta(oracle_lib):
    for k, c, alpha, beta, rho in halfspace_cases(30, 43, 0.05, 0.999):
        K = oracle_lib.halfspace_stiffness_complex(k, c, alpha, beta, rho)
        Kr = oracle_lib.halfspace_stiffness(k, c, alpha, beta, rho)
        assert np.abs(K.imag).max() == 0.0
        assert np.abs(K.real - Kr).max() <= 1e-14 * np.abs(Kr).max()


@pytest.mark.parametrize("nu", [0.25, 0.33, 0.45])
def test_bare_halfspace_re_det_follows_the_rayleigh_function(oracle_lib, nu):
    """N = 0: sign Re det K = sign Re(-R / (1 - r s)) at c from 0.5 beta to
    5 beta, and the whole-grid scan changes sign only at the Rayleigh root
    (a half-space has no leaky zero on the real axis)."""
    beta = 300.0
    h, a, b, r = np.zeros(0), workloads.alpha_from_nu(np.array([beta]), nu), \
        np.array([beta]), np.array([2000.0])
    alpha = float(a[0])
    k = 2 * np.pi / 10.0
    for c in np.linspace(0.5 * beta, 5.0 * beta, 301):
        q = c * c / beta ** 2
        rr = cmath.sqrt(1 - c * c / alpha ** 2)
        ss = cmath.sqrt(1 - q)
        R = (2 - q) ** 2 - 4 * rr * ss
        want = -R / (1 - rr * ss)
        if abs(want.real) < 1e-9 * abs(want):
            continue
        sg, _ = oracle_lib.det_leaky(h, a, b, r, k, float(c))
        assert sg == (1 if want.real > 0 else -1), c / beta
    c0 = 0.5 * beta
    st, ct, idx = oracle_lib.scan_leaky(h, a, b, r, 10.0, c0, 0.5, 2000)
    st0, ct0, idx0 = oracle_lib.scan(h, a, b, r, 10.0, c0, 0.5, 2000)
    assert st == st0 == oracle_lib.OK and idx == idx0
    st, _, idx = oracle_lib.scan_leaky(h, a, b, r, 10.0, beta, 0.5, 2000)
    assert st == oracle_lib.NO_ROOT and idx == -1


def test_complex_lu_matches_numpy(oracle_lib):
    rng = np.random.default_rng(44)
    for n in (1, 2, 3, 6, 12):
        for _ in range(10):
            A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
            ph, la = oracle_lib.lu_det_complex(A)
            d = np.linalg.det(A)
            assert abs(ph * math.exp(la) - d) <= 1e-12 * abs(d)
    ph, la = oracle_lib.lu_det_complex(np.zeros((3, 3)))
    assert ph == 0 and la == -math.inf


def test_below_the_half_space_speed_it_is_algorithm_1(oracle_lib):
    """Where K is real, the complex route gives the real oracle's sign at every
    point, and the whole-grid scan gives Algorithm 1's index wherever that
    finds one."""
    m, g = workloads.uniform_batch(n_models=6, n_layers=5, n_lambda=12, seed=45)
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    rng = np.random.default_rng(45)
    for it in range(m.n_items):
        h, a, b, r, _ = m.model(item_model[it])
        lam = m.lam[it]
        k = 2 * np.pi / lam
        for c in rng.uniform(g.c0, b[-1], 4):
            assert oracle_lib.det_leaky(h, a, b, r, k, c)[0] == oracle_lib.det(h, a, b, r, k, c)[0]
        st, _, idx = oracle_lib.scan(h, a, b, r, lam, g.c0, g.dc, g.n_c)
        st2, ct2, idx2 = oracle_lib.scan_leaky(h, a, b, r, lam, g.c0, g.dc, g.n_c)
        assert st == oracle_lib.OK and (st2, idx2) == (st, idx)
        assert ct2 == oracle_lib.grid_velocity(g.c0, g.dc, idx2)


def test_scan_equals_brute_force_sign_sweep(oracle_lib):
    """Grids that start below and above the half-space speed: the first index
    where sgn Re det (numpy's determinant of the dense complex K) changes."""
    m, _ = workloads.uniform_batch(n_models=3, n_layers=3, n_lambda=4, lam_max=60.0, seed=46)
    found_above = 0
    for mi in range(m.n_models):
        h, a, b, r, lams = m.model(mi)
        for c0, dc, n_c in ((60.0, 2.0, 500), (float(b[-1]), 1.0, 400)):
            for lam in lams:
                k = 2 * np.pi / lam
                signs = []
                for n in range(n_c):
                    d = np.linalg.det(oracle_lib.assemble_complex(
                        h, a, b, r, k, oracle_lib.grid_velocity(c0, dc, n)))
                    signs.append(int(np.sign(d.real)))
                first = next((n for n in range(1, n_c) if signs[n] != signs[n - 1]), None)
                st, ct, idx = oracle_lib.scan_leaky(h, a, b, r, lam, c0, dc, n_c)
                if first is None:
                    assert st == oracle_lib.NO_ROOT and idx == -1 and math.isnan(ct)
                else:
                    assert (st, idx) == (oracle_lib.OK, first)
                    found_above += oracle_lib.grid_velocity(c0, dc, idx) > b[-1]
    assert found_above >= 6


def test_invalid_inputs(oracle_lib):
    h, a, b, r = np.array([6.0]), np.array([500.0, 900.0]), np.array([200.0, 380.0]), \
        np.array([1800.0, 2000.0])
    assert oracle_lib.scan_leaky(h, a, b, r, 0.1, 50.0, 1.0, 100)[0] == oracle_lib.EINVAL
    assert oracle_lib.scan_leaky(h, a, b, r, 10.0, 0.0, 1.0, 100)[0] == oracle_lib.EINVAL
    with pytest.raises(ValueError):
        oracle_lib.det_leaky(h, a, b, r, 1.0, -5.0)
