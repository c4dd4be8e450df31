"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one part of the oracle (``oracle/masw_oracle.c``) to an
independent route: a high-precision matrix exponential of the P-SV
motion-stress system, its decaying eigenvectors, the textbook Rayleigh
cubic, brute-force determinants, eigenvalue inertia, exact identities of the
stiffness method (static condensation, velocity homogeneity) and the
definitions of Algorithms 1 and 2 applied to tiny hand cases.
"""
import itertools
import math

import mpmath as mp
import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads

pytestmark = pytest.mark.usefixtures("oracle_lib")


# ----------------------------------------------------------------- helpers

def A_dimensional(k, omega, lam_l, mu, rho):
    """Motion-stress matrix of P-SV waves, fields ~ exp(i(omega t - k x)),
    vector (U_x, U_z/i, T_xz, T_zz/i) with z down; written out from
    Newton's law and Hooke's law (not from the oracle's closed form)."""
    lp2m = lam_l + 2 * mu
    zeta = 4 * mu * (lam_l + mu) / lp2m
    return mp.matrix([
        [0, -k, 1 / mu, 0],
        [k * lam_l / lp2m, 0, 0, 1 / lp2m],
        [k * k * zeta - rho * omega ** 2, 0, 0, -k * lam_l / lp2m],
        [0, -rho * omega ** 2, k, 0],
    ])


def layer_K_expm(k, c, h, alpha, beta, rho, dps=90):
    """Layer stiffness through the transfer matrix P = expm(A h): with
    y(h) = P y(0), forces (-tau(0), tau(h)) in terms of (u(0), u(h))."""
    with mp.workdps(dps):
        k, c, h, alpha, beta, rho = (mp.mpf(x) for x in (k, c, h, alpha, beta, rho))
        mu = rho * beta ** 2
        lam_l = rho * alpha ** 2 - 2 * mu
        P = mp.expm(A_dimensional(k, k * c, lam_l, mu, rho) * h)
        Puu = P[0:2, 0:2]
        Put = P[0:2, 2:4]
        Ptu = P[2:4, 0:2]
        Ptt = P[2:4, 2:4]
        Pi = mp.inverse(Put)
        K11 = Pi * Puu
        K12 = -Pi
        K21 = Ptu - Ptt * Pi * Puu
        K22 = Ptt * Pi
        K = np.zeros((4, 4))
        for i in range(2):
            for j in range(2):
                K[i, j] = float(K11[i, j])
                K[i, j + 2] = float(K12[i, j])
                K[i + 2, j] = float(K21[i, j])
                K[i + 2, j + 2] = float(K22[i, j])
        return K


def halfspace_K_eig(k, c, alpha, beta, rho, dps=50):
    """Half-space stiffness from the two eigenvectors of A that decay with
    depth: with y = E a, forces on the top face are -tau(0) = -E_t E_u^-1 u."""
    with mp.workdps(dps):
        k, c, alpha, beta, rho = (mp.mpf(x) for x in (k, c, alpha, beta, rho))
        mu = rho * beta ** 2
        lam_l = rho * alpha ** 2 - 2 * mu
        A = A_dimensional(k, k * c, lam_l, mu, rho)
        ev, V = mp.eig(A)
        cols = [i for i in range(4) if mp.re(ev[i]) < 0]
        assert len(cols) == 2
        E = mp.matrix(4, 2)
        for j, col in enumerate(cols):
            for i in range(4):
                E[i, j] = V[i, col]
        Eu = E[0:2, 0:2]
        Et = E[2:4, 0:2]
        Kh = -(Et * mp.inverse(Eu))
        out = np.zeros((2, 2))
        for i in range(2):
            for j in range(2):
                assert abs(mp.im(Kh[i, j])) <= 1e-30 * (1 + abs(Kh[i, j]))
                out[i, j] = float(mp.re(Kh[i, j]))
        return out


def rayleigh_ratio(nu):
    """c_R / beta from the Rayleigh cubic x^3 - 8x^2 + (24 - 16g)x - 16(1 - g)
    with x = c^2/beta^2, g = beta^2/alpha^2 (the root in (0, 1))."""
    g = (1 - 2 * nu) / (2 * (1 - nu))
    roots = np.roots([1.0, -8.0, 24.0 - 16.0 * g, -16.0 * (1.0 - g)])
    real = [r.real for r in roots if abs(r.imag) < 1e-12 and 0 < r.real < 1]
    assert len(real) == 1
    return math.sqrt(real[0])


def leibniz_det(M):
    n = M.shape[0]
    total = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1.0
        for i in range(n):
            prod *= M[i, perm[i]]
        total += -prod if inv % 2 else prod
    return total


def half_space_model(beta, nu, rho=2000.0):
    b = np.array([beta])
    return np.zeros(0), workloads.alpha_from_nu(b, nu), b, np.array([rho])


# ------------------------------------------------------- element matrices

def test_motion_stress_eigenvalues_are_pm_kr_pm_ks():
    rng = np.random.default_rng(1)
    for _ in range(20):
        beta = rng.uniform(100, 800)
        alpha = beta * rng.uniform(1.5, 3.0)
        rho = rng.uniform(1500, 2500)
        k = rng.uniform(0.01, 5.0)
        c = beta * rng.uniform(0.05, 2.5)
        mu = rho * beta ** 2
        with mp.workdps(60):
            A = A_dimensional(mp.mpf(k), mp.mpf(k) * c, mp.mpf(rho) * alpha ** 2 - 2 * mu,
                              mp.mpf(mu), mp.mpf(rho))
            ev = [complex(e) for e in mp.eig(A)[0]]
        r = np.sqrt(complex(1 - c ** 2 / alpha ** 2))
        s = np.sqrt(complex(1 - c ** 2 / beta ** 2))
        for w in (k * r, -k * r, k * s, -k * s):
            j = int(np.argmin([abs(e - w) for e in ev]))
            assert abs(ev.pop(j) - w) <= 1e-10 * k
        assert not ev


def _layer_cases():
    rng = np.random.default_rng(2)
    cases = []
    for _ in range(60):
        beta = rng.uniform(100, 800)
        alpha = beta * rng.uniform(1.5, 3.0)
        rho = rng.uniform(1500, 2500)
        h = rng.uniform(0.5, 10)
        k = rng.uniform(0.005, 5.0)
        c = beta * rng.uniform(0.05, 2.5)
        cases.append((k, c, h, alpha, beta, rho))
    # exact r = 0 and s = 0 (c equal to alpha or beta), and kh spanning 1e-3..40
    cases += [(0.7, 250.0, 3.0, 600.0, 250.0, 1900.0), (0.3, 600.0, 2.0, 600.0, 250.0, 1900.0),
              (2 * np.pi / 1.0, 150.0, 2.0, 150.0 * np.sqrt(3.5), 150.0, 1850.0),
              (2 * np.pi / 1.0, 140.0, 6.4, 280.0, 160.0, 1800.0),
              (2 * np.pi / 5000.0, 120.0, 0.8, 280.0, 160.0, 1800.0)]
    return cases


@pytest.mark.parametrize("case", _layer_cases())
def test_layer_closed_form_matches_matrix_exponential(oracle_lib, case):
    k, c, h, alpha, beta, rho = case
    K = oracle_lib.layer_stiffness(k, c, h, alpha, beta, rho)
    Kx = layer_K_expm(k, c, h, alpha, beta, rho)
    scale = np.abs(Kx).max()
    km = k * rho * beta ** 2
    if scale > 1e4 * km:  # next to a clamped-layer resonance: skip
        pytest.skip("near a pole of the layer stiffness")
    assert np.abs(K - K.T).max() <= 1e-12 * scale
    assert np.abs(K - Kx).max() <= 1e-9 * scale


def test_halfspace_closed_form_matches_decaying_eigenvectors(oracle_lib):
    rng = np.random.default_rng(3)
    for _ in range(40):
        beta = rng.uniform(100, 800)
        alpha = beta * rng.uniform(1.5, 3.0)
        rho = rng.uniform(1500, 2500)
        k = rng.uniform(0.01, 5.0)
        c = beta * rng.uniform(0.05, 0.999)
        K = oracle_lib.halfspace_stiffness(k, c, alpha, beta, rho)
        Ke = halfspace_K_eig(k, c, alpha, beta, rho)
        assert np.abs(K - Ke).max() <= 1e-10 * np.abs(Ke).max()


def test_thick_layer_top_block_tends_to_halfspace(oracle_lib):
    k, c, alpha, beta, rho = 1.3, 180.0, 520.0, 230.0, 1900.0
    K = oracle_lib.layer_stiffness(k, c, 40.0, alpha, beta, rho)  # k h = 52
    Kh = oracle_lib.halfspace_stiffness(k, c, alpha, beta, rho)
    assert np.abs(K[:2, :2] - Kh).max() <= 1e-12 * np.abs(Kh).max()


def test_static_condensation_of_split_layer(oracle_lib):
    """A layer of thickness h1+h2 equals two stacked layers with the middle
    node condensed out (exact identity of the stiffness method)."""
    rng = np.random.default_rng(4)
    done = 0
    for _ in range(40):
        beta = rng.uniform(100, 600)
        alpha = beta * rng.uniform(1.6, 2.5)
        rho = rng.uniform(1600, 2200)
        k = rng.uniform(0.05, 3.0)
        c = beta * rng.uniform(0.1, 1.8)
        h1, h2 = rng.uniform(0.3, 4.0, 2)
        A = oracle_lib.layer_stiffness(k, c, h1, alpha, beta, rho)
        B = oracle_lib.layer_stiffness(k, c, h2, alpha, beta, rho)
        T = oracle_lib.layer_stiffness(k, c, h1 + h2, alpha, beta, rho)
        G = np.zeros((6, 6))
        G[:4, :4] += A
        G[2:, 2:] += B
        keep = [0, 1, 4, 5]
        mid = [2, 3]
        Gmm = G[np.ix_(mid, mid)]
        if np.linalg.cond(Gmm) > 1e8 or np.abs(T).max() > 1e4 * k * rho * beta ** 2:
            continue
        Kc = G[np.ix_(keep, keep)] - G[np.ix_(keep, mid)] @ np.linalg.solve(Gmm, G[np.ix_(mid, keep)])
        assert np.abs(Kc - T).max() <= 1e-8 * np.abs(T).max()
        done += 1
    assert done >= 20


# ---------------------------------------------------------- determinants

def test_lu_det_matches_leibniz(oracle_lib):
    rng = np.random.default_rng(5)
    for n in range(1, 7):
        for _ in range(5):
            M = rng.standard_normal((n, n))
            s, la = oracle_lib.lu_det(M)
            ref = leibniz_det(M)
            assert s == int(np.sign(ref))
            assert la == pytest.approx(math.log(abs(ref)), rel=1e-12, abs=1e-12)
    s, la = oracle_lib.lu_det(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert s == 0


def test_assembled_one_layer_det_matches_leibniz(oracle_lib):
    h, a, b, r = np.array([3.0]), np.array([500.0, 900.0]), np.array([200.0, 380.0]), \
        np.array([1800.0, 2000.0])
    for c in (80.0, 150.0, 185.0, 260.0, 350.0):
        K = oracle_lib.assemble(h, a, b, r, 2 * np.pi / 7.0, c)
        assert K.shape == (4, 4)
        assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()
        ref = leibniz_det(K)
        s, la = oracle_lib.det(h, a, b, r, 2 * np.pi / 7.0, c)
        assert s == int(np.sign(ref))
        assert la == pytest.approx(math.log(abs(ref)), rel=1e-11)


def test_assembled_det_matches_numpy_slogdet(oracle_lib):
    m, _ = workloads.uniform_batch(n_models=6, n_layers=5, n_lambda=3)
    rng = np.random.default_rng(6)
    for mi in range(m.n_models):
        h, a, b, r, lam = m.model(mi)
        for _ in range(10):
            c = rng.uniform(50, b[-1] * 0.999)
            k = 2 * np.pi / rng.choice(lam)
            K = oracle_lib.assemble(h, a, b, r, k, c)
            sn, ln = np.linalg.slogdet(K)
            s, la = oracle_lib.det(h, a, b, r, k, c)
            assert s == int(sn)
            assert la == pytest.approx(ln, rel=1e-10, abs=1e-8)


# ------------------------------------------------------------------ scan

def test_grid_velocity_and_scan_limit(oracle_lib):
    assert oracle_lib.grid_velocity(50.0, 0.25, 4600) == 1200.0
    assert oracle_lib.grid_velocity(50.0, 0.5, 0) == 50.0
    # V[n] < 400 for n = 0..699 with c0=50, dc=0.5
    assert oracle_lib.scan_limit(400.0, 50.0, 0.5, 901) == 700
    assert oracle_lib.scan_limit(400.0, 50.0, 0.5, 10) == 10
    assert oracle_lib.scan_limit(40.0, 50.0, 0.5, 901) == 0


def test_scan_equals_brute_force_first_sign_change(oracle_lib):
    m, _ = workloads.uniform_batch(n_models=4, n_layers=3, n_lambda=4, lam_max=60.0)
    c0, dc, n_c = 60.0, 2.0, 400
    for mi in range(m.n_models):
        h, a, b, r, lams = m.model(mi)
        for lam in lams:
            n_lim = oracle_lib.scan_limit(b[-1], c0, dc, n_c)
            signs = [oracle_lib.det(h, a, b, r, 2 * np.pi / lam, c0 + n * dc)[0]
                     for n in range(n_lim)]
            first = next((n for n in range(1, n_lim) if signs[n] != signs[n - 1]), None)
            st, ct, idx = oracle_lib.scan(h, a, b, r, lam, c0, dc, n_c)
            if first is None:
                assert st == oracle_lib.NO_ROOT and idx == -1 and math.isnan(ct)
            else:
                assert (st, idx, ct) == (oracle_lib.OK, first, c0 + first * dc)


def test_out_of_domain_wavelength_is_rejected(oracle_lib):
    h, a, b, r = np.array([6.0]), np.array([500.0, 900.0]), np.array([200.0, 380.0]), \
        np.array([1800.0, 2000.0])
    st, ct, idx = oracle_lib.scan(h, a, b, r, 0.1, 50.0, 1.0, 100)  # k h = 377
    assert st == oracle_lib.EINVAL and idx == -1 and math.isnan(ct)


def test_no_root_cases(oracle_lib):
    h, a, b, r = np.array([3.0]), np.array([500.0, 900.0]), np.array([200.0, 380.0]), \
        np.array([1800.0, 2000.0])
    # grid entirely above the half-space shear speed
    st, ct, idx = oracle_lib.scan(h, a, b, r, 10.0, 400.0, 1.0, 100)
    assert st == oracle_lib.NO_ROOT and idx == -1 and math.isnan(ct)
    # grid that stops below the root
    st, ct, idx = oracle_lib.scan(h, a, b, r, 10.0, 50.0, 1.0, 20)
    assert st == oracle_lib.NO_ROOT and idx == -1
    # a single point below beta_hs cannot hold a sign change
    st, _, _ = oracle_lib.scan(h, a, b, r, 10.0, 379.5, 1.0, 5)
    assert st == oracle_lib.NO_ROOT


@pytest.mark.parametrize("nu", [0.25, 0.3])
def test_half_space_gives_rayleigh_root_at_every_wavelength(oracle_lib, nu):
    beta = 200.0
    h, a, b, r = half_space_model(beta, nu)
    if nu == 0.25:
        cr = beta * math.sqrt(2.0 - 2.0 / math.sqrt(3.0))  # closed form for nu = 1/4
        assert cr / beta == pytest.approx(0.9194016867, rel=1e-9)
    else:
        cr = beta * rayleigh_ratio(nu)
    c0, dc, n_c = 50.0, 0.25, 4601
    want_idx = int(math.floor((cr - c0) / dc)) + 1
    for lam in (0.5, 1.0, 7.0, 60.0, 150.0, 5000.0):
        st, ct, idx = oracle_lib.scan(h, a, b, r, lam, c0, dc, n_c)
        assert st == oracle_lib.OK and idx == want_idx and ct == c0 + want_idx * dc
        root = oracle_lib.root(h, a, b, r, lam, c0, dc, n_c, idx)
        assert root == pytest.approx(cr, rel=1e-11)


@pytest.mark.parametrize("nu", [0.2, 0.35, 0.45])
def test_half_space_root_matches_rayleigh_cubic(oracle_lib, nu):
    beta = 333.0
    h, a, b, r = half_space_model(beta, nu)
    st, ct, idx = oracle_lib.scan(h, a, b, r, 12.0, 50.0, 0.25, 4601)
    assert st == oracle_lib.OK
    root = oracle_lib.root(h, a, b, r, 12.0, 50.0, 0.25, 4601, idx)
    assert root == pytest.approx(beta * rayleigh_ratio(nu), rel=1e-11)


def test_layer_identical_to_half_space_changes_nothing(oracle_lib):
    beta, nu, rho = 240.0, 0.3, 1950.0
    _, a0, b0, r0 = half_space_model(beta, nu, rho)
    h = np.array([3.7])
    a, b, r = np.repeat(a0, 2), np.repeat(b0, 2), np.repeat(r0, 2)
    for lam in (1.0, 3.0, 10.0, 40.0):
        s0 = oracle_lib.scan(np.zeros(0), a0, b0, r0, lam, 50.0, 0.25, 4601)
        s1 = oracle_lib.scan(h, a, b, r, lam, 50.0, 0.25, 4601)
        assert s0 == s1
        r_0 = oracle_lib.root(np.zeros(0), a0, b0, r0, lam, 50.0, 0.25, 4601, s0[2])
        r_1 = oracle_lib.root(h, a, b, r, lam, 50.0, 0.25, 4601, s1[2])
        assert r_1 == pytest.approx(r_0, rel=1e-11)


def test_splitting_a_layer_keeps_every_index(oracle_lib):
    m, grid = workloads.single_curve()
    h, a, b, r, lams = m.model(0)
    # split layer 3 (h = 4 m) into 1.5 m + 2.5 m of the same material
    h2 = np.array([2.0, 2.0, 1.5, 2.5, 6.0])
    a2, b2, r2 = (np.insert(x, 2, x[2]) for x in (a, b, r))
    for lam in lams[::7]:
        assert oracle_lib.scan(h, a, b, r, lam, grid.c0, grid.dc, grid.n_c) == \
            oracle_lib.scan(h2, a2, b2, r2, lam, grid.c0, grid.dc, grid.n_c)


@pytest.mark.parametrize("lam", [1.0, 20.0, 60.0])
def test_spd_before_root_and_one_negative_eigenvalue_at_root(oracle_lib, lam):
    m, grid = workloads.single_curve()
    h, a, b, r, _ = m.model(0)
    st, ct, idx = oracle_lib.scan(h, a, b, r, lam, grid.c0, grid.dc, grid.n_c)
    assert st == oracle_lib.OK
    k = 2 * np.pi / lam
    for n in list(range(0, idx, 5)) + [idx - 1]:
        ev = np.linalg.eigvalsh(oracle_lib.assemble(h, a, b, r, k, grid.c0 + n * grid.dc))
        assert (ev > 0).all(), n
    ev = np.linalg.eigvalsh(oracle_lib.assemble(h, a, b, r, k, ct))
    assert (ev < 0).sum() == 1


def test_short_and_long_wavelength_limits(oracle_lib):
    m, _ = workloads.single_curve()
    h, a, b, r, _ = m.model(0)
    kappa = rayleigh_ratio(0.3)
    c0, dc, n_c = 50.0, 0.05, 20000
    # short wavelength: only the top layer is felt
    st, _, idx = oracle_lib.scan(h, a, b, r, 0.15, c0, dc, n_c)
    root = oracle_lib.root(h, a, b, r, 0.15, c0, dc, n_c, idx)
    assert root == pytest.approx(kappa * b[0], rel=1e-6)
    # very long wavelength: the half-space dominates
    st, _, idx = oracle_lib.scan(h, a, b, r, 1e5, c0, dc, n_c)
    root = oracle_lib.root(h, a, b, r, 1e5, c0, dc, n_c, idx)
    assert root == pytest.approx(kappa * b[-1], rel=1e-3)


# --------------------------------------------------------------- misfit

def test_misfit_definitions_on_hand_cases(oracle_lib):
    ct = np.array([100.0, 200.0, 300.0])
    ce = np.array([110.0, 190.0, 300.0])
    assert oracle_lib.misfit_paper(ct, ce) == pytest.approx((10 / 110 + 10 / 190 + 0) / 3, rel=1e-15)
    assert oracle_lib.misfit_lsq(ct, ce, 2.0) == pytest.approx((100 + 100) / 8.0, rel=1e-15)


# ------------------------------------------------------------- gradient

def test_fd_gradient_half_space_is_rayleigh_ratio(oracle_lib):
    h, a, b, r = half_space_model(250.0, 0.3)
    st, _, idx = oracle_lib.scan(h, a, b, r, 10.0, 50.0, 0.25, 4601)
    gb, gh = oracle_lib.root_grad_fd(h, a, b, r, 10.0, 50.0, 0.25, 4601, idx)
    assert gh.size == 0
    assert gb[0] == pytest.approx(rayleigh_ratio(0.3), rel=1e-7)


def test_fd_gradient_velocity_homogeneity(oracle_lib):
    """Scaling every velocity by t scales the root by t, so
    sum_i beta_i dC/dbeta_i = C (Euler's theorem)."""
    m, grid = workloads.single_curve()
    h, a, b, r, _ = m.model(0)
    for lam in (3.0, 20.0, 45.0):
        st, _, idx = oracle_lib.scan(h, a, b, r, lam, grid.c0, grid.dc, grid.n_c)
        root = oracle_lib.root(h, a, b, r, lam, grid.c0, grid.dc, grid.n_c, idx)
        gb, gh = oracle_lib.root_grad_fd(h, a, b, r, lam, grid.c0, grid.dc, grid.n_c, idx)
        assert float(np.dot(b, gb)) == pytest.approx(root, rel=1e-7)
        # a thicker slow top layer can only slow the wave down
        assert gh[0] < 0


def test_fd_gradient_of_layer_identical_to_half_space_thickness_is_zero(oracle_lib):
    beta, nu, rho = 240.0, 0.3, 1950.0
    _, a0, b0, r0 = half_space_model(beta, nu, rho)
    h = np.array([3.7])
    a, b, r = np.repeat(a0, 2), np.repeat(b0, 2), np.repeat(r0, 2)
    st, _, idx = oracle_lib.scan(h, a, b, r, 8.0, 50.0, 0.25, 4601)
    gb, gh = oracle_lib.root_grad_fd(h, a, b, r, 8.0, 50.0, 0.25, 4601, idx)
    assert abs(gh[0]) < 1e-6
    assert float(gb.sum()) == pytest.approx(rayleigh_ratio(nu), rel=1e-7)


def test_uniform_stress_roots_land_near_their_targets(oracle_lib):
    """Input recipe of the uniform stress curves: the oracle's first change
    lies within 1.5 m/s of the targeted fundamental-mode limits (top-layer
    Rayleigh speed at 0.5 m, half-space Rayleigh speed at 2000 m), and every
    repeat of the wavelength gives the same index."""
    for target in workloads.STRESS_TARGETS:
        m, g = workloads.uniform_stress(target, 4, n_models=2)
        ct, idx, st = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
        assert (st == 0).all() and (idx == idx[0]).all()
        assert abs(ct[0] - target) <= 1.5, (target, ct[0])
