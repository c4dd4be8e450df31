"""Gradient reference and bar shared by the GPU gradient tests.

The reference is the oracle's central difference of the refined root
(reading: the derivative is taken on the zero of det K inside the first
sign-changing bracket, with the Poisson ratio held under d/dbeta),
Richardson-extrapolated over the relative steps 1e-4 and 2e-4 and with the
bisection run to about two ulps of the root. With the default bracket
width of 1e-13 the difference quotient alone carries up to ~1e-5 relative
noise on single components (1e-13 of the root over a step of 1e-4); the
extrapolated, fully refined form agrees with itself under step halving
(steps 5e-5 and 1e-4) to below 2e-6 relative per component on the
differentiation workload's 150 wavelengths, inside the 1e-5 bar.

The bar is per component: |got - ref| <= 1e-5 |ref| wherever |ref| is at
least 1e-3 of the largest component, and |got - ref| <= 1e-8 of the largest
component below that floor (those components are under the difference
quotient's own noise as a relative quantity).
"""
import numpy as np

REL = 1e-5
FLOOR = 1e-3
# relative bracket width of the reference's bisection: about two ulps
BISECT_TOL = 4e-16


def root_grad_reference(oracle_lib, h, alpha, beta, rho, lam, grid, idx):
    """d C*/d(beta_1..beta_{N+1}, h_1..h_N) of one item, Richardson-
    extrapolated central differences of the oracle's refined root."""
    g = (grid.c0, grid.dc, grid.n_c)
    a1, b1 = oracle_lib.root_grad_fd(h, alpha, beta, rho, lam, *g, int(idx), rel_step=1e-4,
                                     rel_tol=BISECT_TOL)
    a2, b2 = oracle_lib.root_grad_fd(h, alpha, beta, rho, lam, *g, int(idx), rel_step=2e-4,
                                     rel_tol=BISECT_TOL)
    return (4.0 * np.r_[a1, b1] - np.r_[a2, b2]) / 3.0


def assert_grad_close(got, ref, where=""):
    """The per-component bar (module docstring)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape and np.isfinite(got).all() and np.isfinite(ref).all(), where
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    big = np.abs(ref) >= FLOOR * scale
    rel = err[big] / np.abs(ref[big])
    assert (rel <= REL).all(), (where, float(rel.max()), np.nonzero(big)[0][np.argmax(rel)])
    assert (err[~big] <= REL * FLOOR * scale).all(), (where, float(err[~big].max(initial=0)))
    return float(rel.max(initial=0.0))
