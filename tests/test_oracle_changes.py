"""Pins of the oracle's continued scan (higher modes: Algorithm 1 carried past
its first sign change) and of the label it puts on each change.

- Positions: the sign of det K at every grid point, taken with numpy's
  slogdet (LAPACK LU) on the oracle's dense matrix, changes exactly at the
  listed indices, in order, and nowhere else before the last one.
- First change: equals Algorithm 1's index (oracle.scan).
- Labels: across a root of det K the number of negative eigenvalues rises by
  one (a mode of the layered structure is crossed), across a pole (a mode of
  a clamped layer) it falls by one. Checked without eigenvalues: bisection on
  the sign inside the bracket to 1e-12 relative width, then ln|det K| at the
  narrowed bracket is far below its grid values at a root and far above them
  at a pole.
"""
import math

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def slogdet_sign(oracle_lib, h, a, b, r, k, c):
    sign, _ = np.linalg.slogdet(oracle_lib.assemble(h, a, b, r, k, c))
    return int(sign)


def cases():
    m, g = workloads.single_curve()
    h, a, b, r, _ = m.model(0)
    yield (h, a, b, r, g, (1.0, 3.0, 5.0, 12.0, 40.0))
    mu, gu = workloads.uniform_batch(n_models=3, n_layers=4, n_lambda=3, seed=17)
    for q in range(mu.n_models):
        hq, aq, bq, rq, lq = mu.model(q)
        yield (hq, aq, bq, rq, workloads.Grid(50.0, 0.5, 1400), tuple(lq))


def test_changes_match_a_brute_force_sign_scan(oracle_lib):
    for h, a, b, r, g, lams in cases():
        nlim = oracle_lib.scan_limit(b[-1], g.c0, g.dc, g.n_c)
        for lam in lams:
            st, idx, _ = oracle_lib.scan_changes(h, a, b, r, lam, g.c0, g.dc, g.n_c, 5)
            k = 2.0 * math.pi / lam
            signs = [slogdet_sign(oracle_lib, h, a, b, r, k, oracle_lib.grid_velocity(g.c0, g.dc, n))
                     for n in range(nlim)]
            brute = [n for n in range(1, nlim) if signs[n] != signs[n - 1]][:5]
            found = [int(x) for x in idx if x >= 0]
            assert found == brute, (lam, found, brute)
            assert (st == oracle_lib.OK) == (len(brute) == 5)


def test_first_change_is_algorithm_1(oracle_lib):
    for h, a, b, r, g, lams in cases():
        for lam in lams:
            st1, _, idx1 = oracle_lib.scan(h, a, b, r, lam, g.c0, g.dc, g.n_c)
            _, idx, _ = oracle_lib.scan_changes(h, a, b, r, lam, g.c0, g.dc, g.n_c, 3)
            assert idx[0] == (idx1 if st1 == oracle_lib.OK else -1)


def test_labels_separate_roots_from_poles(oracle_lib):
    seen = {1: 0, -1: 0}
    for h, a, b, r, g, lams in cases():
        for lam in lams:
            k = 2.0 * math.pi / lam
            _, idx, delta = oracle_lib.scan_changes(h, a, b, r, lam, g.c0, g.dc, g.n_c, 6)
            for n, d in zip(idx, delta):
                if n < 0:
                    continue
                lo = oracle_lib.grid_velocity(g.c0, g.dc, int(n) - 1)
                hi = oracle_lib.grid_velocity(g.c0, g.dc, int(n))
                s_lo, l_lo = oracle_lib.det(h, a, b, r, k, lo)
                _, l_hi = oracle_lib.det(h, a, b, r, k, hi)
                x, y = lo, hi
                for _ in range(60):
                    mid = 0.5 * (x + y)
                    s_mid, _ = oracle_lib.det(h, a, b, r, k, mid)
                    if s_mid == s_lo:
                        x = mid
                    else:
                        y = mid
                    if y - x < 1e-12 * y:
                        break
                l_near = max(oracle_lib.det(h, a, b, r, k, x)[1], oracle_lib.det(h, a, b, r, k, y)[1])
                l_far = min(l_lo, l_hi)
                if d == 1:
                    assert l_near < max(l_lo, l_hi) - 5.0, (lam, n, l_near, l_lo, l_hi)
                elif d == -1:
                    assert l_near > l_far + 5.0, (lam, n, l_near, l_lo, l_hi)
                else:
                    pytest.fail(f"change {n} at lambda {lam}: count jumps by {d}")
                seen[int(d)] += 1
    assert seen[1] >= 10 and seen[-1] >= 2, seen
