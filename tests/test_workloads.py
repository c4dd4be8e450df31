"""The seeded synthetic workloads (CPU only): the recipes stated for the
benchmark and the tests hold (sizes, ranges, the half-space and bulk-modulus
rules the library validates), and every generator is deterministic in its
seed."""
import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W


def valid(m):
    """Creation rules of the library: h, rho, beta > 0, alpha^2 > 4/3 beta^2."""
    return ((m.h > 0).all() and (m.rho > 0).all() and (m.beta > 0).all()
            and (3 * m.alpha ** 2 > 4 * m.beta ** 2).all())


def test_uniform_batch_recipe():
    m, g = W.uniform_batch()
    assert m.n_models == 1024 and (m.n_layers == 8).all() and (m.n_lambda == 200).all()
    assert (g.c0, g.dc, g.n_c) == (50.0, 0.25, 4601)
    assert valid(m) and m.h.min() >= 1.0 and m.h.max() <= 8.0
    lam = m.model(0)[4]
    assert np.isclose(lam[0], 1.0) and np.isclose(lam[-1], 150.0)
    for q in (0, 511, 1023):
        b = m.model(q)[2]
        assert (np.diff(b) > 0).all() and 100.0 <= b[0] <= 250.0


def test_extreme_batch_recipe():
    m, g = W.extreme_batch()
    assert m.n_models == 256 and (m.n_lambda == 32).all()
    assert m.n_layers.min() >= 1 and m.n_layers.max() <= 30
    assert valid(m) and m.h.min() >= 0.05 and m.h.max() <= 50.0
    assert (g.c0, g.dc, g.n_c) == (50.0, 0.5, 4901)
    unsorted = 0
    for q in range(m.n_models):
        h, a, b, r, lam = m.model(q)
        assert b[-1] >= b[:-1].max() and b[-1] <= 1.5 * b[:-1].max() + 1e-9
        assert 1000.0 <= r.min() and r.max() <= 3000.0
        unsorted += len(b) > 2 and not (np.diff(b[:-1]) > 0).all()
        assert np.isclose(lam[0], 0.5) and np.isclose(lam[-1], 500.0)
    assert unsorted > 100  # low-velocity layers are common


def test_leaky_batch_is_the_uniform_models_on_a_higher_grid():
    m, g = W.leaky_batch(n_models=64, n_lambda=50)
    u, _ = W.uniform_batch(n_models=64, n_lambda=50)
    for f in ("n_layers", "h", "alpha", "beta", "rho", "n_lambda", "lam"):
        assert np.array_equal(getattr(m, f), getattr(u, f)), f
    assert (g.c0, g.dc, g.n_c) == (700.0, 0.25, 4001)
    beta_hs = np.array([m.model(q)[2][-1] for q in range(m.n_models)])
    assert (beta_hs < g.c0).any() and (beta_hs > g.c0).any()


@pytest.mark.parametrize("gen", [lambda s: W.uniform_batch(n_models=8, n_lambda=5, seed=s),
                                 lambda s: W.ragged_batch(n_models=8, seed=s),
                                 lambda s: W.extreme_batch(n_models=8, seed=s),
                                 lambda s: W.differentiation_batch(n_models=4, seed=s)])
def test_generators_are_deterministic_in_their_seed(gen):
    a, b, c = gen(7), gen(7), gen(8)
    ma, mb, mc = a[0], b[0], c[0]
    for f in ("h", "alpha", "beta", "rho", "lam"):
        assert np.array_equal(getattr(ma, f), getattr(mb, f)), f
    assert not all(np.array_equal(getattr(ma, f), getattr(mc, f)) for f in ("beta", "h"))
