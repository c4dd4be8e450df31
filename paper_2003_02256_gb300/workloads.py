"""Seeded synthetic inputs for the dispersion-curve workloads.

This module only draws layered models, wavelength sets and test-velocity
grids from seeded random distributions; it holds none of the method's
arithmetic (no stiffness, determinant or scan). Both the CUDA library's tests
and the CPU oracle consume its output.

Model arrays follow the C ABI layout: models are concatenated; model m has
``n_layers[m]`` finite layers, ``h`` holds their thicknesses, and ``alpha``,
``beta``, ``rho`` hold ``n_layers[m] + 1`` values each (the last one is the
half-space). Wavelengths are concatenated the same way by ``n_lambda``.

The paper's own datasets ("uniform" and "variable" curves, Section 3) are not
given numerically; these distributions stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 20032256


@dataclass
class Grid:
    """Test velocities V[n] = c0 + n*dc, n = 0..n_c-1 (Algorithm 1's V)."""
    c0: float
    dc: float
    n_c: int


@dataclass
class Models:
    n_layers: np.ndarray  # int32 [M]
    h: np.ndarray         # f64 [sum N]
    alpha: np.ndarray     # f64 [sum N+1]
    beta: np.ndarray      # f64 [sum N+1]
    rho: np.ndarray       # f64 [sum N+1]
    n_lambda: np.ndarray  # int32 [M]
    lam: np.ndarray       # f64 [sum n_lambda]
    meta: dict = field(default_factory=dict)

    @property
    def n_models(self) -> int:
        return int(self.n_layers.size)

    @property
    def n_items(self) -> int:
        return int(self.lam.size)

    def as_dict(self) -> dict:
        return {"n_layers": self.n_layers, "h": self.h, "alpha": self.alpha,
                "beta": self.beta, "rho": self.rho, "n_lambda": self.n_lambda,
                "lambda": self.lam}

    def layer_offsets(self):
        hoff = np.concatenate([[0], np.cumsum(self.n_layers)]).astype(np.int64)
        loff = np.concatenate([[0], np.cumsum(self.n_layers + 1)]).astype(np.int64)
        woff = np.concatenate([[0], np.cumsum(self.n_lambda)]).astype(np.int64)
        return hoff, loff, woff

    def model(self, m: int):
        """(h, alpha, beta, rho, lam) of model m."""
        hoff, loff, woff = self.layer_offsets()
        return (self.h[hoff[m]:hoff[m + 1]], self.alpha[loff[m]:loff[m + 1]],
                self.beta[loff[m]:loff[m + 1]], self.rho[loff[m]:loff[m + 1]],
                self.lam[woff[m]:woff[m + 1]])

    def subset(self, ms) -> "Models":
        """The models with indices ``ms``, in that order."""
        parts = [self.model(int(m)) for m in ms]
        return Models(
            n_layers=np.array([p[0].size for p in parts], dtype=np.int32),
            h=np.concatenate([p[0] for p in parts]) if parts else np.zeros(0),
            alpha=np.concatenate([p[1] for p in parts]),
            beta=np.concatenate([p[2] for p in parts]),
            rho=np.concatenate([p[3] for p in parts]),
            n_lambda=np.array([p[4].size for p in parts], dtype=np.int32),
            lam=np.concatenate([p[4] for p in parts]),
            meta=dict(self.meta, subset=True))


def concat(parts) -> Models:
    return Models(
        n_layers=np.concatenate([p.n_layers for p in parts]).astype(np.int32),
        h=np.concatenate([p.h for p in parts]),
        alpha=np.concatenate([p.alpha for p in parts]),
        beta=np.concatenate([p.beta for p in parts]),
        rho=np.concatenate([p.rho for p in parts]),
        n_lambda=np.concatenate([p.n_lambda for p in parts]).astype(np.int32),
        lam=np.concatenate([p.lam for p in parts]),
        meta={"concat": len(parts)})


def alpha_from_nu(beta, nu):
    """P speed from S speed and Poisson ratio (input recipe, isotropic)."""
    return beta * np.sqrt(2.0 * (1.0 - nu) / (1.0 - 2.0 * nu))


def _draw_profile(rng, N, *, invert: bool = False):
    """One model: h~U[1,8]; beta_1~U[100,250], each deeper layer
    +U[10,120]; nu~U[0.25,0.4]; rho~U[1700,2100]. With ``invert`` one finite
    layer j>=2 is slowed to beta_{j-1}*U[0.6,0.9] (a low-velocity layer)."""
    h = rng.uniform(1.0, 8.0, N)
    beta = np.empty(N + 1)
    beta[0] = rng.uniform(100.0, 250.0)
    for i in range(1, N + 1):
        beta[i] = beta[i - 1] + rng.uniform(10.0, 120.0)
    if invert and N >= 2:
        j = int(rng.integers(1, N))  # finite layer index 1..N-1 (0-based), i.e. j>=2 1-based
        beta[j] = beta[j - 1] * rng.uniform(0.6, 0.9)
    nu = rng.uniform(0.25, 0.4, N + 1)
    rho = rng.uniform(1700.0, 2100.0, N + 1)
    return h, alpha_from_nu(beta, nu), beta, rho


def _pack(profiles, lams, meta) -> Models:
    return Models(
        n_layers=np.array([p[0].size for p in profiles], dtype=np.int32),
        h=np.concatenate([p[0] for p in profiles]),
        alpha=np.concatenate([p[1] for p in profiles]),
        beta=np.concatenate([p[2] for p in profiles]),
        rho=np.concatenate([p[3] for p in profiles]),
        n_lambda=np.array([l.size for l in lams], dtype=np.int32),
        lam=np.concatenate(lams),
        meta=meta)


# ---------------------------------------------------------------- workloads

def single_curve() -> tuple[Models, Grid]:
    """Single plain curve: 4 layers + half-space, h=[2,2,4,6] m,
    beta=[150,180,220,300,400] m/s, nu=0.3, rho=[1850,1850,1900,1900,2000];
    wavelengths 1..60 m step 1; c grid 50..500 step 0.5 (901 points)."""
    beta = np.array([150.0, 180.0, 220.0, 300.0, 400.0])
    h = np.array([2.0, 2.0, 4.0, 6.0])
    rho = np.array([1850.0, 1850.0, 1900.0, 1900.0, 2000.0])
    alpha = alpha_from_nu(beta, 0.3)
    lam = np.arange(1.0, 61.0)
    m = _pack([(h, alpha, beta, rho)], [lam], {"workload": "single_curve"})
    return m, Grid(50.0, 0.5, 901)


def uniform_batch(n_models: int = 1024, n_layers: int = 8, n_lambda: int = 200,
                  lam_max: float = 150.0, grid: Grid | None = None,
                  seed: int = SEED) -> tuple[Models, Grid]:
    """Uniform batch: n_models models of n_layers layers + half-space from
    the profile distribution, n_lambda log-spaced wavelengths 1..lam_max m,
    c grid 50..1200 step 0.25 (4601 points) unless ``grid`` is given."""
    rng = np.random.default_rng(seed)
    profiles = [_draw_profile(rng, n_layers) for _ in range(n_models)]
    lam = np.geomspace(1.0, lam_max, n_lambda)
    m = _pack(profiles, [lam] * n_models,
              {"workload": "uniform_batch", "seed": seed, "n_models": n_models,
               "n_layers": n_layers, "n_lambda": n_lambda})
    return m, grid or Grid(50.0, 0.25, 4601)


def ragged_batch(n_models: int = 8192, layers=(3, 30), lambdas=(30, 400),
                 invert_frac: float = 0.10, grid: Grid | None = None,
                 seed: int = SEED + 3) -> tuple[Models, Grid]:
    """Ragged batch: layer count uniform in ``layers``, wavelength count
    uniform in ``lambdas``, log-spaced from 1 m to twice the total layer
    thickness; ``invert_frac`` of the models carry a low-velocity layer."""
    rng = np.random.default_rng(seed)
    profiles, lams = [], []
    for _ in range(n_models):
        N = int(rng.integers(layers[0], layers[1] + 1))
        nw = int(rng.integers(lambdas[0], lambdas[1] + 1))
        inv = bool(rng.random() < invert_frac)
        p = _draw_profile(rng, N, invert=inv)
        profiles.append(p)
        lams.append(np.geomspace(1.0, 2.0 * float(p[0].sum()), nw))
    m = _pack(profiles, lams, {"workload": "ragged_batch", "seed": seed,
                               "n_models": n_models})
    return m, grid or Grid(50.0, 0.25, 4601)


STRESS_TARGETS = (72.0, 238.0, 256.0)


def uniform_stress(target: float, repeats: int, n_models: int = 256) -> tuple[Models, Grid]:
    """Uniform-work stress curves (the paper's uniform runs: one wavelength
    repeated many times per curve). Each of the n_models identical curves
    holds `repeats` copies of one wavelength, chosen so that the root lies
    near `target` m/s, from the textbook limits of the fundamental mode (the
    Rayleigh speed of the top layer at short wavelengths, of the half-space
    at long ones; 0.9194 beta for nu = 0.25):
      72  -> model S (h = [4, 6] m, beta = [78.3, 180, 278.4] m/s), lambda 0.5 m;
      238 -> model U (h = [4, 6] m, beta = [200, 230, 258.9] m/s), lambda 2000 m;
      256 -> model S, lambda 2000 m.
    nu = 0.25, rho = 1900 kg/m^3; c grid 50..1200 m/s step 0.25."""
    models = {"S": np.array([78.3, 180.0, 278.4]), "U": np.array([200.0, 230.0, 258.9])}
    case = {72.0: ("S", 0.5), 238.0: ("U", 2000.0), 256.0: ("S", 2000.0)}
    if float(target) not in case:
        raise ValueError(f"target must be one of {STRESS_TARGETS}")
    name, lam = case[float(target)]
    beta = models[name]
    h = np.array([4.0, 6.0])
    alpha = alpha_from_nu(beta, 0.25)
    rho = np.full(3, 1900.0)
    profiles = [(h, alpha, beta, rho)] * n_models
    lams = [np.full(int(repeats), lam)] * n_models
    m = _pack(profiles, lams, {"workload": f"uniform_stress target {target:g} m/s, "
                                           f"lambda {lam:g} m x {repeats}"})
    return m, Grid(50.0, 0.25, 4601)


def extreme_batch(n_models: int = 256, n_lambda: int = 32, seed: int = SEED + 8
                  ) -> tuple[Models, Grid]:
    """Models outside the paper's ranges, for robustness tests: 1..30 layers
    with log-uniform thicknesses 0.05..50 m, unsorted shear speeds 60..1500 m/s
    (low-velocity layers, strong contrasts), Poisson ratios 0.1..0.45,
    densities 1000..3000 kg/m^3, a half-space 1.0..1.5 times faster than the
    fastest layer, and n_lambda log-spaced wavelengths 0.5..500 m per model;
    c grid 50..2500 m/s step 0.5."""
    rng = np.random.default_rng(seed)
    profiles = []
    for N in rng.integers(1, 31, n_models):
        beta = rng.uniform(60.0, 1500.0, N + 1)
        beta[N] = beta[:N].max() * rng.uniform(1.0, 1.5)
        nu = rng.uniform(0.1, 0.45, N + 1)
        h = np.exp(rng.uniform(np.log(0.05), np.log(50.0), N))
        profiles.append((h, alpha_from_nu(beta, nu), beta, rng.uniform(1000.0, 3000.0, N + 1)))
    lams = [np.geomspace(0.5, 500.0, n_lambda)] * n_models
    m = _pack(profiles, lams, {"workload": f"extreme models x {n_models}, seed {seed}"})
    return m, Grid(50.0, 0.5, 4901)


def leaky_batch(n_models: int = 1024, n_lambda: int = 200) -> tuple[Models, Grid]:
    """The uniform batch's models on a c grid 700..1700 m/s step 0.25, which
    starts above most of their fundamental modes and above about half of
    their half-space shear speeds (5 / 50 / 95 % at 526 / 691 / 855 m/s for
    the full batch), so most first sign changes lie where the half-space
    block is complex."""
    m, _ = uniform_batch(n_models=n_models, n_lambda=n_lambda)
    m.meta = dict(m.meta, workload=f"uniform_batch models x {n_models}, {n_lambda} lambda; "
                                   "c grid 700..1700 step 0.25 (leaky continuation)")
    return m, Grid(700.0, 0.25, 4001)


def differentiation_batch(n_models: int = 512, n_layers: int = 12, n_lambda: int = 150,
                          grid: Grid | None = None, seed: int = SEED + 4,
                          spread: float = 0.05) -> tuple[Models, Grid, Models]:
    """Differentiation workload: a seeded true model (12 layers + half-space
    from the profile distribution) and ``n_models`` candidate models drawn
    around it (each beta and h scaled by 1 + N(0, spread^2)); 150 log-spaced
    wavelengths 1..150 m. Returns (candidates, grid, true_model)."""
    rng = np.random.default_rng(seed)
    h0, a0, b0, r0 = _draw_profile(rng, n_layers)
    lam = np.geomspace(1.0, 150.0, n_lambda)
    true = _pack([(h0, a0, b0, r0)], [lam], {"workload": "differentiation_true", "seed": seed})
    ratio = a0 / b0
    profiles = []
    for _ in range(n_models):
        b = b0 * (1.0 + spread * rng.standard_normal(n_layers + 1))
        b = np.maximum(b, 50.0)
        h = h0 * np.clip(1.0 + spread * rng.standard_normal(n_layers), 0.5, 1.5)
        profiles.append((h, b * ratio, b, r0.copy()))
    m = _pack(profiles, [lam] * n_models,
              {"workload": "differentiation", "seed": seed, "n_models": n_models})
    return m, grid or Grid(50.0, 0.25, 4601), true


def noisy_observation(curve, sigma: float = 2.0, seed: int = SEED + 5):
    """C_e = curve + N(0, sigma^2), seeded."""
    rng = np.random.default_rng(seed)
    return np.asarray(curve, dtype=np.float64) + sigma * rng.standard_normal(np.size(curve))


class RandomWalkSampler:
    """Seeded random-walk model sampler (the request source of the serving
    workload): each step perturbs one beta_i or h_i of the current model by
    N(0, (2%)^2) of its value. Models start from the ragged-batch
    distribution; ``restart`` draws a fresh chain start."""

    def __init__(self, seed: int = SEED + 6, layers=(3, 30), lambdas=(30, 400),
                 step: float = 0.02, chain_len: int = 64):
        self.rng = np.random.default_rng(seed)
        self.layers, self.lambdas, self.step, self.chain_len = layers, lambdas, step, chain_len
        self._restart()

    def _restart(self):
        rng = self.rng
        N = int(rng.integers(self.layers[0], self.layers[1] + 1))
        nw = int(rng.integers(self.lambdas[0], self.lambdas[1] + 1))
        h, a, b, r = _draw_profile(rng, N)
        self.cur = [h, a, b, r]
        self.ratio = a / b
        self.lam = np.geomspace(1.0, 2.0 * float(h.sum()), nw)
        self.left = self.chain_len

    def next(self) -> Models:
        if self.left <= 0:
            self._restart()
        self.left -= 1
        h, a, b, r = (x.copy() for x in self.cur)
        N = h.size
        p = int(self.rng.integers(0, 2 * N + 1))
        if p <= N:
            b[p] *= 1.0 + self.step * self.rng.standard_normal()
            b[p] = max(b[p], 50.0)
            a[p] = b[p] * self.ratio[p]
        else:
            h[p - N - 1] *= max(0.2, 1.0 + self.step * self.rng.standard_normal())
        self.cur = [h, a, b, r]
        return _pack([(h, a, b, r)], [self.lam.copy()], {"workload": "random_walk"})


def poisson_arrivals(n: int, rate: float, seed: int = SEED + 7) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))
