"""The double-float element of the counting certificate (csrc/masw_df.cuh)
against a 50-digit evaluation of the closed-form element stiffness, and
beside the FP64 element, through masw_element_check.

Points: random (item, layer, c) of uniform, ragged and extreme models, with
c below the layer's pole-free bound (where the certificate evaluates
elements: no element is near one of its own poles there) and below the
half-space shear speed. The element's entries K = numerator / D are
compared relative to the largest of the element's six entries. Bar: at
the median 1e-13; at every point no worse than the FP64 element by more
than a factor 30 (the ratio of the two unit roundoffs), or 1e-11; on the
uniform and ragged workloads 1e-11 everywhere. (On the extreme models the
worst double-float point, 9.6e-10, sits where the FP64 element is off by
3.5e-6: such points are ill-conditioned for both.)"""
import math

import mpmath as mp
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


def reference_entries(h, a, b, rho, k, c, dps=50):
    """K11 (00, 01, 11) and K12 (00, 01, 11) of one layer in units of k, from
    the closed form (the FP64 element's, with rho c^2 in the denominator),
    at dps digits."""
    with mp.workdps(dps):
        h, a, b, rho, k, c = (mp.mpf(float(v)) for v in (h, a, b, rho, k, c))
        c2 = c * c
        kh = k * h
        q = c2 / b ** 2
        r2 = 1 - c2 / a ** 2
        s2 = 1 - q

        def wave(w2):
            if w2 > 0:
                w = mp.sqrt(w2)
                x = kh * w
                return 1, mp.cosh(x), mp.sinh(x) / w, w * mp.sinh(x)
            if w2 == 0:
                return 1, 1, kh, 0
            w = mp.sqrt(-w2)
            x = kh * w
            return 1, mp.cos(x), mp.sin(x) / w, -w * mp.sin(x)

        RE, RC, RSd, RSm = wave(r2)
        SE, SC, SSd, SSm = wave(s2)
        u = RE * SE - RC * SC
        SdSd = RSd * SSd
        D = (2 * u + RSm * SSm + SdSd) / (rho * c2)
        num = [RC * SSd - SC * RSm,
               (b * b / c2) * -((s2 + 3) * u + SSm * (2 * RSm + RSd) + SdSd),
               SC * RSd - RC * SSm,
               RSm * SE - RE * SSd,
               RE * SC - RC * SE,
               SSm * RE - SE * RSd]
        return np.array([float(x / D) for x in num])


def sample_points(models, grid, rng, n):
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    pts = []
    while len(pts) < n:
        it = int(rng.integers(models.n_items))
        h, a, b, r, _ = models.model(item_model[it])
        if h.size == 0:
            continue
        j = int(rng.integers(h.size))
        k = 2 * math.pi / models.lam[it]
        cpf = b[j] * math.sqrt(1 + (math.pi / (k * h[j])) ** 2) * (1 - 1e-4)
        top = min(cpf, b[-1] * 0.9999)
        if top <= grid.c0:
            continue
        c = float(rng.uniform(grid.c0, top))
        pts.append((it, j, c, h[j], a[j], b[j], r[j], k))
    return pts


@pytest.mark.parametrize("which", ["uniform", "ragged", "extreme"])
def test_double_float_element_against_50_digits(masw, which):
    if which == "uniform":
        m, g = W.uniform_batch(n_models=32)
    elif which == "ragged":
        m, g = W.ragged_batch(n_models=32)
    else:
        m, g = W.extreme_batch(n_models=32, seed=W.SEED + 11)
    rng = np.random.default_rng(17)
    pts = sample_points(m, g, rng, 300)
    with masw.Batch(m, g) as b:
        fp, df = masw.element_check(b.handle, [p[0] for p in pts], [p[1] for p in pts],
                                    [p[2] for p in pts])
    err_df, err_fp = [], []
    for t, (_, _, c, h, a, bb, r, k) in enumerate(pts):
        ref = reference_entries(h, a, bb, r, k, c)
        scale = np.abs(ref).max()
        err_df.append(np.abs(df[t, 1:] / df[t, 0] - ref).max() / scale)
        err_fp.append(np.abs(fp[t, 1:] / fp[t, 0] - ref).max() / scale)
    err_df, err_fp = np.array(err_df), np.array(err_fp)
    print(f"{which}: double-float max {err_df.max():.1e} median {np.median(err_df):.1e}; "
          f"FP64 max {err_fp.max():.1e} median {np.median(err_fp):.1e}")
    assert np.isfinite(err_df).all()
    assert np.median(err_df) <= 1e-13
    assert (err_df <= np.maximum(30 * err_fp, 1e-11)).all()
    if which != "extreme":
        assert err_df.max() <= 1e-11


def leaky_points(models, grid, rng, n):
    """(item, layer, c) with c between the half-space shear speed and the top
    of the grid: the leaky continuation's points, where most finite layers
    are above their shear speed (trigonometric branch, arguments k h |s| up
    to a few hundred)."""
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    top = grid.c0 + grid.dc * (grid.n_c - 1)
    pts = []
    while len(pts) < n:
        it = int(rng.integers(models.n_items))
        h, a, b, r, _ = models.model(item_model[it])
        if h.size == 0 or b[-1] >= top:
            continue
        j = int(rng.integers(h.size))
        c = float(rng.uniform(b[-1], top))
        pts.append((it, j, c, h[j], a[j], b[j], r[j], 2 * math.pi / models.lam[it]))
    return pts


@pytest.mark.parametrize("which", ["leaky", "ragged"])
def test_leaky_double_float_element_against_50_digits(masw, which):
    """The leaky continuation's element (dd_trig: the trigonometric branch in
    double-float, dsincos) against 50 digits. There the phase x = k h |w|
    of a wave reaches several hundred radians, and a double-float phase
    carries an absolute error of a few units of 2^-48 |x| (k h, w = sqrt(-w2)
    and their product each round once or twice), which sine and cosine pass
    on unchanged. Above the shear speeds the element takes its plain forms,
    which cancel at some points for both forms alike; there the error scales
    with the unit roundoff, 2^-47 for a double-float product or sum against
    2^-53, a ratio of 64. Bar, at every point: no worse than the FP64 element
    by more than a factor 100, or than 1e-11, or than 64 x 2^-48 x the
    point's largest phase; median 1e-12."""
    if which == "leaky":
        m, g = W.leaky_batch(n_models=32)
    else:
        m, _ = W.ragged_batch(n_models=32)
        g = W.Grid(500.0, 0.25, 3001)
    rng = np.random.default_rng(19)
    pts = leaky_points(m, g, rng, 300)

    def phase(c, h, a, bb, k):
        return k * h * max(math.sqrt(max(c * c / (bb * bb) - 1.0, 0.0)),
                           math.sqrt(max(c * c / (a * a) - 1.0, 0.0)))

    x = np.array([phase(c, h, a, bb, k) for _, _, c, h, a, bb, _, k in pts])
    assert x.max() > 20.0  # the reduction by pi/2 takes several quadrants
    with masw.Batch(m, g) as b:
        fp, df = masw.element_check(b.handle, [p[0] for p in pts], [p[1] for p in pts],
                                    [p[2] for p in pts], dd_trig=True)
    err_df, err_fp = [], []
    for t, (_, _, c, h, a, bb, r, k) in enumerate(pts):
        ref = reference_entries(h, a, bb, r, k, c)
        scale = np.abs(ref).max()
        err_df.append(np.abs(df[t, 1:] / df[t, 0] - ref).max() / scale)
        err_fp.append(np.abs(fp[t, 1:] / fp[t, 0] - ref).max() / scale)
    err_df, err_fp = np.array(err_df), np.array(err_fp)
    w = int(np.argmax(err_df))
    print(f"{which}: double-float max {err_df.max():.1e} (phase {x[w]:.0f}, FP64 there "
          f"{err_fp[w]:.1e}) median {np.median(err_df):.1e}; FP64 max {err_fp.max():.1e} "
          f"median {np.median(err_fp):.1e}; largest phase {x.max():.0f}")
    assert np.isfinite(err_df).all()
    assert np.median(err_df) <= 1e-12
    bar = np.maximum(np.maximum(100 * err_fp, 1e-11), 64 * 2.0 ** -48 * x)
    assert (err_df <= bar).all(), np.nonzero(err_df > bar)
