"""The benchmark's evaluation model follows the library's split search (CPU
only): its anchor stride is the one the kernels are built with."""
import math
import os
import re

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_search_stride_matches_the_kernels():
    src = open(os.path.join(HERE, "..", "paper_2003_02256_gb300", "csrc", "masw_internal.h")).read()
    m = re.search(r"constexpr int SEARCH_STRIDE = (\d+);", src)
    assert m and int(m.group(1)) == bench.SEARCH_STRIDE


def _single(npf, r):
    # count_search_single on a count that turns nonzero at r
    if npf < 1:
        return 0
    lo, hi, ev = -1, npf - 1, 0
    while hi - lo > 1:
        mid = lo + ((hi - lo) >> 1)
        ev += 1
        if mid >= r:
            hi = mid
        else:
            lo = mid
    return ev + (hi == npf - 1)


def _guess(npf, r, na, nb, x, d):
    # search_guess and count_search_guess, item by item
    if npf < 1:
        return 0
    if na < 1 or nb < 1:
        return _single(npf, r)
    g = min(max(math.floor(na + (nb - na) * x / d - 0.25), 0), npf - 1)
    ev = 1
    if g >= r:
        hi, lo, step = g, -1, 1
        while hi > 0:
            p = max(hi - step, 0)
            ev += 1
            if p < r:
                lo = p
                break
            hi, step = p, step * 2
    else:
        lo, hi, step = g, -1, 1
        while lo < npf - 1:
            p = min(lo + step, npf - 1)
            ev += 1
            if p >= r:
                hi = p
                break
            lo, step = p, step * 2
        if hi < 0:
            return ev
    while hi - lo > 1:
        mid = lo + ((hi - lo) >> 1)
        ev += 1
        if mid >= r:
            hi = mid
        else:
            lo = mid
    return ev


def test_search_evaluation_model_matches_the_step_by_step_search():
    import numpy as np

    rng = np.random.default_rng(3)

    class Models:
        n_models = 40
        n_lambda = rng.integers(1, 50, 40)

    Models.n_items = int(Models.n_lambda.sum())
    npf = rng.integers(0, 400, Models.n_items)
    root = rng.integers(0, 420, Models.n_items)
    got = bench.split_search_evals(Models, npf, root)
    S = bench.SEARCH_STRIDE
    woff = np.concatenate([[0], np.cumsum(Models.n_lambda)])
    loc = lambda q: int(root[q]) if root[q] < npf[q] else -1
    for m in range(Models.n_models):
        first, last = int(woff[m]), int(woff[m + 1]) - 1
        for j in range(first, last + 1):
            r = int(root[j]) if root[j] < npf[j] else 10 ** 9
            if (j - first) % S == 0 or j == last:
                want = _single(int(npf[j]), r)
            else:
                ja = first + ((j - first) // S) * S
                jb = min(ja + S, last)
                want = _guess(int(npf[j]), r, loc(ja), loc(jb), j - ja, jb - ja)
            assert got[j] == want, (m, j)
