"""The constants of the double-float element (csrc/masw_df.cuh) are what
their definitions say: each table entry (hi, lo) is hi = the nearest float
of the exact value v and lo = the nearest float of v - hi (60-digit mpmath),
for 2^(j/256), 2^(-i/256) - 1, 2^(-i/256), 1/(2n)! and 1/(2n+1)!; ln 2/256
splits into L1 + L2 + L3 with L1 and L2 of at most 9 significant bits (so
n L1 and n L2 are exact floats for |n| < 2^15) and the three summing to
ln 2/256 within 2^-48 of it. CPU only: the source file is read as text."""
import os
import re
import struct

import mpmath as mp
import pytest

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2003_02256_gb300", "csrc",
                      "masw_df.cuh")


def f32(x):
    return struct.unpack("f", struct.pack("f", float(x)))[0]


def hexfloat(tok):
    return float.fromhex(tok.rstrip("f"))


def table(src, name):
    m = re.search(name + r"\[(\d+)\] = \{(.*?)\n\};", src, re.S)
    pairs = re.findall(r"\{(-?0x[0-9a-f.]+p[+-]\d+f), (-?0x[0-9a-f.]+p[+-]\d+f)\}", m.group(2))
    assert len(pairs) == int(m.group(1))
    return [(hexfloat(a), hexfloat(b)) for a, b in pairs]


def constant(src, name):
    return hexfloat(re.search(name + r" = (-?0x[0-9a-f.]+p[+-]\d+f);", src).group(1))


@pytest.fixture(scope="module")
def src():
    with open(HEADER) as f:
        return f.read()


def nearest_pair(v):
    hi = f32(v)
    return hi, f32(v - mp.mpf(hi))


@pytest.mark.parametrize("name,value", [
    ("EXP2_DF", lambda j: mp.power(2, mp.mpf(j) / 256)),
    ("EXPM1_DF", lambda i: mp.power(2, -mp.mpf(i) / 256) - 1),
    ("EXP2N_DF", lambda i: mp.power(2, -mp.mpf(i) / 256)),
    ("COSH_DF", lambda n: 1 / mp.factorial(2 * n)),
    ("SINH_DF", lambda n: 1 / mp.factorial(2 * n + 1)),
])
def test_table_entries_are_nearest_float_pairs(src, name, value):
    with mp.workdps(60):
        for j, (hi, lo) in enumerate(table(src, name)):
            v = value(j)
            assert (hi, lo) == nearest_pair(v), (name, j)
            assert abs((mp.mpf(hi) + mp.mpf(lo)) - v) <= abs(v) * mp.mpf(2) ** -48, (name, j)


def test_table_sizes_cover_the_reductions(src):
    # e^-x for x < 87: n = round(-x 256/ln2) >= -32132, so j = n mod 256 and
    # 2^(n >> 8) >= 2^-126; e^y - 1 for -0.35 < y: i = -n <= 130
    assert len(table(src, "EXP2_DF")) == 256
    assert len(table(src, "EXPM1_DF")) == len(table(src, "EXP2N_DF")) == 131
    assert int(round(-87 * 256 / 0.6931471805599453)) >> 8 >= -126
    assert round(0.35 * 256 / 0.6931471805599453) <= 130


def test_reduction_constants(src):
    L1, L2, L3 = (constant(src, f"DF_LN2_256_{i}") for i in (1, 2, 3))
    inv = constant(src, "DF_INV_LN2_256")
    for v in (L1, L2):
        m, e = mp.frexp(mp.mpf(v))
        assert int(abs(m) * 2 ** 9) == abs(m) * 2 ** 9  # at most 9 significant bits
    with mp.workdps(60):
        L = mp.log(2) / 256
        assert abs(mp.mpf(L1) + mp.mpf(L2) + mp.mpf(L3) - L) <= L * mp.mpf(2) ** -48
        assert inv == f32(256 / mp.log(2))
    # n L1 and n L2 exact in float for |n| < 2^15
    for n in (1, 129, 32132, 32767):
        assert f32(n * L1) == n * L1 and f32(n * L2) == n * L2


def test_pi_over_2_reduction_constants(src):
    """pi/2 = P1 + P2 + P3 + P4 within 2^-80 of it, P1 and P2 of at most 12
    significant bits (j P1 and j P2 exact floats for 0 <= j < 2^12), P3 and
    P4 the nearest floats of the successive remainders; 2/pi the nearest
    float. The double-float sine and cosine reduce by these."""
    P = [constant(src, f"DF_PIO2_{i}") for i in (1, 2, 3, 4)]
    for v in P[:2]:
        m, e = mp.frexp(mp.mpf(v))
        assert int(abs(m) * 2 ** 12) == abs(m) * 2 ** 12
    with mp.workdps(60):
        H = mp.pi / 2
        assert P[2] == f32(H - P[0] - P[1])
        assert P[3] == f32(H - P[0] - P[1] - mp.mpf(P[2]))
        assert abs(sum(mp.mpf(p) for p in P) - H) <= mp.mpf(2) ** -80
        assert constant(src, "DF_TWO_OVER_PI") == f32(2 / mp.pi)
    for j in (1, 3, 1000, 4095):
        assert f32(j * P[0]) == j * P[0] and f32(j * P[1]) == j * P[1]
