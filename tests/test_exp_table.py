"""The constants of the library's FP64 exponential (csrc/masw_device.cuh,
exp_neg: table-driven after Tang, ACM TOMS 1989) are the nearest doubles of
their exact values: 2^(j/2048) for j = 0..2047, 2048/ln 2, ln 2/2048 and the
remainder of ln 2/2048 after its nearest double (60-digit mpmath). CPU only:
the source file is read as text."""
import os
import re

import mpmath as mp

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2003_02256_gb300", "csrc",
                      "masw_device.cuh")


def read_header():
    with open(HEADER) as f:
        return f.read()


def test_table_entries_are_the_nearest_doubles():
    src = read_header()
    body = re.search(r"EXP2_TABLE\[2048\] = \{(.*?)\};", src, re.S).group(1)
    vals = [float.fromhex(t) for t in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 2048
    with mp.workdps(60):
        for j, v in enumerate(vals):
            assert v == float(mp.power(2, mp.mpf(j) / 2048)), j


def test_reduction_constants_are_the_nearest_doubles():
    src = read_header()

    def const(name):
        return float.fromhex(re.search(name + r" = (0x[0-9a-f.]+p[+-]\d+);", src).group(1))

    with mp.workdps(60):
        ln2_n = mp.log(2) / 2048
        assert const("INV_LN2_N") == float(2048 / mp.log(2))
        hi = const("LN2_N_HI")
        assert hi == float(ln2_n)
        assert const("LN2_N_LO") == float(ln2_n - mp.mpf(hi))
