"""Write the double-float constants of masw_df.cuh (run by hand; the CPU test
tests/test_df_tables.py checks the header against the same definitions).

Each value v is stored as the pair (hi, lo) of floats with hi the nearest
float of v and lo the nearest float of v - hi, from 60-digit mpmath:
  EXP2_DF[j]   = 2^(j/256),          j = 0..255
  EXPM1_DF[i]  = 2^(-i/256) - 1,     i = 0..130
  EXP2N_DF[i]  = 2^(-i/256),         i = 0..130
  COSH_DF[n]   = 1/(2n)!,            n = 0..9
  SINH_DF[n]   = 1/(2n+1)!,          n = 0..8
the reduction constants of ln 2 / 256 as three floats L1 + L2 + L3 with
L1 and L2 rounded to 9 significant bits (so n L1 and n L2 are exact for
|n| < 2^15) and L3 the nearest float of the rest, and those of pi / 2 as
four floats P1 + P2 + P3 + P4 with P1 and P2 rounded to 12 significant bits
(j P1 and j P2 exact for 0 <= j < 2^12), P3 the nearest float of the rest
and P4 the nearest float of what remains, with 2 / pi as a float."""
import struct

import mpmath as mp


def f32(x):
    return struct.unpack("f", struct.pack("f", float(x)))[0]


def hexf(x):
    return float(x).hex()


def split(v):
    hi = f32(v)
    lo = f32(v - mp.mpf(hi))
    return hi, lo


def round_bits(v, bits):
    e = mp.floor(mp.log(abs(v), 2))
    q = mp.mpf(2) ** (e - bits + 1)
    return mp.nint(v / q) * q


def tables():
    with mp.workdps(60):
        exp2 = [split(mp.power(2, mp.mpf(j) / 256)) for j in range(256)]
        expm1 = [split(mp.power(2, -mp.mpf(i) / 256) - 1) for i in range(131)]
        exp2n = [split(mp.power(2, -mp.mpf(i) / 256)) for i in range(131)]
        L = mp.log(2) / 256
        L1 = round_bits(L, 9)
        L2 = round_bits(L - L1, 9)
        L3 = f32(L - L1 - L2)
        inv = f32(256 / mp.log(2))
        H = mp.pi / 2
        P1 = round_bits(H, 12)
        P2 = round_bits(H - P1, 12)
        P3 = f32(H - P1 - P2)
        P4 = f32(H - P1 - P2 - mp.mpf(P3))
        pio2 = (float(P1), float(P2), P3, P4, f32(2 / mp.pi))
        # Taylor coefficients of cosh(x) and sinh(x)/x in u = x^2
        cosh_c = [split(1 / mp.factorial(2 * n)) for n in range(10)]
        sinh_c = [split(1 / mp.factorial(2 * n + 1)) for n in range(9)]
    return exp2, expm1, exp2n, (float(L1), float(L2), L3), inv, cosh_c, sinh_c, pio2


def emit():
    exp2, expm1, exp2n, (L1, L2, L3), inv, cosh_c, sinh_c, pio2 = tables()
    out = []
    def arr(name, vals):
        out.append(f"__device__ const float2 {name}[{len(vals)}] = {{")
        for i in range(0, len(vals), 2):
            out.append("    " + " ".join(f"{{{hexf(h)}f, {hexf(l)}f}}," for h, l in vals[i:i + 2]))
        out.append("};")
    arr("EXP2_DF", exp2)
    arr("EXPM1_DF", expm1)
    arr("EXP2N_DF", exp2n)
    arr("COSH_DF", cosh_c)
    arr("SINH_DF", sinh_c)
    out.append(f"constexpr float DF_LN2_256_1 = {hexf(L1)}f;")
    out.append(f"constexpr float DF_LN2_256_2 = {hexf(L2)}f;")
    out.append(f"constexpr float DF_LN2_256_3 = {hexf(L3)}f;")
    out.append(f"constexpr float DF_INV_LN2_256 = {hexf(inv)}f;")
    for i in range(4):
        out.append(f"constexpr float DF_PIO2_{i + 1} = {hexf(pio2[i])}f;")
    out.append(f"constexpr float DF_TWO_OVER_PI = {hexf(pio2[4])}f;")
    return "\n".join(out)


if __name__ == "__main__":
    print(emit())
