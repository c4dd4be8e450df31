// masw_screen.cuh -- FP32 screen of the determinant sign (GB300 two-precision
// scan).
//
// GB300 issues 2 FP64 FMAs per clock per SM against 128 FP32 FMAs, so the
// FP64 recurrence of masw_device.cuh costs ~64x the same arithmetic in FP32.
// The screen evaluates the same element stiffness and the same homogeneous
// Schur recurrence in FP32 to LOCATE the first sign change n32; the result
// reported by the library is always decided in FP64: the Wittrick-Williams
// mode count of the FP64 recurrence over double-float elements
// (masw_df.cuh::mode_count_T_df) at V[0],
// V[n32-1] and V[n32], and when it does not confirm, the FP64 search on that
// count (masw_modes.cuh) or finally the FP64 scan.
//
// FP32-specific care: stiffnesses are divided by the half-space shear
// modulus (a positive common factor, so no sign changes) to keep the
// recurrence far from FP32 overflow; the Taylor series is cut where its
// remainder falls below FP32 rounding; exponentials and reciprocal square
// roots and reciprocals use the SFU.
//
// Below a layer's shear speed (r, s real) the plain denominator
// D = 2(1 - C_r C_s) + Sd_r Sd_s + Sm_r Sm_s cancels to O(q^2) of its terms
// (q = c^2/beta^2 small for stiff layers at low c), which in FP32 gives the
// wrong sign. There the screen uses the exact rearrangement
//   D = (1 - rs)^2 Sd_r Sd_s - 4 sinh^2(k h (r - s) / 2),
//   1 - rs = (p + q - pq) / (1 + rs),  r - s = (q - p) / (r + s),
// and C_r - C_s = 2 sinh((x_r + x_s)/2) sinh((x_r - x_s)/2); the K11 and
// coupling numerators are rearranged the same way,
//   A1 s = (1 - rs) C_s S_r - sinh(x_r - x_s),
//   D1 r = (1 - rs) C_r S_s + sinh(x_r - x_s),
//   B1 rs = sinh^2((x_r + x_s)/2) (1 - rs)(q - 2(1 - rs))
//         + sinh^2((x_r - x_s)/2) ((4 - q) rs + 2 r^2 s^2 + s^2 + 1),
// whose terms carry no cancellation (scaled by exp(-x_r - x_s) like every
// other term).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace masw {

// FP32 layer record: h, mu/mu_ref, rho/mu_ref, 1/alpha^2, 1/beta^2,
// 1/beta^2 - 1/alpha^2 (rounded once from FP64), pad x2.
enum LayerField32 { F_H = 0, F_MU = 1, F_RHO = 2, F_IA2 = 3, F_IB2 = 4, F_DIB = 5 };
constexpr int LAYER_STRIDE32 = 8;

__device__ __forceinline__ int sgnf(float x) { return (x > 0.0f) - (x < 0.0f); }

struct WaveF { float E, C, Sd, Sm; };

__device__ __forceinline__ WaveF wave_fns_f(float kh, float w2) {
    float u = kh * kh * w2;
    WaveF o;
    if (fabsf(u) < 1.0f) {
        // cosh(x), sinh(x)/x as series in u = x^2, remainder < 2^-25
        float pc = fmaf(u, 1.0f / 3628800.0f, 1.0f / 40320.0f);
        pc = fmaf(pc, u, 1.0f / 720.0f);
        pc = fmaf(pc, u, 1.0f / 24.0f);
        pc = fmaf(pc, u, 0.5f);
        pc = fmaf(pc, u, 1.0f);
        float ps = fmaf(u, 1.0f / 39916800.0f, 1.0f / 362880.0f);
        ps = fmaf(ps, u, 1.0f / 5040.0f);
        ps = fmaf(ps, u, 1.0f / 120.0f);
        ps = fmaf(ps, u, 1.0f / 6.0f);
        ps = fmaf(ps, u, 1.0f);
        float khps = kh * ps;
        o.E = 1.0f;
        o.C = pc;
        o.Sd = khps;
        o.Sm = w2 * khps;
    } else if (w2 > 0.0f) {
        float rw = rsqrtf(w2);
        float w = w2 * rw;
        float E = __expf(-kh * w);
        float E2 = E * E;
        float t = fmaf(-0.5f, E2, 0.5f);
        o.E = E;
        o.C = fmaf(0.5f, E2, 0.5f);
        o.Sd = t * rw;
        o.Sm = t * w;
    } else {
        float rw = rsqrtf(-w2);
        float w = -w2 * rw;
        float sn, cs;
        sincosf(kh * w, &sn, &cs);
        o.E = 1.0f;
        o.C = cs;
        o.Sd = sn * rw;
        o.Sm = -w * sn;
    }
    return o;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// exp(y) - 1 for y <= 0: Taylor polynomial near 0 (remainder < 2e-8
// relative for y > -0.35), exp(y) - 1 from the SFU otherwise.
__device__ __forceinline__ float expm1_neg(float y) {
    if (y > -0.35f) {
        float p = fmaf(y, 1.0f / 5040.0f, 1.0f / 720.0f);
        p = fmaf(p, y, 1.0f / 120.0f);
        p = fmaf(p, y, 1.0f / 24.0f);
        p = fmaf(p, y, 1.0f / 6.0f);
        p = fmaf(p, y, 0.5f);
        p = fmaf(p, y, 1.0f);
        return p * y;
    }
    return __expf(y) - 1.0f;
}

// Number of negative eigenvalues of a symmetric 2x2 block from its det and
// first diagonal entry (a zero determinant counts as one).
__device__ __forceinline__ int neg_eigs_2x2(float det, float s00) {
    return det < 0.0f ? 1 : (det > 0.0f ? (s00 < 0.0f ? 2 : 0) : 1);
}

// Sign of det K at (k, c) in FP32 (MODE 0), or the number of its negative
// eigenvalues by Sylvester's law of inertia over the 2x2 Schur pivots
// (MODE 1). Same element stiffness as det_sign (in units of the half-space
// shear modulus) but the plain Schur recurrence S = P + K11,
// P' = K22 - K21 S^-1 K12 with SFU reciprocals: on the FP32 pipe a
// reciprocal is cheaper than the homogeneous bookkeeping the FP64 path uses
// to avoid divisions.
template <int MODE>
__device__ __forceinline__ int det_core_f(const float* __restrict__ lay, int N, float k, float c) {
    float c2 = c * c;
    float p00 = 0.0f, p01 = 0.0f, p11 = 0.0f;
    int sg = MODE == 0 ? 1 : 0;
    for (int j = 0; j < N; ++j) {
        const float4 LA = *reinterpret_cast<const float4*>(lay + j * LAYER_STRIDE32);
        const float2 LB = *reinterpret_cast<const float2*>(lay + j * LAYER_STRIDE32 + 4);
        // LA = (h, mu, rho, 1/alpha^2), LB = (1/beta^2, 1/beta^2 - 1/alpha^2)
        float kh = k * LA.x;
        float q = c2 * LB.x;
        float pp = c2 * LA.w;
        float r2 = 1.0f - pp;
        float s2 = 1.0f - q;
        float Dh, A1, D1, B1, E1, F1, G1;
        if (s2 > 0.0f) {
            // r, s real (c below the layer's shear speed): every term scaled
            // by exp(-x_r - x_s) and written without cancellation
            float rwr = rsqrtf(r2), rws = rsqrtf(s2);
            float r = r2 * rwr, s = s2 * rws;
            float emr1 = expm1_neg(-kh * r), ems1 = expm1_neg(-kh * s);  // exp(-x) - 1
            float Er = 1.0f + emr1, Es = 1.0f + ems1;
            float hr = -0.5f * emr1 * (1.0f + Er), hs = -0.5f * ems1 * (1.0f + Es);  // exp(-x) sinh x
            float cr = 1.0f - hr, cs = 1.0f - hs;                                  // exp(-x) cosh x
            float rs = r * s;
            float irs = rcp_approx(r + s);
            float dE = -Es * expm1_neg(-kh * c2 * LB.y * irs);  // E_s - E_r, x_r - x_s >= 0
            float omP = fmaf(-Er, Es, 1.0f);                     // 1 - E_r E_s
            float om = fmaf(-pp, q, pp + q) * rcp_approx(1.0f + rs);  // 1 - rs
            float shd = 0.5f * dE * (Es + Er);                   // exp(-x_r-x_s) sinh(x_r-x_s)
            float sdr = hr * rwr, sds = hs * rws;
            Dh = fmaf(om * om * sdr, sds, -dE * dE);
            A1 = fmaf(om * cs, hr, -shd) * rws;
            D1 = fmaf(om * cr, hs, shd) * rwr;
            float K2 = fmaf(4.0f - q, rs, fmaf(2.0f * rs, rs, s2 + 1.0f));
            B1 = 0.25f * fmaf(omP * omP, om * fmaf(-2.0f, om, q), dE * dE * K2) * (rwr * rws);
            F1 = -0.5f * dE * omP;
            E1 = fmaf(hr * r, Es, -Er * sds);
            G1 = fmaf(hs * s, Er, -Es * sdr);
        } else {
            WaveF R = wave_fns_f(kh, r2);
            WaveF S = wave_fns_f(kh, s2);
            float ErEs = R.E * S.E;
            float CrCs = R.C * S.C;
            Dh = fmaf(2.0f, ErEs - CrCs, fmaf(R.Sd, S.Sd, R.Sm * S.Sm));
            A1 = fmaf(R.C, S.Sd, -S.C * R.Sm);
            D1 = fmaf(S.C, R.Sd, -R.C * S.Sm);
            B1 = fmaf(s2 + 3.0f, CrCs - ErEs, -fmaf(S.Sm, fmaf(2.0f, R.Sm, R.Sd), R.Sd * S.Sd));
            E1 = fmaf(R.Sm, S.E, -R.E * S.Sd);
            F1 = fmaf(R.E, S.C, -R.C * S.E);
            G1 = fmaf(S.Sm, R.E, -S.E * R.Sd);
        }
        // element blocks K = numerators / Dh (k and mu_ref dropped)
        float iD = rcp_approx(Dh);
        float fr = LA.z * c2 * iD, fm = LA.y * iD;
        float n00 = fr * A1, n01 = fm * B1, n11 = fr * D1;
        float ce = fr * E1, cf = fr * F1, cg = fr * G1;
        float s00 = p00 + n00, s01 = p01 + n01, s11 = p11 + n11;
        float det = fmaf(s00, s11, -s01 * s01);
        if (MODE == 0) sg *= sgnf(det);
        else sg += neg_eigs_2x2(det, s00);
        float idet = rcp_approx(det);
        // P' = K22 - K21 adj(S) K12 / det,  K12 = [[ce, cf], [-cf, cg]]
        float t00 = fmaf(s11, ce, s01 * cf);
        float t01 = fmaf(s11, cf, -s01 * cg);
        float t10 = -fmaf(s01, ce, s00 * cf);
        float t11 = fmaf(s00, cg, -s01 * cf);
        float q00 = fmaf(ce, t00, -cf * t10);
        float q01 = fmaf(ce, t01, -cf * t11);
        float q11 = fmaf(cf, t01, cg * t11);
        p00 = fmaf(-idet, q00, n00);
        p01 = fmaf(-idet, q01, -n01);
        p11 = fmaf(-idet, q11, n11);
    }
    const float4 LA = *reinterpret_cast<const float4*>(lay + N * LAYER_STRIDE32);
    const float LBx = lay[N * LAYER_STRIDE32 + 4];
    float q = c2 * LBx;
    float p = c2 * LA.w;
    float r = sqrtf(1.0f - p);
    float s = sqrtf(1.0f - q);
    float g = fmaf(r, s, 1.0f);
    float iden = rcp_approx(fmaf(-p, q, p + q));
    float rc2g = LA.z * c2 * g * iden;
    float s00 = fmaf(rc2g, r, p00);
    float s01 = fmaf(LA.y * iden, fmaf(g, q, -2.0f * fmaf(-p, q, p + q)), p01);
    float s11 = fmaf(rc2g, s, p11);
    float dl = fmaf(s00, s11, -s01 * s01);
    if (MODE == 0) return sg * sgnf(dl);
    return sg + neg_eigs_2x2(dl, s00);
}

__device__ __forceinline__ int det_sign_f(const float* __restrict__ lay, int N, float k, float c) {
    return det_core_f<0>(lay, N, k, c);
}
__device__ __forceinline__ int inertia_f(const float* __restrict__ lay, int N, float k, float c) {
    return det_core_f<1>(lay, N, k, c);
}

// J0 of one layer (modes with both faces clamped below c) in FP32 from the
// FP32 record: the thickness-halving count of clamped_modes (masw_device.cuh)
// with wave_fns_f at the finest level, h / 2^lv with 2^lv > x =
// k h sqrt(c^2/beta^2 - 1) / pi >= 2^(lv-1), and the doubling
// E(2x) = E^2, C(2x) = 2C^2 - E^2, Sd(2x) = 2 Sd C, Sm(2x) = 2 Sm C up to h.
// For locating events only: every located event is certified on the FP64
// count.
__device__ __forceinline__ int clamped_modes_f(const float* __restrict__ L, float k, float c2) {
    const float q = c2 * L[F_IB2];
    if (!(q > 1.0f)) return 0;
    const float kh = k * L[F_H];
    const float x = kh * sqrtf(q - 1.0f) * 0.318309886f;  // 1/pi
    if (!(x >= 1.0f && x < 1.0e30f)) return 0;
    const int lv = ((__float_as_int(x) >> 23) & 0xff) - 126;  // 2^lv > x >= 2^(lv-1)
    const float khf = kh * __int_as_float((127 - lv) << 23);  // kh 2^-lv, exact
    WaveF R = wave_fns_f(khf, fmaf(-c2, L[F_IA2], 1.0f));
    WaveF S = wave_fns_f(khf, 1.0f - q);
    int J = 0;
    for (int j = lv; j >= 1; --j) {
        if (j < lv) {
            R = WaveF{R.E * R.E, fmaf(2.0f * R.C, R.C, -R.E * R.E), 2.0f * R.Sd * R.C,
                      2.0f * R.Sm * R.C};
            S = WaveF{S.E * S.E, fmaf(2.0f * S.C, S.C, -S.E * S.E), 2.0f * S.Sd * S.C,
                      2.0f * S.Sm * S.C};
        }
        const float D = fmaf(2.0f, fmaf(R.E, S.E, -R.C * S.C), fmaf(R.Sd, S.Sd, R.Sm * S.Sm));
        const float an = fmaf(R.C, S.Sd, -S.C * R.Sm);
        const float dn = fmaf(S.C, R.Sd, -R.C * S.Sm);
        J = 2 * J + (int)((an < 0.0f) != (D < 0.0f)) + (int)((dn < 0.0f) != (D < 0.0f));
    }
    return J;
}

// The Wittrick-Williams mode count T = s + 2 J0 in FP32 (inertia_f and
// clamped_modes_f): exact T never decreases along the grid and jumps by an odd
// amount where det K changes sign; the FP32 value may be off next to an event.
// Requires c < beta_halfspace.
__device__ __forceinline__ int mode_count_T_f(const float* __restrict__ lay, int N, float k,
                                              float c) {
    const int s = inertia_f(lay, N, k, c);
    const float c2 = c * c;
    int j0 = 0;
    for (int j = 0; j < N; ++j) j0 += clamped_modes_f(lay + j * LAYER_STRIDE32, k, c2);
    return s + 2 * j0;
}

}  // namespace masw

// ---------------------------------------------------------------------
// Paired evaluation: two test velocities per thread in packed FP32x2
// arithmetic (fma/mul/add.rn.f32x2). The FP32 pipe runs the same number of
// lane operations either way, but one packed instruction issues two of them,
// and the screen is issue-bound. SFU operations stay per element. When the
// two points of a layer take different branches the layer is evaluated per
// element with the scalar code.
namespace masw {

struct f2 { unsigned long long v; };

__device__ __forceinline__ f2 P2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 B2(float a) { return P2(a, a); }
__device__ __forceinline__ float X(f2 a) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
    return x;
}
__device__ __forceinline__ float Y(f2 a) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
    return y;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// a * b - c
__device__ __forceinline__ f2 fms2(f2 a, f2 b, f2 c) { return fma2(a, b, mul2(c, B2(-1.0f))); }

__device__ __forceinline__ f2 expm1_neg2(f2 y) {
    float yx = X(y), yy = Y(y);
    if (yx > -0.35f && yy > -0.35f) {
        f2 p = fma2(y, B2(1.0f / 5040.0f), B2(1.0f / 720.0f));
        p = fma2(p, y, B2(1.0f / 120.0f));
        p = fma2(p, y, B2(1.0f / 24.0f));
        p = fma2(p, y, B2(1.0f / 6.0f));
        p = fma2(p, y, B2(0.5f));
        p = fma2(p, y, B2(1.0f));
        return mul2(p, y);
    }
    return P2(expm1_neg(yx), expm1_neg(yy));
}

// One layer's element numerators (scalar, any branch), for the mixed case.
__device__ __forceinline__ void layer_nums_f(float kh, float c2, float pp, float q, float dib,
                                             float* Dh, float* A1, float* B1, float* D1, float* E1,
                                             float* F1, float* G1) {
    float r2 = 1.0f - pp, s2 = 1.0f - q;
    if (s2 > 0.0f) {
        float rwr = rsqrtf(r2), rws = rsqrtf(s2);
        float r = r2 * rwr, s = s2 * rws;
        float emr1 = expm1_neg(-kh * r), ems1 = expm1_neg(-kh * s);
        float Er = 1.0f + emr1, Es = 1.0f + ems1;
        float hr = -0.5f * emr1 * (1.0f + Er), hs = -0.5f * ems1 * (1.0f + Es);
        float cr = 1.0f - hr, cs = 1.0f - hs;
        float rs = r * s;
        float dE = -Es * expm1_neg(-kh * c2 * dib * rcp_approx(r + s));
        float omP = fmaf(-Er, Es, 1.0f);
        float om = fmaf(-pp, q, pp + q) * rcp_approx(1.0f + rs);
        float shd = 0.5f * dE * (Es + Er);
        float sdr = hr * rwr, sds = hs * rws;
        *Dh = fmaf(om * om * sdr, sds, -dE * dE);
        *A1 = fmaf(om * cs, hr, -shd) * rws;
        *D1 = fmaf(om * cr, hs, shd) * rwr;
        float K2 = fmaf(4.0f - q, rs, fmaf(2.0f * rs, rs, s2 + 1.0f));
        *B1 = 0.25f * fmaf(omP * omP, om * fmaf(-2.0f, om, q), dE * dE * K2) * (rwr * rws);
        *F1 = -0.5f * dE * omP;
        *E1 = fmaf(hr * r, Es, -Er * sds);
        *G1 = fmaf(hs * s, Er, -Es * sdr);
    } else {
        WaveF R = wave_fns_f(kh, r2);
        WaveF S = wave_fns_f(kh, s2);
        float ErEs = R.E * S.E;
        float CrCs = R.C * S.C;
        *Dh = fmaf(2.0f, ErEs - CrCs, fmaf(R.Sd, S.Sd, R.Sm * S.Sm));
        *A1 = fmaf(R.C, S.Sd, -S.C * R.Sm);
        *D1 = fmaf(S.C, R.Sd, -R.C * S.Sm);
        *B1 = fmaf(s2 + 3.0f, CrCs - ErEs, -fmaf(S.Sm, fmaf(2.0f, R.Sm, R.Sd), R.Sd * S.Sd));
        *E1 = fmaf(R.Sm, S.E, -R.E * S.Sd);
        *F1 = fmaf(R.E, S.C, -R.C * S.E);
        *G1 = fmaf(S.Sm, R.E, -S.E * R.Sd);
    }
}

// Signs of det K at two test velocities (ca, cb) in packed FP32.
__device__ __forceinline__ void det_sign_f2(const float* __restrict__ lay, int N, float k, float ca,
                                            float cb, int* sa, int* sb) {
    const f2 one = B2(1.0f);
    f2 c2 = P2(ca * ca, cb * cb);
    f2 p00 = B2(0.0f), p01 = B2(0.0f), p11 = B2(0.0f);
    unsigned neg_a = 0, neg_b = 0, zero = 0;
    for (int j = 0; j < N; ++j) {
        const float4 LA = *reinterpret_cast<const float4*>(lay + j * LAYER_STRIDE32);
        const float2 LB = *reinterpret_cast<const float2*>(lay + j * LAYER_STRIDE32 + 4);
        float kh = k * LA.x;
        f2 q = mul2(c2, B2(LB.x));
        f2 pp = mul2(c2, B2(LA.w));
        f2 s2 = sub2(one, q);
        f2 Dh, A1, B1, D1, E1, F1, G1;
        bool ra = X(s2) > 0.0f, rb = Y(s2) > 0.0f;
        if (ra && rb) {
            f2 r2 = sub2(one, pp);
            f2 rwr = P2(rsqrtf(X(r2)), rsqrtf(Y(r2)));
            f2 rws = P2(rsqrtf(X(s2)), rsqrtf(Y(s2)));
            f2 r = mul2(r2, rwr), s = mul2(s2, rws);
            f2 nkh = B2(-kh);
            f2 emr1 = expm1_neg2(mul2(nkh, r)), ems1 = expm1_neg2(mul2(nkh, s));
            f2 Er = add2(one, emr1), Es = add2(one, ems1);
            f2 hr = mul2(emr1, fma2(B2(-0.5f), emr1, B2(-1.0f)));  // exp(-x) sinh x
            f2 hs = mul2(ems1, fma2(B2(-0.5f), ems1, B2(-1.0f)));
            f2 cr = sub2(one, hr), cs = sub2(one, hs);
            f2 rs = mul2(r, s);
            f2 rps = add2(r, s);
            f2 irs = P2(rcp_approx(X(rps)), rcp_approx(Y(rps)));
            f2 dlt = mul2(mul2(B2(-kh * LB.y), c2), irs);  // -(x_r - x_s)
            f2 dE = mul2(mul2(Es, expm1_neg2(dlt)), B2(-1.0f));  // E_s - E_r
            f2 omP = fms2(B2(-1.0f), mul2(Er, Es), B2(-1.0f));     // 1 - Er Es
            f2 ops = add2(one, rs);
            f2 num = fms2(add2(pp, q), one, mul2(pp, q));
            f2 om = mul2(num, P2(rcp_approx(X(ops)), rcp_approx(Y(ops))));  // 1 - rs
            f2 shd = mul2(mul2(B2(0.5f), dE), add2(Es, Er));
            f2 sdr = mul2(hr, rwr), sds = mul2(hs, rws);
            f2 dE2 = mul2(dE, dE);
            Dh = fms2(mul2(mul2(om, om), sdr), sds, dE2);
            A1 = mul2(fms2(mul2(om, cs), hr, shd), rws);
            D1 = mul2(fma2(mul2(om, cr), hs, shd), rwr);
            f2 K2 = fma2(sub2(B2(4.0f), q), rs, fma2(add2(rs, rs), rs, sub2(B2(2.0f), q)));
            f2 t1 = mul2(mul2(omP, omP), mul2(om, fma2(B2(-2.0f), om, q)));
            B1 = mul2(mul2(B2(0.25f), fma2(dE2, K2, t1)), mul2(rwr, rws));
            F1 = mul2(mul2(B2(-0.5f), dE), omP);
            E1 = fms2(mul2(hr, r), Es, mul2(Er, sds));
            G1 = fms2(mul2(hs, s), Er, mul2(Es, sdr));
        } else {
            float da, aa, ba, dda, ea, fa, ga, db, ab, bb, ddb, eb, fb, gb;
            layer_nums_f(kh, X(c2), X(pp), X(q), LB.y, &da, &aa, &ba, &dda, &ea, &fa, &ga);
            layer_nums_f(kh, Y(c2), Y(pp), Y(q), LB.y, &db, &ab, &bb, &ddb, &eb, &fb, &gb);
            Dh = P2(da, db);
            A1 = P2(aa, ab);
            B1 = P2(ba, bb);
            D1 = P2(dda, ddb);
            E1 = P2(ea, eb);
            F1 = P2(fa, fb);
            G1 = P2(ga, gb);
        }
        f2 iD = P2(rcp_approx(X(Dh)), rcp_approx(Y(Dh)));
        f2 fr = mul2(mul2(B2(LA.z), c2), iD), fm = mul2(B2(LA.y), iD);
        f2 n00 = mul2(fr, A1), n01 = mul2(fm, B1), n11 = mul2(fr, D1);
        f2 ce = mul2(fr, E1), cf = mul2(fr, F1), cg = mul2(fr, G1);
        f2 s00 = add2(p00, n00), s01 = add2(p01, n01), s11 = add2(p11, n11);
        f2 det = fms2(s00, s11, mul2(s01, s01));
        float dx = X(det), dy = Y(det);
        neg_a ^= __float_as_uint(dx);
        neg_b ^= __float_as_uint(dy);
        zero |= (dx == 0.0f) | ((dy == 0.0f) << 1);
        f2 idet = P2(rcp_approx(dx), rcp_approx(dy));
        f2 t00 = fma2(s11, ce, mul2(s01, cf));
        f2 t01 = fms2(s11, cf, mul2(s01, cg));
        f2 t10 = mul2(fma2(s01, ce, mul2(s00, cf)), B2(-1.0f));
        f2 t11 = fms2(s00, cg, mul2(s01, cf));
        f2 q00 = fms2(ce, t00, mul2(cf, t10));
        f2 q01 = fms2(ce, t01, mul2(cf, t11));
        f2 q11 = fma2(cf, t01, mul2(cg, t11));
        f2 nid = mul2(idet, B2(-1.0f));
        p00 = fma2(nid, q00, n00);
        p01 = fms2(nid, q01, n01);
        p11 = fma2(nid, q11, n11);
    }
    const float4 LA = *reinterpret_cast<const float4*>(lay + N * LAYER_STRIDE32);
    const float LBx = lay[N * LAYER_STRIDE32 + 4];
    int out[2];
    for (int e = 0; e < 2; ++e) {
        float c2e = e ? Y(c2) : X(c2);
        float q = c2e * LBx, p = c2e * LA.w;
        float r = sqrtf(1.0f - p), s = sqrtf(1.0f - q);
        float g = fmaf(r, s, 1.0f);
        float den = fmaf(-p, q, p + q);
        float iden = rcp_approx(den);
        float rc2g = LA.z * c2e * g * iden;
        float s00 = fmaf(rc2g, r, e ? Y(p00) : X(p00));
        float s01 = fmaf(LA.y * iden, fmaf(g, q, -2.0f * den), e ? Y(p01) : X(p01));
        float s11 = fmaf(rc2g, s, e ? Y(p11) : X(p11));
        float dl = fmaf(s00, s11, -s01 * s01);
        unsigned nb = (e ? neg_b : neg_a) ^ __float_as_uint(dl);
        bool z = (dl == 0.0f) || ((zero >> e) & 1);
        out[e] = z ? 0 : ((nb >> 31) ? -1 : 1);
    }
    *sa = out[0];
    *sb = out[1];
}

// Counting search (Wittrick-Williams). With both faces of layer i clamped,
// its energy is mu |grad u|^2 + (lambda + mu) |div u|^2 >= mu |grad u|^2
// (lambda + mu = rho (alpha^2 - beta^2) > 0), and Poincare's inequality in
// depth bounds |grad u|^2 >= (k^2 + (pi/h_i)^2) |u|^2; so no clamped-layer
// mode lies below c_i = beta_i sqrt(1 + (pi / (k h_i))^2). Below
// min_i c_i the element stiffnesses have no pole, the number of negative
// eigenvalues of K(k, c) equals the number of modes below omega = k c, and
// it is non-decreasing in c from 0 at c = 0 (static stiffness positive
// definite). Returns the number of grid points V[n] < (1 - 1e-4) min_i c_i,
// at most nlim (the margin covers the FP32 rounding of the bound).
__device__ __forceinline__ int pole_free_points_f(const float* __restrict__ lay, int N, float k,
                                                  float c0, float dc, int nlim) {
    float cb2 = 3.0e38f;
    for (int j = 0; j < N; ++j) {
        float t = 3.14159265f / (k * lay[j * LAYER_STRIDE32 + F_H]);
        cb2 = fminf(cb2, fmaf(t, t, 1.0f) / lay[j * LAYER_STRIDE32 + F_IB2]);
    }
    float x = (sqrtf(cb2) * (1.0f - 1.0e-4f) - c0) / dc;  // V[n] below the bound: n < x
    if (!(x > 0.0f)) return 0;
    if (x >= (float)nlim) return nlim;
    return min((int)ceilf(x), nlim);
}

}  // namespace masw
