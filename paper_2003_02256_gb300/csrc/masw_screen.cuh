// masw_screen.cuh -- FP32 screen of the determinant sign (GB300 two-precision
// scan).
//
// GB300 issues 2 FP64 FMAs per clock per SM against 128 FP32 FMAs, so the
// FP64 recurrence of masw_device.cuh costs ~64x the same arithmetic in FP32.
// The screen evaluates the same element stiffness and the same homogeneous
// Schur recurrence in FP32 to LOCATE the first sign change n32; the result
// reported by the library is always decided by the FP64 recurrence
// (masw_device.cuh::det_sign) at V[0], V[n32-1] and V[n32], with an FP64
// window re-scan and finally a full FP64 scan whenever they disagree.
//
// FP32-specific care: stiffnesses are divided by the half-space shear
// modulus (a positive common factor, so no sign changes) to keep the
// recurrence far from FP32 overflow; the Taylor series is cut where its
// remainder falls below FP32 rounding; exponentials and reciprocal square
// roots use the SFU; the power-of-two rescaling works on FP32 exponent bits,
// both for the recurrence weight and for each layer's numerators and
// denominator (a common factor of K_e's numerator and denominator).
//
// Below a layer's shear speed (r, s real) the plain denominator
// D = 2(1 - C_r C_s) + Sd_r Sd_s + Sm_r Sm_s cancels to O(q^2) of its terms
// (q = c^2/beta^2 small for stiff layers at low c), which in FP32 gives the
// wrong sign. There the screen uses the exact rearrangement
//   D = (1 - rs)^2 Sd_r Sd_s - 4 sinh^2(k h (r - s) / 2),
//   1 - rs = (p + q - pq) / (1 + rs),  r - s = (q - p) / (r + s),
// and C_r - C_s = 2 sinh((x_r + x_s)/2) sinh((x_r - x_s)/2), whose terms
// carry no cancellation (scaled by exp(-x_r - x_s) like every other term).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace masw {

// FP32 layer record: h, mu/mu_ref, rho/mu_ref, 1/alpha^2, 1/beta^2,
// 1/beta^2 - 1/alpha^2 (rounded once from FP64), pad x2.
enum LayerField32 { F_H = 0, F_MU = 1, F_RHO = 2, F_IA2 = 3, F_IB2 = 4, F_DIB = 5 };
constexpr int LAYER_STRIDE32 = 8;

__device__ __forceinline__ int sgnf(float x) { return (x > 0.0f) - (x < 0.0f); }

__device__ __forceinline__ bool pow2_normaliser_f(float x, float* scale) {
    int bits = __float_as_int(x);
    int be = (bits >> 23) & 0xff;
    if (be == 0 || be >= 253) return false;
    *scale = __int_as_float((253 - be) << 23);  // 2^-(be - 126): |x * scale| in [0.5, 1)
    return true;
}

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

// Sign of det K at (k, c) in FP32 (same recurrence as det_sign).
__device__ __forceinline__ int det_sign_f(const float* __restrict__ lay, int N, float k, float c) {
    float c2 = c * c;
    float p00 = 0.0f, p01 = 0.0f, p11 = 0.0f, w = 1.0f;
    int sg = 1;
    for (int j = 0; j < N; ++j) {
        const float* L = lay + j * LAYER_STRIDE32;
        float kh = k * L[F_H];
        float q = c2 * L[F_IB2];
        float pp = c2 * L[F_IA2];
        float r2 = 1.0f - pp;
        float s2 = 1.0f - q;
        float Dh, A1, D1, B1, E1, F1, G1;
        if (s2 > 0.0f) {
            // r, s real (c below the layer's shear speed): every term scaled
            // by exp(-x_r - x_s) and written without cancellation
            float rwr = rsqrtf(r2), rws = rsqrtf(s2);
            float r = r2 * rwr, s = s2 * rws;
            float xr = kh * r, xs = kh * s;
            float emr = expm1f(-2.0f * xr), ems = expm1f(-2.0f * xs);
            float hr = -0.5f * emr, hs = -0.5f * ems;             // exp(-x) sinh(x)
            float cr = fmaf(0.5f, emr, 1.0f), cs = fmaf(0.5f, ems, 1.0f);  // exp(-x) cosh(x)
            float Er = __expf(-xr), Es = __expf(-xs);
            float dlt = __fdividef(kh * c2 * L[F_DIB], r + s);  // x_r - x_s >= 0
            float dE = -Es * expm1f(-dlt);                    // E_s - E_r
            float sE = Es + Er;
            float omP = fmaf(-Er, Es, 1.0f);                  // 1 - E_r E_s
            float rs = r * s;
            float om = __fdividef(fmaf(-pp, q, pp + q), 1.0f + rs);  // 1 - rs
            float shd = 0.5f * dE * sE;                       // exp(-x_r-x_s) sinh(x_r-x_s)
            Dh = fmaf(om * om * (hr * rwr), hs * rws, -dE * dE);
            A1 = fmaf(om * cs, hr, -shd) * rws;
            D1 = fmaf(om * cr, hs, shd) * rwr;
            float K2 = fmaf(4.0f - q, rs, fmaf(2.0f * rs, rs, s2 + 1.0f));
            B1 = 0.25f * fmaf(omP * omP, om * fmaf(-2.0f, om, q), dE * dE * K2) * (rwr * rws);
            F1 = -0.5f * dE * omP;
            E1 = fmaf(hr * r, Es, -Er * (hs * rws));
            G1 = fmaf(hs * s, Er, -Es * (hr * rwr));
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
        // K_e = numerators / Dh is unchanged by a common factor: bring Dh to
        // [0.5, 1) so that long wavelengths (Dh ~ (kh)^2 p q) cannot drive the
        // recurrence into FP32 underflow
        float nrm;
        if (!pow2_normaliser_f(Dh, &nrm)) return 0;
        Dh *= nrm;
        A1 *= nrm;
        B1 *= nrm;
        D1 *= nrm;
        E1 *= nrm;
        F1 *= nrm;
        G1 *= nrm;
        float rc2 = L[F_RHO] * c2, mu = L[F_MU];
        float n00 = rc2 * A1, n01 = mu * B1, n11 = rc2 * D1;
        float ce = rc2 * E1, cf = rc2 * F1, cg = rc2 * G1;
        float s00 = fmaf(Dh, p00, w * n00);
        float s01 = fmaf(Dh, p01, w * n01);
        float s11 = fmaf(Dh, p11, w * n11);
        float det = fmaf(s00, s11, -s01 * s01);
        sg *= sgnf(det);
        float t00 = fmaf(s11, ce, s01 * cf);
        float t01 = fmaf(s11, cf, -s01 * cg);
        float t10 = -fmaf(s01, ce, s00 * cf);
        float t11 = fmaf(s00, cg, -s01 * cf);
        float q00 = fmaf(ce, t00, -cf * t10);
        float q01 = fmaf(ce, t01, -cf * t11);
        float q11 = fmaf(cf, t01, cg * t11);
        p00 = fmaf(n00, det, -w * q00);
        p01 = fmaf(-n01, det, -w * q01);
        p11 = fmaf(n11, det, -w * q11);
        float wn = Dh * det;
        float sc;
        if (!pow2_normaliser_f(wn, &sc)) return 0;
        p00 *= sc;
        p01 *= sc;
        p11 *= sc;
        w = wn * sc;
    }
    const float* L = lay + N * LAYER_STRIDE32;
    float q = c2 * L[F_IB2];
    float p = c2 * L[F_IA2];
    float r = sqrtf(1.0f - p);
    float s = sqrtf(1.0f - q);
    float g = fmaf(r, s, 1.0f);
    float den = fmaf(-p, q, p + q);
    float rc2g = L[F_RHO] * c2 * g;
    float m00 = rc2g * r, m01 = L[F_MU] * fmaf(g, q, -2.0f * den), m11 = rc2g * s;
    float s00 = fmaf(den, p00, w * m00);
    float s01 = fmaf(den, p01, w * m01);
    float s11 = fmaf(den, p11, w * m11);
    return sg * sgnf(fmaf(s00, s11, -s01 * s01));
}

}  // namespace masw
