// masw_adjoint.cuh -- forward-mode dual numbers for the element stiffness and
// the null-vector adjoint of the refined root.
//
// At a simple root C* of det K(c; theta) = 0, Jacobi's formula with the
// rank-one adjugate adj K = kappa u u^T (u the null vector of the symmetric K)
// gives the implicit-function derivative
//   dC*/dtheta = - (u^T dK/dtheta u) / (u^T dK/dc u).
// The paper has no gradient ("no backpropagation", Section 2.1); this is the
// differentiation extension of the same stiffness matrix. dK/dtheta comes
// from evaluating each 4x4 element (and the half-space 2x2) in dual numbers
// with three directions: c, the layer's beta (Poisson ratio held, so alpha
// moves with beta) and the layer's thickness h.
#pragma once

#include "masw_device.cuh"

namespace masw {

struct D4 { double v, d0, d1, d2; };

__device__ __forceinline__ D4 mk(double v) { return {v, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ D4 operator+(D4 a, D4 b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
__device__ __forceinline__ D4 operator-(D4 a, D4 b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
__device__ __forceinline__ D4 operator-(D4 a) { return {-a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ D4 operator*(D4 a, D4 b) {
    return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
__device__ __forceinline__ D4 operator*(double s, D4 a) { return {s * a.v, s * a.d0, s * a.d1, s * a.d2}; }
__device__ __forceinline__ D4 operator+(double s, D4 a) { return {s + a.v, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ D4 operator/(D4 a, D4 b) {
    double iv = 1.0 / b.v;
    double q = a.v * iv;
    return {q, (a.d0 - q * b.d0) * iv, (a.d1 - q * b.d1) * iv, (a.d2 - q * b.d2) * iv};
}
__device__ __forceinline__ D4 chain(D4 a, double f, double df) {
    return {f, df * a.d0, df * a.d1, df * a.d2};
}
__device__ __forceinline__ D4 dexp(D4 a) { double e = exp(a.v); return chain(a, e, e); }
__device__ __forceinline__ D4 dsqrt(D4 a) { double s = sqrt(a.v); return chain(a, s, 0.5 / s); }
__device__ __forceinline__ D4 drsqrt(D4 a) {
    double r = rsqrt(a.v);
    return chain(a, r, -0.5 * r * r * r);
}
__device__ __forceinline__ void dsincos(D4 a, D4* s, D4* c) {
    double sn, cs;
    sincos(a.v, &sn, &cs);
    *s = chain(a, sn, cs);
    *c = chain(a, cs, -sn);
}

struct WaveD { D4 E, C, Sd, Sm; };

// Dual version of wave_fns (same branches, same scaling).
__device__ inline WaveD wave_fns_d(D4 kh, D4 w2) {
    D4 u = kh * kh * w2;
    WaveD o;
    if (fabs(u.v) < SERIES_U) {
        D4 pc = mk(inv_fact(18));
        const double cc[9] = {inv_fact(16), inv_fact(14), inv_fact(12), inv_fact(10), inv_fact(8),
                              inv_fact(6), inv_fact(4), inv_fact(2), 1.0};
        for (int i = 0; i < 9; ++i) pc = cc[i] + pc * u;
        D4 ps = mk(inv_fact(17));
        const double cs[8] = {inv_fact(15), inv_fact(13), inv_fact(11), inv_fact(9), inv_fact(7),
                              inv_fact(5), inv_fact(3), 1.0};
        for (int i = 0; i < 8; ++i) ps = cs[i] + ps * u;
        D4 khps = kh * ps;
        o.E = mk(1.0);
        o.C = pc;
        o.Sd = khps;
        o.Sm = w2 * khps;
    } else if (w2.v > 0.0) {
        D4 rw = drsqrt(w2);
        D4 w = w2 * rw;
        D4 E = dexp(-(kh * w));
        D4 E2 = E * E;
        D4 t = 0.5 + (-0.5) * E2;
        o.E = E;
        o.C = 0.5 + 0.5 * E2;
        o.Sd = t * rw;
        o.Sm = t * w;
    } else {
        D4 rw = drsqrt(-w2);
        D4 w = (-w2) * rw;
        D4 sn, cs;
        dsincos(kh * w, &sn, &cs);
        o.E = mk(1.0);
        o.C = cs;
        o.Sd = sn * rw;
        o.Sm = -(w * sn);
    }
    return o;
}

// Element stiffness entries (k dropped) of one finite layer as duals in the
// directions (c, beta, h): K = [[A, B, E, F], [B, Dd, -F, G],
// [E, -F, A, -B], [F, G, -B, Dd]].
struct ElemD { D4 A, B, Dd, E, F, G; };

__device__ inline ElemD layer_element_d(const double* __restrict__ L, double k, double c) {
    D4 cc = {c, 1.0, 0.0, 0.0};
    D4 be = {L[L_BETA], 0.0, 1.0, 0.0};
    D4 hh = {L[L_H], 0.0, 0.0, 1.0};
    double rho = L[L_RHO], ratio = L[L_RATIO];
    D4 c2 = cc * cc;
    D4 b2 = be * be;
    D4 mu = rho * b2;
    D4 q = c2 / b2;
    D4 r2 = 1.0 + (-1.0) * (c2 / ((ratio * ratio) * b2));
    D4 s2 = 1.0 + (-1.0) * q;
    D4 kh = k * hh;
    WaveD R = wave_fns_d(kh, r2);
    WaveD S = wave_fns_d(kh, s2);
    D4 ErEs = R.E * S.E;
    D4 CrCs = R.C * S.C;
    D4 Dh = 2.0 * (ErEs - CrCs) + R.Sd * S.Sd + R.Sm * S.Sm;
    D4 A1 = R.C * S.Sd - S.C * R.Sm;
    D4 D1 = S.C * R.Sd - R.C * S.Sm;
    D4 B1 = (s2 + mk(3.0)) * (CrCs - ErEs) - S.Sm * (2.0 * R.Sm + R.Sd) - R.Sd * S.Sd;
    D4 E1 = R.Sm * S.E - R.E * S.Sd;
    D4 F1 = R.E * S.C - R.C * S.E;
    D4 G1 = S.Sm * R.E - S.E * R.Sd;
    D4 rc2 = rho * c2;
    ElemD o;
    o.A = rc2 * A1 / Dh;
    o.B = mu * B1 / Dh;
    o.Dd = rc2 * D1 / Dh;
    o.E = rc2 * E1 / Dh;
    o.F = rc2 * F1 / Dh;
    o.G = rc2 * G1 / Dh;
    return o;
}

// Half-space 2x2 (k dropped) as duals in (c, beta_hs, unused).
struct HalfD { D4 H00, H01, H11; };

__device__ inline HalfD halfspace_d(const double* __restrict__ L, double c) {
    D4 cc = {c, 1.0, 0.0, 0.0};
    D4 be = {L[L_BETA], 0.0, 1.0, 0.0};
    double rho = L[L_RHO], ratio = L[L_RATIO];
    D4 c2 = cc * cc;
    D4 b2 = be * be;
    D4 mu = rho * b2;
    D4 q = c2 / b2;
    D4 p = c2 / ((ratio * ratio) * b2);
    D4 r = dsqrt(1.0 + (-1.0) * p);
    D4 s = dsqrt(1.0 + (-1.0) * q);
    D4 g = 1.0 + r * s;
    D4 den = (p + q - p * q) / g;  // 1 - r s
    D4 rc2 = rho * c2;
    HalfD o;
    o.H00 = rc2 * r / den;
    o.H01 = mu * (q - 2.0 * den) / den;
    o.H11 = rc2 * s / den;
    return o;
}

// Quadratic form u_e^T K u_e of an element and its three directional
// derivatives; u = (x0, z0, x1, z1).
__device__ __forceinline__ D4 elem_quad(const ElemD& K, double x0, double z0, double x1, double z1) {
    double xx = x0 * x0 + x1 * x1, zz = z0 * z0 + z1 * z1;
    double b = 2.0 * (x0 * z0 - x1 * z1), e = 2.0 * x0 * x1, f = 2.0 * (x0 * z1 - z0 * x1),
           g = 2.0 * z0 * z1;
    return xx * K.A + zz * K.Dd + b * K.B + e * K.E + f * K.F + g * K.G;
}

__device__ __forceinline__ D4 half_quad(const HalfD& H, double x, double z) {
    return (x * x) * H.H00 + (2.0 * x * z) * H.H01 + (z * z) * H.H11;
}

}  // namespace masw
