// masw_count.cuh -- counting search with its FP64 certificate for one
// (model, wavenumber) item, run by a pair of adjacent lanes (plan precision 2
// of the batch path and the serving tick).
//
//  * Search (FP32). Inside the pole-free range [0, npf) of pole_free_points_f
//    the negative-eigenvalue count of K (inertia_f) is a non-decreasing step
//    function of the grid index, 0 at c = 0 (Wittrick-Williams below the
//    lowest clamped-layer mode). The pair evaluates the top of the range and
//    its midpoint, then splits the bracket in three per step (one point per
//    lane): about log3(npf) steps instead of Algorithm 1's linear walk. An
//    odd count at the first nonzero point is Algorithm 1's first change.
//  * Certificate (FP64). The count (det_inertia) is 0 at V[n-1] (so 0, and
//    V[0]'s sign, at every point below) and odd at V[n] (the sign differs).
//    When the FP32 count was off by one next to the change (count 0 at both
//    points: the change is higher; nonzero at V[n-1]: lower), the pair takes
//    one FP64 step of two points in that direction, inside the range.
#pragma once

#include "masw_device.cuh"
#include "masw_screen.cuh"

namespace masw {

struct PairCount {
    int cert;   // certified first change (>= 1), or -1
    int n;      // the search's index when the certificate failed (>= 1), or -1
    int start;  // n < 1: the linear scan's start (npf when the range holds no change, else 0)
};

// Both lanes of the pair (lane bit 0 = half, `pair` = their shuffle mask)
// call this with the same item and get the same result. Requires nlim >= 2.
__device__ __forceinline__ PairCount count_certify_pair(const float* __restrict__ lay32,
                                                        const double* __restrict__ lay, int N,
                                                        double k, double c0, double dc, int nlim,
                                                        int half, unsigned pair) {
    const float kf = (float)k;
    const float c0f = (float)c0, dcf = (float)dc;
    const int npf = pole_free_points_f(lay32, N, kf, c0f, dcf, nlim);
    PairCount out{-1, -1, 0};
    int n = -1;
    if (npf >= 1) {
        int lo = -1, hi = npf - 1;
        const int mid = (hi - 1) >> 1;  // midpoint of (lo, hi); -1 when hi == 0
        const int pt = half ? mid : hi;
        const int cnt = pt >= 0 ? inertia_f(lay32, N, kf, fmaf((float)pt, dcf, c0f)) : 0;
        const int oth = __shfl_xor_sync(pair, cnt, 1);
        const int c_top = half ? oth : cnt, c_mid = half ? cnt : oth;
        if (c_top == 0) {
            out.start = npf;  // no mode below the bound: scan linearly above it
        } else {
            int chi = c_top;
            if (mid >= 0) {
                if (c_mid >= 1) {
                    hi = mid;
                    chi = c_mid;
                } else {
                    lo = mid;
                }
            }
            while (hi - lo > 1) {
                const int len = hi - lo;
                const int a = lo + (len + 1) / 3, bq = lo + (2 * len + 1) / 3;  // lo < a <= bq < hi
                const int q = half ? bq : a;
                const int c = inertia_f(lay32, N, kf, fmaf((float)q, dcf, c0f));
                const int co = __shfl_xor_sync(pair, c, 1);
                const int ca = half ? co : c, cb = half ? c : co;
                if (ca >= 1) {
                    hi = a;
                    chi = ca;
                } else if (cb >= 1) {
                    lo = a;
                    hi = bq;
                    chi = cb;
                } else {
                    lo = bq;
                }
            }
            if (hi >= 1 && (chi & 1)) n = hi;
        }
    }
    if (n < 1) return out;
    const int v = det_inertia(lay, N, k, grid_c(c0, dc, n - 1 + half));
    const int vo = __shfl_xor_sync(pair, v, 1);
    const int va = half ? vo : v;  // V[n-1]
    const int vb = half ? v : vo;  // V[n]
    int cert = (va == 0 && vb > 0 && (vb & 1)) ? n : -1;
    if (cert < 0 && va >= 0 && vb >= 0) {
        const bool up = va == 0 && vb == 0;
        const bool down = va > 0 && n >= 3;
        if (up || down) {
            const int p = (up ? n + 1 : n - 3) + half;
            const int w = p < nlim ? det_inertia(lay, N, k, grid_c(c0, dc, p)) : -1;
            const int wo = __shfl_xor_sync(pair, w, 1);
            const int c_lo = half ? wo : w, c_hi = half ? w : wo;
            if (up) {
                // count 0 at n; first nonzero at n+1, or at n+2 with n+1 inside the range
                if (c_lo > 0) {
                    if (c_lo & 1) cert = n + 1;
                } else if (c_lo == 0 && c_hi > 0 && (c_hi & 1) && n + 1 < npf) {
                    cert = n + 2;
                }
            } else {
                // count nonzero at n-1; first nonzero at n-1 or n-2
                if (c_hi == 0) {
                    if (va & 1) cert = n - 1;
                } else if (c_hi > 0 && c_lo == 0 && (c_hi & 1)) {
                    cert = n - 2;
                }
            }
        }
    }
    out.cert = cert;
    out.n = cert >= 1 ? -1 : n;
    return out;
}

}  // namespace masw
