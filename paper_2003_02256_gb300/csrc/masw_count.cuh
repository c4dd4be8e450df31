// masw_count.cuh -- counting search with its FP64 certificate for one
// (model, wavenumber) item (plan precision 2 of the batch path and the
// serving tick).
//
//  * Search (FP32). Inside the pole-free range [0, npf) of pole_free_points_f
//    the negative-eigenvalue count of K (inertia_f) is a non-decreasing step
//    function of the grid index, 0 at c = 0 (Wittrick-Williams below the
//    lowest clamped-layer mode). One thread bisects it (count_search_single,
//    or count_search_guess from a guess interpolated between the indices of
//    neighbouring wavelengths),
//    or a pair of lanes evaluates the top of the range and its midpoint, then
//    splits the bracket in three per step, one point per lane (the fused
//    kernel and the serving tick, where the certificate's lanes follow):
//    about log2(npf), or log3(npf) steps, instead of Algorithm 1's linear
//    walk. The first nonzero point goes to the certificate whatever its FP32
//    parity.
//  * Certificate (a pair of adjacent lanes; the recurrence over
//    double-float elements, det_inertia_dd in masw_df.cuh: the Schur step in
//    double-float too, the half-space's in FP64; points above the pole-free
//    range take det_inertia_df, the FP64 step). The count is 0 at V[n-1] (so
//    0, and V[0]'s sign, at every point below) and odd at V[n] (the sign
//    differs).
//    When the FP32 count was off by one next to the change (count 0 at both
//    points: the change is higher; nonzero at V[n-1]: lower), the pair takes
//    one FP64 step of two points in that direction, inside the range. An
//    even FP64 count (two or more) after count 0 means no sign change there:
//    a second search looks for the first odd count above it, certified the
//    same way. Items left without a certificate fall back: the batch path
//    searches the FP64 mode count s + 2 J0 from V[0] (masw_modes.cuh), the
//    serving tick scans linearly from `start`.
#pragma once

#include "masw_device.cuh"
#include "masw_df.cuh"
#include "masw_screen.cuh"

namespace masw {

struct PairCount {
    int cert;   // certified first change (>= 1), or -1
    int n;      // the search's index when the certificate failed (>= 1), or -1
    int start;  // cert and n < 1: a linear scan's start (npf when the range holds no
                // change, the located point after an even FP64 count, else 0)
    int counts; // cert inside the pole-free range: the certificate's FP64 counts,
                // s(V[cert]) << 16 | s(V[cert-1]) (there J0 = 0, so T = s); else -1
};

__device__ __forceinline__ int pack_counts(int s_lo, int s_hi) {
    return (s_lo >= 0 && s_hi >= s_lo && s_hi < 32768) ? (s_hi << 16) | s_lo : -1;
}

// First grid index in (lo, top] whose FP32 negative-eigenvalue count is at
// least `target`, the count being non-decreasing there and below `target` at
// lo; -1 when the count at `top` is below `target`. The pair evaluates `top`
// and the bracket's midpoint, then splits the bracket in three per step (one
// point per lane). Both lanes return the same index.
static __device__ __noinline__ int pair_search(const float* __restrict__ lay32, int N, float kf,
                                           float c0f, float dcf, int lo, int top, int target,
                                           int half, unsigned pair) {
    int hi = top;
    const int mid = lo + ((hi - lo) >> 1);
    const int pt = half ? mid : hi;
    const int cnt = pt > lo ? inertia_f(lay32, N, kf, fmaf((float)pt, dcf, c0f)) : 0;
    const int oth = __shfl_xor_sync(pair, cnt, 1);
    const int c_top = half ? oth : cnt, c_mid = half ? cnt : oth;
    if (c_top < target) return -1;
    if (mid > lo) {
        if (c_mid >= target) hi = mid;
        else lo = mid;
    }
    while (hi - lo > 1) {
        const int len = hi - lo;
        const int a = lo + (len + 1) / 3, bq = lo + (2 * len + 1) / 3;  // lo < a <= bq < hi
        const int q = half ? bq : a;
        const int c = inertia_f(lay32, N, kf, fmaf((float)q, dcf, c0f));
        const int co = __shfl_xor_sync(pair, c, 1);
        const int ca = half ? co : c, cb = half ? c : co;
        if (ca >= target) {
            hi = a;
        } else if (cb >= target) {
            lo = a;
            hi = bq;
        } else {
            lo = bq;
        }
    }
    return hi;
}

// The search stage: the first grid point in [0, npf) with a nonzero FP32
// count (count 0 at c = 0: static stiffness positive definite), -1 when
// there is none or npf < 1. Both lanes get the same index.
__device__ __forceinline__ int count_search_pair(const float* __restrict__ lay32, int N, double k,
                                                 double c0, double dc, int npf, int half,
                                                 unsigned pair) {
    if (npf < 1) return -1;
    return pair_search(lay32, N, (float)k, (float)c0, (float)dc, -1, npf - 1, 1, half, pair);
}

// The search stage by one thread (the split search kernel): the same first
// grid point in [0, npf) with a nonzero FP32 count, or -1, by bisection. One
// point per step is one bit per evaluation, against log2(3)/2 for a pair's
// three-way split, so an item takes about 20 % fewer evaluations; the pair
// form stays where the certificate's lanes follow in the same kernel.
__device__ __forceinline__ int count_search_single(const float* __restrict__ lay32, int N,
                                                   double k, double c0, double dc, int npf) {
    if (npf < 1) return -1;
    const float kf = (float)k, c0f = (float)c0, dcf = (float)dc;
    // count 0 at lo (c = 0 when lo = -1), nonzero at hi; the top is taken as
    // nonzero and evaluated only when the bisection ends there (the change
    // lies inside the range for nearly every item: one evaluation fewer)
    int lo = -1, hi = npf - 1;
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if (inertia_f(lay32, N, kf, fmaf((float)mid, dcf, c0f)) >= 1) hi = mid;
        else lo = mid;
    }
    if (hi == npf - 1 && inertia_f(lay32, N, kf, fmaf((float)hi, dcf, c0f)) < 1) return -1;
    return hi;
}

// The guess for an item between two searched wavelengths of its model
// (indices na, nb >= 1, d items apart; the item x after the first): the line
// through them, rounded down from a quarter point below it. A fundamental
// mode's phase velocity is smooth and convex in the wavelength's place on a
// log-spaced set, so the line overestimates: on a ragged batch of 8192 models
// this guess was the change or the point below it (two evaluations) for 85 %
// of the items, the rounded line for 65 % (a parabola through a third
// neighbour, 86 %, cost more in loads and divisions than it saved).
__device__ __forceinline__ int search_guess(int na, int nb, int x, int d) {
    // (a guess: a fast division, any rounding of it gives the same result)
    return __float2int_rd(
        fmaf(__fdividef((float)(nb - na), (float)d), (float)x, (float)na - 0.25f));
}

// The search stage for an item between two searched wavelengths of its
// model, from a guess g (search_guess; g < 0: a neighbour without an index,
// and the item takes count_search_single). The count at g says on which
// side the change lies; steps of 1, 2, 4, ... from g away in that direction
// bracket it, and bisection closes the bracket: 2 evaluations when g is the
// change or the point below it, about 2 log2(e) + 2 for an error of e
// points. The result is the same first nonzero point of a non-decreasing
// count in [0, npf), or -1.
__device__ __forceinline__ int count_search_guess(const float* __restrict__ lay32, int N,
                                                  double k, double c0, double dc, int npf,
                                                  int guess) {
    if (npf < 1) return -1;
    if (guess < 0) return count_search_single(lay32, N, k, c0, dc, npf);
    const float kf = (float)k, c0f = (float)c0, dcf = (float)dc;
    const int g = min(max(guess, 0), npf - 1);
    int lo, hi;  // count 0 at lo (c = 0 when lo = -1), nonzero at hi
    if (inertia_f(lay32, N, kf, fmaf((float)g, dcf, c0f)) >= 1) {
        hi = g;
        lo = -1;
        for (int step = 1; hi > 0; step *= 2) {
            const int p = max(hi - step, 0);
            if (inertia_f(lay32, N, kf, fmaf((float)p, dcf, c0f)) < 1) {
                lo = p;
                break;
            }
            hi = p;
        }
    } else {
        lo = g;
        hi = -1;
        for (int step = 1; lo < npf - 1; step *= 2) {
            const int p = min(lo + step, npf - 1);
            if (inertia_f(lay32, N, kf, fmaf((float)p, dcf, c0f)) >= 1) {
                hi = p;
                break;
            }
            lo = p;
        }
        if (hi < 0) return -1;  // no change inside the range
    }
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if (inertia_f(lay32, N, kf, fmaf((float)mid, dcf, c0f)) >= 1) hi = mid;
        else lo = mid;
    }
    return hi;
}

// The certificate stage for the search's index n (count_search_pair or
// count_search_single) in the
// pole-free range [0, npf). Both lanes of the pair (lane bit 0 = half, `pair`
// = their shuffle mask) call it with the same item and get the same result.
// Requires nlim >= 2.
__device__ __forceinline__ PairCount certify_pair(const float* __restrict__ lay32,
                                                  const float* __restrict__ laydf,
                                                  const double* __restrict__ lay, int N, double k,
                                                  double c0, double dc, int nlim, int npf, int n,
                                                  int half, unsigned pair) {
    const float kf = (float)k;
    const float c0f = (float)c0, dcf = (float)dc;
    PairCount out{-1, -1, 0, -1};
    if (npf < 1) return out;
    // the FP64 certificate decides the parity at the first nonzero point
    if (n < 0) {
        out.start = npf;  // no mode below the bound: scan linearly above it
        return out;
    }
    if (n < 1) return out;  // a mode below V[0]: Algorithm 1 from V[0]
    const int v = det_inertia_dd(laydf, lay, N, k, grid_c(c0, dc, n - 1 + half));
    const int vo = __shfl_xor_sync(pair, v, 1);
    const int va = half ? vo : v;  // V[n-1]
    const int vb = half ? v : vo;  // V[n]
    int cert = (va == 0 && vb > 0 && (vb & 1)) ? n : -1;
    int s_lo = va, s_hi = vb;  // the FP64 counts at cert - 1 and cert
    if (cert < 0 && va >= 0 && vb >= 0) {
        const bool up = va == 0 && vb == 0;
        const bool down = va > 0 && n >= 3;
        if (up || down) {
            const int p = (up ? n + 1 : n - 3) + half;
            // inside the pole-free range the Schur step in double-float, above it in FP64
            const int w = p >= nlim ? -1
                          : p < npf ? det_inertia_dd(laydf, lay, N, k, grid_c(c0, dc, p))
                                    : det_inertia_df(laydf, lay, N, k, grid_c(c0, dc, p));
            const int wo = __shfl_xor_sync(pair, w, 1);
            const int c_lo = half ? wo : w, c_hi = half ? w : wo;
            if (up) {
                // count 0 at n; first nonzero at n+1, or at n+2 with n+1 inside the range
                if (c_lo > 0) {
                    if (c_lo & 1) {
                        cert = n + 1;
                        s_lo = vb;
                        s_hi = c_lo;
                    }
                } else if (c_lo == 0 && c_hi > 0 && (c_hi & 1) && n + 1 < npf) {
                    cert = n + 2;
                    s_lo = c_lo;
                    s_hi = c_hi;
                }
            } else {
                // count nonzero at n-1; first nonzero at n-1 or n-2
                if (c_hi == 0) {
                    if (va & 1) {
                        cert = n - 1;
                        s_lo = c_hi;
                        s_hi = va;
                    }
                } else if (c_hi > 0 && c_lo == 0 && (c_hi & 1)) {
                    cert = n - 2;
                    s_lo = c_lo;
                    s_hi = c_hi;
                }
            }
        }
    }
    if (cert < 0 && va == 0 && vb >= 2 && !(vb & 1)) {
        // FP64: count 0 below n and even at n (two modes inside one interval,
        // no sign change there). The first change is the first point above n
        // whose count is odd: search for the first count above vb and certify
        // count vb one point below it (so vb, an even count, all the way from
        // n) and an odd count at it; otherwise the item falls back with start n.
        const int m = pair_search(lay32, N, kf, c0f, dcf, n, npf - 1, vb + 1, half, pair);
        if (m > n) {
            const int u = det_inertia_dd(laydf, lay, N, k, grid_c(c0, dc, m - 1 + half));
            const int uo = __shfl_xor_sync(pair, u, 1);
            const int ua = half ? uo : u, ub = half ? u : uo;
            if (ua == vb && ub > vb && (ub & 1)) {
                cert = m;
                s_lo = ua;
                s_hi = ub;
            }
        }
        if (cert < 0) {
            out.start = n;
            return out;
        }
    }
    out.cert = cert;
    out.n = cert >= 1 ? -1 : n;
    if (cert >= 1 && cert < npf) out.counts = pack_counts(s_lo, s_hi);
    return out;
}

// Search and certificate in one call (count_search_pair, certify_pair).
// Requires nlim >= 2.
__device__ __forceinline__ PairCount count_certify_pair(const float* __restrict__ lay32,
                                                        const float* __restrict__ laydf,
                                                        const double* __restrict__ lay, int N,
                                                        double k, double c0, double dc, int nlim,
                                                        int half, unsigned pair) {
    const int npf = pole_free_points_f(lay32, N, (float)k, (float)c0, (float)dc, nlim);
    const int n = count_search_pair(lay32, N, k, c0, dc, npf, half, pair);
    return certify_pair(lay32, laydf, lay, N, k, c0, dc, nlim, npf, n, half, pair);
}

}  // namespace masw
