// masw_modes.cuh -- search for sign changes of det K on the Wittrick-Williams
// mode count (FP64 recurrence over double-float elements: mode_count_T_df),
// run by a pair of adjacent lanes.
//
// T = s + 2 J0 (mode_count_T_df: s negative eigenvalues of K, J0 clamped-layer
// modes) never decreases along the grid below the scan limit and jumps by an
// odd amount exactly where det K changes sign, by Delta s there (the change
// in the negative-eigenvalue count: +1 at a root, -1 at a pole). From a point
// P whose T and s are known, the next change is the first grid point above P
// where T grows by an odd amount: the pair finds the first point where T
// grows by splitting a bracket in three per step (one point per lane), takes
// it if the jump is odd and otherwise (a root and a pole, or two modes, inside
// one grid interval: no sign change) starts again from it. The first search
// evaluates V[top] and the bracket's midpoint; later ones reuse the smallest
// evaluated point above the last event, and start from it when its T equals
// the event's. About 2 log3(n_lim) FP64 evaluations per event.
//
// next_change runs from V[0] for the first change of the counting search's
// fallback items (change above the pole-free range, a mode below V[0], double
// crossings), which an FP32 linear screen could miss when a root and a pole
// share a grid interval. The higher modes (Algorithm 1 carried past its first
// change) take next_change_f32, which locates each rise on the FP32 count and
// certifies it on the FP64 count, with next_change as its fallback.
#pragma once

#include "masw_device.cuh"
#include "masw_df.cuh"
#include "masw_screen.cuh"

namespace masw {

struct TPoint {
    int n, T, s;
};

// Both lanes evaluate one point each (n0 on half 0, n1 on half 1; a negative
// index evaluates nothing and gives T = -1) and both get both results.
__device__ __forceinline__ void eval_pair(const float* __restrict__ laydf,
                                          const double* __restrict__ lay, int N, double k,
                                          double c0, double dc, int n0, int n1, int half,
                                          unsigned pair, TPoint* a, TPoint* b) {
    const int n = half ? n1 : n0;
    int sv = 0, T = -1;
    if (n >= 0) T = mode_count_T_df(laydf, lay, N, k, grid_c(c0, dc, n), &sv);
    const int so = __shfl_xor_sync(pair, sv, 1), To = __shfl_xor_sync(pair, T, 1);
    *a = half ? TPoint{n0, To, so} : TPoint{n0, T, sv};
    *b = half ? TPoint{n1, T, sv} : TPoint{n1, To, so};
}

// The three-point check of a linear scan's first change n (n < 1: none below
// the limit) on the mode count: T0 at V[0], Ta at V[n-1] (for n < 1 the last
// point below the limit), Tb at V[n]. T(V[n-1]) = T(V[0]) leaves no event, so
// no change, below n; an odd jump at n is a change. Two changes that a screen
// missed together (a root and a pole inside one grid interval) leave their
// mark on T even where the signs agree.
__device__ __forceinline__ bool mode_count_verified(int n, int T0, int Ta, int Tb) {
    if (T0 < 0 || Ta != T0) return false;
    return n < 1 || (Tb > Ta && ((Tb - Ta) & 1));
}

struct ModeSearch {
    const float* laydf;  // double-float records (nullptr: split on the fly)
    const double* lay;
    int N;
    double k, c0, dc;
    int top;      // last grid index below the scan limit
    int half;
    unsigned pair;
    TPoint P;     // the last event (or the start point)
    TPoint topp;  // V[top], T = -1 until evaluated
    TPoint cand;  // smallest evaluated point above P, n = -1: none
    bool bad;     // the FP64 counts failed (rescaling, or T not monotone)
    int displace; // test routing: added to each FP32-located event (0 normally)
};

__device__ __forceinline__ ModeSearch mode_search_init(const float* laydf, const double* lay,
                                                       int N, double k, double c0, double dc,
                                                       int top, int half, unsigned pair, TPoint P,
                                                       TPoint topp) {
    ModeSearch st;
    st.laydf = laydf;
    st.lay = lay;
    st.N = N;
    st.k = k;
    st.c0 = c0;
    st.dc = dc;
    st.top = top;
    st.half = half;
    st.pair = pair;
    st.P = P;
    st.topp = topp;
    st.cand = TPoint{-1, 0, 0};
    st.bad = P.T < 0 || (topp.T >= 0 && topp.T < P.T);
    st.displace = 0;
    return st;
}

// J0 at c (clamped-layer modes of the N finite layers) with the layers split
// between the pair's lanes; both lanes get the sum.
static __device__ __noinline__ int j0_pair(const double* __restrict__ lay, int N, double k,
                                           double c, int half, unsigned pair) {
    const double c2 = c * c;
    int j0 = 0;
    for (int j = half; j < N; j += 2) j0 += clamped_modes(lay + j * LAYER_STRIDE, k, c2);
    return j0 + __shfl_xor_sync(pair, j0, 1);
}

// eval_pair for two points above the last event, st.P.n < na < nb (na < 0:
// not evaluated, T = -1): s at each point on its own lane (det_inertia_df),
// J0 at V[nb] over both lanes (j0_pair). J0 never decreases along the grid,
// so J0 at V[na] equals J0 at P when J0 at V[nb] does; only otherwise is it
// counted, again over both lanes.
__device__ __forceinline__ void eval_pair_above(const ModeSearch& st, int na, int nb, TPoint* a,
                                                TPoint* b) {
    const int n = st.half ? nb : na;
    const int sv = n >= 0 ? det_inertia_df(st.laydf, st.lay, st.N, st.k, grid_c(st.c0, st.dc, n))
                          : 0;
    const int so = __shfl_xor_sync(st.pair, sv, 1);
    const int sa = st.half ? so : sv, sb = st.half ? sv : so;
    const int jp = (st.P.T - st.P.s) >> 1;
    const int jb = j0_pair(st.lay, st.N, st.k, grid_c(st.c0, st.dc, nb), st.half, st.pair);
    int ja = jp;
    if (na >= 0 && jb != jp)
        ja = j0_pair(st.lay, st.N, st.k, grid_c(st.c0, st.dc, na), st.half, st.pair);
    *a = TPoint{na, (na < 0 || sa < 0) ? -1 : sa + 2 * ja, sa};
    *b = TPoint{nb, sb < 0 ? -1 : sb + 2 * jb, sb};
}

// The first point of (lo, hi.n] with T > P.T, given T(lo) = P.T and
// hi.T > P.T: the bracket split in three per step, one point per lane. Sets
// st.cand to the smallest evaluated point above the result, st.bad when the
// counts are not monotone.
__device__ inline TPoint first_rise(ModeSearch& st, int lo, TPoint hi) {
    while (hi.n - lo > 1) {
        const int len = hi.n - lo;
        const int a = lo + (len + 1) / 3, bq = lo + (2 * len + 1) / 3;  // lo < a <= bq < hi
        TPoint pa, pb;
        if (bq > a) {
            eval_pair_above(st, a, bq, &pa, &pb);
        } else {
            eval_pair_above(st, -1, a, &pa, &pb);
            pa = pb;
        }
        if (pa.T < st.P.T || pb.T < pa.T || pb.T > hi.T) {
            st.bad = true;
            return hi;
        }
        if (pa.T > st.P.T) {
            st.cand = bq > a ? pb : hi;
            hi = pa;
        } else if (pb.T > st.P.T) {
            st.cand = hi;
            lo = a;
            hi = pb;
        } else {
            lo = bq;
        }
    }
    return hi;
}

// The next sign change above st.P: its grid index with *delta = Delta s, or -1
// when there is none up to V[top] or the counts failed (st.bad). Both lanes
// call it together and get the same result; st.P moves to the change.
__device__ inline int next_change(ModeSearch& st, int* delta) {
    while (!st.bad && st.P.n < st.top) {
        int lo = st.P.n;
        TPoint hi;
        if (st.cand.n >= 0 && st.cand.T == st.P.T) {  // no event up to cand: start there
            lo = st.cand.n;
            st.cand.n = -1;
        }
        if (st.cand.n >= 0) {
            hi = st.cand;
            st.cand = st.topp.n > hi.n && st.topp.T >= 0 ? st.topp : TPoint{-1, 0, 0};
        } else if (st.topp.T >= 0) {
            if (st.topp.T == st.P.T || lo >= st.top) return -1;  // no event below the limit
            hi = st.topp;
        } else {
            const int mid = lo + ((st.top - lo) >> 1);
            TPoint mp;
            eval_pair_above(st, mid > lo ? mid : -1, st.top, &mp, &st.topp);
            if (st.topp.T < st.P.T || (mp.n >= 0 && (mp.T < st.P.T || mp.T > st.topp.T))) {
                st.bad = true;
                return -1;
            }
            if (st.topp.T == st.P.T) return -1;
            hi = st.topp;
            if (mp.n >= 0) {
                if (mp.T > st.P.T) {
                    st.cand = st.topp;
                    hi = mp;
                } else {
                    lo = mid;
                }
            }
        }
        hi = first_rise(st, lo, hi);
        if (st.bad) return -1;
        const bool odd = (hi.T - st.P.T) & 1;
        const int ds = hi.s - st.P.s;
        st.P = hi;
        if (odd) {
            *delta = ds;
            return hi.n;
        }
    }
    return -1;
}

// ------------------------------------------------ FP32-located events
//
// The same events located on the FP32 count mode_count_T_f and certified on
// the FP64 count: from the last event P (FP64 T and s), the pair searches
// (lo, top] for the first point n whose FP32 count exceeds T(P), splitting the
// bracket in three per step, then evaluates the FP64 count at V[n-1] and V[n]
// (one point per lane). T(V[n-1]) = T(P) and T(V[n]) > T(P) place the first
// rise of T above P at n, an event when the jump is odd; otherwise the FP32
// count was off next to the rise. Located one point high or low, the pair
// takes one FP64 step of two points down or up; further off, the FP64 search
// (first_rise, next_change) takes over from the certified bracket. Per event
// about log3(n_lim) FP32 steps and one FP64 step, against 2 log3(n_lim) FP64
// evaluations per lane for next_change.

// First index in (lo, top) whose FP32 count is at least target, else top.
static __device__ __noinline__ int pair_search_T32(const float* __restrict__ lay32, int N,
                                                   float kf, float c0f, float dcf, int lo, int top,
                                                   int target, int half, unsigned pair) {
    int hi = top;
    while (hi - lo > 1) {
        const int len = hi - lo;
        const int a = lo + (len + 1) / 3, bq = lo + (2 * len + 1) / 3;  // lo < a <= bq < hi
        const int q = half ? bq : a;
        const int c = mode_count_T_f(lay32, N, kf, fmaf((float)q, dcf, c0f));
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

// next_change with events located on the FP32 count (lay32: the model's FP32
// records). Same contract: both lanes call it and get the same result.
__device__ inline int next_change_f32(ModeSearch& st, const float* __restrict__ lay32,
                                      int* delta) {
    const float kf = (float)st.k, c0f = (float)st.c0, dcf = (float)st.dc;
    int lo = st.P.n;  // T(V[lo]) = T(P)
    st.cand = TPoint{-1, 0, 0};
    while (!st.bad && lo < st.top) {
        if (st.topp.T >= 0 && st.topp.T == st.P.T) return -1;  // no event below the limit
        int n = pair_search_T32(lay32, st.N, kf, c0f, dcf, lo, st.top, st.P.T + 1, st.half,
                                st.pair);
        if (st.displace) n = min(max(n + st.displace, lo + 1), st.top);
        TPoint a, b;
        eval_pair_above(st, n - 1 > lo ? n - 1 : -1, n, &a, &b);
        if (n - 1 <= lo) a = TPoint{lo, st.P.T, st.P.s};
        if (n == st.top) st.topp = b;
        if (a.T < st.P.T || b.T < a.T || (st.topp.T >= 0 && b.T > st.topp.T)) {
            st.bad = true;
            return -1;
        }
        TPoint hi;
        if (a.T == st.P.T && b.T > st.P.T) {
            hi = b;  // certified: the first rise is at n
        } else if (b.T == st.P.T) {
            // no rise up to n: one step of two points up
            if (n >= st.top) return -1;
            TPoint u, v;
            if (n + 2 <= st.top) {
                eval_pair_above(st, n + 1, n + 2, &u, &v);
            } else {
                eval_pair_above(st, -1, n + 1, &v, &u);
                v = TPoint{-1, -1, 0};
            }
            if (u.n == st.top) st.topp = u;
            if (v.n == st.top) st.topp = v;
            if (u.T < st.P.T || (v.n >= 0 && v.T < u.T)) {
                st.bad = true;
                return -1;
            }
            if (u.T > st.P.T) {
                hi = u;
            } else if (v.n >= 0 && v.T > st.P.T) {
                hi = v;
            } else {
                lo = v.n >= 0 ? v.n : n + 1;  // FP32 off: FP64 search from the certified point
                st.cand = TPoint{lo, st.P.T, st.P.s};
                return next_change(st, delta);
            }
        } else {
            // a.T > P.T: the first rise is at or below n - 1; one step down
            TPoint u, v;
            const int n3 = n - 3 > lo ? n - 3 : -1, n2 = n - 2 > lo ? n - 2 : -1;
            if (n2 >= 0) eval_pair_above(st, n3, n2, &u, &v);
            if (n3 < 0) u = TPoint{lo, st.P.T, st.P.s};
            if (n2 < 0) v = u;
            if (u.T < st.P.T || v.T < u.T || v.T > a.T) {
                st.bad = true;
                return -1;
            }
            if (v.T == st.P.T) {
                hi = a;  // rise at n - 1
            } else if (u.T == st.P.T) {
                hi = v;  // rise at n - 2
            } else {
                st.cand = TPoint{-1, 0, 0};
                hi = first_rise(st, lo, u);  // further below: FP64 search in (lo, n - 3]
                if (st.bad) return -1;
                st.cand = TPoint{-1, 0, 0};
            }
        }
        const bool odd = (hi.T - st.P.T) & 1;
        const int ds = hi.s - st.P.s;
        st.P = hi;
        lo = hi.n;
        if (odd) {
            *delta = ds;
            return hi.n;
        }
    }
    return -1;
}

}  // namespace masw
