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
// Used for the higher modes (Algorithm 1 carried past its first change) and,
// from V[0], for the first change of the counting search's fallback items
// (change above the pole-free range, a mode below V[0], double crossings),
// which an FP32 linear screen could miss when a root and a pole share a grid
// interval.
#pragma once

#include "masw_device.cuh"
#include "masw_df.cuh"

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
    return st;
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
            eval_pair(st.laydf, st.lay, st.N, st.k, st.c0, st.dc, st.top, mid > lo ? mid : -1, st.half,
                      st.pair, &st.topp, &mp);
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
        // first point of (lo, hi] with T > P.T (T(lo) = P.T, T(hi) > P.T)
        while (hi.n - lo > 1) {
            const int len = hi.n - lo;
            const int a = lo + (len + 1) / 3, bq = lo + (2 * len + 1) / 3;  // lo < a <= bq < hi
            TPoint pa, pb;
            eval_pair(st.laydf, st.lay, st.N, st.k, st.c0, st.dc, a, bq, st.half, st.pair, &pa, &pb);
            if (pa.T < st.P.T || pb.T < pa.T || pb.T > hi.T) {
                st.bad = true;
                return -1;
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

}  // namespace masw
