// The taut string of one chain (Sec. 3.2) without rescans: the funnel form
// used by the lane-group scan.
//
// With the running sum G(j) = v_r + ... + v_j of a lane (r its first
// element), the string is the shortest path through the tube between the
// lower points (j, G(j) - a_j) and the upper points (j, G(j) + a_j), ending
// at the chain end where a = 0; the prox value of element j is the slope of
// the string on [j - 1, j].  From the apex (the last point where the string
// is known to bend, or a start with multiplier 0), the funnel keeps two hull
// chains:
//   U  the greatest convex minorant of the upper points seen so far (edge
//      slopes increasing; its first edge bounds every feasible slope from
//      above: th of the local form),
//   L  the least concave majorant of the lower points (slopes decreasing; its
//      first edge is tl).
// A new knot's lower point above U's first edge (or its upper point below L's
// first edge) makes that edge final: the segment from the apex to the edge's
// end is output with the edge's slope and the apex moves there; the other
// chain then reduces to the new point (every earlier point of its side lies
// beyond the segment from the new apex to it).  Otherwise the point joins its
// chain after popping the vertices it hides.  Each point is pushed and popped
// at most once, so a chain costs O(m) however long its segments are; the
// local form (taut_string.cuh) restarts behind a bend instead, which is
// quadratic on long plateaus.
//
// Residual form.  A vertex is stored as (knot, slope of the chain edge into
// it); heights are never formed.  For each end of each chain (U's and L's
// first and last vertex) the kernel keeps C = G(i) - (that edge's line at
// i), updated per knot by C += v_i - slope, exactly like the local form's
// multipliers; a knot's upper point lies C + a_i above the line and its lower
// point C - a_i.  A pushed vertex starts at C = -+a_i (the point itself);
// moving an end to a neighbouring vertex shifts C by the slope difference
// times the distance.  In FP32 the slopes are unevaluated pairs hi + lo (a
// drifting state makes them large, and a rounded slope would tilt its line
// by eps |slope| per element of distance); FP64 keeps lo = 0.
#pragma once
#include <stdint.h>

#include "taut_string.cuh"

namespace tvcut {

template <typename T>
struct FSlope {
    T h, l;
};

template <typename T>
struct FVert;
template <>
struct __align__(16) FVert<float> {
    float h, l;
    int j, pad;
};
template <>
struct __align__(16) FVert<double> {
    double h;
    int j, pad;
};

template <typename T>
__device__ __forceinline__ FSlope<T> fv_slope(const FVert<T>& v)
{
    if constexpr (sizeof(T) == 4) return FSlope<T>{v.h, v.l};
    else return FSlope<T>{v.h, T(0)};
}

template <typename T>
__device__ __forceinline__ FVert<T> fv_make(FSlope<T> s, int j)
{
    if constexpr (sizeof(T) == 4) return FVert<T>{s.h, s.l, j, 0};
    else return FVert<T>{s.h, j, 0};
}

// a + b with the rounding error of the sum kept in lo (two-sum)
template <typename T>
__device__ __forceinline__ FSlope<T> fs_add(FSlope<T> a, T b)
{
    if constexpr (sizeof(T) == 4) {
        const T s = a.h + b;
        const T bb = s - a.h;
        return FSlope<T>{s, ((a.h - (s - bb)) + (b - bb)) + a.l};
    } else {
        return FSlope<T>{a.h + b, T(0)};
    }
}

// a - b
template <typename T>
__device__ __forceinline__ T fs_sub(FSlope<T> a, FSlope<T> b)
{
    if constexpr (sizeof(T) == 4) return (a.h - b.h) + (a.l - b.l);
    else return a.h - b.h;
}

// v - s
template <typename T>
__device__ __forceinline__ T fs_vm(T v, FSlope<T> s)
{
    if constexpr (sizeof(T) == 4) return (v - s.h) - s.l;
    else return v - s.h;
}

template <typename T>
__device__ __forceinline__ T fs_val(FSlope<T> s)
{
    return s.h + s.l;
}

template <typename T>
struct FunnelState {
    int i;             // next knot
    int pa;            // apex knot: the open segment starts at pa + 1
    int ad;            // apex kind: 0 start with multiplier 0, 1 upper point (+a_pa), 2 lower point (-a_pa)
    FSlope<T> sa;      // a line through the apex, where a chain has to restart from it,
    T ca;              //   and the running sum's residual against it
    int uh, ut, lh, lt;                  // U = ring entries [uh, ut), L = [lh, lt)
    int juf, jub, jlf, jlb;              // knots of U's and L's first and last vertex
    FSlope<T> suf, sub, slf, slb;        // their edge slopes
    T cuf, cub, clf, clb;                // residuals against their edge lines
};

// Funnel state of a segment starting at knot p with multiplier 0 (a chain
// start, or a lane's guessed piece start).
template <typename T>
__device__ __forceinline__ FunnelState<T> funnel_start(int p)
{
    FunnelState<T> f;
    f.i = p;
    f.pa = p - 1;
    f.ad = 0;
    f.sa = FSlope<T>{T(0), T(0)};
    f.ca = T(0);
    f.uh = f.ut = f.lh = f.lt = 0;
    f.juf = f.jub = f.jlf = f.jlb = p;
    f.suf = f.sub = f.slf = f.slb = FSlope<T>{T(0), T(0)};
    f.cuf = f.cub = f.clf = f.clb = T(0);
    return f;
}

// Advance the funnel through knots f.i .. stop-1 (data in shared memory,
// skewed; U and L are rings of KQ vertices, KQ a power of two).
// on_bend(s, e, d, t) receives every finished segment [s, e] with value t
// (d = 1: the string bends at the upper point e, 2: at the lower point, 0:
// chain end) and returns true to stop.  Returns 0 at stop, 1 when stopped by
// on_bend, 2 at the chain end, 3 when a chain is full: the apex (pa, ad) is
// then valid and the scan resumes in local form from pa + 1
// (funnel_to_local).
template <typename T, int KQ, class OnBend>
__device__ __forceinline__ int funnel_scan(FunnelState<T>& f, int m, int stop, const T* sv, const T* sa,
                                           FVert<T>* U, FVert<T>* L, OnBend on_bend)
{
    constexpr int M = KQ - 1;
    while (f.i < stop) {
        const int i = f.i;
        const T vi = sv[skew32(i)];
        const T Ai = (i < m - 1) ? sa[skew32(i)] : T(0);
        if (f.ut == f.uh && f.lt == f.lh) {     // first knot: the line of slope v_i through the apex
            f.sa = FSlope<T>{vi, T(0)};
            f.ca = T(0);
        }
        f.cuf += fs_vm(vi, f.suf);
        f.cub += fs_vm(vi, f.sub);
        f.clf += fs_vm(vi, f.slf);
        f.clb += fs_vm(vi, f.slb);
        // the lower point above U's first edge: the string bends at U's front
        while (f.ut != f.uh && f.cuf - Ai > T(0)) {
            const int s0 = f.pa + 1, e = f.juf;
            const FSlope<T> t = f.suf;
            f.pa = e;
            f.ad = 1;
            f.sa = f.suf;
            f.ca = f.cuf;
            ++f.uh;
            if (f.ut - f.uh == 1) {
                f.juf = f.jub;
                f.suf = f.sub;
                f.cuf = f.cub;
            } else if (f.ut != f.uh) {
                const FVert<T> nx = U[f.uh & M];
                const FSlope<T> ns = fv_slope(nx);
                f.cuf -= fs_sub(ns, f.suf) * (T)(i - f.juf);
                f.juf = nx.j;
                f.suf = ns;
            }
            f.lh = f.lt = 0;
            if (on_bend(s0, e, 1, fs_val(t))) {
                f.i = e + 1;
                return 1;
            }
        }
        // the lower point joins L (pop the vertices on or below its edge)
        {
            while (f.lt != f.lh && f.clb - Ai >= T(0)) {
                f.sa = f.slb;                    // the last vertex's edge runs through the apex
                f.ca = f.clb;
                --f.lt;
                if (f.lt - f.lh == 1) {
                    f.jlb = f.jlf;
                    f.slb = f.slf;
                    f.clb = f.clf;
                } else if (f.lt != f.lh) {
                    const FVert<T> b = L[(f.lt - 1) & M];
                    const FSlope<T> bs = fv_slope(b);
                    f.clb += fs_sub(f.slb, bs) * (T)(i - b.j);
                    f.jlb = b.j;
                    f.slb = bs;
                }
            }
            const bool empty = f.lt == f.lh;
            if (f.lt - f.lh == KQ) return 3;
            const T r = (empty ? f.ca : f.clb) - Ai;
            const FSlope<T> sn = fs_add(empty ? f.sa : f.slb, div_len<T>(r, i - (empty ? f.pa : f.jlb)));
            L[f.lt & M] = fv_make(sn, i);
            ++f.lt;
            f.jlb = i;
            f.slb = sn;
            f.clb = Ai;
            if (empty) {
                f.jlf = i;
                f.slf = sn;
                f.clf = Ai;
            }
        }
        // the upper point below L's first edge: the string bends at L's front
        while (f.lt != f.lh && f.jlf != i && f.clf + Ai < T(0)) {
            const int s0 = f.pa + 1, e = f.jlf;
            const FSlope<T> t = f.slf;
            f.pa = e;
            f.ad = 2;
            f.sa = f.slf;
            f.ca = f.clf;
            ++f.lh;
            if (f.lt - f.lh == 1) {
                f.jlf = f.jlb;
                f.slf = f.slb;
                f.clf = f.clb;
            } else if (f.lt != f.lh) {
                const FVert<T> nx = L[f.lh & M];
                const FSlope<T> ns = fv_slope(nx);
                f.clf -= fs_sub(ns, f.slf) * (T)(i - f.jlf);
                f.jlf = nx.j;
                f.slf = ns;
            }
            f.uh = f.ut = 0;
            if (on_bend(s0, e, 2, fs_val(t))) {
                f.i = e + 1;
                return 1;
            }
        }
        // the upper point joins U (pop the vertices on or above its edge)
        {
            while (f.ut != f.uh && f.cub + Ai <= T(0)) {
                f.sa = f.sub;
                f.ca = f.cub;
                --f.ut;
                if (f.ut - f.uh == 1) {
                    f.jub = f.juf;
                    f.sub = f.suf;
                    f.cub = f.cuf;
                } else if (f.ut != f.uh) {
                    const FVert<T> b = U[(f.ut - 1) & M];
                    const FSlope<T> bs = fv_slope(b);
                    f.cub += fs_sub(f.sub, bs) * (T)(i - b.j);
                    f.jub = b.j;
                    f.sub = bs;
                }
            }
            const bool empty = f.ut == f.uh;
            if (f.ut - f.uh == KQ) return 3;
            const T r = (empty ? f.ca : f.cub) + Ai;
            const FSlope<T> sn = fs_add(empty ? f.sa : f.sub, div_len<T>(r, i - (empty ? f.pa : f.jub)));
            U[f.ut & M] = fv_make(sn, i);
            ++f.ut;
            f.jub = i;
            f.sub = sn;
            f.cub = -Ai;
            if (empty) {
                f.juf = i;
                f.suf = sn;
                f.cuf = -Ai;
            }
        }
        if (i == m - 1) {   // a_{m-1} = 0: both chains end at the last point
            on_bend(f.pa + 1, m - 1, 0, fs_val(f.suf));
            f.i = m;
            return 2;
        }
        f.i = i + 1;
    }
    return 0;
}

// The local-form state that restarts the scan at the funnel's apex.
template <typename T>
__device__ __forceinline__ LaneState<T> funnel_to_local(const FunnelState<T>& f, const T* sa)
{
    const T a0 = f.ad ? sa[skew32(f.pa)] : T(0);
    const T u0 = f.ad == 1 ? a0 : f.ad == 2 ? -a0 : T(0);
    const int s = f.pa + 1;
    return LaneState<T>{s, s, s, s, u0, T(0), T(0), T(0), T(0), T(0), T(0)};
}

}  // namespace tvcut
