// The taut-string scan of one chain (Sec. 3.2), shared by every kernel that
// runs it: the per-thread chain prox of the scan launches, single grid and
// batched.
#pragma once
#include <stdint.h>

namespace tvcut {

// A lane's local-form scan state (scan_chain's variables): segment start s,
// next element i, the points ih/il that last limited th/tl, the incoming
// multiplier u0 and the weights ah/al at ih/il.
template <typename T>
struct LaneState {
    int s, i, ih, il;
    T u0, th, tl, uh, ul, ah, al;
};

// Shared-memory index of element j of a staged chain (one pad word per 32,
// so that lanes reading consecutive pieces hit different banks).
__host__ __device__ __forceinline__ int skew32(int j) { return j + (j >> 5); }

// Taut-string scan of one chain: element j of v at v[j*stride], weight of
// edge (j, j+1) at a[j*stride]; writes x[j*stride] = prox value.  From a
// segment start s with incoming multiplier u0, a common value t on s..i gives
// u_i = u0 + sum_{j=s..i} (t - v_j), which must stay in [-a_i, a_i] (and be 0
// at the chain end).  th/tl are the largest/smallest feasible t and uh/ul the
// matching u_i; when the feasible set empties, the segment ends at the point
// that last limited the violated bound (the string bends there) and the scan
// resumes after it.  Pointers advance by `stride` per element; only a rescan
// recomputes them.
// num / len for the segment updates of every scan kernel (all of them use
// this one helper, so the thread and warp scans agree bit for bit): exact
// division in FP64; in FP32 a product with one approximate reciprocal
// instruction (relative error below 2^-22).
template <typename T>
__device__ __forceinline__ T div_len(T num, int len)
{
    if constexpr (sizeof(T) == 4) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((float)len));
        return num * r;
    } else {
        return num / (T)len;
    }
}

// The step with branches: lanes that bend, clamp or start a segment take
// different paths.  Identical arithmetic to scan_chain_predicated below.
//
// SHADOW: write v_j - t (the projection of v onto the block's polytope,
// Sec. 3.1) instead of the prox value t; x must not alias v then.
template <typename T, bool SHADOW = false>
__device__ __forceinline__ void scan_chain(int m, const T* __restrict__ v, const T* __restrict__ a,
                                           T* __restrict__ x, int64_t stride)
{
    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    const T* pv = v;
    const T* pa = a;
    T* px = x;                                   // next element to write
    for (;;) {
        const T vi = *pv;
        const T Ai = (i < m - 1) ? *pa : T(0);
        bool init = (i == s);
        if (!init) {
            uh += th - vi;
            ul += tl - vi;
            const bool bhi = uh < -Ai;
            const bool blo = !bhi && ul > Ai;
            if (bhi || blo) {                        // the string bends at e
                const int e = bhi ? ih : il;
                const T t = bhi ? th : tl;
                u0 = bhi ? ah : -al;
                for (int j = s; j <= e; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - t : t;
                s = e + 1;
                if (s < i) {                         // rescan from the bend
                    i = s;
                    pv = v + (int64_t)s * stride;
                    pa = a + (int64_t)s * stride;
                    continue;
                }
                init = true;                         // the new segment starts at i
            } else {
                const int len = i - s + 1;
                if (uh > Ai) {
                    th -= div_len<T>(uh - Ai, len);
                    uh = Ai;
                    ih = i;
                    ah = Ai;
                }
                if (ul < -Ai) {
                    tl += div_len<T>(-Ai - ul, len);
                    ul = -Ai;
                    il = i;
                    al = Ai;
                }
            }
        }
        if (init) {
            th = vi + Ai - u0;
            tl = vi - Ai - u0;
            uh = Ai;
            ul = -Ai;
            ih = il = i;
            ah = al = Ai;
        }
        if (i == m - 1) {
            for (int j = s; j <= m - 1; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - th : th;
            break;
        }
        ++i;
        pv += stride;
        pa += stride;
    }
}

// scan_chain on padded weights: a holds one value per element, 0 at the
// chain's last one (the state's own layout), so element i+1's value and
// weight are loaded one step ahead with no bounds test on the weight.  The
// loads of a step then overlap the arithmetic of the previous one; the
// arithmetic and the order of the writes are those of scan_chain.
template <typename T, bool SHADOW = false>
__device__ __forceinline__ void scan_chain_padded(int m, const T* __restrict__ v, const T* __restrict__ a,
                                                  T* __restrict__ x, int64_t stride)
{
    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    const T* pv = v;
    const T* pa = a;
    T* px = x;                                   // next element to write
    T cv = v[0], ca = a[0];                      // element i
    for (;;) {
        const T vi = cv;
        const T Ai = ca;
        T nv = T(0), na = T(0);                  // element i + 1
        if (i + 1 < m) {
            nv = pv[stride];
            na = pa[stride];
        }
        bool init = (i == s);
        if (!init) {
            uh += th - vi;
            ul += tl - vi;
            const bool bhi = uh < -Ai;
            const bool blo = !bhi && ul > Ai;
            if (bhi || blo) {
                const int e = bhi ? ih : il;
                const T t = bhi ? th : tl;
                u0 = bhi ? ah : -al;
                for (int j = s; j <= e; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - t : t;
                s = e + 1;
                if (s < i) {
                    i = s;
                    pv = v + (int64_t)s * stride;
                    pa = a + (int64_t)s * stride;
                    cv = *pv;
                    ca = *pa;
                    continue;
                }
                init = true;
            } else {
                const int len = i - s + 1;
                if (uh > Ai) {
                    th -= div_len<T>(uh - Ai, len);
                    uh = Ai;
                    ih = i;
                    ah = Ai;
                }
                if (ul < -Ai) {
                    tl += div_len<T>(-Ai - ul, len);
                    ul = -Ai;
                    il = i;
                    al = Ai;
                }
            }
        }
        if (init) {
            th = vi + Ai - u0;
            tl = vi - Ai - u0;
            uh = Ai;
            ul = -Ai;
            ih = il = i;
            ah = al = Ai;
        }
        if (i == m - 1) {
            for (int j = s; j <= m - 1; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - th : th;
            break;
        }
        ++i;
        pv += stride;
        pa += stride;
        cv = nv;
        ca = na;
    }
}

// The per-element step is written without branches except two rare ones
// (writing a finished segment and restarting behind the current element), so
// that the lanes of a warp, which bend, clamp and restart at different
// elements, stay on one instruction stream: every candidate update is
// computed and the valid one selected.
template <typename T, bool SHADOW = false>
__device__ __forceinline__ void scan_chain_predicated(int m, const T* __restrict__ v, const T* __restrict__ a,
                                           T* __restrict__ x, int64_t stride)
{
    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    const T* pv = v;
    const T* pa = a;
    T* px = x;                                   // next element to write
    for (;;) {
        const T vi = *pv;
        const T Ai = (i < m - 1) ? *pa : T(0);
        const bool fresh = (i == s);             // first element of a segment
        const T uhn = uh + (th - vi);
        const T uln = ul + (tl - vi);
        const bool bhi = !fresh && uhn < -Ai;    // the string bends up at ih
        const bool blo = !fresh && !bhi && uln > Ai;
        const bool bend = bhi || blo;
        if (bend) {
            const int e = bhi ? ih : il;
            const T t = bhi ? th : tl;
            u0 = bhi ? ah : -al;
            for (int j = s; j <= e; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - t : t;
            s = e + 1;
            if (s < i) {                         // rescan from the bend
                i = s;
                pv = v + (int64_t)s * stride;
                pa = a + (int64_t)s * stride;
                continue;
            }
        }
        const bool start = fresh || bend;        // a segment starts at i
        const int len = i - s + 1;
        const bool ch = !start && uhn > Ai;      // the upper slope is cut at i
        const bool cl = !start && uln < -Ai;     // the lower slope is cut at i
        const T thc = ch ? th - div_len<T>(uhn - Ai, len) : th;
        const T tlc = cl ? tl + div_len<T>(-Ai - uln, len) : tl;
        th = start ? vi + Ai - u0 : thc;
        tl = start ? vi - Ai - u0 : tlc;
        uh = (start || ch) ? Ai : uhn;
        ul = (start || cl) ? -Ai : uln;
        ih = (start || ch) ? i : ih;
        il = (start || cl) ? i : il;
        ah = (start || ch) ? Ai : ah;
        al = (start || cl) ? Ai : al;
        if (i == m - 1) {
            for (int j = s; j <= m - 1; ++j, px += stride) *px = SHADOW ? v[(int64_t)j * stride] - th : th;
            break;
        }
        ++i;
        pv += stride;
        pa += stride;
    }
}

}  // namespace tvcut
