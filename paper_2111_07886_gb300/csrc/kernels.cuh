// Device helpers shared by the projector and update kernels: plane-group loads, packed
// FP32x2 arithmetic (sm_100+ f32x2 instructions), compensated sums, the pixel-driven
// backprojection gather, and the deterministic last-block FP64 reduction.
#pragma once

#include <type_traits>

#include "pet_common.cuh"

namespace pet {

constexpr float kQ32 = 2.3283064365386963e-10f;   // 2^-32
constexpr double kQ32d = 2.3283064365386963e-10;

template <int AR> struct ArithT { using T = float; };
template <> struct ArithT<AR_FP64> { using T = double; };

// ------------------------------------------------------------------------------------------
// Loads of G consecutive planes (G * sizeof(T) bytes, aligned) through the read-only path.
// ------------------------------------------------------------------------------------------
template <int G, typename T>
__device__ __forceinline__ void load_group(const T *__restrict__ p, T (&v)[G])
{
    if constexpr (G == 1) {
        v[0] = __ldg(p);
    } else if constexpr (G == 8 && sizeof(T) == 4) {
        // one 256-bit load per plane group (sm_100+; the group is 32-byte aligned)
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                       "=f"(v[6]), "=f"(v[7])
                     : "l"(p));
    } else if constexpr (G == 8 && sizeof(T) == 8) {
        asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
                     : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
        asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
                     : "=d"(v[4]), "=d"(v[5]), "=d"(v[6]), "=d"(v[7]) : "l"(p + 4));
    } else if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < G / 4; ++q) {
            float4 x = __ldg(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < G / 2; ++q) {
            double2 x = __ldg(reinterpret_cast<const double2 *>(p) + q);
            v[2 * q] = x.x; v[2 * q + 1] = x.y;
        }
    }
}

template <int G>
__device__ __forceinline__ void load_group_i(const int *__restrict__ p, int (&v)[G])
{
    if constexpr (G == 1) {
        v[0] = __ldg(p);
    } else if constexpr (G == 8) {
        asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7])
                     : "l"(p));
    } else {
#pragma unroll
        for (int q = 0; q < G / 4; ++q) {
            int4 x = __ldg(reinterpret_cast<const int4 *>(p) + q);
            v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
    }
}

template <int G, typename T>
__device__ __forceinline__ void store_group(T *__restrict__ p, const T (&v)[G])
{
    if constexpr (G == 1) {
        p[0] = v[0];
    } else if constexpr (G == 8 && sizeof(T) == 4) {
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                     :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]),
                        "f"(v[6]), "f"(v[7])
                     : "memory");
    } else if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < G / 4; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                           v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < G / 2; ++q)
            reinterpret_cast<double2 *>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
    }
}

// ------------------------------------------------------------------------------------------
// Packed FP32x2 arithmetic: one instruction updates two planes (round-to-nearest, IEEE).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// ------------------------------------------------------------------------------------------
// Two FP32 planes in one 64-bit register pair (low word = even plane): the operands of the
// f32x2 instructions stay paired, with no repacking between instructions.
// ------------------------------------------------------------------------------------------
typedef unsigned long long f2x;

__device__ __forceinline__ f2x vpk(float lo, float hi)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2x vsplat(float v) { return vpk(v, v); }
__device__ __forceinline__ void vunpk(f2x v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x vfma(f2x a, f2x b, f2x c)
{
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2x vadd(f2x a, f2x b)
{
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x vsub(f2x a, f2x b)
{
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x vmul(f2x a, f2x b)
{
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x vabs(f2x a)       // clears both sign bits
{
    f2x r;
    asm("and.b64 %0, %1, 0x7FFFFFFF7FFFFFFF;" : "=l"(r) : "l"(a));
    return r;
}
// Hardware approximate reciprocal and 1/sqrt per lane; subnormal inputs are flushed to zero
// (1/0 = inf), so callers keep their arguments normal or test for it.
__device__ __forceinline__ f2x vrcp(f2x a)
{
    float x, y;
    vunpk(a, x, y);
    asm("rcp.approx.ftz.f32 %0, %0;" : "+f"(x));
    asm("rcp.approx.ftz.f32 %0, %0;" : "+f"(y));
    return vpk(x, y);
}
__device__ __forceinline__ f2x vrsqrt(f2x a)
{
    float x, y;
    vunpk(a, x, y);
    asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x));
    asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(y));
    return vpk(x, y);
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start before the previous kernel of its stream has finished; grid_dependency_wait() blocks
// until that kernel has completed and its memory operations are visible (a no-op for a kernel
// launched without the attribute).  grid_dependents_launch() lets such a dependent kernel be
// scheduled before this one completes.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only), its commit and the
// wait for all of this thread's copies
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// one 8-plane FP32 group (32-byte aligned) as four pairs, through the read-only path
__device__ __forceinline__ void load8x(const float *__restrict__ p, f2x (&v)[4])
{
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
        : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
}
// as load8x when `on`, else four zero pairs (no memory access)
__device__ __forceinline__ void load8x_if(const float *__restrict__ p, bool on, f2x (&v)[4])
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
        "mov.b64 %0, 0;\n\tmov.b64 %1, 0;\n\tmov.b64 %2, 0;\n\tmov.b64 %3, 0;\n\t"
        "@q ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];\n\t}"
        : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p), "r"((unsigned)on));
}
__device__ __forceinline__ void store8x(float *__restrict__ p, const f2x (&v)[4])
{
    asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "l"(v[0]), "l"(v[1]), "l"(v[2]), "l"(v[3]) : "memory");
}

// ------------------------------------------------------------------------------------------
// Sums of G planes.  Each step adds the two-term contribution w0 x0 + w1 x1 of one driving
// step (forward) or one view (backward).
//   AR_FP32 : s += w0 x0 + w1 x1 with FMAs
//   AR_KAHAN: compensated: y = w0 x0 + w1 x1 + e; t = s + y; e = y - (t - s); s = t
//   AR_FP64 : double FMAs
// The final value is s + e.
// ------------------------------------------------------------------------------------------
template <int G, int AR> struct GroupSum {
    using T = typename ArithT<AR>::T;
    static constexpr bool PACK = (AR != AR_FP64) && (G % 2 == 0);
    static constexpr int NS = PACK ? G / 2 : G;
    // packed: s2[q] holds planes (2q, 2q+1), so every f32x2 operand is an aligned register pair
    typename std::conditional<PACK, float2, T>::type s2[NS], e2[NS];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if constexpr (PACK) { s2[q] = make_float2(0.f, 0.f); e2[q] = make_float2(0.f, 0.f); }
            else { s2[q] = T(0); e2[q] = T(0); }
        }
    }

    __device__ __forceinline__ T s_at(int p) const
    {
        if constexpr (PACK) return (p & 1) ? s2[p >> 1].y : s2[p >> 1].x;
        else return s2[p];
    }
    __device__ __forceinline__ T e_at(int p) const
    {
        if constexpr (PACK) return (p & 1) ? e2[p >> 1].y : e2[p >> 1].x;
        else return e2[p];
    }

    // y_p = w0 x0_p + w1 x1_p (+ e_p for Kahan), then accumulate
    __device__ __forceinline__ void add2terms(T w0, const T (&x0)[G], T w1, const T (&x1)[G])
    {
        if constexpr (PACK) {
            const float2 W0 = make_float2(w0, w0), W1 = make_float2(w1, w1);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const float2 X0 = make_float2(x0[2 * q], x0[2 * q + 1]);
                const float2 X1 = make_float2(x1[2 * q], x1[2 * q + 1]);
                if constexpr (AR == AR_KAHAN) {
                    float2 y = fma2(W0, X0, e2[q]);
                    y = fma2(W1, X1, y);
                    const float2 t = add2(s2[q], y);
                    e2[q] = sub2(y, sub2(t, s2[q]));
                    s2[q] = t;
                } else {
                    s2[q] = fma2(W1, X1, fma2(W0, X0, s2[q]));
                }
            }
        } else if constexpr (AR == AR_KAHAN) {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                float y = fmaf(w0, x0[p], e2[p]);
                y = fmaf(w1, x1[p], y);
                const float t = s2[p] + y;
                e2[p] = y - (t - s2[p]);
                s2[p] = t;
            }
        } else {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                s2[p] = fma(w0, x0[p], s2[p]);
                s2[p] = fma(w1, x1[p], s2[p]);
            }
        }
    }

    // scalar-weight-only form (sensitivity: x == 1)
    __device__ __forceinline__ void add_scalar(T y0)
    {
        T x0[G], x1[G];
#pragma unroll
        for (int p = 0; p < G; ++p) { x0[p] = T(1); x1[p] = T(0); }
        add2terms(y0, x0, T(0), x1);
    }

    __device__ __forceinline__ T value(int p) const { return s_at(p) + e_at(p); }

    // overwrite plane p's sum and compensation
    __device__ __forceinline__ void set(int p, T s, T e)
    {
        if constexpr (PACK) {
            if (p & 1) { s2[p >> 1].y = s; e2[p >> 1].y = e; }
            else { s2[p >> 1].x = s; e2[p >> 1].x = e; }
        } else {
            s2[p] = s;
            e2[p] = e;
        }
    }
};

// ------------------------------------------------------------------------------------------
// Pixel-driven gather backprojection, in two phases per block.
//
// Phase 1 (bp_weights): for every (pixel, view) pair of the block, the first candidate bin b0
// and the exact lengths w[k] of the lines of bins b0 + k (k < KC) inside the pixel square go to a
// shared-memory table.  Oblique views: the trapezoid min(L, (h - |delta|) rho / (major minor))
// of the pixel's footprint, delta = b - t(ix, iy) in bins, from Q32.32 integers so that the
// feet of the trapezoid keep relative precision.  Views along an axis: length L for each ray
// inside the pixel's half-open column, membership decided from the very start coordinate the
// forward walk uses, so ties on pixel edges match the forward projector exactly.
// Phase 2 (bp_accumulate): every plane group of the pixel adds, view by view in order, the
// <= KC-term partial with one compensated step (fixed order: deterministic, no atomics).
// ------------------------------------------------------------------------------------------
template <int KC, int AR> struct BpEntry {
    using T = typename ArithT<AR>::T;
    unsigned off;      // element offset of the group row (u NB + b0) Pp, b0 clamped to [0, NB - KC]
    T w[KC];           // lengths for bins b0 .. b0 + KC - 1 (zero outside the footprint)
};

template <int KC, int AR, int CAPX = 0> struct BpTable {
    static constexpr int CAP = CAPX > 0 ? CAPX : (AR == AR_FP64 ? 1024 : 2048) / (KC > 2 ? 2 : 1);
    // one entry per (pixel, view): read with one or two wide shared-memory loads
    struct __align__(16) E : BpEntry<KC, AR> {};
    E e[CAP];
};

// Sub-ray model (g.R > 1): the weight of bin b is the sum over its R lines, at offsets
// (2 s + 1 - R) / (2 R) bins from its centre, of the single-line length (the trapezoid of oblique
// views; for views along an axis, L for each line whose forward-walk start coordinate lies in the
// pixel's column, the forward projector's own membership test); scale carries the 1 / R.  The
// first candidate is floor(t - h - (R - 1) / (2 R)).
// Ring-sampled bins (g.ring): bin b's R lines lie at c0_b + s ds_b (pixel units, from the bin
// table); the weight of bin b is the sum of their lengths in the pixel: the trapezoid
// min(L, (hp - |r - p|) / (major minor)) of the pixel's footprint, p the pixel centre's offset
// along the view's normal, hp its half-width; views along an axis use the forward walk's start
// coordinates as for uniform sub-rays.  Candidates start one bin before the bin coordinate
// asin((p - hp) / Rd) / dbeta + (NB - 1) / 2 of the footprint's low edge, rounded to the bin
// whose width contains it (K covers the footprint over the narrowest bins).
template <int KC, int AR>
__device__ __forceinline__ void bp_weights_ring(const GeoDev &g, const ViewGeo &vw, int slot, int ix,
                                                int iy, int &b0, typename ArithT<AR>::T (&w)[KC])
{
    using T = typename ArithT<AR>::T;
    const int NB = g.NB, R = g.R;
#pragma unroll
    for (int k = 0; k < KC; ++k) w[k] = T(0);
    if constexpr (AR == AR_FP64) {
        const double p = vw.pn0 + (double)ix * vw.pnx + (double)iy * vw.pny;
        const double x = fmin(1.0, fmax(-1.0, (p - vw.hp) / g.ring_r));
        b0 = (int)floor(asin(x) / g.ring_db + 0.5 * NB) - 1;
    } else {
        const float p = (float)vw.pn0 + (float)ix * (float)vw.pnx + (float)iy * (float)vw.pny;
        const float x = fminf(1.f, fmaxf(-1.f, (p - (float)vw.hp) / g.ring_rf));
        b0 = (int)floorf(asinf(x) / g.ring_dbf + 0.5f * NB) - 1;
    }
    const BinGeo *bg = g.bins;
    if (vw.axis) {
        const int cross = vw.xdrive ? iy : ix;
        const RayGeo *rr = g.rays + (size_t)slot * NB;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            int cnt = 0;
            for (int sr = 0; sr < R; ++sr) {
                if constexpr (AR == AR_FP64) cnt += (int)floor(rr[b].lo + (2 * sr + 1 - R) * rr[b].sh) == cross;
                else cnt += (int)((rr[b].loq + (long long)(2 * sr + 1 - R) * rr[b].shq) >> 32) == cross;
            }
            w[k] = (T)cnt * (T)vw.L;
        }
        return;
    }
    if constexpr (AR == AR_FP64) {
        const double p = vw.pn0 + (double)ix * vw.pnx + (double)iy * vw.pny;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            double ww = 0.0;
            for (int sr = 0; sr < R; ++sr) {
                const double dd = vw.hp - fabs(bg[b].c0 + sr * bg[b].ds - p);
                ww += dd > 0.0 ? fmin(vw.L, dd * vw.islope) : 0.0;
            }
            w[k] = ww;
        }
    } else {
        const long long pq = vw.pn0q + (long long)ix * vw.pnxq + (long long)iy * vw.pnyq;
        const float ws = vw.islopef * (kQ32 * 256.f);
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            float ww = 0.f;
            for (int sr = 0; sr < R; ++sr) {
                const long long dq = bg[b].c0q + (long long)sr * bg[b].dsq - pq;
                const long long dd = vw.hpq - (dq < 0 ? -dq : dq);
                ww += dd > 0 ? fminf(vw.Lf, __int2float_rn((int)(dd >> 8)) * ws) : 0.f;
            }
            w[k] = ww;
        }
    }
}

template <int KC, int AR>
__device__ __forceinline__ void bp_weights_sub(const GeoDev &g, const ViewGeo &vw, int slot, int ix,
                                            int iy, int &b0, typename ArithT<AR>::T (&w)[KC])
{
    using T = typename ArithT<AR>::T;
    if (g.ring) {
        bp_weights_ring<KC, AR>(g, vw, slot, ix, iy, b0, w);
        return;
    }
    const int NB = g.NB, R = g.R;
#pragma unroll
    for (int k = 0; k < KC; ++k) w[k] = T(0);
    if constexpr (AR == AR_FP64) {
        const double t = vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy;
        b0 = (int)floor(t - vw.h - (0.5 - 0.5 / R));
    } else {
        const long long tq = vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq;
        b0 = (int)((tq - vw.hq - (long long)(R - 1) * g.offq) >> 32);
    }
    if (vw.axis) {
        const int cross = vw.xdrive ? iy : ix;
        const RayGeo *rr = g.rays + (size_t)slot * NB;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            int cnt = 0;
            for (int sr = 0; sr < R; ++sr) {
                if constexpr (AR == AR_FP64) cnt += (int)floor(rr[b].lo + (2 * sr + 1 - R) * vw.half) == cross;
                else cnt += (int)((rr[b].loq + (long long)(2 * sr + 1 - R) * vw.halfq) >> 32) == cross;
            }
            w[k] = (T)cnt * (T)vw.L;
        }
        return;
    }
    if constexpr (AR == AR_FP64) {
        const double t = vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            double ww = 0.0;
            for (int sr = 0; sr < R; ++sr) {
                const double dd = vw.h - fabs((double)b + (2 * sr + 1 - R) * (0.5 / R) - t);
                ww += dd > 0.0 ? fmin(vw.L, dd * vw.wslope) : 0.0;
            }
            w[k] = ww;
        }
    } else {
        const long long tq = vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq;
        const float ws = vw.wslopef * (kQ32 * 256.f);
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            if ((unsigned)b >= (unsigned)NB) continue;
            float ww = 0.f;
            for (int sr = 0; sr < R; ++sr) {
                const long long dq = ((long long)b << 32) + (long long)(2 * sr + 1 - R) * g.offq - tq;
                const long long dd = vw.hq - (dq < 0 ? -dq : dq);
                ww += dd > 0 ? fminf(vw.Lf, __int2float_rn((int)(dd >> 8)) * ws) : 0.f;
            }
            w[k] = ww;
        }
    }
}

// SUB: the kernel instantiation that serves sub-ray geometries (g.R > 1); the others never
// contain the sub-ray code
template <int KC, int AR, bool SUB = false>
__device__ __forceinline__ void bp_weights(const GeoDev &g, const ViewGeo &vw, int slot, int ix,
                                           int iy, int &b0, typename ArithT<AR>::T (&w)[KC])
{
    using T = typename ArithT<AR>::T;
    const int NB = g.NB;
    if constexpr (SUB) {
        bp_weights_sub<KC, AR>(g, vw, slot, ix, iy, b0, w);
        return;
    }
    if (vw.axis) {
        const int cross = vw.xdrive ? iy : ix;
        const RayGeo *rr = g.rays + (size_t)slot * NB;
        int bs;
        if constexpr (AR == AR_FP64)
            bs = (int)floor(vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy - vw.h);
        else
            bs = (int)((vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq - vw.hq) >> 32);
        auto member = [&](int b) -> bool {
            if ((unsigned)b >= (unsigned)NB) return false;
            if constexpr (AR == AR_FP64) return (int)floor(rr[b].lo) == cross;
            else return (int)(rr[b].loq >> 32) == cross;
        };
        b0 = member(bs) ? bs : bs + 1;
#pragma unroll
        for (int k = 0; k < KC; ++k) w[k] = member(b0 + k) ? (T)vw.L : T(0);
        return;
    }
    if constexpr (AR == AR_FP64) {
        const double t = vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy;
        b0 = (int)ceil(t - vw.h);
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            const double dd = vw.h - fabs((double)b - t);
            const double ww = dd > 0.0 ? fmin(vw.L, dd * vw.wslope) : 0.0;
            w[k] = (unsigned)b < (unsigned)NB ? ww : 0.0;
        }
    } else {
        const long long tq = vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq;
        b0 = (int)((tq - vw.hq + 0xFFFFFFFFLL) >> 32);          // ceil(t - h)
        // dd in (0, h 2^32] fits 32 bits after dropping its 8 lowest bits (2^-24 bin): a 32-bit
        // integer conversion instead of a 64-bit one, which runs on the (narrow) FP64 pipe
        const float ws = vw.wslopef * (kQ32 * 256.f);
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int b = b0 + k;
            const long long dq = ((long long)b << 32) - tq;
            const long long dd = vw.hq - (dq < 0 ? -dq : dq);
            const float ww = dd > 0 ? fminf(vw.Lf, __int2float_rn((int)(dd >> 8)) * ws) : 0.f;
            w[k] = (unsigned)b < (unsigned)NB ? ww : 0.f;
        }
    }
}

// One table entry: pixel (ix, iy) (inside the image when `in`) against view u of the subset.
template <int KC, int AR, int CAPX, bool SUB = false>
__device__ __forceinline__ typename BpTable<KC, AR, CAPX>::E bp_entry(const GeoDev &g, int slot0, int u,
                                                                    bool in, int ix, int iy)
{
    using T = typename ArithT<AR>::T;
    int b0 = 0;
    T w[KC];
    if (in) {
        bp_weights<KC, AR, SUB>(g, g.views[slot0 + u], slot0 + u, ix, iy, b0, w);
    } else {
#pragma unroll
        for (int k = 0; k < KC; ++k) w[k] = T(0);
    }
    // Clamp the first bin into [0, NB - KC] and shift the lengths with it, so that all KC
    // rows of the entry exist (bins outside [0, NB) already carry zero length).
    const int bc = min(max(b0, 0), g.NB - KC);
    typename BpTable<KC, AR, CAPX>::E ent;
    ent.off = ((unsigned)u * (unsigned)g.NB + (unsigned)bc) * (unsigned)g.Pp;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int src = k + bc - b0;
        T v = T(0);
#pragma unroll
        for (int m = 0; m < KC; ++m) v = (m == src) ? w[m] : v;
        ent.w[k] = v;
    }
    return ent;
}

// Fill the table for pixels [j0, j0 + np) x views [u0, u0 + nvc), view-major: the entry of local
// pixel pl and view u0 + uu is tb.e[uu * np + pl], so that threads of consecutive pixels touch
// consecutive entries.  With one pixel per thread (single-plane images) each thread computes its
// pixel's coordinates once and walks the views.
template <int KC, int AR, int CAPX, bool SUB = false>
__device__ __forceinline__ void bp_fill(const GeoDev &g, int slot0, int u0, int nvc, int j0,
                                        int np, BpTable<KC, AR, CAPX> &tb)
{
    const int nthr = blockDim.x, npix = g.N * g.N;
    if (np == nthr) {
        const int pl = threadIdx.x, j = j0 + pl;
        const bool in = j < npix;
        const int ix = in ? j % g.N : 0, iy = in ? j / g.N : 0;
        for (int uu = 0; uu < nvc; ++uu)
            tb.e[uu * np + pl] = bp_entry<KC, AR, CAPX, SUB>(g, slot0, u0 + uu, in, ix, iy);
        return;
    }
    for (int e = threadIdx.x; e < np * nvc; e += nthr) {
        const int uu = e / np, pl = e - uu * np;
        const int j = j0 + pl;
        const bool in = j < npix;
        tb.e[e] = bp_entry<KC, AR, CAPX, SUB>(g, slot0, u0 + uu, in, in ? j % g.N : 0, in ? j / g.N : 0);
    }
}

// Accumulate the nvc views of the table (np pixels) into acc for local pixel pl and plane group grp.
// proj (subset rows [u][NB][Pp]) == nullptr backprojects ones.
template <int G, int KC, int AR, int CAPX>
__device__ __forceinline__ void bp_accumulate(const GeoDev &g, const BpTable<KC, AR, CAPX> &tb,
                                              const typename ArithT<AR>::T *__restrict__ proj,
                                              int np, int nvc, int pl, int grp,
                                              GroupSum<G, AR> &acc)
{
    using T = typename ArithT<AR>::T;
    const unsigned Pp = (unsigned)g.Pp;
    const T *base = proj + grp * G;
    for (int uu = 0; uu < nvc; ++uu) {
        const typename BpTable<KC, AR, CAPX>::E ent = tb.e[uu * np + pl];
        if (proj == nullptr) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < KC; ++k) s += ent.w[k];
            acc.add_scalar(s);
            continue;
        }
        // 32-bit element offsets (sinograms hold < 2^32 elements)
        const T *row = base + ent.off;
#pragma unroll
        for (int k = 0; k < KC; k += 2) {
            T x0[G], x1[G];
            load_group<G, T>(row + k * Pp, x0);
            load_group<G, T>(row + (k + 1) * Pp, x1);
            acc.add2terms(ent.w[k], x0, ent.w[k + 1], x1);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Time of flight.  TOF bin t of a line spans [e_t, e_t+1) along it, e_t = (t - T/2) d, and
// h_t(tau) = Phi((e_t+1 - tau) / sigma) - Phi((e_t - tau) / sigma) is the Gaussian timing kernel
// at position tau integrated over the bin.  With z = (e - tau) / (sigma sqrt 2) at the two edges
// (z0 < z1), h = (erfc(-z1) - erfc(-z0)) / 2, taken from the tail masses in the form that has
// no cancellation.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T tof_h(T z0, T z1)
{
    if constexpr (sizeof(T) == 8) {
        if (z0 >= 0.0) return 0.5 * (erfc(z0) - erfc(z1));
        if (z1 <= 0.0) return 0.5 * (erfc(-z1) - erfc(-z0));
        return 1.0 - 0.5 * (erfc(-z0) + erfc(z1));
    } else {
        if (z0 >= 0.f) return 0.5f * (erfcf(z0) - erfcf(z1));
        if (z1 <= 0.f) return 0.5f * (erfcf(-z1) - erfcf(-z0));
        return 1.f - 0.5f * (erfcf(-z0) + erfcf(z1));
    }
}

// h_t(tau) for one TOF bin (tau in pixel units)
template <typename T>
__device__ __forceinline__ T tof_weight(const GeoDev &g, int t, T tau)
{
    const T d = sizeof(T) == 8 ? (T)g.tof_d : (T)g.tof_df, k = sizeof(T) == 8 ? (T)g.tof_k : (T)g.tof_kf;
    const T e0 = (T)(2 * t - g.T) * T(0.5) * d;
    return tof_h<T>((e0 - tau) * k, (e0 + d - tau) * k);
}

// TOF form of bp_accumulate: rows [u][NB][T][Pp]; for each view the pixel's centre position
// tau along the view's lines picks the TOF bins within the kernel's window, each weighted by
// h_t(tau) (its bin edges evaluated once and shared by neighbouring bins).  ix, iy: the pixel;
// slot0 + u0: the table's first view.
template <int G, int KC, int AR, int CAPX>
__device__ __forceinline__ void bp_accumulate_tof(const GeoDev &g, const BpTable<KC, AR, CAPX> &tb,
                                                  const typename ArithT<AR>::T *__restrict__ proj,
                                                  int np, int nvc, int pl, int grp,
                                                  GroupSum<G, AR> &acc, int ix, int iy, int slot0,
                                                  int u0)
{
    using T = typename ArithT<AR>::T;
    constexpr bool D = AR == AR_FP64;
    const unsigned Pp = (unsigned)g.Pp, TT = (unsigned)g.T;
    const T d = D ? (T)g.tof_d : (T)g.tof_df, kk = D ? (T)g.tof_k : (T)g.tof_kf;
    const T W = D ? (T)g.tof_w : (T)g.tof_wf;
    const T *base = proj + grp * G;
    for (int uu = 0; uu < nvc; ++uu) {
        const typename BpTable<KC, AR, CAPX>::E ent = tb.e[uu * np + pl];
        const ViewGeo &vw = g.views[slot0 + u0 + uu];
        const T tau = D ? (T)(vw.tau0 + ix * vw.taux + iy * vw.tauy)
                        : (T)vw.tau0f + (T)ix * (T)vw.tauxf + (T)iy * (T)vw.tauyf;
        // bins whose centre (t - (T-1)/2) d lies within W of tau
        const T tc = tau / d + T(0.5) * (T)(g.T - 1);
        const int t_lo = max(0, (int)ceil(tc - W / d));
        const int t_hi = min(g.T - 1, (int)floor(tc + W / d));
        T z0 = ((T)(2 * t_lo - g.T) * T(0.5) * d - tau) * kk;
        for (int t = t_lo; t <= t_hi; ++t) {
            const T z1 = ((T)(2 * t + 2 - g.T) * T(0.5) * d - tau) * kk;
            const T h = tof_h<T>(z0, z1);
            z0 = z1;
            if (proj == nullptr) {
                T sw = T(0);
#pragma unroll
                for (int k = 0; k < KC; ++k) sw += ent.w[k];
                acc.add_scalar(h * sw);
                continue;
            }
            const T *row = base + ent.off * TT + (unsigned)t * Pp;
#pragma unroll
            for (int k = 0; k < KC; k += 2) {
                T x0[G], x1[G];
                load_group<G, T>(row + (unsigned)k * TT * Pp, x0);
                load_group<G, T>(row + (unsigned)(k + 1) * TT * Pp, x1);
                acc.add2terms(h * ent.w[k], x0, h * ent.w[k + 1], x1);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Deterministic FP64 reduction of NV values over the whole grid: each block writes its
// partial, the last block to finish (atomic ticket) adds the partials in block order and
// writes result[0..NV).  No waits.  blockDim.x must be a multiple of 32, <= 1024.
// ------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[32])
{
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, wid = t >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < nw ? sh[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[k] = x;
        }
    }
}

// Reduction over the nblocks virtual blocks of one scan; bid is this virtual block's index.
template <int NV>
__device__ void grid_reduce(double (&v)[NV], const Reducer &red, double *result, int bid,
                            int nblocks)
{
    __shared__ double sh[NV][32];
    __shared__ bool last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    block_sum<NV>(v, sh);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red.partials[(size_t)k * red.capacity + bid] = v[k];
        __threadfence();
        const unsigned prev = atomicAdd(red.ticket, 1u);
        last = (prev == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nthr = blockDim.x * blockDim.y;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        acc[k] = 0.0;
        for (int i = tid; i < nblocks; i += nthr) acc[k] += __ldcg(&red.partials[(size_t)k * red.capacity + i]);
    }
    block_sum<NV>(acc, sh);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) result[k] = acc[k];
        *red.ticket = 0u;
    }
    __syncthreads();
}

template <int NV>
__device__ void grid_reduce(double (&v)[NV], const Reducer &red, double *result)
{
    grid_reduce<NV>(v, red, result,
                    (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x,
                    gridDim.x * gridDim.y * gridDim.z);
}

// Virtual-block dispatch: returns the arguments of the scan owning virtual block vb and its
// index / count within that scan.
template <class A>
__device__ __forceinline__ const A *scan_of(const A &one, const Batch &b, int vb, int &local,
                                            int &count)
{
    if (b.nscans == 0) { local = vb; count = one.nvb; return &one; }
    int lo = 0, hi = b.nscans;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&b.prefix[mid]) <= vb) lo = mid;
        else hi = mid;
    }
    local = vb - __ldg(&b.prefix[lo]);
    count = __ldg(&b.prefix[lo + 1]) - __ldg(&b.prefix[lo]);
    return reinterpret_cast<const A *>(b.args) + lo;
}

// As scan_of, for a whole block: in a batched launch the scan's argument struct is copied into
// the block's shared memory `sh` (one cooperative copy per virtual block; the kernel's field
// reads are then shared-memory loads instead of global ones); a single scan's arguments are
// used where they are (the kernel parameters).  Every thread of the block must call it with the
// same vb.
template <class A>
__device__ __forceinline__ const A &scan_args(const A &one, const Batch &b, int vb, int &local,
                                              int &count, A &sh)
{
    const A *src = scan_of(one, b, vb, local, count);
    if (b.nscans == 0) return one;
    static_assert(sizeof(A) % 4 == 0, "argument structs are copied as 32-bit words");
    __syncthreads();                                  // the previous virtual block is done with sh
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const unsigned *s = reinterpret_cast<const unsigned *>(src);
    unsigned *d = reinterpret_cast<unsigned *>(&sh);
    for (int k = tid; k < (int)(sizeof(A) / 4); k += nthr) d[k] = __ldg(s + k);
    __syncthreads();
    return sh;
}

template <class A>
__device__ __forceinline__ int total_vblocks(const A &one, const Batch &b)
{
    return b.nscans == 0 ? one.nvb : __ldg(&b.prefix[b.nscans]);
}

}  // namespace pet
