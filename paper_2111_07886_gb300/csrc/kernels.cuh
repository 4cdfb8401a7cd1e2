// Device helpers shared by the projector and update kernels: plane-group loads, packed
// FP32x2 arithmetic (sm_100+ f32x2 instructions), compensated sums, the pixel-driven
// backprojection gather, and the deterministic last-block FP64 reduction.
#pragma once

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
// Sums of G planes.  Each step adds the two-term contribution w0 x0 + w1 x1 of one driving
// step (forward) or one view (backward).
//   AR_FP32 : s += w0 x0 + w1 x1 with FMAs
//   AR_KAHAN: compensated: y = w0 x0 + w1 x1 + e; t = s + y; e = y - (t - s); s = t
//   AR_FP64 : double FMAs
// The final value is s + e.
// ------------------------------------------------------------------------------------------
template <int G, int AR> struct GroupSum {
    using T = typename ArithT<AR>::T;
    T s[G], e[G];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int p = 0; p < G; ++p) { s[p] = T(0); e[p] = T(0); }
    }

    // y_p = w0 x0_p + w1 x1_p (+ e_p for Kahan), then accumulate
    __device__ __forceinline__ void add2terms(T w0, const T (&x0)[G], T w1, const T (&x1)[G])
    {
        if constexpr (AR == AR_KAHAN && G % 2 == 0) {
            const float2 W0 = make_float2(w0, w0), W1 = make_float2(w1, w1);
#pragma unroll
            for (int p = 0; p < G; p += 2) {
                float2 S = make_float2(s[p], s[p + 1]), E = make_float2(e[p], e[p + 1]);
                float2 y = fma2(W0, make_float2(x0[p], x0[p + 1]), E);
                y = fma2(W1, make_float2(x1[p], x1[p + 1]), y);
                float2 t = add2(S, y);
                E = sub2(y, sub2(t, S));
                s[p] = t.x; s[p + 1] = t.y; e[p] = E.x; e[p + 1] = E.y;
            }
        } else if constexpr (AR == AR_KAHAN) {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                float y = fmaf(w0, x0[p], e[p]);
                y = fmaf(w1, x1[p], y);
                float t = s[p] + y;
                e[p] = y - (t - s[p]);
                s[p] = t;
            }
        } else if constexpr (AR == AR_FP32 && G % 2 == 0) {
            const float2 W0 = make_float2(w0, w0), W1 = make_float2(w1, w1);
#pragma unroll
            for (int p = 0; p < G; p += 2) {
                float2 S = make_float2(s[p], s[p + 1]);
                S = fma2(W0, make_float2(x0[p], x0[p + 1]), S);
                S = fma2(W1, make_float2(x1[p], x1[p + 1]), S);
                s[p] = S.x; s[p + 1] = S.y;
            }
        } else {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                s[p] = fma(w0, x0[p], s[p]);
                s[p] = fma(w1, x1[p], s[p]);
            }
        }
    }

    // scalar-weight-only form (sensitivity: x == 1)
    __device__ __forceinline__ void add_scalar(T y0)
    {
        if constexpr (AR == AR_KAHAN) {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                float y = y0 + e[p];
                float t = s[p] + y;
                e[p] = y - (t - s[p]);
                s[p] = t;
            }
        } else {
#pragma unroll
            for (int p = 0; p < G; ++p) s[p] += y0;
        }
    }

    __device__ __forceinline__ T value(int p) const { return s[p] + e[p]; }
};

// ------------------------------------------------------------------------------------------
// Pixel-driven gather backprojection for pixel (ix, iy) and one plane group:
//   acc_p += sum_{u < nviews} sum_b len(view u, bin b, pixel) * proj[u][b][plane p]
// len is the exact length of the line of bin b inside the pixel square: the trapezoid
// min(L, (h - |delta|) rho / (major minor)) of the pixel's footprint, or, for views along an
// axis, L for the rays inside the pixel's half-open column.  delta = b - t(ix, iy), in bins.
// proj == nullptr backprojects ones.  Views are taken in order and each view's candidate bins
// are added in pairs with one compensated step: the sum order is fixed (deterministic).
// ------------------------------------------------------------------------------------------
template <int G, int AR>
__device__ __forceinline__ void gather_bp(const GeoDev &g, int slot0, int nviews,
                                          const typename ArithT<AR>::T *__restrict__ proj,
                                          int grp, int ix, int iy, GroupSum<G, AR> &acc)
{
    using T = typename ArithT<AR>::T;
    const int NB = g.NB, Pp = g.Pp, K = g.K;
    T zero[G];
#pragma unroll
    for (int p = 0; p < G; ++p) zero[p] = T(0);
    for (int u = 0; u < nviews; ++u) {
        const ViewGeo &vw = g.views[slot0 + u];
        const T *base = proj ? proj + (size_t)u * NB * Pp + (size_t)grp * G : nullptr;
        if (vw.axis) {
            // Views along an axis: every ray runs along one pixel column (row).  Ray b belongs
            // to the pixel whose half-open column contains it, decided from the very start
            // coordinate the forward walk uses, so ties on pixel edges match it exactly.
            const int cross = vw.xdrive ? iy : ix;
            const RayGeo *rr = g.rays + (size_t)(slot0 + u) * NB;
            int bs;
            if constexpr (AR == AR_FP64)
                bs = (int)floor(vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy - vw.h);
            else
                bs = (int)((vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq - vw.hq) >> 32);
            for (int k = 0; k <= K; ++k) {
                const int b = bs + k;
                if ((unsigned)b >= (unsigned)NB) continue;
                int c;
                if constexpr (AR == AR_FP64) c = (int)floor(rr[b].lo);
                else c = (int)(rr[b].loq >> 32);
                if (c != cross) continue;
                if (base == nullptr) {
                    acc.add_scalar((T)vw.L);
                } else {
                    T x[G];
                    load_group<G, T>(base + (size_t)b * Pp, x);
                    acc.add2terms((T)vw.L, x, T(0), zero);
                }
            }
            continue;
        }
        // Oblique views: trapezoid footprint; the candidate bins are ceil(t - h) + k, k < K.
        for (int k0 = 0; k0 < K; k0 += 2) {
            T w[2];
            int bc[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                T ww;
                int b;
                if constexpr (AR == AR_FP64) {
                    const double t = vw.t0 + (double)ix * vw.cx + (double)iy * vw.cy;
                    b = (int)ceil(t - vw.h) + k0 + k;
                    const double dd = vw.h - fabs((double)b - t);
                    ww = dd > 0.0 ? fmin(vw.L, dd * vw.wslope) : 0.0;
                } else {
                    const long long tq = vw.t0q + (long long)ix * vw.cxq + (long long)iy * vw.cyq;
                    b = (int)((tq - vw.hq + 0xFFFFFFFFLL) >> 32) + k0 + k;   // ceil(t - h) + k
                    const long long dq = ((long long)b << 32) - tq;
                    const long long dd = vw.hq - (dq < 0 ? -dq : dq);
                    ww = dd > 0 ? fminf(vw.Lf, __ll2float_rn(dd) * kQ32 * vw.wslopef) : 0.f;
                }
                const bool ok = (unsigned)b < (unsigned)NB && k0 + k < K;
                w[k] = ok ? ww : T(0);
                bc[k] = ok ? b : 0;
            }
            if (base == nullptr) {
                acc.add_scalar(w[0] + w[1]);
            } else {
                T x0[G], x1[G];
                load_group<G, T>(base + (size_t)bc[0] * Pp, x0);
                load_group<G, T>(base + (size_t)bc[1] * Pp, x1);
                acc.add2terms(w[0], x0, w[1], x1);
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

template <int NV>
__device__ void grid_reduce(double (&v)[NV], const Reducer &red, double *result)
{
    __shared__ double sh[NV][32];
    __shared__ bool last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
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
}

}  // namespace pet
