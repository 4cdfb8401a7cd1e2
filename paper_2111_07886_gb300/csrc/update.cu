// Image-space kernels of one SDP-BSREM subiteration (Table I):
//   - the fused update: gather backprojection b = A_i^T w, RDP gradient (Eq. gradRD, 8-point
//     in-plane neighbourhood), the smoothness map nu (Sec. III, Eq. nuki), the preconditioner
//     S (Eq. preconditioner) and the clamp P_t (Eq. OperatorPt), with the FP64 sum of the new
//     iterate in the epilogue;
//   - the mu reduction that feeds mean(mu), the plain sum behind mean(f), and the stand-alone
//     RDP value / gradient and nu maps.
// Pixel-driven: one thread handles one pixel and one group of G planes; neighbours come
// through L1; the gather's (pixel, view) weights are shared by all groups through shared memory.
#include "kernels.cuh"
#include "profile.cuh"

#ifndef UPDATE_G1_BLOCKS
#define UPDATE_G1_BLOCKS 4      // resident blocks per SM the single-plane update kernel is built for
#endif
#ifndef UPDATE_X8_BLOCKS
#define UPDATE_X8_BLOCKS 3      // resident blocks per SM the packed update kernel is built for
#endif

namespace pet {

// Loads the 3x3 in-plane neighbourhood of pixel (ix, iy) for one plane group.
//   RG: gr_p = 2 sum_k (f_j - f_k)(gamma_R |f_j - f_k| + f_j + 3 f_k + 2 eps) / den^2
//       (den = f_j + f_k + gamma_R |f_j - f_k| + eps; FP32 kernels use the fast reciprocal)
//   MU: gx_p, gy_p of the Matlab-style gradient: central differences inside, one-sided at
//       the edges (the missing side counts as the centre value)
//   RV: rv_p = sum_k (f_j - f_k)^2 / den
// z3: the neighbourhood is the 26 voxels around (ix, iy, plane) in the volume (neighbours
// outside it are absent), and MU also gives gz_p, the gradient across the planes (central
// inside, one-sided at the first and last plane, 0 for one plane).  Each position's plane group
// is loaded with the planes just below and above it.
template <int G, int AR, bool RG, bool MU, bool RV>
__device__ __forceinline__ void stencil(const GeoDev &g, const typename ArithT<AR>::T *f, int grp,
                                        int ix, int iy, typename ArithT<AR>::T gamma_r,
                                        typename ArithT<AR>::T eps,
                                        typename ArithT<AR>::T (&fc)[G],
                                        typename ArithT<AR>::T (&gr)[G],
                                        typename ArithT<AR>::T (&gx)[G],
                                        typename ArithT<AR>::T (&gy)[G],
                                        typename ArithT<AR>::T (&rv)[G],
                                        bool z3 = false, typename ArithT<AR>::T *gz = nullptr)
{
    using T = typename ArithT<AR>::T;
    const int N = g.N, Pp = g.Pp;
    const T *base = f + grp * G;
    const unsigned jc = (unsigned)iy * (unsigned)N + (unsigned)ix;   // images hold < 2^32 elements
    load_group<G, T>(base + jc * (unsigned)Pp, fc);
    const T hx = (ix > 0 && ix < N - 1) ? T(0.5) : T(1);
    const T hy = (iy > 0 && iy < N - 1) ? T(0.5) : T(1);
#pragma unroll
    for (int p = 0; p < G; ++p) { gr[p] = T(0); gx[p] = T(0); gy[p] = T(0); rv[p] = T(0); }
    if constexpr (MU) {
        // a missing neighbour on one side is replaced by the centre value
        const T sx = (ix == 0 ? -hx : T(0)) + (ix == N - 1 ? hx : T(0));
        const T sy = (iy == 0 ? -hy : T(0)) + (iy == N - 1 ? hy : T(0));
#pragma unroll
        for (int p = 0; p < G; ++p) { gx[p] = sx * fc[p]; gy[p] = sy * fc[p]; }
    }
    // one (centre, neighbour) pair of Eq. RDP / Eq. gradRD
    auto pair = [&](int p, T c, T k) {
        const T d = c - k;
        const T ad = d < T(0) ? -d : d;
        const T den = c + k + gamma_r * ad + eps;
        if constexpr (RG) {
            const T num = d * (gamma_r * ad + c + T(3) * k + T(2) * eps);
            if constexpr (AR == AR_FP64) gr[p] += num / (den * den);
            else gr[p] += __fdividef(num, den * den);
        }
        if constexpr (RV) {
            if constexpr (AR == AR_FP64) rv[p] += d * d / den;
            else rv[p] += __fdividef(d * d, den);
        }
    };
    const int z0 = grp * G;                  // plane of element 0 of the group
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int dx = q % 3 - 1, dy = q / 3 - 1;
        if (q == 4 && !z3) continue;
        if (!RG && !RV && dx != 0 && dy != 0) continue;    // gradient only: axial neighbours
        const int x = ix + dx, y = iy + dy;
        if (x < 0 || y < 0 || x >= N || y >= N) continue;
        const unsigned jn = (unsigned)((int)jc + dy * N + dx) * (unsigned)Pp;
        T fk[G];
        if (q == 4) {
#pragma unroll
            for (int p = 0; p < G; ++p) fk[p] = fc[p];
        } else {
            load_group<G, T>(base + jn, fk);
        }
        if (z3) {
            // the planes just below and above this position's group
            const T lo = z0 > 0 ? f[jn + z0 - 1] : T(0);
            const T hi = z0 + G < g.P ? f[jn + z0 + G] : T(0);
#pragma unroll
            for (int p = 0; p < G; ++p) {
                const int z = z0 + p;
                if (z >= g.P) continue;
                if (RG || RV) {
                    if (q != 4) pair(p, fc[p], fk[p]);
                    if (z > 0) pair(p, fc[p], p > 0 ? fk[p - 1] : lo);
                    if (z + 1 < g.P) pair(p, fc[p], p + 1 < G ? fk[p + 1] : hi);
                }
                if constexpr (MU) {
                    if (q == 4 && gz) {
                        const T dn = z > 0 ? (p > 0 ? fk[p - 1] : lo) : fc[p];
                        const T up = z + 1 < g.P ? (p + 1 < G ? fk[p + 1] : hi) : fc[p];
                        gz[p] = (z > 0 && z + 1 < g.P ? T(0.5) : T(1)) * (up - dn);
                    }
                }
            }
        } else if constexpr (RG && AR != AR_FP64 && G % 2 == 0) {
            // packed FP32x2: two planes per instruction; 1/den^2 from the fast reciprocal
            const float2 GR = make_float2(gamma_r, gamma_r), THREE = make_float2(3.f, 3.f);
#pragma unroll
            for (int p = 0; p < G; p += 2) {
                const float2 c2 = make_float2(fc[p], fc[p + 1]), k2 = make_float2(fk[p], fk[p + 1]);
                const float2 d = sub2(c2, k2);
                const float2 ad = make_float2(fabsf(d.x), fabsf(d.y));
                const float2 den = fma2(GR, ad, add2(add2(c2, k2), make_float2(eps, eps)));
                const float2 t = fma2(GR, ad, fma2(THREE, k2, add2(c2, make_float2(2.f * eps, 2.f * eps))));
                const float2 num = mul2(d, t);
                const float2 den2 = mul2(den, den);
                const float2 qq = make_float2(__fdividef(num.x, den2.x), __fdividef(num.y, den2.y));
                gr[p] += qq.x;
                gr[p + 1] += qq.y;
            }
        } else if constexpr (RG || RV) {
#pragma unroll
            for (int p = 0; p < G; ++p) pair(p, fc[p], fk[p]);
        }
        if constexpr (MU) {
            if (q == 4) continue;
            if (dy == 0) {
                const T sgn = dx < 0 ? -hx : hx;
#pragma unroll
                for (int p = 0; p < G; ++p) gx[p] += sgn * fk[p];
            } else if (dx == 0) {
                const T sgn = dy < 0 ? -hy : hy;
#pragma unroll
                for (int p = 0; p < G; ++p) gy[p] += sgn * fk[p];
            }
        }
    }
    if constexpr (RG) {
#pragma unroll
        for (int p = 0; p < G; ++p) gr[p] *= T(2);
    }
}

template <typename T>
__device__ __forceinline__ T clampT(T v, T lo, T hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T>
__device__ __forceinline__ T fast_div(T a, T b)
{
    if constexpr (sizeof(T) == 8) return a / b;
    else return __fdividef(a, b);
}

// |(gx, gy)|: FP32 kernels use x rsqrt(x) (two instructions, a few ulp)
template <typename T>
__device__ __forceinline__ T grad_norm(T gx, T gy)
{
    const T x = gx * gx + gy * gy;
    if constexpr (sizeof(T) == 8) return sqrt(x);
    else return x > 0.f ? x * rsqrtf(x) : 0.f;
}

// |(gx, gy, gz)|
template <typename T>
__device__ __forceinline__ T grad_norm3(T gx, T gy, T gz)
{
    const T x = gx * gx + gy * gy + gz * gz;
    if constexpr (sizeof(T) == 8) return sqrt(x);
    else return x > 0.f ? x * rsqrtf(x) : 0.f;
}

// mu = max(0.01, |grad f| / mean(f)); nu = P_{nu1}^{nu2}(mean(mu) / mu)
template <typename T>
__device__ __forceinline__ T nu_of(T gx, T gy, T gz, T inv_mean_f, T mean_mu, T nu1, T nu2)
{
    T mu = grad_norm3(gx, gy, gz) * inv_mean_f;
    mu = mu < T(0.01) ? T(0.01) : mu;
    return clampT<T>(fast_div(mean_mu, mu), nu1, nu2);
}

int sm_count();

void update_fp32_scalars(UpdateArgs &a)
{
    a.fs_lam = (float)a.lam_alpha;
    a.fs_bm = (float)a.beta_over_M;
    a.fs_gamma_r = (float)a.gamma_r;
    a.fs_eps = (float)a.eps;
    a.fs_t = (float)a.t;
    a.fs_U = (float)a.U;
    a.fs_nu1 = (float)a.nu1;
    a.fs_nu2 = (float)a.nu2;
    a.fs_ips = (float)a.invp_scale;
    a.fs_scale = (float)a.g.scale;
}

// the scalar in the kernel's arithmetic: the host-converted FP32 copy, or the double
template <typename T>
__device__ __forceinline__ T scal(double d, float f)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

// f^{k,i} = P_t(f - lambda_k alpha_{k,i} nu S(f) (A_i^T w + (beta/M) grad R(f)))
// Virtual block: tpv tiles of TP consecutive pixels x NG plane groups (thread = pixel * NG +
// group); the (pixel, view) weights of each tile are computed once into shared memory.  A
// persistent grid strides over the virtual blocks of one scan or of a batch of scans.
template <int G, int KC, int AR, bool SUB = false, bool TOF = false>
__global__ void __launch_bounds__(256, G == 1 ? UPDATE_G1_BLOCKS : 3) update_kernel(
    const __grid_constant__ UpdateArgs one, const Batch bt)
{
    using T = typename ArithT<AR>::T;
    __shared__ BpTable<KC, AR> tb;
    grid_dependents_launch();                    // as in update_kernel_x8
    const int total = total_vblocks(one, bt);
    __shared__ UpdateArgs sh_args;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const UpdateArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int N = g.N, NG = g.NG, Pp = g.Pp, npix = N * N;
        const int TP = 256 / NG;
        const int pl = threadIdx.x / NG, grp = threadIdx.x % NG;
        const int VC = max(1, min(a.nviews, BpTable<KC, AR>::CAP / TP));
        const bool dyn = a.nu_mode == 1 || a.nu_mode == 2;
        const double q = (double)npix * g.P;
        // per-scan scalars in the kernel's arithmetic: an FP64 division in every thread of every
        // virtual block is costly at GB300's FP64 rate
        const T inv_mean_f = dyn ? (T)q / (T)*a.sum_f : T(1);
        const T mean_mu = dyn ? (T)*a.sum_mu / (T)q : T(1);
        const T lam = scal<T>(a.lam_alpha, a.fs_lam), bm = scal<T>(a.beta_over_M, a.fs_bm);
        const T U = scal<T>(a.U, a.fs_U), tt = scal<T>(a.t, a.fs_t);
        const T nu1 = scal<T>(a.nu1, a.fs_nu1), nu2 = scal<T>(a.nu2, a.fs_nu2), halfU = T(0.5) * U;
        const T *w = reinterpret_cast<const T *>(a.w);
        const T *f = reinterpret_cast<const T *>(a.f);
        const T *invp = reinterpret_cast<const T *>(a.invp);
        const T scale = scal<T>(g.scale, a.fs_scale);
        const int ntiles = (npix + TP - 1) / TP;
        T part = T(0);
        for (int tile = vloc * a.tpv; tile < min(ntiles, (vloc + 1) * a.tpv); ++tile) {
            const int j0 = tile * TP, j = j0 + pl;
            const bool active = pl < TP && j < npix;
            // 1. stencil first, folded into fc, coef = lambda alpha nu S and rg = (beta/M) grad R,
            //    so that the backprojection's accumulators do not coexist with the stencil state
            T fc[G], coef[G], rg[G];
            if (active) {
                const int ix = j % N, iy = j / N;
                T gr[G], gx[G], gy[G], rv[G], gz[G];
#pragma unroll
                for (int p = 0; p < G; ++p) gz[p] = T(0);
                const T gam_r = scal<T>(a.gamma_r, a.fs_gamma_r), eps_t = scal<T>(a.eps, a.fs_eps);
                if (dyn) stencil<G, AR, true, true, false>(g, f, grp, ix, iy, gam_r, eps_t, fc, gr, gx, gy, rv, a.z3, gz);
                else stencil<G, AR, true, false, false>(g, f, grp, ix, iy, gam_r, eps_t, fc, gr, gx, gy, rv, a.z3, gz);
                T nu[G];
                if (a.nu_mode == 3) {
                    load_group<G, T>(reinterpret_cast<const T *>(a.nu_frozen) + (unsigned)j * (unsigned)Pp + grp * G, nu);
                } else if (!dyn) {
#pragma unroll
                    for (int p = 0; p < G; ++p) nu[p] = T(1);
                } else {
#pragma unroll
                    for (int p = 0; p < G; ++p) nu[p] = nu_of<T>(gx[p], gy[p], gz[p], inv_mean_f, mean_mu, nu1, nu2);
                    if (a.nu_mode == 2)
                        store_group<G, T>(reinterpret_cast<T *>(a.nu_frozen) + (unsigned)j * (unsigned)Pp + grp * G, nu);
                }
                T ipv[G];
                if (a.vox) {
                    load_group<G, T>(invp + (unsigned)j * (unsigned)Pp + grp * G, ipv);
#pragma unroll
                    for (int p = 0; p < G; ++p) ipv[p] *= scal<T>(a.invp_scale, a.fs_ips);
                } else {
                    const T ip = invp[j] * scal<T>(a.invp_scale, a.fs_ips);
#pragma unroll
                    for (int p = 0; p < G; ++p) ipv[p] = ip;
                }
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    const T S = (fc[p] < halfU ? fc[p] : U - fc[p]) * ipv[p];
                    coef[p] = lam * nu[p] * S;
                    rg[p] = bm * gr[p];
                }
            }
            // 2. gather backprojection A_i^T w with the tile's shared (pixel, view) weights
            GroupSum<G, AR> bp;
            bp.zero();
            for (int u0 = 0; u0 < a.nviews; u0 += VC) {
                const int nvc = min(VC, a.nviews - u0);
                __syncthreads();
                bp_fill<KC, AR, 0, SUB>(g, a.slot0, u0, nvc, j0, TP, tb);
                __syncthreads();
                if (!active) continue;
                if constexpr (TOF)
                    bp_accumulate_tof<G, KC, AR>(g, tb, w, TP, nvc, pl, grp, bp, j % N, j / N,
                                                 a.slot0, u0);
                else
                    bp_accumulate<G, KC, AR>(g, tb, w, TP, nvc, pl, grp, bp);
            }
            if (!active) continue;
            // 3. step and clamp P_t (TV variant: the unclamped z and the metric W = coef, for the
            //    proximal step that follows)
            T out[G], wv[G];
#pragma unroll
            for (int p = 0; p < G; ++p) {
                const T d = scale * bp.value(p) + rg[p];
                T ft = fc[p] - coef[p] * d;
                if (!a.tv) ft = ft <= T(0) ? tt : (ft >= U ? U - tt : ft);
                const bool valid = grp * G + p < g.P;
                out[p] = valid ? ft : T(0);
                wv[p] = valid ? coef[p] : T(1);
                part += out[p];
            }
            const unsigned o = (unsigned)j * (unsigned)Pp + grp * G;
            store_group<G, T>(reinterpret_cast<T *>(a.fout) + o, out);
            if (a.tv) {
                store_group<G, T>(reinterpret_cast<T *>(a.zbuf) + o, out);
                store_group<G, T>(reinterpret_cast<T *>(a.wbuf) + o, wv);
            }
        }
        double v[1] = {(double)part};
        grid_reduce<1>(v, a.red, a.sum_fout, vloc, nv);
    }
}

// FP32 update for 8-plane groups held as four f32x2 pairs.  Same step as update_kernel, with:
//   - the 3x3 stencil loading every neighbour with missing ones (image border) replaced by the
//     centre value: their RDP term is exactly zero (d = 0) and the Matlab-style gradient becomes
//     the one-sided difference, as in the generic stencil;
//   - the RDP pair term written as d (den + 2 f_k + eps) / den^2 (the numerator
//     gamma_R |d| + f_j + 3 f_k + 2 eps equals den + 2 f_k + eps), from one reciprocal of den;
//   - nu = P_{nu1}^{nu2}(mean(mu) / mu) from 1 / mu = min(100, mean(f) / |grad f|);
//   - the step folded into two per-plane constants before the gather,
//     f^{k,i} = P_t(A + B b) with A = f - c (beta/M) grad R, B = -c scale, c = lambda alpha nu S,
//     so that only A, B and the sums of b = A_i^T w stay live across the gather.
template <int KC, int AR>
__global__ void __launch_bounds__(256, UPDATE_X8_BLOCKS) update_kernel_x8(
    const __grid_constant__ UpdateArgs one, const Batch bt)
{
    static_assert(AR != AR_FP64, "FP32 arithmetic only");
    // 16 KB of (pixel, view) entries: the rest of the SM's shared memory stays L1 for the gather
    using Table = BpTable<KC, AR, 1024 / (KC > 2 ? 2 : 1)>;
    __shared__ Table tb;
    // the next subiteration's projection (launched after this kernel with programmatic stream
    // serialization) may be scheduled as this kernel's blocks retire; it waits for completion
    grid_dependents_launch();
    const int total = total_vblocks(one, bt);
    __shared__ UpdateArgs sh_args;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const UpdateArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int N = g.N, NG = g.NG, npix = N * N;
        const unsigned Pp = (unsigned)g.Pp;
        const int TP = 256 / NG;
        const int pl = threadIdx.x / NG, grp = threadIdx.x % NG;
        const int VC = max(1, min(a.nviews, Table::CAP / TP));
        const bool dyn = a.nu_mode == 1 || a.nu_mode == 2;
        const double q = (double)npix * g.P;
        // per-scan scalars in FP32 (an FP64 division per thread is costly at GB300's FP64 rate)
        const float mean_f = dyn ? (float)*a.sum_f / (float)q : 1.f;
        const float mean_mu = dyn ? (float)*a.sum_mu / (float)q : 1.f;
        const float U = a.fs_U, tt = a.fs_t;
        // eps >= 1e-30 keeps 1/den finite, so that a zero-difference term stays exactly zero
        const float eps = fmaxf(a.fs_eps, 1e-30f);
        const float *f = reinterpret_cast<const float *>(a.f) + grp * 8;
        const float *w = reinterpret_cast<const float *>(a.w) + grp * 8;
        const float *invp = reinterpret_cast<const float *>(a.invp);
        const int ntiles = (npix + TP - 1) / TP;
        // the subset's precomputed entries (one contiguous block per tile) when two tiles' entries
        // fit the table: double-buffered, the next tile's block copied with cp.async while this
        // tile is gathered and the next one's stencil runs (one barrier per tile)
        const bool pre = a.bptab && 2 * a.nviews * TP <= Table::CAP;
        const int t0 = vloc * a.tpv, t1 = min(ntiles, (vloc + 1) * a.tpv);
        auto copy_tile = [&](int tile) {
            const int tbytes = a.nviews * TP * (int)sizeof(typename Table::E);
            const char *src = static_cast<const char *>(a.bptab) + (size_t)tile * tbytes;
            char *dst = reinterpret_cast<char *>(tb.e) + ((tile - t0) & 1) * tbytes;
            for (int o = threadIdx.x * 16; o < tbytes; o += 256 * 16) cp_async16(dst + o, src + o);
            cp_async_commit();
        };
        if (pre && t0 < t1) copy_tile(t0);
        float part = 0.f;
        for (int tile = t0; tile < t1; ++tile) {
            const int j0 = tile * TP, j = j0 + pl;
            const bool active = pl < TP && j < npix;
            f2x A[4], B[4];
            if (active) {
                const int ix = j % N, iy = j / N;
                const unsigned jc = (unsigned)j;
                const unsigned xm = ix > 0 ? jc - 1 : jc, xp = ix < N - 1 ? jc + 1 : jc;
                const unsigned ym = iy > 0 ? jc - N : jc, yp = iy < N - 1 ? jc + N : jc;
                const f2x GR = vsplat(a.fs_gamma_r), EP = vsplat(eps), TWO = vsplat(2.f);
                f2x c[4], ce[4], gr[4], g2[4], nb0[4], nb1[4];
                load8x(f + jc * Pp, c);
#pragma unroll
                for (int k = 0; k < 4; ++k) { ce[k] = vadd(c[k], EP); gr[k] = 0ull; }
                auto rdp = [&](const f2x(&x)[4]) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const f2x d = vsub(c[k], x[k]);
                        const f2x den = vfma(GR, vabs(d), vadd(ce[k], x[k]));
                        const f2x num = vadd(den, vfma(TWO, x[k], EP));
                        const f2x r = vrcp(den);
                        gr[k] = vfma(vmul(d, vmul(num, r)), r, gr[k]);
                    }
                };
                // axial neighbours: RDP terms and the Matlab-style gradient
                load8x(f + xm * Pp, nb0);
                load8x(f + xp * Pp, nb1);
                rdp(nb0);
                rdp(nb1);
                if (dyn) {
                    const f2x HX = vsplat((ix > 0 && ix < N - 1) ? 0.5f : 1.f);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const f2x t = vmul(HX, vsub(nb1[k], nb0[k]));
                        g2[k] = vmul(t, t);
                    }
                }
                load8x(f + ym * Pp, nb0);
                load8x(f + yp * Pp, nb1);
                rdp(nb0);
                rdp(nb1);
                f2x nu[4];
                if (dyn) {
                    const f2x HY = vsplat((iy > 0 && iy < N - 1) ? 0.5f : 1.f);
                    const float nu1 = a.fs_nu1, nu2 = a.fs_nu2;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const f2x t = vmul(HY, vsub(nb1[k], nb0[k]));
                        float r0, r1;
                        vunpk(vrsqrt(vfma(t, t, g2[k])), r0, r1);
                        // 1 / mu = 1 / max(0.01, |grad f| / mean f) = min(100, mean f / |grad f|)
                        r0 = fminf(100.f, r0 * mean_f);
                        r1 = fminf(100.f, r1 * mean_f);
                        nu[k] = vpk(fminf(fmaxf(mean_mu * r0, nu1), nu2),
                                    fminf(fmaxf(mean_mu * r1, nu1), nu2));
                    }
                    if (a.nu_mode == 2)
                        store8x(reinterpret_cast<float *>(a.nu_frozen) + jc * Pp + grp * 8, nu);
                } else if (a.nu_mode == 3) {
                    load8x(reinterpret_cast<const float *>(a.nu_frozen) + jc * Pp + grp * 8, nu);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) nu[k] = vsplat(1.f);
                }
                // diagonal neighbours
                const unsigned dm = iy > 0 ? jc - N : jc, dp = iy < N - 1 ? jc + N : jc;
                load8x(f + (ix > 0 && iy > 0 ? dm - 1 : jc) * Pp, nb0);
                load8x(f + (ix < N - 1 && iy > 0 ? dm + 1 : jc) * Pp, nb1);
                rdp(nb0);
                rdp(nb1);
                load8x(f + (ix > 0 && iy < N - 1 ? dp - 1 : jc) * Pp, nb0);
                load8x(f + (ix < N - 1 && iy < N - 1 ? dp + 1 : jc) * Pp, nb1);
                rdp(nb0);
                rdp(nb1);
                // c = lambda alpha nu S, S = min(f, U - f) / p;  A = f - c (beta/M) 2 gr;  B = -c scale
                const f2x NK = vsplat(-a.fs_lam * invp[j] * a.fs_ips);
                const f2x BM = vsplat(2.f * a.fs_bm), SC = vsplat(a.fs_scale);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float c0, c1;
                    vunpk(c[k], c0, c1);
                    const f2x S = vpk(fminf(c0, U - c0), fminf(c1, U - c1));
                    const f2x cn = vmul(vmul(nu[k], S), NK);
                    A[k] = vfma(cn, vmul(BM, gr[k]), c[k]);
                    B[k] = vmul(cn, SC);
                }
            }
            // gather backprojection b = A_i^T w with the tile's shared (pixel, view) weights
            f2x sm[4], er[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) { sm[k] = 0ull; er[k] = 0ull; }
            for (int u0 = 0; u0 < a.nviews; u0 += VC) {
                const int nvc = min(VC, a.nviews - u0);
                if (pre) {
                    cp_async_wait_all();             // this tile's block (this thread's part)
                    __syncthreads();                 // all parts; the previous gather is done
                    if (tile + 1 < t1) copy_tile(tile + 1);
                } else {
                    __syncthreads();
                    bp_fill<KC, AR>(g, a.slot0, u0, nvc, j0, TP, tb);
                    __syncthreads();
                }
                if (!active) continue;
                const typename Table::E *te = tb.e + (pre ? ((tile - t0) & 1) * a.nviews * TP : 0);
                for (int uu = 0; uu < nvc; ++uu) {
                    const typename Table::E ent = te[uu * TP + pl];
                    const float *row = w + ent.off;
#pragma unroll
                    for (int kb = 0; kb < KC; kb += 2) {
                        f2x x0[4], x1[4];
                        load8x(row + kb * Pp, x0);
                        load8x(row + (kb + 1) * Pp, x1);
                        const f2x W0 = vsplat(ent.w[kb]), W1 = vsplat(ent.w[kb + 1]);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if constexpr (AR == AR_KAHAN) {
                                const f2x y = vfma(W1, x1[k], vfma(W0, x0[k], er[k]));
                                const f2x t = vadd(sm[k], y);
                                er[k] = vsub(y, vsub(t, sm[k]));
                                sm[k] = t;
                            } else {
                                sm[k] = vfma(W1, x1[k], vfma(W0, x0[k], sm[k]));
                            }
                        }
                    }
                }
            }
            if (!active) continue;
            // step and clamp P_t
            f2x out[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const f2x b = AR == AR_KAHAN ? vadd(sm[k], er[k]) : sm[k];
                float f0, f1;
                vunpk(vfma(B[k], b, A[k]), f0, f1);
                f0 = f0 <= 0.f ? tt : (f0 >= U ? U - tt : f0);
                f1 = f1 <= 0.f ? tt : (f1 >= U ? U - tt : f1);
                const int p0 = grp * 8 + 2 * k;
                f0 = p0 < g.P ? f0 : 0.f;
                f1 = p0 + 1 < g.P ? f1 : 0.f;
                part += f0 + f1;
                out[k] = vpk(f0, f1);
            }
            store8x(reinterpret_cast<float *>(a.fout) + (unsigned)j * Pp + grp * 8, out);
        }
        double v[1] = {(double)part};
        grid_reduce<1>(v, a.red, a.sum_fout, vloc, nv);
    }
}

// Stand-alone gather backprojection (also the sensitivity, proj == nullptr); one pixel tile
// per virtual block.
template <int G, int KC, int AR, bool SUB = false, bool TOF = false>
__global__ void __launch_bounds__(256) back_kernel(const __grid_constant__ BackArgs a)
{
    using T = typename ArithT<AR>::T;
    __shared__ BpTable<KC, AR> tb;
    const GeoDev &g = a.g;
    const int N = g.N, NG = g.NG, npix = N * N;
    const int TP = 256 / NG;
    const int pl = threadIdx.x / NG, grp = threadIdx.x % NG;
    const int VC = max(1, min(a.nviews, BpTable<KC, AR>::CAP / TP));
    const T *proj = reinterpret_cast<const T *>(a.proj);
    const int ntiles = (npix + TP - 1) / TP;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j0 = tile * TP, j = j0 + pl;
        const bool active = pl < TP && j < npix;
        GroupSum<G, AR> acc;
        acc.zero();
        for (int u0 = 0; u0 < a.nviews; u0 += VC) {
            const int nvc = min(VC, a.nviews - u0);
            __syncthreads();
            bp_fill<KC, AR, 0, SUB>(g, a.slot0, u0, nvc, j0, TP, tb);
            __syncthreads();
            if (!active) continue;
            if constexpr (TOF)
                bp_accumulate_tof<G, KC, AR>(g, tb, proj, TP, nvc, pl, grp, acc, j % N, j / N,
                                             a.slot0, u0);
            else
                bp_accumulate<G, KC, AR>(g, tb, proj, TP, nvc, pl, grp, acc);
        }
        if (!active) continue;
        T b[G];
        const T scale = (T)g.scale;
#pragma unroll
        for (int p = 0; p < G; ++p) b[p] = (grp * G + p < g.P) ? scale * acc.value(p) : T(0);
        store_group<G, T>(reinterpret_cast<T *>(a.img) + (size_t)j * g.Pp + (size_t)grp * G, b);
    }
}

// KIND 0: sum f; 1: sum mu; 2: nu map; 3: RDP gradient; 4: RDP value.  Virtual block: 256 x ipt
// (pixel, plane group) items, item = thread + 256 k.
template <int G, int AR, int KIND>
__global__ void __launch_bounds__(256) image_kernel(const __grid_constant__ ImageArgs one,
                                                    const Batch bt)
{
    using T = typename ArithT<AR>::T;
    const int total = total_vblocks(one, bt);
    __shared__ ImageArgs sh_args;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const ImageArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int N = g.N, NG = g.NG, Pp = g.Pp;
        const unsigned items = (unsigned)N * (unsigned)N * (unsigned)NG;    // < 2^32 (geometry limits)
        const double q = (double)N * N * g.P;
        const T *f = reinterpret_cast<const T *>(a.f);
        const T inv_mean_f = (KIND == 1 || KIND == 2) ? (T)q / (T)*a.sum_f : T(1);
        const T mean_mu = KIND == 2 ? (T)*a.sum_mu / (T)q : T(1);
        T part = T(0);
        for (int k = 0; k < a.ipt; ++k) {
            const unsigned tid = ((unsigned)vloc * (unsigned)a.ipt + (unsigned)k) * 256u + threadIdx.x;
            if (tid >= items) break;
            const int grp = NG == 1 ? 0 : (int)(tid % (unsigned)NG);
            const int j = NG == 1 ? (int)tid : (int)(tid / (unsigned)NG);
            const int ix = j % N, iy = j / N;
            T fc[G], gr[G], gx[G], gy[G], rv[G], out[G], gz[G];
#pragma unroll
            for (int p = 0; p < G; ++p) gz[p] = T(0);
            if constexpr (KIND == 0) {
                load_group<G, T>(f + (size_t)j * Pp + (size_t)grp * G, fc);
#pragma unroll
                for (int p = 0; p < G; ++p) part += (grp * G + p < g.P) ? fc[p] : T(0);
            } else if constexpr (KIND == 1 || KIND == 2) {
                stencil<G, AR, false, true, false>(g, f, grp, ix, iy, T(0), T(0), fc, gr, gx, gy, rv, a.z3, gz);
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    T mu = grad_norm3(gx[p], gy[p], gz[p]) * inv_mean_f;
                    mu = mu < T(0.01) ? T(0.01) : mu;
                    if constexpr (KIND == 1) {
                        part += (grp * G + p < g.P) ? mu : T(0);
                    } else {
                        out[p] = grp * G + p < g.P ? clampT<T>(fast_div(mean_mu, mu), (T)a.nu1, (T)a.nu2) : T(0);
                    }
                }
                if constexpr (KIND == 2)
                    store_group<G, T>(reinterpret_cast<T *>(a.out) + (size_t)j * Pp + (size_t)grp * G, out);
            } else if constexpr (KIND == 3) {
                stencil<G, AR, true, false, false>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gx, gy, rv, a.z3, gz);
#pragma unroll
                for (int p = 0; p < G; ++p) out[p] = grp * G + p < g.P ? gr[p] : T(0);
                store_group<G, T>(reinterpret_cast<T *>(a.out) + (size_t)j * Pp + (size_t)grp * G, out);
            } else if (a.tv) {
                // R_TV: |(f_{j+x} - f_j, f_{j+y} - f_j)|, a component 0 across the last column / row
                T fx[G], fy[G];
                load_group<G, T>(f + (size_t)j * Pp + (size_t)grp * G, fc);
                if (ix + 1 < N) load_group<G, T>(f + (size_t)(j + 1) * Pp + (size_t)grp * G, fx);
                if (iy + 1 < N) load_group<G, T>(f + (size_t)(j + N) * Pp + (size_t)grp * G, fy);
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    const T dx = ix + 1 < N ? fx[p] - fc[p] : T(0);
                    const T dy = iy + 1 < N ? fy[p] - fc[p] : T(0);
                    part += (grp * G + p < g.P) ? sqrt(dx * dx + dy * dy) : T(0);
                }
            } else {
                stencil<G, AR, false, false, true>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gx, gy, rv, a.z3, gz);
#pragma unroll
                for (int p = 0; p < G; ++p) part += (grp * G + p < g.P) ? rv[p] : T(0);
            }
        }
        if constexpr (KIND == 0 || KIND == 1 || KIND == 4) {
            double v[1] = {(double)part};
            grid_reduce<1>(v, a.red, a.result, vloc, nv);
        }
    }
}

// FP32 mu pass for 8-plane groups: sum over voxels of mu = max(0.01, |grad f| / mean(f))
// (Matlab-style gradient: central differences inside, one-sided at the border, where the
// missing neighbour is the centre value).  Thread layout of the update kernel (pixel x plane
// group, TP = 256 / NG pixels per tile); a virtual block takes a.ipt tiles.
__global__ void __launch_bounds__(256) mu_kernel_x8(const __grid_constant__ ImageArgs one, const Batch bt)
{
    const int total = total_vblocks(one, bt);
    __shared__ ImageArgs sh_args;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const ImageArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int N = g.N, NG = g.NG, npix = N * N;
        const unsigned Pp = (unsigned)g.Pp;
        const int TP = 256 / NG;
        const int pl = threadIdx.x / NG, grp = threadIdx.x % NG;
        const int ntiles = (npix + TP - 1) / TP;
        const float inv_mean_f = (float)((double)npix * g.P) / (float)*a.sum_f;
        const float *f = reinterpret_cast<const float *>(a.f) + grp * 8;
        const int nvalid = min(8, g.P - grp * 8);             // real planes of this group
        float part = 0.f;
        for (int tile = vloc * a.ipt; tile < min(ntiles, (vloc + 1) * a.ipt); ++tile) {
            const int j = tile * TP + pl;
            if (pl >= TP || j >= npix) continue;
            const int ix = j % N, iy = j / N;
            const unsigned jc = (unsigned)j;
            f2x w_[4], e_[4], n_[4], s_[4];
            load8x(f + (ix > 0 ? jc - 1 : jc) * Pp, w_);
            load8x(f + (ix < N - 1 ? jc + 1 : jc) * Pp, e_);
            load8x(f + (iy > 0 ? jc - N : jc) * Pp, n_);
            load8x(f + (iy < N - 1 ? jc + N : jc) * Pp, s_);
            const f2x HX = vsplat((ix > 0 && ix < N - 1) ? 0.5f : 1.f);
            const f2x HY = vsplat((iy > 0 && iy < N - 1) ? 0.5f : 1.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const f2x gx = vmul(HX, vsub(e_[k], w_[k])), gy = vmul(HY, vsub(s_[k], n_[k]));
                const f2x x2 = vfma(gx, gx, vmul(gy, gy));
                float x0, x1, r0, r1;
                vunpk(x2, x0, x1);
                vunpk(vrsqrt(x2), r0, r1);
                // |grad f|^2 below the smallest normal float (|grad f| < 1.1e-19, met on decayed
                // backgrounds) counts as zero: mu = 0.01 there, and the flushed rsqrt would be inf
                const float m0 = fmaxf(0.01f, x0 >= 1.17549435e-38f ? x0 * r0 * inv_mean_f : 0.f);
                const float m1 = fmaxf(0.01f, x1 >= 1.17549435e-38f ? x1 * r1 * inv_mean_f : 0.f);
                part += (2 * k < nvalid ? m0 : 0.f) + (2 * k + 1 < nvalid ? m1 : 0.f);
            }
        }
        double v[1] = {(double)part};
        grid_reduce<1>(v, a.red, a.result, vloc, nv);
    }
}

// Plane grouping of the update kernel: the full 8-plane groups (measured faster at three blocks
// per SM than 4-plane half groups, whose per-thread overheads double).
GeoDev update_geo(const GeoDev &g) { return g; }

// pixel tiles per virtual block so that a scan never needs more partial sums than its reducer
int resident_blocks(const void *fn);

template <int G, int KC>
static const void *update_fn(int arith, int z3 = 0, int sub = 0, int tof = 0)
{
    if (tof && sub) {                            // TOF on ring-sampled bins: KC = 4
        if (arith == AR_FP32) return (const void *)update_kernel<G, 4, AR_FP32, true, true>;
        if (arith == AR_KAHAN) return (const void *)update_kernel<G, 4, AR_KAHAN, true, true>;
        return (const void *)update_kernel<G, 4, AR_FP64, true, true>;
    }
    if (tof) {                                   // TOF geometries: generic kernel
        if (arith == AR_FP32) return (const void *)update_kernel<G, KC, AR_FP32, false, true>;
        if (arith == AR_KAHAN) return (const void *)update_kernel<G, KC, AR_KAHAN, false, true>;
        return (const void *)update_kernel<G, KC, AR_FP64, false, true>;
    }
    if (sub) {                                   // sub-ray geometries: KC = 4, generic kernel
        if (arith == AR_FP32) return (const void *)update_kernel<G, 4, AR_FP32, true>;
        if (arith == AR_KAHAN) return (const void *)update_kernel<G, 4, AR_KAHAN, true>;
        return (const void *)update_kernel<G, 4, AR_FP64, true>;
    }
    if constexpr (G == 8) {
        if (z3 && arith == AR_FP32) return (const void *)update_kernel<G, KC, AR_FP32>;
        if (z3 && arith == AR_KAHAN) return (const void *)update_kernel<G, KC, AR_KAHAN>;
        if (arith == AR_FP32) return (const void *)update_kernel_x8<KC, AR_FP32>;
        if (arith == AR_KAHAN) return (const void *)update_kernel_x8<KC, AR_KAHAN>;
    } else {
        if (arith == AR_FP32) return (const void *)update_kernel<G, KC, AR_FP32>;
        if (arith == AR_KAHAN) return (const void *)update_kernel<G, KC, AR_KAHAN>;
    }
    return (const void *)update_kernel<G, KC, AR_FP64>;
}

// Entries of update_kernel_x8's (pixel, view) table for one subset, computed once per geometry:
// entry e = (tile t, view u, pixel pl of the tile) is bp_entry(pixel t TP + pl, view u), in the
// kernel's shared-memory order, so that one tile's entries are one contiguous block.  bp_entry
// has no arithmetic that differs between the FP32 kernels (the FP32 and FP32 + Kahan tables are
// the same bits as those the kernel computes).
template <int KC>
__global__ void __launch_bounds__(256) bp_table_kernel(const __grid_constant__ GeoDev g, int slot0,
                                                      int nviews, int TP, long long nent, void *out)
{
    using E = typename BpTable<KC, AR_KAHAN, 1024 / (KC > 2 ? 2 : 1)>::E;
    const long long per = (long long)nviews * TP;
    const int npix = g.N * g.N;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < nent; e += (long long)gridDim.x * 256) {
        const long long tile = e / per;
        const int r = (int)(e - tile * per);
        const int uu = r / TP, pl = r - uu * TP;
        const long long j = tile * TP + pl;
        const bool in = j < npix;
        reinterpret_cast<E *>(out)[e] = bp_entry<KC, AR_KAHAN, 1024 / (KC > 2 ? 2 : 1)>(
            g, slot0, uu, in, in ? (int)(j % g.N) : 0, in ? (int)(j / g.N) : 0);
    }
}

// The packed update kernel runs for 8-plane groups with uniform bins and without TOF; its table
// holds 1024 (KC = 2) or 512 (KC = 4) entries of 16 or 32 bytes, two tiles' worth when copied.
size_t bp_table_bytes_bound(const pet_geometry_desc &d)
{
    if (d.nplanes <= 1 || d.subrays > 1 || d.ring_mm > 0 || d.tof_bins > 1) return 0;
    const long long NG = (d.nplanes + 7) / 8, TP = 256 / NG;
    const long long npix = (long long)d.n * d.n, ntiles = (npix + TP - 1) / TP;
    const long long vmax = (d.nviews + d.nsubsets - 1) / d.nsubsets;
    if (TP < 1 || 2 * vmax * TP > 1024) return 0;
    return (size_t)(ntiles * d.nviews * TP * 32);
}

pet_status build_bp_table(pet_geometry *g, cudaStream_t st)
{
    const GeoDev &gd = g->dev;
    g->bptab_off.clear();
    if (gd.G != 8 || gd.table || gd.T > 1) return PET_OK;
    const int KC = gd.K <= 2 ? 2 : 4;
    const int CAP = KC > 2 ? 512 : 1024;
    const int TP = 256 / gd.NG;
    if (TP < 1) return PET_OK;
    const size_t esz = KC > 2 ? sizeof(BpTable<4, AR_KAHAN, 512>::E) : sizeof(BpTable<2, AR_KAHAN, 1024>::E);
    const long long ntiles = ((long long)gd.N * gd.N + TP - 1) / TP;
    std::vector<size_t> off(gd.M);
    size_t total = 0;
    for (int i = 0; i < gd.M; ++i) {
        const int nv = g->voff[i + 1] - g->voff[i];
        if (2 * nv * TP > CAP) return PET_OK;       // the kernel computes this geometry's entries
        off[i] = total;
        total += (size_t)ntiles * nv * TP * esz;
    }
    if (total == 0) return PET_OK;
    void *tab = nullptr;
    PET_CUDA(dev_malloc(&tab, total));
    for (int i = 0; i < gd.M; ++i) {
        const int nv = g->voff[i + 1] - g->voff[i];
        const long long nent = ntiles * nv * TP;
        const int grid = (int)std::min<long long>((nent + 255) / 256, (long long)sm_count() * 16);
        char *out = static_cast<char *>(tab) + off[i];
        if (KC == 2) bp_table_kernel<2><<<grid, 256, 0, st>>>(gd, g->voff[i], nv, TP, nent, out);
        else bp_table_kernel<4><<<grid, 256, 0, st>>>(gd, g->voff[i], nv, TP, nent, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFree(tab);
            return cuda_fail(e, "bp_table_kernel launch");
        }
    }
    g->d_bptab = tab;                                // set together with the offsets
    g->bptab_off = off;
    return PET_OK;
}

// Pixel tiles per virtual block: each virtual block ends in a block reduction and a grid-wide
// ticket, so the tiles are grouped into one wave of virtual blocks over the resident block
// slots (and never more virtual blocks than the reducer has partial sums for).
void update_shape(UpdateArgs &a, int arith)
{
    const int TP = 256 / a.g.NG;
    const int ntiles = (a.g.N * a.g.N + TP - 1) / TP;
    const int sub = a.g.table, tof = a.g.T > 1;
    const void *fn = a.g.G == 1 ? (a.g.K <= 2 ? update_fn<1, 2>(arith, 0, sub, tof) : update_fn<1, 4>(arith, 0, sub, tof))
                                : (a.g.K <= 2 ? update_fn<8, 2>(arith, a.z3 || a.tv || a.vox, sub, tof)
                                              : update_fn<8, 4>(arith, a.z3 || a.tv || a.vox, sub, tof));
    const int slots = sm_count() * resident_blocks(fn);
    a.tpv = std::max({1, (ntiles + a.red.capacity - 1) / a.red.capacity, (ntiles + slots - 1) / slots});
    a.nvb = (ntiles + a.tpv - 1) / a.tpv;
}

// items per thread: at most ~4 virtual blocks per SM (each ends in a block reduction) and never
// more virtual blocks than reduction slots
void image_shape(ImageArgs &a)
{
    const long long items = (long long)a.g.N * a.g.N * a.g.NG;
    const long long nblk = (items + 255) / 256;
    const int cap = a.red.capacity > 0 ? a.red.capacity : (1 << 30);
    const long long target = (long long)sm_count() * 4;
    a.ipt = (int)std::max<long long>({1, (nblk + cap - 1) / cap, (nblk + target - 1) / target});
    a.nvb = (int)((nblk + a.ipt - 1) / a.ipt);
}

static int persistent_grid(int nvb) { return std::max(1, std::min(nvb, sm_count() * 8)); }

template <int G, int KC>
static void update_dispatch(const UpdateArgs &a, const Batch &b, int arith, int grid, cudaStream_t st)
{
    if (a.g.T > 1 && a.g.table) {                // TOF on ring-sampled bins: KC = 4
        if (arith == AR_FP32) update_kernel<G, 4, AR_FP32, true, true><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_KAHAN) update_kernel<G, 4, AR_KAHAN, true, true><<<grid, 256, 0, st>>>(a, b);
        else update_kernel<G, 4, AR_FP64, true, true><<<grid, 256, 0, st>>>(a, b);
        return;
    }
    if (a.g.T > 1) {                             // TOF geometries: generic kernel
        if (arith == AR_FP32) update_kernel<G, KC, AR_FP32, false, true><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_KAHAN) update_kernel<G, KC, AR_KAHAN, false, true><<<grid, 256, 0, st>>>(a, b);
        else update_kernel<G, KC, AR_FP64, false, true><<<grid, 256, 0, st>>>(a, b);
        return;
    }
    if (a.g.table) {                             // sub-ray / ring geometries: KC = 4, generic kernel
        if (arith == AR_FP32) update_kernel<G, 4, AR_FP32, true><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_KAHAN) update_kernel<G, 4, AR_KAHAN, true><<<grid, 256, 0, st>>>(a, b);
        else update_kernel<G, 4, AR_FP64, true><<<grid, 256, 0, st>>>(a, b);
        return;
    }
    if constexpr (G == 8) {
        // the packed kernel has the in-plane RDP step and p per pixel only; the 3-D prior, the
        // TV variant and scans with detection factors (p per voxel) run the generic kernel
        const bool gen = a.z3 || a.tv || a.vox;
        if (gen && arith == AR_FP32) update_kernel<G, KC, AR_FP32><<<grid, 256, 0, st>>>(a, b);
        else if (gen && arith == AR_KAHAN) update_kernel<G, KC, AR_KAHAN><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_FP32) update_kernel_x8<KC, AR_FP32><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_KAHAN) update_kernel_x8<KC, AR_KAHAN><<<grid, 256, 0, st>>>(a, b);
        else update_kernel<G, KC, AR_FP64><<<grid, 256, 0, st>>>(a, b);
    } else {
        if (arith == AR_FP32) update_kernel<G, KC, AR_FP32><<<grid, 256, 0, st>>>(a, b);
        else if (arith == AR_KAHAN) update_kernel<G, KC, AR_KAHAN><<<grid, 256, 0, st>>>(a, b);
        else update_kernel<G, KC, AR_FP64><<<grid, 256, 0, st>>>(a, b);
    }
}

static pet_status update_any(const UpdateArgs &a, const Batch &b, int arith, int grid, cudaStream_t st)
{
    LaunchScope ls(PET_K_UPDATE, st);
    if (a.g.G == 1) {
        if (a.g.K <= 2) update_dispatch<1, 2>(a, b, arith, grid, st);
        else update_dispatch<1, 4>(a, b, arith, grid, st);
    } else {
        if (a.g.K <= 2) update_dispatch<8, 2>(a, b, arith, grid, st);
        else update_dispatch<8, 4>(a, b, arith, grid, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "update_kernel launch");
    return PET_OK;
}

pet_status launch_update(const UpdateArgs &a0, int arith, cudaStream_t st)
{
    UpdateArgs a = a0;
    update_shape(a, arith);
    update_fp32_scalars(a);
    return update_any(a, Batch{nullptr, nullptr, 0, 0}, arith, persistent_grid(a.nvb), st);
}

pet_status launch_update_batch(const UpdateArgs &shape, const Batch &b, int arith, cudaStream_t st)
{
    return update_any(shape, b, arith, b.grid, st);
}

template <int G, int KC>
static void back_dispatch(const BackArgs &a, int arith, int grid, cudaStream_t st)
{
    if (a.g.T > 1 && a.g.table) {
        if (arith == AR_FP32) back_kernel<G, 4, AR_FP32, true, true><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) back_kernel<G, 4, AR_KAHAN, true, true><<<grid, 256, 0, st>>>(a);
        else back_kernel<G, 4, AR_FP64, true, true><<<grid, 256, 0, st>>>(a);
        return;
    }
    if (a.g.T > 1) {
        if (arith == AR_FP32) back_kernel<G, KC, AR_FP32, false, true><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) back_kernel<G, KC, AR_KAHAN, false, true><<<grid, 256, 0, st>>>(a);
        else back_kernel<G, KC, AR_FP64, false, true><<<grid, 256, 0, st>>>(a);
        return;
    }
    if (a.g.table) {
        if (arith == AR_FP32) back_kernel<G, 4, AR_FP32, true><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) back_kernel<G, 4, AR_KAHAN, true><<<grid, 256, 0, st>>>(a);
        else back_kernel<G, 4, AR_FP64, true><<<grid, 256, 0, st>>>(a);
        return;
    }
    if (arith == AR_FP32) back_kernel<G, KC, AR_FP32><<<grid, 256, 0, st>>>(a);
    else if (arith == AR_KAHAN) back_kernel<G, KC, AR_KAHAN><<<grid, 256, 0, st>>>(a);
    else back_kernel<G, KC, AR_FP64><<<grid, 256, 0, st>>>(a);
}

pet_status launch_back(const BackArgs &a, int arith, cudaStream_t st)
{
    const int TP = 256 / a.g.NG;
    const int ntiles = (a.g.N * a.g.N + TP - 1) / TP;
    const int grid = persistent_grid(ntiles);
    LaunchScope ls(PET_K_OTHER, st);
    if (a.g.G == 1) {
        if (a.g.K <= 2) back_dispatch<1, 2>(a, arith, grid, st);
        else back_dispatch<1, 4>(a, arith, grid, st);
    } else {
        if (a.g.K <= 2) back_dispatch<8, 2>(a, arith, grid, st);
        else back_dispatch<8, 4>(a, arith, grid, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "back_kernel launch");
    return PET_OK;
}

template <int KIND>
static pet_status image_any(const ImageArgs &a, const Batch &b, int arith, int grid, cudaStream_t st)
{
    LaunchScope ls(KIND == 1 ? PET_K_MU_SUM : (KIND == 4 ? PET_K_RDP_VALUE : PET_K_OTHER), st);
    // FP32 and Kahan modes share the FP32 image arithmetic
    if (a.g.G == 1) {
        if (arith == AR_FP64) image_kernel<1, AR_FP64, KIND><<<grid, 256, 0, st>>>(a, b);
        else image_kernel<1, AR_FP32, KIND><<<grid, 256, 0, st>>>(a, b);
    } else {
        if (arith == AR_FP64) image_kernel<8, AR_FP64, KIND><<<grid, 256, 0, st>>>(a, b);
        else image_kernel<8, AR_FP32, KIND><<<grid, 256, 0, st>>>(a, b);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "image_kernel launch");
    return PET_OK;
}

template <int KIND>
static pet_status launch_image(const ImageArgs &a0, int arith, cudaStream_t st)
{
    ImageArgs a = a0;
    image_shape(a);
    return image_any<KIND>(a, Batch{nullptr, nullptr, 0, 0}, arith, persistent_grid(a.nvb), st);
}

pet_status launch_sum(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<0>(a, arith, st); }
// Shape of the mu pass: the packed kernel (8-plane groups, FP32) takes a.ipt pixel tiles per
// virtual block, one wave of virtual blocks over the resident block slots; otherwise the
// items-per-thread shape of image_kernel.
void mu_shape(ImageArgs &a, int arith)
{
    if (a.g.G != 8 || arith == AR_FP64 || a.z3) {
        image_shape(a);
        return;
    }
    const int TP = 256 / a.g.NG;
    const int ntiles = (a.g.N * a.g.N + TP - 1) / TP;
    const int slots = sm_count() * resident_blocks((const void *)mu_kernel_x8);
    const int cap = a.red.capacity > 0 ? a.red.capacity : (1 << 30);
    a.ipt = std::max({1, (ntiles + cap - 1) / cap, (ntiles + slots - 1) / slots});
    a.nvb = (ntiles + a.ipt - 1) / a.ipt;
}

static pet_status mu_any(const ImageArgs &a, const Batch &b, int arith, int grid, cudaStream_t st)
{
    if (a.g.G != 8 || arith == AR_FP64 || a.z3) return image_any<1>(a, b, arith, grid, st);
    LaunchScope ls(PET_K_MU_SUM, st);
    mu_kernel_x8<<<grid, 256, 0, st>>>(a, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mu_kernel_x8 launch");
    return PET_OK;
}

pet_status launch_mu_sum(const ImageArgs &a0, int arith, cudaStream_t st)
{
    ImageArgs a = a0;
    mu_shape(a, arith);
    return mu_any(a, Batch{nullptr, nullptr, 0, 0}, arith, persistent_grid(a.nvb), st);
}
pet_status launch_nu_map(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<2>(a, arith, st); }
pet_status launch_rdp_grad(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<3>(a, arith, st); }
pet_status launch_rdp_value(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<4>(a, arith, st); }
pet_status launch_mu_sum_batch(const ImageArgs &shape, const Batch &b, int arith, cudaStream_t st)
{
    return mu_any(shape, b, arith, b.grid, st);
}
pet_status launch_rdp_value_batch(const ImageArgs &shape, const Batch &b, int arith, cudaStream_t st)
{
    return image_any<4>(shape, b, arith, b.grid, st);
}

}  // namespace pet
