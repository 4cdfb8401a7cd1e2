// Time-of-flight forward projector (the TOF data of the clinical reconstructions, Sec. IV-C):
// y_(i,t) = sum_j A_ij h_t(tau_j) f_j, A_ij the one-line Siddon lengths of bin i = (v, b),
// h_t the Gaussian timing kernel integrated over TOF bin t at the position tau_j of pixel j's
// centre along the line.  One thread walks one (ray, TOF bin, plane group) over the part of
// the ray where h_t can be non-zero (|tau - tau_t| <= the kernel's window), with the same
// column-by-column walk and exact lengths as the non-TOF projector, each length weighted by h_t
// at its pixel's centre.  Epilogues as in fwd_kernel: plain, ratio (with the per-bin detection
// factors), or the objective's FP64 sums.  Outputs are [nviews][NB][T][Pp].  One scan, or a batch
// of TOF scans (per-scan arguments and virtual blocks, as in fwd_kernel).
#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

// FP32 kernels take h_t from a table of h(u) = h_t(c_t + u) (the kernel relative to the TOF
// bin's centre c_t, the same for every bin) over the window |u| <= W: values and derivatives at
// TAB nodes, cubic Hermite interpolation in between (error below 1e-7 of the peak for the node
// spacing of at most sigma / 16; the table is built per block with the tail-mass form of h).
constexpr int TOF_TAB = 2048;

template <int G, int AR, int MODE>
__global__ void __launch_bounds__(256) tof_fwd_kernel(const __grid_constant__ FwdArgs one,
                                                      const Batch bt)
{
    using T = typename ArithT<AR>::T;
    constexpr bool D = AR == AR_FP64;
    __shared__ float2 tab[D ? 1 : TOF_TAB];
    __shared__ float tab_key[3];                       // the TOF kernel the table holds
    __shared__ FwdArgs sh_args;
    if (threadIdx.x == 0) tab_key[0] = tab_key[1] = tab_key[2] = -1.f;
    __syncthreads();
    const int total = total_vblocks(one, bt);
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const FwdArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int NG = g.NG, NB = g.NB, N = g.N, Pp = g.Pp, TT = g.T;
        const long long items = (long long)a.nviews * NB * TT * NG;
        const T d = D ? (T)g.tof_d : (T)g.tof_df, kk = D ? (T)g.tof_k : (T)g.tof_kf;
        const T W = (D ? (T)g.tof_w : (T)g.tof_wf) + T(1);   // + 1: pixel centres vs the line
        const float Wt = g.tof_wf, dt_ = (2.f * Wt) / (float)(TOF_TAB - 1), idt = 1.f / dt_;
        if constexpr (!D) {
            // (re)build the table when this scan's kernel differs from the one it holds
            // (block-uniform: every thread reads the same arguments)
            if (tab_key[0] != g.tof_df || tab_key[1] != g.tof_kf || tab_key[2] != g.tof_wf) {
                __syncthreads();
                const float k = g.tof_kf, hd = 0.5f * g.tof_df;
                const float dphi = 1.1283791670955126f * k;   // 2 k / sqrt(pi)
                for (int i = threadIdx.x; i < TOF_TAB; i += blockDim.x) {
                    const float u = -Wt + (float)i * dt_;
                    const float z0 = (-hd - u) * k, z1 = (hd - u) * k;
                    // h(u) = Phi(sqrt2 z1) - Phi(sqrt2 z0); h'(u) = k / sqrt(pi) (e^{-z0^2} - e^{-z1^2})
                    tab[i] = make_float2(tof_h<float>(z0, z1),
                                         0.5f * dphi * (expf(-z0 * z0) - expf(-z1 * z1)));
                }
                __syncthreads();
                if (threadIdx.x == 0) { tab_key[0] = g.tof_df; tab_key[1] = g.tof_kf; tab_key[2] = g.tof_wf; }
                __syncthreads();
            }
        }
        double obj[2] = {0.0, 0.0};
        for (int k = 0; k < a.tpv; ++k) {
            const long long it = ((long long)vloc * a.tpv + k) * 256 + threadIdx.x;
            if (it >= items) continue;
            const int grp = (int)(it % NG);
            const long long rt = it / NG;
            const int t = (int)(rt % TT);
            const int ray = (int)(rt / TT);              // subset-local u * NB + b
            const int slot = a.slot0 + ray / NB, b = ray % NB;
            const ViewGeo &vw = g.views[slot];
            const RayGeo &rg = g.rays[(size_t)a.slot0 * NB + ray];
            // driving columns whose line point lies within the window of TOF bin t
            const T r = g.ring ? (T)g.bins[b].c0
                               : (T)(2 * b - (NB - 1)) * T(0.5) * (D ? (T)g.rho : (T)(float)g.rho);
            const T tauA = D ? (T)vw.tdr * r + (T)vw.tdc : (T)vw.tdrf * r + (T)vw.tdcf;
            const T tdd = D ? (T)vw.tdd : (T)vw.tddf;
            const T ct = (T)(2 * t - (TT - 1)) * T(0.5) * d;
            T lo_d = (ct - W - tauA) / tdd, hi_d = (ct + W - tauA) / tdd;
            if (lo_d > hi_d) { const T x = lo_d; lo_d = hi_d; hi_d = x; }
            const int k0 = max(0, (int)ceil(lo_d) - rg.d0);
            const int k1 = min(rg.nd, (int)floor(hi_d) - rg.d0 + 1);
            const int ds = vw.xdrive ? 1 : N;
            const int cs = vw.xdrive ? N : 1;
            // pixel (d, r) of the walk is (ix, iy) = (d, r) or (r, d)
            const T tpd = D ? (T)(vw.xdrive ? vw.taux : vw.tauy) : (T)(vw.xdrive ? vw.tauxf : vw.tauyf);
            const T tpr = D ? (T)(vw.xdrive ? vw.tauy : vw.taux) : (T)(vw.xdrive ? vw.tauyf : vw.tauxf);
            const T tp0 = D ? (T)vw.tau0 : (T)vw.tau0f;
            const T e0 = (T)(2 * t - TT) * T(0.5) * d;  // lower edge of the TOF bin
            auto hw = [&](int dd, int rr) -> T {
                const T tau = tp0 + (T)dd * tpd + (T)rr * tpr;
                if constexpr (D) {
                    return tof_h<T>((e0 - tau) * kk, (e0 + d - tau) * kk);
                } else {
                    const float x = (tau - ct + Wt) * idt;
                    if (!(x >= 0.f && x < (float)(TOF_TAB - 1))) return 0.f;
                    const int i = (int)x;
                    const float f = x - (float)i;
                    const float2 p0 = tab[i], p1 = tab[i + 1];
                    const float f2 = f * f, f3 = f2 * f;
                    const float h00 = 2.f * f3 - 3.f * f2 + 1.f, h01 = 3.f * f2 - 2.f * f3;
                    const float h10 = f3 - 2.f * f2 + f, h11 = f3 - f2;
                    return h00 * p0.x + h01 * p1.x + dt_ * (h10 * p0.y + h11 * p1.y);
                }
            };
            const T *img = reinterpret_cast<const T *>(a.img) + (size_t)grp * G;
            GroupSum<G, AR> acc;
            acc.zero();
            if constexpr (D) {
                const double step = vw.step, ast = fabs(vw.step), L = vw.L, im = vw.inv_minor;
                for (int kd = k0; kd < k1; ++kd) {
                    const int dd = rg.d0 + kd;
                    const double lo = fma((double)kd, step, rg.lo);
                    const double hi = lo + ast;
                    const double f0 = floor(lo), f1 = floor(hi);
                    const int r0 = (int)f0, r1 = (int)f1;
                    double l1 = (r1 != r0) ? (hi - f1) * im : 0.0;
                    double l0 = L - l1;
                    const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                    l0 = ok0 ? l0 * hw(dd, r0) : 0.0;
                    l1 = (ok1 && l1 > 0.0) ? l1 * hw(dd, r1) : 0.0;
                    T x0[G], x1[G];
                    load_group<G, T>(img + (unsigned)(dd * ds + (ok0 ? r0 : 0) * cs) * (unsigned)Pp, x0);
                    load_group<G, T>(img + (unsigned)(dd * ds + (ok1 ? r1 : 0) * cs) * (unsigned)Pp, x1);
                    acc.add2terms(l0, x0, l1, x1);
                }
            } else {
                const long long stp = vw.stepq, ast = vw.absstepq;
                const float L = vw.Lf, im = vw.inv_minorf * kQ32;
                long long lo = rg.loq + (long long)k0 * stp;
                for (int kd = k0; kd < k1; ++kd) {
                    const int dd = rg.d0 + kd;
                    const long long hi = lo + ast;
                    const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
                    float l1 = (r1 != r0) ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f;
                    float l0 = L - l1;
                    const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                    l0 = ok0 ? l0 * hw(dd, r0) : 0.f;
                    l1 = (ok1 && l1 > 0.f) ? l1 * hw(dd, r1) : 0.f;
                    T x0[G], x1[G];
                    load_group<G, T>(img + (unsigned)(dd * ds + (ok0 ? r0 : 0) * cs) * (unsigned)Pp, x0);
                    load_group<G, T>(img + (unsigned)(dd * ds + (ok1 ? r1 : 0) * cs) * (unsigned)Pp, x1);
                    acc.add2terms(l0, x0, l1, x1);
                    lo += stp;
                }
            }
            const size_t o = ((size_t)ray * TT + t) * Pp + (size_t)grp * G;
            const T scale = (T)g.scale;
            if constexpr (MODE == FWD_PLAIN) {
                T y[G];
#pragma unroll
                for (int p = 0; p < G; ++p) y[p] = scale * acc.value(p);
                store_group<G, T>(reinterpret_cast<T *>(a.out) + o, y);
            } else {
                int cnt[G];
                float gam[G];
                load_group_i<G>(a.counts + o, cnt);
                load_group<G, float>(a.gamma + o, gam);
                const float *mp = a.mult ? a.mult + o : nullptr;
                if constexpr (MODE == FWD_RATIO) {
                    T w[G];
#pragma unroll
                    for (int p = 0; p < G; ++p) {
                        const T m = mp ? (T)__ldg(mp + p) : T(1);
                        const T y = scale * (acc.value(p) * m) + (T)gam[p];
                        w[p] = (grp * G + p < g.P) ? m * (T(1) - (T)cnt[p] / y) : T(0);
                    }
                    store_group<G, T>(reinterpret_cast<T *>(a.out) + o, w);
                } else {
                    T s_af = T(0);
                    double s_gl = 0.0;
#pragma unroll
                    for (int p = 0; p < G; ++p) {
                        if (grp * G + p < g.P) {
                            const T v = acc.value(p);
                            const T af = scale * (mp ? v * (T)__ldg(mp + p) : v);
                            s_af += af;
                            if (cnt[p] != 0) s_gl += (double)cnt[p] * log((double)af + (double)gam[p]);
                        }
                    }
                    obj[0] += (double)s_af;
                    obj[1] += s_gl;
                }
            }
        }
        if constexpr (MODE == FWD_OBJECTIVE) grid_reduce<2>(obj, a.red, a.result, vloc, nv);
    }
}

int sm_count();
int resident_blocks(const void *fn);

template <int G>
static const void *tof_fwd_fn(int mode, int arith)
{
#define PET_TOF_FN(AR)                                                                      \
    (mode == FWD_PLAIN ? (const void *)tof_fwd_kernel<G, AR, FWD_PLAIN>                     \
     : mode == FWD_RATIO ? (const void *)tof_fwd_kernel<G, AR, FWD_RATIO>                   \
                         : (const void *)tof_fwd_kernel<G, AR, FWD_OBJECTIVE>)
    if (arith == AR_FP64) return PET_TOF_FN(AR_FP64);
    if (arith == AR_FP32) return PET_TOF_FN(AR_FP32);
    return PET_TOF_FN(AR_KAHAN);
#undef PET_TOF_FN
}

// 256 (ray, TOF bin, group) items per block; the objective groups blocks into one wave of
// virtual blocks (each ends in a reduction step), never more than its reducer holds.
void forward_shape_tof(FwdArgs &a, int mode, int arith)
{
    const long long items = (long long)a.nviews * a.g.NB * a.g.T * a.g.NG;
    const long long blocks = std::max(1LL, (items + 255) / 256);
    a.S = 1;
    a.R = 1;
    a.tpv = 1;
    if (mode == FWD_OBJECTIVE) {
        const void *fn = a.g.G == 1 ? tof_fwd_fn<1>(mode, arith) : tof_fwd_fn<8>(mode, arith);
        const long long slots = (long long)sm_count() * resident_blocks(fn);
        long long tpv = (blocks + slots - 1) / slots;
        if (a.red.capacity > 0) tpv = std::max(tpv, (blocks + a.red.capacity - 1) / a.red.capacity);
        a.tpv = (int)std::max(1LL, tpv);
    }
    a.nvb = (int)((blocks + a.tpv - 1) / a.tpv);
}

template <int G, int AR>
static void tof_launch_mode(const FwdArgs &a, const Batch &b, int mode, int grid, cudaStream_t st)
{
    if (mode == FWD_PLAIN) tof_fwd_kernel<G, AR, FWD_PLAIN><<<grid, 256, 0, st>>>(a, b);
    else if (mode == FWD_RATIO) tof_fwd_kernel<G, AR, FWD_RATIO><<<grid, 256, 0, st>>>(a, b);
    else tof_fwd_kernel<G, AR, FWD_OBJECTIVE><<<grid, 256, 0, st>>>(a, b);
}

template <int G>
static void tof_launch(const FwdArgs &a, const Batch &b, int mode, int arith, int grid, cudaStream_t st)
{
    if (arith == AR_FP64) tof_launch_mode<G, AR_FP64>(a, b, mode, grid, st);
    else if (arith == AR_FP32) tof_launch_mode<G, AR_FP32>(a, b, mode, grid, st);
    else tof_launch_mode<G, AR_KAHAN>(a, b, mode, grid, st);
}

pet_status launch_forward_tof(const FwdArgs &a0, int mode, int arith, cudaStream_t st)
{
    FwdArgs a = a0;
    if ((long long)a.nviews * a.g.NB == 0) return PET_OK;
    forward_shape_tof(a, mode, arith);
    const int grid = std::max(1, std::min(a.nvb, sm_count() * 8));
    LaunchScope ls(mode == FWD_RATIO ? PET_K_FORWARD_RATIO
                   : (mode == FWD_OBJECTIVE ? PET_K_OBJ_FORWARD : PET_K_OTHER), st);
    const Batch b{nullptr, nullptr, 0, grid};
    if (a.g.G == 1) tof_launch<1>(a, b, mode, arith, grid, st);
    else tof_launch<8>(a, b, mode, arith, grid, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tof_fwd_kernel launch");
    return PET_OK;
}

// Batched launch: every scan of the batch has TOF bins and the plane-group size of `shape`.
pet_status launch_forward_tof_batch(const FwdArgs &shape, const Batch &b, int mode, int arith,
                                    cudaStream_t st)
{
    LaunchScope ls(mode == FWD_RATIO ? PET_K_FORWARD_RATIO
                   : (mode == FWD_OBJECTIVE ? PET_K_OBJ_FORWARD : PET_K_OTHER), st);
    if (shape.g.G == 1) tof_launch<1>(shape, b, mode, arith, b.grid, st);
    else tof_launch<8>(shape, b, mode, arith, b.grid, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tof_fwd_kernel batch launch");
    return PET_OK;
}

}  // namespace pet
