// Ray-driven Siddon forward projector (with the Poisson-ratio and objective epilogues) and the
// pixel-driven gather backprojector.
//
// Forward (Sec. II-B, y = A_i f; App. A, w = 1 - g_i / (A_i f + gamma_i)): one thread walks one
// ray for one group of G planes (planes innermost in memory, so one walk serves G planes and
// each pixel fetch is one 32-byte sector for G = 8).  The ray is walked one pixel column (or
// row) at a time along its driving axis, the axis it advances fastest along: inside one such
// step the line meets at most two pixels of the cross axis, and their exact intersection
// lengths are l1 = frac(hi) / minor and l0 = L - l1, which is Siddon's length set computed in
// a fixed-trip loop without a merge.  The cross coordinate is stepped exactly in Q32.32 fixed
// point (FP32 kernels) so positions keep 32 fractional bits at any image size.
#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

template <int G, int AR, int MODE>
__global__ void __launch_bounds__(256) fwd_kernel(FwdArgs a)
{
    using T = typename ArithT<AR>::T;
    const GeoDev &g = a.g;
    const int NG = g.NG, NB = g.NB, N = g.N, Pp = g.Pp;
    const long long total = (long long)a.nviews * NB * NG;
    double obj[2] = {0.0, 0.0};
    for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < total;
         tid += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(tid % NG);
        const int ray = (int)(tid / NG);          // subset-local ray index u * NB + b
        const int slot = a.slot0 + ray / NB;
        const ViewGeo &vw = g.views[slot];
        const RayGeo &rg = g.rays[(size_t)a.slot0 * NB + ray];
        const int ds = vw.xdrive ? 1 : N;         // pixel stride along the driving axis
        const int cs = vw.xdrive ? N : 1;         // pixel stride along the cross axis
        const T *img = reinterpret_cast<const T *>(a.img) + (size_t)grp * G;
        GroupSum<G, AR> acc;
        acc.zero();
        const int nd = rg.nd;
        if constexpr (AR == AR_FP64) {
            const double step = vw.step, ast = fabs(vw.step), L = vw.L, im = vw.inv_minor;
            for (int k = 0; k < nd; ++k) {
                const int d = rg.d0 + k;
                const double lo = fma((double)k, step, rg.lo);
                const double hi = lo + ast;
                const double f0 = floor(lo), f1 = floor(hi);
                const int r0 = (int)f0, r1 = (int)f1;
                double l1 = (r1 != r0) ? (hi - f1) * im : 0.0;
                double l0 = L - l1;
                const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                l0 = ok0 ? l0 : 0.0;
                l1 = ok1 ? l1 : 0.0;
                const int c0 = ok0 ? r0 : 0, c1 = ok1 ? r1 : 0;
                T x0[G], x1[G];
                load_group<G, T>(img + (size_t)(d * ds + c0 * cs) * Pp, x0);
                load_group<G, T>(img + (size_t)(d * ds + c1 * cs) * Pp, x1);
                acc.add2terms(l0, x0, l1, x1);
            }
        } else {
            const long long stp = vw.stepq, ast = vw.absstepq;
            const float L = vw.Lf, im = vw.inv_minorf * kQ32;
            long long lo = rg.loq;
            for (int k = 0; k < nd; ++k) {
                const int d = rg.d0 + k;
                const long long hi = lo + ast;
                const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
                float l1 = (r1 != r0) ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f;
                float l0 = L - l1;
                const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                l0 = ok0 ? l0 : 0.f;
                l1 = ok1 ? l1 : 0.f;
                const int c0 = ok0 ? r0 : 0, c1 = ok1 ? r1 : 0;
                T x0[G], x1[G];
                load_group<G, T>(img + (size_t)(d * ds + c0 * cs) * Pp, x0);
                load_group<G, T>(img + (size_t)(d * ds + c1 * cs) * Pp, x1);
                acc.add2terms(l0, x0, l1, x1);
                lo += stp;
            }
        }
        const size_t o = (size_t)ray * Pp + (size_t)grp * G;
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
            if constexpr (MODE == FWD_RATIO) {
                T w[G];
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    const T y = scale * acc.value(p) + (T)gam[p];
                    w[p] = (grp * G + p < g.P) ? T(1) - (T)cnt[p] / y : T(0);
                }
                store_group<G, T>(reinterpret_cast<T *>(a.out) + o, w);
            } else {
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    if (grp * G + p < g.P) {
                        const T af = scale * acc.value(p);
                        obj[0] += (double)af;
                        if (cnt[p] != 0) obj[1] += (double)cnt[p] * (double)log(af + (T)gam[p]);
                    }
                }
            }
        }
    }
    if constexpr (MODE == FWD_OBJECTIVE) grid_reduce<2>(obj, a.red, a.result);
}

// Pixel-driven gather backprojection: one thread per (pixel, plane group).
template <int G, int AR>
__global__ void __launch_bounds__(256) back_kernel(BackArgs a)
{
    using T = typename ArithT<AR>::T;
    const GeoDev &g = a.g;
    const int NG = g.NG, N = g.N;
    const long long total = (long long)N * N * NG;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= total) return;
    const int grp = (int)(tid % NG);
    const int j = (int)(tid / NG);
    const int ix = j % N, iy = j / N;
    GroupSum<G, AR> acc;
    acc.zero();
    gather_bp<G, AR>(g, a.slot0, a.nviews, reinterpret_cast<const T *>(a.proj), grp, ix, iy, acc);
    T b[G];
    const T scale = (T)g.scale;
#pragma unroll
    for (int p = 0; p < G; ++p) b[p] = (grp * G + p < g.P) ? scale * acc.value(p) : T(0);
    store_group<G, T>(reinterpret_cast<T *>(a.img) + (size_t)j * g.Pp + (size_t)grp * G, b);
}

template <int G, int AR>
static void fwd_dispatch_mode(const FwdArgs &a, int mode, int grid, cudaStream_t st)
{
    if (mode == FWD_PLAIN) fwd_kernel<G, AR, FWD_PLAIN><<<grid, 256, 0, st>>>(a);
    else if (mode == FWD_RATIO) fwd_kernel<G, AR, FWD_RATIO><<<grid, 256, 0, st>>>(a);
    else fwd_kernel<G, AR, FWD_OBJECTIVE><<<grid, 256, 0, st>>>(a);
}

template <int G>
static void fwd_dispatch(const FwdArgs &a, int mode, int arith, int grid, cudaStream_t st)
{
    if (arith == AR_FP32) fwd_dispatch_mode<G, AR_FP32>(a, mode, grid, st);
    else if (arith == AR_KAHAN) fwd_dispatch_mode<G, AR_KAHAN>(a, mode, grid, st);
    else fwd_dispatch_mode<G, AR_FP64>(a, mode, grid, st);
}

pet_status launch_forward(const FwdArgs &a, int mode, int arith, cudaStream_t st)
{
    const long long total = (long long)a.nviews * a.g.NB * a.g.NG;
    if (total == 0) return PET_OK;
    long long grid = (total + 255) / 256;
    if (mode == FWD_OBJECTIVE && grid > a.red.capacity) grid = a.red.capacity;
    LaunchScope ls(mode == FWD_RATIO ? PET_K_FORWARD_RATIO
                   : (mode == FWD_OBJECTIVE ? PET_K_OBJ_FORWARD : PET_K_OTHER), st);
    if (a.g.G == 1) fwd_dispatch<1>(a, mode, arith, (int)grid, st);
    else fwd_dispatch<8>(a, mode, arith, (int)grid, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fwd_kernel launch");
    return PET_OK;
}

pet_status launch_back(const BackArgs &a, int arith, cudaStream_t st)
{
    const long long total = (long long)a.g.N * a.g.N * a.g.NG;
    const int grid = (int)((total + 255) / 256);
    LaunchScope ls(PET_K_OTHER, st);
    if (a.g.G == 1) {
        if (arith == AR_FP32) back_kernel<1, AR_FP32><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) back_kernel<1, AR_KAHAN><<<grid, 256, 0, st>>>(a);
        else back_kernel<1, AR_FP64><<<grid, 256, 0, st>>>(a);
    } else {
        if (arith == AR_FP32) back_kernel<8, AR_FP32><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) back_kernel<8, AR_KAHAN><<<grid, 256, 0, st>>>(a);
        else back_kernel<8, AR_FP64><<<grid, 256, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "back_kernel launch");
    return PET_OK;
}

}  // namespace pet
