// Image-space kernels of one SDP-BSREM subiteration (Table I):
//   - the fused update: gather backprojection b = A_i^T w, RDP gradient (Eq. gradRD, 8-point
//     in-plane neighbourhood), the smoothness map nu (Sec. III, Eq. nuki), the preconditioner
//     S (Eq. preconditioner) and the clamp P_t (Eq. OperatorPt), with the FP64 sum of the new
//     iterate in the epilogue;
//   - the mu reduction that feeds mean(mu), the plain sum behind mean(f), and the stand-alone
//     RDP value / gradient and nu maps.
// One thread handles one pixel and one group of G planes; neighbours come through L1.
#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

// Loads the 3x3 in-plane neighbourhood of pixel (ix, iy) for one plane group and returns
// the RDP gradient sum, the RDP value and the Matlab-style gradient magnitude as requested.
//   RG: gr_p = 2 sum_k (f_j - f_k)(gamma_R |f_j - f_k| + f_j + 3 f_k + 2 eps) / den^2
//   RV: rv  += sum_k (f_j - f_k)^2 / den             (den = f_j + f_k + gamma_R|f_j-f_k| + eps)
//   MU: gm_p = sqrt(gx^2 + gy^2), central differences inside, one-sided at the edges
template <int G, int AR, bool RG, bool RV, bool MU>
__device__ __forceinline__ void stencil(const GeoDev &g, const typename ArithT<AR>::T *f, int grp,
                                        int ix, int iy, typename ArithT<AR>::T gamma_r,
                                        typename ArithT<AR>::T eps,
                                        typename ArithT<AR>::T (&fc)[G],
                                        typename ArithT<AR>::T (&gr)[G],
                                        typename ArithT<AR>::T (&gm)[G], double &rv)
{
    using T = typename ArithT<AR>::T;
    const int N = g.N, Pp = g.Pp;
    const T *base = f + (size_t)grp * G;
    load_group<G, T>(base + ((size_t)iy * N + ix) * Pp, fc);
    T xl[G], xr[G], yd[G], yu[G];
#pragma unroll
    for (int p = 0; p < G; ++p) {
        gr[p] = T(0);
        xl[p] = xr[p] = yd[p] = yu[p] = fc[p];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        if (q == 4) continue;
        const int dx = q % 3 - 1, dy = q / 3 - 1;
        const int x = ix + dx, y = iy + dy;
        if (x < 0 || y < 0 || x >= N || y >= N) continue;
        T fk[G];
        load_group<G, T>(base + ((size_t)y * N + x) * Pp, fk);
        if constexpr (RG || RV) {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                const T d = fc[p] - fk[p];
                const T ad = d < T(0) ? -d : d;
                const T den = fc[p] + fk[p] + gamma_r * ad + eps;
                if constexpr (RG) gr[p] += d * (gamma_r * ad + fc[p] + T(3) * fk[p] + T(2) * eps) / (den * den);
                if constexpr (RV) {
                    if (grp * G + p < g.P) rv += (double)(d * d / den);
                }
            }
        }
        if constexpr (MU) {
            if (dy == 0 && dx == -1) {
#pragma unroll
                for (int p = 0; p < G; ++p) xl[p] = fk[p];
            } else if (dy == 0 && dx == 1) {
#pragma unroll
                for (int p = 0; p < G; ++p) xr[p] = fk[p];
            } else if (dx == 0 && dy == -1) {
#pragma unroll
                for (int p = 0; p < G; ++p) yd[p] = fk[p];
            } else if (dx == 0 && dy == 1) {
#pragma unroll
                for (int p = 0; p < G; ++p) yu[p] = fk[p];
            }
        }
    }
#pragma unroll
    for (int p = 0; p < G; ++p) {
        if constexpr (RG) gr[p] *= T(2);
        if constexpr (MU) {
            // interior: (f[+1] - f[-1]) / 2; edges: one-sided (the missing side equals fc)
            const T hx = (ix > 0 && ix < N - 1) ? T(0.5) : T(1);
            const T hy = (iy > 0 && iy < N - 1) ? T(0.5) : T(1);
            const T gx = (xr[p] - xl[p]) * hx, gy = (yu[p] - yd[p]) * hy;
            gm[p] = sqrt(gx * gx + gy * gy);
        }
    }
}

template <typename T>
__device__ __forceinline__ T clampT(T v, T lo, T hi) { return v < lo ? lo : (v > hi ? hi : v); }

// f^{k,i} = P_t(f - lambda_k alpha_{k,i} nu S(f) (A_i^T w + (beta/M) grad R(f)))
template <int G, int AR>
__global__ void __launch_bounds__(256) update_kernel(UpdateArgs a)
{
    using T = typename ArithT<AR>::T;
    const GeoDev &g = a.g;
    const int N = g.N, NG = g.NG, Pp = g.Pp;
    const long long total = (long long)N * N * NG;
    const double q = (double)N * N * g.P;
    const T mean_f = a.nu_mode == 1 || a.nu_mode == 2 ? (T)(*a.sum_f / q) : T(1);
    const T mean_mu = a.nu_mode == 1 || a.nu_mode == 2 ? (T)(*a.sum_mu / q) : T(1);
    const T lam = (T)a.lam_alpha, bm = (T)a.beta_over_M, U = (T)a.U, tt = (T)a.t;
    const T nu1 = (T)a.nu1, nu2 = (T)a.nu2, halfU = T(0.5) * U;
    const T *w = reinterpret_cast<const T *>(a.w);
    const T *f = reinterpret_cast<const T *>(a.f);
    const T *invp = reinterpret_cast<const T *>(a.invp);
    double s = 0.0;
    for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < total;
         tid += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(tid % NG);
        const int j = (int)(tid / NG);
        const int ix = j % N, iy = j / N;
        GroupSum<G, AR> bp;
        bp.zero();
        gather_bp<G, AR>(g, a.slot0, a.nviews, w, grp, ix, iy, bp);
        T fc[G], gr[G], gm[G];
        if (a.nu_mode == 1 || a.nu_mode == 2)
            stencil<G, AR, true, false, true>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gm, s);
        else
            stencil<G, AR, true, false, false>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gm, s);
        T nu[G];
        if (a.nu_mode == 3) {
            load_group<G, T>(reinterpret_cast<const T *>(a.nu_frozen) + (size_t)j * Pp + (size_t)grp * G, nu);
        } else if (a.nu_mode == 0) {
#pragma unroll
            for (int p = 0; p < G; ++p) nu[p] = T(1);
        } else {
#pragma unroll
            for (int p = 0; p < G; ++p) {
                T mu = gm[p] / mean_f;
                mu = mu < T(0.01) ? T(0.01) : mu;
                nu[p] = clampT<T>(mean_mu / mu, nu1, nu2);
            }
            if (a.nu_mode == 2)
                store_group<G, T>(reinterpret_cast<T *>(a.nu_frozen) + (size_t)j * Pp + (size_t)grp * G, nu);
        }
        const T ip = invp[j];
        const T scale = (T)g.scale;
        T out[G];
#pragma unroll
        for (int p = 0; p < G; ++p) {
            const T fj = fc[p];
            const T d = scale * bp.value(p) + bm * gr[p];
            const T S = (fj < halfU ? fj : U - fj) * ip;
            T ft = fj - lam * nu[p] * S * d;
            ft = ft <= T(0) ? tt : (ft >= U ? U - tt : ft);
            const bool valid = grp * G + p < g.P;
            out[p] = valid ? ft : T(0);
            if (valid) s += (double)ft;
        }
        store_group<G, T>(reinterpret_cast<T *>(a.fout) + (size_t)j * Pp + (size_t)grp * G, out);
    }
    double v[1] = {s};
    grid_reduce<1>(v, a.red, a.sum_fout);
}

// KIND 0: sum f; 1: sum mu; 2: nu map; 3: RDP gradient; 4: RDP value
template <int G, int AR, int KIND>
__global__ void __launch_bounds__(256) image_kernel(ImageArgs a)
{
    using T = typename ArithT<AR>::T;
    const GeoDev &g = a.g;
    const int N = g.N, NG = g.NG, Pp = g.Pp;
    const long long total = (long long)N * N * NG;
    const double q = (double)N * N * g.P;
    const T *f = reinterpret_cast<const T *>(a.f);
    const T mean_f = (KIND == 1 || KIND == 2) ? (T)(*a.sum_f / q) : T(1);
    const T mean_mu = KIND == 2 ? (T)(*a.sum_mu / q) : T(1);
    double s = 0.0;
    for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < total;
         tid += (long long)gridDim.x * blockDim.x) {
        const int grp = (int)(tid % NG);
        const int j = (int)(tid / NG);
        const int ix = j % N, iy = j / N;
        T fc[G], gr[G], gm[G], out[G];
        if constexpr (KIND == 0) {
            load_group<G, T>(f + (size_t)j * Pp + (size_t)grp * G, fc);
#pragma unroll
            for (int p = 0; p < G; ++p)
                if (grp * G + p < g.P) s += (double)fc[p];
        } else if constexpr (KIND == 1 || KIND == 2) {
            stencil<G, AR, false, false, true>(g, f, grp, ix, iy, T(0), T(0), fc, gr, gm, s);
#pragma unroll
            for (int p = 0; p < G; ++p) {
                T mu = gm[p] / mean_f;
                mu = mu < T(0.01) ? T(0.01) : mu;
                if constexpr (KIND == 1) {
                    if (grp * G + p < g.P) s += (double)mu;
                } else {
                    out[p] = grp * G + p < g.P ? clampT<T>(mean_mu / mu, (T)a.nu1, (T)a.nu2) : T(0);
                }
            }
            if constexpr (KIND == 2)
                store_group<G, T>(reinterpret_cast<T *>(a.out) + (size_t)j * Pp + (size_t)grp * G, out);
        } else if constexpr (KIND == 3) {
            stencil<G, AR, true, false, false>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gm, s);
#pragma unroll
            for (int p = 0; p < G; ++p) out[p] = grp * G + p < g.P ? gr[p] : T(0);
            store_group<G, T>(reinterpret_cast<T *>(a.out) + (size_t)j * Pp + (size_t)grp * G, out);
        } else {
            stencil<G, AR, false, true, false>(g, f, grp, ix, iy, (T)a.gamma_r, (T)a.eps, fc, gr, gm, s);
        }
    }
    if constexpr (KIND == 0 || KIND == 1 || KIND == 4) {
        double v[1] = {s};
        grid_reduce<1>(v, a.red, a.result);
    }
}

static int reduce_grid(const GeoDev &g, int capacity)
{
    const long long total = (long long)g.N * g.N * g.NG;
    long long grid = (total + 255) / 256;
    if (grid > capacity) grid = capacity;
    return (int)grid;
}

pet_status launch_update(const UpdateArgs &a, int arith, cudaStream_t st)
{
    const int grid = reduce_grid(a.g, a.red.capacity);
    LaunchScope ls(PET_K_UPDATE, st);
    if (a.g.G == 1) {
        if (arith == AR_FP32) update_kernel<1, AR_FP32><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) update_kernel<1, AR_KAHAN><<<grid, 256, 0, st>>>(a);
        else update_kernel<1, AR_FP64><<<grid, 256, 0, st>>>(a);
    } else {
        if (arith == AR_FP32) update_kernel<8, AR_FP32><<<grid, 256, 0, st>>>(a);
        else if (arith == AR_KAHAN) update_kernel<8, AR_KAHAN><<<grid, 256, 0, st>>>(a);
        else update_kernel<8, AR_FP64><<<grid, 256, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "update_kernel launch");
    return PET_OK;
}

template <int KIND>
static pet_status launch_image(const ImageArgs &a, int arith, cudaStream_t st)
{
    const int grid = reduce_grid(a.g, a.red.capacity > 0 ? a.red.capacity : (1 << 30));
    LaunchScope ls(KIND == 1 ? PET_K_MU_SUM : (KIND == 4 ? PET_K_RDP_VALUE : PET_K_OTHER), st);
    // FP32 and Kahan modes share the FP32 image arithmetic
    if (a.g.G == 1) {
        if (arith == AR_FP64) image_kernel<1, AR_FP64, KIND><<<grid, 256, 0, st>>>(a);
        else image_kernel<1, AR_FP32, KIND><<<grid, 256, 0, st>>>(a);
    } else {
        if (arith == AR_FP64) image_kernel<8, AR_FP64, KIND><<<grid, 256, 0, st>>>(a);
        else image_kernel<8, AR_FP32, KIND><<<grid, 256, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "image_kernel launch");
    return PET_OK;
}

pet_status launch_sum(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<0>(a, arith, st); }
pet_status launch_mu_sum(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<1>(a, arith, st); }
pet_status launch_nu_map(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<2>(a, arith, st); }
pet_status launch_rdp_grad(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<3>(a, arith, st); }
pet_status launch_rdp_value(const ImageArgs &a, int arith, cudaStream_t st) { return launch_image<4>(a, arith, st); }

}  // namespace pet
