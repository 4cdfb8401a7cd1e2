// TV variant of the regulariser: the proximal step of (beta/M) R_TV in the metric W of the
// subiteration's step sizes, approximated by primal-dual iterations (Chambolle and Pock, J. Math.
// Imaging Vis. 40, 2011) with the diagonal steps of Pock and Chambolle (ICCV 2011) for K = b D:
//   p    <- proj_{|p_j| <= 1}(p + D xbar / 2)                   (sigma = 1 / (2 b))
//   x'    = (x + div(p) / 4 + (tau / W) z) / (1 + tau / W)      (tau = 1 / (4 b))
//   xbar  = 2 x' - x,   x = x'
// from x = xbar = z.  R_TV(f) = sum_j |(D f)_j| with D the in-plane forward differences (zero
// across the last column / row) and div(p)_j = p^x_j - p^x_{j-x} + p^y_j - p^y_{j-y}.  The paper's
// own prior (RDP) is smooth and handled by its gradient; TV is named there only as the typical
// non-smooth prior, and this is how such a prior enters the same preconditioned step.
// Element-parallel kernels over the internal layout [N*N][Pp] (planes innermost, pad planes kept
// at zero); the last primal step applies P_t and reduces the sum of f^{k,i} (FP64, per virtual
// block in order, like every reduction of the library).
#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

int sm_count();

template <typename T>
__global__ void __launch_bounds__(256) tv_dual_kernel(const __grid_constant__ TvArgs a, const T *xb)
{
    const GeoDev &g = a.g;
    const unsigned N = (unsigned)g.N, Pp = (unsigned)g.Pp;
    const unsigned items = N * N * Pp;                       // < 2^32 (geometry limits)
    T *px = reinterpret_cast<T *>(a.px);
    T *py = reinterpret_cast<T *>(a.py);
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const unsigned z = it % Pp, j = it / Pp;
        if ((int)z >= g.P) continue;                          // pad planes: p stays 0
        const unsigned ix = j % N, iy = j / N;
        const T c = xb[it];
        const T gx = ix + 1 < N ? xb[it + Pp] - c : T(0);
        const T gy = iy + 1 < N ? xb[it + N * Pp] - c : T(0);
        const T qx = px[it] + T(0.5) * gx, qy = py[it] + T(0.5) * gy;
        const T nq = sqrt(qx * qx + qy * qy);
        const T sc = nq > T(1) ? T(1) / nq : T(1);
        px[it] = qx * sc;
        py[it] = qy * sc;
    }
}

template <typename T, bool LAST>
__global__ void __launch_bounds__(256) tv_primal_kernel(const __grid_constant__ TvArgs a)
{
    const GeoDev &g = a.g;
    const unsigned N = (unsigned)g.N, Pp = (unsigned)g.Pp;
    const unsigned items = N * N * Pp;
    T *x = reinterpret_cast<T *>(a.x);
    T *xbar = reinterpret_cast<T *>(a.xbar);
    const T *zz = reinterpret_cast<const T *>(a.z);
    const T *w = reinterpret_cast<const T *>(a.w);
    const T *px = reinterpret_cast<const T *>(a.px);
    const T *py = reinterpret_cast<const T *>(a.py);
    const T tau = T(0.25) / (T)a.b, tt = (T)a.t, U = (T)a.U;
    for (int vb = blockIdx.x; vb < a.nvb; vb += gridDim.x) {
        T part = T(0);
        for (int k = 0; k < a.ipt; ++k) {
            const unsigned it = ((unsigned)vb * (unsigned)a.ipt + (unsigned)k) * 256u + threadIdx.x;
            if (it >= items) break;
            const unsigned z = it % Pp, j = it / Pp;
            if ((int)z >= g.P) continue;                      // pad planes stay 0
            const unsigned ix = j % N, iy = j / N;
            const T div = px[it] - (ix > 0 ? px[it - Pp] : T(0)) + py[it] - (iy > 0 ? py[it - N * Pp] : T(0));
            const T xo = x[it];
            T xn = zz[it];                                    // b = 0: the proximal point is z
            if (a.b > 0.0) {
                const T r = tau / w[it];
                xn = (xo + T(0.25) * div + r * zz[it]) / (T(1) + r);
            }
            if constexpr (LAST) {
                // P_t (Eq. OperatorPt); t <= 0 asks for the bare proximal point
                const T f = tt <= T(0) ? xn : (xn <= T(0) ? tt : (xn >= U ? U - tt : xn));
                x[it] = f;
                part += f;
            } else {
                xbar[it] = T(2) * xn - xo;
                x[it] = xn;
            }
        }
        if constexpr (LAST) {
            double v[1] = {(double)part};
            grid_reduce<1>(v, a.red, a.sum_out, vb, a.nvb);
        }
    }
}

// items per thread so that the reduction's virtual blocks fit the reducer and about four of
// them fall on each SM
void tv_shape(TvArgs &a)
{
    const long long items = (long long)a.g.N * a.g.N * a.g.Pp;
    const long long nblk = (items + 255) / 256;
    const int cap = a.red.capacity > 0 ? a.red.capacity : (1 << 30);
    const long long target = (long long)sm_count() * 4;
    a.ipt = (int)std::max<long long>({1, (nblk + cap - 1) / cap, (nblk + target - 1) / target});
    a.nvb = (int)((nblk + a.ipt - 1) / a.ipt);
}

template <typename T>
static pet_status tv_run(const TvArgs &a, int iters, cudaStream_t st)
{
    const long long items = (long long)a.g.N * a.g.N * a.g.Pp;
    const int grid = (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, sm_count() * 8));
    const int pgrid = std::max(1, std::min(a.nvb, sm_count() * 8));
    if (iters == 0) {                  // b = 0: P_t(z) and its sum only
        LaunchScope ls(PET_K_OTHER, st);
        tv_primal_kernel<T, true><<<pgrid, 256, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? PET_OK : cuda_fail(e, "tv kernels launch");
    }
    for (int k = 0; k < iters; ++k) {
        {
            LaunchScope ls(PET_K_OTHER, st);
            tv_dual_kernel<T><<<grid, 256, 0, st>>>(a, reinterpret_cast<const T *>(k == 0 ? a.z : a.xbar));
        }
        LaunchScope ls(PET_K_OTHER, st);
        if (k + 1 < iters) tv_primal_kernel<T, false><<<pgrid, 256, 0, st>>>(a);
        else tv_primal_kernel<T, true><<<pgrid, 256, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tv kernels launch");
    }
    return PET_OK;
}

// iters primal-dual steps (iters = 0 for b = 0: the proximal point is z); the last one clamps
// by P_t and writes the sum to a.sum_out.
pet_status launch_tv_prox(const TvArgs &a, int iters, int arith, cudaStream_t st)
{
    if (iters < 0) return fail(PET_ERR_INVALID, "TV proximal step: negative iteration count");
    return arith == AR_FP64 ? tv_run<double>(a, iters, st) : tv_run<float>(a, iters, st);
}

}  // namespace pet

using namespace pet;

extern "C" pet_status pet_tv_prox(const pet_geometry *g, const float *d_z, const float *d_w, double b,
                                  int iters, float *d_px, float *d_py, float *d_x, void *stream)
{
    if (!g || !d_z || !d_w || !d_px || !d_py || !d_x)
        return fail(PET_ERR_INVALID, "pet_tv_prox: NULL argument");
    if (!(b >= 0) || iters < 0 || iters > 10000)
        return fail(PET_ERR_INVALID, "pet_tv_prox: need b >= 0 and 0 <= iters <= 10000");
    cudaStream_t st = as_stream(stream);
    const GeoDev &gd = g->dev;
    const size_t qb = ((size_t)gd.N * gd.N * gd.Pp * 4 + 255) / 256 * 256;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, 6 * qb, &scr));
    char *base = reinterpret_cast<char *>(scr);
    TvArgs a{};
    a.g = gd;
    a.z = base;
    a.w = base + qb;
    a.x = base + 2 * qb;
    a.xbar = base + 3 * qb;
    a.px = base + 4 * qb;
    a.py = base + 5 * qb;
    a.b = b;
    a.t = 0.0;                         // no clamp: the bare proximal point
    a.U = 0.0;
    a.red = g->red;
    a.sum_out = g->d_sums + 7;
    PET_TRY(to_internal_image(gd, d_z, const_cast<void *>(a.z), 0, 0, st));
    PET_TRY(to_internal_image(gd, d_w, const_cast<void *>(a.w), 0, 0, st));
    PET_TRY(to_internal_image(gd, d_z, a.x, 0, 0, st));
    PET_TRY(to_internal_image(gd, d_px, a.px, 0, 0, st));
    PET_TRY(to_internal_image(gd, d_py, a.py, 0, 0, st));
    if (b > 0 && iters > 0) {
        tv_shape(a);
        PET_TRY(launch_tv_prox(a, iters, AR_KAHAN, st));
    }
    // b = 0 or no iterations: x = z as copied above
    PET_TRY(from_internal_image(gd, a.x, d_x, 0, 0, st));
    PET_TRY(from_internal_image(gd, a.px, d_px, 0, 0, st));
    return from_internal_image(gd, a.py, d_py, 0, 0, st);
}
