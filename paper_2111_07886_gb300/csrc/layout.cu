// Layout conversions between the C-ABI layouts (plane outermost) and the internal ones
// (planes innermost, padded to the plane group; sinogram views sorted by subset), and the
// input check of the data (counts >= 0, gamma > 0 and finite: Eq. model-Poisson needs
// gamma in R_{++}^p).
#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

// [P][N*N] -> [N*N][Pp]; pad planes are zero.
template <typename S, typename D>
__global__ void img_to_internal(const S *src, D *dst, int npix, int P, int Pp)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)npix * Pp) return;
    const int p = (int)(tid % Pp);
    const long long j = tid / Pp;
    dst[tid] = p < P ? (D)src[(size_t)p * npix + j] : (D)0;
}

// [N*N][Pp] -> [P][N*N]
template <typename S, typename D>
__global__ void img_from_internal(const S *src, D *dst, int npix, int P, int Pp)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)npix * P) return;
    const int p = (int)(tid / npix);
    const long long j = tid % npix;
    dst[tid] = (D)src[(size_t)j * Pp + p];
}

// full [P][V][NB] (original view order) or subset [P][nviews][NB] -> [nviews][NB][Pp]
template <typename E, typename D = E>
__global__ void sino_to_internal(const E *src, D *dst, const int *view_of_slot, int slot0,
                                 int nviews, int V, int NB, int P, int Pp, int src_is_subset,
                                 D pad)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)nviews * NB * Pp) return;
    const int p = (int)(tid % Pp);
    const long long rb = tid / Pp;
    const int b = (int)(rb % NB);
    const int u = (int)(rb / NB);
    if (p >= P) { dst[tid] = pad; return; }
    const int v = src_is_subset ? u : view_of_slot[slot0 + u];
    const int vn = src_is_subset ? nviews : V;
    dst[tid] = (D)src[((size_t)p * vn + v) * NB + b];
}

// [nviews][NB][Pp] -> [P][nviews][NB], or -> [P][V][NB] in original view order when
// view_of_slot is given (all views, slot0 = 0)
template <typename E>
__global__ void sino_from_internal(const E *src, E *dst, const int *view_of_slot, int nviews,
                                   int NB, int P, int Pp)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)P * nviews * NB) return;
    const long long per = (long long)nviews * NB;
    const int p = (int)(tid / per);
    const long long rb = tid % per;
    const int u = (int)(rb / NB), b = (int)(rb % NB);
    const int v = view_of_slot ? view_of_slot[u] : u;
    dst[((size_t)p * nviews + v) * NB + b] = src[(size_t)rb * Pp + p];
}

// ones in the valid planes, zero in the pad planes
template <typename D>
__global__ void img_ones_internal(D *dst, long long n, int P, int Pp)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n) return;
    dst[tid] = (int)(tid % Pp) < P ? (D)1 : (D)0;
}

__global__ void check_data(const int *counts, const float *gamma, size_t n, int *flag)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gm = gamma[i];
    if (counts[i] < 0 || !(gm > 0.f) || !isfinite(gm)) atomicOr(flag, 1);
}

__global__ void check_factors(const float *mult, size_t n, int *flag)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = mult[i];
    if (!(a >= 0.f) || !isfinite(a)) atomicOr(flag, 1);
}

static inline unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

pet_status to_internal_image(const GeoDev &g, const void *src, void *dst, int sd, int dd,
                             cudaStream_t st)
{
    const int npix = g.N * g.N;
    const long long n = (long long)npix * g.Pp;
    LaunchScope ls(PET_K_LAYOUT, st);
    if (!sd && !dd) img_to_internal<float, float><<<blocks(n), 256, 0, st>>>((const float *)src, (float *)dst, npix, g.P, g.Pp);
    else if (!sd && dd) img_to_internal<float, double><<<blocks(n), 256, 0, st>>>((const float *)src, (double *)dst, npix, g.P, g.Pp);
    else if (sd && !dd) img_to_internal<double, float><<<blocks(n), 256, 0, st>>>((const double *)src, (float *)dst, npix, g.P, g.Pp);
    else img_to_internal<double, double><<<blocks(n), 256, 0, st>>>((const double *)src, (double *)dst, npix, g.P, g.Pp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "img_to_internal");
}

pet_status from_internal_image(const GeoDev &g, const void *src, void *dst, int sd, int dd,
                               cudaStream_t st)
{
    const int npix = g.N * g.N;
    const long long n = (long long)npix * g.P;
    LaunchScope ls(PET_K_LAYOUT, st);
    if (!sd && !dd) img_from_internal<float, float><<<blocks(n), 256, 0, st>>>((const float *)src, (float *)dst, npix, g.P, g.Pp);
    else if (!sd && dd) img_from_internal<float, double><<<blocks(n), 256, 0, st>>>((const float *)src, (double *)dst, npix, g.P, g.Pp);
    else if (sd && !dd) img_from_internal<double, float><<<blocks(n), 256, 0, st>>>((const double *)src, (float *)dst, npix, g.P, g.Pp);
    else img_from_internal<double, double><<<blocks(n), 256, 0, st>>>((const double *)src, (double *)dst, npix, g.P, g.Pp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "img_from_internal");
}

pet_status to_internal_sino(const GeoDev &g, const int *d_view_of_slot, int slot0, int nviews,
                            const void *src, void *dst, int elem, int src_is_subset,
                            cudaStream_t st)
{
    const long long n = (long long)nviews * g.SB * g.Pp;    // SB: bins x TOF bins
    if (n == 0) return PET_OK;
    LaunchScope ls(PET_K_LAYOUT, st);
    // elem: 0 int32 counts (pad 0), 1 float gamma (pad 1), 2 float data (pad 0), 3 double
    // data, 4 float data to double (pad 0)
    if (elem == 4)
        sino_to_internal<float, double><<<blocks(n), 256, 0, st>>>((const float *)src, (double *)dst, d_view_of_slot, slot0, nviews, g.V, g.SB, g.P, g.Pp, src_is_subset, 0.0);
    else if (elem == 0)
        sino_to_internal<int><<<blocks(n), 256, 0, st>>>((const int *)src, (int *)dst, d_view_of_slot, slot0, nviews, g.V, g.SB, g.P, g.Pp, src_is_subset, 0);
    else if (elem == 1)
        sino_to_internal<float><<<blocks(n), 256, 0, st>>>((const float *)src, (float *)dst, d_view_of_slot, slot0, nviews, g.V, g.SB, g.P, g.Pp, src_is_subset, 1.f);
    else if (elem == 2)
        sino_to_internal<float><<<blocks(n), 256, 0, st>>>((const float *)src, (float *)dst, d_view_of_slot, slot0, nviews, g.V, g.SB, g.P, g.Pp, src_is_subset, 0.f);
    else
        sino_to_internal<double><<<blocks(n), 256, 0, st>>>((const double *)src, (double *)dst, d_view_of_slot, slot0, nviews, g.V, g.SB, g.P, g.Pp, src_is_subset, 0.0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "sino_to_internal");
}

pet_status from_internal_sino(const GeoDev &g, const int *d_view_of_slot, int nviews,
                              const void *src, void *dst, int is_double, cudaStream_t st)
{
    const long long n = (long long)g.P * nviews * g.SB;
    if (n == 0) return PET_OK;
    LaunchScope ls(PET_K_LAYOUT, st);
    if (is_double) sino_from_internal<double><<<blocks(n), 256, 0, st>>>((const double *)src, (double *)dst, d_view_of_slot, nviews, g.SB, g.P, g.Pp);
    else sino_from_internal<float><<<blocks(n), 256, 0, st>>>((const float *)src, (float *)dst, d_view_of_slot, nviews, g.SB, g.P, g.Pp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "sino_from_internal");
}

pet_status fill_internal_ones(const GeoDev &g, void *dst, int is_double, cudaStream_t st)
{
    const long long n = (long long)g.N * g.N * g.Pp;
    LaunchScope ls(PET_K_LAYOUT, st);
    if (is_double) img_ones_internal<double><<<blocks(n), 256, 0, st>>>((double *)dst, n, g.P, g.Pp);
    else img_ones_internal<float><<<blocks(n), 256, 0, st>>>((float *)dst, n, g.P, g.Pp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "img_ones_internal");
}

// Per-bin detection factors: finite and >= 0 (sets *d_flag, which the caller cleared, else).
pet_status validate_factors(const float *mult, size_t n, int *d_flag, cudaStream_t st)
{
    if (n == 0) return PET_OK;
    LaunchScope ls(PET_K_LAYOUT, st);
    check_factors<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mult, n, d_flag);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "check_factors");
}

pet_status validate_data(const GeoDev &g, const int *counts, const float *gamma, size_t n,
                         int *d_flag, cudaStream_t st)
{
    (void)g;
    PET_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    if (n == 0) return PET_OK;
    LaunchScope ls(PET_K_LAYOUT, st);
    check_data<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(counts, gamma, n, d_flag);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PET_OK : cuda_fail(e, "check_data");
}

}  // namespace pet
