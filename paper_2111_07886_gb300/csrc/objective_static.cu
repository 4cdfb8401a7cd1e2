// pet_objective_static: the objective Phi(f) computed without allocating any memory.
//
// Who needs this: a host that is not allowed to allocate device memory on its own, for
// example a scanner pipeline that hands every byte of device memory to a fixed-size pool at
// start-up, or a real-time acquisition loop in which a cudaMalloc (with its implicit device
// synchronisation) would stall the stream.  pet_objective stages the image and sinograms into
// geometry-owned scratch (allocated on first use) and reduces through a scratch partials
// buffer; this variant reads the caller's buffers in their C-ABI layouts directly and reduces
// through one fixed array in this file's device memory.
//
// The scratch (g_static_scratch) is a file-scope __device__ array: every GPU that loads the
// library holds it (kStaticBlocks * 3 + 64 doubles, about 49 KB) until the process exits.  In
// host code its name is only a host-side stand-in, so the device address is looked up once
// per device with cudaGetSymbolAddress while that device is current, and passed to the kernel.
// All calls share the array: calls that overlap on the GPU (other streams, other threads)
// race on it and must be serialised by the caller.  The call ends by reading the three sums
// back to the host and synchronising its stream.
#include <math.h>

#include <mutex>

#include "kernels.cuh"
#include "profile.cuh"

namespace pet {

constexpr int kStaticBlocks = 2048;                  // reduction grid cap (partials per value)
constexpr int kStaticDoubles = kStaticBlocks * 3 + 64;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// One launch: a grid-stride pass over every (plane, ray) for the data terms and every
// (plane, pixel) for the RDP value, then one deterministic FP64 reduction of three sums.
// Image float [P][N][N], counts int32 / gamma float [P][V][NB] (original view order).
__global__ void __launch_bounds__(256) objective_static_kernel(
    GeoDev g, const int *view_of_slot, const float *img, const int *counts, const float *gamma,
    float gamma_r, float eps, Reducer red, double *result)
{
    const int N = g.N, NB = g.NB, V = g.V, P = g.P;
    const long long nrays = (long long)V * NB * P;
    const long long npix = (long long)N * N * P;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nrays; t += stride) {
        const int p = (int)(t / ((long long)V * NB));
        const int rs = (int)(t % ((long long)V * NB));      // ray in slot order
        const int slot = rs / NB, b = rs % NB;
        const ViewGeo &vw = g.views[slot];
        const RayGeo &rg = g.rays[rs];
        const int ds = vw.xdrive ? 1 : N, cs = vw.xdrive ? N : 1;
        const float *fp = img + (size_t)p * N * N;
        GroupSum<1, AR_KAHAN> s;
        s.zero();
        const long long stp = vw.stepq, ast = vw.absstepq;
        const float L = vw.Lf, im = vw.inv_minorf * kQ32;
        long long lo = rg.loq;
        for (int k = 0; k < rg.nd; ++k) {
            const int d = rg.d0 + k;
            const long long hi = lo + ast;
            const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
            float l1 = (r1 != r0) ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f;
            float l0 = L - l1;
            const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
            l0 = ok0 ? l0 : 0.f;
            l1 = ok1 ? l1 : 0.f;
            float x0[1] = {fp[d * ds + (ok0 ? r0 : 0) * cs]};
            float x1[1] = {fp[d * ds + (ok1 ? r1 : 0) * cs]};
            s.add2terms(l0, x0, l1, x1);
            lo += stp;
        }
        const size_t o = ((size_t)p * V + view_of_slot[slot]) * NB + b;
        const float af = (float)g.scale * s.value(0);
        acc[0] += (double)af;
        const int c = counts[o];
        // the likelihood term in FP64: ln((double) Af + gamma)
        if (c != 0) acc[1] += (double)c * log((double)af + (double)gamma[o]);
    }
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npix; t += stride) {
        const int p = (int)(t / ((long long)N * N));
        const int j = (int)(t % ((long long)N * N));
        const int ix = j % N, iy = j / N;
        const float *fp = img + (size_t)p * N * N;
        const float fj = fp[j];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (q == 4) continue;
            const int x = ix + q % 3 - 1, y = iy + q / 3 - 1;
            if (x < 0 || y < 0 || x >= N || y >= N) continue;
            const float fk = fp[y * N + x];
            const float dd = fj - fk;
            acc[2] += (double)(dd * dd / (fj + fk + gamma_r * fabsf(dd) + eps));
        }
    }
    grid_reduce<3>(acc, red, result);
}

// device address of g_static_scratch, looked up once per device
static std::mutex g_mu;
static double *g_addr[64];

static pet_status static_scratch(double **out)
{
    int dev = 0;
    PET_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PET_ERR_INVALID, "pet_objective_static: device id >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        PET_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_addr[dev] = reinterpret_cast<double *>(p);
    }
    *out = g_addr[dev];
    return PET_OK;
}

}  // namespace pet

using namespace pet;

extern "C" pet_status pet_objective_static(const pet_geometry *g, const int32_t *d_counts,
                                           const float *d_gamma, const float *d_img,
                                           double beta, double gamma_r, double eps,
                                           double *h_phi, double *h_parts, void *stream)
{
    if (!g || !d_counts || !d_gamma || !d_img || !h_phi)
        return fail(PET_ERR_INVALID, "pet_objective_static: NULL argument");
    const GeoDev &gd = g->dev;
    if (gd.table || gd.T > 1)
        return fail(PET_ERR_INVALID, "pet_objective_static: one line per uniform bin without TOF only "
                                     "(use pet_objective for sub-ray, ring and TOF geometries)");
    const double nrays = (double)gd.V * gd.NB * gd.P, npix = (double)gd.N * gd.N * gd.P;
    if (nrays > 2147483647.0 || npix > 2147483647.0)
        return fail(PET_ERR_INVALID, "pet_objective_static: at most 2^31 - 1 rays x planes and "
                                     "2^31 - 1 pixels x planes (use pet_objective)");
    cudaStream_t st = as_stream(stream);
    double *scr = nullptr;
    PET_TRY(static_scratch(&scr));
    Reducer red;
    red.partials = scr;
    red.capacity = kStaticBlocks;
    red.ticket = reinterpret_cast<unsigned int *>(scr + kStaticBlocks * 3);
    double *result = scr + kStaticBlocks * 3 + 8;
    // the ticket must start at zero; results are overwritten
    PET_CUDA(cudaMemsetAsync(red.ticket, 0, sizeof(double), st));
    const double work = nrays > npix ? nrays : npix;
    long long grid = (long long)((work + 255) / 256);
    if (grid > kStaticBlocks) grid = kStaticBlocks;
    if (grid < 1) grid = 1;
    {
        LaunchScope ls(PET_K_OTHER, st);
        objective_static_kernel<<<(unsigned)grid, 256, 0, st>>>(
            gd, g->d_view_of_slot, d_img, d_counts, d_gamma, (float)gamma_r, (float)eps, red,
            result);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "objective_static_kernel launch");
    }
    double h[3];
    PET_CUDA(cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    *h_phi = h[0] - h[1] + beta * h[2];
    if (h_parts) { h_parts[0] = h[0]; h_parts[1] = h[1]; h_parts[2] = h[2]; }
    return PET_OK;
}
