// Geometry: per-view / per-ray tables of the ray-driven projector and the pixel-driven
// backprojector (built in FP64 on the host), the subset ordering of Sec. II-B, and the
// sensitivity p_j of Eq. pj.  Also the error plumbing of the C ABI.
#include <atomic>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "pet_common.cuh"
#include "profile.cuh"

namespace pet {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

pet_status fail(pet_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

static std::atomic<long long> g_fail_alloc{0};
static std::atomic<int> g_bp_table{1};   // pet_debug_bp_table

bool alloc_fault()
{
    long long n = g_fail_alloc.load();
    while (n > 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
    }
    return false;
}

pet_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PET_ERR_OOM : PET_ERR_CUDA;
}

static inline long long to_q32(double x) { return llround(ldexp(x, 32)); }

size_t reducer_bytes(int capacity, int nvals)
{
    return (size_t)capacity * nvals * sizeof(double) + 256;
}

void reducer_bind(Reducer &r, void *mem, int capacity, int nvals)
{
    r.partials = reinterpret_cast<double *>(mem);
    r.ticket = reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(mem) +
                                                (size_t)capacity * nvals * sizeof(double));
    r.capacity = capacity;
}

pet_status geometry_scratch(const pet_geometry *gc, size_t bytes, void **out)
{
    pet_geometry *g = const_cast<pet_geometry *>(gc);
    if (g->scratch_bytes < bytes) {
        if (g->d_scratch) PET_CUDA(cudaFree(g->d_scratch));
        g->d_scratch = nullptr;
        g->scratch_bytes = 0;
        PET_CUDA(dev_malloc(&g->d_scratch, bytes));
        g->scratch_bytes = bytes;
    }
    *out = g->d_scratch;
    return PET_OK;
}

// p_j = (A^T 1)_j / M, or 1/M where (A^T 1)_j == 0 (Eq. pj); also 1/p_j in FP32 and FP64.
__global__ void finish_sensitivity(const double *bp, int npix, int M, float *p, float *invp,
                                   double *invp64)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npix) return;
    double v = bp[j];
    double pj = v > 0.0 ? v / M : 1.0 / M;
    p[j] = (float)pj;
    invp[j] = (float)(1.0 / pj);
    invp64[j] = 1.0 / pj;
}

}  // namespace pet

using namespace pet;

extern "C" const char *pet_last_error(void) { return pet::g_last_error.c_str(); }

extern "C" void pet_debug_fail_alloc(int n) { pet::g_fail_alloc.store(n > 0 ? n : 0); }
extern "C" void pet_debug_bp_table(int enable) { pet::g_bp_table.store(enable ? 1 : 0); }

static pet_status build_tables(pet_geometry *g, std::vector<ViewGeo> &views,
                               std::vector<RayGeo> &rays, std::vector<BinGeo> &bins)
{
    const pet_geometry_desc &d = g->desc;
    const int N = d.n, V = d.nviews, NB = d.nbins, M = d.nsubsets;
    const int R = d.subrays > 1 ? d.subrays : 1;
    const double rho = d.bin_mm / d.pixel_mm;
    const double half = 0.5 * N;
    // bins: the line offset of bin b (pixel units) and the lines of its R sub-rays.  Uniform:
    // r_b = (b - (NB-1)/2) rho, width rho.  Ring: r_b = Rd sin(beta_b), beta_b = (b - (NB-1)/2)
    // dbeta, width [Rd sin(beta_b - dbeta/2), Rd sin(beta_b + dbeta/2)]; R > 1 lines spread
    // uniformly over the width, around its middle m_b (= r_b for uniform bins).
    const bool ring = d.ring_mm > 0.0;
    const double Rd = ring ? d.ring_mm / d.pixel_mm : 0.0, db = ring ? d.bin_mm / d.ring_mm : 0.0;
    std::vector<double> rc(NB), wd(NB);          // centre of the bin's lines, width
    double wmin = 1e300;
    bins.assign(NB, BinGeo{});
    for (int b = 0; b < NB; ++b) {
        const double k = (double)b - 0.5 * (NB - 1);
        double lo, hi, rb;
        if (ring) { lo = Rd * sin((k - 0.5) * db); hi = Rd * sin((k + 0.5) * db); rb = Rd * sin(k * db); }
        else { rb = k * rho; lo = rb - 0.5 * rho; hi = rb + 0.5 * rho; }
        wd[b] = ring ? hi - lo : rho;
        wmin = std::min(wmin, wd[b]);
        rc[b] = (R > 1 && ring) ? 0.5 * (lo + hi) : rb;
        BinGeo bg;
        bg.ds = wd[b] / R;
        bg.c0 = R > 1 ? lo + 0.5 * bg.ds : rb;
        bg.c0q = to_q32(bg.c0);
        bg.dsq = to_q32(bg.ds);
        bins[b] = bg;
    }
    g->voff.assign(M + 1, 0);
    g->view_of_slot.clear();
    for (int i = 0; i < M; ++i) {
        g->voff[i] = (int)g->view_of_slot.size();
        for (int v = i; v < V; v += M) g->view_of_slot.push_back(v);
    }
    g->voff[M] = V;
    views.resize(V);
    rays.resize((size_t)V * NB);
    int K = 1;
    for (int u = 0; u < V; ++u) {
        const int v = g->view_of_slot[u];
        const double th = (double)v * 3.14159265358979323846 / (double)V;
        double c = cos(th), s = sin(th);
        if (fabs(c) < 1e-12) { c = 0.0; s = s > 0 ? 1.0 : -1.0; }
        if (fabs(s) < 1e-12) { s = 0.0; c = c > 0 ? 1.0 : -1.0; }
        const double ac = fabs(c), as = fabs(s);
        const double major = std::max(ac, as), minor = std::min(ac, as);
        ViewGeo vg;
        std::memset(&vg, 0, sizeof(vg));
        vg.xdrive = as >= ac ? 1 : 0;
        const double B = vg.xdrive ? -c / s : -s / c;
        vg.step = B;
        vg.stepq = to_q32(B);
        vg.absstepq = vg.stepq < 0 ? -vg.stepq : vg.stepq;
        vg.L = 1.0 / major;
        vg.inv_minor = minor > 0.0 ? 1.0 / minor : 0.0;
        vg.Lf = (float)vg.L;
        vg.inv_minorf = (float)vg.inv_minor;
        // backprojection: bin coordinate of the centre of pixel (ix, iy)
        vg.t0 = ((0.5 - half) * c + (0.5 - half) * s) / rho + 0.5 * (NB - 1);
        vg.cx = c / rho;
        vg.cy = s / rho;
        vg.h = (ac + as) / (2.0 * rho);
        vg.t0q = to_q32(vg.t0);
        vg.cxq = to_q32(vg.cx);
        vg.cyq = to_q32(vg.cy);
        vg.hq = to_q32(vg.h);
        vg.axis = minor == 0.0 ? 1 : 0;
        vg.wslope = minor > 0.0 ? rho / (major * minor) : 0.0;
        vg.wslopef = (float)vg.wslope;
        // forward walk: cross coordinate (grid units) at the start of driving step 0
        const double a = vg.xdrive ? s : c;        // divisor
        const double o = vg.xdrive ? c : s;        // other component
        vg.half = R > 1 ? rho / (2.0 * R * a) : 0.0;
        vg.halfq = to_q32(vg.half);
        // time of flight: the line is r (c, s) + tau (-s, c); pixel centre (X, Y) lies at
        // tau = -X s + Y c, X = ix + 1/2 - N/2, Y = iy + 1/2 - N/2 (pixel units)
        vg.taux = -s;
        vg.tauy = c;
        vg.tau0 = (0.5 - half) * (c - s);
        if (vg.xdrive) {           // X = d + 1/2 - N/2 on the line: tau = (r c - X) / s
            vg.tdr = c / s; vg.tdc = -(0.5 - half) / s; vg.tdd = -1.0 / s;
        } else {                   // Y = d + 1/2 - N/2: tau = (Y - r s) / c
            vg.tdr = -s / c; vg.tdc = (0.5 - half) / c; vg.tdd = 1.0 / c;
        }
        vg.tau0f = (float)vg.tau0; vg.tauxf = (float)vg.taux; vg.tauyf = (float)vg.tauy;
        vg.tdrf = (float)vg.tdr; vg.tdcf = (float)vg.tdc; vg.tddf = (float)vg.tdd;
        // table-driven bins: the pixel centre's offset along the normal (c, s), pixel units
        vg.pnx = c;
        vg.pny = s;
        vg.pn0 = (0.5 - half) * (c + s);
        vg.hp = 0.5 * (ac + as);
        vg.islope = minor > 0.0 ? 1.0 / (major * minor) : 0.0;
        vg.islopef = (float)vg.islope;
        vg.pn0q = to_q32(vg.pn0); vg.pnxq = to_q32(vg.pnx); vg.pnyq = to_q32(vg.pny);
        vg.hpq = to_q32(vg.hp);
        // candidate bins of a pixel's footprint: one line per bin, or sub-lines within
        // (R - 1) / (2 R) bins of the bin centre on either side (first candidate floor(t - hh));
        // ring bins: any bin whose width meets the footprint, from one bin before the bin
        // coordinate of its low edge (the narrowest bins, at the edge of the field, decide)
        if (ring) K = std::max(K, (int)floor(2.0 * (0.5 * (ac + as)) / wmin) + 3);
        else if (R == 1) K = std::max(K, (int)floor(2.0 * vg.h) + 1);
        else K = std::max(K, (int)floor(2.0 * (vg.h + 0.5 - 0.5 / R)) + 2);
        views[u] = vg;
        // driving steps the line at offset r meets the image (+- one step of margin)
        auto range = [&](double r, long long &dlo, long long &dhi, double &LO0) {
            const double A0 = (r + half * o) / a + half;
            LO0 = A0 + std::min(0.0, B);
            const double aB = fabs(B);
            double lower, upper;
            if (B > 0) { lower = (-LO0 - aB) / B; upper = (N - LO0) / B; }
            else if (B < 0) { lower = (LO0 - N) / aB; upper = (LO0 + aB) / aB; }
            else {
                lower = (LO0 >= -1.0 && LO0 < N + 1.0) ? 0.0 : 1e30;
                upper = (LO0 >= -1.0 && LO0 < N + 1.0) ? N : -1e30;
            }
            dlo = (long long)floor(std::max(-1e9, lower)) - 1;
            dhi = (long long)ceil(std::min(1e9, upper)) + 1;
        };
        for (int b = 0; b < NB; ++b) {
            const double r = rc[b];
            long long dlo, dhi;
            double LO0;
            range(r, dlo, dhi, LO0);
            if (R > 1) {
                // the union of the ranges of the bin's outermost sub-lines and its centre line
                const double e = (0.5 - 0.5 / R) * wd[b];
                for (double rr : {r - e, r + e}) {
                    long long l2, h2;
                    double unused;
                    range(rr, l2, h2, unused);
                    if (l2 <= h2) {
                        if (dlo > dhi) { dlo = l2; dhi = h2; }
                        else { dlo = std::min(dlo, l2); dhi = std::max(dhi, h2); }
                    }
                }
            }
            dlo = std::max(0LL, dlo);
            dhi = std::min((long long)N - 1, dhi);
            RayGeo rg;
            std::memset(&rg, 0, sizeof(rg));
            if (dlo > dhi) { rg.d0 = 0; rg.nd = 0; }
            else { rg.d0 = (int)dlo; rg.nd = (int)(dhi - dlo + 1); }
            rg.lo = LO0 + rg.d0 * B;
            rg.loq = to_q32(rg.lo);
            rg.sh = R > 1 ? wd[b] / (2.0 * R * a) : 0.0;
            rg.shq = to_q32(rg.sh);
            rays[(size_t)u * NB + b] = rg;
        }
    }
    // sub-ray and ring kernels are built for 4 candidates
    g->dev.K = (R > 1 || ring) ? std::max(K, 3) : K;
    g->dev.R = R;
    g->dev.ring = ring ? 1 : 0;
    g->dev.table = (R > 1 || ring) ? 1 : 0;
    g->dev.ring_r = Rd;
    g->dev.ring_db = db;
    g->dev.ring_rf = (float)Rd;
    g->dev.ring_dbf = (float)db;
    g->dev.offq = to_q32(0.5 / R);
    return PET_OK;
}

static pet_status geometry_init(pet_geometry *g, cudaStream_t st)
{
    const pet_geometry_desc &d = g->desc;
    std::vector<ViewGeo> views;
    std::vector<RayGeo> rays;
    std::vector<BinGeo> bins;
    PET_TRY(build_tables(g, views, rays, bins));
    GeoDev &gd = g->dev;
    if (gd.K > 4)
        return fail(PET_ERR_INVALID, "pet_geometry_create: a pixel's footprint spans more than 4 "
                                     "bins of one view (bins too fine for the sub-ray width)");
    gd.N = d.n;
    gd.P = d.nplanes;
    gd.G = d.nplanes == 1 ? 1 : 8;
    gd.Pp = (d.nplanes + gd.G - 1) / gd.G * gd.G;
    gd.NG = gd.Pp / gd.G;
    gd.V = d.nviews;
    gd.NB = d.nbins;
    gd.M = d.nsubsets;
    gd.scale = d.sens * d.pixel_mm / gd.R;
    gd.rho = d.bin_mm / d.pixel_mm;
    gd.T = d.tof_bins > 1 ? d.tof_bins : 1;
    gd.SB = gd.NB * gd.T;
    if (gd.T > 1) {
        // h_t(tau) < 1e-12 farther than 7.1 sigma beyond the bin's edges
        const double sigma = d.tof_fwhm_mm / (2.0 * sqrt(2.0 * log(2.0))) / d.pixel_mm;
        gd.tof_d = d.tof_bin_mm / d.pixel_mm;
        gd.tof_k = 1.0 / (sigma * sqrt(2.0));
        gd.tof_w = 0.5 * gd.tof_d + 7.1 * sigma;
    } else {
        gd.tof_d = gd.tof_k = gd.tof_w = 0.0;
    }
    gd.tof_df = (float)gd.tof_d; gd.tof_kf = (float)gd.tof_k; gd.tof_wf = (float)gd.tof_w;
    PET_CUDA(dev_malloc(&g->d_views, sizeof(ViewGeo) * views.size()));
    PET_CUDA(dev_malloc(&g->d_rays, sizeof(RayGeo) * rays.size()));
    PET_CUDA(dev_malloc(&g->d_view_of_slot, sizeof(int) * g->view_of_slot.size()));
    PET_CUDA(dev_malloc(&g->d_bins, sizeof(BinGeo) * bins.size()));
    PET_CUDA(cudaMemcpyAsync(g->d_bins, bins.data(), sizeof(BinGeo) * bins.size(),
                             cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(g->d_views, views.data(), sizeof(ViewGeo) * views.size(),
                             cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(g->d_rays, rays.data(), sizeof(RayGeo) * rays.size(),
                             cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(g->d_view_of_slot, g->view_of_slot.data(),
                             sizeof(int) * g->view_of_slot.size(), cudaMemcpyHostToDevice, st));
    gd.views = g->d_views;
    gd.rays = g->d_rays;
    gd.bins = g->d_bins;
    const size_t npix = (size_t)d.n * d.n;
    PET_CUDA(dev_malloc(&g->d_p, sizeof(float) * npix));
    PET_CUDA(dev_malloc(&g->d_invp, sizeof(float) * npix));
    PET_CUDA(dev_malloc(&g->d_invp64, sizeof(double) * npix));
    const int cap = 4096;
    void *redmem = nullptr;
    PET_CUDA(dev_malloc(&redmem, reducer_bytes(cap, 4)));
    PET_CUDA(cudaMemsetAsync(redmem, 0, reducer_bytes(cap, 4), st));
    reducer_bind(g->red, redmem, cap, 4);
    PET_CUDA(dev_malloc(&g->d_sums, 16 * sizeof(double)));
    // sensitivity: one FP64 backprojection of ones over all views, single plane
    double *bp = nullptr;
    PET_CUDA(dev_malloc_async((void **)&bp, sizeof(double) * npix, st));
    BackArgs ba;
    ba.g = gd;
    ba.g.P = 1; ba.g.Pp = 1; ba.g.G = 1; ba.g.NG = 1;
    ba.slot0 = 0;
    ba.nviews = d.nviews;
    ba.proj = nullptr;
    ba.img = bp;
    pet_status s = launch_back(ba, AR_FP64, st);
    if (s == PET_OK) {
        LaunchScope ls(PET_K_OTHER, st);
        finish_sensitivity<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(
            bp, (int)npix, d.nsubsets, g->d_p, g->d_invp, g->d_invp64);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "finish_sensitivity");
    }
    cudaFreeAsync(bp, st);
    if (s == PET_OK && g_bp_table.load()) s = build_bp_table(g, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (s != PET_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "pet_geometry_create");
    return PET_OK;
}

extern "C" pet_status pet_geometry_create(const pet_geometry_desc *desc, void *stream,
                                          pet_geometry **out)
{
    if (!desc || !out) return fail(PET_ERR_INVALID, "pet_geometry_create: NULL argument");
    *out = nullptr;
    const pet_geometry_desc &d = *desc;
    if (d.n < 1 || d.n > 8192 || d.nplanes < 1 || d.nviews < 1 || d.nbins < 4 ||
        d.nsubsets < 1 || d.nsubsets > d.nviews || !(d.pixel_mm > 0) || !(d.bin_mm > 0) ||
        !(d.sens > 0) || !std::isfinite(d.pixel_mm) || !std::isfinite(d.bin_mm) ||
        !std::isfinite(d.sens))
        return fail(PET_ERR_INVALID, "pet_geometry_create: invalid geometry description "
                                     "(need n in [1,8192], nplanes, nviews >= 1, nbins >= 4, "
                                     "1 <= nsubsets <= nviews, pixel_mm, bin_mm, sens > 0)");
    if (d.nplanes > 2048)
        return fail(PET_ERR_INVALID, "pet_geometry_create: at most 2048 planes");
    if (d.subrays < 0 || d.subrays > 64)
        return fail(PET_ERR_INVALID, "pet_geometry_create: subrays must be in 0..64");
    if (d.bin_mm < 0.36 * d.pixel_mm)
        return fail(PET_ERR_INVALID, "pet_geometry_create: bin_mm must be >= 0.36 pixel_mm "
                                     "(at most 4 rays of one view cross a pixel)");
    if (!(d.ring_mm >= 0) || !std::isfinite(d.ring_mm) ||
        (d.ring_mm > 0 && 0.5 * d.nbins * d.bin_mm / d.ring_mm >= 1.5707963267948966))
        return fail(PET_ERR_INVALID, "pet_geometry_create: ring_mm must be 0 or > 0 with the bins "
                                     "spanning less than a half circle (nbins bin_mm / ring_mm < pi)");
    if (d.tof_bins < 0 || d.tof_bins > 64 ||
        (d.tof_bins > 1 && (!(d.tof_bin_mm > 0) || !(d.tof_fwhm_mm > 0) ||
                            !std::isfinite(d.tof_bin_mm) || !std::isfinite(d.tof_fwhm_mm) ||
                            d.subrays > 1)))
        return fail(PET_ERR_INVALID, "pet_geometry_create: tof_bins must be in 0..64, with "
                                     "tof_bin_mm, tof_fwhm_mm > 0 and subrays <= 1 when > 1");
    if ((double)d.n * d.n * ((d.nplanes + 7) / 8 * 8) > 4.0e9 ||
        (double)d.nviews * d.nbins * (d.tof_bins > 1 ? d.tof_bins : 1) *
                ((d.nplanes + 7) / 8 * 8) > 4.0e9)
        return fail(PET_ERR_INVALID, "pet_geometry_create: problem too large (> 4e9 elements)");
    pet_geometry *g = new pet_geometry();
    g->desc = d;
    pet_status s = geometry_init(g, as_stream(stream));
    if (s != PET_OK) {
        std::string msg = pet_last_error();
        pet_geometry_destroy(g);
        return fail(s, msg);
    }
    *out = g;
    return PET_OK;
}

extern "C" void pet_geometry_destroy(pet_geometry *g)
{
    if (!g) return;
    pet::workspace_free(g->workspace);
    cudaFree(g->d_views);
    cudaFree(g->d_rays);
    cudaFree(g->d_bins);
    cudaFree(g->d_view_of_slot);
    cudaFree(g->d_p);
    cudaFree(g->d_invp);
    cudaFree(g->d_invp64);
    cudaFree(g->d_scratch);
    cudaFree(g->red.partials);
    cudaFree(g->d_sums);
    cudaFree(g->d_bptab);
    delete g;
}

extern "C" int pet_subset_size(const pet_geometry *g, int subset)
{
    if (!g || subset < 0 || subset >= g->desc.nsubsets) return -1;
    return g->voff[subset + 1] - g->voff[subset];
}

extern "C" pet_status pet_sensitivity(const pet_geometry *g, float *d_p, void *stream)
{
    if (!g || !d_p) return fail(PET_ERR_INVALID, "pet_sensitivity: NULL argument");
    PET_CUDA(cudaMemcpyAsync(d_p, g->d_p, sizeof(float) * g->desc.n * g->desc.n,
                             cudaMemcpyDeviceToDevice, as_stream(stream)));
    return PET_OK;
}
