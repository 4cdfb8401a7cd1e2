// Internal definitions shared by the libpet CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pet.h"

namespace pet {

// ------------------------------------------------------------------------------------------
// Error handling: thread-local message, status codes, no exceptions across the ABI.
// ------------------------------------------------------------------------------------------
void set_error(const std::string &msg);
pet_status fail(pet_status st, const std::string &msg);
pet_status cuda_fail(cudaError_t e, const char *what);

// Device and pinned-host allocations of the library go through these, so that the test hook
// pet_debug_fail_alloc can make the n-th of them fail as out of memory (host-side fault
// injection: no GPU fault is involved).
bool alloc_fault();
template <class T> inline cudaError_t dev_malloc(T **p, size_t n)
{
    return alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc((void **)p, n);
}
template <class T> inline cudaError_t dev_malloc_async(T **p, size_t n, cudaStream_t st)
{
    return alloc_fault() ? cudaErrorMemoryAllocation : cudaMallocAsync((void **)p, n, st);
}
template <class T> inline cudaError_t host_malloc(T **p, size_t n)
{
    return alloc_fault() ? cudaErrorMemoryAllocation : cudaMallocHost((void **)p, n);
}
inline pet_status cuda_ok(cudaError_t e, const char *what)
{
    return e == cudaSuccess ? PET_OK : cuda_fail(e, what);
}

#define PET_CUDA(call)                                                       \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::pet::cuda_fail(e_, #call);           \
    } while (0)
#define PET_TRY(call)                                                        \
    do {                                                                     \
        pet_status s_ = (call);                                              \
        if (s_ != PET_OK) return s_;                                         \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------------------------------
// Geometry tables.  Positions are fixed point Q32.32 (int64) for the FP32 kernels, so that the
// fractional position of a ray inside a pixel keeps 32 bits whatever the image size; the FP64
// kernels use the double fields.  All values are computed in FP64 on the host.
// ------------------------------------------------------------------------------------------
struct ViewGeo {
    // forward walk along the driving axis (x if |sin| >= |cos|, else y)
    long long stepq;      // cross-coordinate change per driving step, Q32.32
    long long absstepq;   // |stepq|
    double step;          // same, double
    double L;             // length per driving step = 1 / major, pixel units
    double inv_minor;     // 1 / minor (0 when minor == 0)
    float Lf, inv_minorf;
    int xdrive;           // 1: driving index is ix (columns), cross index is iy
    // backprojection footprint (bin units, measured from bin 0)
    long long t0q, cxq, cyq, hq;   // t(ix,iy) = t0 + ix cx + iy cy; half-width h; Q32.32
    double t0, cx, cy, h;
    double wslope;        // length per bin unit of (h - |delta|): rho / (major * minor)
    float wslopef;
    int axis;             // minor == 0: half-open rule, length L for delta in [-h, h)
    // sub-ray model: cross-coordinate shift of half a sub-ray spacing (rho / (2 R a), a the
    // driving component of the view's direction), grid units; sub-ray s of a bin starts
    // (2 s + 1 - R) of them away from the bin's centre line
    long long halfq;
    double half;
    // time of flight: position along the line (pixel units) of pixel (ix, iy)'s centre,
    // tau = tau0 + ix taux + iy tauy; and of the line at the centre of driving column d,
    // tau = tdr r + tdc + d tdd (r the line's offset in pixel units)
    double tau0, taux, tauy, tdr, tdc, tdd;
    float tau0f, tauxf, tauyf, tdrf, tdcf, tddf;
    // table-driven bins (ring sampling): offset of pixel (ix, iy)'s centre along the view's
    // normal in pixel units, pn = pn0 + ix pnx + iy pny (double and Q32.32), the pixel's
    // half-footprint hp = (|c| + |s|) / 2 and 1 / (major minor) (pixel units)
    long long pn0q, pnxq, pnyq, hpq;
    double pn0, pnx, pny, hp, islope;
    float islopef;
};

// One bin of a table-driven geometry: its first line's offset c0 and the spacing ds of its R
// lines (pixel units, double and Q32.32): line s lies at c0 + s ds.
struct BinGeo {
    long long c0q, dsq;
    double c0, ds;
};

struct RayGeo {
    long long loq;        // low cross coordinate of the first driving step, Q32.32 (grid units)
    double lo;            // same, double (the bin's line; with sub-rays, the centre of its lines)
    int d0, nd;           // driving range [d0, d0 + nd)
    long long shq;        // sub-rays: half the cross-coordinate spacing of the bin's lines
    double sh;            //   (line s starts (2 s + 1 - R) sh from lo)
};

// Kernel-side view of a geometry.
struct GeoDev {
    int N, P, Pp, G, NG;      // image side, planes, padded planes, group size, groups
    int V, NB, M, K;          // views, bins, subsets, max candidate bins per view in the gather
    int tuneS;                // forward projector chunks per ray picked by pet_autotune (0: heuristic)
    int R;                    // sub-rays per bin (1: one line); scale includes the 1 / R
    int ring;                 // 1: bins sampled like a detector ring's lines (table-driven)
    int table;                // 1: table-driven bins (sub-rays or ring): the SUB kernels
    double ring_r, ring_db;   // ring radius (pixel units) and angular bin spacing
    float ring_rf, ring_dbf;
    const BinGeo *bins;       // [NB] (table-driven geometries)
    int T;                    // TOF bins per bin (1: no TOF)
    int SB;                   // sinogram entries per view and plane: NB T
    double rho;               // bin spacing / pixel size
    double tof_d, tof_k, tof_w;   // TOF bin width, 1 / (sigma sqrt 2), window half-width
    float tof_df, tof_kf, tof_wf; //   (pixel units; h_t < 1e-12 beyond the window)
    long long offq;           // half a sub-ray spacing in bin units, Q32.32 (2^32 / (2 R))
    double scale;             // sens * pixel_mm
    const ViewGeo *views;     // [V] in subset order
    const RayGeo *rays;       // [V * NB] in subset order
};

struct Reducer {              // deterministic last-block reduction scratch
    double *partials;         // [capacity * nvals]
    unsigned int *ticket;     // one counter, returns to 0 after each launch
    int capacity;
};

}  // namespace pet

struct pet_geometry {
    pet_geometry_desc desc;
    pet::GeoDev dev;
    std::vector<int> voff;          // subset view offsets (M + 1), views sorted by subset
    std::vector<int> view_of_slot;  // original view index of each sorted slot
    pet::ViewGeo *d_views = nullptr;
    pet::RayGeo *d_rays = nullptr;
    pet::BinGeo *d_bins = nullptr;  // table-driven geometries
    float *d_p = nullptr;           // p_j, FP32, [N*N]
    float *d_invp = nullptr;        // 1 / p_j, FP32
    double *d_invp64 = nullptr;     // 1 / p_j, FP64
    int *d_view_of_slot = nullptr;
    // scratch for the standalone projector / step calls (not thread-safe across streams)
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    pet::Reducer red{};
    double *d_sums = nullptr;       // small FP64 scalar area
    void *workspace = nullptr;      // reconstruction workspace reused by pet_reconstruct*
    // precomputed (pixel, view) backprojection entries of the packed update kernel (8-plane
    // groups, uniform bins, no TOF): per subset, [pixel tile][view][pixel of the tile], the
    // kernel's shared-memory order; nullptr: the kernel computes them per tile
    void *d_bptab = nullptr;
    std::vector<size_t> bptab_off;  // byte offset of each subset's block
};

namespace pet {

// kernels implemented in project.cu / update.cu, launched from the host files
// A launch over several scans: the virtual blocks of scan s are [prefix[s], prefix[s+1]);
// a persistent grid strides over all of them.  nscans == 0 means a single scan passed by value.
struct Batch {
    const void *args;          // device array of per-scan argument structs
    const int *prefix;         // device, nscans + 1 entries
    int nscans;
    int grid;                  // CTAs of the persistent grid
};
struct FwdArgs {
    GeoDev g;
    int slot0;                 // first sorted view slot of the subset
    int nviews;                // views in the subset
    const void *img;           // [N*N][Pp] (float or double)
    void *out;                 // [nviews*NB][Pp]: y, or w = 1 - counts/(y + gamma)
    const int *counts;         // [nviews*NB][Pp] (ratio / objective modes)
    const float *gamma;        // [nviews*NB][Pp]
    const float *mult;         // [nviews*NB][Pp] per-bin detection factors a_i (ratio /
                               // objective modes; NULL: a_i = 1): y = a_i (A f)_i + gamma_i
    Reducer red;               // objective mode
    double *result;            // objective mode: 2 doubles (sum y, sum g ln(y + gamma))
    int S, R;                  // launch shape: chunks per ray, rays per ray tile
    int tpv;                   // ray tiles per virtual block
    int nvb;                   // virtual blocks of this scan
};

enum FwdMode { FWD_PLAIN = 0, FWD_RATIO = 1, FWD_OBJECTIVE = 2 };
enum Arith { AR_FP32 = 0, AR_KAHAN = 1, AR_FP64 = 2 };

// after_kernel: the launch directly follows a kernel of the same stream that produces the
// image (a subiteration's update); the projection is then launched with programmatic stream
// serialization, so that its blocks are scheduled while that kernel's last blocks finish and
// wait (griddepcontrol.wait) for its completion before their first memory access.
pet_status launch_forward(const FwdArgs &a, int mode, int arith, cudaStream_t st,
                          bool after_kernel = false);
void forward_shape(FwdArgs &a, int mode, int arith);      // fills S, R, tpv, nvb
// time-of-flight geometries (g.T > 1; launch_forward / forward_shape forward to these)
pet_status launch_forward_tof(const FwdArgs &a, int mode, int arith, cudaStream_t st);
pet_status launch_forward_tof_batch(const FwdArgs &shape, const Batch &b, int mode, int arith,
                                    cudaStream_t st);
void forward_shape_tof(FwdArgs &a, int mode, int arith);
pet_status launch_forward_batch(const FwdArgs &shape, const Batch &b, int mode, int arith,
                                cudaStream_t st);

struct BackArgs {
    GeoDev g;
    int slot0, nviews;
    const void *proj;          // [nviews*NB][Pp]; NULL = ones (sensitivity)
    void *img;                 // [N*N][Pp] out
    int nvb;
};

pet_status launch_back(const BackArgs &a, int arith, cudaStream_t st);

struct UpdateArgs {
    GeoDev g;
    int slot0, nviews;
    const void *w;             // subset ratio term [nviews*NB][Pp]
    const void *f;             // f^{k,i-1} [N*N][Pp]
    void *fout;                // f^{k,i}
    const void *invp;          // [N*N], or [N*N][Pp] when vox (float or double)
    int vox;                   // 1: p differs per voxel (a scan with per-bin detection factors)
    const void *bptab;         // the subset's precomputed (pixel, view) entries (pet_geometry::
                               // d_bptab), or NULL: computed in the kernel
    double invp_scale;         // multiplies invp (a scan whose sens differs from the geometry's)
    void *nu_frozen;           // [N*N][Pp]
    int nu_mode;               // 0: nu = 1, 1: from f, 2: from f and stored, 3: frozen
    double lam_alpha;          // lambda_k alpha_{k,i}
    double beta_over_M, gamma_r, eps, t, U, nu1, nu2;
    const double *sum_f;       // sum of f^{k,i-1} (FP64, device)
    const double *sum_mu;      // sum of mu (FP64, device)
    double *sum_fout;          // sum of f^{k,i} (FP64, device, written)
    Reducer red;
    int tpv;                   // pixel tiles per virtual block
    int nvb;                   // virtual blocks of this scan
    int z3;                    // 1: RDP over the 26 neighbours in 3-D, nu from the 3-D gradient
    int tv;                    // 1: TV variant: write z = f - W grad F_i (no clamp) to fout and
    void *zbuf, *wbuf;         //    zbuf, and W = lambda alpha nu S to wbuf ([N*N][Pp])
    // the scalars above as FP32 for the FP32 kernels (converted once on the host: a conversion
    // from double on the device runs on the narrow FP64 pipe)
    float fs_lam, fs_bm, fs_gamma_r, fs_eps, fs_t, fs_U, fs_nu1, fs_nu2, fs_ips, fs_scale;
};
// FP32 copies of the update's scalars (call after filling the double fields and g)
void update_fp32_scalars(UpdateArgs &a);
pet_status launch_update(const UpdateArgs &a, int arith, cudaStream_t st);
void update_shape(UpdateArgs &a, int arith);               // fills tpv, nvb
GeoDev update_geo(const GeoDev &g);                        // plane grouping of the update kernel
pet_status launch_update_batch(const UpdateArgs &shape, const Batch &b, int arith,
                               cudaStream_t st);
// the geometry's precomputed backprojection entries (d_bptab; left empty where the packed
// update kernel does not run or a subset's views do not fit its table), and an upper bound
// of their size from the description alone (memory accounting before creation)
pet_status build_bp_table(pet_geometry *g, cudaStream_t st);
size_t bp_table_bytes_bound(const pet_geometry_desc &d);

struct ImageArgs {
    GeoDev g;
    const void *f;             // [N*N][Pp]
    void *out;                 // per-kernel output
    double gamma_r, eps, nu1, nu2;
    const double *sum_f;       // mu pass / nu map: sum of f
    const double *sum_mu;      // nu map: sum of mu
    double *result;            // reductions
    Reducer red;
    int ipt, nvb;              // items per thread, virtual blocks of this scan
    int z3;                    // 1: RDP over the 26 neighbours in 3-D, gradient with its z part
    int tv;                    // RDP value kernel: the total variation R_TV instead
};
pet_status launch_sum(const ImageArgs &a, int arith, cudaStream_t st);        // result[0] = sum f
pet_status launch_mu_sum(const ImageArgs &a, int arith, cudaStream_t st);     // result[0] = sum mu
pet_status launch_nu_map(const ImageArgs &a, int arith, cudaStream_t st);     // out = nu
pet_status launch_rdp_grad(const ImageArgs &a, int arith, cudaStream_t st);   // out = grad R
pet_status launch_rdp_value(const ImageArgs &a, int arith, cudaStream_t st);  // result[0] = R
void image_shape(ImageArgs &a);                            // fills ipt, nvb
void mu_shape(ImageArgs &a, int arith);                    // shape of the mu pass
pet_status launch_mu_sum_batch(const ImageArgs &shape, const Batch &b, int arith, cudaStream_t st);
pet_status launch_rdp_value_batch(const ImageArgs &shape, const Batch &b, int arith,
                                  cudaStream_t st);

// per-scan reconstruction state (state.cu)
}  // namespace pet
struct pet_state {
    const pet_geometry *g = nullptr;
    pet_params prm{};
    int arith = pet::AR_KAHAN;
    size_t esz = 4;                 // bytes per image / ratio element
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    void *w = nullptr;              // ratio term of the largest subset
    int *counts = nullptr;          // [V][NB][Pp], views sorted by subset
    float *gamma = nullptr;
    float *mult = nullptr;          // per-bin detection factors [V][NB][Pp] (buffer)
    bool attn = false;              // the loaded scan has per-bin detection factors (mult)
    void *invp_vox = nullptr;       // 1 / p_j per voxel [N*N][Pp] for diag(a) A (with mult)
    void *nu_frozen = nullptr;
    bool have_frozen = false;
    void *tvmem = nullptr;          // TV variant: z, W, xbar, px, py (each q_bytes)
    double *sums = nullptr;         // [0..1] sum f (ping-pong), [2] sum mu, [3..5] objective
    double *objhist = nullptr;      // [(T+1) * 3] objective parts per outer iteration
    int objcap = 0;
    pet::Reducer red{};
    void *redmem = nullptr;
    int *flag = nullptr;
    int k = 0, i = 0, J = 0;        // next subiteration is (k, i+1) of the paper; J done
    double tn = 1.0;                // Nesterov t_{k,i}
    double sens_ratio = 1.0;        // this scan's sens / the geometry's sens (A and p scale with it)
    cudaStream_t alloc_stream = nullptr;   // non-null: buffers are stream-ordered allocations
    cudaStream_t side = nullptr;           // the mu pass runs here, beside the forward projection
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // objective history of a whole reconstruction, evaluated beside the next subiterations
    void *fobj = nullptr;                  // snapshot of f^k
    void *redobj_mem = nullptr;
    pet::Reducer red_obj{};
    cudaStream_t ostream = nullptr;
    cudaEvent_t ev_ofork = nullptr, ev_odone = nullptr;
    bool obj_pending = false;
    cudaStream_t hstream = nullptr;        // whole reconstructions: subiterations at top priority
    cudaEvent_t ev_h0 = nullptr, ev_h1 = nullptr;
    size_t q_bytes = 0, sino_elems = 0, w_bytes = 0;
};

namespace pet {

// Proximal step of the TV variant: primal-dual iterations on internal images [N*N][Pp].
struct TvArgs {
    GeoDev g;
    void *x;                   // in: z, out: the proximal point (clamped by P_t on the last step)
    void *xbar;                // extrapolated primal iterate
    const void *z, *w;         // z = f - W grad F_i and the metric W
    void *px, *py;             // dual variable (kept across subiterations)
    double b;                  // beta / M
    double t, U;               // P_t
    Reducer red;
    double *sum_out;           // sum of the clamped result (last step)
    int ipt, nvb;
};
void tv_shape(TvArgs &a);
pet_status launch_tv_prox(const TvArgs &a, int iters, int arith, cudaStream_t st);

struct SubiterPlan {
    int arith;
    bool tv;                   // TV variant: proximal step after the update
    int tv_iters;
    TvArgs tv_args;
    bool mu;                   // mu pass needed (dynamic nu)
    ImageArgs mu_args;
    FwdArgs fwd;               // subset forward projection + ratio
    UpdateArgs upd;            // fused update
    bool objective;            // Phi(f^{k+1}) after this subiteration
    FwdArgs obj_fwd;
    ImageArgs obj_rdp;
};
void plan_subiter(pet_state *s, SubiterPlan *pl, bool with_objective);
pet_status state_create_loaded(const pet_geometry *g, double sens, const int32_t *d_counts,
                               const float *d_gamma, const float *d_mult, const float *d_img,
                               const pet_params *p, cudaStream_t st, pet_state **out);
size_t state_bytes(const pet_geometry *g, int precision, int iterations);
void state_release(pet_state *s, cudaStream_t st);
pet_status check_params(const pet_params *p);
pet_status fill_internal_ones(const GeoDev &g, void *dst, int is_double, cudaStream_t st);
void objective_args(pet_state *s, double *out3, FwdArgs *fa, ImageArgs *ra);

// layout conversions (layout.cu)
pet_status to_internal_image(const GeoDev &g, const void *src, void *dst, int src_is_double,
                             int dst_is_double, cudaStream_t st);
pet_status from_internal_image(const GeoDev &g, const void *src, void *dst, int src_is_double,
                               int dst_is_double, cudaStream_t st);
pet_status to_internal_sino(const GeoDev &g, const int *d_view_of_slot, int slot0, int nviews,
                            const void *src, void *dst, int elem, int src_is_subset,
                            cudaStream_t st);
pet_status from_internal_sino(const GeoDev &g, const int *d_view_of_slot, int nviews,
                              const void *src, void *dst, int is_double, cudaStream_t st);
pet_status validate_factors(const float *mult, size_t n, int *d_flag, cudaStream_t st);
pet_status validate_data(const GeoDev &g, const int *counts, const float *gamma, size_t n,
                         int *d_flag, cudaStream_t st);

void workspace_free(void *w);     // state.cu
bool batch_can_step(const pet_batch *b);   // batch.cu: a step would not wait for earlier ticks

// geometry helpers (geometry.cu)
pet_status geometry_scratch(const pet_geometry *g, size_t bytes, void **out);
size_t reducer_bytes(int capacity, int nvals);
void reducer_bind(Reducer &r, void *mem, int capacity, int nvals);

}  // namespace pet
