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
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "profile.cuh"

#ifndef FWD_MAX_CHUNKS
#define FWD_MAX_CHUNKS 16       // most threads sharing one ray (built-in chunking and autotuner)
#endif
#ifndef FWD_FAST
#define FWD_FAST 1               // blocked compensated walk (see the G == 8 branch of fwd_kernel)
#endif
#ifndef FWD_TILE_ORDER
#define FWD_TILE_ORDER 1         // ray tiles within one view, centre bins first (long rays first),
#endif                           // in the ratio mode (2: in the objective mode too; 0: neither)

namespace pet {

// Thread layout: a virtual block is R rays x S chunks x NG plane groups (thread = (ray * S +
// chunk) * NG + group; threads beyond R S NG idle).  Chunk c walks driving steps
// [c Lc, (c + 1) Lc) of its ray, Lc = ceil(nd / S), so that short subsets still fill the GPU; the
// S partial sums of a (ray, group) are combined in chunk order through shared memory
// (deterministic).  A persistent grid strides over the virtual blocks of one scan or a batch.
template <int G, int AR, int MODE, bool SUB = false>
__global__ void __launch_bounds__(256, 3) fwd_kernel(const __grid_constant__ FwdArgs one, const Batch bt)
{
    grid_dependency_wait();                      // before any memory access
    using T = typename ArithT<AR>::T;
    __shared__ T comb_s[256 * G];
    __shared__ T comb_e[256 * G];
    const int total = total_vblocks(one, bt);
    __shared__ FwdArgs sh_args;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int vloc, nv;
        const FwdArgs &a = scan_args(one, bt, vb, vloc, nv, sh_args);
        const GeoDev &g = a.g;
        const int NG = g.NG, NB = g.NB, N = g.N, Pp = g.Pp, S = a.S, R = a.R;
        const int nrays = a.nviews * NB;
        constexpr bool kOrder = FWD_TILE_ORDER && (MODE != FWD_OBJECTIVE || FWD_TILE_ORDER > 1);
        const int tpv_view = (NB + R - 1) / R;       // tiles of one view
        const int ntiles = kOrder ? a.nviews * tpv_view : (nrays + R - 1) / R;
        const bool lane_ok = (int)threadIdx.x < R * S * NG;
        double obj[2] = {0.0, 0.0};
        // with the centre-first order, virtual block v of a scan takes tiles v, v + nv, ...: a
        // mix of long and short rays in every block (the objective mode's blocks hold several)
        const int t_end = kOrder ? ntiles : min(ntiles, (vloc + 1) * a.tpv);
        for (int tile = kOrder ? vloc : vloc * a.tpv; tile < t_end; tile += kOrder ? nv : 1) {
        const int grp = threadIdx.x % NG;
        const int c = (threadIdx.x / NG) % S;
        const int rl = threadIdx.x / (NG * S);
        // centre-first order: tile rank t -> (view, tile of the view) with the view's tiles
        // taken from its centre outwards (c, c + 1, c - 1, c + 2, ...; c the lower middle), so
        // that the longest rays run first and the launch ends on short ones
        const int tr = kOrder ? tile / a.nviews : 0;
        const int tb = (tpv_view - 1) / 2 + ((tr & 1) ? (tr + 1) / 2 : -(tr / 2));
        const int bin = tb * R + rl;
        // subset-local ray index u * NB + b
        const int ray = kOrder ? (tile % a.nviews) * NB + bin : tile * R + rl;
        const bool live = lane_ok && (kOrder ? bin < NB : ray < nrays);
        GroupSum<G, AR> acc;
        acc.zero();
        if (live) {
            const int slot = a.slot0 + ray / NB;
            const ViewGeo &vw = g.views[slot];
            const RayGeo &rg = g.rays[(size_t)a.slot0 * NB + ray];
            const int ds = vw.xdrive ? 1 : N;        // pixel stride along the driving axis
            const int cs = vw.xdrive ? N : 1;        // pixel stride along the cross axis
            const T *img = reinterpret_cast<const T *>(a.img) + (size_t)grp * G;
            const int Lc = (rg.nd + S - 1) / S;
            const int k0 = c * Lc, k1 = min(rg.nd, k0 + Lc);
            // sub-rays of the bin (SUB instantiations only; the others walk its centre line)
            const int nsr = SUB ? g.R : 1;
            if constexpr (AR == AR_FP64) {
                const double step = vw.step, ast = fabs(vw.step), L = vw.L, im = vw.inv_minor;
                for (int sr = 0; sr < nsr; ++sr)
                for (int k = k0; k < k1; ++k) {
                    const int d = rg.d0 + k;
                    const double lo = fma((double)k, step, rg.lo + (2 * sr + 1 - nsr) * (SUB ? rg.sh : vw.half));
                    const double hi = lo + ast;
                    const double f0 = floor(lo), f1 = floor(hi);
                    const int r0 = (int)f0, r1 = (int)f1;
                    double l1 = (r1 != r0) ? (hi - f1) * im : 0.0;
                    double l0 = L - l1;
                    const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                    l0 = ok0 ? l0 : 0.0;
                    l1 = ok1 ? l1 : 0.0;
                    T x0[G], x1[G];
                    load_group<G, T>(img + (unsigned)(d * ds + (ok0 ? r0 : 0) * cs) * (unsigned)Pp, x0);
                    load_group<G, T>(img + (unsigned)(d * ds + (ok1 ? r1 : 0) * cs) * (unsigned)Pp, x1);
                    acc.add2terms(l0, x0, l1, x1);
                }
            } else if constexpr (G == 8 && FWD_FAST) {
                // FP32 pairs, as below, with three changes: the fraction of the cross coordinate
                // is read from its top 23 bits as the mantissa of a float in [1, 2) (no integer-
                // to-float conversion), the pixel offsets advance incrementally along the driving
                // axis, and the compensated sum takes blocks of 8 steps summed by FMAs (one
                // compensated step per block instead of one per driving step)
                const long long stp = vw.stepq, ast = vw.absstepq;
                const float L = vw.Lf, imb = vw.inv_minorf;
                const float *imf = reinterpret_cast<const float *>(img);
                const unsigned dstep = (unsigned)ds * (unsigned)Pp, cstep = (unsigned)cs * (unsigned)Pp;
                f2x sm[4], er[4], bl[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { sm[q] = 0ull; er[q] = 0ull; bl[q] = 0ull; }
                auto merge = [&]() {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if constexpr (AR == AR_KAHAN) {
                            const f2x y = vadd(bl[q], er[q]);
                            const f2x t = vadd(sm[q], y);
                            er[q] = vsub(y, vsub(t, sm[q]));
                            sm[q] = t;
                        } else {
                            sm[q] = vadd(sm[q], bl[q]);
                        }
                        bl[q] = 0ull;
                    }
                };
                int nb = 0;
                for (int sr = 0; sr < nsr; ++sr) {
                unsigned base = (unsigned)(rg.d0 + k0) * dstep;
                long long lo = rg.loq + (long long)(2 * sr + 1 - nsr) * (SUB ? rg.shq : vw.halfq) + (long long)k0 * stp;
                for (int k = k0; k < k1; ++k) {
                    const long long hi = lo + ast;
                    const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
                    const bool cross = r1 != r0;
                    const bool ok0 = (unsigned)r0 < (unsigned)N;
                    const bool ok1 = cross && (unsigned)r1 < (unsigned)N;
                    const float fr = __uint_as_float(0x3F800000u | ((unsigned)hi >> 9)) - 1.f;
                    const float t1 = cross ? fr * imb : 0.f;
                    const float l1 = ok1 ? t1 : 0.f;
                    const float l0 = ok0 ? L - t1 : 0.f;
                    const unsigned o0 = base + (ok0 ? (unsigned)r0 * cstep : 0u);
                    const unsigned o1 = base + (ok1 ? (unsigned)r1 * cstep : 0u);
                    f2x x0[4], x1[4];
                    load8x(imf + o0, x0);
                    load8x_if(imf + o1, ok1, x1);
                    const f2x W0 = vsplat(l0), W1 = vsplat(l1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) bl[q] = vfma(W1, x1[q], vfma(W0, x0[q], bl[q]));
                    if (++nb == 8) { merge(); nb = 0; }
                    lo += stp;
                    base += dstep;
                }
                }
                merge();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float a0, a1, b0, b1;
                    vunpk(sm[q], a0, a1);
                    vunpk(er[q], b0, b1);
                    acc.set(2 * q, a0, b0);
                    acc.set(2 * q + 1, a1, b1);
                }
            } else if constexpr (G == 8) {
                // FP32 pairs; the second pixel of a step is read only when the line crosses
                // into it (l1 > 0), on about |slope| of the steps
                const long long stp = vw.stepq, ast = vw.absstepq;
                const float L = vw.Lf, im = vw.inv_minorf * kQ32;
                const float *imf = reinterpret_cast<const float *>(img);
                f2x sm[4], er[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { sm[q] = 0ull; er[q] = 0ull; }
                for (int sr = 0; sr < nsr; ++sr) {
                long long lo = rg.loq + (long long)(2 * sr + 1 - nsr) * (SUB ? rg.shq : vw.halfq) + (long long)k0 * stp;
                for (int k = k0; k < k1; ++k) {
                    const int d = rg.d0 + k;
                    const long long hi = lo + ast;
                    const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
                    const bool ok0 = (unsigned)r0 < (unsigned)N;
                    const bool ok1 = r1 != r0 && (unsigned)r1 < (unsigned)N;
                    const float l1 = ok1 ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f;
                    const float l0 = ok0 ? L - (r1 != r0 ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f) : 0.f;
                    f2x x0[4], x1[4];
                    load8x(imf + (unsigned)(d * ds + (ok0 ? r0 : 0) * cs) * (unsigned)Pp, x0);
                    load8x_if(imf + (unsigned)(d * ds + (ok1 ? r1 : 0) * cs) * (unsigned)Pp, ok1, x1);
                    const f2x W0 = vsplat(l0), W1 = vsplat(l1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if constexpr (AR == AR_KAHAN) {
                            const f2x y = vfma(W1, x1[q], vfma(W0, x0[q], er[q]));
                            const f2x t = vadd(sm[q], y);
                            er[q] = vsub(y, vsub(t, sm[q]));
                            sm[q] = t;
                        } else {
                            sm[q] = vfma(W1, x1[q], vfma(W0, x0[q], sm[q]));
                        }
                    }
                    lo += stp;
                }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float a0, a1, b0, b1;
                    vunpk(sm[q], a0, a1);
                    vunpk(er[q], b0, b1);
                    acc.set(2 * q, a0, b0);
                    acc.set(2 * q + 1, a1, b1);
                }
            } else {
                const long long stp = vw.stepq, ast = vw.absstepq;
                const float L = vw.Lf, im = vw.inv_minorf * kQ32;
                for (int sr = 0; sr < nsr; ++sr) {
                long long lo = rg.loq + (long long)(2 * sr + 1 - nsr) * (SUB ? rg.shq : vw.halfq) + (long long)k0 * stp;
                for (int k = k0; k < k1; ++k) {
                    const int d = rg.d0 + k;
                    const long long hi = lo + ast;
                    const int r0 = (int)(lo >> 32), r1 = (int)(hi >> 32);
                    float l1 = (r1 != r0) ? __uint2float_rn((unsigned)(hi & 0xFFFFFFFFLL)) * im : 0.f;
                    float l0 = L - l1;
                    const bool ok0 = (unsigned)r0 < (unsigned)N, ok1 = (unsigned)r1 < (unsigned)N;
                    l0 = ok0 ? l0 : 0.f;
                    l1 = ok1 ? l1 : 0.f;
                    T x0[G], x1[G];
                    load_group<G, T>(img + (unsigned)(d * ds + (ok0 ? r0 : 0) * cs) * (unsigned)Pp, x0);
                    load_group<G, T>(img + (unsigned)(d * ds + (ok1 ? r1 : 0) * cs) * (unsigned)Pp, x1);
                    acc.add2terms(l0, x0, l1, x1);
                    lo += stp;
                }
                }
            }
        }
        // combine the S chunks of each (ray, group) in chunk order
        T tot[G];
        if (S > 1) {
            __syncthreads();
#pragma unroll
            for (int p = 0; p < G; ++p) {
                comb_s[p * 256 + threadIdx.x] = acc.s_at(p);
                comb_e[p * 256 + threadIdx.x] = acc.e_at(p);
            }
            __syncthreads();
#pragma unroll
            for (int p = 0; p < G; ++p) {
                T s0 = acc.s_at(p), e0 = acc.e_at(p);
                if (c == 0 && lane_ok) {            // idle lanes (>= R S NG) have no chunks
                    for (int cc = 1; cc < S; ++cc) {
                        const int o = p * 256 + (rl * S + cc) * NG + grp;
                        if constexpr (AR == AR_KAHAN) {
                            const T y = comb_s[o] + (comb_e[o] + e0);
                            const T t = s0 + y;
                            e0 = y - (t - s0);
                            s0 = t;
                        } else {
                            s0 += comb_s[o];
                        }
                    }
                }
                tot[p] = s0 + e0;
            }
        } else {
#pragma unroll
            for (int p = 0; p < G; ++p) tot[p] = acc.value(p);
        }
        if (live && c == 0) {
            const size_t o = (size_t)ray * Pp + (size_t)grp * G;
            const T scale = (T)g.scale;
            if constexpr (MODE == FWD_PLAIN) {
                T y[G];
#pragma unroll
                for (int p = 0; p < G; ++p) y[p] = scale * tot[p];
                store_group<G, T>(reinterpret_cast<T *>(a.out) + o, y);
            } else {
                int cnt[G];
                float gam[G];
                load_group_i<G>(a.counts + o, cnt);
                load_group<G, float>(a.gamma + o, gam);
                // per-bin detection factors: the system matrix is diag(a) A, so the mean is
                // a_i (A f)_i + gamma_i and the backprojected ratio carries a_i (a_i = 1, exact
                // in the products, without factors)
                const float *mp = a.mult ? a.mult + o : nullptr;
                if constexpr (MODE == FWD_RATIO) {
                    T w[G];
#pragma unroll
                    for (int p = 0; p < G; ++p) {
                        const T m = mp ? (T)__ldg(mp + p) : T(1);
                        const T y = scale * (tot[p] * m) + (T)gam[p];
                        w[p] = (grp * G + p < g.P) ? m * (T(1) - (T)cnt[p] / y) : T(0);
                    }
                    store_group<G, T>(reinterpret_cast<T *>(a.out) + o, w);
                } else {
                    // the likelihood terms in FP64 in every mode: ln((double) Af + gamma)
                    T s_af = T(0);
                    double s_gl = 0.0;
#pragma unroll
                    for (int p = 0; p < G; ++p) {
                        if (grp * G + p < g.P) {
                            const T af = scale * (mp ? tot[p] * (T)__ldg(mp + p) : tot[p]);
                            s_af += af;
                            if (cnt[p] != 0) s_gl += (double)cnt[p] * log((double)af + (double)gam[p]);
                        }
                    }
                    obj[0] += (double)s_af;
                    obj[1] += s_gl;
                }
            }
        }
        }  // tiles of this virtual block
        if constexpr (MODE == FWD_OBJECTIVE) grid_reduce<2>(obj, a.red, a.result, vloc, nv);
    }
}

// One launch of a forward-projection instantiation; `pdl`: with programmatic stream
// serialization (the kernel waits for the previous kernel of the stream before its first
// memory access).
template <typename K>
static void fwd_launch(K kernel, int grid, cudaStream_t st, bool pdl, const FwdArgs &a, const Batch &b)
{
    if (!pdl) {
        kernel<<<grid, 256, 0, st>>>(a, b);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, a, b);
}

template <int G, int AR>
static void fwd_dispatch_mode(const FwdArgs &a, const Batch &b, int mode, int grid, cudaStream_t st,
                              bool pdl)
{
    if (a.g.table) {
        if (mode == FWD_PLAIN) fwd_launch(fwd_kernel<G, AR, FWD_PLAIN, true>, grid, st, pdl, a, b);
        else if (mode == FWD_RATIO) fwd_launch(fwd_kernel<G, AR, FWD_RATIO, true>, grid, st, pdl, a, b);
        else fwd_launch(fwd_kernel<G, AR, FWD_OBJECTIVE, true>, grid, st, pdl, a, b);
        return;
    }
    if (mode == FWD_PLAIN) fwd_launch(fwd_kernel<G, AR, FWD_PLAIN>, grid, st, pdl, a, b);
    else if (mode == FWD_RATIO) fwd_launch(fwd_kernel<G, AR, FWD_RATIO>, grid, st, pdl, a, b);
    else fwd_launch(fwd_kernel<G, AR, FWD_OBJECTIVE>, grid, st, pdl, a, b);
}

template <int G>
static void fwd_dispatch(const FwdArgs &a, const Batch &b, int mode, int arith, int grid,
                         cudaStream_t st, bool pdl = false)
{
    if (arith == AR_FP32) fwd_dispatch_mode<G, AR_FP32>(a, b, mode, grid, st, pdl);
    else if (arith == AR_KAHAN) fwd_dispatch_mode<G, AR_KAHAN>(a, b, mode, grid, st, pdl);
    else fwd_dispatch_mode<G, AR_FP64>(a, b, mode, grid, st, pdl);
}

template <int G, int AR>
static const void *fwd_fn_mode(int mode, int sub)
{
    if (sub) {
        if (mode == FWD_PLAIN) return (const void *)fwd_kernel<G, AR, FWD_PLAIN, true>;
        if (mode == FWD_RATIO) return (const void *)fwd_kernel<G, AR, FWD_RATIO, true>;
        return (const void *)fwd_kernel<G, AR, FWD_OBJECTIVE, true>;
    }
    if (mode == FWD_PLAIN) return (const void *)fwd_kernel<G, AR, FWD_PLAIN>;
    if (mode == FWD_RATIO) return (const void *)fwd_kernel<G, AR, FWD_RATIO>;
    return (const void *)fwd_kernel<G, AR, FWD_OBJECTIVE>;
}

template <int G>
static const void *fwd_fn_g(int mode, int arith, int sub)
{
    if (arith == AR_FP32) return fwd_fn_mode<G, AR_FP32>(mode, sub);
    if (arith == AR_KAHAN) return fwd_fn_mode<G, AR_KAHAN>(mode, sub);
    return fwd_fn_mode<G, AR_FP64>(mode, sub);
}

// Resident 256-thread blocks per SM of one kernel instantiation (cached per function).
int resident_blocks(const void *fn)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &c : cache)
        if (c.first == fn) return c.second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 256, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cache.emplace_back(fn, n);
    return n;
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

// Chunks per ray (S, at most FWD_MAX_CHUNKS) so that one subset projection has about one
// full-occupancy wave of threads, with >= 16 driving steps per chunk; R rays per 256-thread virtual block.  The
// objective mode groups its ray tiles into one wave of virtual blocks (each ends in a reduction
// step), never more than its reducer holds partial sums for.
void forward_shape(FwdArgs &a, int mode, int arith)
{
    if (a.g.T > 1) { forward_shape_tof(a, mode, arith); return; }
    const long long nrays = (long long)a.nviews * a.g.NB;
    const long long want = (long long)sm_count() * 2048;
    const long long have = std::max<long long>(1, nrays * a.g.NG);
    int S = (int)std::min<long long>(FWD_MAX_CHUNKS, std::max<long long>(1, (want + have - 1) / have));
    S = std::max(1, std::min(S, a.g.N / 16));
    if (a.g.tuneS > 0 && mode != FWD_OBJECTIVE) S = a.g.tuneS;
    while (S > 1 && (256 / a.g.NG) % S) --S;          // S divides the rays-per-block budget
    a.S = S;
    a.R = std::max(1, 256 / (S * a.g.NG));
    const bool order = FWD_TILE_ORDER && (mode != FWD_OBJECTIVE || FWD_TILE_ORDER > 1);
    const long long ntiles = order ? (long long)a.nviews * ((a.g.NB + a.R - 1) / a.R)
                                   : (nrays + a.R - 1) / a.R;
    a.tpv = 1;
    if (mode == FWD_OBJECTIVE) {
        // each virtual block ends in a block reduction and a grid-wide ticket: one wave of them
        const void *fn = a.g.G == 1 ? fwd_fn_g<1>(mode, arith, a.g.table) : fwd_fn_g<8>(mode, arith, a.g.table);
        const long long slots = (long long)sm_count() * resident_blocks(fn);
        long long tpv = (ntiles + slots - 1) / slots;
        if (a.red.capacity > 0) tpv = std::max(tpv, (ntiles + a.red.capacity - 1) / a.red.capacity);
        a.tpv = (int)std::max(1LL, tpv);
    }
    a.nvb = (int)((ntiles + a.tpv - 1) / a.tpv);
}

pet_status launch_forward(const FwdArgs &a0, int mode, int arith, cudaStream_t st,
                          bool after_kernel)
{
    if (a0.g.T > 1) return launch_forward_tof(a0, mode, arith, st);
    FwdArgs a = a0;
    const long long nrays = (long long)a.nviews * a.g.NB;
    if (nrays == 0) return PET_OK;
    forward_shape(a, mode, arith);
    const int grid = std::max(1, std::min(a.nvb, sm_count() * 8));
    Batch b{nullptr, nullptr, 0, grid};
    LaunchScope ls(mode == FWD_RATIO ? PET_K_FORWARD_RATIO
                   : (mode == FWD_OBJECTIVE ? PET_K_OBJ_FORWARD : PET_K_OTHER), st);
    if (a.g.G == 1) fwd_dispatch<1>(a, b, mode, arith, grid, st, after_kernel);
    else fwd_dispatch<8>(a, b, mode, arith, grid, st, after_kernel);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fwd_kernel launch");
    return PET_OK;
}

// Batched launch: all scans share the plane-group size of `shape` (G and the kernel template).
pet_status launch_forward_batch(const FwdArgs &shape, const Batch &b, int mode, int arith,
                                cudaStream_t st)
{
    if (shape.g.T > 1) return launch_forward_tof_batch(shape, b, mode, arith, st);
    LaunchScope ls(mode == FWD_RATIO ? PET_K_FORWARD_RATIO
                   : (mode == FWD_OBJECTIVE ? PET_K_OBJ_FORWARD : PET_K_OTHER), st);
    if (shape.g.G == 1) fwd_dispatch<1>(shape, b, mode, arith, b.grid, st);
    else fwd_dispatch<8>(shape, b, mode, arith, b.grid, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fwd_kernel batch launch");
    return PET_OK;
}

}  // namespace pet

using namespace pet;

// Autotuner: times the subset-0 forward projection of an image of ones for every admissible
// chunk count S (1..16, dividing the 256-thread block budget; best of 7 runs of 4 launches, or
// of 5 single launches of the batched copies) and
// keeps the fastest in the geometry, a larger S only when it is faster by more than 3 %.
// `concurrent` copies of the projection run as one batched launch (the persistent grid of
// pet_batch), so that a geometry whose scans run in a batch is tuned with the GPU shared the way
// the batch shares it; concurrent = 1 is a scan alone.  The choice is per geometry, so
// every scan using it (alone or batched) runs the same shapes and computes the same bits.
static pet_status autotune_any(pet_geometry *g, int concurrent, cudaStream_t st, int *best_S)
{
    GeoDev &gd = g->dev;
    if (gd.T > 1) {                      // the TOF projector has no ray chunking to tune
        gd.tuneS = 0;
        if (best_S) *best_S = 1;
        return PET_OK;
    }
    const int nv = g->voff[1] - g->voff[0];
    const size_t qb = ((size_t)gd.N * gd.N * gd.Pp * 4 + 255) / 256 * 256;
    const size_t pb = ((size_t)nv * gd.NB * gd.Pp * 4 + 255) / 256 * 256;
    const size_t ab = ((size_t)concurrent * sizeof(FwdArgs) + 255) / 256 * 256;
    const size_t prb = ((size_t)(concurrent + 1) * sizeof(int) + 255) / 256 * 256;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, qb + (size_t)concurrent * pb + ab + prb, &scr));
    char *base = reinterpret_cast<char *>(scr);
    char *img = base, *outs = base + qb;
    FwdArgs *d_args = reinterpret_cast<FwdArgs *>(outs + (size_t)concurrent * pb);
    int *d_pre = reinterpret_cast<int *>(reinterpret_cast<char *>(d_args) + ab);
    PET_TRY(fill_internal_ones(gd, img, 0, st));
    std::vector<FwdArgs> h_args(concurrent);
    std::vector<int> h_pre(concurrent + 1);
    cudaEvent_t a, b;
    PET_CUDA(cudaEventCreate(&a));
    PET_CUDA(cudaEventCreate(&b));
    float best = 1e30f;
    int bestS = 0;
    const int save = gd.tuneS;
    pet_status r = PET_OK;
    for (int S = 1; S <= FWD_MAX_CHUNKS && r == PET_OK; ++S) {
        if ((256 / gd.NG) % S) continue;
        gd.tuneS = S;
        FwdArgs fa{};
        fa.g = gd;
        fa.slot0 = g->voff[0];
        fa.nviews = nv;
        fa.img = img;
        forward_shape(fa, FWD_PLAIN, AR_KAHAN);
        for (int c = 0; c < concurrent; ++c) {
            h_args[c] = fa;
            h_args[c].out = outs + (size_t)c * pb;
            h_pre[c] = c * fa.nvb;
        }
        h_pre[concurrent] = concurrent * fa.nvb;
        r = cuda_ok(cudaMemcpyAsync(d_args, h_args.data(), sizeof(FwdArgs) * concurrent,
                                    cudaMemcpyHostToDevice, st), "pet_autotune: arguments");
        if (r == PET_OK)
            r = cuda_ok(cudaMemcpyAsync(d_pre, h_pre.data(), sizeof(int) * (concurrent + 1),
                                        cudaMemcpyHostToDevice, st), "pet_autotune: arguments");
        const Batch bt{d_args, d_pre, concurrent, sm_count() * 4};
        auto once = [&]() {
            return concurrent == 1 ? launch_forward(h_args[0], FWD_PLAIN, AR_KAHAN, st)
                                   : launch_forward_batch(fa, bt, FWD_PLAIN, AR_KAHAN, st);
        };
        if (r == PET_OK) r = once();                         // warm-up
        float tmin = 1e30f;
        // a scan alone: runs of 4 launches (one is ~50 us); batched copies: one launch a run
        // (each takes milliseconds, and a server tunes every geometry it meets)
        const int per_run = concurrent == 1 ? 4 : 1;
        for (int rep = 0; rep < (concurrent == 1 ? 7 : 5) && r == PET_OK; ++rep) {
            cudaEventRecord(a, st);
            for (int k = 0; k < per_run && r == PET_OK; ++k) r = once();
            cudaEventRecord(b, st);
            if (r == PET_OK) r = cuda_ok(cudaEventSynchronize(b), "pet_autotune: timing");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            tmin = std::min(tmin, ms);
        }
        // a larger S must win by more than 3 %: timings that close are noise, and fewer chunks
        // leave more of the GPU to whatever runs beside the projection
        if (r == PET_OK && tmin < best * 0.97f) { best = tmin; bestS = S; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r != PET_OK) { gd.tuneS = save; return r; }
    gd.tuneS = bestS;
    if (best_S) *best_S = bestS;
    return PET_OK;
}

extern "C" pet_status pet_autotune(pet_geometry *g, void *stream, int *best_S)
{
    if (!g) return fail(PET_ERR_INVALID, "pet_autotune: NULL geometry");
    return autotune_any(g, 1, as_stream(stream), best_S);
}

extern "C" pet_status pet_autotune_batch(pet_geometry *g, int concurrent, void *stream, int *best_S)
{
    if (!g) return fail(PET_ERR_INVALID, "pet_autotune_batch: NULL geometry");
    if (concurrent < 1 || concurrent > 4096)
        return fail(PET_ERR_INVALID, "pet_autotune_batch: need 1 <= concurrent <= 4096");
    return autotune_any(g, concurrent, as_stream(stream), best_S);
}

extern "C" pet_status pet_set_ray_chunks(pet_geometry *g, int S)
{
    if (!g) return fail(PET_ERR_INVALID, "pet_set_ray_chunks: NULL geometry");
    if (S < 0 || S > FWD_MAX_CHUNKS || (S > 0 && (256 / g->dev.NG) % S))
        return fail(PET_ERR_INVALID, "pet_set_ray_chunks: S must be 0 or in 1..16 and divide 256 / plane groups");
    g->dev.tuneS = S;
    return PET_OK;
}
