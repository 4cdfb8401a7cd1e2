// Reconstruction state and the SDP-BSREM subiteration (Table I), the whole-reconstruction
// entry points, and the stand-alone projector / step calls of the C ABI.
//
// Per subiteration (k, i), J = kM + i, subset I_i:
//   host FP64: lambda_k = lambda0 / (a k + 1) (Theorem 2); alpha_{k,i} (Eq.
//     preconditioner:Nesterov or preconditioner:KM); the nu mode of Eq. nuki;
//   [J0 < J <= J1] mu pass: sum of mu = max(0.01, grad(f)/mean(f)) in FP64 (Sec. III);
//   forward + ratio: w = 1 - g_i / (A_i f + gamma_i) (App. A);
//   fused update: f <- P_t(f - lambda_k alpha_{k,i} nu S(f) (A_i^T w + (beta/M) grad R(f)))
//     with the FP64 sum of the new f (feeds mean(f) of the next mu pass).
// Everything stays on the device; the scalars travel as kernel arguments.
#include <math.h>

#include <cstring>

#include "pet_common.cuh"
#include "profile.cuh"

using namespace pet;

static const int kRedCap = 4096;   // reduction partials per scan

pet_status pet::check_params(const pet_params *p)
{
    if (!p) return fail(PET_ERR_INVALID, "pet_params is NULL");
    if (p->iterations < 0 || !(p->beta >= 0) || !(p->gamma_r >= 0) || !(p->eps > 0) ||
        !(p->U > 0) || !(p->t > 0) || !(p->t < p->U) || !(p->lambda0 > 0) || !(p->a >= 0) ||
        !(p->nu1 > 0) || !(p->nu2 >= p->nu1) || p->precond < 0 || p->precond > 4 ||
        p->precision < 0 || p->precision > 2 || !(p->delta1 > 0) || !(p->rho > 0) ||
        !(p->delta2 > 0) || p->J0 < 0 || p->J1 < p->J0 || p->rdp_3d < 0 || p->rdp_3d > 1 ||
        p->regularizer < 0 || p->regularizer > 1 ||
        (p->regularizer == PET_REG_TV && (p->tv_iters < 1 || p->tv_iters > 10000 || p->rdp_3d)))
        return fail(PET_ERR_INVALID,
                    "invalid pet_params (need iterations >= 0, beta, gamma_r, a >= 0, eps, "
                    "lambda0, rho, delta1, delta2 > 0, 0 < t < U, 0 < nu1 <= nu2, "
                    "0 <= J0 <= J1, precond in 0..4, precision in 0..2, rdp_3d in 0..1, "
                    "regularizer in 0..1, TV: 1 <= tv_iters <= 10000 and rdp_3d = 0)");
    return PET_OK;
}

static void state_free(pet_state *s)
{
    if (!s) return;
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
        cudaEventDestroy(s->ev_fork);
        cudaEventDestroy(s->ev_join);
        s->side = nullptr;
        s->ev_fork = s->ev_join = nullptr;
    }
    if (s->hstream) {
        cudaStreamSynchronize(s->hstream);
        cudaStreamDestroy(s->hstream);
        cudaEventDestroy(s->ev_h0);
        cudaEventDestroy(s->ev_h1);
        s->hstream = nullptr;
        s->ev_h0 = s->ev_h1 = nullptr;
    }
    if (s->ostream) {
        cudaStreamSynchronize(s->ostream);
        cudaStreamDestroy(s->ostream);
        cudaEventDestroy(s->ev_ofork);
        cudaEventDestroy(s->ev_odone);
        cudaFree(s->fobj);
        cudaFree(s->redobj_mem);
        s->ostream = nullptr;
        s->ev_ofork = s->ev_odone = nullptr;
        s->fobj = s->redobj_mem = nullptr;
        s->obj_pending = false;
    }
    auto rel = [&](void *p) {
        if (!p) return;
        if (s->alloc_stream) cudaFreeAsync(p, s->alloc_stream);
        else cudaFree(p);
    };
    rel(s->f[0]);
    rel(s->f[1]);
    rel(s->w);
    rel(s->counts);
    rel(s->gamma);
    rel(s->nu_frozen);
    rel(s->sums);
    rel(s->objhist);
    rel(s->redmem);
    rel(s->flag);
    rel(s->tvmem);
    rel(s->mult);
    rel(s->invp_vox);
    s->tvmem = nullptr;
    s->mult = nullptr;
    s->invp_vox = nullptr;
    s->attn = false;
    s->f[0] = s->f[1] = s->w = s->nu_frozen = s->redmem = nullptr;
    s->counts = nullptr;
    s->gamma = nullptr;
    s->sums = s->objhist = nullptr;
    s->flag = nullptr;
}

// (Re)allocate the state's buffers for geometry g and arithmetic `arith` (no-op when they fit);
// tv: also the buffers of the TV variant's proximal step (z, W, xbar and the dual variable);
// attn: also the per-bin detection factors and the per-voxel 1 / p_j they imply.
static pet_status state_alloc(pet_state *s, const pet_geometry *g, int arith, int iterations,
                              bool tv = false, bool attn = false)
{
    const GeoDev &gd = g->dev;
    const size_t esz = arith == AR_FP64 ? 8 : 4;
    const size_t q_bytes = (size_t)gd.N * gd.N * gd.Pp * esz;
    int maxv = 0;
    for (int i = 0; i < gd.M; ++i) maxv = std::max(maxv, g->voff[i + 1] - g->voff[i]);
    const size_t w_bytes = (size_t)maxv * gd.SB * gd.Pp * esz;
    const size_t sino = (size_t)gd.V * gd.SB * gd.Pp;
    if (s->g == g && s->esz == esz && s->f[0] && s->objcap >= iterations + 1 && (!tv || s->tvmem) &&
        (!attn || s->mult)) {
        s->arith = arith;
        return PET_OK;
    }
    state_free(s);
    s->g = g;
    s->esz = esz;
    s->arith = arith;
    s->q_bytes = q_bytes;
    s->w_bytes = w_bytes;
    s->sino_elems = sino;
    cudaStream_t as = s->alloc_stream;
    auto get = [&](void **p, size_t n) -> cudaError_t {
        return as ? dev_malloc_async(p, n, as) : dev_malloc(p, n);
    };
    PET_CUDA(get(&s->f[0], q_bytes));
    PET_CUDA(get(&s->f[1], q_bytes));
    PET_CUDA(get(&s->w, w_bytes));
    PET_CUDA(get((void **)&s->counts, sino * sizeof(int)));
    PET_CUDA(get((void **)&s->gamma, sino * sizeof(float)));
    PET_CUDA(get(&s->nu_frozen, q_bytes));
    PET_CUDA(get((void **)&s->sums, 16 * sizeof(double)));
    s->objcap = std::max(iterations + 1, 1);
    PET_CUDA(get((void **)&s->objhist, (size_t)s->objcap * 3 * sizeof(double)));
    PET_CUDA(get(&s->redmem, reducer_bytes(kRedCap, 2)));
    PET_CUDA(cudaMemsetAsync(s->redmem, 0, reducer_bytes(kRedCap, 2), as));
    reducer_bind(s->red, s->redmem, kRedCap, 2);
    PET_CUDA(get((void **)&s->flag, sizeof(int)));
    if (tv) PET_CUDA(get(&s->tvmem, 5 * q_bytes));
    if (attn) {
        PET_CUDA(get((void **)&s->mult, sino * sizeof(float)));
        PET_CUDA(get(&s->invp_vox, q_bytes));
    }
    if (!as) PET_CUDA(cudaStreamSynchronize(nullptr));
    return PET_OK;
}

// TV variant: the dual variable starts at zero with every (re)started reconstruction.
static pet_status tv_reset(pet_state *s, cudaStream_t st)
{
    if (s->prm.regularizer != PET_REG_TV) return PET_OK;
    if (!s->tvmem) return fail(PET_ERR_INVALID, "TV variant: state has no TV buffers");
    PET_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(s->tvmem) + 3 * s->q_bytes, 0, 2 * s->q_bytes, st));
    return PET_OK;
}

static pet_status state_sum_f(pet_state *s, cudaStream_t st)
{
    ImageArgs a{};
    a.g = s->g->dev;
    a.f = s->f[s->cur];
    a.result = s->sums + s->cur;
    a.red = s->red;
    return launch_sum(a, s->arith, st);
}

// 1 / p_j per voxel from the FP64 backprojection bp = A^T a (Eq. pj for diag(a) A).
template <typename T>
__global__ void finish_sensitivity_vox(const double *bp, size_t q, int M, T *invp)
{
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= q) return;
    const double v = bp[j];
    invp[j] = (T)(1.0 / (v > 0.0 ? v / M : 1.0 / M));
}

// The per-bin detection factors of a scan ([P][V][NB], device): their internal copy, and
// p_j = (A^T a)_j / M per voxel (1/M where it is 0) by one FP64 backprojection of a over all
// views, kept as 1 / p_j in the state's arithmetic.
static pet_status load_factors(pet_state *s, const float *d_mult, cudaStream_t st)
{
    const pet_geometry *g = s->g;
    const GeoDev &gd = g->dev;
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_mult, s->mult, 2, 0, st));
    const size_t nsino = (size_t)gd.V * gd.SB * gd.Pp, q = (size_t)gd.N * gd.N * gd.Pp;
    double *ad = nullptr, *bp = nullptr;
    PET_CUDA(dev_malloc_async((void **)&ad, nsino * sizeof(double), st));
    pet_status r = cuda_ok(dev_malloc_async((void **)&bp, q * sizeof(double), st),
                           "per-voxel sensitivity");
    if (r == PET_OK) r = to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_mult, ad, 4, 0, st);
    if (r == PET_OK) {
        BackArgs ba{};
        ba.g = gd;
        ba.slot0 = 0;
        ba.nviews = gd.V;
        ba.proj = ad;
        ba.img = bp;
        r = launch_back(ba, AR_FP64, st);
    }
    if (r == PET_OK) {
        LaunchScope ls(PET_K_OTHER, st);
        const unsigned blk = (unsigned)((q + 255) / 256);
        if (s->arith == AR_FP64)
            finish_sensitivity_vox<double><<<blk, 256, 0, st>>>(bp, q, gd.M, (double *)s->invp_vox);
        else
            finish_sensitivity_vox<float><<<blk, 256, 0, st>>>(bp, q, gd.M, (float *)s->invp_vox);
        r = cuda_ok(cudaGetLastError(), "finish_sensitivity_vox");
    }
    if (ad) cudaFreeAsync(ad, st);
    if (bp) cudaFreeAsync(bp, st);
    return r;
}

// Load data (counts, gamma and, when not NULL, the per-bin detection factors mult: [P][V][NB],
// device) and f^0 ([P][N][N] float, device) into an allocated state and reset the schedule to
// (k, i) = (0, 1).  Validates the data (synchronises).
static pet_status state_load(pet_state *s, const int32_t *d_counts, const float *d_gamma,
                             const float *d_mult, const pet_params *p, const float *d_img,
                             cudaStream_t st, bool validate)
{
    const pet_geometry *g = s->g;
    const GeoDev &gd = g->dev;
    s->prm = *p;
    if (d_mult && !s->mult) return fail(PET_ERR_INVALID, "state has no buffers for detection factors");
    if (validate) {
        const size_t n = (size_t)gd.P * gd.V * gd.SB;
        PET_TRY(validate_data(gd, d_counts, d_gamma, n, s->flag, st));
        if (d_mult) PET_TRY(validate_factors(d_mult, n, s->flag, st));
        int h = 0;
        PET_CUDA(cudaMemcpyAsync(&h, s->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        PET_CUDA(cudaStreamSynchronize(st));
        if (h) return fail(PET_ERR_INVALID, "data check failed: need counts >= 0, 0 < gamma < inf "
                                            "and finite detection factors >= 0");
    }
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_counts, s->counts, 0, 0, st));
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_gamma, s->gamma, 1, 0, st));
    s->attn = d_mult != nullptr;
    if (d_mult) PET_TRY(load_factors(s, d_mult, st));
    s->cur = 0;
    PET_TRY(to_internal_image(gd, d_img, s->f[0], 0, s->arith == AR_FP64, st));
    s->k = s->i = s->J = 0;
    s->tn = 1.0;
    s->have_frozen = false;
    PET_TRY(tv_reset(s, st));
    return state_sum_f(s, st);
}

// Plan the next subiteration of s (host FP64 scalars, argument structs) and advance its
// schedule.  Shapes depend on the scan alone, so a scan computes the same bits on its own and
// inside any batch.  with_objective: also plan Phi(f^{k+1}) when this subiteration ends an
// outer iteration (written to objhist[3 (k+1) ..]).
void pet::plan_subiter(pet_state *s, SubiterPlan *pl, bool with_objective)
{
    const pet_geometry *g = s->g;
    const pet_params &p = s->prm;
    const int M = g->dev.M;
    const int J = s->k * M + s->i + 1;                 // J_{k,i} = kM + i (1-based i)
    const double lam = p.lambda0 / (p.a * s->k + 1.0);
    double alpha = 1.0;
    if (p.precond == PET_PRECOND_M1 || p.precond == PET_PRECOND_P1) {
        const double tn1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * s->tn * s->tn));
        alpha = 1.0 + (s->tn - 1.0) / tn1;
        s->tn = tn1;
    } else if (p.precond == PET_PRECOND_M2 || p.precond == PET_PRECOND_P2) {
        alpha = (p.rho * (J - 1) + p.delta2) / ((double)(J - 1) + p.delta1);
    }
    const bool use_nu = p.precond == PET_PRECOND_P1 || p.precond == PET_PRECOND_P2;
    int nu_mode = 0;
    if (use_nu && J > p.J0) {
        if (J <= p.J1) nu_mode = (J == p.J1) ? 2 : 1;
        else nu_mode = s->have_frozen ? 3 : 0;
    }
    const int slot0 = g->voff[s->i], nv = g->voff[s->i + 1] - g->voff[s->i];
    *pl = SubiterPlan{};
    GeoDev gd = g->dev;
    gd.scale *= s->sens_ratio;
    pl->arith = s->arith;
    pl->mu = nu_mode == 1 || nu_mode == 2;
    ImageArgs &a = pl->mu_args;
    a.g = gd;
    a.f = s->f[s->cur];
    a.sum_f = s->sums + s->cur;
    a.result = s->sums + 2;
    a.red = s->red;
    a.z3 = p.rdp_3d;
    mu_shape(a, s->arith);
    FwdArgs &fa = pl->fwd;
    fa.g = gd;
    fa.slot0 = slot0;
    fa.nviews = nv;
    fa.img = s->f[s->cur];
    fa.out = s->w;
    fa.counts = s->counts + (size_t)slot0 * gd.SB * gd.Pp;
    fa.gamma = s->gamma + (size_t)slot0 * gd.SB * gd.Pp;
    fa.mult = s->attn ? s->mult + (size_t)slot0 * gd.SB * gd.Pp : nullptr;
    forward_shape(fa, FWD_RATIO, s->arith);
    UpdateArgs &ua = pl->upd;
    ua.g = update_geo(gd);
    ua.slot0 = slot0;
    ua.nviews = nv;
    ua.w = s->w;
    ua.f = s->f[s->cur];
    ua.fout = s->f[1 - s->cur];
    ua.invp = s->attn ? (const void *)s->invp_vox
                      : (s->arith == AR_FP64 ? (const void *)g->d_invp64 : (const void *)g->d_invp);
    ua.vox = s->attn ? 1 : 0;
    ua.bptab = g->d_bptab && s->arith != AR_FP64 ? static_cast<const char *>(g->d_bptab) +
                                                       g->bptab_off[s->i]
                                                 : nullptr;
    ua.invp_scale = 1.0 / s->sens_ratio;
    ua.nu_frozen = s->nu_frozen;
    ua.nu_mode = nu_mode;
    ua.lam_alpha = lam * alpha;
    ua.beta_over_M = p.beta / M;
    ua.gamma_r = p.gamma_r;
    ua.eps = p.eps;
    ua.t = p.t;
    ua.U = p.U;
    ua.nu1 = p.nu1;
    ua.nu2 = p.nu2;
    ua.sum_f = s->sums + s->cur;
    ua.sum_mu = s->sums + 2;
    ua.sum_fout = s->sums + (1 - s->cur);
    ua.red = s->red;
    ua.z3 = p.rdp_3d;
    pl->tv = p.regularizer == PET_REG_TV;
    if (pl->tv) {
        // TV variant: the update writes z = f - W grad F_i and W; the proximal step follows
        char *tvm = reinterpret_cast<char *>(s->tvmem);
        ua.tv = 1;
        ua.beta_over_M = 0.0;
        ua.zbuf = tvm;
        ua.wbuf = tvm + s->q_bytes;
        TvArgs &ta = pl->tv_args;
        ta.g = gd;
        ta.x = ua.fout;
        ta.z = tvm;
        ta.w = tvm + s->q_bytes;
        ta.xbar = tvm + 2 * s->q_bytes;
        ta.px = tvm + 3 * s->q_bytes;
        ta.py = tvm + 4 * s->q_bytes;
        ta.b = p.beta / M;
        ta.t = p.t;
        ta.U = p.U;
        ta.red = s->red;
        ta.sum_out = ua.sum_fout;
        tv_shape(ta);
        pl->tv_iters = ta.b > 0 ? p.tv_iters : 0;
    }
    update_shape(ua, s->arith);
    update_fp32_scalars(ua);
    if (nu_mode == 2) s->have_frozen = true;
    s->cur ^= 1;
    s->J = J;
    const bool iter_end = (s->i + 1 == M);
    if (++s->i == M) { s->i = 0; ++s->k; }
    pl->objective = with_objective && iter_end && s->k < s->objcap;
    if (pl->objective) objective_args(s, s->objhist + 3 * s->k, &pl->obj_fwd, &pl->obj_rdp);
}

// TV variant: the proximal step on the update's z (beta = 0: P_t(z)).
static pet_status tv_step(const SubiterPlan &pl, cudaStream_t st)
{
    if (!pl.tv) return PET_OK;
    return launch_tv_prox(pl.tv_args, pl.tv_iters, pl.arith, st);
}

// The mu pass and the forward projection only read f^{k,i-1}: the mu pass runs on a side stream
// forked from `st` and joined before the update.
static pet_status state_subiter(pet_state *s, cudaStream_t st)
{
    TraceRange tr("pet_subiter");
    SubiterPlan pl;
    plan_subiter(s, &pl, false);
    if (pl.mu && profile_active()) {
        PET_TRY(launch_mu_sum(pl.mu_args, pl.arith, st));
        PET_TRY(launch_forward(pl.fwd, FWD_RATIO, pl.arith, st));
        PET_TRY(launch_update(pl.upd, pl.arith, st));
        return tv_step(pl, st);
    }
    if (pl.mu) {
        if (!s->side) {
            int lo = 0, hi = 0;
            PET_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            PET_CUDA(cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, hi));
            PET_CUDA(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
            PET_CUDA(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
        }
        PET_CUDA(cudaEventRecord(s->ev_fork, st));
        PET_CUDA(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
        PET_TRY(launch_mu_sum(pl.mu_args, pl.arith, s->side));
        PET_CUDA(cudaEventRecord(s->ev_join, s->side));
    }
    // the projection follows the previous subiteration's update on `st` (or the host's own
    // work, where the launch attribute has no effect): see launch_forward
    PET_TRY(launch_forward(pl.fwd, FWD_RATIO, pl.arith, st, true));
    if (pl.mu) PET_CUDA(cudaStreamWaitEvent(st, s->ev_join, 0));
    PET_TRY(launch_update(pl.upd, pl.arith, st));
    return tv_step(pl, st);
}

// Argument structs for Phi(current f): parts sum(Af), sum(g ln(Af+gamma)) -> out3[0..1],
// R(f) -> out3[2].
void pet::objective_args(pet_state *s, double *out3, FwdArgs *fa, ImageArgs *ra)
{
    GeoDev gd = s->g->dev;
    gd.scale *= s->sens_ratio;
    *fa = FwdArgs{};
    fa->g = gd;
    fa->slot0 = 0;
    fa->nviews = gd.V;
    fa->img = s->f[s->cur];
    fa->counts = s->counts;
    fa->gamma = s->gamma;
    fa->mult = s->attn ? s->mult : nullptr;
    fa->red = s->red;
    fa->result = out3;
    forward_shape(*fa, FWD_OBJECTIVE, s->arith);
    *ra = ImageArgs{};
    ra->g = gd;
    ra->f = s->f[s->cur];
    ra->gamma_r = s->prm.gamma_r;
    ra->eps = s->prm.eps;
    ra->result = out3 + 2;
    ra->red = s->red;
    ra->z3 = s->prm.rdp_3d;
    ra->tv = s->prm.regularizer == PET_REG_TV;
    image_shape(*ra);
}

static pet_status state_objective_async(pet_state *s, double *out3, cudaStream_t st)
{
    FwdArgs fa;
    ImageArgs ra;
    objective_args(s, out3, &fa, &ra);
    PET_TRY(launch_forward(fa, FWD_OBJECTIVE, s->arith, st));
    return launch_rdp_value(ra, s->arith, st);
}

static int arith_of(int precision)
{
    return precision == PET_PREC_FP64 ? AR_FP64 : (precision == PET_PREC_FP32 ? AR_FP32 : AR_KAHAN);
}

// Internal creation for the serving loop: allocate a state for geometry g and parameters p and
// load it from device buffers in the C-ABI layouts (d_img may be NULL: f^0 = 1).  The data were
// validated by the caller.  sens: this scan's sensitivity (may differ from the geometry's).
pet_status pet::state_create_loaded(const pet_geometry *g, double sens, const int32_t *d_counts,
                                    const float *d_gamma, const float *d_mult, const float *d_img,
                                    const pet_params *p, cudaStream_t st, pet_state **out)
{
    *out = nullptr;
    PET_TRY(check_params(p));
    pet_state *s = new pet_state();
    s->alloc_stream = st;                       // stream-ordered memory: no device-wide syncs
    pet_status r = state_alloc(s, g, arith_of(p->precision), p->iterations, false, d_mult != nullptr);
    if (r == PET_OK) {
        s->sens_ratio = sens / g->desc.sens;
        if (d_img) {
            r = state_load(s, d_counts, d_gamma, d_mult, p, d_img, st, false);
        } else {
            // f^0 = 1: fill the internal image, then load data
            s->prm = *p;
            const GeoDev &gd = g->dev;
            r = to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_counts, s->counts, 0, 0, st);
            if (r == PET_OK) r = to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_gamma, s->gamma, 1, 0, st);
            s->attn = d_mult != nullptr;
            if (r == PET_OK && d_mult) r = load_factors(s, d_mult, st);
            if (r == PET_OK) r = fill_internal_ones(gd, s->f[0], s->arith == AR_FP64, st);
            s->cur = 0;
            s->k = s->i = s->J = 0;
            s->tn = 1.0;
            s->have_frozen = false;
            if (r == PET_OK) r = state_sum_f(s, st);
        }
    }
    if (r != PET_OK) {
        std::string msg = pet_last_error();
        state_free(s);
        delete s;
        return fail(r, msg);
    }
    *out = s;
    return PET_OK;
}

size_t pet::state_bytes(const pet_geometry *g, int precision, int iterations)
{
    const GeoDev &gd = g->dev;
    const size_t esz = precision == PET_PREC_FP64 ? 8 : 4;
    const size_t q = (size_t)gd.N * gd.N * gd.Pp * esz;
    int maxv = 0;
    for (int i = 0; i < gd.M; ++i) maxv = std::max(maxv, g->voff[i + 1] - g->voff[i]);
    const size_t sino = (size_t)gd.V * gd.SB * gd.Pp;
    return 3 * q + (size_t)maxv * gd.SB * gd.Pp * esz + sino * 8 + reducer_bytes(kRedCap, 2) +
           (size_t)(iterations + 1) * 24 + 1024;
}

void pet::state_release(pet_state *s, cudaStream_t st)
{
    if (s->alloc_stream) s->alloc_stream = st;  // free in the order of the last user's stream
    state_free(s);
    delete s;
}

static pet_status state_create_any(const pet_geometry *g, const int32_t *d_counts,
                                   const float *d_gamma, const float *d_mult,
                                   const pet_params *params, const float *d_img_init,
                                   void *stream, pet_state **out)
{
    if (!g || !d_counts || !d_gamma || !d_img_init || !out)
        return fail(PET_ERR_INVALID, "pet_state_create: NULL argument");
    *out = nullptr;
    PET_TRY(check_params(params));
    cudaStream_t st = as_stream(stream);
    pet_state *s = new pet_state();
    pet_status r = state_alloc(s, g, arith_of(params->precision), params->iterations,
                               params->regularizer == PET_REG_TV, d_mult != nullptr);
    if (r == PET_OK) r = state_load(s, d_counts, d_gamma, d_mult, params, d_img_init, st, true);
    if (r == PET_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "pet_state_create");
    }
    if (r != PET_OK) {
        std::string msg = pet_last_error();
        state_free(s);
        delete s;
        return fail(r, msg);
    }
    *out = s;
    return PET_OK;
}

extern "C" pet_status pet_state_create(const pet_geometry *g, const int32_t *d_counts,
                                       const float *d_gamma, const pet_params *params,
                                       const float *d_img_init, void *stream, pet_state **out)
{
    return state_create_any(g, d_counts, d_gamma, nullptr, params, d_img_init, stream, out);
}

extern "C" pet_status pet_state_create_attn(const pet_geometry *g, const int32_t *d_counts,
                                            const float *d_gamma, const float *d_mult,
                                            const pet_params *params, const float *d_img_init,
                                            void *stream, pet_state **out)
{
    if (!d_mult) return fail(PET_ERR_INVALID, "pet_state_create_attn: NULL detection factors");
    return state_create_any(g, d_counts, d_gamma, d_mult, params, d_img_init, stream, out);
}

extern "C" pet_status pet_subiter(pet_state *s, void *stream)
{
    if (!s) return fail(PET_ERR_INVALID, "pet_subiter: NULL state");
    return state_subiter(s, as_stream(stream));
}

extern "C" pet_status pet_state_read_image(const pet_state *s, float *d_img, void *stream)
{
    if (!s || !d_img) return fail(PET_ERR_INVALID, "pet_state_read_image: NULL argument");
    return from_internal_image(s->g->dev, s->f[s->cur], d_img, s->arith == AR_FP64, 0,
                               as_stream(stream));
}

extern "C" pet_status pet_state_read_image_f64(const pet_state *s, double *d_img, void *stream)
{
    if (!s || !d_img) return fail(PET_ERR_INVALID, "pet_state_read_image_f64: NULL argument");
    return from_internal_image(s->g->dev, s->f[s->cur], d_img, s->arith == AR_FP64, 1,
                               as_stream(stream));
}

extern "C" pet_status pet_state_objective(pet_state *s, double *h_phi, double *h_parts,
                                         void *stream)
{
    if (!s || !h_phi) return fail(PET_ERR_INVALID, "pet_state_objective: NULL argument");
    cudaStream_t st = as_stream(stream);
    PET_TRY(state_objective_async(s, s->sums + 3, st));
    double h[3];
    PET_CUDA(cudaMemcpyAsync(h, s->sums + 3, sizeof(h), cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    *h_phi = h[0] - h[1] + s->prm.beta * h[2];
    if (h_parts) { h_parts[0] = h[0]; h_parts[1] = h[1]; h_parts[2] = h[2]; }
    return PET_OK;
}

extern "C" pet_status pet_state_reset(pet_state *s, const float *d_img_init, void *stream)
{
    if (!s) return fail(PET_ERR_INVALID, "pet_state_reset: NULL state");
    cudaStream_t st = as_stream(stream);
    const GeoDev &gd = s->g->dev;
    if (d_img_init) PET_TRY(to_internal_image(gd, d_img_init, s->f[0], 0, s->arith == AR_FP64, st));
    else PET_TRY(fill_internal_ones(gd, s->f[0], s->arith == AR_FP64, st));
    s->cur = 0;
    s->k = s->i = s->J = 0;
    s->tn = 1.0;
    s->have_frozen = false;
    PET_TRY(tv_reset(s, st));
    return state_sum_f(s, st);
}

extern "C" int pet_state_subiters(const pet_state *s) { return s ? s->J : -1; }

// ------------------------------------------------------------------------------------------
// Checkpoint / resume: everything a state carries from one subiteration to the next (schedule
// position, Nesterov t, the current image in the internal layout, the frozen nu, the FP64 sums,
// the objective history, the TV dual variable), as one host blob.
// ------------------------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];                  // "PETCKPT1"
    int n, nplanes, nviews, nbins, nsubsets, subrays, precision, regularizer, rdp_3d, iterations;
    int attn;                       // the scan has per-bin detection factors
    int k, i, J, cur, have_frozen, objcap;
    double tn;
    unsigned long long q_bytes, tv_bytes;
};
const char kMagic[8] = {'P', 'E', 'T', 'C', 'K', 'P', 'T', '1'};

size_t ckpt_bytes(const pet_state *s)
{
    const size_t tv = s->prm.regularizer == PET_REG_TV ? 2 * s->q_bytes : 0;
    return sizeof(CkptHeader) + 2 * s->q_bytes + 16 * sizeof(double) +
           (size_t)s->objcap * 3 * sizeof(double) + tv;
}
}  // namespace

extern "C" pet_status pet_state_export(const pet_state *s, void *h_buf, size_t *bytes, void *stream)
{
    if (!s || !bytes) return fail(PET_ERR_INVALID, "pet_state_export: NULL argument");
    const size_t need = ckpt_bytes(s);
    if (!h_buf) { *bytes = need; return PET_OK; }
    if (*bytes < need) return fail(PET_ERR_INVALID, "pet_state_export: buffer too small");
    cudaStream_t st = as_stream(stream);
    const pet_geometry_desc &d = s->g->desc;
    CkptHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.n = d.n; h.nplanes = d.nplanes; h.nviews = d.nviews; h.nbins = d.nbins;
    h.nsubsets = d.nsubsets; h.subrays = s->g->dev.R; h.precision = s->prm.precision;
    h.regularizer = s->prm.regularizer; h.rdp_3d = s->prm.rdp_3d; h.iterations = s->prm.iterations;
    h.attn = s->attn ? 1 : 0;
    h.k = s->k; h.i = s->i; h.J = s->J; h.cur = s->cur; h.have_frozen = s->have_frozen;
    h.objcap = s->objcap; h.tn = s->tn;
    h.q_bytes = s->q_bytes;
    h.tv_bytes = s->prm.regularizer == PET_REG_TV ? 2 * s->q_bytes : 0;
    char *o = reinterpret_cast<char *>(h_buf);
    memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    PET_CUDA(cudaMemcpyAsync(o, s->f[s->cur], s->q_bytes, cudaMemcpyDeviceToHost, st));
    o += s->q_bytes;
    PET_CUDA(cudaMemcpyAsync(o, s->nu_frozen, s->q_bytes, cudaMemcpyDeviceToHost, st));
    o += s->q_bytes;
    PET_CUDA(cudaMemcpyAsync(o, s->sums, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
    o += 16 * sizeof(double);
    PET_CUDA(cudaMemcpyAsync(o, s->objhist, (size_t)s->objcap * 3 * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    o += (size_t)s->objcap * 3 * sizeof(double);
    if (h.tv_bytes)
        PET_CUDA(cudaMemcpyAsync(o, reinterpret_cast<char *>(s->tvmem) + 3 * s->q_bytes, h.tv_bytes,
                                 cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    *bytes = need;
    return PET_OK;
}

extern "C" pet_status pet_state_import(pet_state *s, const void *h_buf, size_t bytes, void *stream)
{
    if (!s || !h_buf) return fail(PET_ERR_INVALID, "pet_state_import: NULL argument");
    if (bytes < sizeof(CkptHeader)) return fail(PET_ERR_INVALID, "pet_state_import: truncated checkpoint");
    CkptHeader h;
    memcpy(&h, h_buf, sizeof(h));
    const pet_geometry_desc &d = s->g->desc;
    if (memcmp(h.magic, kMagic, 8) != 0)
        return fail(PET_ERR_INVALID, "pet_state_import: not a checkpoint of this library");
    if (h.n != d.n || h.nplanes != d.nplanes || h.nviews != d.nviews || h.nbins != d.nbins ||
        h.nsubsets != d.nsubsets || h.subrays != s->g->dev.R || h.precision != s->prm.precision ||
        h.regularizer != s->prm.regularizer || h.rdp_3d != s->prm.rdp_3d ||
        h.iterations != s->prm.iterations || h.q_bytes != s->q_bytes || h.objcap != s->objcap ||
        h.attn != (s->attn ? 1 : 0))
        return fail(PET_ERR_INVALID, "pet_state_import: checkpoint of another geometry or parameters");
    if (bytes < ckpt_bytes(s)) return fail(PET_ERR_INVALID, "pet_state_import: truncated checkpoint");
    cudaStream_t st = as_stream(stream);
    const char *o = reinterpret_cast<const char *>(h_buf) + sizeof(h);
    s->cur = h.cur;
    PET_CUDA(cudaMemcpyAsync(s->f[s->cur], o, s->q_bytes, cudaMemcpyHostToDevice, st));
    o += s->q_bytes;
    PET_CUDA(cudaMemcpyAsync(s->nu_frozen, o, s->q_bytes, cudaMemcpyHostToDevice, st));
    o += s->q_bytes;
    PET_CUDA(cudaMemcpyAsync(s->sums, o, 16 * sizeof(double), cudaMemcpyHostToDevice, st));
    o += 16 * sizeof(double);
    PET_CUDA(cudaMemcpyAsync(s->objhist, o, (size_t)s->objcap * 3 * sizeof(double),
                             cudaMemcpyHostToDevice, st));
    o += (size_t)s->objcap * 3 * sizeof(double);
    if (h.tv_bytes)
        PET_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(s->tvmem) + 3 * s->q_bytes, o, h.tv_bytes,
                                 cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaStreamSynchronize(st));
    s->k = h.k;
    s->i = h.i;
    s->J = h.J;
    s->tn = h.tn;
    s->have_frozen = h.have_frozen != 0;
    return PET_OK;
}

extern "C" pet_status pet_state_objective_history(pet_state *s, double *h_obj, void *stream)
{
    if (!s || !h_obj) return fail(PET_ERR_INVALID, "pet_state_objective_history: NULL argument");
    cudaStream_t st = as_stream(stream);
    const int T = s->prm.iterations;
    std::vector<double> h((size_t)(T + 1) * 3);
    PET_CUDA(cudaMemcpyAsync(h.data(), s->objhist, h.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    const int M = s->g->dev.M;
    const int kdone = s->J / M;                       // objectives recorded for k <= kdone
    for (int k = 0; k <= T; ++k)
        h_obj[k] = k <= kdone ? h[3 * k] - h[3 * k + 1] + s->prm.beta * h[3 * k + 2]
                              : __builtin_nan("");
    return PET_OK;
}

extern "C" void pet_state_destroy(pet_state *s)
{
    if (!s) return;
    state_free(s);
    delete s;
}

// Phi(f^k) beside the following subiterations: f^k is copied to a snapshot on `st`, and the
// objective projection and RDP value run on their own stream (own reduction scratch) from the
// snapshot while `st` goes on with iteration k + 1.  `st` waits for the previous evaluation
// before overwriting the snapshot, and for the last one before the reconstruction returns.
static pet_status state_objective_beside(pet_state *s, double *out3, cudaStream_t st)
{
    if (profile_active()) {
        if (s->obj_pending) {
            PET_CUDA(cudaStreamWaitEvent(st, s->ev_odone, 0));
            s->obj_pending = false;
        }
        return state_objective_async(s, out3, st);
    }
    if (!s->ostream) {
        PET_CUDA(cudaStreamCreateWithFlags(&s->ostream, cudaStreamNonBlocking));
        PET_CUDA(cudaEventCreateWithFlags(&s->ev_ofork, cudaEventDisableTiming));
        PET_CUDA(cudaEventCreateWithFlags(&s->ev_odone, cudaEventDisableTiming));
        PET_CUDA(dev_malloc(&s->fobj, s->q_bytes));
        PET_CUDA(dev_malloc(&s->redobj_mem, reducer_bytes(kRedCap, 2)));
        PET_CUDA(cudaMemset(s->redobj_mem, 0, reducer_bytes(kRedCap, 2)));
        reducer_bind(s->red_obj, s->redobj_mem, kRedCap, 2);
    }
    if (s->obj_pending) PET_CUDA(cudaStreamWaitEvent(st, s->ev_odone, 0));
    PET_CUDA(cudaMemcpyAsync(s->fobj, s->f[s->cur], s->q_bytes, cudaMemcpyDeviceToDevice, st));
    PET_CUDA(cudaEventRecord(s->ev_ofork, st));
    PET_CUDA(cudaStreamWaitEvent(s->ostream, s->ev_ofork, 0));
    FwdArgs fa;
    ImageArgs ra;
    objective_args(s, out3, &fa, &ra);
    fa.img = ra.f = s->fobj;
    fa.red = ra.red = s->red_obj;
    PET_TRY(launch_forward(fa, FWD_OBJECTIVE, s->arith, s->ostream));
    PET_TRY(launch_rdp_value(ra, s->arith, s->ostream));
    PET_CUDA(cudaEventRecord(s->ev_odone, s->ostream));
    s->obj_pending = true;
    return PET_OK;
}

// Whole reconstruction on an allocated state: T outer iterations, objective history on device.
// The subiterations run on an internal stream of the highest priority forked from `st` (joined
// back at the end), so that the objective evaluations beside them, at default priority, take
// only the SM slots the subiterations leave.
static pet_status run_reconstruct(pet_state *s, double *h_objective, cudaStream_t st0)
{
    TraceRange tr("pet_reconstruct");
    const int T = s->prm.iterations, M = s->g->dev.M;
    cudaStream_t st = st0;
    if (h_objective && !profile_active()) {
        if (!s->hstream) {
            int lo = 0, hi = 0;
            PET_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            PET_CUDA(cudaStreamCreateWithPriority(&s->hstream, cudaStreamNonBlocking, hi));
            PET_CUDA(cudaEventCreateWithFlags(&s->ev_h0, cudaEventDisableTiming));
            PET_CUDA(cudaEventCreateWithFlags(&s->ev_h1, cudaEventDisableTiming));
        }
        PET_CUDA(cudaEventRecord(s->ev_h0, st0));
        PET_CUDA(cudaStreamWaitEvent(s->hstream, s->ev_h0, 0));
        st = s->hstream;
    }
    if (h_objective) PET_TRY(state_objective_beside(s, s->objhist, st));
    for (int k = 0; k < T; ++k) {
        for (int i = 0; i < M; ++i) PET_TRY(state_subiter(s, st));
        if (h_objective) PET_TRY(state_objective_beside(s, s->objhist + 3 * (k + 1), st));
    }
    if (s->obj_pending) {
        PET_CUDA(cudaStreamWaitEvent(st, s->ev_odone, 0));
        s->obj_pending = false;
    }
    if (st != st0) {
        PET_CUDA(cudaEventRecord(s->ev_h1, st));
        PET_CUDA(cudaStreamWaitEvent(st0, s->ev_h1, 0));
    }
    return PET_OK;
}

static pet_status finish_objective(pet_state *s, double *h_objective, cudaStream_t st)
{
    if (!h_objective) return PET_OK;
    const int T = s->prm.iterations;
    std::vector<double> h((size_t)(T + 1) * 3);
    PET_CUDA(cudaMemcpyAsync(h.data(), s->objhist, h.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k <= T; ++k)
        h_objective[k] = h[3 * k] - h[3 * k + 1] + s->prm.beta * h[3 * k + 2];
    return PET_OK;
}

// The reconstruction entry points keep one workspace per geometry (allocated on first use and
// reused), so repeated calls do not allocate.  Calls on one geometry must not overlap.
struct GeoWorkspace {
    pet_state st;
    int32_t *counts = nullptr;      // host-entry staging
    float *gamma = nullptr;
    float *img = nullptr;
    size_t cap_counts = 0, cap_img = 0;
};

static GeoWorkspace *workspace_of(const pet_geometry *g)
{
    pet_geometry *gm = const_cast<pet_geometry *>(g);
    if (!gm->workspace) gm->workspace = new GeoWorkspace();
    return reinterpret_cast<GeoWorkspace *>(gm->workspace);
}

namespace pet {
void workspace_free(void *w)
{
    GeoWorkspace *ws = reinterpret_cast<GeoWorkspace *>(w);
    if (!ws) return;
    state_free(&ws->st);
    cudaFree(ws->counts);
    cudaFree(ws->gamma);
    cudaFree(ws->img);
    delete ws;
}
}  // namespace pet

static pet_status reconstruct_any(const pet_geometry *g, const int32_t *d_counts,
                                  const float *d_gamma, const float *d_mult,
                                  const pet_params *params, float *d_img_inout,
                                  double *h_objective, void *stream)
{
    if (!g || !d_counts || !d_gamma || !d_img_inout)
        return fail(PET_ERR_INVALID, "pet_reconstruct: NULL argument");
    PET_TRY(check_params(params));
    cudaStream_t st = as_stream(stream);
    GeoWorkspace *ws = workspace_of(g);
    pet_state *s = &ws->st;
    PET_TRY(state_alloc(s, g, arith_of(params->precision), params->iterations,
                        params->regularizer == PET_REG_TV, d_mult != nullptr));
    PET_TRY(state_load(s, d_counts, d_gamma, d_mult, params, d_img_inout, st, true));
    PET_TRY(run_reconstruct(s, h_objective, st));
    PET_TRY(from_internal_image(g->dev, s->f[s->cur], d_img_inout, s->arith == AR_FP64, 0, st));
    PET_TRY(finish_objective(s, h_objective, st));
    PET_CUDA(cudaStreamSynchronize(st));
    return PET_OK;
}

extern "C" pet_status pet_reconstruct(const pet_geometry *g, const int32_t *d_counts,
                                      const float *d_gamma, const pet_params *params,
                                      float *d_img_inout, double *h_objective, void *stream)
{
    return reconstruct_any(g, d_counts, d_gamma, nullptr, params, d_img_inout, h_objective, stream);
}

extern "C" pet_status pet_reconstruct_attn(const pet_geometry *g, const int32_t *d_counts,
                                           const float *d_gamma, const float *d_mult,
                                           const pet_params *params, float *d_img_inout,
                                           double *h_objective, void *stream)
{
    if (!d_mult) return fail(PET_ERR_INVALID, "pet_reconstruct_attn: NULL detection factors");
    return reconstruct_any(g, d_counts, d_gamma, d_mult, params, d_img_inout, h_objective, stream);
}

extern "C" pet_status pet_reconstruct_host(const pet_geometry *g, const int32_t *h_counts,
                                           const float *h_gamma, const pet_params *params,
                                           float *h_img_inout, double *h_objective, void *stream)
{
    if (!g || !h_counts || !h_gamma || !h_img_inout)
        return fail(PET_ERR_INVALID, "pet_reconstruct_host: NULL argument");
    PET_TRY(check_params(params));
    cudaStream_t st = as_stream(stream);
    GeoWorkspace *ws = workspace_of(g);
    const GeoDev &gd = g->dev;
    const size_t nsino = (size_t)gd.P * gd.V * gd.SB, nimg = (size_t)gd.P * gd.N * gd.N;
    if (ws->cap_counts < nsino) {
        cudaFree(ws->counts);
        cudaFree(ws->gamma);
        ws->counts = nullptr;
        ws->gamma = nullptr;
        ws->cap_counts = 0;
        PET_CUDA(dev_malloc(&ws->counts, nsino * sizeof(int32_t)));
        PET_CUDA(dev_malloc(&ws->gamma, nsino * sizeof(float)));
        ws->cap_counts = nsino;
    }
    if (ws->cap_img < nimg) {
        cudaFree(ws->img);
        ws->img = nullptr;
        ws->cap_img = 0;
        PET_CUDA(dev_malloc(&ws->img, nimg * sizeof(float)));
        ws->cap_img = nimg;
    }
    PET_CUDA(cudaMemcpyAsync(ws->counts, h_counts, nsino * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(ws->gamma, h_gamma, nsino * sizeof(float), cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(ws->img, h_img_inout, nimg * sizeof(float), cudaMemcpyHostToDevice, st));
    pet_state *s = &ws->st;
    PET_TRY(state_alloc(s, g, arith_of(params->precision), params->iterations,
                        params->regularizer == PET_REG_TV));
    PET_TRY(state_load(s, ws->counts, ws->gamma, nullptr, params, ws->img, st, true));
    PET_TRY(run_reconstruct(s, h_objective, st));
    PET_TRY(from_internal_image(gd, s->f[s->cur], ws->img, s->arith == AR_FP64, 0, st));
    PET_CUDA(cudaMemcpyAsync(h_img_inout, ws->img, nimg * sizeof(float), cudaMemcpyDeviceToHost, st));
    PET_TRY(finish_objective(s, h_objective, st));
    PET_CUDA(cudaStreamSynchronize(st));
    return PET_OK;
}

// ------------------------------------------------------------------------------------------
// Stand-alone projectors and steps (geometry scratch: calls on one geometry must not overlap)
// ------------------------------------------------------------------------------------------
static pet_status subset_range(const pet_geometry *g, int subset, int *slot0, int *nv)
{
    if (subset == -1) { *slot0 = 0; *nv = g->desc.nviews; return PET_OK; }
    if (subset < 0 || subset >= g->desc.nsubsets)
        return fail(PET_ERR_INVALID, "subset index out of range (need -1 or 0 <= subset < M)");
    *slot0 = g->voff[subset];
    *nv = g->voff[subset + 1] - g->voff[subset];
    return PET_OK;
}

static pet_status forward_any(const pet_geometry *g, int subset, const void *d_img, void *d_proj,
                              int is_double, void *stream)
{
    if (!g || !d_img || !d_proj) return fail(PET_ERR_INVALID, "forward projection: NULL argument");
    int slot0, nv;
    PET_TRY(subset_range(g, subset, &slot0, &nv));
    cudaStream_t st = as_stream(stream);
    const GeoDev &gd = g->dev;
    const size_t esz = is_double ? 8 : 4;
    const size_t qb = (size_t)gd.N * gd.N * gd.Pp * esz, pb = (size_t)nv * gd.SB * gd.Pp * esz;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, qb + pb + 256, &scr));
    void *img_i = scr, *proj_i = reinterpret_cast<char *>(scr) + ((qb + 255) / 256) * 256;
    PET_TRY(to_internal_image(gd, d_img, img_i, is_double, is_double, st));
    FwdArgs fa{};
    fa.g = gd;
    fa.slot0 = slot0;
    fa.nviews = nv;
    fa.img = img_i;
    fa.out = proj_i;
    PET_TRY(launch_forward(fa, FWD_PLAIN, is_double ? AR_FP64 : AR_KAHAN, st));
    return from_internal_sino(gd, subset == -1 ? g->d_view_of_slot : nullptr, nv, proj_i, d_proj,
                              is_double, st);
}

static pet_status back_any(const pet_geometry *g, int subset, const void *d_proj, void *d_img,
                           int is_double, void *stream)
{
    if (!g || !d_img || !d_proj) return fail(PET_ERR_INVALID, "backprojection: NULL argument");
    int slot0, nv;
    PET_TRY(subset_range(g, subset, &slot0, &nv));
    cudaStream_t st = as_stream(stream);
    const GeoDev &gd = g->dev;
    const size_t esz = is_double ? 8 : 4;
    const size_t qb = (size_t)gd.N * gd.N * gd.Pp * esz, pb = (size_t)nv * gd.SB * gd.Pp * esz;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, qb + pb + 256, &scr));
    void *img_i = scr, *proj_i = reinterpret_cast<char *>(scr) + ((qb + 255) / 256) * 256;
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, slot0, nv, d_proj, proj_i, is_double ? 3 : 2,
                             subset == -1 ? 0 : 1, st));
    BackArgs ba{};
    ba.g = gd;
    ba.slot0 = slot0;
    ba.nviews = nv;
    ba.proj = proj_i;
    ba.img = img_i;
    PET_TRY(launch_back(ba, is_double ? AR_FP64 : AR_KAHAN, st));
    return from_internal_image(gd, img_i, d_img, is_double, is_double, st);
}

extern "C" pet_status pet_forward_subset(const pet_geometry *g, int subset, const float *d_img,
                                         float *d_proj, void *stream)
{
    return forward_any(g, subset, d_img, d_proj, 0, stream);
}

extern "C" pet_status pet_back_subset(const pet_geometry *g, int subset, const float *d_proj,
                                      float *d_img, void *stream)
{
    return back_any(g, subset, d_proj, d_img, 0, stream);
}

extern "C" pet_status pet_forward_subset_f64(const pet_geometry *g, int subset,
                                             const double *d_img, double *d_proj, void *stream)
{
    return forward_any(g, subset, d_img, d_proj, 1, stream);
}

extern "C" pet_status pet_back_subset_f64(const pet_geometry *g, int subset, const double *d_proj,
                                          double *d_img, void *stream)
{
    return back_any(g, subset, d_proj, d_img, 1, stream);
}

// image -> internal image in geometry scratch (two internal images of room)
static pet_status stage_image(const pet_geometry *g, const float *d_img, void **img_i,
                              void **out_i, cudaStream_t st)
{
    const GeoDev &gd = g->dev;
    const size_t qb = ((size_t)gd.N * gd.N * gd.Pp * 4 + 255) / 256 * 256;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, 2 * qb, &scr));
    *img_i = scr;
    *out_i = reinterpret_cast<char *>(scr) + qb;
    return to_internal_image(gd, d_img, *img_i, 0, 0, st);
}

static pet_status rdp_gradient_any(const pet_geometry *g, const float *d_img, double gamma_r,
                                   double eps, float *d_grad, void *stream, int z3)
{
    if (!g || !d_img || !d_grad) return fail(PET_ERR_INVALID, "pet_rdp_gradient: NULL argument");
    cudaStream_t st = as_stream(stream);
    void *img_i, *out_i;
    PET_TRY(stage_image(g, d_img, &img_i, &out_i, st));
    ImageArgs a{};
    a.g = g->dev;
    a.f = img_i;
    a.out = out_i;
    a.gamma_r = gamma_r;
    a.eps = eps;
    a.red = g->red;
    a.z3 = z3;
    PET_TRY(launch_rdp_grad(a, AR_FP32, st));
    return from_internal_image(g->dev, out_i, d_grad, 0, 0, st);
}

extern "C" pet_status pet_rdp_gradient(const pet_geometry *g, const float *d_img, double gamma_r,
                                       double eps, float *d_grad, void *stream)
{
    return rdp_gradient_any(g, d_img, gamma_r, eps, d_grad, stream, 0);
}

extern "C" pet_status pet_rdp_gradient_3d(const pet_geometry *g, const float *d_img, double gamma_r,
                                          double eps, float *d_grad, void *stream)
{
    return rdp_gradient_any(g, d_img, gamma_r, eps, d_grad, stream, 1);
}

static pet_status smoothness_nu_any(const pet_geometry *g, const float *d_img, double nu1,
                                    double nu2, float *d_nu, void *stream, int z3)
{
    if (!g || !d_img || !d_nu) return fail(PET_ERR_INVALID, "pet_smoothness_nu: NULL argument");
    if (!(nu1 > 0) || !(nu2 >= nu1)) return fail(PET_ERR_INVALID, "pet_smoothness_nu: need 0 < nu1 <= nu2");
    cudaStream_t st = as_stream(stream);
    void *img_i, *out_i;
    PET_TRY(stage_image(g, d_img, &img_i, &out_i, st));
    ImageArgs a{};
    a.g = g->dev;
    a.f = img_i;
    a.out = out_i;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.red = g->red;
    a.z3 = z3;
    a.result = g->d_sums;
    PET_TRY(launch_sum(a, AR_FP32, st));                  // d_sums[0] = sum f
    a.sum_f = g->d_sums;
    a.result = g->d_sums + 1;
    PET_TRY(launch_mu_sum(a, AR_FP32, st));               // d_sums[1] = sum mu
    a.sum_mu = g->d_sums + 1;
    PET_TRY(launch_nu_map(a, AR_FP32, st));
    return from_internal_image(g->dev, out_i, d_nu, 0, 0, st);
}

extern "C" pet_status pet_smoothness_nu(const pet_geometry *g, const float *d_img, double nu1,
                                        double nu2, float *d_nu, void *stream)
{
    return smoothness_nu_any(g, d_img, nu1, nu2, d_nu, stream, 0);
}

extern "C" pet_status pet_smoothness_nu_3d(const pet_geometry *g, const float *d_img, double nu1,
                                           double nu2, float *d_nu, void *stream)
{
    return smoothness_nu_any(g, d_img, nu1, nu2, d_nu, stream, 1);
}

static pet_status objective_any(const pet_geometry *g, const int32_t *d_counts,
                                const float *d_gamma, const float *d_img, double beta,
                                double gamma_r, double eps, double *h_phi, double *h_parts,
                                void *stream, int z3, int tv = 0)
{
    if (!g || !d_counts || !d_gamma || !d_img || !h_phi)
        return fail(PET_ERR_INVALID, "pet_objective: NULL argument");
    cudaStream_t st = as_stream(stream);
    const GeoDev &gd = g->dev;
    const size_t qb = ((size_t)gd.N * gd.N * gd.Pp * 4 + 255) / 256 * 256;
    const size_t sino = (size_t)gd.V * gd.SB * gd.Pp;
    const size_t sb = (sino * 4 + 255) / 256 * 256;
    void *scr = nullptr;
    PET_TRY(geometry_scratch(g, qb + 2 * sb, &scr));
    char *base = reinterpret_cast<char *>(scr);
    void *img_i = base;
    int *cnt_i = reinterpret_cast<int *>(base + qb);
    float *gam_i = reinterpret_cast<float *>(base + qb + sb);
    PET_TRY(to_internal_image(gd, d_img, img_i, 0, 0, st));
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_counts, cnt_i, 0, 0, st));
    PET_TRY(to_internal_sino(gd, g->d_view_of_slot, 0, gd.V, d_gamma, gam_i, 1, 0, st));
    FwdArgs fa{};
    fa.g = gd;
    fa.slot0 = 0;
    fa.nviews = gd.V;
    fa.img = img_i;
    fa.counts = cnt_i;
    fa.gamma = gam_i;
    fa.red = g->red;
    fa.result = g->d_sums + 4;
    PET_TRY(launch_forward(fa, FWD_OBJECTIVE, AR_KAHAN, st));
    ImageArgs a{};
    a.g = gd;
    a.f = img_i;
    a.gamma_r = gamma_r;
    a.eps = eps;
    a.red = g->red;
    a.result = g->d_sums + 6;
    a.z3 = z3;
    a.tv = tv;
    PET_TRY(launch_rdp_value(a, AR_FP32, st));
    double h[3];
    PET_CUDA(cudaMemcpyAsync(h, g->d_sums + 4, sizeof(h), cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaStreamSynchronize(st));
    *h_phi = h[0] - h[1] + beta * h[2];
    if (h_parts) { h_parts[0] = h[0]; h_parts[1] = h[1]; h_parts[2] = h[2]; }
    return PET_OK;
}

extern "C" pet_status pet_objective(const pet_geometry *g, const int32_t *d_counts,
                                    const float *d_gamma, const float *d_img, double beta,
                                    double gamma_r, double eps, double *h_phi, double *h_parts,
                                    void *stream)
{
    return objective_any(g, d_counts, d_gamma, d_img, beta, gamma_r, eps, h_phi, h_parts, stream, 0);
}

extern "C" pet_status pet_objective_3d(const pet_geometry *g, const int32_t *d_counts,
                                       const float *d_gamma, const float *d_img, double beta,
                                       double gamma_r, double eps, double *h_phi, double *h_parts,
                                       void *stream)
{
    return objective_any(g, d_counts, d_gamma, d_img, beta, gamma_r, eps, h_phi, h_parts, stream, 1);
}

extern "C" pet_status pet_objective_tv(const pet_geometry *g, const int32_t *d_counts,
                                       const float *d_gamma, const float *d_img, double beta,
                                       double *h_phi, double *h_parts, void *stream)
{
    return objective_any(g, d_counts, d_gamma, d_img, beta, 2.0, 1e-12, h_phi, h_parts, stream, 0, 1);
}
