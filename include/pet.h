/*
 * libpet — GB300-native SDP-BSREM PET reconstruction (arXiv 2111.07886), C ABI.
 *
 * The library computes penalised-likelihood PET reconstruction with the relative difference
 * prior (RDP) by BSREM with subiteration-dependent diagonal preconditioners (SDP-BSREM,
 * Table I).  Every step of the path runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Geometry (Sec. II-A, Eq. model-Poisson; one line per detector bin, parallel beam):
 *   - image: N x N pixels of side pixel_mm, P stacked planes, centred at the origin; pixel
 *     (ix, iy) is the half-open square [ix - N/2, ix + 1 - N/2) x [iy - N/2, iy + 1 - N/2) in
 *     pixel units, so a ray lying on a pixel edge belongs to the pixel on its + side only;
 *   - views theta_v = v pi / V, v = 0..V-1; bins at offsets r_b = (b - (n_b - 1)/2) bin_mm;
 *     ray (v, b) is the line {x cos theta_v + y sin theta_v = r_b};
 *   - system matrix A_ij = sens * (length in mm of ray i inside pixel j) (or the mean over
 *     desc.subrays parallel lines across the bin, see pet_geometry_desc);
 *   - ordered subsets (Sec. II-B): subset i (0-based) holds the views v with v mod M == i,
 *     processed i = 0..M-1 within an iteration; subset projections list the subset's views
 *     in increasing order.
 * Layouts (row-major, x fastest):
 *   - images  float [P][N][N];
 *   - sinograms: counts int32 [P][V][n_b], background gamma float [P][V][n_b] (gamma > 0);
 *   - subset projections float [P][V_i][n_b].
 * Memory: pointers named d_* are device memory owned by the caller (the library never frees
 *   them); pointers named h_* are host memory owned by the caller.  Handles are owned by the
 *   library and freed by the matching *_destroy.  `stream` is a cudaStream_t passed as void*
 *   (NULL = the legacy default stream); device work is enqueued on it and the call returns
 *   without synchronising unless it says otherwise.
 * Errors: every call returns a pet_status and never aborts; on failure pet_last_error()
 *   gives a message for the calling thread.  CUDA failures map to PET_ERR_CUDA.
 * Precision: PET_PREC_FP32 sums in plain FP32; PET_PREC_FP32_KAHAN adds compensated (Kahan)
 *   sums along rays and in the backprojection gather; PET_PREC_FP64 runs every kernel in
 *   double.  In all modes the objective, the global sums behind mean(f) and mean(mu), and the
 *   step-size scalars are FP64; counts stay exact int32.
 */
#ifndef PET_H_
#define PET_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PET_OK = 0,
    PET_ERR_INVALID = 1,    /* bad argument, shape, or input value (e.g. gamma <= 0) */
    PET_ERR_OOM = 2,        /* device or host allocation failed / over budget */
    PET_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    PET_ERR_TIMEOUT = 4,    /* a bounded wait ran out */
    PET_PENDING = 5,        /* serving: request not finished yet */
    PET_ERR_NOT_FOUND = 6   /* serving: unknown ticket */
} pet_status;

typedef struct {
    int n;              /* image side N (pixels) */
    int nplanes;        /* P stacked 2-D planes */
    double pixel_mm;    /* pixel side */
    int nviews;         /* V views over [0, pi) */
    int nbins;          /* n_b radial bins */
    double bin_mm;      /* bin spacing */
    int nsubsets;       /* M ordered subsets, 1 <= M <= V */
    double sens;        /* A_ij = sens * length_mm (counts per activity per mm), > 0 */
    int subrays;        /* R parallel lines per bin, spread uniformly across its width (offsets
                           ((s + 1/2)/R - 1/2) bin_mm from its centre, s = 0..R-1), and
                           A_ij = sens / R * (sum of their lengths in mm inside pixel j): the
                           paper's ray-driven model with parallel rays per detector pair
                           (Sec. IV-A, 32 there).  0 or 1: one line at the bin centre; at most 64 */
    int tof_bins;       /* T time-of-flight bins per bin (the TOF data of the clinical
                           reconstructions, Sec. IV-C); 0 or 1: no TOF.  TOF bin t of bin i is
                           centred at tau_t = (t - (T-1)/2) tof_bin_mm along the line from its
                           point nearest the centre, and A_{(i,t) j} = A_ij h_t(tau_j) with tau_j
                           the position of pixel j's centre along the line and h_t the Gaussian
                           timing kernel (FWHM tof_fwhm_mm) integrated over the TOF bin.
                           Sinograms then hold [P][V][n_b][T].  At most 64; with subrays <= 1 */
    double tof_bin_mm;  /* TOF bin width along the line (> 0 with TOF) */
    double tof_fwhm_mm; /* FWHM of the timing kernel as a distance along the line (> 0 with TOF) */
    double ring_mm;     /* 0: uniform bins bin_mm apart.  > 0: the bins of a view are the lines of
                           a detector ring of this radius equally spaced in angle (the paper's
                           576-detector ring, Sec. IV-A): bin b lies at r_b = ring_mm sin(beta_b),
                           beta_b = (b - (n_b-1)/2) bin_mm / ring_mm (bin_mm is then the arc
                           spacing on the ring), spans [ring_mm sin(beta_b - d/2),
                           ring_mm sin(beta_b + d/2)] with d = bin_mm / ring_mm, and its subrays
                           spread uniformly over that width.  Needs n_b bin_mm < pi ring_mm */
} pet_geometry_desc;

typedef enum {
    PET_PRECOND_BSREM = 0,  /* S^{k,i} = S                         (Sec. II-B)           */
    PET_PRECOND_M1 = 1,     /* alpha Nesterov, nu = 1              (Eq. preconditioner:Nesterov) */
    PET_PRECOND_M2 = 2,     /* alpha KM, nu = 1                    (Eq. preconditioner:KM) */
    PET_PRECOND_P1 = 3,     /* alpha Nesterov, nu from Eq. nuki                          */
    PET_PRECOND_P2 = 4      /* alpha KM, nu from Eq. nuki                                */
} pet_precond;

typedef enum { PET_PREC_FP32 = 0, PET_PREC_FP32_KAHAN = 1, PET_PREC_FP64 = 2 } pet_precision;

/* Parameters of SDP-BSREM (Table I; Eqs. RDP, preconditioner, OperatorPt,
 * preconditioner:Nesterov, preconditioner:KM, nuki; relaxation lambda_k of Theorem 2). */
typedef struct {
    int iterations;     /* T outer iterations (pet_reconstruct) */
    double beta;        /* RDP weight beta >= 0 (Eq. ObjectiveFunction) */
    double gamma_r;     /* RDP edge parameter gamma_R >= 0 (Eq. RDP) */
    double eps;         /* RDP epsilon > 0 (Eq. RDP) */
    double t;           /* clamp margin of P_t, 0 < t < U (Eq. OperatorPt) */
    double U;           /* upper bound of the box B (Eq. BoundedSet) */
    double lambda0;     /* lambda_k = lambda0 / (a k + 1), lambda0 > 0 */
    double a;           /* a >= 0 */
    double rho;         /* KM alpha: (rho (J-1) + delta2) / (J - 1 + delta1) */
    double delta1;
    double delta2;
    double nu1;         /* nu = P_{nu1}^{nu2}(mean(mu) / mu), 0 < nu1 <= nu2 */
    double nu2;
    int J0;             /* nu = 1 for J <= J0 */
    int J1;             /* nu frozen at its J1 value for J > J1 */
    int precond;        /* pet_precond */
    int precision;      /* pet_precision */
    int rdp_3d;         /* 0: RDP over the 8 in-plane neighbours and nu from the in-plane gradient
                           (Sec. IV-A); 1: the volume as one 3-D image (the fully 3-D
                           reconstructions of Sec. IV-C): RDP over the 26 neighbours in the volume
                           (Eqs. RDP, gradRD) and nu from the gradient with its component across
                           the planes (Sec. III) */
    int regularizer;    /* pet_regularizer: PET_REG_RDP (the paper's prior, by its gradient) or
                           PET_REG_TV (no counterpart in the paper's method, which names TV only as
                           a non-smooth example): R_TV(f) = sum_j |(D f)_j|, D the in-plane forward
                           differences, entering each subiteration through a proximal step in the
                           metric of the step sizes, W = lambda_k alpha_{k,i} nu S(f):
                           z = f - W grad F_i(f); f = P_t(argmin_x 1/2 |x - z|^2_{W^-1}
                           + (beta/M) R_TV(x)), the argmin approximated by tv_iters primal-dual
                           (Chambolle-Pock) iterations warm-started from the previous dual
                           variable.  TV runs through pet_subiter / pet_reconstruct (not in
                           batches or the server), in-plane only (rdp_3d = 0). */
    int tv_iters;       /* primal-dual iterations per subiteration (PET_REG_TV), 1..10000 */
} pet_params;

typedef enum { PET_REG_RDP = 0, PET_REG_TV = 1 } pet_regularizer;

typedef struct pet_geometry pet_geometry;
typedef struct pet_state pet_state;
typedef struct pet_server pet_server;

/* Message describing the last failure on the calling thread ("" if none). */
const char *pet_last_error(void);

/* Test hook (no counterpart in the paper): host-side fault injection.  The n-th device or pinned
 * host allocation the library makes from now on (on any thread) fails as out of memory, and
 * the call that made it returns PET_ERR_OOM (a serving request finishes with it); n <= 0
 * disarms the hook.  One failure per arming.  No GPU fault is involved. */
void pet_debug_fail_alloc(int n);

/* Test hook (no counterpart in the paper): enable = 0 makes geometries created from now on (on
 * any thread) skip the precomputed backprojection entries described at pet_geometry_create,
 * so that their FP32 update computes the entries per tile; a nonzero value restores the
 * default.  Both give the same results, bit for bit; the hook lets a test show it. */
void pet_debug_bp_table(int enable);

/* ------------------------------------------------------------------------------------------
 * Geometry (Sec. II-A/II-B).  Builds the per-view / per-ray walk tables in FP64 on the host,
 * uploads them, and computes the sensitivity p_j of Eq. pj (one backprojection of ones over all
 * views) on the device.  With nplanes > 1, uniform bins (subrays <= 1, ring_mm = 0) and no TOF
 * it also stores the backprojection's (pixel, view) entries for the FP32 update (16 or 32 bytes
 * per pixel and view: 302 MB for 256 x 256 pixels and 288 views), unless a subset has more
 * views than half the update's table holds.  Synchronises `stream` before returning.
 * PET_ERR_INVALID for a bad desc
 * (limits: 1 <= n <= 8192, 1 <= nplanes <= 2048, nbins >= 4, 1 <= nsubsets <= nviews,
 * bin_mm >= 0.36 pixel_mm, 0 <= subrays <= 64, 0 <= tof_bins <= 64 (TOF with subrays <= 1),
 * at most 4 bins per view in a pixel's footprint, fewer than 4e9 image or sinogram elements).
 * With TOF bins every sinogram argument and result of the library is [P][V][n_b][T] (also the
 * server's request data).
 * ---------------------------------------------------------------------------------------- */
pet_status pet_geometry_create(const pet_geometry_desc *desc, void *stream, pet_geometry **out);
void pet_geometry_destroy(pet_geometry *g);

/* Autotuner (no counterpart in the paper): times the forward projector of subset 0 for each
 * admissible number of ray chunks (threads sharing one ray) and keeps the fastest in the
 * geometry; *best_S (optional) receives it.  Tune before creating states on the geometry (the
 * chunking changes the order of the ray sums, within rounding).  The projection is timed on an
 * image of ones, best of 7 runs of 4 launches after a warm-up (pet_autotune_batch: best of 5
 * single batched launches); a larger chunk count replaces a smaller one only when it is more
 * than 3 % faster.  Synchronises `stream`.  TOF geometries have no ray chunking (*best_S = 1).
 * pet_autotune_batch: the same, with `concurrent` (1..4096) copies of the projection running as
 * one batched launch, as they do when that many scans of the geometry step together in a
 * pet_batch or a server; the choice is kept in the geometry and used alone and in batches alike,
 * so a scan computes the same bits either way. */
pet_status pet_autotune(pet_geometry *g, void *stream, int *best_S);
pet_status pet_autotune_batch(pet_geometry *g, int concurrent, void *stream, int *best_S);

/* Sets the forward projector's ray chunks S directly (no counterpart in the paper): a choice
 * taken from an earlier pet_autotune, or fixed for a profiling run, where the profiler's own
 * per-launch cost distorts the autotuner's timings.  S = 0 returns to the built-in heuristic.
 * PET_ERR_INVALID unless S == 0 or 1 <= S <= 16 with S dividing 256 / ceil(nplanes / 8) (256 for
 * one plane).  Same rule as pet_autotune: set it before creating states on the geometry. */
pet_status pet_set_ray_chunks(pet_geometry *g, int S);

/* Number of views V_i in subset `subset` (0 <= subset < M), or -1 if out of range. */
int pet_subset_size(const pet_geometry *g, int subset);

/* p_j of Eq. pj: (A^T 1)_j / M, or 1/M where (A^T 1)_j = 0.  d_p: float [N][N] (identical for
 * every plane).  Copies the FP32 table computed at creation. */
pet_status pet_sensitivity(const pet_geometry *g, float *d_p, void *stream);

/* ------------------------------------------------------------------------------------------
 * Projectors (Sec. II-B: the row block A_i of A; App. A: grad F = A^T(1 - g/(Af + gamma))).
 * pet_forward_subset: d_proj = A_i d_img (no background added); float [P][N][N] ->
 *   float [P][V_i][n_b].  Ray-driven Siddon line integrals, FP32 with Kahan sums.
 * pet_back_subset: d_img = A_i^T d_proj; float [P][V_i][n_b] -> float [P][N][N] (overwritten).
 *   Pixel-driven gather (deterministic, no float atomics), FP32 with Kahan sums.
 * *_f64 variants: the same in double throughout.
 * subset = -1 means all views (d_proj then [P][V][n_b]).  Calls on one geometry use its scratch
 * buffers: do not overlap them on different streams.
 * ---------------------------------------------------------------------------------------- */
pet_status pet_forward_subset(const pet_geometry *g, int subset, const float *d_img, float *d_proj,
                              void *stream);
pet_status pet_back_subset(const pet_geometry *g, int subset, const float *d_proj, float *d_img,
                           void *stream);
pet_status pet_forward_subset_f64(const pet_geometry *g, int subset, const double *d_img,
                                  double *d_proj, void *stream);
pet_status pet_back_subset_f64(const pet_geometry *g, int subset, const double *d_proj,
                               double *d_img, void *stream);

/* ------------------------------------------------------------------------------------------
 * Reconstruction state (Table I).  pet_state_create copies counts, gamma and the initial image
 * into library-owned device buffers (reordered by subset, planes innermost), validates that
 * counts >= 0 and gamma > 0 and finite (PET_ERR_INVALID otherwise), and positions the state at
 * (k, i) = (0, 1).  The state keeps f, the frozen nu, the scalar schedule and the FP64 global
 * sums resident across subiterations.  Synchronises `stream`.
 * pet_subiter: one subiteration f^{k,i} = P_t(f^{k,i-1} - lambda_k S^{k,i}(f^{k,i-1})
 *   grad Phi_i(f^{k,i-1})), then advances (k, i).  Asynchronous.
 * pet_state_read_image: d_img = current f as float [P][N][N].
 * pet_state_read_image_f64: the same as double [P][N][N] (exact for PET_PREC_FP64 states).
 * pet_state_objective: *h_phi = Phi(current f) (Eqs. FidelityTerm, ObjectiveFunction), FP64;
 *   h_parts (optional, 3 doubles) = sum(Af), sum(g ln(Af + gamma)), R(f).  Synchronises.
 * pet_state_subiters: completed subiterations J.
 * pet_state_reset: restart at (k, i) = (0, 1) from d_img_init (float [P][N][N]; NULL: f^0 = 1),
 *   keeping the data; asynchronous.
 * ---------------------------------------------------------------------------------------- */
pet_status pet_state_create(const pet_geometry *g, const int32_t *d_counts, const float *d_gamma,
                            const pet_params *params, const float *d_img_init, void *stream,
                            pet_state **out);
/* pet_state_create_attn: a scan whose system matrix carries per-bin detection factors a_i
 * (attenuation, times normalisation where wanted; the simulated system of Sec. IV-A includes
 * uniform water attenuation): A becomes diag(a) A, so the mean data are a_i (A f)_i + gamma_i,
 * the ratio term backprojected by each subiteration is a_i (1 - g_i / (a_i (A f)_i + gamma_i)),
 * and p_j of Eq. pj is (A^T a)_j / M for every voxel (1/M where it is 0), computed once at
 * creation by an FP64 backprojection of a.  d_mult: float [P][V][NB] like gamma, finite and
 * >= 0 (PET_ERR_INVALID otherwise), copied into the state.  Objectives of the state
 * (pet_state_objective, the objective history) use diag(a) A.  Such states step alone, in
 * batches and in the server (pet_request.h_mult).  Synchronises `stream`. */
pet_status pet_state_create_attn(const pet_geometry *g, const int32_t *d_counts,
                                 const float *d_gamma, const float *d_mult,
                                 const pet_params *params, const float *d_img_init, void *stream,
                                 pet_state **out);
pet_status pet_subiter(pet_state *s, void *stream);
pet_status pet_state_read_image(const pet_state *s, float *d_img, void *stream);
pet_status pet_state_read_image_f64(const pet_state *s, double *d_img, void *stream);
pet_status pet_state_objective(pet_state *s, double *h_phi, double *h_parts, void *stream);
int pet_state_subiters(const pet_state *s);
/* Checkpoint / resume (no counterpart in the paper).  pet_state_export: with h_buf NULL,
 * *bytes = the size of the state's checkpoint; otherwise writes it to h_buf (*bytes >= that
 * size; host memory, caller-owned) and synchronises `stream`.  The checkpoint holds the position
 * (k, i), the Nesterov t, the current image, the frozen nu, the FP64 sums, the objective history
 * and the TV dual variable.  pet_state_import: loads a checkpoint into a state created for the
 * same geometry and parameters (same data: counts, gamma and detection factors are not in the
 * checkpoint, but whether the scan has detection factors is checked);
 * PET_ERR_INVALID for another geometry or parameters or a truncated buffer.  Subiterations after
 * an import give the same bits as the uninterrupted run.  Synchronises `stream`. */
pet_status pet_state_export(const pet_state *s, void *h_buf, size_t *bytes, void *stream);
pet_status pet_state_import(pet_state *s, const void *h_buf, size_t bytes, void *stream);
pet_status pet_state_reset(pet_state *s, const float *d_img_init, void *stream);
void pet_state_destroy(pet_state *s);

/* ------------------------------------------------------------------------------------------
 * Whole reconstruction (Table I, T = params->iterations outer iterations of M subiterations).
 * d_img_inout: f^0 in, f^T out (float [P][N][N]).  h_objective: NULL, or T+1 doubles receiving
 * Phi(f^k), k = 0..T.  Synchronises `stream`.
 * pet_reconstruct_host: the same from host buffers (copies in and out inside the call).
 * pet_reconstruct_attn: the same for a scan with per-bin detection factors d_mult (float
 *   [P][V][NB], device; see pet_state_create_attn).
 * ---------------------------------------------------------------------------------------- */
pet_status pet_reconstruct(const pet_geometry *g, const int32_t *d_counts, const float *d_gamma,
                           const pet_params *params, float *d_img_inout, double *h_objective,
                           void *stream);
pet_status pet_reconstruct_host(const pet_geometry *g, const int32_t *h_counts,
                                const float *h_gamma, const pet_params *params,
                                float *h_img_inout, double *h_objective, void *stream);
pet_status pet_reconstruct_attn(const pet_geometry *g, const int32_t *d_counts,
                                const float *d_gamma, const float *d_mult,
                                const pet_params *params, float *d_img_inout,
                                double *h_objective, void *stream);

/* ------------------------------------------------------------------------------------------
 * Single steps of the hot path, for parity checks (same kernels as pet_subiter).
 * pet_rdp_gradient: d_grad = grad R(d_img) (Eq. gradRD, 8-neighbourhood in-plane), float.
 * pet_smoothness_nu: d_nu = P_{nu1}^{nu2}(mean(mu) / mu), mu = max(0.01, grad(f)/mean(f))
 *   (Sec. III, Eq. nuki), grad = Matlab-style numerical gradient magnitude; float.
 * pet_objective: Phi(d_img) for given data (Eqs. FidelityTerm, ObjectiveFunction, RDP), FP64
 *   sums; h_parts as for pet_state_objective.  Synchronises.
 * Images float [P][N][N].
 * ---------------------------------------------------------------------------------------- */
pet_status pet_rdp_gradient(const pet_geometry *g, const float *d_img, double gamma_r, double eps,
                            float *d_grad, void *stream);
pet_status pet_smoothness_nu(const pet_geometry *g, const float *d_img, double nu1, double nu2,
                             float *d_nu, void *stream);
pet_status pet_objective(const pet_geometry *g, const int32_t *d_counts, const float *d_gamma,
                         const float *d_img, double beta, double gamma_r, double eps,
                         double *h_phi, double *h_parts, void *stream);
/* The same three calls with the fully 3-D prior (pet_params.rdp_3d = 1): RDP over the 26
 * neighbours of each voxel in the volume, nu from the gradient including its component across
 * the planes. */
pet_status pet_rdp_gradient_3d(const pet_geometry *g, const float *d_img, double gamma_r,
                               double eps, float *d_grad, void *stream);
pet_status pet_smoothness_nu_3d(const pet_geometry *g, const float *d_img, double nu1, double nu2,
                                float *d_nu, void *stream);
pet_status pet_objective_3d(const pet_geometry *g, const int32_t *d_counts, const float *d_gamma,
                            const float *d_img, double beta, double gamma_r, double eps,
                            double *h_phi, double *h_parts, void *stream);
/* TV variant (pet_params.regularizer = PET_REG_TV; no counterpart in the paper's method).
 * pet_objective_tv: Phi with R = R_TV; h_parts[2] = R_TV(d_img).  Synchronises.
 * pet_tv_prox: d_x = the primal-dual approximation (iters Chambolle-Pock iterations, steps
 *   sigma = 1/(2b), tau = 1/(4b)) of argmin_x 1/2 sum_j (x_j - z_j)^2 / W_j + b R_TV(x), from
 *   x = z and the dual variable (d_px, d_py), which is updated in place.  All arrays float
 *   [P][N][N]; W > 0; b >= 0 (b = 0 copies z). */
pet_status pet_objective_tv(const pet_geometry *g, const int32_t *d_counts, const float *d_gamma,
                            const float *d_img, double beta, double *h_phi, double *h_parts,
                            void *stream);
pet_status pet_tv_prox(const pet_geometry *g, const float *d_z, const float *d_w, double b,
                       int iters, float *d_px, float *d_py, float *d_x, void *stream);

/* ------------------------------------------------------------------------------------------
 * Batches (Table I for many independent scans at once; no counterpart in the paper).
 * A batch holds up to `capacity` reconstruction states of any geometries.  pet_batch_step
 * advances every running state of the batch by one subiteration: scans sharing one kernel
 * instantiation (plane-group size, precision) are processed by one persistent kernel per step
 * kind (mu pass, forward + ratio, fused update, objective projection, RDP value); with
 * use_graph != 0 and a non-default stream, each class's step is captured once as a CUDA graph
 * and replayed.  A state runs until it has done params.iterations x M subiterations; with
 * with_objective, Phi(f^k) is recorded for k = 0..T (read it with pet_state_objective_history).
 * Results of a scan are bitwise the same alone (pet_subiter) and in any batch.
 * pet_batch_add: the state joins at its current subiteration (Phi(f^0) is enqueued on `stream`
 *   when requested and J = 0); PET_ERR_OOM if the batch is full.
 * pet_batch_step: *running_after (optional) = states still running after this step.  The step is
 *   asynchronous; the host waits only to reuse its descriptor memory (four buffers per class, so
 *   up to four steps are in flight).  A class with a single running state launches that state's
 *   kernels directly (as pet_subiter does); with more, only the running states' arguments are
 *   uploaded and the replayed graph runs just the kernels the step needs.
 * pet_batch_remove: detach a state (waits for in-flight steps that read its descriptors).
 * pet_batch_size: running states.  The batch does not own the states.
 * pet_state_objective_history: h_obj[k] = Phi(f^k) for k = 0..T recorded so far (synchronises);
 *   entries not computed yet are NaN.
 * ---------------------------------------------------------------------------------------- */
typedef struct pet_batch pet_batch;
pet_status pet_batch_create(int capacity, int use_graph, pet_batch **out);
pet_status pet_batch_add(pet_batch *b, pet_state *s, int with_objective, void *stream);
pet_status pet_batch_remove(pet_batch *b, pet_state *s);
pet_status pet_batch_step(pet_batch *b, void *stream, int *running_after);
int pet_batch_size(const pet_batch *b);
void pet_batch_destroy(pet_batch *b);
pet_status pet_state_objective_history(pet_state *s, double *h_obj, void *stream);

/* ------------------------------------------------------------------------------------------
 * Serving (continuous batching of reconstruction requests; no counterpart in the paper).
 * pet_serve_create: a server on CUDA device `device` with a device-memory budget (bytes, for
 *   scan states, geometry tables and upload staging) and at most `max_slots` scans resident at
 *   once.  It runs two host threads: a preparer that admits queued requests in arrival order
 *   while slots and the budget allow (geometry tables cached by description; upload; resident
 *   state), and a runner that keeps one pet_batch of all resident scans stepping: requests that
 *   arrive while others are on the GPU join at the next step; finished scans are read back and
 *   their memory and slot freed.  Scans are kept in one batch per kernel class (plane-group size,
 *   arithmetic, gather width), each stepped on its own stream so that the classes advance
 *   independently and overlap on the device; the stacked (multi-plane) class runs at the higher
 *   stream priority.
 * pet_serve_submit: copies the request's host data (validated: counts >= 0, 0 < gamma < inf,
 *   detection factors when given finite and >= 0)
 *   and returns a ticket; the caller may free its buffers on return.  A request larger than the
 *   whole budget fails with PET_ERR_OOM (reported by poll).
 * pet_serve_poll: PET_PENDING while queued or running; otherwise the request's final status,
 *   with f^T copied to h_img_out (float [P][N][N], may be NULL), Phi(f^k) k = 0..T to h_obj_out
 *   (T+1 doubles, NaN without with_objective; may be NULL) and *latency_s = seconds from submit
 *   to result available; the ticket is then forgotten (PET_ERR_NOT_FOUND afterwards).
 * pet_serve_stats_get: counters, p50/p99/mean latency of completed requests, scans/s from first
 *   submit to last completion, device bytes in use, and the mean per-request breakdown of the
 *   latency: queue (submit to admission), prepare (geometry, upload, state), run (joining the
 *   batch to the last subiteration issued) and readback (to the result on the host).
 * pet_serve_autotune: concurrent > 0 makes the preparer tune every geometry it creates with
 *   pet_autotune_batch(g, concurrent) before the geometry's first scan runs (0: built-in shapes);
 *   set it before submitting.
 * pet_serve_destroy: drops queued requests, finishes resident ones, joins the threads.
 * Thread-safe: submit/poll/stats may be called from any host thread.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    pet_geometry_desc geom;
    const int32_t *h_counts;     /* [P][V][n_b] */
    const float *h_gamma;        /* [P][V][n_b] */
    const float *h_img_init;     /* [P][N][N], or NULL for f^0 = 1 */
    pet_params params;
    int with_objective;
    const float *h_mult;         /* [P][V][n_b] per-bin detection factors (pet_state_create_attn),
                                    finite and >= 0, or NULL for none */
} pet_request;

typedef struct {
    long long submitted, completed, failed, running, queued;
    double p50_s, p99_s, mean_s, scans_per_s;
    size_t hbm_in_use;
    double mean_queue_s, mean_prepare_s, mean_run_s, mean_readback_s;
    long long tuned_geometries;
} pet_serve_stats;

pet_status pet_serve_create(size_t hbm_budget_bytes, int max_slots, int device, pet_server **out);
pet_status pet_serve_submit(pet_server *sv, const pet_request *req, uint64_t *ticket);
pet_status pet_serve_poll(pet_server *sv, uint64_t ticket, float *h_img_out, double *h_obj_out,
                          double *latency_s);
pet_status pet_serve_stats_get(pet_server *sv, pet_serve_stats *out);
pet_status pet_serve_autotune(pet_server *sv, int concurrent);
void pet_serve_destroy(pet_server *sv);

/* ------------------------------------------------------------------------------------------
 * pet_objective_static: the same values as pet_objective, from a call that allocates nothing.
 * The paper has no counterpart; this serves callers that may not allocate device memory at the
 * moment they need the objective: a pipeline whose device memory is handed to a fixed pool at
 * start-up, or a real-time loop in which a cudaMalloc (such as the scratch pet_objective
 * allocates on first use) would stall the stream.  Inputs are read in their C-ABI layouts
 * (float image [P][N][N], counts int32 and gamma float [P][V][n_b]); the log-likelihood terms
 * are evaluated in FP64; the reduction uses one static device array of about 49 KB that every
 * GPU loading the library holds until exit.  The geometry must exist already
 * (pet_geometry_create allocates).  The first call on a device looks up that array's device
 * address; every call then shares the array, so calls that overlap on the GPU race and must be
 * serialised.  Problems above 2^31 - 1 rays x planes or pixels x planes are rejected with
 * PET_ERR_INVALID.  The call reads the result back to the host and synchronises `stream`.
 * ---------------------------------------------------------------------------------------- */
pet_status pet_objective_static(const pet_geometry *g, const int32_t *d_counts,
                                const float *d_gamma, const float *d_img, double beta,
                                double gamma_r, double eps, double *h_phi, double *h_parts,
                                void *stream);

/* ------------------------------------------------------------------------------------------
 * Launch accounting (no counterpart in the paper; instrumentation of this library).
 * pet_launch_count: kernels launched by this library since load (all threads).
 * pet_profile_enable(1): from now on, every launch is bracketed by CUDA events on its stream;
 *   pet_profile_read(kind, ...) waits for the recorded events and returns the accumulated
 *   device time (ms) and launch count of one kernel kind; pet_profile_reset clears them.
 * ---------------------------------------------------------------------------------------- */
typedef enum {
    PET_K_FORWARD_RATIO = 0,  /* subset forward projection + Poisson ratio (a2, a3) */
    PET_K_UPDATE = 1,         /* gather backprojection + RDP + nu + update + clamp (a4, a6, a7) */
    PET_K_MU_SUM = 2,         /* smoothness reduction sum(mu) (a5) */
    PET_K_OBJ_FORWARD = 3,    /* full forward projection with objective sums (a8) */
    PET_K_RDP_VALUE = 4,      /* RDP value (a8) */
    PET_K_LAYOUT = 5,         /* layout conversions and input checks */
    PET_K_OTHER = 6,          /* stand-alone projectors, sums, maps */
    PET_K_COUNT = 7
} pet_kernel_kind;

long long pet_launch_count(void);
void pet_profile_enable(int on);
pet_status pet_profile_read(int kind, double *total_ms, long long *launches);
void pet_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* PET_H_ */
