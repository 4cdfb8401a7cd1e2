/*
 * FP64 CPU oracle for SDP-BSREM PET reconstruction (arXiv 2111.07886).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links it, and it
 * shares no code, header, table or helper with the CUDA sources.
 *
 * Everything is double precision.  Each function cites the passage it follows:
 *   - Poisson data model, fidelity F ................ Sec. II-A, Eqs. model-Poisson, FidelityTerm
 *   - objective Phi = F + beta R, RDP R ............... Sec. II-A, Eqs. ObjectiveFunction, RDP
 *   - subset objective Phi_i ......................... Sec. II-B, Eq. SubObjFunc
 *   - preconditioner S, p_j, clamp P_t .............. Sec. II-B, Eqs. preconditioner, pj, OperatorPt
 *   - SDP-BSREM loop ................................. Sec. II-C, Table I
 *   - alpha (Nesterov / KM), mu, nu, lambda_k ......... Sec. III, Eqs. preconditioner:Nesterov,
 *                                                      preconditioner:KM, nuki; Theorem 2
 *   - grad F, dR/df_j ................................ Appendix A, Eq. gradRD
 *   - fully 3-D RDP (26 neighbours) and 3-D smoothness map, for volumes reconstructed as one
 *     3-D image (Sec. IV-C) ......................... Eqs. RDP, gradRD, nuki over 3-D neighbours
 *   - TV variant: total variation (named in Sec. I as the typical non-smooth prior) entering
 *     Table I's step through a proximal step in the preconditioner's metric, computed by the
 *     primal-dual method of Chambolle and Pock (2011) ...... see ora_tv_prox
 *
 * System model: one line per detector bin, parallel beam; A_ij = sens * (length in mm of
 * ray i inside pixel j), where a pixel is the half-open square [x, x+1) x [y, y+1) in pixel
 * units (a ray lying on a pixel edge belongs to the pixel on its + side only).  With R > 1
 * sub-rays (the "parallel rays per detector pair" of the paper's ray-driven system model,
 * Sec. IV-A, 32 there) bin i is R parallel lines spread uniformly across its width, at offsets
 * ((s + 1/2) / R - 1/2) bin_mm from its centre, s = 0..R-1, and A_ij = sens / R * (the sum of
 * their lengths in mm inside pixel j).  Lengths are
 * found by Siddon's method: all crossings of the ray with the grid lines are sorted, and each
 * piece between consecutive crossings is charged to the pixel that contains its midpoint.
 *
 * Ring sampling (the paper's scanner is a ring of 576 detectors, Sec. IV-A): with ring_mm = Rd
 * > 0 the bins are the lines of a ring of radius Rd seen in one view, equally spaced in angle:
 * bin b sits at r_b = Rd sin(beta_b), beta_b = (b - (n_b - 1)/2) dbeta, dbeta = bin_mm / Rd (so
 * bin_mm is the arc spacing on the ring; the radial spacing shrinks by cos beta towards the edge
 * of the field), and spans [Rd sin(beta_b - dbeta/2), Rd sin(beta_b + dbeta/2)]: its R sub-rays
 * are spread uniformly over that width.  ring_mm = 0: the uniform parallel-beam bins above.
 *
 * Time of flight (the clinical reconstructions of Sec. IV-C use TOF data): with T > 1 TOF bins,
 * bin i = (v, b) splits into (v, b, t), t = 0..T-1, centred at tau_t = (t - (T-1)/2) dtau along
 * the line from its point nearest the centre, and A_{(v,b,t) j} = A_{(v,b) j} h_t(tau_j), where
 * tau_j is the position of the centre of pixel j along the line and
 * h_t(tau) = Phi((tau - tau_t + dtau/2) / sigma) - Phi((tau - tau_t - dtau/2) / sigma) is the
 * Gaussian timing kernel (sigma = FWHM / (2 sqrt(2 ln 2))) integrated over the TOF bin.  When
 * the TOF bins cover the image with margin, sum_t h_t = 1 and the TOF bins add up to A.
 * Sinograms then hold [P][V][n_b][T].
 *
 * Per-bin detection factors (the simulated system of Sec. IV-A includes uniform water
 * attenuation): given a_i > 0 for every bin i, the system matrix is diag(a) A, i.e. the mean
 * data are a_i (A f)_i + gamma_i, its transpose weights bin i by a_i, and p_j of Eq. pj becomes
 * (A^T a)_j / M, which differs from plane to plane.  a = NULL stands for a_i = 1.
 *
 * Layouts: images [P][N][N] (x fastest), full sinograms [P][V][n_b], subset sinograms
 * [P][V_i][n_b] with the subset's views in increasing order.  Subset i (0-based) holds the
 * views v with v mod M == i.
 */
#define _DEFAULT_SOURCE 1
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;           /* image side N */
    int nplanes;     /* P */
    int nviews;      /* V */
    int nbins;       /* n_b */
    int nsubsets;    /* M */
    double pixel_mm;
    double bin_mm;
    double sens;     /* A_ij = sens * length_mm */
    int subrays;     /* R parallel lines per bin (<= 1: one line at the bin centre) */
    int tof_bins;    /* T time-of-flight bins per bin (<= 1: no TOF) */
    double tof_bin_mm;   /* width of a TOF bin along the line */
    double tof_fwhm_mm;  /* FWHM of the Gaussian timing kernel, as a distance along the line */
    double ring_mm;  /* detector ring radius (> 0: bins sampled like a ring's lines, below) */
} ora_geom;

typedef struct {
    int iterations;
    double beta, gamma_r, eps, t, U, lambda0, a, rho, delta1, delta2, nu1, nu2;
    int J0, J1;
    int precond;     /* 0 BSREM, 1 M1, 2 M2, 3 P1, 4 P2 */
    int rdp3d;       /* 0: 8 in-plane neighbours (Sec. IV-A); 1: 26 neighbours in 3-D */
    int reg;         /* 0: RDP by its gradient (the paper); 1: TV by a proximal step */
    int tv_iters;    /* primal-dual iterations per proximal step (reg = 1) */
} ora_params;

/* ---------------------------------------------------------------------------------------
 * Geometry.  theta_v = v pi / V; cos/sin values within 1e-12 of 0 are set to exactly 0 (and
 * the other to exactly +-1) so that rays at theta = 0 and pi/2 lie exactly on grid lines.
 * ------------------------------------------------------------------------------------- */
static void view_dir(const ora_geom *g, int v, double *c, double *s)
{
    double th = (double)v * 3.14159265358979323846 / (double)g->nviews;
    double cc = cos(th), ss = sin(th);
    if (fabs(cc) < 1e-12) { cc = 0.0; ss = ss > 0 ? 1.0 : -1.0; }
    if (fabs(ss) < 1e-12) { ss = 0.0; cc = cc > 0 ? 1.0 : -1.0; }
    *c = cc; *s = ss;
}

/* offset of bin b from the centre, in pixel units (uniform bins, or ring sampling) */
static double bin_offset(const ora_geom *g, int b)
{
    const double k = (double)b - 0.5 * (double)(g->nbins - 1);
    if (g->ring_mm > 0.0) return g->ring_mm * sin(k * g->bin_mm / g->ring_mm) / g->pixel_mm;
    return k * (g->bin_mm / g->pixel_mm);
}

/* the edges of bin b's width, in pixel units */
static void bin_edges(const ora_geom *g, int b, double *lo, double *hi)
{
    const double k = (double)b - 0.5 * (double)(g->nbins - 1);
    if (g->ring_mm > 0.0) {
        const double db = g->bin_mm / g->ring_mm;
        *lo = g->ring_mm * sin((k - 0.5) * db) / g->pixel_mm;
        *hi = g->ring_mm * sin((k + 0.5) * db) / g->pixel_mm;
    } else {
        *lo = (k - 0.5) * (g->bin_mm / g->pixel_mm);
        *hi = (k + 0.5) * (g->bin_mm / g->pixel_mm);
    }
}

int ora_subset_size(const ora_geom *g, int subset)
{
    int cnt = 0;
    for (int v = subset; v < g->nviews; v += g->nsubsets) cnt++;
    return cnt;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/*
 * Siddon's method for ray (v, b): fills pix[] (flat in-plane index iy*N+ix) and len[]
 * (length in pixel units) and returns the number of pieces.  Buffers need 2N+2 entries.
 * The ray is P(tau) = r (c, s) + tau (-s, c); the image is [-N/2, N/2]^2 in pixel units.
 */
static int line_pieces(const ora_geom *g, int v, double r, int *pix, double *len);

int ora_ray_pieces(const ora_geom *g, int v, int b, int *pix, double *len)
{
    return line_pieces(g, v, bin_offset(g, b), pix, len);
}

static int nsub_of(const ora_geom *g) { return g->subrays > 1 ? g->subrays : 1; }

/*
 * Pieces of bin (v, b) under the sub-ray model: the Siddon pieces of each of its R lines, each
 * length divided by R (pixels may repeat).  Buffers need R (2N + 2) entries.
 */
int ora_bin_pieces(const ora_geom *g, int v, int b, int *pix, double *len)
{
    const int R = nsub_of(g), N = g->n;
    if (R == 1) return ora_ray_pieces(g, v, b, pix, len);
    const double rho = g->bin_mm / g->pixel_mm;
    double lo, hi;
    bin_edges(g, b, &lo, &hi);
    int np = 0;
    for (int s = 0; s < R; ++s) {
        const double r = g->ring_mm > 0.0 ? lo + (s + 0.5) / R * (hi - lo)
                                          : bin_offset(g, b) + ((s + 0.5) / R - 0.5) * rho;
        const int k = line_pieces(g, v, r, pix + np, len + np);
        for (int m = np; m < np + k; ++m) len[m] /= R;
        np += k;
    }
    (void)N;
    return np;
}

/* Siddon's method for the line of view v at offset r (pixel units) from the centre. */
static int line_pieces(const ora_geom *g, int v, double r, int *pix, double *len)
{
    const int N = g->n;
    double c, s;
    view_dir(g, v, &c, &s);
    const double half = 0.5 * N;
    double *tau = (double *)malloc(sizeof(double) * (2 * N + 2));
    int nt = 0;
    /* crossings with the vertical lines X = k - N/2: X(tau) = r c - tau s */
    if (s != 0.0)
        for (int k = 0; k <= N; ++k) tau[nt++] = (r * c - ((double)k - half)) / s;
    /* crossings with the horizontal lines Y = k - N/2: Y(tau) = r s + tau c */
    if (c != 0.0)
        for (int k = 0; k <= N; ++k) tau[nt++] = (((double)k - half) - r * s) / c;
    qsort(tau, (size_t)nt, sizeof(double), cmp_double);
    int np = 0;
    for (int m = 0; m + 1 < nt; ++m) {
        double ta = tau[m], tb = tau[m + 1];
        if (!(tb > ta)) continue;
        double tm = 0.5 * (ta + tb);
        double X = r * c - tm * s, Y = r * s + tm * c;
        double fx = floor(X + half), fy = floor(Y + half);
        if (fx < 0 || fy < 0 || fx >= N || fy >= N) continue;
        pix[np] = (int)fy * N + (int)fx;
        len[np] = tb - ta;
        ++np;
    }
    free(tau);
    return np;
}

/* TOF bins per bin (1 without TOF) and "bins" per view of the sinogram (n_b T) */
static int ntof(const ora_geom *g) { return g->tof_bins > 1 ? g->tof_bins : 1; }
static int nbt(const ora_geom *g) { return g->nbins * ntof(g); }

/* h_t(tau) for TOF bin t at position tau (mm) along the line, in the form without cancellation */
double ora_tof_weight(const ora_geom *g, int t, double tau_mm)
{
    const int T = ntof(g);
    if (T == 1) return 1.0;
    const double sigma = g->tof_fwhm_mm / (2.0 * sqrt(2.0 * log(2.0)));
    const double c = ((double)t - 0.5 * (T - 1)) * g->tof_bin_mm;
    const double k = 1.0 / (sigma * sqrt(2.0));
    const double a = (tau_mm - c - 0.5 * g->tof_bin_mm) * k;   /* lower edge, scaled */
    const double b = (tau_mm - c + 0.5 * g->tof_bin_mm) * k;   /* upper edge, scaled */
    /* h = Phi(b') - Phi(a') with Phi(z) = erfc(-z / sqrt 2) / 2 */
    if (a > 0.0) return 0.5 * (erfc(a) - erfc(b));
    if (b < 0.0) return 0.5 * (erfc(-b) - erfc(-a));
    return 0.5 * (erf(b) - erf(a));
}

/* position (mm) of the centre of pixel j along the lines of view v */
static double pixel_tau_mm(const ora_geom *g, int v, int j)
{
    double c, s;
    view_dir(g, v, &c, &s);
    const double X = (double)(j % g->n) + 0.5 - 0.5 * g->n;
    const double Y = (double)(j / g->n) + 0.5 - 0.5 * g->n;
    return (-X * s + Y * c) * g->pixel_mm;
}

/* views of subset `subset` in increasing order; returns count */
static int subset_views(const ora_geom *g, int subset, int *views)
{
    int cnt = 0;
    for (int v = subset; v < g->nviews; v += g->nsubsets) views[cnt++] = v;
    return cnt;
}

/* Piece table of a list of views: for every ray (u, b), its Siddon pieces. */
typedef struct { int *pix; double *len; int *cnt; int stride; } piece_table;

static void build_pieces(const ora_geom *g, const int *views, int nv, piece_table *tb)
{
    const int N = g->n, NB = g->nbins, T = ntof(g);
    tb->stride = nsub_of(g) * (2 * N + 2);
    tb->pix = (int *)malloc(sizeof(int) * (size_t)nv * NB * T * tb->stride);
    tb->len = (double *)malloc(sizeof(double) * (size_t)nv * NB * T * tb->stride);
    tb->cnt = (int *)malloc(sizeof(int) * (size_t)nv * NB * T);
    /* ray index (u * n_b + b) * T + t: the pieces of bin (u, b), weighted by h_t at each
       piece's pixel centre */
    #pragma omp parallel for schedule(dynamic)
    for (int ray = 0; ray < nv * NB; ++ray) {
        int *pix0 = tb->pix + (size_t)ray * T * tb->stride;
        double *len0 = tb->len + (size_t)ray * T * tb->stride;
        const int cnt = ora_bin_pieces(g, views[ray / NB], ray % NB, pix0, len0);
        for (int t = T - 1; t >= 0; --t) {
            int *pix = pix0 + (size_t)t * tb->stride;
            double *len = len0 + (size_t)t * tb->stride;
            for (int m = 0; m < cnt; ++m) {
                pix[m] = pix0[m];
                len[m] = T > 1 ? len0[m] * ora_tof_weight(g, t, pixel_tau_mm(g, views[ray / NB], pix0[m]))
                               : len0[m];
            }
            tb->cnt[(size_t)ray * T + t] = cnt;
        }
    }
}

static void free_pieces(piece_table *tb) { free(tb->pix); free(tb->len); free(tb->cnt); }

static int view_list(const ora_geom *g, int subset, int *views)
{
    if (subset < 0) { for (int v = 0; v < g->nviews; ++v) views[v] = v; return g->nviews; }
    return subset_views(g, subset, views);
}

/*
 * Forward projection of one subset: y = A_i f  (Sec. II-B, the row block A_i of A).
 * f: [P][N][N]; y: [P][V_i][n_b] ([P][V_i][n_b][T] with TOF).  subset = -1 projects all
 * views into [P][V][n_b] ([P][V][n_b][T]).
 */
void ora_forward(const ora_geom *g, int subset, const double *f, double *y)
{
    const int N = g->n, P = g->nplanes, NB = nbt(g);   /* bins x TOF bins */
    int *views = (int *)malloc(sizeof(int) * g->nviews);
    const int nv = view_list(g, subset, views);
    const double scale = g->sens * g->pixel_mm;
    piece_table tb;
    build_pieces(g, views, nv, &tb);
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < P; ++p) {
        const double *fp = f + (size_t)p * N * N;
        for (int ray = 0; ray < nv * NB; ++ray) {
            const int *pix = tb.pix + (size_t)ray * tb.stride;
            const double *len = tb.len + (size_t)ray * tb.stride;
            double acc = 0.0;
            for (int m = 0; m < tb.cnt[ray]; ++m) acc += len[m] * fp[pix[m]];
            y[(size_t)p * nv * NB + ray] = scale * acc;
        }
    }
    free_pieces(&tb);
    free(views);
}

/*
 * Back projection of one subset: out = A_i^T y (ray-driven scatter, the plain transpose).
 * y: [P][V_i][n_b] (or [P][V][n_b] for subset = -1); out: [P][N][N] (overwritten).
 */
void ora_back(const ora_geom *g, int subset, const double *y, double *out)
{
    const int N = g->n, P = g->nplanes, NB = nbt(g);   /* bins x TOF bins */
    int *views = (int *)malloc(sizeof(int) * g->nviews);
    const int nv = view_list(g, subset, views);
    const double scale = g->sens * g->pixel_mm;
    piece_table tb;
    build_pieces(g, views, nv, &tb);
    memset(out, 0, sizeof(double) * (size_t)P * N * N);
    /* planes are independent: parallel over planes, each plane scatters serially */
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < P; ++p) {
        double *op = out + (size_t)p * N * N;
        for (int ray = 0; ray < nv * NB; ++ray) {
            const double w = y[(size_t)p * nv * NB + ray];
            const int *pix = tb.pix + (size_t)ray * tb.stride;
            const double *len = tb.len + (size_t)ray * tb.stride;
            for (int m = 0; m < tb.cnt[ray]; ++m) op[pix[m]] += scale * len[m] * w;
        }
    }
    free_pieces(&tb);
    free(views);
}

/* p_j of Eq. pj: (A^T 1)_j / M, or 1/M where (A^T 1)_j = 0.  p: [N][N] (same every plane). */
void ora_sensitivity(const ora_geom *g, double *pj)
{
    ora_geom g1 = *g;
    g1.nplanes = 1;
    const int N = g->n;
    double *ones = (double *)malloc(sizeof(double) * (size_t)g->nviews * nbt(g));
    for (size_t k = 0; k < (size_t)g->nviews * nbt(g); ++k) ones[k] = 1.0;
    ora_back(&g1, -1, ones, pj);
    for (int j = 0; j < N * N; ++j)
        pj[j] = pj[j] > 0.0 ? pj[j] / g->nsubsets : 1.0 / g->nsubsets;
    free(ones);
}

/* p_j of Eq. pj for the system matrix diag(a) A: (A^T a)_j / M, or 1/M where it is 0.
   a: [P][V][n_b] (NULL: a_i = 1); p: [P][N][N], one value per voxel. */
void ora_sensitivity_m(const ora_geom *g, const float *a, double *pj)
{
    const size_t q = (size_t)g->nplanes * g->n * g->n;
    const size_t nsino = (size_t)g->nplanes * g->nviews * nbt(g);
    double *ad = (double *)malloc(sizeof(double) * nsino);
    for (size_t k = 0; k < nsino; ++k) ad[k] = a ? (double)a[k] : 1.0;
    ora_back(g, -1, ad, pj);
    for (size_t j = 0; j < q; ++j)
        pj[j] = pj[j] > 0.0 ? pj[j] / g->nsubsets : 1.0 / g->nsubsets;
    free(ad);
}

/* ---------------------------------------------------------------------------------------
 * RDP (Eq. RDP) and its gradient (Eq. gradRD).  8-point in-plane neighbourhood (Sec. IV-A),
 * unweighted; neighbours outside the image do not exist.  Sum over ordered pairs (j, k).
 * ------------------------------------------------------------------------------------- */
static const int NBR_DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int NBR_DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

double ora_rdp_value(int N, int P, const double *f, double gamma_r, double eps)
{
    double R = 0.0;
    for (int p = 0; p < P; ++p) {
        const double *fp = f + (size_t)p * N * N;
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double fj = fp[iy * N + ix];
                for (int k = 0; k < 8; ++k) {
                    int x = ix + NBR_DX[k], y = iy + NBR_DY[k];
                    if (x < 0 || y < 0 || x >= N || y >= N) continue;
                    double fk = fp[y * N + x];
                    double d = fj - fk;
                    R += d * d / (fj + fk + gamma_r * fabs(d) + eps);
                }
            }
    }
    return R;
}

void ora_rdp_grad(int N, int P, const double *f, double gamma_r, double eps, double *grad)
{
    for (int p = 0; p < P; ++p) {
        const double *fp = f + (size_t)p * N * N;
        double *gp = grad + (size_t)p * N * N;
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double fj = fp[iy * N + ix], acc = 0.0;
                for (int k = 0; k < 8; ++k) {
                    int x = ix + NBR_DX[k], y = iy + NBR_DY[k];
                    if (x < 0 || y < 0 || x >= N || y >= N) continue;
                    double fk = fp[y * N + x];
                    double d = fj - fk;
                    double den = fj + fk + gamma_r * fabs(d) + eps;
                    acc += d * (gamma_r * fabs(d) + fj + 3.0 * fk + 2.0 * eps) / (den * den);
                }
                gp[iy * N + ix] = 2.0 * acc;
            }
    }
}

/*
 * Fully 3-D RDP (Eq. RDP, Eq. gradRD with the neighbourhood N_j of voxel j taken as its 26
 * neighbours in the volume: offsets (dx, dy, dz) in {-1, 0, 1}^3 other than 0, unweighted, absent
 * outside the volume).  f: [P][N][N] with the planes as the third axis.
 */
double ora_rdp_value3(int N, int P, const double *f, double gamma_r, double eps)
{
    double R = 0.0;
    for (int p = 0; p < P; ++p)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                const double fj = f[((size_t)p * N + iy) * N + ix];
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dx && !dy && !dz) continue;
                            const int x = ix + dx, y = iy + dy, z = p + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= P) continue;
                            const double fk = f[((size_t)z * N + y) * N + x];
                            const double d = fj - fk;
                            R += d * d / (fj + fk + gamma_r * fabs(d) + eps);
                        }
            }
    return R;
}

void ora_rdp_grad3(int N, int P, const double *f, double gamma_r, double eps, double *grad)
{
    for (int p = 0; p < P; ++p)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                const double fj = f[((size_t)p * N + iy) * N + ix];
                double acc = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dx && !dy && !dz) continue;
                            const int x = ix + dx, y = iy + dy, z = p + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= P) continue;
                            const double fk = f[((size_t)z * N + y) * N + x];
                            const double d = fj - fk;
                            const double den = fj + fk + gamma_r * fabs(d) + eps;
                            acc += d * (gamma_r * fabs(d) + fj + 3.0 * fk + 2.0 * eps) / (den * den);
                        }
                grad[((size_t)p * N + iy) * N + ix] = 2.0 * acc;
            }
}

/*
 * Numerical gradient of mat(f) along x and y (Sec. III, "gradient function in Matlab"):
 * central differences (f[j+1] - f[j-1]) / 2 inside, one-sided differences at the two edges,
 * unit spacing, in-plane.  gx along ix, gy along iy.
 */
void ora_matlab_gradient(int N, int P, const double *f, double *gx, double *gy)
{
    for (int p = 0; p < P; ++p) {
        const double *fp = f + (size_t)p * N * N;
        double *ox = gx + (size_t)p * N * N, *oy = gy + (size_t)p * N * N;
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double dx, dy;
                if (N == 1) dx = 0.0;
                else if (ix == 0) dx = fp[iy * N + 1] - fp[iy * N];
                else if (ix == N - 1) dx = fp[iy * N + N - 1] - fp[iy * N + N - 2];
                else dx = 0.5 * (fp[iy * N + ix + 1] - fp[iy * N + ix - 1]);
                if (N == 1) dy = 0.0;
                else if (iy == 0) dy = fp[N + ix] - fp[ix];
                else if (iy == N - 1) dy = fp[(N - 1) * N + ix] - fp[(N - 2) * N + ix];
                else dy = 0.5 * (fp[(iy + 1) * N + ix] - fp[(iy - 1) * N + ix]);
                ox[iy * N + ix] = dx;
                oy[iy * N + ix] = dy;
            }
    }
}

/*
 * The third component of Matlab's gradient of a 3-D array (planes as the third axis): central
 * differences (f[z+1] - f[z-1]) / 2 between planes, one-sided at the first and last plane, zero
 * for a single plane.
 */
void ora_matlab_gradient_z(int N, int P, const double *f, double *gz)
{
    const size_t np = (size_t)N * N;
    for (int p = 0; p < P; ++p)
        for (size_t j = 0; j < np; ++j) {
            double d;
            if (P == 1) d = 0.0;
            else if (p == 0) d = f[np + j] - f[j];
            else if (p == P - 1) d = f[(size_t)(P - 1) * np + j] - f[(size_t)(P - 2) * np + j];
            else d = 0.5 * (f[(size_t)(p + 1) * np + j] - f[(size_t)(p - 1) * np + j]);
            gz[(size_t)p * np + j] = d;
        }
}

/*
 * nu from f (Sec. III): mu = max(0.01, grad(f) / mean(f)), nu = P_{nu1}^{nu2}(mean(mu) / mu),
 * with grad(f) = sqrt(gx^2 + gy^2) (+ gz^2 for a 3-D volume, three_d != 0) and means over all
 * q = N^2 P pixels.
 */
void ora_nu_from_image3(int N, int P, const double *f, double nu1, double nu2, int three_d,
                        double *nu)
{
    size_t q = (size_t)N * N * P;
    double *gx = (double *)malloc(sizeof(double) * q), *gy = (double *)malloc(sizeof(double) * q);
    double *gz = (double *)calloc(q, sizeof(double));
    ora_matlab_gradient(N, P, f, gx, gy);
    if (three_d) ora_matlab_gradient_z(N, P, f, gz);
    double mf = 0.0;
    for (size_t j = 0; j < q; ++j) mf += f[j];
    mf /= (double)q;
    double mmu = 0.0;
    for (size_t j = 0; j < q; ++j) {
        double mu = sqrt(gx[j] * gx[j] + gy[j] * gy[j] + gz[j] * gz[j]) / mf;
        if (mu < 0.01) mu = 0.01;
        gx[j] = mu;
        mmu += mu;
    }
    mmu /= (double)q;
    for (size_t j = 0; j < q; ++j) {
        double v = mmu / gx[j];
        nu[j] = v < nu1 ? nu1 : (v > nu2 ? nu2 : v);
    }
    free(gx); free(gy); free(gz);
}

void ora_nu_from_image(int N, int P, const double *f, double nu1, double nu2, double *nu)
{
    ora_nu_from_image3(N, P, f, nu1, nu2, 0, nu);
}

/* ---------------------------------------------------------------------------------------
 * TV variant.  R_TV(f) = sum_j |(D f)_j| (isotropic total variation, in-plane): (D f)_j =
 * (f_{j+x} - f_j, f_{j+y} - f_j), a component being 0 across the last column / row, |.| the
 * Euclidean norm.  The paper handles its smooth prior by the gradient; a non-smooth prior enters
 * the same preconditioned step through its proximal operator in the metric of the step sizes:
 *   z = f - W grad F_i(f),   W_j = lambda_k alpha_{k,i} nu_j S_jj(f)
 *   x = argmin_x 1/2 sum_j (x_j - z_j)^2 / W_j + b R_TV(x),   b = beta / M,   f+ = P_t(x)
 * ora_tv_prox approximates x by `iters` iterations of the first-order primal-dual algorithm of
 * Chambolle and Pock (J. Math. Imaging Vis. 40, 2011) for min_x G(x) + F(K x), G the weighted
 * quadratic, K = b D, F the sum of Euclidean norms, with the diagonal step sizes of Pock and
 * Chambolle (ICCV 2011) for this K: sigma = 1 / (2 b) for every dual component (each row of K
 * holds b and -b) and tau = 1 / (4 b) for every voxel (a column holds at most four entries
 * +-b).  One iteration, from x = xbar = z and the dual p (one 2-vector per voxel):
 *   p    <- proj_{|p_j| <= 1}(p + sigma K xbar)            (sigma K = D / 2)
 *   x'    = (x - tau K^T p + (tau / W) z) / (1 + tau / W)  (tau K^T p = -div(p) / 4)
 *   xbar  = 2 x' - x,   x = x'
 * div(p)_j = p^x_j - p^x_{j-x} + p^y_j - p^y_{j-y}, terms outside the plane are 0.  p is in/out:
 * the loop keeps it from one subiteration to the next (0 at the start).  b = 0 gives x = z.
 * ------------------------------------------------------------------------------------- */
double ora_tv_value(int N, int P, const double *f)
{
    double R = 0.0;
    for (int p = 0; p < P; ++p) {
        const double *fp = f + (size_t)p * N * N;
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                const double c = fp[iy * N + ix];
                const double gx = ix + 1 < N ? fp[iy * N + ix + 1] - c : 0.0;
                const double gy = iy + 1 < N ? fp[(iy + 1) * N + ix] - c : 0.0;
                R += sqrt(gx * gx + gy * gy);
            }
    }
    return R;
}

void ora_tv_prox(int N, int P, const double *z, const double *W, double b, int iters,
                 double *px, double *py, double *x)
{
    const size_t q = (size_t)N * N * P;
    memcpy(x, z, sizeof(double) * q);
    if (!(b > 0.0)) return;
    double *xbar = (double *)malloc(sizeof(double) * q);
    memcpy(xbar, z, sizeof(double) * q);
    const double sigma_b = 0.5, tau = 1.0 / (4.0 * b);
    for (int it = 0; it < iters; ++it) {
        for (int p = 0; p < P; ++p)
            for (int iy = 0; iy < N; ++iy)
                for (int ix = 0; ix < N; ++ix) {
                    const size_t j = ((size_t)p * N + iy) * N + ix;
                    const double gx = ix + 1 < N ? xbar[j + 1] - xbar[j] : 0.0;
                    const double gy = iy + 1 < N ? xbar[j + N] - xbar[j] : 0.0;
                    const double qx = px[j] + sigma_b * gx, qy = py[j] + sigma_b * gy;
                    const double nq = sqrt(qx * qx + qy * qy);
                    const double sc = nq > 1.0 ? 1.0 / nq : 1.0;
                    px[j] = qx * sc;
                    py[j] = qy * sc;
                }
        for (int p = 0; p < P; ++p)
            for (int iy = 0; iy < N; ++iy)
                for (int ix = 0; ix < N; ++ix) {
                    const size_t j = ((size_t)p * N + iy) * N + ix;
                    const double div = px[j] - (ix > 0 ? px[j - 1] : 0.0) + py[j] -
                                       (iy > 0 ? py[j - N] : 0.0);
                    const double r = tau / W[j];
                    const double xn = (x[j] + 0.25 * div + r * z[j]) / (1.0 + r);
                    xbar[j] = 2.0 * xn - x[j];
                    x[j] = xn;
                }
    }
    free(xbar);
}

/* ---------------------------------------------------------------------------------------
 * Scalar schedules (Sec. III).  alpha for subiterations J = 1..nsub in order.
 * ------------------------------------------------------------------------------------- */
/* Eq. preconditioner:Nesterov: alpha = 1 + (t_J - 1) / t_{J+1}, t_{J+1} = (1 + sqrt(1 + 4 t_J^2)) / 2,
   t_1 = 1, the t sequence running on across outer iterations (t_{k+1,1} = t_{k,M+1}). */
void ora_alpha_nesterov(int nsub, double *alpha)
{
    double t = 1.0;
    for (int J = 0; J < nsub; ++J) {
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        alpha[J] = 1.0 + (t - 1.0) / tn;
        t = tn;
    }
}

/* Eq. preconditioner:KM: alpha_{k,i} = (rho (kM + i - 1) + delta2) / (kM + i - 1 + delta1). */
void ora_alpha_km(int nsub, double rho, double delta1, double delta2, double *alpha)
{
    for (int J = 1; J <= nsub; ++J)
        alpha[J - 1] = (rho * (J - 1) + delta2) / ((double)(J - 1) + delta1);
}

/* ---------------------------------------------------------------------------------------
 * Objective Phi(f) = <Af, 1> - <ln(Af + gamma), g> + beta R(f)   (Eqs. FidelityTerm,
 * ObjectiveFunction, RDP).  out[0] = <Af,1>, out[1] = <ln(Af+gamma), g>, out[2] = R, out[3] = Phi.
 * ------------------------------------------------------------------------------------- */
void ora_objective_m(const ora_geom *g, const int *counts, const float *gamma, const float *a,
                     const double *f, double beta, double gamma_r, double eps, int three_d,
                     double *out);

void ora_objective(const ora_geom *g, const int *counts, const float *gamma, const double *f,
                   double beta, double gamma_r, double eps, double *out)
{
    ora_objective_m(g, counts, gamma, NULL, f, beta, gamma_r, eps, 0, out);
}

/* As ora_objective; three_d == 1 takes R over the 26 neighbours of each voxel, three_d == 2
   takes R = R_TV (the TV variant). */
void ora_objective3(const ora_geom *g, const int *counts, const float *gamma, const double *f,
                    double beta, double gamma_r, double eps, int three_d, double *out)
{
    ora_objective_m(g, counts, gamma, NULL, f, beta, gamma_r, eps, three_d, out);
}

/* As ora_objective3 for the system matrix diag(a) A (a: [P][V][n_b], NULL: a_i = 1): the sums
   run over a_i (A f)_i. */
void ora_objective_m(const ora_geom *g, const int *counts, const float *gamma, const float *a,
                     const double *f, double beta, double gamma_r, double eps, int three_d,
                     double *out)
{
    size_t nsino = (size_t)g->nplanes * g->nviews * nbt(g);
    double *y = (double *)malloc(sizeof(double) * nsino);
    ora_forward(g, -1, f, y);
    if (a)
        for (size_t k = 0; k < nsino; ++k) y[k] *= (double)a[k];
    double s1 = 0.0, s2 = 0.0;
    for (size_t k = 0; k < nsino; ++k) {
        s1 += y[k];
        s2 += (double)counts[k] * log(y[k] + (double)gamma[k]);
    }
    double R = three_d == 2 ? ora_tv_value(g->n, g->nplanes, f)
               : three_d ? ora_rdp_value3(g->n, g->nplanes, f, gamma_r, eps)
                         : ora_rdp_value(g->n, g->nplanes, f, gamma_r, eps);
    out[0] = s1; out[1] = s2; out[2] = R; out[3] = s1 - s2 + beta * R;
    free(y);
}

/* ---------------------------------------------------------------------------------------
 * SDP-BSREM (Table I), run for `nsub` subiterations from (k, i) = (0, 1); nsub < 0 runs all
 * T M subiterations.  f: [P][N][N] in/out.  obj (optional, length T+1): Phi(f^k) at each
 * completed outer iteration k = 0..T (only for iterations reached).
 *
 * One subiteration, with J = kM + i and the subset I_i = views v == i-1 (mod M):
 *   grad   = A_i^T (1 - g_i / (A_i f + gamma_i)) + (beta / M) grad R(f)      (Eq. SubObjFunc, App. A)
 *   S_jj   = f_j / p_j  if f_j < U/2,  (U - f_j) / p_j  otherwise              (Eq. preconditioner)
 *   nu     = 1 (J <= J0) | P(mean(mu)/mu) from f (J0 < J <= J1) | frozen (J > J1)   (Eq. nuki)
 *   f~     = f - lambda_k alpha_{k,i} nu_j S_jj grad_j                             (Table I)
 *   f      = P_t(f~)                                                           (Eq. OperatorPt)
 * nu is computed from f^{k,i-1}, the iterate the preconditioner is applied to.
 * ------------------------------------------------------------------------------------- */
void ora_reconstruct_m(const ora_geom *g, const int *counts, const float *gamma, const float *a,
                       const ora_params *prm, double *f, int nsub, double *obj, double *snaps);

void ora_reconstruct(const ora_geom *g, const int *counts, const float *gamma,
                     const ora_params *prm, double *f, int nsub, double *obj)
{
    ora_reconstruct_m(g, counts, gamma, NULL, prm, f, nsub, obj, NULL);
}

/* As ora_reconstruct; snaps (optional, T x q doubles) receives f^{k+1} after each completed
   outer iteration k. */
void ora_reconstruct_snap(const ora_geom *g, const int *counts, const float *gamma,
                          const ora_params *prm, double *f, int nsub, double *obj, double *snaps)
{
    ora_reconstruct_m(g, counts, gamma, NULL, prm, f, nsub, obj, snaps);
}

/* As ora_reconstruct_snap for the system matrix diag(a) A (a: [P][V][n_b], NULL: a_i = 1):
   the forward projection is scaled by a_i before the ratio, the backprojected ratio carries
   a_i, and p_j is (A^T a)_j / M per voxel. */
void ora_reconstruct_m(const ora_geom *g, const int *counts, const float *gamma, const float *a,
                       const ora_params *prm, double *f, int nsub, double *obj, double *snaps)
{
    const int N = g->n, P = g->nplanes, M = g->nsubsets, NB = nbt(g);   /* bins x TOF bins */
    const size_t q = (size_t)N * N * P;
    const int T = prm->iterations;
    const int total = T * M;
    if (nsub < 0 || nsub > total) nsub = total;
    double *pj = (double *)malloc(sizeof(double) * q);
    ora_sensitivity_m(g, a, pj);
    double *alpha = (double *)malloc(sizeof(double) * (total > 0 ? total : 1));
    int kind = prm->precond;
    if (kind == 1 || kind == 3) ora_alpha_nesterov(total, alpha);
    else if (kind == 2 || kind == 4) ora_alpha_km(total, prm->rho, prm->delta1, prm->delta2, alpha);
    else for (int J = 0; J < total; ++J) alpha[J] = 1.0;
    const int use_nu = (kind == 3 || kind == 4);

    double *nu = (double *)malloc(sizeof(double) * q);
    double *nu_frozen = (double *)malloc(sizeof(double) * q);
    int have_frozen = 0;
    double *grad = (double *)malloc(sizeof(double) * q);
    double *rgrad = (double *)malloc(sizeof(double) * q);
    int *views = (int *)malloc(sizeof(int) * g->nviews);
    double *ysub = (double *)malloc(sizeof(double) * (size_t)P * g->nviews * NB);

    const int z3 = prm->rdp3d, tv = prm->reg == 1;
    const int rmode = tv ? 2 : z3;                      /* regulariser of the objective */
    double *px = NULL, *py = NULL, *W = NULL, *zz = NULL;
    if (tv) {
        px = (double *)calloc(q, sizeof(double));
        py = (double *)calloc(q, sizeof(double));
        W = (double *)malloc(sizeof(double) * q);
        zz = (double *)malloc(sizeof(double) * q);
    }
    if (obj) { double o[4]; ora_objective_m(g, counts, gamma, a, f, prm->beta, prm->gamma_r, prm->eps, rmode, o); obj[0] = o[3]; }
    for (int J = 1; J <= nsub; ++J) {
        const int k = (J - 1) / M, i = (J - 1) % M + 1;
        const double lambda = prm->lambda0 / (prm->a * k + 1.0);
        const int subset = i - 1;
        const int nv = subset_views(g, subset, views);
        /* nu^{k,i} (Eq. nuki) from f^{k,i-1} */
        if (!use_nu || J <= prm->J0) { for (size_t j = 0; j < q; ++j) nu[j] = 1.0; }
        else if (J <= prm->J1) {
            ora_nu_from_image3(N, P, f, prm->nu1, prm->nu2, z3, nu);
            if (J == prm->J1) { memcpy(nu_frozen, nu, sizeof(double) * q); have_frozen = 1; }
        } else {
            if (!have_frozen) { /* J1 < first dynamic J: nu^{k1,i1} with J_{k1,i1} = J1 <= J0 is 1 */
                for (size_t j = 0; j < q; ++j) nu_frozen[j] = 1.0;
                have_frozen = 1;
            }
            memcpy(nu, nu_frozen, sizeof(double) * q);
        }
        /* data term of grad Phi_i: A_i^T (1 - g_i / (A_i f + gamma_i))  (App. A); with factors
           the matrix is diag(a_i) A_i: A_i^T diag(a_i) (1 - g_i / (a_i A_i f + gamma_i)) */
        ora_forward(g, subset, f, ysub);
        for (int p = 0; p < P; ++p)
            for (int u = 0; u < nv; ++u)
                for (int b = 0; b < NB; ++b) {
                    size_t ks = ((size_t)p * nv + u) * NB + b;
                    size_t kf = ((size_t)p * g->nviews + views[u]) * NB + b;
                    if (a) {
                        const double ai = (double)a[kf];
                        ysub[ks] = ai * (1.0 - (double)counts[kf] / (ai * ysub[ks] + (double)gamma[kf]));
                    } else {
                        ysub[ks] = 1.0 - (double)counts[kf] / (ysub[ks] + (double)gamma[kf]);
                    }
                }
        ora_back(g, subset, ysub, grad);
        if (tv) {
            /* TV variant: the data step, then the proximal step of (beta / M) R_TV */
            for (size_t j = 0; j < q; ++j) {
                const double fj = f[j], pjj = pj[j];
                const double S = fj < 0.5 * prm->U ? fj / pjj : (prm->U - fj) / pjj;
                W[j] = lambda * alpha[J - 1] * nu[j] * S;
                zz[j] = fj - W[j] * grad[j];
            }
            ora_tv_prox(N, P, zz, W, prm->beta / M, prm->tv_iters, px, py, f);
            for (size_t j = 0; j < q; ++j) {
                if (f[j] <= 0.0) f[j] = prm->t;
                else if (f[j] >= prm->U) f[j] = prm->U - prm->t;
            }
        } else {
        /* penalty term (beta / M) grad R  (Eq. SubObjFunc, Eq. gradRD) */
        if (z3) ora_rdp_grad3(N, P, f, prm->gamma_r, prm->eps, rgrad);
        else ora_rdp_grad(N, P, f, prm->gamma_r, prm->eps, rgrad);
        for (size_t j = 0; j < q; ++j) {
            const double d = grad[j] + prm->beta / M * rgrad[j];
            const double fj = f[j], pjj = pj[j];
            const double S = fj < 0.5 * prm->U ? fj / pjj : (prm->U - fj) / pjj;
            double ft = fj - lambda * alpha[J - 1] * nu[j] * S * d;
            if (ft <= 0.0) ft = prm->t;
            else if (ft >= prm->U) ft = prm->U - prm->t;
            f[j] = ft;
        }
        }
        if (obj && i == M) {
            double o[4];
            ora_objective_m(g, counts, gamma, a, f, prm->beta, prm->gamma_r, prm->eps, rmode, o);
            obj[k + 1] = o[3];
        }
        if (snaps && i == M) memcpy(snaps + (size_t)k * q, f, sizeof(double) * q);
    }
    free(pj); free(alpha); free(nu); free(nu_frozen); free(grad); free(rgrad);
    free(views); free(ysub); free(px); free(py); free(W); free(zz);
}
