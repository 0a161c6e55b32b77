/*
 * FP64 oracle of the FoE-regularised Poisson denoiser (Feng, Qiao, Chen, arXiv:1609.05722).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * legs may load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every quantity is computed in double precision by direct loops, in the order the paper
 * states it.  No blocking, no fusion, no reordering beyond the formulas.  The only
 * parallelism is an optional split of image rows over threads; every output element is
 * computed by the same sequence of operations whatever the thread count, so results do not
 * depend on it.
 *
 * Conventions (readings of places where the paper is silent; each is listed in the design
 * notes):
 *   - images are row-major H x W;
 *   - filters are convolution kernels, k[i*49 + (a+3)*7 + (b+3)] = k_i(a, b), a, b in -3..3,
 *     and (k * u)_p = sum_{a,b} k(a, b) u(p - (a, b))  (Sec. 2.3, Eq. FOEmodel: "convolution");
 *   - responses exist only at the N pixels of the image (K_i is N x N, Sec. 2.5.2); they are
 *     taken on a padded image P u.  bc = 0: half-sample symmetric padding (index -1 -> 0,
 *     -2 -> 1, ...); bc = 1: zero padding.  K_i = K_i,valid P and K_i^T = P^T K_i,valid^T;
 *   - model 0 = direct I-divergence model (Eq. straightforward), 1 = Anscombe-domain
 *     quadratic model (Eq. overallModel), 2 = Anscombe-domain I-divergence model (Eq. lowcase,
 *     with the weights alpha_i kept as in Eq. FOEscheme).
 *
 * Parity pins: see the "-m 'not gpu'" oracle tests.  Every function below is pinned.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KS 7
#define ORC_KK 49
#define ORC_R 3

/* ------------------------------------------------------------------------------------------
 * Scalars: Anscombe transform (Eq. Anscombetransform), closed-form unbiased inverse (Eq.
 * invAns) and its derivative (Sec. 3.2, I_C'), potential rho and its derivatives (Eq. STfunc,
 * Sec. 2.5.2).
 * ---------------------------------------------------------------------------------------- */
double orc_anscombe1(double y) { return 2.0 * sqrt(y + 3.0 / 8.0); }

double orc_ic1(double z)
{
    const double s = sqrt(1.5);
    return 0.25 * z * z + 0.25 * s / z - (11.0 / 8.0) / (z * z) + (5.0 / 8.0) * s / (z * z * z) - 0.125;
}

double orc_ic_deriv1(double z)
{
    const double s = sqrt(1.5);
    return 0.5 * z - 0.25 * s / (z * z) + (11.0 / 4.0) / (z * z * z) - (15.0 / 8.0) * s / (z * z * z * z);
}

double orc_rho(double z) { return log1p(z * z); }
double orc_rho1(double z) { return 2.0 * z / (1.0 + z * z); }
double orc_rho2(double z)
{
    const double q = 1.0 + z * z;
    return 2.0 * (1.0 - z * z) / (q * q);
}

void orc_anscombe(long n, const double *y, double *v)
{
    for (long i = 0; i < n; ++i) v[i] = orc_anscombe1(y[i]);
}

/* x = I_C(max(z, sqrt(3/2))): the clamp keeps the output >= 0 (I_C(sqrt(3/2)) = 0). */
void orc_inverse(long n, const double *z, double *x)
{
    const double zmin = sqrt(1.5);
    for (long i = 0; i < n; ++i) x[i] = orc_ic1(z[i] > zmin ? z[i] : zmin);
}

/* ------------------------------------------------------------------------------------------
 * Padding operator P.
 * ---------------------------------------------------------------------------------------- */
long orc_pad_index(long i, long n, int bc)
{
    if (bc == 1) return (i >= 0 && i < n) ? i : -1;
    while (i < 0 || i >= n) {
        if (i < 0) i = -1 - i;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

/* ------------------------------------------------------------------------------------------
 * Row-parallel helper.
 * ---------------------------------------------------------------------------------------- */
typedef void (*orc_rowfn)(void *ctx, long r0, long r1);
typedef struct { orc_rowfn fn; void *ctx; long r0, r1; } orc_job;

static void *orc_job_run(void *p)
{
    orc_job *j = (orc_job *)p;
    j->fn(j->ctx, j->r0, j->r1);
    return NULL;
}

static void orc_par_rows(long nrows, int nthreads, orc_rowfn fn, void *ctx)
{
    if (nthreads <= 1 || nrows < 2 * nthreads) {
        fn(ctx, 0, nrows);
        return;
    }
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    orc_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].r0 = nrows * t / nthreads;
        jobs[t].r1 = nrows * (t + 1) / nthreads;
    }
    int started[256];
    for (int t = 0; t < nthreads; ++t) started[t] = pthread_create(&th[t], NULL, orc_job_run, &jobs[t]) == 0;
    for (int t = 0; t < nthreads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else orc_job_run(&jobs[t]);
    }
}

/* ------------------------------------------------------------------------------------------
 * K_i u: r(y, x) = sum_{a,b} k_i(a, b) (P u)(y - a, x - b) for (y, x) in the image.
 * Each output accumulates its 49 products in tap order (a, then b); the loop over x is innermost
 * only so that the compiler can vectorise it; this does not change any element's arithmetic.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int nf;
    const double *k;  /* nf x 49 */
    const double *pu; /* padded image, (H+6) x (W+6), origin at (-3, -3) */
    int H, W;
    double *r;        /* nf x H x W */
} orc_resp_ctx;

static void orc_resp_rows(void *c, long r0, long r1)
{
    orc_resp_ctx *q = (orc_resp_ctx *)c;
    const long PW = q->W + 2 * ORC_R;
    for (int i = 0; i < q->nf; ++i)
        for (long y = r0; y < r1; ++y) {
            double *row = q->r + (size_t)i * q->H * q->W + y * q->W;
            for (long x = 0; x < q->W; ++x) row[x] = 0.0;
            for (int a = -ORC_R; a <= ORC_R; ++a)
                for (int b = -ORC_R; b <= ORC_R; ++b) {
                    const double kv = q->k[(size_t)i * ORC_KK + (a + ORC_R) * ORC_KS + (b + ORC_R)];
                    const double *src = q->pu + (y - a + ORC_R) * PW + (ORC_R - b);
                    for (long x = 0; x < q->W; ++x) row[x] += kv * src[x];
                }
        }
}

static void orc_pad_image(int H, int W, const double *u, int bc, double *pu)
{
    const long PW = W + 2 * ORC_R;
    for (long yp = -ORC_R; yp < H + ORC_R; ++yp)
        for (long xp = -ORC_R; xp < W + ORC_R; ++xp) {
            long sy = orc_pad_index(yp, H, bc), sx = orc_pad_index(xp, W, bc);
            pu[(yp + ORC_R) * PW + (xp + ORC_R)] = (sy < 0 || sx < 0) ? 0.0 : u[sy * W + sx];
        }
}

/* r[i*H*W + p] = (K_i u)_p for all filters. */
void orc_responses(int nf, const double *k, int H, int W, const double *u, int bc, double *r, int nthreads)
{
    double *pu = (double *)malloc(sizeof(double) * (size_t)(H + 2 * ORC_R) * (W + 2 * ORC_R));
    if (!pu) return;
    orc_pad_image(H, W, u, bc, pu);
    orc_resp_ctx c = {nf, k, pu, H, W, r};
    orc_par_rows(H, nthreads, orc_resp_rows, &c);
    free(pu);
}

/* ------------------------------------------------------------------------------------------
 * K^T psi = sum_i P^T K_i,valid^T psi_i.
 *   h(q') = sum_i sum_{a,b} k_i(a, b) psi_i(q' + (a, b)) over q' + (a, b) in the image, for
 *           every padded position q' (3-pixel border);
 *   g(q)  = sum of h(q') over the padded positions q' that P maps to q.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int nf;
    const double *k;
    const double *psi;
    int H, W;
    double *h; /* (H+6) x (W+6), origin at (-3, -3) */
} orc_adj_ctx;

static void orc_adj_rows(void *c, long r0, long r1)
{
    orc_adj_ctx *q = (orc_adj_ctx *)c;
    const long PW = q->W + 2 * ORC_R;
    for (long row = r0; row < r1; ++row) {
        const long yp = row - ORC_R;
        double *hrow = q->h + row * PW; /* hrow[xp + 3] = h(yp, xp) */
        for (long j = 0; j < PW; ++j) hrow[j] = 0.0;
        for (int i = 0; i < q->nf; ++i)
            for (int a = -ORC_R; a <= ORC_R; ++a) {
                const long py = yp + a;
                if (py < 0 || py >= q->H) continue;
                const double *prow = q->psi + (size_t)i * q->H * q->W + py * q->W;
                for (int b = -ORC_R; b <= ORC_R; ++b) {
                    const double kv = q->k[(size_t)i * ORC_KK + (a + ORC_R) * ORC_KS + (b + ORC_R)];
                    /* xp + b must lie in [0, W) */
                    long x0 = -ORC_R, x1 = q->W + ORC_R;
                    if (x0 < -b) x0 = -b;
                    if (x1 > q->W - b) x1 = q->W - b;
                    for (long xp = x0; xp < x1; ++xp) hrow[xp + ORC_R] += kv * prow[xp + b];
                }
            }
    }
}

void orc_adjoint(int nf, const double *k, int H, int W, const double *psi, int bc, double *g, int nthreads)
{
    const long PH = H + 2 * ORC_R, PW = W + 2 * ORC_R;
    double *h = (double *)malloc(sizeof(double) * (size_t)PH * PW);
    if (!h) return;
    orc_adj_ctx c = {nf, k, psi, H, W, h};
    orc_par_rows(PH, nthreads, orc_adj_rows, &c);
    for (long i = 0; i < (long)H * W; ++i) g[i] = 0.0;
    for (long yp = -ORC_R; yp < H + ORC_R; ++yp)
        for (long xp = -ORC_R; xp < W + ORC_R; ++xp) {
            long sy = orc_pad_index(yp, H, bc), sx = orc_pad_index(xp, W, bc);
            if (sy < 0 || sx < 0) continue;
            g[sy * W + sx] += h[(yp + ORC_R) * PW + (xp + ORC_R)];
        }
    free(h);
}

/* ------------------------------------------------------------------------------------------
 * FoE prior energy (Eq. FOEmodel) and its gradient (Eq. FoEF).
 * ---------------------------------------------------------------------------------------- */
double orc_prior_energy(int nf, const double *k, const double *alpha, int H, int W, const double *u, int bc,
                        int nthreads)
{
    const long N = (long)H * W;
    double *r = (double *)malloc(sizeof(double) * (size_t)nf * N);
    if (!r) return NAN;
    orc_responses(nf, k, H, W, u, bc, r, nthreads);
    double e = 0.0;
    for (int i = 0; i < nf; ++i) {
        double ei = 0.0;
        for (long p = 0; p < N; ++p) ei += orc_rho(r[(size_t)i * N + p]);
        e += alpha[i] * ei;
    }
    free(r);
    return e;
}

void orc_prior_grad(int nf, const double *k, const double *alpha, int H, int W, const double *u, int bc, double *g,
                    int nthreads)
{
    const long N = (long)H * W;
    double *r = (double *)malloc(sizeof(double) * (size_t)nf * N);
    if (!r) return;
    orc_responses(nf, k, H, W, u, bc, r, nthreads);
    for (int i = 0; i < nf; ++i)
        for (long p = 0; p < N; ++p) r[(size_t)i * N + p] = alpha[i] * orc_rho1(r[(size_t)i * N + p]);
    orc_adjoint(nf, k, H, W, r, bc, g, nthreads);
    free(r);
}

/* ------------------------------------------------------------------------------------------
 * Data terms: I-divergence <u - d log u, 1> (Eq. poissonfidelity; models 0 and 2) and the
 * quadratic 1/2 ||u - d||^2 (Eq. overallModel; model 1), each times lambda.  0 log 0 = 0.
 * ---------------------------------------------------------------------------------------- */
double orc_data_energy(int model, double lambda, long n, const double *u, const double *d)
{
    double e = 0.0;
    for (long i = 0; i < n; ++i) {
        if (model == 1) {
            e += 0.5 * (u[i] - d[i]) * (u[i] - d[i]);
        } else {
            if (d[i] == 0.0) e += u[i];
            else if (u[i] <= 0.0) return INFINITY;
            else e += u[i] - d[i] * log(u[i]);
        }
    }
    return lambda * e;
}

void orc_data_grad(int model, double lambda, long n, const double *u, const double *d, double *g)
{
    for (long i = 0; i < n; ++i) g[i] = (model == 1) ? lambda * (u[i] - d[i]) : lambda * (1.0 - d[i] / u[i]);
}

/* Proximal map (I + tau dG)^{-1}, tl = tau * lambda:
 *   I-divergence (Eq. subproblemGIdiv): (ut - tl + sqrt((ut - tl)^2 + 4 tl d)) / 2;
 *   quadratic    (Eq. subproblemGL2):   (ut + tl d) / (1 + tl). */
void orc_prox(int model, double tl, long n, const double *ut, const double *d, double *out)
{
    for (long i = 0; i < n; ++i) {
        if (model == 1) out[i] = (ut[i] + tl * d[i]) / (1.0 + tl);
        else {
            double t = ut[i] - tl;
            out[i] = 0.5 * (t + sqrt(t * t + 4.0 * tl * d[i]));
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * iPiano (Eq. iPianoupdate): u+ = prox_{tau G}(u - tau grad F(u) + gamma (u - u-)).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int nf;
    const double *k;
    const double *alpha;
    int H, W, bc, model;
    double lambda, tau, gamma;
    int nthreads;
} orc_params;

double orc_energy(const orc_params *p, const double *u, const double *d)
{
    return orc_prior_energy(p->nf, p->k, p->alpha, p->H, p->W, u, p->bc, p->nthreads) +
           orc_data_energy(p->model, p->lambda, (long)p->H * p->W, u, d);
}

/* Energy and gradient of the whole objective E = F + G at u. */
double orc_energy_grad(const orc_params *p, const double *u, const double *d, double *g)
{
    const long N = (long)p->H * p->W;
    double *gd = (double *)malloc(sizeof(double) * (size_t)N);
    if (!gd) return NAN;
    orc_prior_grad(p->nf, p->k, p->alpha, p->H, p->W, u, p->bc, g, p->nthreads);
    orc_data_grad(p->model, p->lambda, N, u, d, gd);
    for (long i = 0; i < N; ++i) g[i] += gd[i];
    free(gd);
    return orc_energy(p, u, d);
}

/* One step: u_next from (u, u_prev). */
void orc_ipiano_step(const orc_params *p, const double *d, const double *u, const double *u_prev, double *u_next)
{
    const long N = (long)p->H * p->W;
    double *g = (double *)malloc(sizeof(double) * (size_t)N);
    double *ut = (double *)malloc(sizeof(double) * (size_t)N);
    if (!g || !ut) { free(g); free(ut); return; }
    orc_prior_grad(p->nf, p->k, p->alpha, p->H, p->W, u, p->bc, g, p->nthreads);
    for (long i = 0; i < N; ++i) ut[i] = u[i] - p->tau * g[i] + p->gamma * (u[i] - u_prev[i]);
    orc_prox(p->model, p->tau * p->lambda, N, ut, d, u_next);
    free(g);
    free(ut);
}

/* Runs iters steps.  On entry u = u^0, u_prev = u^{-1}; on exit u = u^iters, u_prev = u^{iters-1}.
 * energy (nullable, iters + 1 values) receives E(u^n) for n = 0..iters. */
int orc_ipiano(const orc_params *p, const double *d, double *u, double *u_prev, int iters, double *energy)
{
    const long N = (long)p->H * p->W;
    double *un = (double *)malloc(sizeof(double) * (size_t)N);
    if (!un) return -1;
    if (energy) energy[0] = orc_energy(p, u, d);
    for (int n = 0; n < iters; ++n) {
        orc_ipiano_step(p, d, u, u_prev, un);
        memcpy(u_prev, u, sizeof(double) * (size_t)N);
        memcpy(u, un, sizeof(double) * (size_t)N);
        if (energy) energy[n + 1] = orc_energy(p, u, d);
    }
    free(un);
    return 0;
}

/* Stopping rule (the paper fixes none; it reports the iteration counts of its runs, Sec. 5.1): after step n, for n
 * a multiple of check_every, the solve stops at u^n once ||u^n - u^{n-1}||_2 <= tol ||u^n||_2 (sums in FP64).  Runs
 * at most iters steps like orc_ipiano and returns the number of steps taken (tol <= 0: never stops early). */
int orc_ipiano_tol(const orc_params *p, const double *d, double *u, double *u_prev, int iters, double tol,
                   int check_every)
{
    const long N = (long)p->H * p->W;
    double *un = (double *)malloc(sizeof(double) * (size_t)N);
    if (!un) return -1;
    int n = 0;
    while (n < iters) {
        orc_ipiano_step(p, d, u, u_prev, un);
        memcpy(u_prev, u, sizeof(double) * (size_t)N);
        memcpy(u, un, sizeof(double) * (size_t)N);
        ++n;
        if (tol > 0.0 && check_every > 0 && n % check_every == 0) {
            double dd = 0.0, uu = 0.0;
            for (long i = 0; i < N; ++i) {
                const double e = u[i] - u_prev[i];
                dd += e * e;
                uu += u[i] * u[i];
            }
            if (sqrt(dd) <= tol * sqrt(uu)) break;
        }
    }
    free(un);
    return n;
}

/* Whole denoiser for one image: data -> iPiano -> output.
 *   model 0 (direct, Eq. straightforward): d = y with zeros replaced by zero_c (Sec. 3.1.1),
 *           x = u^T;
 *   model 1/2 (Eq. overallModel / lowcase): d = Anscombe(y), x = I_C(max(u^T, sqrt(3/2)));
 *   model 3 (Eq. FOEscheme): 1 if peak >= 5 else 2.
 * Initial iterates u^0 = u^{-1} = d. */
int orc_denoise_tol(const orc_params *p_in, const double *y, double peak, double zero_c, int iters, double tol,
                    int check_every, double *x, int *iters_done);

int orc_denoise(const orc_params *p_in, const double *y, double peak, double zero_c, int iters, double *x)
{
    return orc_denoise_tol(p_in, y, peak, zero_c, iters, 0.0, 0, x, NULL);
}

/* The same with the stopping rule of orc_ipiano_tol; *iters_done (nullable) receives the steps taken. */
int orc_denoise_tol(const orc_params *p_in, const double *y, double peak, double zero_c, int iters, double tol,
                    int check_every, double *x, int *iters_done)
{
    orc_params p = *p_in;
    if (p.model == 3) p.model = (peak >= 5.0) ? 1 : 2;
    const long N = (long)p.H * p.W;
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    double *u = (double *)malloc(sizeof(double) * (size_t)N);
    double *up = (double *)malloc(sizeof(double) * (size_t)N);
    if (!d || !u || !up) { free(d); free(u); free(up); return -1; }
    if (p.model == 0) {
        for (long i = 0; i < N; ++i) d[i] = (y[i] == 0.0) ? zero_c : y[i];
    } else {
        orc_anscombe(N, y, d);
    }
    memcpy(u, d, sizeof(double) * (size_t)N);
    memcpy(up, d, sizeof(double) * (size_t)N);
    const int done = orc_ipiano_tol(&p, d, u, up, iters, tol, check_every);
    if (iters_done) *iters_done = done;
    if (p.model == 0) memcpy(x, u, sizeof(double) * (size_t)N);
    else orc_inverse(N, u, x);
    free(d);
    free(u);
    free(up);
    return p.model;
}

/* ------------------------------------------------------------------------------------------
 * Binning variant (FoEPNRbin, Sec. 4, comparison to the state of the art): a 3x3 ones kernel sums the counts of
 * each bin, which raises the peak nine-fold; the binned image is denoised with the binned peak deciding the data
 * term (Sec. 3.4 after Eq. FOEscheme: the threshold stays at peak 5, applied to the binned image); the low-resolution estimate is
 * brought back to full size by bilinear interpolation.  The paper fixes neither the bin grid at ragged borders
 * nor the interpolation grid; the readings taken here:
 *   - bins are the non-overlapping 3x3 blocks starting at pixel (0, 0), ceil(H/3) x ceil(W/3) of them; a block
 *     cut by the image border sums its n < 9 pixels and is scaled by 9 / n, so that every bin estimates nine
 *     times the local intensity;
 *   - the estimate at pixel (r, c) is the bilinear interpolation of the bin image at ((r - 1) / 3, (c - 1) / 3)
 *     (bin (I, J) centred on pixel (3I + 1, 3J + 1)), with coordinates clamped to the edge bins, divided by 9.
 * ---------------------------------------------------------------------------------------- */
void orc_bin3(int H, int W, const double *y, double *yb)
{
    const int Hb = (H + 2) / 3, Wb = (W + 2) / 3;
    for (int I = 0; I < Hb; ++I)
        for (int J = 0; J < Wb; ++J) {
            double s = 0.0;
            int n = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const int r = 3 * I + a, c = 3 * J + b;
                    if (r < H && c < W) {
                        s += y[(long)r * W + c];
                        ++n;
                    }
                }
            yb[(long)I * Wb + J] = s * 9.0 / n;
        }
}

static int orc_clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

void orc_upscale3(int Hb, int Wb, const double *xb, int H, int W, double *x)
{
    for (int r = 0; r < H; ++r) {
        const double fy = (r - 1) / 3.0;
        const int y0 = (int)floor(fy);
        const double wy = fy - y0;
        const int ya = orc_clampi(y0, 0, Hb - 1), yc = orc_clampi(y0 + 1, 0, Hb - 1);
        for (int c = 0; c < W; ++c) {
            const double fx = (c - 1) / 3.0;
            const int x0 = (int)floor(fx);
            const double wx = fx - x0;
            const int xa = orc_clampi(x0, 0, Wb - 1), xc = orc_clampi(x0 + 1, 0, Wb - 1);
            const double top = (1.0 - wx) * xb[(long)ya * Wb + xa] + wx * xb[(long)ya * Wb + xc];
            const double bot = (1.0 - wx) * xb[(long)yc * Wb + xa] + wx * xb[(long)yc * Wb + xc];
            x[(long)r * W + c] = ((1.0 - wy) * top + wy * bot) / 9.0;
        }
    }
}

/* Bin, denoise at nine times the peak, upscale.  p_in->H, p_in->W are the full image sizes; returns the model
 * used on the binned image (or -1). */
int orc_denoise_binned(const orc_params *p_in, const double *y, double peak, double zero_c, int iters, double *x)
{
    orc_params p = *p_in;
    const int Hb = (p.H + 2) / 3, Wb = (p.W + 2) / 3;
    double *yb = (double *)malloc(sizeof(double) * (size_t)Hb * Wb);
    double *xb = (double *)malloc(sizeof(double) * (size_t)Hb * Wb);
    if (!yb || !xb) {
        free(yb);
        free(xb);
        return -1;
    }
    orc_bin3(p.H, p.W, y, yb);
    p.H = Hb;
    p.W = Wb;
    const int used = orc_denoise(&p, yb, 9.0 * peak, zero_c, iters, xb);
    orc_upscale3(Hb, Wb, xb, p_in->H, p_in->W, x);
    free(yb);
    free(xb);
    return used;
}

/* ------------------------------------------------------------------------------------------
 * Step size.  L = 2 kappa max_w sum_i alpha_i |k_i^(w)|^2 bounds the Lipschitz constant of grad F
 * (|rho''| <= 2; the symbol maximum bounds sum_i alpha_i K_i,valid^T K_i,valid; ||P||^2 <= kappa with
 * kappa = 4 for symmetric padding when H, W >= 6, 1 for zero padding).  The maximum is taken on an
 * ngrid x ngrid DTFT grid.
 * ---------------------------------------------------------------------------------------- */
double orc_lipschitz(int nf, const double *k, const double *alpha, int bc, int ngrid)
{
    double best = 0.0;
    for (int iy = 0; iy < ngrid; ++iy)
        for (int ix = 0; ix < ngrid; ++ix) {
            double wy = 2.0 * M_PI * iy / ngrid, wx = 2.0 * M_PI * ix / ngrid;
            double s = 0.0;
            for (int i = 0; i < nf; ++i) {
                double re = 0.0, im = 0.0;
                for (int a = -ORC_R; a <= ORC_R; ++a)
                    for (int b = -ORC_R; b <= ORC_R; ++b) {
                        double kv = k[(size_t)i * ORC_KK + (a + ORC_R) * ORC_KS + (b + ORC_R)];
                        re += kv * cos(wy * a + wx * b);
                        im -= kv * sin(wy * a + wx * b);
                    }
                s += alpha[i] * (re * re + im * im);
            }
            if (s > best) best = s;
        }
    return 2.0 * (bc == 1 ? 1.0 : 4.0) * best;
}

/* PSNR on the [0, 255] scale: both images are scaled by 255 / peak. */
double orc_psnr(long n, const double *a, const double *b, double peak)
{
    double s = 0.0, f = 255.0 / peak;
    for (long i = 0; i < n; ++i) {
        double e = f * (a[i] - b[i]);
        s += e * e;
    }
    double mse = s / (double)n;
    return 10.0 * log10(255.0 * 255.0 / mse);
}

/* ------------------------------------------------------------------------------------------
 * Training (Sec. 2.5, Eq. learningmodel; loss of Sec. 3.2: l = 1/2 ||I_C(u) - g||^2 per image).
 * The lower-level solve is T unrolled iPiano steps of the Anscombe quadratic model (Eq. overallModel,
 * prox Eq. subproblemGL2) from u^0 = u^{-1} = v; the parameters are the filters k_i (convolution
 * orientation) and the log-weights a_i, alpha_i = e^{a_i} (Eq. learningmodel).  The gradient is taken by
 * reverse-mode differentiation of the unrolled iteration:
 *   u^{n+1} = c1 (u^n - tau grad F(u^n) + gamma (u^n - u^{n-1})) + c2 v,   c1 = 1/(1+tau lambda),
 *   gbar^T = I_C'(u^T) (I_C(u^T) - g)   (0 where the output clamp max(u, sqrt(3/2)) is active),
 *   w = c1 gbar^{n+1},
 *   gbar^n = (1 + gamma) w - tau H(u^n) w - gamma c1 gbar^{n+2},  H(u) w = sum_i alpha_i K_i^T (rho''(K_i u) K_i w)
 *            (Hessian of the prior, Sec. 2.5.2),
 *   dL/da_i     += -tau alpha_i sum_p (K_i w)_p rho'((K_i u^n)_p),
 *   dL/dk_i(a,b) += -tau alpha_i sum_p [ (P w)(p - (a,b)) rho'(r_i(p)) + (K_i w)_p rho''(r_i(p)) (P u^n)(p - (a,b)) ].
 * ---------------------------------------------------------------------------------------- */
static double orc_loss_one(const double *u, const double *g, long N, double *gbar)
{
    const double zmin = sqrt(1.5);
    double L = 0.0;
    for (long i = 0; i < N; ++i) {
        const double z = u[i] > zmin ? u[i] : zmin;
        const double e = orc_ic1(z) - g[i];
        L += 0.5 * e * e;
        if (gbar) gbar[i] = u[i] > zmin ? orc_ic_deriv1(u[i]) * e : 0.0;
    }
    return L;
}

/* Runs the T-step forward solve of one image; U receives u^0..u^T ((T+1) x N). */
static void orc_train_forward(const orc_params *p, const double *y, int T, double *v, double *U)
{
    const long N = (long)p->H * p->W;
    orc_anscombe(N, y, v);
    memcpy(U, v, sizeof(double) * (size_t)N);
    for (int n = 0; n < T; ++n)
        orc_ipiano_step(p, v, U + (size_t)n * N, n == 0 ? v : U + (size_t)(n - 1) * N, U + (size_t)(n + 1) * N);
}

double orc_train_loss(const orc_params *p, int B, const double *clean, const double *noisy, int T)
{
    const long N = (long)p->H * p->W;
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
    double *U = (double *)malloc(sizeof(double) * (size_t)N * (T + 1));
    if (!v || !U) { free(v); free(U); return NAN; }
    double L = 0.0;
    for (int s = 0; s < B; ++s) {
        orc_train_forward(p, noisy + (size_t)s * N, T, v, U);
        L += orc_loss_one(U + (size_t)T * N, clean + (size_t)s * N, N, NULL);
    }
    free(v);
    free(U);
    return L;
}

double orc_train_grad(const orc_params *p, int B, const double *clean, const double *noisy, int T, double *dk,
                      double *dlogalpha)
{
    const int nf = p->nf, H = p->H, W = p->W;
    const long N = (long)H * W, PW = W + 2 * ORC_R, PN = (long)(H + 2 * ORC_R) * PW;
    const double c1 = 1.0 / (1.0 + p->tau * p->lambda);
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
    double *U = (double *)malloc(sizeof(double) * (size_t)N * (T + 1));
    double *gb1 = (double *)calloc((size_t)N, sizeof(double));   /* gbar^{n+1} */
    double *gb2 = (double *)calloc((size_t)N, sizeof(double));   /* gbar^{n+2} */
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *r = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *sv = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *psi = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *Hw = (double *)malloc(sizeof(double) * (size_t)N);
    double *pu = (double *)malloc(sizeof(double) * (size_t)PN);
    double *pw = (double *)malloc(sizeof(double) * (size_t)PN);
    double L = NAN;
    if (!v || !U || !gb1 || !gb2 || !w || !r || !sv || !psi || !Hw || !pu || !pw) goto done;
    for (int i = 0; i < nf * ORC_KK; ++i) dk[i] = 0.0;
    for (int i = 0; i < nf; ++i) dlogalpha[i] = 0.0;
    L = 0.0;
    for (int s = 0; s < B; ++s) {
        orc_train_forward(p, noisy + (size_t)s * N, T, v, U);
        L += orc_loss_one(U + (size_t)T * N, clean + (size_t)s * N, N, gb1);
        for (long i = 0; i < N; ++i) gb2[i] = 0.0;
        for (int n = T - 1; n >= 0; --n) {
            const double *un = U + (size_t)n * N;
            for (long i = 0; i < N; ++i) w[i] = c1 * gb1[i];
            orc_responses(nf, p->k, H, W, un, p->bc, r, p->nthreads);
            orc_responses(nf, p->k, H, W, w, p->bc, sv, p->nthreads);
            orc_pad_image(H, W, un, p->bc, pu);
            orc_pad_image(H, W, w, p->bc, pw);
            for (int f = 0; f < nf; ++f) {
                const double *rf = r + (size_t)f * N, *sf = sv + (size_t)f * N;
                double ga = 0.0;
                for (long q = 0; q < N; ++q) ga += sf[q] * orc_rho1(rf[q]);
                dlogalpha[f] += -p->tau * p->alpha[f] * ga;
                for (int a = -ORC_R; a <= ORC_R; ++a)
                    for (int b = -ORC_R; b <= ORC_R; ++b) {
                        double gk = 0.0;
                        for (long y = 0; y < H; ++y)
                            for (long x = 0; x < W; ++x) {
                                const long q = y * W + x, pi = (y - a + ORC_R) * PW + (x - b + ORC_R);
                                gk += pw[pi] * orc_rho1(rf[q]) + sf[q] * orc_rho2(rf[q]) * pu[pi];
                            }
                        dk[(size_t)f * ORC_KK + (a + ORC_R) * ORC_KS + (b + ORC_R)] += -p->tau * p->alpha[f] * gk;
                    }
                for (long q = 0; q < N; ++q) psi[(size_t)f * N + q] = p->alpha[f] * orc_rho2(rf[q]) * sf[q];
            }
            if (n >= 1) {
                orc_adjoint(nf, p->k, H, W, psi, p->bc, Hw, p->nthreads);
                for (long i = 0; i < N; ++i) {
                    const double gn = (1.0 + p->gamma) * w[i] - p->tau * Hw[i] - p->gamma * c1 * gb2[i];
                    gb2[i] = gb1[i];
                    gb1[i] = gn;
                }
            }
        }
    }
done:
    free(v); free(U); free(gb1); free(gb2); free(w); free(r); free(sv); free(psi); free(Hw); free(pu); free(pw);
    return L;
}

/* ------------------------------------------------------------------------------------------
 * The paper's own training gradient (Sec. 2.5, Eq. implicitdifferentiation and Eq. overallderivative), for the
 * Anscombe quadratic model E(w) = E_FoE(w) + lambda/2 ||w - v||^2 and the loss of Sec. 3.2:
 *   q = H_E(w*)^{-1} dL/dw at the minimiser w*,
 *   H_E(w) = sum_i alpha_i K_i^T Gamma_i K_i + lambda I,   Gamma_i = diag(rho''(K_i w))        (Sec. 2.5),
 *   dL/da_i      = -alpha_i (K_i^T rho'(K_i w*))^T q = -alpha_i sum_p (K_i q)_p rho'(r_i(p)),
 *   dL/dk_i(a,b) = -alpha_i sum_p [ (P q)(p - (a,b)) rho'(r_i(p)) + (K_i q)_p rho''(r_i(p)) (P w*)(p - (a,b)) ],
 * with r_i = K_i w* and the filter coefficients themselves as parameters (the basis B of Eq. filtercoe is the
 * identity).  w* is approximated by T iPiano steps from v; q by conjugate gradients from q = 0, stopped when
 * ||dL/dw - H_E q|| <= tol ||dL/dw|| or after max_cg iterations, or when p^T H_E p <= 0 (H_E is positive definite
 * at a strict minimiser; elsewhere the solve stops there).
 * ---------------------------------------------------------------------------------------- */
/* out = H_E(w) x */
void orc_hvp(const orc_params *p, const double *w, const double *x, double *out)
{
    const int nf = p->nf;
    const long N = (long)p->H * p->W;
    double *r = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *sv = (double *)malloc(sizeof(double) * (size_t)nf * N);
    if (!r || !sv) { free(r); free(sv); return; }
    orc_responses(nf, p->k, p->H, p->W, w, p->bc, r, p->nthreads);
    orc_responses(nf, p->k, p->H, p->W, x, p->bc, sv, p->nthreads);
    for (int f = 0; f < nf; ++f)
        for (long q = 0; q < N; ++q) sv[(size_t)f * N + q] *= p->alpha[f] * orc_rho2(r[(size_t)f * N + q]);
    orc_adjoint(nf, p->k, p->H, p->W, sv, p->bc, out, p->nthreads);
    for (long q = 0; q < N; ++q) out[q] += p->lambda * x[q];
    free(r);
    free(sv);
}

static double orc_dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Conjugate gradients for H_E(w) q = b from q = 0; returns the iterations taken, *relres = ||b - H q|| / ||b||
 * from the recurrence. */
int orc_cg(const orc_params *p, const double *w, const double *b, int max_cg, double tol, double *q, double *relres)
{
    const long N = (long)p->H * p->W;
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    double *Ad = (double *)malloc(sizeof(double) * (size_t)N);
    if (!r || !d || !Ad) { free(r); free(d); free(Ad); return -1; }
    for (long i = 0; i < N; ++i) {
        q[i] = 0.0;
        r[i] = b[i];
        d[i] = b[i];
    }
    const double rr0 = orc_dot(N, r, r);
    double rr = rr0;
    int it = 0;
    while (it < max_cg && rr > tol * tol * rr0) {
        orc_hvp(p, w, d, Ad);
        const double dAd = orc_dot(N, d, Ad);
        if (!(dAd > 0.0)) break;
        const double al = rr / dAd;
        for (long i = 0; i < N; ++i) {
            q[i] += al * d[i];
            r[i] -= al * Ad[i];
        }
        const double rr1 = orc_dot(N, r, r);
        const double be = rr1 / rr;
        for (long i = 0; i < N; ++i) d[i] = r[i] + be * d[i];
        rr = rr1;
        ++it;
    }
    if (relres) *relres = rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
    free(r);
    free(d);
    free(Ad);
    return it;
}

double orc_train_grad_implicit(const orc_params *p, int B, const double *clean, const double *noisy, int T,
                               int max_cg, double tol, double *dk, double *dlogalpha, int *cg_iters_max,
                               double *relres_max)
{
    const int nf = p->nf, H = p->H, W = p->W;
    const long N = (long)H * W, PW = W + 2 * ORC_R, PN = (long)(H + 2 * ORC_R) * PW;
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
    double *U = (double *)malloc(sizeof(double) * (size_t)N * (T + 1));
    double *b = (double *)malloc(sizeof(double) * (size_t)N);
    double *q = (double *)malloc(sizeof(double) * (size_t)N);
    double *r = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *sv = (double *)malloc(sizeof(double) * (size_t)nf * N);
    double *pw = (double *)malloc(sizeof(double) * (size_t)PN);
    double *pq = (double *)malloc(sizeof(double) * (size_t)PN);
    double L = NAN;
    int itmax = 0;
    double rmax = 0.0;
    if (!v || !U || !b || !q || !r || !sv || !pw || !pq) goto done;
    for (int i = 0; i < nf * ORC_KK; ++i) dk[i] = 0.0;
    for (int i = 0; i < nf; ++i) dlogalpha[i] = 0.0;
    L = 0.0;
    for (int s = 0; s < B; ++s) {
        orc_train_forward(p, noisy + (size_t)s * N, T, v, U);
        const double *w = U + (size_t)T * N;
        L += orc_loss_one(w, clean + (size_t)s * N, N, b);
        double rel = 0.0;
        const int it = orc_cg(p, w, b, max_cg, tol, q, &rel);
        if (it > itmax) itmax = it;
        if (rel > rmax) rmax = rel;
        orc_responses(nf, p->k, H, W, w, p->bc, r, p->nthreads);
        orc_responses(nf, p->k, H, W, q, p->bc, sv, p->nthreads);
        orc_pad_image(H, W, w, p->bc, pw);
        orc_pad_image(H, W, q, p->bc, pq);
        for (int f = 0; f < nf; ++f) {
            const double *rf = r + (size_t)f * N, *sf = sv + (size_t)f * N;
            double ga = 0.0;
            for (long k = 0; k < N; ++k) ga += sf[k] * orc_rho1(rf[k]);
            dlogalpha[f] += -p->alpha[f] * ga;
            for (int a = -ORC_R; a <= ORC_R; ++a)
                for (int bb = -ORC_R; bb <= ORC_R; ++bb) {
                    double gk = 0.0;
                    for (long y = 0; y < H; ++y)
                        for (long x = 0; x < W; ++x) {
                            const long k = y * W + x, pi = (y - a + ORC_R) * PW + (x - bb + ORC_R);
                            gk += pq[pi] * orc_rho1(rf[k]) + sf[k] * orc_rho2(rf[k]) * pw[pi];
                        }
                    dk[(size_t)f * ORC_KK + (a + ORC_R) * ORC_KS + (bb + ORC_R)] += -p->alpha[f] * gk;
                }
        }
    }
done:
    if (cg_iters_max) *cg_iters_max = itmax;
    if (relres_max) *relres_max = rmax;
    free(v); free(U); free(b); free(q); free(r); free(sv); free(pw); free(pq);
    return L;
}
