/*
 * FP64 CPU oracle for the PDE dehazing method (arXiv 2506.08793).
 *
 * TEST INFRASTRUCTURE ONLY: see oracle.h.  Every loop below follows the
 * definition it cites term by term; there is no blocking, fusion or
 * reordering.  Per-pixel loops may run on several OpenMP threads because each
 * output element is computed on its own; every reduction runs serially in
 * index order, so results do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Half-sample symmetric extension (... c b a | a b c ... | z y x | x y z ...),
 * the 'reflect' boundary of scipy.ndimage that App. A-B-2 names.  Period 2n. */
static long reflect(long i, long n) {
    long p = 2 * n;
    long m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

/* ---------------------------------------------------------------- Sec. II-D */

void or_dark_channel(const float *I, int H, int W, int patch, const double *A, double *out) {
    const int r = patch / 2;
    const long N = (long)H * W;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double best = INFINITY;
            for (int c = 0; c < 3; ++c) {
                const double a = A ? A[c] : 1.0;
                /* inner minimum over the patch Omega(x), clipped to the image */
                double m = INFINITY;
                for (int yy = y - r; yy <= y + r; ++yy) {
                    if (yy < 0 || yy >= H) continue;
                    for (int xx = x - r; xx <= x + r; ++xx) {
                        if (xx < 0 || xx >= W) continue;
                        const double v = (double)I[c * N + (long)yy * W + xx] / a;
                        if (v < m) m = v;
                    }
                }
                /* outer minimum over the colour channels */
                if (m < best) best = m;
            }
            out[(long)y * W + x] = best;
        }
    }
}

/* ------------------------------------------------- atmospheric light (DCP) */

static const double *g_sort_dc; /* qsort has no context argument */

static int cmp_desc_dc_then_index(const void *pa, const void *pb) {
    const long a = *(const long *)pa, b = *(const long *)pb;
    const double da = g_sort_dc[a], db = g_sort_dc[b];
    if (da > db) return -1;
    if (da < db) return 1;
    return (a > b) - (a < b);
}

int or_atmospheric_light(const float *I, const double *dc, int H, int W, int permille,
                         double A[3], long *index) {
    const long N = (long)H * W;
    long k = (N * (long)permille) / 1000;
    if (k < 1) k = 1;
    if (k > N) k = N;
    long *order = (long *)malloc(sizeof(long) * (size_t)N);
    for (long i = 0; i < N; ++i) order[i] = i;
    g_sort_dc = dc;
    qsort(order, (size_t)N, sizeof(long), cmp_desc_dc_then_index);
    /* among the k haziest pixels, the brightest; ties go to the lower index */
    long best = -1;
    double best_sum = -INFINITY;
    for (long q = 0; q < k; ++q) {
        const long i = order[q];
        const double s = ((double)I[i] + (double)I[N + i]) + (double)I[2 * N + i];
        if (best < 0 || s > best_sum || (s == best_sum && i < best)) {
            best = i;
            best_sum = s;
        }
    }
    free(order);
    int clamped = 0;
    for (int c = 0; c < 3; ++c) {
        A[c] = (double)I[c * N + best];
        if (!(A[c] > 0.0)) {
            A[c] = 1e-6;
            clamped = 1;
        }
    }
    if (index) *index = best;
    return clamped;
}

/* ------------------------------------------------- Sec. II-D and Sec. II-A */

/* mean of v over the (2r+1)x(2r+1) window at (x, y), clipped to the image */
static double box_mean(const double *v, int H, int W, int x, int y, int r) {
    const int x0 = x - r < 0 ? 0 : x - r, x1 = x + r >= W ? W - 1 : x + r;
    const int y0 = y - r < 0 ? 0 : y - r, y1 = y + r >= H ? H - 1 : y + r;
    double s = 0.0;
    for (int j = y0; j <= y1; ++j)
        for (int i = x0; i <= x1; ++i) s += v[(long)j * W + i];
    return s / (double)((x1 - x0 + 1) * (y1 - y0 + 1));
}

void or_guided_filter(const double *g, const double *p, int H, int W, int r, double eps, double *q) {
    const long N = (long)H * W;
    double *gp = (double *)malloc(sizeof(double) * (size_t)N), *gg = (double *)malloc(sizeof(double) * (size_t)N);
    double *a = (double *)malloc(sizeof(double) * (size_t)N), *b = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; ++i) {
        gp[i] = g[i] * p[i];
        gg[i] = g[i] * g[i];
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double mg = box_mean(g, H, W, x, y, r), mp = box_mean(p, H, W, x, y, r);
            const double cov = box_mean(gp, H, W, x, y, r) - mg * mp;
            const double var = box_mean(gg, H, W, x, y, r) - mg * mg;
            const long i = (long)y * W + x;
            a[i] = cov / (var + eps);
            b[i] = mp - a[i] * mg;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long i = (long)y * W + x;
            q[i] = box_mean(a, H, W, x, y, r) * g[i] + box_mean(b, H, W, x, y, r);
        }
    free(gp);
    free(gg);
    free(a);
    free(b);
}

void or_transmission(const float *I, const double A[3], const double *td, int H, int W,
                     const or_params *p, double *t, double *lam, double *Phi) {
    const long N = (long)H * W;
    for (long i = 0; i < N; ++i) t[i] = 1.0 - p->omega * td[i];
    if (p->gf_radius > 0) {
        double *g = (double *)malloc(sizeof(double) * (size_t)N), *t0 = (double *)malloc(sizeof(double) * (size_t)N);
        for (long i = 0; i < N; ++i) {
            g[i] = (((double)I[i] + (double)I[N + i]) + (double)I[2 * N + i]) / 3.0;
            t0[i] = t[i];
        }
        or_guided_filter(g, t0, H, W, p->gf_radius, p->gf_eps, t);
        free(g);
        free(t0);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        const double ti = t[i];
        lam[i] = p->lambda0 * exp(-p->beta * (1.0 - ti));
        if (p->variant & 1) lam[i] = p->lambda0; /* w/o adaptive regularisation */
        if (p->variant & 4) lam[i] = 0.0;        /* w/o nonlocal regularisation */
        const double den = ti > p->t0 ? ti : p->t0;
        for (int c = 0; c < 3; ++c)
            Phi[c * N + i] = ((double)I[c * N + i] - A[c] * (1.0 - ti)) / den;
    }
}

/* ------------------------------------------------------------- App. A-B-2 */

void or_gauss_weights(double sigma, int radius, double *w) {
    double s = 0.0;
    for (int k = -radius; k <= radius; ++k) {
        w[k + radius] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        s += w[k + radius];
    }
    for (int k = 0; k <= 2 * radius; ++k) w[k] /= s;
}

/* u at column i, row j outside the image: the reflecting boundary, or zero
 * for the Dirichlet (H^1_0) setting */
static double U(const double *u, int H, int W, long i, long j, int boundary) {
    if (boundary == 1 && (i < 0 || i >= W || j < 0 || j >= H)) return 0.0;
    return u[reflect(j, H) * W + reflect(i, W)];
}

void or_gauss(const double *u, int H, int W, double sigma, int radius, int boundary, double *out) {
    double w[64];
    or_gauss_weights(sigma, radius, w);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            /* G(u)(x) = sum_y K(x,y) u(y) with the separable normalised kernel */
            double g = 0.0;
            for (int b = -radius; b <= radius; ++b)
                for (int a = -radius; a <= radius; ++a)
                    g += w[b + radius] * w[a + radius] * U(u, H, W, x + a, y + b, boundary);
            out[(long)y * W + x] = g;
        }
    }
}

/* ------------------------------------------------------------- App. A-B-1 */

/* D on the x-face (i+1/2, j): forward difference in x, central difference in
 * y at cell (i, j), D = (|grad u| + eps)^-1, Delta x = Delta y = 1 (D == 1
 * for the "w/o edge-preserving term" ablation); *ux receives the difference
 * across the face. */
static double coef_x(const double *u, int H, int W, long i, long j, double eps, int bnd, int no_edge, double *ux) {
    *ux = U(u, H, W, i + 1, j, bnd) - U(u, H, W, i, j, bnd);
    const double uy = (U(u, H, W, i, j + 1, bnd) - U(u, H, W, i, j - 1, bnd)) / 2.0;
    return no_edge ? 1.0 : 1.0 / (sqrt(*ux * *ux + uy * uy) + eps);
}

/* The y-face (i, j+1/2): the same with the roles of x and y swapped. */
static double coef_y(const double *u, int H, int W, long i, long j, double eps, int bnd, int no_edge, double *uy) {
    *uy = U(u, H, W, i, j + 1, bnd) - U(u, H, W, i, j, bnd);
    const double ux = (U(u, H, W, i + 1, j, bnd) - U(u, H, W, i - 1, j, bnd)) / 2.0;
    return no_edge ? 1.0 : 1.0 / (sqrt(ux * ux + *uy * *uy) + eps);
}

/* D u_x on the x-face (i+1/2, j) and D u_y on the y-face (i, j+1/2). */
static double flux_x(const double *u, int H, int W, long i, long j, double eps, int bnd, int no_edge) {
    double ux;
    const double D = coef_x(u, H, W, i, j, eps, bnd, no_edge, &ux);
    return D * ux;
}
static double flux_y(const double *u, int H, int W, long i, long j, double eps, int bnd, int no_edge) {
    double uy;
    const double D = coef_y(u, H, W, i, j, eps, bnd, no_edge, &uy);
    return D * uy;
}

void or_faces(const double *u, int H, int W, double eps, int boundary, int no_edge, double *Dx, double *Dy) {
    double d;
    for (int j = 0; j < H; ++j)
        for (int i = -1; i < W; ++i) Dx[(long)j * (W + 1) + i + 1] = coef_x(u, H, W, i, j, eps, boundary, no_edge, &d);
    for (int j = -1; j < H; ++j)
        for (int i = 0; i < W; ++i) Dy[(long)(j + 1) * W + i] = coef_y(u, H, W, i, j, eps, boundary, no_edge, &d);
}

void or_div(const double *u, int H, int W, double eps, int boundary, int no_edge, double *out) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            const double dx = flux_x(u, H, W, i, j, eps, boundary, no_edge) -
                              flux_x(u, H, W, i - 1, j, eps, boundary, no_edge);
            const double dy = flux_y(u, H, W, i, j, eps, boundary, no_edge) -
                              flux_y(u, H, W, i, j - 1, eps, boundary, no_edge);
            out[(long)j * W + i] = dx + dy;
        }
    }
}

void or_F(const double *u, const double *Phi, const double *lam, int H, int W,
          const or_params *p, double *F) {
    const long N = (long)H * W;
    double *dv = (double *)malloc(sizeof(double) * (size_t)N);
    double *g = (double *)malloc(sizeof(double) * (size_t)N);
    for (int c = 0; c < 3; ++c) {
        or_div(u + c * N, H, W, p->eps, p->boundary, (p->variant & 2) != 0, dv);
        or_gauss(u + c * N, H, W, p->sigma, p->radius, p->boundary, g);
        for (long i = 0; i < N; ++i)
            F[c * N + i] = dv[i] - lam[i] * g[i] + Phi[c * N + i];
    }
    free(dv);
    free(g);
}

/* --------------------------------------------------------------- App. A-A */

int or_solve(double *u, const double *Phi, const double *lam, int H, int W,
             const or_params *p, int max_iter, double tol, double *rho) {
    const long N = (long)H * W;
    double *F = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double phin[3];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (long i = 0; i < N; ++i) s += Phi[c * N + i] * Phi[c * N + i];
        phin[c] = sqrt(s);
    }
    int n = 0;
    for (;; ++n) {
        or_F(u, Phi, lam, H, W, p, F);
        double worst = 0.0;
        int finite = 1;
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (long i = 0; i < N; ++i) s += F[c * N + i] * F[c * N + i];
            const double r = phin[c] > 0.0 ? sqrt(s) / phin[c] : sqrt(s);
            rho[3 * n + c] = r;
            if (!isfinite(r)) finite = 0; /* a non-finite residual never converges */
            else if (r > worst) worst = r;
        }
        if ((finite && worst <= tol) || n == max_iter) break;
        for (long i = 0; i < 3 * N; ++i) u[i] = u[i] + p->tau * F[i];
    }
    free(F);
    return n;
}
