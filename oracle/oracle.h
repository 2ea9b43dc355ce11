/*
 * FP64 CPU oracle for the PDE dehazing method of Hu, Wang, Gao, Wang and
 * Zheng, "A PDE-Based Image Dehazing Method via Atmospheric Scattering
 * Theory" (arXiv 2506.08793).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * restatement of what the method computes, used to judge the CUDA library.
 * Only the test-suite, the package's smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Layout: images are planar, row-major; channel c, row y, column x lives at
 * [(c*H + y)*W + x].  Pixel (i, j) in the paper's notation is column i, row j.
 * All arithmetic is IEEE binary64 (built with -ffp-contract=off, so no fused
 * multiply-add changes rounding between hosts).
 *
 * Parity status per function (pins live in tests/test_oracle_pins.py):
 *   or_dark_channel        pinned (scipy minimum_filter, brute force, prior scenes)
 *   or_atmospheric_light   pinned (numpy lexsort selection, prior scenes)
 *   or_transmission        pinned (closed form on constant images, prior scenes)
 *   or_gauss_weights / or_F pinned (scipy gaussian_filter, scipy laplace linear
 *                          limit, 1-D step closed form, conservation)
 *   or_solve               pinned (constant-image trajectory closed form,
 *                          Newton root, uniqueness, resume)
 *   boundary = 1 / variant  pinned (scipy zero-padded gaussian_filter and laplace;
 *                          D == 1 is the 5-point Laplacian; lambda ablations)
 *   or_faces               pinned (the frozen operator applied to u equals -or_div(u))
 *   or_guided_filter       pinned (scipy uniform_filter composition, constant input, eps -> infinity,
 *                          linear guide)
 */
#ifndef DEHAZE_ORACLE_H
#define DEHAZE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int    patch;          /* dark-channel window side, Sec. II-D: 15 */
    int    topk_permille;  /* atmospheric light: top max(1, N*p/1000) pixels (He et al. DCP rule) */
    double omega;          /* Sec. II-D: 0.95 */
    double t0;             /* floor of t in Phi, Sec. II-A (value not given: 0.1) */
    double lambda0;        /* Sec. II-D: 0.5 */
    double beta;           /* Sec. II-D: 3.0 */
    double eps;            /* D = (|grad u| + eps)^-1, Sec. II-B: 1e-3 */
    double sigma;          /* Gaussian width, Sec. II-C: 2.0 */
    int    radius;         /* Gaussian half-width; 5x5 kernel => 2 (App. A-B-2) */
    double tau;            /* relaxation parameter, App. A-A: 0.2 */
    int    boundary;       /* 0: half-sample reflection (zero flux); 1: u = 0 outside (H^1_0, Sec. III) */
    int    variant;        /* ablations of Sec. IV-E: 1 lambda == lambda0, 2 D == 1, 4 lambda == 0 */
    int    dc_scales;      /* 1: one patch; 3: mean of the normalised dark channels at patch/2|1, patch,
                              2*patch+1 (the "multiscale dark channel" of Sec. IV-E; used by the Python
                              composition, not by the C functions) */
    int    gf_radius;      /* > 0: guided-filter refinement of t (Sec. IV-E "guided filter") */
    double gf_eps;         /* its regularisation */
} or_params;

/* Sec. II-D dark channel: out(x) = min_c min_{y in Omega(x)} I^c(y)/A^c over a
 * patch x patch window clipped at the image border.  A == NULL means A = 1
 * (the un-normalised dark channel used to locate the atmospheric light). */
void or_dark_channel(const float *I, int H, int W, int patch, const double *A, double *out);

/* Atmospheric light (the paper cites the DCP rule of He et al. without
 * restating it): the k = max(1, N*permille/1000) pixels with the largest dark
 * channel (ties to the lower row-major index), then among them the pixel with
 * the largest ((double)I^R + (double)I^G) + (double)I^B (ties to the lower
 * index).  A = I at that pixel.  Returns 1 when some A^c <= 0 was clamped to
 * 1e-6, else 0; *index receives the chosen pixel. */
int or_atmospheric_light(const float *I, const double *dc, int H, int W, int permille,
                         double A[3], long *index);

/* Sec. II-D and II-A: t = 1 - omega*td, lambda = lambda0*exp(-beta*(1-t)),
 * Phi^c = (I^c - A^c (1-t)) / max(t, t0).  t, lam: HxW; Phi: 3xHxW.
 * With p->gf_radius > 0, t is first refined by or_guided_filter with the
 * gray guide g = ((I^R + I^G) + I^B) / 3 (t, lambda and Phi then use it). */
void or_transmission(const float *I, const double A[3], const double *td, int H, int W,
                     const or_params *p, double *t, double *lam, double *Phi);

/* The guided filter of He, Sun and Tang (the paper names it in Sec. IV-E
 * without defining it): with mean_r(v)(x) the average of v over the
 * (2r+1)x(2r+1) window around x clipped to the image,
 *   a = (mean(g p) - mean(g) mean(p)) / (mean(g g) - mean(g)^2 + eps),
 *   b = mean(p) - a mean(g),   q = mean(a) g + mean(b).
 * g, p, q: HxW. */
void or_guided_filter(const double *g, const double *p, int H, int W, int r, double eps, double *q);

/* App. A-B-2: the 2*radius+1 normalised 1-D Gaussian weights. */
void or_gauss_weights(double sigma, int radius, double *w);

/* App. A-A / A-B: F(u) = div(D(grad u) grad u) - lambda*G(u) + Phi for the
 * three channels.  u, Phi, F: 3xHxW; lam: HxW. */
void or_F(const double *u, const double *Phi, const double *lam, int H, int W,
          const or_params *p, double *F);

/* The diffusion term alone, div(D grad u), one channel (HxW); boundary as in
 * or_params; no_edge: D == 1. */
void or_div(const double *u, int H, int W, double eps, int boundary, int no_edge, double *out);

/* The face coefficients of the diffusion term frozen at u (one channel), for
 * the semi-implicit scheme: D = (|grad u| + eps)^-1 (1 for no_edge) with the
 * same differences as or_div.  x-faces (i+1/2, j), i = -1..W-1, at
 * Dx[j*(W+1) + i+1]; y-faces (i, j+1/2), j = -1..H-1, at Dy[(j+1)*W + i].
 * Border faces are included; what they couple to is the boundary rule's. */
void or_faces(const double *u, int H, int W, double eps, int boundary, int no_edge, double *Dx, double *Dy);

/* The Gaussian term alone, G(u), one channel (HxW). */
void or_gauss(const double *u, int H, int W, double sigma, int radius, int boundary, double *out);

/* App. A-A fixed-point iteration u <- u + tau*F(u) from u (in/out).
 * For n = 0, 1, ...: rho_n^c = ||F^c(u^n)|| / ||Phi^c|| (||F^c|| when
 * ||Phi^c|| = 0) is stored in rho[3n + c] (rho must hold 3*(max_iter+1));
 * the loop stops at the first n with max_c rho_n^c <= tol or n == max_iter,
 * leaving u = u^n.  Returns n (the number of updates applied). */
int or_solve(double *u, const double *Phi, const double *lam, int H, int W,
             const or_params *p, int max_iter, double tol, double *rho);

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
