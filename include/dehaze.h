/*
 * dehaze.h -- C ABI of the GB300 (sm_103a) CUDA library for the PDE-based
 * dehazing method of Hu, Wang, Gao, Wang and Zheng, "A PDE-Based Image
 * Dehazing Method via Atmospheric Scattering Theory" (arXiv 2506.08793).
 *
 * The method (Sec. II and App. A):
 *   dark channel      t_d(x) = min_c min_{y in Omega(x)} I^c(y)/A^c      (Sec. II-D)
 *   transmission      t = 1 - omega*t_d, lambda(t) = lambda0*exp(-beta(1-t)) (Sec. II-D)
 *   data term         Phi^c = (I^c - A^c (1-t)) / max(t, t0)             (Sec. II-A)
 *   PDE, per channel  -div(D(grad u) grad u) + lambda(t) G(u) = Phi      (Sec. II-A, eq. main_pde)
 *                     D = (|grad u| + eps)^-1 (Sec. II-B), G = 5x5 Gaussian, sigma 2 (Sec. II-C)
 *   solver            u <- u + tau [div(D_n grad u) - lambda G(u) + Phi] (App. A-A)
 *                     flux-form stencil of App. A-B-1, separable Gaussian of App. A-B-2
 * The atmospheric light A is not defined by the paper; the library uses the
 * dark-channel-prior rule of He et al. that the paper cites: the brightest
 * (largest R+G+B) of the 0.1 % pixels with the largest dark channel.
 *
 * Conventions for every call below
 *   - Images are planar float32, row-major: channel c, row y, column x at
 *     [(c*H + y)*W + x].  Maps (t, lambda, dark channel) are HxW.
 *   - Every array argument is a DEVICE pointer owned by the caller, unless
 *     marked "host".  The library allocates no device memory: scratch space
 *     is the caller's workspace (size from dh_workspace_bytes, 256-byte
 *     aligned).  Pointers passed in one call must not overlap unless stated.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     queued asynchronously; a call with a non-NULL host `report` waits for
 *     the stream and fills the report.
 *   - Return value: DH_OK (0), a positive warning (outputs valid) or a
 *     negative error (outputs unspecified).  Errors found on the host
 *     (shapes, parameters, workspace) are returned before any work is queued.
 *   - 1 <= H, W <= 32768 and H*W <= 2^28.  There is no CPU fallback: on a
 *     machine without a usable GB300 every compute call returns DH_ECUDA.
 */
#ifndef DEHAZE_H
#define DEHAZE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DH_VERSION 1

/* status codes */
#define DH_OK 0
#define DH_WDEGENERATE 1  /* warning: some A^c <= 0 was clamped to 1e-6 */
#define DH_WNOCONV 2      /* warning: max_iter reached with residual above tol */
#define DH_EINVAL (-1)    /* bad shape, pointer, alignment or parameter */
#define DH_ENONFINITE (-2)/* a non-finite residual appeared; iteration stopped */
#define DH_EWORKSPACE (-3)/* workspace missing, too small or misaligned */
#define DH_ECUDA (-4)     /* a CUDA runtime call failed (no GPU, launch error ...) */
#define DH_ETIMEOUT (-5)  /* a bounded device-side wait ran out */

/* presets for dh_params_default */
#define DH_PRESET_PAPER 0  /* the paper's constants (Sec. IV-B), eps = 1e-3 */
#define DH_PRESET_STABLE 1 /* the same with eps = 1.0, which satisfies App. A-A's step bound */

/* iterate storage (u and its halos); Phi, lambda and all arithmetic stay
 * float32.  The 16-bit forms stall at a residual set by their quantum (u is
 * O(10) at the fixed point); the switched forms run 16-bit storage until the
 * residual stops falling (less than 2 % over 16 iterations), then convert the
 * iterate and finish in float32. */
#define DH_STORE_F32 0
#define DH_STORE_BF16 1
#define DH_STORE_F16 2
#define DH_STORE_BF16_F32 3
#define DH_STORE_F16_F32 4

/* boundary of the PDE (dh_params.boundary) */
#define DH_BOUNDARY_REFLECT 0 /* half-sample symmetric extension: zero flux (default) */
#define DH_BOUNDARY_ZERO 1    /* u = 0 outside the image: the H^1_0 setting of Sec. III */

/* ablation switches (Sec. IV-E, Table II), OR-ed into dh_params.variant */
#define DH_VAR_NO_ADAPTIVE 1 /* lambda(t) == lambda0 */
#define DH_VAR_NO_EDGE 2     /* D == 1 (linear diffusion) */
#define DH_VAR_NO_NONLOCAL 4 /* lambda == 0 */

typedef struct dh_params {
    int patch;          /* dark-channel window side, odd, 1..31 (Sec. II-D: 15) */
    int topk_permille;  /* A from the top max(1, H*W*p/1000) dark-channel pixels (1) */
    float omega;        /* Sec. II-D: 0.95 */
    float t0;           /* floor of t in Phi (Sec. II-A; no value given: 0.1) */
    float lambda0;      /* Sec. II-D: 0.5 */
    float beta;         /* Sec. II-D: 3.0 */
    float eps;          /* Sec. II-B: 1e-3 (paper) / 1.0 (stable) */
    float sigma;        /* Sec. II-C: 2.0 */
    int radius;         /* Gaussian half-width; only 2 (5x5, App. A-B-2) is built */
    float tau;          /* App. A-A: 0.2 */
    float tol;          /* stop when max_c ||F^c(u^n)|| / ||Phi^c|| <= tol (1e-4) */
    int max_iter;       /* at most this many updates (default 5000) */
    int tb_depth;       /* fixed-point iterations per tile load: 0 = library choice (tuned or
                           default), 1 = one, 2..4 = the temporally blocked sweeps (W % 4 == 0,
                           float32 storage; otherwise one) */
    int storage;        /* DH_STORE_* */
    int variant;        /* DH_VAR_* bits, 0 = the full method */
    int use_graph;      /* 1: iteration loop in a CUDA graph with a device-side
                           while condition (default); 0: host-queued launches */
    int sweep_variant;  /* sweep kernel variant (1..dh_sweep_variants()-1); 0 = the
                           tuned choice for this shape if dh_tune ran, else default */
    int boundary;       /* DH_BOUNDARY_* for the flux stencil and the Gaussian */
    /* Front-end refinements the Sec. IV-E ablation names ("multiscale dark
     * channel", "guided filter") without defining them; both off by default.
     * They need workspace (dh_workspace_bytes accounts for them). */
    int dc_scales;      /* 1: one patch; 3: t_d = mean of the normalised dark channels at
                           patch sizes patch/2 (odd), patch and 2*patch+1 (patch <= 15) */
    int gf_radius;      /* 0: off; 1..24: t refined by the guided filter (He et al.) with
                           the gray guide (I^R + I^G + I^B)/3 over (2r+1)^2 windows */
    float gf_eps;       /* its regularisation (default 1e-3) */
} dh_params;

typedef struct dh_report {
    int status;         /* as returned */
    int n_iter;         /* updates applied: the returned u is u^n_iter */
    float rho[3];       /* ||F^c(u^n_iter)|| / ||Phi^c|| (||F^c|| if ||Phi^c|| = 0) */
    float A[3];         /* atmospheric light (dh_dehaze only) */
    long long a_index;  /* row-major index of the pixel A was taken from, or -1 */
    float ms;           /* device time of the call (CUDA events on `stream`) */
    float ms_loop;      /* device time of the fixed-point loop alone */
    int launches;       /* kernels the call ran; sweep launches are counted on the device
                           (a multi-iteration launch runs up to 64 iterations) */
} dh_report;

/* Fill *p with a preset.  Returns DH_OK or DH_EINVAL (NULL p, unknown preset). */
int dh_params_default(dh_params *p, int preset);

/* Static description of a status code (never NULL). */
const char *dh_strerror(int status);

/* DH_VERSION of the built library. */
int dh_version(void);

/* Bytes of device workspace dh_dehaze / dh_fixed_point / dh_atmospheric_light
 * need for an HxW image under *p (p may be NULL for the defaults); 0 when the
 * shape or parameters are invalid.  About 44 bytes per pixel: the dark
 * channel, lambda, Phi and two iterate buffers besides the caller's u (the
 * multi-iteration sweep rotates u^n over three buffers so that it can start
 * the next iteration before the stop rule on u^n is decided), plus the
 * refinements' scratch when they are on. */
size_t dh_workspace_bytes(int H, int W, const dh_params *p);

/* Sec. II-D dark channel:
 *   out(x) = min_c min_{|dy|,|dx| <= patch/2} I^c(x+(dx,dy)) / A^c,
 * the window clipped at the image border.  A = NULL means A = (1,1,1) (the
 * un-normalised dark channel that locates the atmospheric light); otherwise
 * A is a device float[3] and each quotient is the IEEE float32 quotient.
 * I: 3xHxW; out: HxW.  Bit-exact (no rounding beyond the quotient). */
int dh_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out,
                    void *stream);

/* Atmospheric light by the DCP rule (not defined by the paper; He et al.):
 * k = max(1, H*W*topk_permille/1000) pixels with the largest dc (ties: lower
 * row-major index), then the one with the largest
 * ((double)I^R + (double)I^G) + (double)I^B (ties: lower index).
 * I: 3xHxW; dc: HxW (from dh_dark_channel with A = NULL); A_out: device
 * float[3] receives I at that pixel, each A^c <= 0 replaced by 1e-6;
 * index_out: device long long[1] (may be NULL).  Needs workspace.  Returns
 * DH_WDEGENERATE (with report) when a component was clamped. */
int dh_atmospheric_light(const float *I, const float *dc, int H, int W, int topk_permille,
                         float *A_out, long long *index_out, void *workspace,
                         size_t workspace_bytes, void *stream, dh_report *report);

/* Sec. II-D and II-A: from I and A (device float[3]) computes
 *   t_d = dark channel of I/A (as dh_dark_channel), t = 1 - omega*t_d,
 *   lambda = lambda0*exp(-beta(1-t)), Phi^c = (I^c - A^c(1-t))/max(t, t0).
 * t, lam: HxW; Phi: 3xHxW; td may be NULL. */
int dh_transmission(const float *I, const float *A, int H, int W, const dh_params *p,
                    float *td, float *t, float *lam, float *Phi, void *stream);

/* dh_transmission with the front-end refinements of p (dc_scales = 3: t_d is
 * the mean of the three normalised dark channels; gf_radius > 0: t is refined
 * by the guided filter before lambda and Phi; window sums in FP64), which
 * need scratch: workspace of dh_workspace_bytes(H, W, p) bytes, 256-byte
 * aligned (dh_transmission itself returns DH_EINVAL for those parameters). */
int dh_transmission_ws(const float *I, const float *A, int H, int W, const dh_params *p, float *td, float *t,
                       float *lam, float *Phi, void *workspace, size_t workspace_bytes, void *stream);

/* App. A-A fixed-point iteration, per channel, from u (in: u^0, out: u^n):
 *   F(u) = div(D(grad u) grad u) - lambda G(u) + Phi   (App. A-B-1, A-B-2)
 *   for n = 0, 1, ...: rho_n^c = ||F^c(u^n)|| / ||Phi^c||;
 *   stop at the first n with max_c rho_n^c <= p->tol or n == p->max_iter,
 *   else u^{n+1} = u^n + tau F(u^n).
 * Boundary: half-sample symmetric reflection for both the flux stencil (zero
 * flux across the border) and the Gaussian.
 * u, Phi: 3xHxW; lam: HxW; rho_hist: device float[3*(max_iter+1)] or NULL,
 * receives rho_n for n = 0 .. the returned n.  Returns DH_WNOCONV when max_iter
 * was reached (only known with a report), DH_ENONFINITE on a non-finite
 * residual.  (The float32 multi-iteration sweep decides the stop rule one
 * update late, computing u^{n+2} into a scratch buffer it then discards; the
 * returned u, n and rho are those of the rule above.) */
int dh_fixed_point(float *u, const float *Phi, const float *lam, int H, int W,
                   const dh_params *p, float *rho_hist, void *workspace, size_t workspace_bytes,
                   void *stream, dh_report *report);

/* The whole method on one image: dark channel -> A -> t, lambda, Phi ->
 * fixed point from u0 (NULL: u0 = Phi) -> J = clamp(u, 0, 1).
 * I: 3xHxW; u0: 3xHxW or NULL; outputs J, u: 3xHxW; t: HxW; A: float[3]. */
int dh_dehaze(const float *I, int H, int W, const dh_params *p, const float *u0, float *J,
              float *u, float *t, float *A, void *workspace, size_t workspace_bytes,
              void *stream, dh_report *report);

/* Timings of one dh_tune run. */
typedef struct dh_tune_result {
    int best;               /* fastest usable variant */
    int count;              /* entries below */
    int variant[64];        /* variant ids timed */
    float us_per_iter[64];  /* device time per iteration (graph loop, faster of two rounds) */
} dh_tune_result;

/* Number of sweep variants (valid ids are 1 .. count-1). */
int dh_sweep_variants(void);

/* Autotuner (not in the paper): times every sweep variant usable for an HxW
 * image under *p (float32 storage) on the caller's Phi, lambda (as for
 * dh_fixed_point) for `iters` fixed-point iterations each, in the graph loop,
 * with CUDA events on `stream`, in two rounds over all variants (each keeps its
 * faster time); u_scratch (3xHxW) is overwritten.  The fastest is recorded for (current device, H, W) and used by later calls with
 * sweep_variant = 0.  Waits for the stream.  out may be NULL. */
int dh_tune(const float *Phi, const float *lam, float *u_scratch, int H, int W, const dh_params *p,
            int iters, void *workspace, size_t workspace_bytes, void *stream, dh_tune_result *out);

/* Records / reads the tuned variant for (current device, H, W, storage), e.g.
 * from a saved tuning table.  dh_tune_get returns 0 when none is recorded. */
int dh_tune_set(int H, int W, int storage, int variant);
int dh_tune_get(int H, int W, int storage);

/* One image of a batch: inputs I (3xHxW) and optional u0, outputs J, u
 * (3xHxW), t (HxW) and A (float[3]); all device pointers, caller-owned. */
typedef struct dh_image {
    const float *I;
    int H, W;
    const float *u0;
    float *J, *u, *t, *A;
} dh_image;

/* Workspace bytes dh_dehaze_batch needs for these images (0 if invalid). */
size_t dh_batch_workspace_bytes(int n, const dh_image *imgs, const dh_params *p);

/* The whole method on n <= 256 images of any sizes.  The front end (Sec.
 * II-D, II-A) runs per image; the fixed-point loops (App. A-A) of all images
 * run in one CUDA graph while loop whose body is ONE persistent sweep launch
 * over the (128x24 tile, channel) items of every image still iterating; each
 * image stops on its own residual or max_iter, exactly as in dh_dehaze, and
 * leaves the batch's work list.  p->storage may be any DH_STORE_*: with the
 * switched forms every image runs 16-bit until its own residual stalls, then
 * all such images continue in float32 from their n in a second loop.  reports: host array of n or
 * NULL; with reports the call waits and reports[i].ms is the batch's time.
 * Returns the first error, else the first warning, else DH_OK. */
int dh_dehaze_batch(int n, const dh_image *imgs, const dh_params *p, void *workspace,
                    size_t workspace_bytes, void *stream, dh_report *reports);

/* ---- Learned warm start (not in the paper, which only points at hybrids of
 * the PDE with learned models, Sec. I and V): a 4-level U-Net over (I, t, A)
 * and Phi predicts y = lambda * u* as Phi + a learned correction (y = Phi, i.e.
 * u0 = Phi / lambda, is the fixed point without diffusion and with G = 1), and
 * u0 = y / lambda starts the fixed-point loop.
 * Architecture: 14 3x3 convolutions (zero padding, bias, ReLU) with `base`
 * (16 or 32) channels at full resolution doubling per level, 2x2 average
 * pooling, nearest 2x upsampling, skip concatenation (upsampled channels
 * first), a 1x1 head to 3 channels added to Phi.  Parameters are one float32 vector:
 * per convolution k weights [cout][3][3][cin] then bias [cout]; then the head
 * weights [3][base] and bias [3].  The input has 16 channels (I^R, I^G, I^B, t,
 * A^R, A^G, A^B, Phi^R, Phi^G, Phi^B, zeros).  Activations are bf16 NHWC in the workspace;
 * convolutions run on the tensor cores (bf16 in, fp32 accumulate).  Images
 * are N x H x W with H, W multiples of 8 and N*H*W <= 2^26.  I, Phi: N x 3 x H x W,
 * t: N x H x W, A: N x 3, y / target: N x 3 x H x W, all float32 device. */
size_t dh_unet_param_count(int base);
size_t dh_unet_workspace_bytes(int base, int N, int H, int W, int train);
/* He-normal weights from a counter-based generator, zero biases. */
int dh_unet_init(float *params, int base, unsigned long long seed, void *stream);
int dh_unet_forward(const float *params, int base, const float *I, const float *t, const float *A,
                    const float *Phi, int N, int H, int W, float *y, void *workspace, size_t workspace_bytes,
                    void *stream);
/* Forward, MSE loss mean((y - target)^2) into loss (device float[1]), and the
 * gradient of every parameter into grads (same layout as params). */
int dh_unet_backward(const float *params, int base, const float *I, const float *t, const float *A,
                     const float *Phi, const float *target, int N, int H, int W, float *grads, float *loss,
                     void *workspace, size_t workspace_bytes, void *stream);
/* One Adam step (bias-corrected; step counts from 1) over n parameters. */
int dh_unet_adam(float *params, const float *grads, float *m, float *v, size_t n, float lr, float beta1,
                 float beta2, float eps, int step, void *stream);
/* u0^c = y^c / lambda (3xHxW planar, lambda HxW), and the training target
 * y^c = lambda * u^c of a solved u. */
int dh_warm_start(const float *y, const float *lam, int H, int W, float *u0, void *stream);
int dh_warm_target(const float *u, const float *lam, int H, int W, float *y, void *stream);
/* One 3x3 convolution layer on bf16 NHWC data with channel pitch ldx / ldy
 * (C % 16 == 0, Cout % 8 == 0): y = [ReLU](conv(x, w) + bias), w bf16
 * [Cout][3][3][C]; and its weight / bias gradients (fp32) from dy, with
 * `scratch` (fp32) for per-split partial sums. */
int dh_conv3x3_forward(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *bias,
                       int Cout, int relu, void *y, int ldy, void *stream);
int dh_conv3x3_backward_weights(const void *x, int ldx, int C, const void *dy, int lddy, int Cout, int N, int H,
                                int W, float *dw, float *db, float *scratch, size_t scratch_bytes, void *stream);
/* The whole method with the network's warm start: dark channel, A, t, lambda,
 * Phi, then y = net(I, t, A), u0 = y / lambda, then the fixed-point loop from
 * u0 and J = clamp(u).  net_workspace: dh_unet_workspace_bytes(base, 1, H, W, 0). */
int dh_dehaze_warm(const float *params, int base, const float *I, int H, int W, const dh_params *p, float *J,
                   float *u, float *t, float *A, void *workspace, size_t workspace_bytes, void *net_workspace,
                   size_t net_workspace_bytes, void *stream, dh_report *report);

/* The batched solve of dh_dehaze_batch with the network's warm start for
 * every image: per image the front end, then y = net(I, t, A, Phi) and
 * u0 = y / lambda (as in dh_dehaze_warm), then the fixed-point loops of all
 * images in one graph while loop, each to its own residual; p->storage may be
 * any DH_STORE_* (the 16-bit phase of a switched form starts from the
 * network's u0 rounded to 16 bits).  imgs[i].u0 must be NULL; every image's
 * H and W are multiples of 8.  Images of one shape go through the network
 * together, in groups of up to about 4.2 million pixels (at most 64 images);
 * each image's u0 equals that of its own single-image forward.
 * workspace: dh_batch_workspace_bytes(n, imgs, p); net_workspace:
 * dh_batch_net_workspace_bytes(base, n, imgs) (the largest group's gathered
 * inputs and network workspace, reused group after group), both 256-byte
 * aligned.  The paper only points at hybrids of the PDE with learned models
 * (Sec. I and V). */
size_t dh_batch_net_workspace_bytes(int base, int n, const dh_image *imgs);
int dh_dehaze_batch_warm(const float *params, int base, int n, const dh_image *imgs, const dh_params *p,
                         void *workspace, size_t workspace_bytes, void *net_workspace, size_t net_workspace_bytes,
                         void *stream, dh_report *reports);

/* dh_atmospheric_light without a workspace and without any allocation.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc, such as a plug-in whose host application owns all device memory,
 * or a real-time frame loop that may not allocate.  Same inputs, outputs and
 * result as dh_atmospheric_light (no report).  Its scratch is one fixed
 * 32 KiB array in device memory that every GPU which loads the library keeps
 * until the process exits; it does not grow with the image, so the size limit
 * is the library's own (1 <= H, W <= 32768, H*W <= 2^28; DH_EINVAL beyond).
 * Every call looks up the array's device address for the current device
 * (cheap, no allocation); the first call on a device also loads the library's
 * device code there, so it should come before any stream capture on that
 * device.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. */
int dh_atmospheric_light_noalloc(const float *I, const float *dc, int H, int W, int topk_permille,
                                 float *A_out, long long *index_out, void *stream);

/* ---------------------------------------------------------------- semi-implicit scheme
 * The explicit iteration of App. A-A is stable only for tau < 2/(||D Delta|| +
 * lambda M), and ||D Delta|| grows like 8/eps (App. A-A): at the paper's
 * eps = 1e-3 no usable tau exists.  dh_semi_implicit solves the same equation
 * (Sec. II: -div(D grad u) + lambda G(u) = Phi) by the lagged-diffusivity
 * scheme: each outer step freezes the face coefficients D of App. A-B-1 at
 * u^n and solves (I/step + L_n) u^{n+1} = u^n/step - lambda G(u^n) + Phi,
 * L_n v = -div(D(u^n) grad v), with cg_iters Jacobi-preconditioned
 * conjugate-gradient iterations per channel started from u^n.  The paper has
 * no such scheme; its fixed point is the explicit scheme's.
 *
 * Workspace: dh_semi_implicit_workspace_bytes(H, W) bytes, 256-byte aligned
 * (about 108 B per pixel), owned by the caller; the call allocates nothing. */
size_t dh_semi_implicit_workspace_bytes(int H, int W);

/* u: 3xHxW float32 device, holds u^0 on entry and u^n on return (in place).
 * The iterate is kept as a double-float pair u + u_lo: at eps = 1e-3 the face
 * coefficients reach 1/eps, and a float32 iterate alone would leave F(u) a
 * rounding floor of about ulp(u)/eps (rho ~ 3e-4 on typical scenes).  u_lo
 * (3xHxW, may be NULL) is the trailing part, in and out (NULL: zero on entry,
 * kept in the workspace); u alone is u^n rounded to float32.
 * Phi: 3xHxW, lam: HxW (from dh_transmission).  p: eps, sigma, tol, max_iter,
 * boundary and variant (DH_VAR_NO_EDGE) are used; storage must be
 * DH_STORE_F32.  step: the outer step s > 0 (stable for s * lambda < 2; 2.0
 * is a good default).  The residual, stop rule, n and rho_hist are those of
 * dh_fixed_point: rho_n = ||F(u^n)|| / ||Phi||, F the residual of App. A-A.
 * J (3xHxW, may be NULL) receives clamp(u^n, 0, 1).  One cooperative launch runs the whole solve on `stream`; report (may be
 * NULL; when given the call synchronises the stream) as for dh_fixed_point.
 * Returns DH_OK / DH_WNOCONV / DH_ENONFINITE / DH_ETIMEOUT, or DH_EINVAL,
 * DH_EWORKSPACE, DH_ECUDA before any work is queued. */
int dh_semi_implicit(float *u, float *u_lo, const float *Phi, const float *lam, int H, int W, const dh_params *p,
                     float step, int cg_iters, float *rho_hist, float *J, void *workspace, size_t workspace_bytes,
                     void *stream, dh_report *report);

/* Diagnostic, no counterpart in the paper: runs one wait on a device barrier
 * that nothing completes, bounded by limit_cycles SM clocks (1 .. 4e9), the
 * way every wait of the library is bounded.  Returns DH_ETIMEOUT when the
 * bound is honoured (the expected result), DH_EINVAL for a bad limit,
 * DH_ECUDA on a CUDA error.  Synchronises the stream. */
int dh_selftest_bounded_wait(long long limit_cycles, void *stream);

#ifdef __cplusplus
}
#endif
#endif
