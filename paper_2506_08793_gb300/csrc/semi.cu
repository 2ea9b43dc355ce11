// Semi-implicit (lagged-diffusivity) fixed-point scheme for
// -div(D(grad u) grad u) + lambda G(u) = Phi (Sec. II, App. A).
//
// The explicit iteration of App. A-A needs tau < 2/(||D Delta|| + lambda M)
// with ||D Delta|| up to 8/eps, so the paper's eps = 1e-3 leaves no usable
// tau.  Here each outer step freezes the face coefficients D at u^n and takes
// the diffusion implicitly, the nonlocal term explicitly:
//
//     (I/s + L_n) u^{n+1} = u^n/s - lambda G(u^n) + Phi,
//     (L_n v)_i = sum over the faces f of pixel i of D_f(u^n) (v_i - v_nb(f)),
//
// v_nb extended by the boundary rule (reflecting: border faces drop out;
// Dirichlet: the ghost is 0).  I/s + L_n is symmetric positive definite; it is
// solved per channel by cg_iters Jacobi-preconditioned conjugate-gradient
// iterations started from u^n, whose initial residual is exactly F(u^n) of
// App. A-A, so rho_n = ||F(u^n)|| / ||Phi|| and the stop rule are the
// explicit solver's.  A fixed point of the outer iteration solves the PDE
// whatever the inner accuracy.
//
// One cooperative launch runs the whole solve: grid-stride passes over the
// 3 x H x W elements separated by grid barriers (the last CTA to arrive
// reduces the per-CTA partial sums in a fixed order and updates the scalars).
// Arrays the launch writes are read with plain L1-cached loads only in the
// phases after the grid barrier that follows their writing (the barrier's
// acquire makes the writes visible); the scalars and partial sums go through
// L2 (ld.global.cg).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace dh {

namespace {

constexpr int kSiThreads = 256;
constexpr int kSiMaxGrid = 4096;
constexpr long long kSiWaitCycles = 4000000000LL;  // about 2 s

struct SiState {
    unsigned arrive;
    int n, done, status, n_final, err;
    float rho[3], phin2[3], rz[3], alpha[3], beta[3];
    alignas(128) unsigned gen;  // barrier generation, alone in its line
    int pad[31];
};

struct SiDesc {
    float *x;                  // u^n (in/out), 3 planes: the leading part of the iterate
    float *xlo;                // its trailing part (u = x + xlo, a double-float pair)
    const float *phi, *lam;
    float *r, *z, *p[2], *q, *dg;
    float *fx, *fy;            // faces: 3 x H x wf (W+1 used), 3 x (H+1) x W
    float2 *part;              // [6][grid] per-CTA (sum, compensation)
    SiState *st;
    float *rho_hist;
    int H, W, wf, max_iter, cg_iters, dirichlet, no_edge, zero_lo;
    int vec;                   // W % 4 == 0, 16-byte aligned planes: the CG passes take 4 pixels a thread
    float tol, inv_s, eps, wg0, wg1, wg2;
};

// Reflecting (scipy 'reflect') or Dirichlet extension of one plane.
__device__ __forceinline__ float ext(const float *v, int H, int W, int i, int j, bool dir) {
    if (i < 0 || i >= W || j < 0 || j >= H) {
        if (dir) return 0.f;
        i = reflect_idx(i, W);
        j = reflect_idx(j, H);
    }
    return __ldca(v + (size_t)j * W + i);
}

// The iterate is a double-float pair (hi, lo): at eps = 1e-3 the face
// coefficients reach 1000, so a float32 u would put a rounding floor of about
// 1000 ulp(u) on F(u), well above a 1e-4 residual.  Differences of pairs are
// taken as (hi_a - hi_b) + (lo_a - lo_b): the first difference is exact for
// neighbouring values (Sterbenz), so the gradient carries ~2^-44 relative error.
struct Pair {
    float hi, lo;
};
__device__ __forceinline__ Pair ext2(const float *hi, const float *lo, int H, int W, int i, int j, bool dir) {
    if (i < 0 || i >= W || j < 0 || j >= H) {
        if (dir) return {0.f, 0.f};
        i = reflect_idx(i, W);
        j = reflect_idx(j, H);
    }
    const size_t o = (size_t)j * W + i;
    return {__ldca(hi + o), __ldca(lo + o)};
}
__device__ __forceinline__ float pdiff(Pair a, Pair b) { return (a.hi - b.hi) + (a.lo - b.lo); }

__device__ __forceinline__ float coef(float a, float b, float eps, bool no_edge) {
    return no_edge ? 1.f : 1.f / (sqrtf(fmaf(a, a, b * b)) + eps);
}

__device__ __forceinline__ float4 ldca4(const float *p) { return __ldca(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ldcg4(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void unpack(const float4 a, float (&v)[4]) {
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ float pick3(const float (&v)[3], int ch) { return ch == 0 ? v[0] : (ch == 1 ? v[1] : v[2]); }
// Neumaier-accumulate x into running sum k (no dynamic register indexing).
template <int K>
__device__ __forceinline__ void add_ch(float (&s)[K], float (&c)[K], int k, float x) {
#pragma unroll
    for (int q = 0; q < K; ++q)
        if (q == k) neumaier_add(s[q], c[q], x);
}
// One face term of (A v)_i: a coupling face (inside) adds D (v - nb); a border
// face adds D v under Dirichlet (ghost 0) and drops out under reflection.
__device__ __forceinline__ float face_term(float a, float D, float v, float nb, bool inside, bool dir) {
    return inside ? fmaf(D, v - nb, a) : (dir ? fmaf(D, v, a) : a);
}

// (A v)_i = v_i/s + sum_f D_f (v_i - v_nb); `get(i, j)` reads v inside the image.
template <class Get>
__device__ __forceinline__ float apply_A(const SiDesc &d, const float *fxc, const float *fyc, int x, int y,
                                         float v0, Get get, float *diag) {
    const int H = d.H, W = d.W;
    const bool dir = d.dirichlet != 0;
    float a = d.inv_s * v0, dg = d.inv_s;
    const float Dl = __ldca(fxc + (size_t)y * d.wf + x), Dr = __ldca(fxc + (size_t)y * d.wf + x + 1);
    const float Du = __ldca(fyc + (size_t)y * W + x), Dd = __ldca(fyc + (size_t)(y + 1) * W + x);
    if (x > 0) { a = fmaf(Dl, v0 - get(x - 1, y), a); dg += Dl; } else if (dir) { a = fmaf(Dl, v0, a); dg += Dl; }
    if (x < W - 1) { a = fmaf(Dr, v0 - get(x + 1, y), a); dg += Dr; } else if (dir) { a = fmaf(Dr, v0, a); dg += Dr; }
    if (y > 0) { a = fmaf(Du, v0 - get(x, y - 1), a); dg += Du; } else if (dir) { a = fmaf(Du, v0, a); dg += Du; }
    if (y < H - 1) { a = fmaf(Dd, v0 - get(x, y + 1), a); dg += Dd; } else if (dir) { a = fmaf(Dd, v0, a); dg += Dd; }
    if (diag) *diag = dg;
    return a;
}

// Per-CTA partial sums of nk quantities (k = quantity*3 + channel), written
// to part[k][blockIdx.x]; deterministic order.
template <int NK>
__device__ void cta_partials(float (&s)[NK], float (&c)[NK], float2 *part) {
    __shared__ float2 red[kSiThreads / 32][6];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[k], off);
            const float c2 = __shfl_down_sync(0xffffffffu, c[k], off);
            neumaier_merge(s[k], c[k], s2, c2);
        }
        if (lane == 0) red[w][k] = make_float2(s[k], c[k]);
    }
    __syncthreads();
    if (threadIdx.x < NK) {
        const int k = threadIdx.x;
        float a = red[0][k].x, b = red[0][k].y;
        for (int q = 1; q < kSiThreads / 32; ++q) neumaier_merge(a, b, red[q][k].x, red[q][k].y);
        part[(size_t)k * gridDim.x + blockIdx.x] = make_float2(a, b);
    }
}

// Last CTA: out[k] = fixed-order sum of part[k][0..grid) for k < nk.
__device__ void reduce_partials(const float2 *part, int nk, float *out) {
    __shared__ float2 red[kSiThreads / 32][6];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, G = gridDim.x;
    for (int k = 0; k < nk; ++k) {
        float s = 0.f, c = 0.f;
        for (int b = threadIdx.x; b < G; b += kSiThreads) {
            const float2 v = __ldcg(part + (size_t)k * G + b);
            neumaier_merge(s, c, v.x, v.y);
        }
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, off);
            const float c2 = __shfl_down_sync(0xffffffffu, c, off);
            neumaier_merge(s, c, s2, c2);
        }
        if (lane == 0) red[w][k] = make_float2(s, c);
    }
    __syncthreads();
    if (threadIdx.x < nk) {
        const int k = threadIdx.x;
        float a = red[0][k].x, b = red[0][k].y;
        for (int q = 1; q < kSiThreads / 32; ++q) neumaier_merge(a, b, red[q][k].x, red[q][k].y);
        out[k] = a + b;
    }
    __syncthreads();
}

// Grid barrier.  The last CTA to arrive runs fin() with all its threads, then
// releases the others; a wait longer than about 2 s records DH_ETIMEOUT and
// returns false.
template <class Fin>
__device__ bool grid_barrier(SiState *st, unsigned &gen, Fin fin) {
    __shared__ int s_last, s_to;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->arrive, 1u) == gridDim.x - 1u;
        s_to = 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        fin();
        __syncthreads();
        if (threadIdx.x == 0) {
            st->arrive = 0;
            __threadfence();
            st_release_gpu(&st->gen, gen + 1u);
        }
    } else if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (ld_acquire_gpu(&st->gen) == gen) {
            if (clock64() - t0 > kSiWaitCycles) {
                s_to = 1;
                break;
            }
            __nanosleep(32);
        }
    }
    ++gen;
    __syncthreads();
    if (s_to) {
        if (threadIdx.x == 0) {
            atomicCAS(&st->err, 0, DH_ETIMEOUT);
            st->status = DH_ETIMEOUT;
            st->done = 1;
        }
        return false;
    }
    return true;
}

__global__ void __launch_bounds__(kSiThreads, 3) k_semi_implicit(const __grid_constant__ SiDesc d) {
    SiState *st = d.st;
    const int H = d.H, W = d.W;
    const int N = H * W, E = 3 * N;
    const int G = gridDim.x, T = G * kSiThreads;
    const int e0 = blockIdx.x * kSiThreads + threadIdx.x;
    const bool dir = d.dirichlet != 0, ne = d.no_edge != 0;
    __shared__ float sc[6];
    unsigned gen = ld_acquire_gpu(&st->gen);

    // ||Phi^c||^2
    {
        float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
        for (int e = e0; e < E; e += T) {
            const int ch = e / N;
            const float v = __ldg(d.phi + e);
            add_ch(s, c, ch, v * v);
            if (d.zero_lo) d.xlo[e] = 0.f;
        }
        cta_partials<3>(s, c, d.part);
        if (!grid_barrier(st, gen, [&] {
                reduce_partials(d.part, 3, sc);
                if (threadIdx.x < 3) st->phin2[threadIdx.x] = sc[threadIdx.x];
            }))
            return;
    }

    for (;;) {
        // faces of u^n
        for (int e = e0; e < E; e += T) {
            const int ch = e / N, pix = e - ch * N, y = pix / W, x = pix - y * W;
            const float *xc = d.x + (size_t)ch * N, *lc = d.xlo + (size_t)ch * N;
            float *fxc = d.fx + (size_t)ch * H * d.wf, *fyc = d.fy + (size_t)ch * (H + 1) * W;
            auto U = [&](int i, int j) { return ext2(xc, lc, H, W, i, j, dir); };
            const Pair u0 = U(x, y);
            {  // x-face (x+1/2, y), tangential difference at cell x
                const float a = pdiff(U(x + 1, y), u0);
                const float b = 0.5f * pdiff(U(x, y + 1), U(x, y - 1));
                fxc[(size_t)y * d.wf + x + 1] = coef(a, b, d.eps, ne);
            }
            if (x == 0) {  // x-face (-1/2, y): tangential difference at the ghost cell
                const float a = pdiff(u0, U(-1, y));
                const float b = 0.5f * pdiff(U(-1, y + 1), U(-1, y - 1));
                fxc[(size_t)y * d.wf] = coef(a, b, d.eps, ne);
            }
            {  // y-face (x, y+1/2)
                const float a = pdiff(U(x, y + 1), u0);
                const float b = 0.5f * pdiff(U(x + 1, y), U(x - 1, y));
                fyc[(size_t)(y + 1) * W + x] = coef(a, b, d.eps, ne);
            }
            if (y == 0) {
                const float a = pdiff(u0, U(x, -1));
                const float b = 0.5f * pdiff(U(x + 1, -1), U(x - 1, -1));
                fyc[x] = coef(a, b, d.eps, ne);
            }
        }
        if (!grid_barrier(st, gen, [] {})) return;

        // r = F(u^n) = Phi - lambda G(u^n) - L_n u^n, z = r / diag, p = z
        {
            float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float wg[5] = {d.wg2, d.wg1, d.wg0, d.wg1, d.wg2};
            for (int e = e0; e < E; e += T) {
                const int ch = e / N, pix = e - ch * N, y = pix / W, x = pix - y * W;
                const float *xc = d.x + (size_t)ch * N, *lc = d.xlo + (size_t)ch * N;
                const float *fxc = d.fx + (size_t)ch * H * d.wf, *fyc = d.fy + (size_t)ch * (H + 1) * W;
                float g = 0.f;
                for (int b = -2; b <= 2; ++b) {
                    float h = 0.f;
                    for (int a = -2; a <= 2; ++a) h = fmaf(wg[a + 2], ext(xc, H, W, x + a, y + b, dir), h);
                    g = fmaf(wg[b + 2], h, g);
                }
                // L_n u^n = sum_f D_f (u_i - u_nb) with pair differences;
                // diag = 1/s + the faces that couple (all four under Dirichlet)
                const Pair u0 = ext2(xc, lc, H, W, x, y, dir);
                const float Dl = __ldca(fxc + (size_t)y * d.wf + x), Dr = __ldca(fxc + (size_t)y * d.wf + x + 1);
                const float Du = __ldca(fyc + (size_t)y * W + x), Dd = __ldca(fyc + (size_t)(y + 1) * W + x);
                float Lu = 0.f, dg = d.inv_s;
                if (x > 0 || dir) { Lu = fmaf(Dl, pdiff(u0, ext2(xc, lc, H, W, x - 1, y, dir)), Lu); dg += Dl; }
                if (x < W - 1 || dir) { Lu = fmaf(Dr, pdiff(u0, ext2(xc, lc, H, W, x + 1, y, dir)), Lu); dg += Dr; }
                if (y > 0 || dir) { Lu = fmaf(Du, pdiff(u0, ext2(xc, lc, H, W, x, y - 1, dir)), Lu); dg += Du; }
                if (y < H - 1 || dir) { Lu = fmaf(Dd, pdiff(u0, ext2(xc, lc, H, W, x, y + 1, dir)), Lu); dg += Dd; }
                const float r = __ldg(d.phi + e) - __ldg(d.lam + pix) * g - Lu;
                const float z = r / dg;
                d.r[e] = r;
                d.z[e] = z;
                d.p[0][e] = z;
                d.dg[e] = dg;
                add_ch(s, c, ch, r * r);
                add_ch(s, c, 3 + ch, r * z);
            }
            cta_partials<6>(s, c, d.part);
        }
        if (!grid_barrier(st, gen, [&] {
                reduce_partials(d.part, 6, sc);
                if (threadIdx.x != 0) return;
                const int n = st->n;
                float rho[3], worst = 0.f;
                bool finite = true;
                for (int ch = 0; ch < 3; ++ch) {
                    const float pn = st->phin2[ch];
                    rho[ch] = pn > 0.f ? sqrtf(sc[ch] / pn) : sqrtf(sc[ch]);
                    if (!isfinite(rho[ch])) finite = false;
                    else worst = fmaxf(worst, rho[ch]);
                    if (d.rho_hist) d.rho_hist[3 * n + ch] = rho[ch];
                    st->rz[ch] = sc[3 + ch];
                }
                const int err = st->err;
                const bool conv = finite && worst <= d.tol;
                if (err || conv || !finite || n >= d.max_iter) {
                    st->done = 1;
                    st->n_final = n;
                    st->status = err ? err : (!finite ? DH_ENONFINITE : (conv ? DH_OK : DH_WNOCONV));
                    for (int ch = 0; ch < 3; ++ch) st->rho[ch] = rho[ch];
                }
            }))
            return;
        if (__ldcg(&st->done)) return;

        for (int k = 0; k < d.cg_iters; ++k) {
            const float *pold = d.p[(k + 1) & 1];
            float *pcur = d.p[k & 1];
            // q = A p (p = z + beta p_old, formed where it is read), p.q
            {
                float beta[3];
                for (int ch = 0; ch < 3; ++ch) beta[ch] = __ldcg(&st->beta[ch]);
                float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
                // four pixels of a row a thread (W % 4 == 0): 16-byte loads of p
                // (or z and p_old) on the quad and the rows above and below, single
                // loads for the left and right neighbours, faces from 16-byte rows;
                // per pixel the same operations in the same order as apply_A
                const int Q = W >> 2, HQ = H * Q, NQ = d.vec ? 3 * HQ : 0;
                for (int g = e0; g < NQ; g += T) {
                    const int ch = g / HQ, rem = g - ch * HQ, y = rem / Q, x0 = (rem - y * Q) << 2;
                    const size_t o = (size_t)ch * N + (size_t)y * W + x0;
                    const bool hu = y > 0, hd = y < H - 1, hl = x0 > 0, hr = x0 + 4 < W;
                    float v[4], vu[4] = {0.f, 0.f, 0.f, 0.f}, vd[4] = {0.f, 0.f, 0.f, 0.f}, vl = 0.f, vr = 0.f;
                    if (k == 0) {
                        unpack(ldca4(pcur + o), v);
                        if (hu) unpack(ldca4(pcur + o - W), vu);
                        if (hd) unpack(ldca4(pcur + o + W), vd);
                        if (hl) vl = __ldca(pcur + o - 1);
                        if (hr) vr = __ldca(pcur + o + 4);
                    } else {
                        const float bt = pick3(beta, ch);
                        auto p4 = [&](size_t q, float (&out)[4]) {
                            float a[4], z[4];
                            unpack(ldca4(pold + q), a);
                            unpack(ldca4(d.z + q), z);
#pragma unroll
                            for (int i = 0; i < 4; ++i) out[i] = fmaf(bt, a[i], z[i]);
                        };
                        auto p1 = [&](size_t q) { return fmaf(bt, __ldca(pold + q), __ldca(d.z + q)); };
                        p4(o, v);
                        if (hu) p4(o - W, vu);
                        if (hd) p4(o + W, vd);
                        if (hl) vl = p1(o - 1);
                        if (hr) vr = p1(o + 4);
                        st4(pcur + o, v);
                    }
                    const float *fxr = d.fx + (size_t)ch * H * d.wf + (size_t)y * d.wf + x0;
                    const float *fyr = d.fy + (size_t)ch * (H + 1) * W + (size_t)y * W + x0;
                    float Dx[5], Du[4], Dd[4];  // Dx[i]: face x0 + i - 1/2
                    {
                        float t[4];
                        unpack(ldca4(fxr), t);
#pragma unroll
                        for (int i = 0; i < 4; ++i) Dx[i] = t[i];
                        Dx[4] = __ldca(fxr + 4);
                    }
                    unpack(ldca4(fyr), Du);
                    unpack(ldca4(fyr + W), Dd);
                    float qv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float a = d.inv_s * v[i];
                        a = face_term(a, Dx[i], v[i], i > 0 ? v[i - 1] : vl, i > 0 || hl, dir);
                        a = face_term(a, Dx[i + 1], v[i], i < 3 ? v[i + 1] : vr, i < 3 || hr, dir);
                        a = face_term(a, Du[i], v[i], vu[i], hu, dir);
                        a = face_term(a, Dd[i], v[i], vd[i], hd, dir);
                        qv[i] = a;
                        add_ch(s, c, ch, v[i] * a);
                    }
                    st4(d.q + o, qv);
                }
                for (int e = d.vec ? E : e0; e < E; e += T) {
                    const int ch = e / N, pix = e - ch * N, y = pix / W, x = pix - y * W;
                    const float *fxc = d.fx + (size_t)ch * H * d.wf, *fyc = d.fy + (size_t)ch * (H + 1) * W;
                    const size_t base = (size_t)ch * N;
                    float pv, qv;
                    if (k == 0) {
                        const float *pc = pcur + base;
                        pv = __ldca(pc + pix);
                        qv = apply_A(d, fxc, fyc, x, y, pv,
                                     [&](int i, int j) { return __ldca(pc + (size_t)j * W + i); }, nullptr);
                    } else {
                        const float *zc = d.z + base, *oc = pold + base;
                        const float bt = pick3(beta, ch);
                        auto get = [&](int i, int j) {
                            const size_t o = (size_t)j * W + i;
                            return fmaf(bt, __ldca(oc + o), __ldca(zc + o));
                        };
                        pv = get(x, y);
                        pcur[e] = pv;
                        qv = apply_A(d, fxc, fyc, x, y, pv, get, nullptr);
                    }
                    d.q[e] = qv;
                    add_ch(s, c, ch, pv * qv);
                }
                cta_partials<3>(s, c, d.part);
            }
            if (!grid_barrier(st, gen, [&] {
                    reduce_partials(d.part, 3, sc);
                    if (threadIdx.x < 3) {
                        const int ch = threadIdx.x;
                        const float pq = sc[ch];
                        st->alpha[ch] = pq > 0.f ? st->rz[ch] / pq : 0.f;
                    }
                }))
                return;
            // x += alpha p, r -= alpha q, z = r / diag, r.z
            {
                float alpha[3];
                for (int ch = 0; ch < 3; ++ch) alpha[ch] = __ldcg(&st->alpha[ch]);
                float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
                // four consecutive elements a thread (one channel: N % 4 == 0)
                const int NQ = d.vec ? E >> 2 : 0;
                for (int g = e0; g < NQ; g += T) {
                    const int e = g << 2, ch = e / N;
                    const float al = pick3(alpha, ch);
                    float hi[4], lo[4], pv[4], qv[4], rv[4], dg[4];
                    unpack(ldcg4(d.x + e), hi);
                    unpack(ldcg4(d.xlo + e), lo);
                    unpack(ldcg4(pcur + e), pv);
                    unpack(ldcg4(d.q + e), qv);
                    unpack(ldcg4(d.r + e), rv);
                    unpack(ldcg4(d.dg + e), dg);
                    float zv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {  // (hi, lo) += alpha p: two-sum, then renormalise
                        const float dlt = al * pv[i];
                        const float s1 = hi[i] + dlt, bb = s1 - hi[i];
                        const float err = (hi[i] - (s1 - bb)) + (dlt - bb);
                        const float l2 = lo[i] + err;
                        const float h2 = s1 + l2;
                        hi[i] = h2;
                        lo[i] = l2 - (h2 - s1);
                        rv[i] = fmaf(-al, qv[i], rv[i]);
                        zv[i] = rv[i] / dg[i];
                        add_ch(s, c, ch, rv[i] * zv[i]);
                    }
                    st4(d.x + e, hi);
                    st4(d.xlo + e, lo);
                    st4(d.r + e, rv);
                    st4(d.z + e, zv);
                }
                for (int e = d.vec ? E : e0; e < E; e += T) {
                    const int ch = e / N;
                    const float al = pick3(alpha, ch);
                    {  // (hi, lo) += alpha p: two-sum, then renormalise
                        const float hi = __ldcg(d.x + e), dlt = al * __ldcg(pcur + e);
                        const float s1 = hi + dlt, bb = s1 - hi;
                        const float err = (hi - (s1 - bb)) + (dlt - bb);
                        const float lo = __ldcg(d.xlo + e) + err;
                        const float h2 = s1 + lo;
                        d.x[e] = h2;
                        d.xlo[e] = lo - (h2 - s1);
                    }
                    const float r = fmaf(-al, __ldcg(d.q + e), __ldcg(d.r + e));
                    const float z = r / __ldcg(d.dg + e);
                    d.r[e] = r;
                    d.z[e] = z;
                    add_ch(s, c, ch, r * z);
                }
                cta_partials<3>(s, c, d.part);
            }
            const bool last = k == d.cg_iters - 1;
            if (!grid_barrier(st, gen, [&] {
                    reduce_partials(d.part, 3, sc);
                    if (threadIdx.x < 3) {
                        const int ch = threadIdx.x;
                        const float rz = st->rz[ch];
                        st->beta[ch] = rz > 0.f ? sc[ch] / rz : 0.f;
                        st->rz[ch] = sc[ch];
                    }
                    if (threadIdx.x == 0 && last) st->n = st->n + 1;
                }))
                return;
        }
    }
}

// J = clamp(u, 0, 1) (the restored image).
__global__ void k_si_clamp(const float *__restrict__ u, float *__restrict__ J, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        J[i] = fminf(fmaxf(u[i], 0.f), 1.f);
}

__global__ void k_si_reset(SiState *st) {
    st->arrive = 0;
    st->n = 0;
    st->done = 0;
    st->status = 0;
    st->n_final = 0;
    st->err = 0;
}

// Row stride of the x-face planes (W + 1 faces a row), a multiple of 4 so
// that every row starts on a 16-byte boundary.
int face_stride(int W) { return (W + 1 + 3) & ~3; }

struct SiLayout {
    size_t state, part, planes, fx, fy, total;
};

SiLayout si_layout(int H, int W) {
    SiLayout L;
    const size_t N = (size_t)H * W;
    size_t o = 0;
    L.state = o; o = align_up(o + sizeof(SiState));
    L.part = o; o = align_up(o + (size_t)6 * kSiMaxGrid * sizeof(float2));
    L.planes = o; o = align_up(o + (size_t)7 * 3 * N * sizeof(float));  // r, z, p0, p1, q, diag, u's low part
    L.fx = o; o = align_up(o + (size_t)3 * H * face_stride(W) * sizeof(float));
    L.fy = o; o = align_up(o + (size_t)3 * (H + 1) * W * sizeof(float));
    L.total = o;
    return L;
}

int si_grid(int E) {
    static std::mutex mu;
    static int cached = 0, cached_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (cached_dev != dev) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_semi_implicit, kSiThreads, 0) != cudaSuccess)
            return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cached = per_sm * sms;
        cached_dev = dev;
    }
    // at least 8 elements per thread: fewer CTAs make the grid barriers cheaper
    int g = (E + 8 * kSiThreads - 1) / (8 * kSiThreads);
    if (g > cached) g = cached;
    if (g > kSiMaxGrid) g = kSiMaxGrid;
    return g;
}

}  // namespace

size_t semi_workspace_bytes(int H, int W) { return si_layout(H, W).total; }

int run_semi_implicit(float *u, float *u_lo, const float *Phi, const float *lam, int H, int W, const dh_params *p,
                      float step, int cg_iters, float *rho_hist, float *J, void *workspace, cudaStream_t s) {
    const SiLayout L = si_layout(H, W);
    char *ws = (char *)workspace;
    const size_t n3 = (size_t)3 * H * W;
    SiDesc d = {};
    d.x = u;
    d.phi = Phi;
    d.lam = lam;
    float *pl = (float *)(ws + L.planes);
    d.r = pl;
    d.z = pl + n3;
    d.p[0] = pl + 2 * n3;
    d.p[1] = pl + 3 * n3;
    d.q = pl + 4 * n3;
    d.dg = pl + 5 * n3;
    d.xlo = u_lo ? u_lo : pl + 6 * n3;
    d.zero_lo = u_lo ? 0 : 1;
    d.fx = (float *)(ws + L.fx);
    d.fy = (float *)(ws + L.fy);
    d.part = (float2 *)(ws + L.part);
    d.st = (SiState *)(ws + L.state);
    d.rho_hist = rho_hist;
    d.H = H;
    d.W = W;
    d.wf = face_stride(W);
    {
        auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
        d.vec = W % 4 == 0 && a16(d.x) && a16(d.xlo);
    }
    d.max_iter = p->max_iter;
    d.cg_iters = cg_iters;
    d.dirichlet = p->boundary == DH_BOUNDARY_ZERO;
    d.no_edge = (p->variant & DH_VAR_NO_EDGE) != 0;
    d.tol = p->tol;
    d.inv_s = 1.0f / step;
    d.eps = p->eps;
    {  // App. A-B-2: normalised 5-tap Gaussian
        double w[3];
        for (int k = 0; k <= 2; ++k) w[k] = exp(-(double)(k * k) / (2.0 * (double)p->sigma * p->sigma));
        const double sum = w[0] + 2.0 * (w[1] + w[2]);
        d.wg0 = (float)(w[0] / sum);
        d.wg1 = (float)(w[1] / sum);
        d.wg2 = (float)(w[2] / sum);
    }
    const int G = si_grid((int)n3);
    if (G <= 0) return DH_ECUDA;
    k_si_reset<<<1, 1, 0, s>>>(d.st);
    DH_CUDA_TRY(cudaGetLastError());
    void *args[1] = {(void *)&d};
    DH_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_semi_implicit, dim3(G), dim3(kSiThreads), args, 0, s));
    if (J) {
        const int g = (int)((n3 + 255) / 256 < 4096 ? (n3 + 255) / 256 : 4096);
        k_si_clamp<<<g, 256, 0, s>>>(u, J, n3);
        DH_CUDA_TRY(cudaGetLastError());
    }
    return DH_OK;
}

// Outcome of the last solve queued on this workspace (synchronises s).
int read_semi_implicit(const void *workspace, cudaStream_t s, int *n_final, int *status, float rho[3]) {
    SiState st;
    const SiLayout L = si_layout(1, 1);
    DH_CUDA_TRY(cudaMemcpyAsync(&st, (const char *)workspace + L.state, sizeof(st), cudaMemcpyDeviceToHost, s));
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    *n_final = st.n_final;
    *status = st.status;
    for (int c = 0; c < 3; ++c) rho[c] = st.rho[c];
    return DH_OK;
}

}  // namespace dh
