// Fixed-point solver of App. A-A for -div(D(grad u) grad u) + lambda G(u) = Phi
// (Sec. II-A), one sweep kernel per iteration:
//   F(u) = div(D grad u) - lambda G(u) + Phi,  u <- u + tau F(u)
// with the flux-form stencil of App. A-B-1 and the 5x5 Gaussian of App. A-B-2,
// plus the per-iteration residual, the stop decision and the loop engine.
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace dh {

// PTX approximations of the square root and the reciprocal (MUFU; relative
// error about 2^-22).  The face flux D*u_x only needs float32-level accuracy.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// D u_n on one face: a = difference across the face, b = the half central
// difference along it, D = (sqrt(a^2 + b^2) + eps)^-1 (Sec. II-B, App. A-B-1).
template <bool EDGE>
__device__ __forceinline__ float face_flux(float a, float b, float eps) {
    if (!EDGE) return a;  // ablation: D == 1
    const float s = fmaf(a, a, b * b);
    return a * rcp_approx(sqrt_approx(s) + eps);
}

__device__ __forceinline__ int ld_state_int(const int *p) { return __ldcg(p); }

// Reduces the per-CTA partials of the launch (last CTA only), decides whether
// to stop, advances the state and sets the graph's while condition.
__device__ void finish_iteration(const SolveDesc *d, SolveState *st) {
    __shared__ float sq[3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __threadfence();
    for (int ch = w; ch < 3; ch += blockDim.x >> 5) {
        float s = 0.f, cc = 0.f;
        const float2 *part = d->part + (size_t)ch * d->nblk;
        for (int b = lane; b < d->nblk; b += 32) {
            const float2 p = __ldcg(part + b);
            neumaier_merge(s, cc, p.x, p.y);
        }
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, off);
            const float c2 = __shfl_down_sync(0xffffffffu, cc, off);
            neumaier_merge(s, cc, s2, c2);
        }
        if (lane == 0) sq[ch] = s + cc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int n = st->n;
    float worst = 0.f;
    bool finite = true;
    float rho[3];
    for (int c = 0; c < 3; ++c) {
        const float pn = st->phin2[c];
        rho[c] = pn > 0.f ? sqrtf(sq[c] / pn) : sqrtf(sq[c]);
        if (!isfinite(rho[c])) finite = false;
        else worst = fmaxf(worst, rho[c]);
        if (d->rho_hist) d->rho_hist[3 * n + c] = rho[c];
    }
    const bool conv = finite && worst <= d->tol;
    unsigned cont = 1;
    if (conv || !finite || n >= d->max_iter) {
        st->done = 1;
        st->n_final = n;
        st->status = !finite ? DH_ENONFINITE : (conv ? DH_OK : DH_WNOCONV);
        for (int c = 0; c < 3; ++c) st->rho[c] = rho[c];
        cont = 0;
    } else {
        st->n = n + 1;
        st->cur ^= 1;
    }
    st->arrive = 0;
    __threadfence();
    if (d->use_cond) cudaGraphSetConditional(d->cond, cont);
}

// One iteration for a TW x (R*NW) tile of one channel (blockIdx.z).
// Shared memory holds the tile of u^n with a 2-row / 4-column halo; each warp
// walks R rows, each lane owns 4 adjacent columns and keeps rolling registers
// of the last rows of u, of the horizontally filtered rows and of the y-face
// fluxes, so every face flux and every Gaussian row is computed once.
template <int R, int NW, bool EDGE>
__global__ void __launch_bounds__(NW * 32)
k_sweep(const SolveDesc *__restrict__ d) {
    constexpr int TH = R * NW;
    constexpr int SW = kTW + 8;
    constexpr int SH = TH + 4;
    __shared__ __align__(16) float s[SH][SW];
    __shared__ float2 red[NW];
    __shared__ int s_last;

    SolveState *st = d->st;
    // The loop ends unless this launch's last CTA sets the condition back to
    // 1, so a launch that failed to count its CTAs cannot spin forever.  CTA
    // (0,0,0) clears it before it arrives, hence before the last CTA decides.
    if (d->use_cond && (blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) {
        cudaGraphSetConditional(d->cond, 0);
        __threadfence();
    }
    if (ld_state_int(&st->done)) return;
    const int H = d->H, W = d->W;
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * TH;
    const int cur = ld_state_int(&st->cur);
    const size_t N = (size_t)H * W;
    const float *__restrict__ u = d->u[cur] + c * N;
    float *__restrict__ un = d->u[cur ^ 1] + c * N;
    const float *__restrict__ phi = d->phi + c * N;
    const float *__restrict__ lam = d->lam;
    const float eps = d->eps, tau = d->tau;
    const float wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;

    // tile of u^n, rows y0-2 .. y0+TH+1, columns x0-4 .. x0+TW+3, reflected
    for (int e = threadIdx.x; e < SH * SW; e += NW * 32) {
        const int r = e / SW, q = e - r * SW;
        const int gy = reflect_idx(y0 - 2 + r, H), gx = reflect_idx(x0 - 4 + q, W);
        s[r][q] = u[(size_t)gy * W + gx];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int sc = 4 * lane;      // smem column of x-4 for this lane's x
    const int x = x0 + 4 * lane;  // first of the lane's 4 columns
    const int r0 = w * R;         // first tile row of this warp
    const bool vec = d->vec != 0;

    // rolling registers: uu[k][j] = u at tile row (r0-1+k) (mod 4 ring),
    // column x-1+j (j = 0..5); gh[k][j] = horizontal Gaussian at tile row
    // (r0-2+k) (mod 5 ring), column x+j.
    float uu[4][6];
    float gh[5][4];
    float fyu[4];

    auto load_row = [&](int tr, float *v6, float *g4) {
        // tr = tile row (may be -2 .. TH+1); smem row tr+2
        const float4 L = *reinterpret_cast<const float4 *>(&s[tr + 2][sc]);
        const float4 C = *reinterpret_cast<const float4 *>(&s[tr + 2][sc + 4]);
        const float4 Rr = *reinterpret_cast<const float4 *>(&s[tr + 2][sc + 8]);
        const float v[8] = {L.z, L.w, C.x, C.y, C.z, C.w, Rr.x, Rr.y};  // x-2 .. x+5
#pragma unroll
        for (int j = 0; j < 4; ++j)
            g4[j] = fmaf(wg2, v[j] + v[j + 4], fmaf(wg1, v[j + 1] + v[j + 3], wg0 * v[j + 2]));
        if (v6) {
#pragma unroll
            for (int j = 0; j < 6; ++j) v6[j] = v[j + 1];
        }
    };

    // prologue: Gaussian rows r0-2, r0-1, r0, r0+1; u rows r0-1, r0, r0+1
    {
        float dummy[6];
        load_row(r0 - 2, dummy, gh[0]);
        load_row(r0 - 1, uu[0], gh[1]);
        load_row(r0, uu[1], gh[2]);
        load_row(r0 + 1, uu[2], gh[3]);
        // y-face flux at r0 - 1/2, tangential difference on row r0-1
#pragma unroll
        for (int j = 0; j < 4; ++j)
            fyu[j] = face_flux<EDGE>(uu[1][j + 1] - uu[0][j + 1], 0.5f * (uu[0][j + 2] - uu[0][j]), eps);
    }

    float rs = 0.f, rc = 0.f;  // compensated sum of F^2 over the lane's pixels
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ty = r0 + i;
        const int y = y0 + ty;
        float *um = uu[(i + 0) & 3];
        float *u0 = uu[(i + 1) & 3];
        float *up = uu[(i + 2) & 3];
        float *upp = uu[(i + 3) & 3];
        load_row(ty + 2, upp, gh[(i + 4) % 5]);
        const float *g_m2 = gh[(i + 0) % 5], *g_m1 = gh[(i + 1) % 5], *g_0 = gh[(i + 2) % 5];
        const float *g_p1 = gh[(i + 3) % 5], *g_p2 = gh[(i + 4) % 5];

        // x-face fluxes at x-1/2 .. x+3+1/2 (tangential difference at the face's left cell)
        float fx[5];
#pragma unroll
        for (int j = 0; j < 5; ++j)
            fx[j] = face_flux<EDGE>(u0[j + 1] - u0[j], 0.5f * (up[j] - um[j]), eps);
        float fyd[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            fyd[j] = face_flux<EDGE>(up[j + 1] - u0[j + 1], 0.5f * (u0[j + 2] - u0[j]), eps);

        float ph[4] = {0.f, 0.f, 0.f, 0.f}, la[4] = {0.f, 0.f, 0.f, 0.f};
        const bool row_ok = y < H;
        const size_t ro = (size_t)y * W;
        if (row_ok) {
            if (vec && x < W) {
                const float4 p4 = __ldg(reinterpret_cast<const float4 *>(phi + ro + x));
                const float4 l4 = __ldg(reinterpret_cast<const float4 *>(lam + ro + x));
                ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
            } else if (!vec) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x + j < W) { ph[j] = __ldg(phi + ro + x + j); la[j] = __ldg(lam + ro + x + j); }
            }
        }
        float nu[4];
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float G = fmaf(wg2, g_m2[j] + g_p2[j], fmaf(wg1, g_m1[j] + g_p1[j], wg0 * g_0[j]));
            const float dv = (fx[j + 1] - fx[j]) + (fyd[j] - fyu[j]);
            const float F = fmaf(-la[j], G, dv) + ph[j];
            nu[j] = fmaf(tau, F, u0[j + 1]);
            if (x + j < W) q = fmaf(F, F, q);
            fyu[j] = fyd[j];
        }
        if (row_ok) {
            neumaier_add(rs, rc, q);
            if (vec && x < W) {
                *reinterpret_cast<float4 *>(un + ro + x) = make_float4(nu[0], nu[1], nu[2], nu[3]);
            } else if (!vec) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x + j < W) un[ro + x + j] = nu[j];
            }
        }
    }

    // deterministic block reduction of the residual partial
    for (int off = 16; off; off >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, rs, off);
        const float c2 = __shfl_down_sync(0xffffffffu, rc, off);
        neumaier_merge(rs, rc, s2, c2);
    }
    if (lane == 0) red[w] = make_float2(rs, rc);
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = red[0].x, b = red[0].y;
#pragma unroll
        for (int k = 1; k < NW; ++k) neumaier_merge(a, b, red[k].x, red[k].y);
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        d->part[(size_t)c * d->nblk + blk] = make_float2(a, b);
        __threadfence();
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        s_last = prev == 3u * d->nblk - 1u;
    }
    __syncthreads();
    if (s_last) finish_iteration(d, st);
}

// ------------------------------------------------------------ small kernels

__global__ void k_set_desc(SolveDesc *dst, SolveDesc v) {
    *dst = v;
    SolveState *st = v.st;
    st->arrive = 0;
    st->n = 0;
    st->cur = 0;
    st->done = 0;
    st->status = 0;
    st->n_final = 0;
}

// J = clamp(u^n, 0, 1) and u^n copied to the caller's u when it sits in the
// workspace buffer.
__global__ void k_output(const SolveDesc *__restrict__ d, float *J) {
    const int cur = ld_state_int(&d->st->cur);
    const size_t n3 = (size_t)3 * d->H * d->W;
    const float *src = d->u[cur];
    float *u0 = d->u[0];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (size_t)gridDim.x * blockDim.x) {
        const float v = src[i];
        if (cur) u0[i] = v;
        if (J) J[i] = fminf(fmaxf(v, 0.f), 1.f);
    }
}

// ------------------------------------------------------------ configuration

struct SweepCfg {
    int R, NW;
    bool edge;
};

typedef void (*SweepFn)(const SolveDesc *);

static SweepFn sweep_fn(int R, int NW, bool edge) {
#define DH_SW(r, nw)                                              \
    if (R == r && NW == nw) return edge ? k_sweep<r, nw, true> : k_sweep<r, nw, false>;
    DH_SW(16, 4)
    DH_SW(8, 4)
    DH_SW(16, 2)
    DH_SW(8, 8)
#undef DH_SW
    return nullptr;
}

int sweep_depth(const dh_params *) { return 1; }
int sweep_tile_h(int) { return 16 * 4; }

// ------------------------------------------------------------ graph cache

struct GraphKey {
    int dev;
    const void *ws;
    int H, W, R, NW, edge;
    bool operator==(const GraphKey &o) const {
        return dev == o.dev && ws == o.ws && H == o.H && W == o.W && R == o.R && NW == o.NW &&
               edge == o.edge;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    cudaGraphConditionalHandle cond;
    unsigned long long last_use;
};

static std::mutex g_mu;
static std::vector<GraphEntry> g_cache;
static unsigned long long g_clock = 0;
constexpr size_t kGraphCacheMax = 16;

// A graph holding one while node whose body is the sweep kernel; the sweep's
// last CTA sets the condition to 0 when the loop has to stop.
static int get_loop_graph(const GraphKey &key, dim3 grid, dim3 block, const SolveDesc *desc_dev,
                          SweepFn fn, GraphEntry *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &e : g_cache)
        if (e.key == key) {
            e.last_use = ++g_clock;
            *out = e;
            return DH_OK;
        }
    cudaGraph_t g = nullptr;
    DH_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNode_t wn;
    cudaGraphNodeParams cp = {};
    if (err == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        err = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &cp);
    }
    if (err == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaKernelNodeParams kp = {};
        void *args[] = {(void *)&desc_dev};
        kp.func = (void *)fn;
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t kn;
        err = cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp);
    }
    cudaGraphExec_t exec = nullptr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return cuda_fail(err);
    if (g_cache.size() >= kGraphCacheMax) {
        size_t old = 0;
        for (size_t i = 1; i < g_cache.size(); ++i)
            if (g_cache[i].last_use < g_cache[old].last_use) old = i;
        cudaGraphExecDestroy(g_cache[old].exec);
        g_cache.erase(g_cache.begin() + old);
    }
    GraphEntry e{key, exec, h, ++g_clock};
    g_cache.push_back(e);
    *out = e;
    return DH_OK;
}

// ------------------------------------------------------------ the solve loop

// Queues the fixed-point loop for buffers u[0] (caller's, holds u^0) and
// u[1] (workspace).  st->phin2 must already be set on the stream.
int run_solve(float *u_caller, const float *phi, const float *lam, int H, int W, const dh_params *p,
              float *rho_hist, char *ws, const WsLayout &L, cudaStream_t s, float *J,
              cudaEvent_t loop_begin, cudaEvent_t loop_end, int *launches) {
    const SweepCfg cfg{16, 4, !(p->variant & DH_VAR_NO_EDGE)};
    SweepFn fn = sweep_fn(cfg.R, cfg.NW, cfg.edge);
    if (!fn) return DH_EINVAL;
    const int TH = cfg.R * cfg.NW;
    dim3 grid((W + kTW - 1) / kTW, (H + TH - 1) / TH, 3);
    dim3 block(cfg.NW * 32);
    SolveDesc *desc_dev = (SolveDesc *)(ws + L.desc);
    SolveDesc v = {};
    v.u[0] = u_caller;
    v.u[1] = (float *)(ws + L.ub);
    v.phi = phi;
    v.lam = lam;
    v.rho_hist = rho_hist;
    v.part = (float2 *)(ws + L.part);
    v.st = (SolveState *)(ws + L.state);
    v.H = H;
    v.W = W;
    v.max_iter = p->max_iter;
    v.depth = 1;
    v.nblk = grid.x * grid.y;
    if (v.nblk > L.nblk_sweep) return DH_EINVAL;  // workspace sized for another tiling
    {
        auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
        v.vec = (W % 4 == 0) && a16(u_caller) && a16(v.u[1]) && a16(phi) && a16(lam);
    }
    v.tol = p->tol;
    v.tau = p->tau;
    v.eps = p->eps;
    {  // App. A-B-2: normalised 5-tap Gaussian, sigma = p->sigma
        double w[3], sum = 0.0;
        for (int k = 0; k <= 2; ++k) w[k] = exp(-(double)(k * k) / (2.0 * (double)p->sigma * p->sigma));
        sum = w[0] + 2.0 * (w[1] + w[2]);
        v.wg0 = (float)(w[0] / sum);
        v.wg1 = (float)(w[1] / sum);
        v.wg2 = (float)(w[2] / sum);
    }
    if (p->use_graph) {
        int dev = 0;
        DH_CUDA_TRY(cudaGetDevice(&dev));
        GraphKey key{dev, ws, H, W, cfg.R, cfg.NW, cfg.edge ? 1 : 0};
        GraphEntry ge;
        int rc = get_loop_graph(key, grid, block, desc_dev, fn, &ge);
        if (rc != DH_OK) return rc;
        v.cond = ge.cond;
        v.use_cond = 1;
        k_set_desc<<<1, 1, 0, s>>>(desc_dev, v);
        DH_CUDA_TRY(cudaGetLastError());
        if (loop_begin) DH_CUDA_TRY(cudaEventRecord(loop_begin, s));
        DH_CUDA_TRY(cudaGraphLaunch(ge.exec, s));
        if (loop_end) DH_CUDA_TRY(cudaEventRecord(loop_end, s));
    } else {
        v.use_cond = 0;
        k_set_desc<<<1, 1, 0, s>>>(desc_dev, v);
        if (loop_begin) DH_CUDA_TRY(cudaEventRecord(loop_begin, s));
        for (int n = 0; n <= p->max_iter; ++n) fn<<<grid, block, 0, s>>>(desc_dev);
        DH_CUDA_TRY(cudaGetLastError());
        if (loop_end) DH_CUDA_TRY(cudaEventRecord(loop_end, s));
        if (launches) *launches += p->max_iter + 1;  // queued; finished ones exit at once
    }
    if (launches) *launches += 2;  // k_set_desc, k_output
    const size_t n3 = (size_t)3 * H * W;
    const int ob = (int)((n3 + 255) / 256 < 152 * 16 ? (n3 + 255) / 256 : 152 * 16);
    k_output<<<ob, 256, 0, s>>>(desc_dev, J);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int read_solve_state(const char *ws, const WsLayout &L, SolveState *out) {
    DH_CUDA_TRY(cudaMemcpy(out, ws + L.state, sizeof(SolveState), cudaMemcpyDeviceToHost));
    return DH_OK;
}

}  // namespace dh
