// Dark-channel-prior front end (Sec. II-D, Sec. II-A): dark channel, the
// atmospheric light A, and the fused t / lambda(t) / Phi / ||Phi||^2 pass.
#include "common.cuh"

namespace dh {

constexpr int kDcTile = 32;      // output tile side of the dark-channel kernels
constexpr int kDcThreads = 256;

int dcp_blocks(int H, int W) {
    return ((W + kDcTile - 1) / kDcTile) * ((H + kDcTile - 1) / kDcTile);
}

struct TransArgs {
    const float *A;        // device float[3] or nullptr (A = 1)
    float *td, *t, *lam, *phi, *u0;  // optional outputs (nullptr = skip)
    float2 *phin_part;     // per-block ||Phi^c||^2 partials or nullptr
    float omega, t0, lambda0, beta;
    int variant;
};

// Dark channel of a 32x32 tile (window clipped at the border: outside pixels
// are +inf and never win the minimum).  With FUSE, the epilogue evaluates
// t, lambda, Phi (and u0 = Phi) for the tile's pixels and the block's
// compensated ||Phi^c||^2.
template <bool NORM, bool FUSE>
__global__ void __launch_bounds__(kDcThreads)
k_dark_channel(const float *__restrict__ I, int H, int W, int r, float *__restrict__ out,
               TransArgs ta) {
    extern __shared__ float sm[];
    const int S = kDcTile + 2 * r;
    float *m = sm;                 // S x S channel minimum
    float *hm = sm + S * S;        // S x 32 horizontal minimum
    const int x0 = blockIdx.x * kDcTile, y0 = blockIdx.y * kDcTile;
    const size_t N = (size_t)H * W;
    float a0 = 1.f, a1 = 1.f, a2 = 1.f;
    if (NORM) { a0 = ta.A[0]; a1 = ta.A[1]; a2 = ta.A[2]; }
    for (int e = threadIdx.x; e < S * S; e += kDcThreads) {
        const int rr = e / S, cc = e - rr * S;
        const int gy = y0 - r + rr, gx = x0 - r + cc;
        float v = __int_as_float(0x7f800000);  // +inf
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const size_t o = (size_t)gy * W + gx;
            float q0 = I[o], q1 = I[N + o], q2 = I[2 * N + o];
            if (NORM) {  // IEEE float32 quotients (Sec. II-D, I^c / A^c)
                q0 = __fdiv_rn(q0, a0);
                q1 = __fdiv_rn(q1, a1);
                q2 = __fdiv_rn(q2, a2);
            }
            v = fminf(fminf(q0, q1), q2);
        }
        m[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < S * kDcTile; e += kDcThreads) {
        const int rr = e / kDcTile, cc = e - rr * kDcTile;
        const float *row = m + rr * S + cc;
        float v = row[0];
        for (int d = 1; d <= 2 * r; ++d) v = fminf(v, row[d]);
        hm[e] = v;
    }
    __syncthreads();
    float ps[3] = {0.f, 0.f, 0.f}, pc[3] = {0.f, 0.f, 0.f};
    for (int e = threadIdx.x; e < kDcTile * kDcTile; e += kDcThreads) {
        const int rr = e / kDcTile, cc = e - rr * kDcTile;
        const int gy = y0 + rr, gx = x0 + cc;
        if (gy >= H || gx >= W) continue;
        float v = hm[rr * kDcTile + cc];
        for (int d = 1; d <= 2 * r; ++d) v = fminf(v, hm[(rr + d) * kDcTile + cc]);
        const size_t o = (size_t)gy * W + gx;
        if (!FUSE) {
            out[o] = v;
            continue;
        }
        if (ta.td) ta.td[o] = v;
        // Sec. II-D: t = 1 - omega t_d; lambda(t) = lambda0 exp(-beta (1 - t))
        const float tt = 1.f - ta.omega * v;
        float lam = ta.lambda0 * expf(-ta.beta * (1.f - tt));
        if (ta.variant & DH_VAR_NO_ADAPTIVE) lam = ta.lambda0;
        if (ta.variant & DH_VAR_NO_NONLOCAL) lam = 0.f;
        if (ta.t) ta.t[o] = tt;
        if (ta.lam) ta.lam[o] = lam;
        // Sec. II-A: Phi = (I - A (1 - t)) / max(t, t0)
        const float den = fmaxf(tt, ta.t0);
        const float one_t = 1.f - tt;
        const float av[3] = {a0, a1, a2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float ph = __fdiv_rn(I[c * N + o] - av[c] * one_t, den);
            if (ta.phi) ta.phi[c * N + o] = ph;
            if (ta.u0) ta.u0[c * N + o] = ph;
            neumaier_add(ps[c], pc[c], ph * ph);
        }
    }
    if (!FUSE || !ta.phin_part) return;
    // block-wide compensated ||Phi^c||^2 in a fixed order
    __shared__ float2 red[3][kDcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, ps[c], off);
            const float c2 = __shfl_down_sync(0xffffffffu, pc[c], off);
            neumaier_merge(ps[c], pc[c], s2, c2);
        }
        if (lane == 0) red[c][w] = make_float2(ps[c], pc[c]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        float s = red[c][0].x, cc = red[c][0].y;
        for (int i = 1; i < kDcThreads / 32; ++i) neumaier_merge(s, cc, red[c][i].x, red[c][i].y);
        ta.phin_part[c * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] =
            make_float2(s, cc);
    }
}

// ||Phi^c||^2 partials of a caller-supplied Phi, same tiling (and so the
// same sums) as the fused transmission pass.
__global__ void __launch_bounds__(kDcThreads)
k_phin_partials(const float *__restrict__ phi, int H, int W, float2 *part) {
    const int x0 = blockIdx.x * kDcTile, y0 = blockIdx.y * kDcTile;
    const size_t N = (size_t)H * W;
    float ps[3] = {0.f, 0.f, 0.f}, pc[3] = {0.f, 0.f, 0.f};
    for (int e = threadIdx.x; e < kDcTile * kDcTile; e += kDcThreads) {
        const int rr = e / kDcTile, cc = e - rr * kDcTile;
        const int gy = y0 + rr, gx = x0 + cc;
        if (gy >= H || gx >= W) continue;
        const size_t o = (size_t)gy * W + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float ph = phi[c * N + o];
            neumaier_add(ps[c], pc[c], ph * ph);
        }
    }
    __shared__ float2 red[3][kDcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, ps[c], off);
            const float c2 = __shfl_down_sync(0xffffffffu, pc[c], off);
            neumaier_merge(ps[c], pc[c], s2, c2);
        }
        if (lane == 0) red[c][w] = make_float2(ps[c], pc[c]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        float s = red[c][0].x, cc = red[c][0].y;
        for (int i = 1; i < kDcThreads / 32; ++i) neumaier_merge(s, cc, red[c][i].x, red[c][i].y);
        part[c * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = make_float2(s, cc);
    }
}

// One warp per channel reduces the partials in block order into st->phin2.
__global__ void k_phin_final(const float2 *__restrict__ part, int nblk, SolveState *st) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= 3) return;
    float s = 0.f, cc = 0.f;
    for (int b = lane; b < nblk; b += 32) {
        const float2 p = part[c * nblk + b];
        neumaier_merge(s, cc, p.x, p.y);
    }
    for (int off = 16; off; off >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, off);
        const float c2 = __shfl_down_sync(0xffffffffu, cc, off);
        neumaier_merge(s, cc, s2, c2);
    }
    if (lane == 0) st->phin2[c] = s + cc;
}

// ------------------------------------------------------------ atmospheric light
// k-th largest dark-channel key by a 4-pass MSB radix select (8-bit digits),
// then the lowest-index equal keys, then the brightest selected pixel.

__global__ void k_sel_init(SelectState *sel, unsigned *hist, unsigned k) {
    const int t = threadIdx.x;
    if (t < 256) hist[t] = 0;
    if (t == 0) {
        sel->prefix = 0;
        sel->krem = k;
        sel->key = 0;
        sel->take = 0;
        sel->cutoff = -1;
        sel->best = -1;
        sel->clamped = 0;
        sel->best_sum = 0.0;
    }
}

__global__ void __launch_bounds__(256)
k_sel_hist(const float *__restrict__ dc, int N, const SelectState *sel, unsigned *hist, int pass) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned prefix = sel->prefix;
    const int shift = 24 - 8 * pass;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < N; i += gridDim.x * 256) {
        const unsigned k = float_key(dc[i]);
        if (pass == 0 || (k >> (shift + 8)) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_sel_digit(SelectState *sel, unsigned *hist, int pass) {
    __shared__ unsigned sc[256];
    const int t = threadIdx.x;
    const unsigned v = hist[255 - t];  // descending digits
    sc[t] = v;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {  // inclusive scan
        const unsigned a = t >= off ? sc[t - off] : 0u;
        __syncthreads();
        sc[t] += a;
        __syncthreads();
    }
    const unsigned krem = sel->krem;
    const unsigned incl = sc[t], excl = incl - v;
    __syncthreads();
    if (v > 0 && excl < krem && krem <= incl) {
        const unsigned d = 255u - t;
        sel->prefix = (sel->prefix << 8) | d;
        sel->krem = krem - excl;
        if (pass == 3) {
            sel->key = (sel->prefix);
            sel->take = krem - excl;
        }
    }
    __syncthreads();
    hist[t] = 0;
}

__global__ void __launch_bounds__(256)
k_sel_eqcount(const float *__restrict__ dc, int N, const SelectState *sel, unsigned *cnt) {
    const int chunk = (N + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
    const unsigned key = sel->key;
    unsigned c = 0;
    for (int i = lo + threadIdx.x; i < hi; i += 256) c += float_key(dc[i]) == key;
    for (int off = 16; off; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    __shared__ unsigned ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned s = 0;
        for (int i = 0; i < 8; ++i) s += ws[i];
        cnt[blockIdx.x] = s;
    }
}

// Finds the index of the take-th key equal to sel->key in index order.
__global__ void __launch_bounds__(256)
k_sel_cutoff(const float *__restrict__ dc, int N, SelectState *sel, const unsigned *cnt, int nchunks) {
    __shared__ int s_chunk;
    __shared__ unsigned s_before;
    __shared__ unsigned sc[256];
    const int t = threadIdx.x;
    const unsigned take = sel->take;
    if (t == 0) {  // serial walk over the chunk counts: nchunks is small
        unsigned acc = 0;
        int ch = nchunks - 1;
        for (int b = 0; b < nchunks; ++b) {
            if (acc + cnt[b] >= take) { ch = b; break; }
            acc += cnt[b];
        }
        s_chunk = ch;
        s_before = acc;
    }
    __syncthreads();
    const int chunk = (N + nchunks - 1) / nchunks;
    const int lo = s_chunk * chunk, hi = min(N, lo + chunk);
    const unsigned key = sel->key;
    unsigned before = s_before;
    for (int base = lo; base < hi; base += 256) {
        const int i = base + t;
        const unsigned e = (i < hi && float_key(dc[i]) == key) ? 1u : 0u;
        sc[t] = e;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            const unsigned a = t >= off ? sc[t - off] : 0u;
            __syncthreads();
            sc[t] += a;
            __syncthreads();
        }
        const unsigned incl = sc[t] + before;
        if (e && incl == take) sel->cutoff = i;
        const unsigned tot = sc[255];
        __syncthreads();
        before += tot;
        if (before >= take) break;
    }
}

struct BestPix {
    double sum;
    int idx;
    int pad;
};

__device__ __forceinline__ bool better(double s1, int i1, double s2, int i2) {
    return s1 > s2 || (s1 == s2 && i1 < i2);
}

__global__ void __launch_bounds__(256)
k_sel_argmax(const float *__restrict__ I, const float *__restrict__ dc, int N, const SelectState *sel,
             BestPix *blk) {
    const unsigned key = sel->key;
    const int cutoff = sel->cutoff;
    double bs = -1.0;
    int bi = -1;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < N; i += gridDim.x * 256) {
        const unsigned k = float_key(dc[i]);
        if (k > key || (k == key && i <= cutoff)) {
            const double s = ((double)I[i] + (double)I[(size_t)N + i]) + (double)I[2 * (size_t)N + i];
            if (bi < 0 || better(s, i, bs, bi)) { bs = s; bi = i; }
        }
    }
    for (int off = 16; off; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, bs, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (i2 >= 0 && (bi < 0 || better(s2, i2, bs, bi))) { bs = s2; bi = i2; }
    }
    __shared__ double wsum[8];
    __shared__ int widx[8];
    if ((threadIdx.x & 31) == 0) { wsum[threadIdx.x >> 5] = bs; widx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w)
            if (widx[w] >= 0 && (bi < 0 || better(wsum[w], widx[w], bs, bi))) { bs = wsum[w]; bi = widx[w]; }
        blk[blockIdx.x].sum = bs;
        blk[blockIdx.x].idx = bi;
    }
}

__global__ void __launch_bounds__(256)
k_sel_final(const float *__restrict__ I, int N, SelectState *sel, const BestPix *blk, int nblk,
            float *A, long long *index_out) {
    double bs = -1.0;
    int bi = -1;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        const BestPix p = blk[b];
        if (p.idx >= 0 && (bi < 0 || better(p.sum, p.idx, bs, bi))) { bs = p.sum; bi = p.idx; }
    }
    for (int off = 16; off; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, bs, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (i2 >= 0 && (bi < 0 || better(s2, i2, bs, bi))) { bs = s2; bi = i2; }
    }
    __shared__ double wsum[8];
    __shared__ int widx[8];
    if ((threadIdx.x & 31) == 0) { wsum[threadIdx.x >> 5] = bs; widx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w)
            if (widx[w] >= 0 && (bi < 0 || better(wsum[w], widx[w], bs, bi))) { bs = wsum[w]; bi = widx[w]; }
        if (bi < 0) bi = 0;  // unreachable for N >= 1
        int clamped = 0;
        for (int c = 0; c < 3; ++c) {
            float a = I[(size_t)c * N + bi];
            if (!(a > 0.f)) { a = 1e-6f; clamped = 1; }
            A[c] = a;
        }
        sel->best = bi;
        sel->best_sum = bs;
        sel->clamped = clamped;
        if (index_out) *index_out = bi;
    }
}

// ------------------------------------------------------------ host launchers

int launch_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out,
                        cudaStream_t s) {
    const int r = patch / 2;
    const int S = kDcTile + 2 * r;
    const size_t smem = (size_t)(S * S + S * kDcTile) * sizeof(float);
    dim3 grid((W + kDcTile - 1) / kDcTile, (H + kDcTile - 1) / kDcTile);
    TransArgs ta{};
    ta.A = A;
    if (A)
        k_dark_channel<true, false><<<grid, kDcThreads, smem, s>>>(I, H, W, r, out, ta);
    else
        k_dark_channel<false, false><<<grid, kDcThreads, smem, s>>>(I, H, W, r, out, ta);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

// ------------------------------------------------------------ front-end refinements
// The Sec. IV-E ablation removes a "multiscale dark channel" and a "guided
// filter" that the method section never defines.  Readings built here:
// t_d = mean of the normalised dark channels at patch sizes patch/2 (odd),
// patch and 2*patch+1; t = 1 - omega t_d refined by the guided filter of He,
// Sun and Tang with the gray guide g = ((I^R + I^G) + I^B)/3 and windows
// clipped to the image.  Window sums run in FP64 (the oracle's precision), so
// the refined t is the FP64 value rounded once to float32.

constexpr int kGfTile = 32;
constexpr int kGfMaxR = 24;

size_t refine_bytes(int H, int W, const dh_params *p) {
    if (!p || (p->dc_scales <= 1 && p->gf_radius <= 0)) return 0;
    const size_t N = (size_t)H * W;
    // dark channels per scale (float), t0 (double), a and b (double), refined t (float)
    return align_up(3 * N * sizeof(float)) + align_up(N * sizeof(double)) + 2 * align_up(N * sizeof(double)) +
           align_up(N * sizeof(float)) + kAlign;
}

// t0 = 1 - omega * mean_s(td_s) in double; td_out = the mean (float), t_out = (float) t0
__global__ void k_refine_t0(const float *__restrict__ tds, int S, size_t N, float omega, double *__restrict__ t0,
                            float *__restrict__ td_out, float *__restrict__ t_out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        double m = tds[i];
        for (int k = 1; k < S; ++k) m += (double)tds[k * N + i];
        m /= (double)S;
        const double t = 1.0 - (double)omega * m;
        t0[i] = t;
        if (td_out) td_out[i] = (float)m;
        if (t_out) t_out[i] = (float)t;
    }
}

__device__ __forceinline__ double gray_of(const float *__restrict__ I, size_t N, size_t o) {
    return (((double)I[o] + (double)I[N + o]) + (double)I[2 * N + o]) / 3.0;
}

// Window means of NQ quantities over a 32x32 output tile.  The NI inputs of
// the (32+2r)^2 region are staged in shared memory (q[NI][S*S]); the
// horizontal pass forms the NQ quantities from them (derive) and sums them
// along rows (h[NQ][S*32]); the vertical pass finishes the (2r+1)^2 sums and
// divides by the number of window pixels inside the image.
template <int NI, int NQ, class FILL, class DERIVE, class OUT>
__device__ void gf_window_means(int H, int W, int r, double *smem, FILL fill, DERIVE derive, OUT out) {
    const int S = kGfTile + 2 * r;
    double *q = smem;                // NI x S x S
    double *h = smem + NI * S * S;   // NQ x S x 32
    const int x0 = blockIdx.x * kGfTile, y0 = blockIdx.y * kGfTile;
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        const int rr = e / S, cc = e - rr * S;
        const int gy = y0 - r + rr, gx = x0 - r + cc;
        double v[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) v[k] = 0.0;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) fill(gy, gx, v);
#pragma unroll
        for (int k = 0; k < NI; ++k) q[k * S * S + e] = v[k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < S * kGfTile; e += blockDim.x) {
        const int rr = e / kGfTile, cc = e - rr * kGfTile;
        double acc[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) acc[k] = 0.0;
        for (int d = 0; d <= 2 * r; ++d) {
            double in[NI], dq[NQ];
#pragma unroll
            for (int k = 0; k < NI; ++k) in[k] = q[k * S * S + rr * S + cc + d];
            derive(in, dq);
#pragma unroll
            for (int k = 0; k < NQ; ++k) acc[k] += dq[k];
        }
#pragma unroll
        for (int k = 0; k < NQ; ++k) h[k * S * kGfTile + e] = acc[k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kGfTile * kGfTile; e += blockDim.x) {
        const int rr = e / kGfTile, cc = e - rr * kGfTile;
        const int gy = y0 + rr, gx = x0 + cc;
        if (gy >= H || gx >= W) continue;
        const int nx = min(gx + r, W - 1) - max(gx - r, 0) + 1, ny = min(gy + r, H - 1) - max(gy - r, 0) + 1;
        const double inv = 1.0 / (double)(nx * ny);
        double m[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            double a = 0.0;
            for (int d = 0; d <= 2 * r; ++d) a += h[k * S * kGfTile + (rr + d) * kGfTile + cc];
            m[k] = a * inv;
        }
        out(gy, gx, m);
    }
}

// a = cov(g, t0) / (var(g) + eps), b = mean(t0) - a mean(g)
__global__ void __launch_bounds__(256) k_gf_stats(const float *__restrict__ I, const double *__restrict__ t0, int H,
                                                  int W, int r, double eps, double *__restrict__ a,
                                                  double *__restrict__ b) {
    extern __shared__ double gsm[];
    const size_t N = (size_t)H * W;
    gf_window_means<2, 4>(
        H, W, r, gsm,
        [&](int gy, int gx, double *v) {
            const size_t o = (size_t)gy * W + gx;
            v[0] = gray_of(I, N, o);
            v[1] = t0[o];
        },
        [](const double *in, double *dq) {
            dq[0] = in[0];
            dq[1] = in[1];
            dq[2] = in[0] * in[1];
            dq[3] = in[0] * in[0];
        },
        [&](int gy, int gx, const double *m) {
            const size_t o = (size_t)gy * W + gx;
            const double av = (m[2] - m[0] * m[1]) / (m[3] - m[0] * m[0] + eps);
            a[o] = av;
            b[o] = m[1] - av * m[0];
        });
}

// refined t = mean(a) g + mean(b)
__global__ void __launch_bounds__(256) k_gf_apply(const float *__restrict__ I, const double *__restrict__ a,
                                                  const double *__restrict__ b, int H, int W, int r,
                                                  float *__restrict__ t_out) {
    extern __shared__ double gsm[];
    const size_t N = (size_t)H * W;
    gf_window_means<2, 2>(
        H, W, r, gsm,
        [&](int gy, int gx, double *v) {
            const size_t o = (size_t)gy * W + gx;
            v[0] = a[o];
            v[1] = b[o];
        },
        [](const double *in, double *dq) {
            dq[0] = in[0];
            dq[1] = in[1];
        },
        [&](int gy, int gx, const double *m) {
            const size_t o = (size_t)gy * W + gx;
            t_out[o] = (float)(m[0] * gray_of(I, N, o) + m[1]);
        });
}

// lambda, Phi, u0 and the ||Phi^c||^2 partials from a given t (the same
// arithmetic, tiling and reduction as the fused dark-channel epilogue).
__global__ void __launch_bounds__(kDcThreads)
k_trans_from_t(const float *__restrict__ I, const float *__restrict__ tin, int H, int W, TransArgs ta) {
    const int x0 = blockIdx.x * kDcTile, y0 = blockIdx.y * kDcTile;
    const size_t N = (size_t)H * W;
    const float a0 = ta.A[0], a1 = ta.A[1], a2 = ta.A[2];
    float ps[3] = {0.f, 0.f, 0.f}, pc[3] = {0.f, 0.f, 0.f};
    for (int e = threadIdx.x; e < kDcTile * kDcTile; e += kDcThreads) {
        const int rr = e / kDcTile, cc = e - rr * kDcTile;
        const int gy = y0 + rr, gx = x0 + cc;
        if (gy >= H || gx >= W) continue;
        const size_t o = (size_t)gy * W + gx;
        const float tt = tin[o];
        float lam = ta.lambda0 * expf(-ta.beta * (1.f - tt));
        if (ta.variant & DH_VAR_NO_ADAPTIVE) lam = ta.lambda0;
        if (ta.variant & DH_VAR_NO_NONLOCAL) lam = 0.f;
        if (ta.t) ta.t[o] = tt;
        if (ta.lam) ta.lam[o] = lam;
        const float den = fmaxf(tt, ta.t0);
        const float one_t = 1.f - tt;
        const float av[3] = {a0, a1, a2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float ph = __fdiv_rn(I[c * N + o] - av[c] * one_t, den);
            if (ta.phi) ta.phi[c * N + o] = ph;
            if (ta.u0) ta.u0[c * N + o] = ph;
            neumaier_add(ps[c], pc[c], ph * ph);
        }
    }
    if (!ta.phin_part) return;
    __shared__ float2 red[3][kDcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, ps[c], off);
            const float c2 = __shfl_down_sync(0xffffffffu, pc[c], off);
            neumaier_merge(ps[c], pc[c], s2, c2);
        }
        if (lane == 0) red[c][w] = make_float2(ps[c], pc[c]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int c = threadIdx.x;
        float s = red[c][0].x, cc = red[c][0].y;
        for (int i = 1; i < kDcThreads / 32; ++i) neumaier_merge(s, cc, red[c][i].x, red[c][i].y);
        ta.phin_part[c * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = make_float2(s, cc);
    }
}

static size_t gf_smem(int r, int ni, int nq) {
    const size_t S = kGfTile + 2 * r;
    return (ni * S * S + nq * S * kGfTile) * sizeof(double);
}

int launch_transmission(const float *I, int H, int W, const dh_params *p, const float *A, float *td,
                        float *t, float *lam, float *phi, float *u0, float2 *phin_part, void *scratch,
                        cudaStream_t s) {
    if (p->dc_scales > 1 || p->gf_radius > 0) {
        if (!scratch || p->gf_radius > kGfMaxR) return DH_EINVAL;
        const size_t N = (size_t)H * W;
        char *sc = (char *)scratch;
        float *tds = (float *)sc; sc += align_up(3 * N * sizeof(float));
        double *t0 = (double *)sc; sc += align_up(N * sizeof(double));
        double *ga = (double *)sc; sc += align_up(N * sizeof(double));
        double *gb = (double *)sc; sc += align_up(N * sizeof(double));
        float *tref = (float *)sc;
        const int S = p->dc_scales > 1 ? 3 : 1;
        const int patches[3] = {S > 1 ? ((p->patch / 2) | 1) : p->patch, p->patch, 2 * p->patch + 1};
        for (int k = 0; k < S; ++k) {
            const int q = S > 1 ? patches[k] : p->patch;
            int rc = launch_dark_channel(I, H, W, q, A, tds + k * N, s);
            if (rc) return rc;
        }
        const int g1 = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
        k_refine_t0<<<g1, 256, 0, s>>>(tds, S, N, p->omega, t0, td, p->gf_radius > 0 ? nullptr : tref);
        if (p->gf_radius > 0) {
            const int r = p->gf_radius;
            const size_t sm4 = gf_smem(r, 2, 4), sm2 = gf_smem(r, 2, 2);
            DH_CUDA_TRY(cudaFuncSetAttribute(k_gf_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4));
            DH_CUDA_TRY(cudaFuncSetAttribute(k_gf_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
            dim3 gg((W + kGfTile - 1) / kGfTile, (H + kGfTile - 1) / kGfTile);
            k_gf_stats<<<gg, 256, sm4, s>>>(I, t0, H, W, r, (double)p->gf_eps, ga, gb);
            k_gf_apply<<<gg, 256, sm2, s>>>(I, ga, gb, H, W, r, tref);
        }
        TransArgs ta{};
        ta.A = A;
        ta.t = t;
        ta.lam = lam;
        ta.phi = phi;
        ta.u0 = u0;
        ta.phin_part = phin_part;
        ta.omega = p->omega;
        ta.t0 = p->t0;
        ta.lambda0 = p->lambda0;
        ta.beta = p->beta;
        ta.variant = p->variant;
        dim3 grid((W + kDcTile - 1) / kDcTile, (H + kDcTile - 1) / kDcTile);
        k_trans_from_t<<<grid, kDcThreads, 0, s>>>(I, tref, H, W, ta);
        DH_CUDA_TRY(cudaGetLastError());
        return DH_OK;
    }
    const int r = p->patch / 2;
    const int S = kDcTile + 2 * r;
    const size_t smem = (size_t)(S * S + S * kDcTile) * sizeof(float);
    dim3 grid((W + kDcTile - 1) / kDcTile, (H + kDcTile - 1) / kDcTile);
    TransArgs ta{};
    ta.A = A;
    ta.td = td;
    ta.t = t;
    ta.lam = lam;
    ta.phi = phi;
    ta.u0 = u0;
    ta.phin_part = phin_part;
    ta.omega = p->omega;
    ta.t0 = p->t0;
    ta.lambda0 = p->lambda0;
    ta.beta = p->beta;
    ta.variant = p->variant;
    k_dark_channel<true, true><<<grid, kDcThreads, smem, s>>>(I, H, W, r, nullptr, ta);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int launch_phin(const float *phi, int H, int W, float2 *part, SolveState *st, cudaStream_t s) {
    dim3 grid((W + kDcTile - 1) / kDcTile, (H + kDcTile - 1) / kDcTile);
    k_phin_partials<<<grid, kDcThreads, 0, s>>>(phi, H, W, part);
    k_phin_final<<<1, 96, 0, s>>>(part, (int)(grid.x * grid.y), st);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int launch_phin_final(const float2 *part, int H, int W, SolveState *st, cudaStream_t s) {
    k_phin_final<<<1, 96, 0, s>>>(part, dcp_blocks(H, W), st);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int launch_select_A(const float *I, const float *dc, int H, int W, int permille, float *A,
                    long long *index_out, char *ws, const WsLayout &L, cudaStream_t s) {
    const int N = H * W;
    long long k = (long long)N * permille / 1000;
    if (k < 1) k = 1;
    if (k > N) k = N;
    SelectState *sel = (SelectState *)(ws + L.sel);
    unsigned *hist = (unsigned *)(ws + L.hist);
    const int nb = min(kSelBlocks, (N + 255) / 256);
    k_sel_init<<<1, 256, 0, s>>>(sel, hist, (unsigned)k);
    for (int pass = 0; pass < 4; ++pass) {
        k_sel_hist<<<nb, 256, 0, s>>>(dc, N, sel, hist, pass);
        k_sel_digit<<<1, 256, 0, s>>>(sel, hist, pass);
    }
    unsigned *cnt = (unsigned *)(ws + L.blk);
    k_sel_eqcount<<<nb, 256, 0, s>>>(dc, N, sel, cnt);
    k_sel_cutoff<<<1, 256, 0, s>>>(dc, N, sel, cnt, nb);
    BestPix *bp = (BestPix *)(ws + L.blk);
    k_sel_argmax<<<nb, 256, 0, s>>>(I, dc, N, sel, bp);
    k_sel_final<<<1, 256, 0, s>>>(I, N, sel, bp, nb, A, index_out);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

}  // namespace dh
