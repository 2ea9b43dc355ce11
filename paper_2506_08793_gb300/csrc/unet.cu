// Learned warm start for the fixed-point solver: a 4-level U-Net (base 32
// channels, 3x3 convolutions, ReLU, 2x2 average pooling, nearest 2x
// upsampling, skip concatenation, 1x1 head) over (I, t, A) and the data term
// Phi that predicts y = lambda * u* as Phi plus a learned correction, so that
// u0 = y / lambda starts the iteration of App. A-A near its fixed point
// (y = Phi, i.e. u0 = Phi / lambda, is the fixed point without diffusion and
// with G = identity).  The paper only points at such hybrids (Sec. I, V);
// the network, its training and the warm start are this library's.
//
// Activations and their gradients are bf16, channels-last (NHWC) with a
// channel pitch so that skip concatenations are views; convolutions are
// implicit GEMMs on the tensor cores (mma.sync m16n8k16 bf16, fp32
// accumulate); parameters, the loss and Adam are fp32.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace dh {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ tensor-core helpers

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t *r, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t *r, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr(p)));
}
// D = A (16x16, row) * B (16x8, col) + D, bf16 inputs, fp32 accumulators
__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------ 3x3 convolution, forward
// y[p][co] = bias[co] + sum_{tap, ci} x[p + tap][ci] * w[co][tap][ci], zero
// padding, optional ReLU.  M = N*H*W pixels, N = Cout, K = 9*C.  The same
// kernel computes the data gradient (x = dy, w = flipped / transposed w).
constexpr int kCBM = 128, kCBN = 64;

template <int BK>
__global__ void __launch_bounds__(128)
k_conv3x3(const bf16 *__restrict__ x, int ldx, int C, int Nimg, int H, int W, const bf16 *__restrict__ w,
          const float *__restrict__ bias, int Cout, int relu, bf16 *__restrict__ y, int ldy) {
    __shared__ __align__(16) bf16 As[kCBM][BK + 8];
    __shared__ __align__(16) bf16 Bs[kCBN][BK + 8];
    const int M = Nimg * H * W;
    const int m0 = blockIdx.x * kCBM, n0 = blockIdx.y * kCBN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 64, wn = (warp & 1) * 32;
    constexpr int VPR = BK / 8;              // 16-byte vectors per row
    constexpr int AV = kCBM * VPR / 128;     // A vectors per thread
    constexpr int BV = (kCBN * VPR + 127) / 128;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    int ar[AV], av[AV], an[AV], ay[AV], ax[AV];
#pragma unroll
    for (int i = 0; i < AV; ++i) {
        const int idx = tid + i * 128;
        ar[i] = idx / VPR;
        av[i] = idx % VPR;
        const int p = m0 + ar[i];
        an[i] = p < M ? p / (H * W) : -1;
        const int rem = p - (p / (H * W)) * (H * W);
        ay[i] = rem / W;
        ax[i] = rem - (rem / W) * W;
    }
    const int KC = C / BK;
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        for (int kc = 0; kc < KC; ++kc) {
            const int c0 = kc * BK;
#pragma unroll
            for (int i = 0; i < AV; ++i) {
                const int yy = ay[i] + dy, xx = ax[i] + dx;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (an[i] >= 0 && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v = *reinterpret_cast<const uint4 *>(x + ((size_t)(an[i] * H + yy) * W + xx) * ldx + c0 + av[i] * 8);
                *reinterpret_cast<uint4 *>(&As[ar[i]][av[i] * 8]) = v;
            }
#pragma unroll
            for (int j = 0; j < BV; ++j) {
                const int idx = tid + j * 128;
                if (idx < kCBN * VPR) {
                    const int nr = idx / VPR, v8 = idx % VPR, co = n0 + nr;
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (co < Cout) v = *reinterpret_cast<const uint4 *>(w + ((size_t)co * 9 + tap) * C + c0 + v8 * 8);
                    *reinterpret_cast<uint4 *>(&Bs[nr][v8 * 8]) = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                uint32_t a[4][4], b[2][4];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
                    ldsm_x4(a[mt], &As[wm + mt * 16 + (lane & 15)][ks * 16 + (lane >> 4) * 8]);
#pragma unroll
                for (int np = 0; np < 2; ++np)
                    ldsm_x4(b[np], &Bs[wn + np * 16 + (lane & 7) + (lane >> 4) * 8][ks * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma_bf16(acc[mt][nt], a[mt], b[nt >> 1][(nt & 1) * 2], b[nt >> 1][(nt & 1) * 2 + 1]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = n0 + wn + nt * 8 + (lane & 3) * 2;
            if (col >= Cout) continue;
            const float b0 = bias ? bias[col] : 0.f, b1 = bias ? bias[col + 1] : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm + mt * 16 + (lane >> 2) + h * 8;
                if (row >= M) continue;
                float v0 = acc[mt][nt][2 * h] + b0, v1 = acc[mt][nt][2 * h + 1] + b1;
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162 *>(y + (size_t)row * ldy + col) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

// ------------------------------------------------------------ 3x3 convolution, weight gradient
// dw[co][tap][ci] = sum_p dy[p][co] * x[p + tap][ci]; each CTA sums one
// pixel split for a 64 (co) x 64 (ci) block of one tap into `part`.
constexpr int kWBK = 32;  // pixels per step

__global__ void __launch_bounds__(128)
k_conv3x3_wgrad(const bf16 *__restrict__ x, int ldx, int C, const bf16 *__restrict__ dy, int lddy, int Cout,
                int Nimg, int H, int W, int split_px, float *__restrict__ part) {
    __shared__ __align__(16) bf16 Ds[kWBK][64 + 8];
    __shared__ __align__(16) bf16 Xs[kWBK][64 + 8];
    const int M = Nimg * H * W;
    const int co0 = blockIdx.x * 64;
    const int nci = (C + 63) / 64;
    const int tap = blockIdx.y / nci, ci0 = (blockIdx.y % nci) * 64;
    const int split = blockIdx.z;
    const int dy_ = tap / 3 - 1, dx_ = tap % 3 - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    const int p_begin = split * split_px, p_end = min(M, p_begin + split_px);
    for (int pb = p_begin; pb < p_end; pb += kWBK) {
        // 32 pixels x 64 channels of dy and of x shifted by the tap: 256 vectors each
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int idx = tid + j * 128;
            const int r = idx >> 3, v8 = idx & 7;
            const int p = pb + r;
            uint4 dv = make_uint4(0, 0, 0, 0), xv = make_uint4(0, 0, 0, 0);
            if (p < p_end) {
                if (co0 + v8 * 8 < Cout) dv = *reinterpret_cast<const uint4 *>(dy + (size_t)p * lddy + co0 + v8 * 8);
                const int n = p / (H * W), rem = p - n * (H * W);
                const int yy = rem / W + dy_, xx = rem % W + dx_;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W && ci0 + v8 * 8 < C)
                    xv = *reinterpret_cast<const uint4 *>(x + ((size_t)(n * H + yy) * W + xx) * ldx + ci0 + v8 * 8);
            }
            *reinterpret_cast<uint4 *>(&Ds[r][v8 * 8]) = dv;
            *reinterpret_cast<uint4 *>(&Xs[r][v8 * 8]) = xv;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kWBK / 16; ++ks) {
            uint32_t a[2][4], b[2][4];
            // A[m = co][k = p] = Ds[p][co]: transposed 8x8 loads
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm_x4_t(a[mt], &Ds[ks * 16 + (lane & 7) + (lane >> 4) * 8][wm + mt * 16 + ((lane >> 3) & 1) * 8]);
            // B[k = p][n = ci] = Xs[p][ci]
#pragma unroll
            for (int np = 0; np < 2; ++np)
                ldsm_x4_t(b[np], &Xs[ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8][wn + np * 16 + (lane >> 4) * 8]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16(acc[mt][nt], a[mt], b[nt >> 1][(nt & 1) * 2], b[nt >> 1][(nt & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    // part[split][co][tap][ci]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = co0 + wm + mt * 16 + (lane >> 2) + h * 8;
                const int ci = ci0 + wn + nt * 8 + (lane & 3) * 2;
                if (co >= Cout || ci >= C) continue;
                float *dst = part + (((size_t)split * Cout + co) * 9 + tap) * C + ci;
                dst[0] = acc[mt][nt][2 * h];
                dst[1] = acc[mt][nt][2 * h + 1];
            }
}

// out[i] (+)= sum_s part[s][i], splits summed in order
__global__ void k_sum_splits(const float *__restrict__ part, int splits, size_t n, float *__restrict__ out, int accumulate) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
        out[i] = accumulate ? out[i] + s : s;
    }
}

// db[co] partial sums over pixel splits: part[split][co].  256 threads:
// channel tid % Cout, pixel lane tid / Cout; lanes are summed in order.
__global__ void __launch_bounds__(256)
k_bias_grad(const bf16 *__restrict__ dy, int lddy, int Cout, int M, int split_px, float *part) {
    __shared__ float red[256];
    const int split = blockIdx.x;
    const int p0 = split * split_px, p1 = min(M, p0 + split_px);
    const int lanes = 256 / Cout;  // Cout divides 256
    const int c = threadIdx.x % Cout, l = threadIdx.x / Cout;
    float s = 0.f;
    if (l < lanes)
        for (int p = p0 + l; p < p1; p += lanes) s += __bfloat162float(dy[(size_t)p * lddy + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < Cout) {
        float t = 0.f;
        for (int k = 0; k < lanes; ++k) t += red[k * Cout + threadIdx.x];
        part[(size_t)split * Cout + threadIdx.x] = t;
    }
}

// ------------------------------------------------------------ elementwise layers
// Every activation of the network is bf16 NHWC with channel counts, pitches
// and channel offsets that are multiples of 8 (16 bytes) and H, W multiples of
// 8 with N*H*W <= 2^26 (unet_shape_ok): a thread moves 8 channels as one 16-byte
// vector and the unit indices fit in 32 bits.  Per element the arithmetic (and
// its order) is that of the plain definitions.

__device__ __forceinline__ uint4 ld8(const bf16 *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ void st8(bf16 *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }
__device__ __forceinline__ void unpack8(uint4 v, float (&f)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 v;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return v;
}
#define DH_GRID_STRIDE(u, n) for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < (n); u += gridDim.x * blockDim.x)

// ReLU backward: g = 0 where the layer's output y is not positive (M pixels x C)
__global__ void k_relu_bwd(bf16 *g, int ldg, const bf16 *__restrict__ y, int ldy, int C, int M) {
    const int G = C / 8;
    DH_GRID_STRIDE(u, M * G) {
        const int p = u / G, c = 8 * (u - p * G);
        bf16 *gp = g + (size_t)p * ldg + c;
        float gv[8], yv[8];
        unpack8(*reinterpret_cast<const uint4 *>(gp), gv);
        unpack8(ld8(y + (size_t)p * ldy + c), yv);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!(yv[j] > 0.f)) gv[j] = 0.f;
        st8(gp, pack8(gv));
    }
}

// 2x2 average pooling: out (H/2 x W/2) from in (H x W)
__global__ void k_avgpool(const bf16 *__restrict__ in, int ldi, int C, int Nimg, int H, int W, bf16 *out, int ldo) {
    const int Ho = H / 2, Wo = W / 2, G = C / 8;
    DH_GRID_STRIDE(u, Nimg * Ho * Wo * G) {
        const int q = u / G, c = 8 * (u - q * G);
        const int xo = q % Wo, r = q / Wo, yo = r % Ho, nn = r / Ho;
        const size_t b = (size_t)(nn * H + 2 * yo) * W + 2 * xo;
        float a[8], e[8], f[8], h[8], o[8];
        unpack8(ld8(in + b * ldi + c), a);
        unpack8(ld8(in + (b + 1) * ldi + c), e);
        unpack8(ld8(in + (b + W) * ldi + c), f);
        unpack8(ld8(in + (b + W + 1) * ldi + c), h);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = 0.25f * (a[j] + e[j] + f[j] + h[j]);
        st8(out + (size_t)q * ldo + c, pack8(o));
    }
}

// d_in (H x W) += d_out (H/2 x W/2) / 4 at each of the four positions
__global__ void k_avgpool_bwd_add(const bf16 *__restrict__ gout, int ldo, int C, int Nimg, int H, int W, bf16 *gin, int ldi) {
    const int G = C / 8;
    DH_GRID_STRIDE(u, Nimg * H * W * G) {
        const int p = u / G, c = 8 * (u - p * G);
        const int xx = p % W, r = p / W, yy = r % H, nn = r / H;
        const size_t q = (size_t)(nn * (H / 2) + yy / 2) * (W / 2) + xx / 2;
        bf16 *gp = gin + (size_t)p * ldi + c;
        float gi[8], go[8];
        unpack8(*reinterpret_cast<const uint4 *>(gp), gi);
        unpack8(ld8(gout + q * ldo + c), go);
#pragma unroll
        for (int j = 0; j < 8; ++j) gi[j] = gi[j] + 0.25f * go[j];
        st8(gp, pack8(gi));
    }
}

// nearest 2x upsampling: out (2H x 2W) from in (H x W); a thread reads one
// input vector and writes its 2x2 block
__global__ void k_upsample(const bf16 *__restrict__ in, int ldi, int C, int Nimg, int H, int W, bf16 *out, int ldo) {
    const int G = C / 8;
    DH_GRID_STRIDE(u, Nimg * H * W * G) {
        const int p = u / G, c = 8 * (u - p * G);
        const int xx = p % W, r = p / W, yy = r % H, nn = r / H;
        const uint4 v = ld8(in + (size_t)p * ldi + c);
        const size_t b = (size_t)(nn * 2 * H + 2 * yy) * (2 * W) + 2 * xx;
        st8(out + b * ldo + c, v);
        st8(out + (b + 1) * ldo + c, v);
        st8(out + (b + 2 * W) * ldo + c, v);
        st8(out + (b + 2 * W + 1) * ldo + c, v);
    }
}

// d_in (H x W) = sum of the four d_out (2H x 2W) it was copied to
__global__ void k_upsample_bwd(const bf16 *__restrict__ gout, int ldo, int C, int Nimg, int H, int W, bf16 *gin, int ldi) {
    const int G = C / 8;
    DH_GRID_STRIDE(u, Nimg * H * W * G) {
        const int p = u / G, c = 8 * (u - p * G);
        const int xx = p % W, r = p / W, yy = r % H, nn = r / H;
        const size_t b = (size_t)(nn * 2 * H + 2 * yy) * (2 * W) + 2 * xx;
        float a[8], e[8], f[8], h[8], o[8];
        unpack8(ld8(gout + b * ldo + c), a);
        unpack8(ld8(gout + (b + 1) * ldo + c), e);
        unpack8(ld8(gout + (b + 2 * W) * ldo + c), f);
        unpack8(ld8(gout + (b + 2 * W + 1) * ldo + c), h);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = a[j] + e[j] + f[j] + h[j];
        st8(gin + (size_t)p * ldi + c, pack8(o));
    }
}

// network input: channels (I^R, I^G, I^B, t, A^R, A^G, A^B, Phi^R, Phi^G,
// Phi^B, 0 ...) padded to 16
__global__ void k_pack_input(const float *__restrict__ I, const float *__restrict__ t, const float *__restrict__ A,
                             const float *__restrict__ Phi, int Nimg, int H, int W, bf16 *x) {
    const int HW = H * W;
    DH_GRID_STRIDE(p, Nimg * HW) {
        const int nn = p / HW, q = p - nn * HW;
        const size_t o = (size_t)nn * 3 * HW + q;
        float v[16];
        for (int c = 0; c < 3; ++c) v[c] = __ldg(I + o + (size_t)c * HW);
        v[3] = __ldg(t + (size_t)nn * HW + q);
        for (int c = 0; c < 3; ++c) v[4 + c] = __ldg(A + nn * 3 + c);
        for (int c = 0; c < 3; ++c) v[7 + c] = __ldg(Phi + o + (size_t)c * HW);
        for (int c = 10; c < 16; ++c) v[c] = 0.f;
        float lo[8], hi[8];
        for (int c = 0; c < 8; ++c) {
            lo[c] = v[c];
            hi[c] = v[8 + c];
        }
        st8(x + (size_t)p * 16, pack8(lo));
        st8(x + (size_t)p * 16 + 8, pack8(hi));
    }
}

// 1x1 head on top of the analytic guess: y[n][o][q] = Phi[n][o][q] + hb[o] +
// sum_c hw[o][c] x[p][c] (fp32 out, planar)
__global__ void k_head(const bf16 *__restrict__ x, int ldx, int C, const float *__restrict__ hw, const float *__restrict__ hb,
                       const float *__restrict__ Phi, int Nimg, int H, int W, float *y) {
    const int HW = H * W;
    DH_GRID_STRIDE(p, Nimg * HW) {
        const int nn = p / HW, q = p - nn * HW;
        const size_t o = (size_t)nn * 3 * HW + q;
        float s[3] = {__ldg(hb) + __ldg(Phi + o), __ldg(hb + 1) + __ldg(Phi + o + HW), __ldg(hb + 2) + __ldg(Phi + o + 2 * (size_t)HW)};
        for (int c0 = 0; c0 < C; c0 += 8) {
            float v[8];
            unpack8(ld8(x + (size_t)p * ldx + c0), v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                for (int k = 0; k < 3; ++k) s[k] = fmaf(__ldg(hw + k * C + c0 + j), v[j], s[k]);
        }
        for (int k = 0; k < 3; ++k) y[o + (size_t)k * HW] = s[k];
    }
}

// MSE loss and its gradient: g = 2 (y - target) / count (fp32, planar);
// per-block partial sums of (y - target)^2 in part[block]
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ tgt, size_t n, float *g, float *part) {
    __shared__ float red[256];
    float s = 0.f;
    const float k = 2.f / (float)n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - tgt[i];
        s = fmaf(d, d, s);
        g[i] = k * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const float *part, int nb, size_t n, float *loss) {
    if (threadIdx.x) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[b];
    *loss = s / (float)n;
}

// head backward: gx[p][c] = sum_o g[n][o][q] hw[o][c] (bf16) and per-block
// partials of dhw[o][c] = sum_p g x and dhb[o] = sum_p g: part[block][3C+3]
template <int C>
__global__ void __launch_bounds__(256)
k_head_bwd(const bf16 *__restrict__ x, int ldx, const float *__restrict__ hw, const float *__restrict__ g, int Nimg,
           int H, int W, bf16 *gx, int ldg, float *part) {
    constexpr int P = 3 * C + 3;
    __shared__ float red[8][P];
    float acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = 0.f;
    const size_t HW = (size_t)H * W, n = (size_t)Nimg * HW;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const size_t nn = p / HW, q = p - nn * HW;
        const float g0 = g[(nn * 3 + 0) * HW + q], g1 = g[(nn * 3 + 1) * HW + q], g2 = g[(nn * 3 + 2) * HW + q];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float v = __bfloat162float(x[p * ldx + c]);
            gx[p * ldg + c] = __float2bfloat16(fmaf(g2, hw[2 * C + c], fmaf(g1, hw[C + c], g0 * hw[c])));
            acc[c] = fmaf(g0, v, acc[c]);
            acc[C + c] = fmaf(g1, v, acc[C + c]);
            acc[2 * C + c] = fmaf(g2, v, acc[2 * C + c]);
        }
        acc[3 * C] += g0;
        acc[3 * C + 1] += g1;
        acc[3 * C + 2] += g2;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        float v = acc[k];
        for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[w][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        float t = 0.f;
        for (int ww = 0; ww < 8; ++ww) t += red[ww][k];
        part[(size_t)blockIdx.x * P + k] = t;
    }
}

// fp32 parameters -> bf16 weights of one conv (forward layout [co][tap][ci])
// and its data-gradient layout wt[ci][tap'][co] with tap' = 8 - tap.
__global__ void k_prep_weights(const float *__restrict__ w, int Cout, int C, bf16 *wf, bf16 *wt) {
    const size_t n = (size_t)Cout * 9 * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % C), tap = (int)((i / C) % 9), co = (int)(i / ((size_t)9 * C));
        const bf16 v = __float2bfloat16(w[i]);
        wf[i] = v;
        if (wt) wt[((size_t)ci * 9 + (8 - tap)) * Cout + co] = v;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// He-normal initialisation from a counter-based hash (SplitMix64 + Box-Muller)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__global__ void k_init_normal(float *p, size_t n, float stdv, unsigned long long seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long a = mix64(seed * 0x9E3779B97F4A7C15ULL + 2 * i);
        const unsigned long long b = mix64(seed * 0x9E3779B97F4A7C15ULL + 2 * i + 1);
        const float u1 = ((a >> 40) + 1) * (1.0f / 16777217.0f), u2 = (b >> 40) * (1.0f / 16777216.0f);
        p[i] = stdv * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
    }
}

// y = lambda * u (per channel, planar): the network's training target
__global__ void k_warm_target(const float *__restrict__ u, const float *__restrict__ lam, size_t HW, float *y) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * HW; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __fmul_rn(u[i], lam[i % HW]);
}

// u0 = y / lambda (per channel, planar), the warm start
__global__ void k_warm_start(const float *__restrict__ y, const float *__restrict__ lam, size_t HW, float *u0) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * HW; i += (size_t)gridDim.x * blockDim.x)
        u0[i] = __fdiv_rn(y[i], lam[i % HW]);
}

static int gs(size_t n) { return (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8); }

// ------------------------------------------------------------ network description

// conv k: input channels, output channels, level (0 = full resolution)
struct ConvSpec {
    int cin, cout, level;
};

static std::vector<ConvSpec> unet_convs(int b) {
    return {{16, b, 0},          {b, b, 0},           {b, 2 * b, 1},       {2 * b, 2 * b, 1},
            {2 * b, 4 * b, 2},   {4 * b, 4 * b, 2},   {4 * b, 8 * b, 3},   {8 * b, 8 * b, 3},
            {12 * b, 4 * b, 2},  {4 * b, 4 * b, 2},   {6 * b, 2 * b, 1},   {2 * b, 2 * b, 1},
            {3 * b, b, 0},       {b, b, 0}};
}

struct ParamLayout {
    std::vector<size_t> w, b;  // offsets in the fp32 parameter vector
    size_t hw, hb, total;
};

static ParamLayout param_layout(int base) {
    ParamLayout L;
    size_t o = 0;
    for (auto &c : unet_convs(base)) {
        L.w.push_back(o);
        o += (size_t)c.cout * 9 * c.cin;
        L.b.push_back(o);
        o += c.cout;
    }
    L.hw = o;
    o += 3 * (size_t)base;
    L.hb = o;
    o += 3;
    L.total = o;
    return L;
}

// Activation buffers (bf16 NHWC, channel pitch ld) and their gradients.
struct Act {
    size_t off;  // byte offset in the workspace
    int C, ld, level;
};

struct NetLayout {
    // activations
    Act x0, a1, cat1, p1, a2, cat2, p2, a3, cat3, p3, a4, e4, d3a, d3, d2a, d2, d1a, d1;
    // gradients (same shapes)
    Act g_a1, g_cat1, g_p1, g_a2, g_cat2, g_p2, g_a3, g_cat3, g_p3, g_a4, g_e4, g_d3a, g_d3, g_d2a, g_d2, g_d1a, g_d1;
    size_t wf, wt, y, gy, part, lpart, loss, total;  // bf16 weights, fp32 y/g, partials
    size_t part_bytes;
};

static NetLayout net_layout(int b, int N, int H, int W, bool train) {
    NetLayout L;
    size_t o = 0;
    auto px = [&](int level) { return (size_t)N * (H >> level) * (W >> level); };
    auto act = [&](int C, int level) {
        Act a{o, C, C, level};
        o = align_up(o + px(level) * C * sizeof(bf16));
        return a;
    };
    L.x0 = act(16, 0);
    L.a1 = act(b, 0);
    L.cat1 = act(3 * b, 0);
    L.p1 = act(b, 1);
    L.a2 = act(2 * b, 1);
    L.cat2 = act(6 * b, 1);
    L.p2 = act(2 * b, 2);
    L.a3 = act(4 * b, 2);
    L.cat3 = act(12 * b, 2);
    L.p3 = act(4 * b, 3);
    L.a4 = act(8 * b, 3);
    L.e4 = act(8 * b, 3);
    L.d3a = act(4 * b, 2);
    L.d3 = act(4 * b, 2);
    L.d2a = act(2 * b, 1);
    L.d2 = act(2 * b, 1);
    L.d1a = act(b, 0);
    L.d1 = act(b, 0);
    if (train) {
        L.g_a1 = act(b, 0);
        L.g_cat1 = act(3 * b, 0);
        L.g_p1 = act(b, 1);
        L.g_a2 = act(2 * b, 1);
        L.g_cat2 = act(6 * b, 1);
        L.g_p2 = act(2 * b, 2);
        L.g_a3 = act(4 * b, 2);
        L.g_cat3 = act(12 * b, 2);
        L.g_p3 = act(4 * b, 3);
        L.g_a4 = act(8 * b, 3);
        L.g_e4 = act(8 * b, 3);
        L.g_d3a = act(4 * b, 2);
        L.g_d3 = act(4 * b, 2);
        L.g_d2a = act(2 * b, 1);
        L.g_d2 = act(2 * b, 1);
        L.g_d1a = act(b, 0);
        L.g_d1 = act(b, 0);
    }
    const size_t nw = param_layout(b).total;
    L.wf = o;
    o = align_up(o + nw * sizeof(bf16));
    L.wt = o;
    o = align_up(o + nw * sizeof(bf16));
    L.y = o;
    o = align_up(o + 3 * px(0) * sizeof(float));
    L.gy = o;
    o = align_up(o + 3 * px(0) * sizeof(float));
    L.part_bytes = (size_t)64 << 20;
    L.part = o;
    o = align_up(o + (train ? L.part_bytes : 0));
    L.lpart = o;
    o = align_up(o + 4096 * sizeof(float));
    L.loss = o;
    o = align_up(o + 256);
    L.total = o;
    return L;
}

static bool unet_shape_ok(int base, int N, int H, int W) {
    return (base == 16 || base == 32) && N >= 1 && H >= 8 && W >= 8 && H % 8 == 0 && W % 8 == 0 &&
           (long long)N * H * W <= (1LL << 26);
}

// ------------------------------------------------------------ layer launchers

int conv3x3_tc(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *b, int Cout, bool relu,
               void *y, int ldy, int *err, cudaStream_t s);
int conv3x3_halo(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *b, int Cout,
                 bool relu, void *y, int ldy, int *err, cudaStream_t s);
int conv3x3_wgrad_tc(const void *x, int ldx, int C, const void *dy, int lddy, int Cout, int N, int H, int W,
                     float *part, int splits, int *err, cudaStream_t s);

// tcgen05 kernel when the channel counts allow it (every layer of the
// network does), else the mma.sync kernel below.
static int conv_fwd(const bf16 *x, int ldx, int C, int N, int H, int W, const bf16 *w, const float *b, int Cout,
                    bool relu, bf16 *y, int ldy, cudaStream_t s) {
    if (C % 16 == 0 && Cout % 16 == 0 && ldx % 8 == 0 && ldy % 8 == 0) {
        const int rc = conv3x3_halo(x, ldx, C, N, H, W, w, b, Cout, relu, y, ldy, nullptr, s);
        if (rc != DH_EINVAL) return rc;  // DH_EINVAL: not one of its channel pairs
        return conv3x3_tc(x, ldx, C, N, H, W, w, b, Cout, relu, y, ldy, nullptr, s);
    }
    const int M = N * H * W;
    dim3 grid((M + kCBM - 1) / kCBM, (Cout + kCBN - 1) / kCBN);
    if (C % 32 == 0)
        k_conv3x3<32><<<grid, 128, 0, s>>>(x, ldx, C, N, H, W, w, b, Cout, relu, y, ldy);
    else if (C % 16 == 0)
        k_conv3x3<16><<<grid, 128, 0, s>>>(x, ldx, C, N, H, W, w, b, Cout, relu, y, ldy);
    else
        return DH_EINVAL;
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

// dw (fp32, [Cout][9][C]) and db (fp32, [Cout]) of y = conv(x), written into
// the gradient vector; `part` is scratch of part_bytes.
static int conv_wgrad(const bf16 *x, int ldx, int C, const bf16 *dy, int lddy, int Cout, int N, int H, int W,
                      float *dw, float *db, float *part, size_t part_bytes, cudaStream_t s) {
    const int M = N * H * W;
    const size_t per_split = (size_t)Cout * 9 * C * sizeof(float);
    int splits = (M + 4095) / 4096;
    const int max_splits = (int)(part_bytes / per_split);
    if (max_splits < 1) return DH_EINVAL;
    if (splits > max_splits) splits = max_splits;
    int split_px = (M + splits - 1) / splits;
    split_px = (split_px + kWBK - 1) / kWBK * kWBK;
    splits = (M + split_px - 1) / split_px;
    // tensor cores (tcgen05) from 96 input or 128 output channels (1.4-1.7x the
    // mma.sync kernel there); below that the M = 128 output-channel tile is
    // mostly empty and the mma.sync kernel is 6-10 % faster
    int rc = (C >= 96 || Cout >= 128) ? conv3x3_wgrad_tc(x, ldx, C, dy, lddy, Cout, N, H, W, part, splits, nullptr, s)
                                      : DH_EINVAL;
    if (rc == DH_EINVAL) {
        dim3 grid((Cout + 63) / 64, 9 * ((C + 63) / 64), splits);
        k_conv3x3_wgrad<<<grid, 128, 0, s>>>(x, ldx, C, dy, lddy, Cout, N, H, W, split_px, part);
    } else if (rc) {
        return rc;
    }
    k_sum_splits<<<gs((size_t)Cout * 9 * C), 256, 0, s>>>(part, splits, (size_t)Cout * 9 * C, dw, 0);
    const int bsplits = (M + 1023) / 1024;
    k_bias_grad<<<bsplits, 256, 0, s>>>(dy, lddy, Cout, M, 1024, part);
    k_sum_splits<<<gs(Cout), 256, 0, s>>>(part, bsplits, (size_t)Cout, db, 0);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

}  // namespace dh

namespace dh {

int launch_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out, cudaStream_t s);
int launch_transmission(const float *I, int H, int W, const dh_params *p, const float *A, float *td, float *t,
                        float *lam, float *phi, float *u0, float2 *phin_part, void *scratch, cudaStream_t s);
int launch_phin(const float *phi, int H, int W, float2 *part, SolveState *st, cudaStream_t s);
int launch_select_A(const float *I, const float *dc, int H, int W, int permille, float *A,
                    long long *index_out, char *ws, const WsLayout &L, cudaStream_t s);
int run_solve(float *u_caller, const float *phi, const float *lam, int H, int W, const dh_params *p,
              float *rho_hist, char *ws, const WsLayout &L, cudaStream_t s, float *J,
              cudaEvent_t loop_begin, cudaEvent_t loop_end, int *launches);
int read_solve_state(const char *ws, const WsLayout &L, SolveState *out);
int sweep_depth(const dh_params *p);
int sweep_tile_h(int depth);

#define BF(off) reinterpret_cast<bf16 *>(ws + (off))
#define RUN(x)                  \
    do {                        \
        int rc_ = (x);          \
        if (rc_) return rc_;    \
    } while (0)

// Forward pass; leaves every activation in the workspace (for the backward).
static int net_forward(const float *params, int b, const float *I, const float *t, const float *A,
                       const float *Phi, int N, int H, int W, char *ws, const NetLayout &L, bool train,
                       cudaStream_t s) {
    const ParamLayout P = param_layout(b);
    const auto convs = unet_convs(b);
    bf16 *wf = BF(L.wf), *wt = BF(L.wt);
    for (size_t k = 0; k < convs.size(); ++k)
        k_prep_weights<<<gs((size_t)convs[k].cout * 9 * convs[k].cin), 256, 0, s>>>(
            params + P.w[k], convs[k].cout, convs[k].cin, wf + P.w[k], train ? wt + P.w[k] : nullptr);
    const size_t M0 = (size_t)N * H * W;
    k_pack_input<<<gs(M0), 256, 0, s>>>(I, t, A, Phi, N, H, W, BF(L.x0.off));
    auto conv = [&](int k, const Act &x, const bf16 *xp, int lvl, bf16 *y, int ldy) {
        return conv_fwd(xp, x.ld, convs[k].cin, N, H >> lvl, W >> lvl, wf + P.w[k], params + P.b[k], convs[k].cout,
                        true, y, ldy, s);
    };
    const int h1 = H >> 1, w1 = W >> 1, h2 = H >> 2, w2 = W >> 2, h3 = H >> 3, w3 = W >> 3;
    // encoder
    RUN(conv(0, L.x0, BF(L.x0.off), 0, BF(L.a1.off), b));
    RUN(conv(1, L.a1, BF(L.a1.off), 0, BF(L.cat1.off) + 2 * b, 3 * b));
    k_avgpool<<<gs(M0 / 4 * b), 256, 0, s>>>(BF(L.cat1.off) + 2 * b, 3 * b, b, N, H, W, BF(L.p1.off), b);
    RUN(conv(2, L.p1, BF(L.p1.off), 1, BF(L.a2.off), 2 * b));
    RUN(conv(3, L.a2, BF(L.a2.off), 1, BF(L.cat2.off) + 4 * b, 6 * b));
    k_avgpool<<<gs(M0 / 16 * 2 * b), 256, 0, s>>>(BF(L.cat2.off) + 4 * b, 6 * b, 2 * b, N, h1, w1, BF(L.p2.off), 2 * b);
    RUN(conv(4, L.p2, BF(L.p2.off), 2, BF(L.a3.off), 4 * b));
    RUN(conv(5, L.a3, BF(L.a3.off), 2, BF(L.cat3.off) + 8 * b, 12 * b));
    k_avgpool<<<gs(M0 / 64 * 4 * b), 256, 0, s>>>(BF(L.cat3.off) + 8 * b, 12 * b, 4 * b, N, h2, w2, BF(L.p3.off), 4 * b);
    RUN(conv(6, L.p3, BF(L.p3.off), 3, BF(L.a4.off), 8 * b));
    RUN(conv(7, L.a4, BF(L.a4.off), 3, BF(L.e4.off), 8 * b));
    // decoder
    k_upsample<<<gs(M0 / 16 * 8 * b), 256, 0, s>>>(BF(L.e4.off), 8 * b, 8 * b, N, h3, w3, BF(L.cat3.off), 12 * b);
    RUN(conv(8, L.cat3, BF(L.cat3.off), 2, BF(L.d3a.off), 4 * b));
    RUN(conv(9, L.d3a, BF(L.d3a.off), 2, BF(L.d3.off), 4 * b));
    k_upsample<<<gs(M0 / 4 * 4 * b), 256, 0, s>>>(BF(L.d3.off), 4 * b, 4 * b, N, h2, w2, BF(L.cat2.off), 6 * b);
    RUN(conv(10, L.cat2, BF(L.cat2.off), 1, BF(L.d2a.off), 2 * b));
    RUN(conv(11, L.d2a, BF(L.d2a.off), 1, BF(L.d2.off), 2 * b));
    k_upsample<<<gs(M0 * 2 * b), 256, 0, s>>>(BF(L.d2.off), 2 * b, 2 * b, N, h1, w1, BF(L.cat1.off), 3 * b);
    RUN(conv(12, L.cat1, BF(L.cat1.off), 0, BF(L.d1a.off), b));
    RUN(conv(13, L.d1a, BF(L.d1a.off), 0, BF(L.d1.off), b));
    k_head<<<gs(M0), 256, 0, s>>>(BF(L.d1.off), b, b, params + P.hw, params + P.hb, Phi, N, H, W,
                                  reinterpret_cast<float *>(ws + L.y));
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

// MSE loss against target and the gradients of every parameter.
static int net_backward(const float *params, int b, const float *target, int N, int H, int W, char *ws,
                        const NetLayout &L, float *grads, float *loss, cudaStream_t s) {
    const ParamLayout P = param_layout(b);
    const auto convs = unet_convs(b);
    bf16 *wt = BF(L.wt);
    float *part = reinterpret_cast<float *>(ws + L.part);
    const size_t M0 = (size_t)N * H * W;
    const int h1 = H >> 1, w1 = W >> 1, h2 = H >> 2, w2 = W >> 2, h3 = H >> 3, w3 = W >> 3;
    float *y = reinterpret_cast<float *>(ws + L.y), *gy = reinterpret_cast<float *>(ws + L.gy);
    float *lpart = reinterpret_cast<float *>(ws + L.lpart);
    const int lb = 1024;
    k_mse<<<lb, 256, 0, s>>>(y, target, 3 * M0, gy, lpart);
    k_loss_final<<<1, 32, 0, s>>>(lpart, lb, 3 * M0, loss);
    // head
    const int hb = 512;
    float *hpart = part;  // 512 blocks x (3b+3) partials
    if (b == 32)
        k_head_bwd<32><<<hb, 256, 0, s>>>(BF(L.d1.off), b, params + P.hw, gy, N, H, W, BF(L.g_d1.off), b, hpart);
    else
        k_head_bwd<16><<<hb, 256, 0, s>>>(BF(L.d1.off), b, params + P.hw, gy, N, H, W, BF(L.g_d1.off), b, hpart);
    k_sum_splits<<<1, 256, 0, s>>>(hpart, hb, (size_t)(3 * b + 3), grads + P.hw, 0);
    auto relu_b = [&](bf16 *g, int ldg, const bf16 *yv, int ldy, int C, int lvl) {
        const int M = N * (H >> lvl) * (W >> lvl);
        k_relu_bwd<<<gs((size_t)M * C / 8), 256, 0, s>>>(g, ldg, yv, ldy, C, M);
    };
    // conv k: y = conv_k(x); dy given -> dw, db, and (if gx) gx = dgrad
    auto conv_b = [&](int k, const bf16 *x, int ldx, const bf16 *dy, int lddy, int lvl, bf16 *gx, int ldgx) {
        const int cin = convs[k].cin, cout = convs[k].cout;
        int rc = conv_wgrad(x, ldx, cin, dy, lddy, cout, N, H >> lvl, W >> lvl, grads + P.w[k], grads + P.b[k], part,
                            L.part_bytes, s);
        if (rc || !gx) return rc;
        return conv_fwd(dy, lddy, cout, N, H >> lvl, W >> lvl, wt + P.w[k], nullptr, cin, false, gx, ldgx, s);
    };
    // decoder level 1
    relu_b(BF(L.g_d1.off), b, BF(L.d1.off), b, b, 0);
    RUN(conv_b(13, BF(L.d1a.off), b, BF(L.g_d1.off), b, 0, BF(L.g_d1a.off), b));
    relu_b(BF(L.g_d1a.off), b, BF(L.d1a.off), b, b, 0);
    RUN(conv_b(12, BF(L.cat1.off), 3 * b, BF(L.g_d1a.off), b, 0, BF(L.g_cat1.off), 3 * b));
    k_upsample_bwd<<<gs(M0 / 4 * 2 * b), 256, 0, s>>>(BF(L.g_cat1.off), 3 * b, 2 * b, N, h1, w1, BF(L.g_d2.off), 2 * b);
    // decoder level 2
    relu_b(BF(L.g_d2.off), 2 * b, BF(L.d2.off), 2 * b, 2 * b, 1);
    RUN(conv_b(11, BF(L.d2a.off), 2 * b, BF(L.g_d2.off), 2 * b, 1, BF(L.g_d2a.off), 2 * b));
    relu_b(BF(L.g_d2a.off), 2 * b, BF(L.d2a.off), 2 * b, 2 * b, 1);
    RUN(conv_b(10, BF(L.cat2.off), 6 * b, BF(L.g_d2a.off), 2 * b, 1, BF(L.g_cat2.off), 6 * b));
    k_upsample_bwd<<<gs(M0 / 16 * 4 * b), 256, 0, s>>>(BF(L.g_cat2.off), 6 * b, 4 * b, N, h2, w2, BF(L.g_d3.off), 4 * b);
    // decoder level 3
    relu_b(BF(L.g_d3.off), 4 * b, BF(L.d3.off), 4 * b, 4 * b, 2);
    RUN(conv_b(9, BF(L.d3a.off), 4 * b, BF(L.g_d3.off), 4 * b, 2, BF(L.g_d3a.off), 4 * b));
    relu_b(BF(L.g_d3a.off), 4 * b, BF(L.d3a.off), 4 * b, 4 * b, 2);
    RUN(conv_b(8, BF(L.cat3.off), 12 * b, BF(L.g_d3a.off), 4 * b, 2, BF(L.g_cat3.off), 12 * b));
    k_upsample_bwd<<<gs(M0 / 64 * 8 * b), 256, 0, s>>>(BF(L.g_cat3.off), 12 * b, 8 * b, N, h3, w3, BF(L.g_e4.off), 8 * b);
    // bottleneck
    relu_b(BF(L.g_e4.off), 8 * b, BF(L.e4.off), 8 * b, 8 * b, 3);
    RUN(conv_b(7, BF(L.a4.off), 8 * b, BF(L.g_e4.off), 8 * b, 3, BF(L.g_a4.off), 8 * b));
    relu_b(BF(L.g_a4.off), 8 * b, BF(L.a4.off), 8 * b, 8 * b, 3);
    RUN(conv_b(6, BF(L.p3.off), 4 * b, BF(L.g_a4.off), 8 * b, 3, BF(L.g_p3.off), 4 * b));
    // encoder level 3: skip gradient + pooled gradient
    k_avgpool_bwd_add<<<gs(M0 / 16 * 4 * b), 256, 0, s>>>(BF(L.g_p3.off), 4 * b, 4 * b, N, h2, w2, BF(L.g_cat3.off) + 8 * b, 12 * b);
    relu_b(BF(L.g_cat3.off) + 8 * b, 12 * b, BF(L.cat3.off) + 8 * b, 12 * b, 4 * b, 2);
    RUN(conv_b(5, BF(L.a3.off), 4 * b, BF(L.g_cat3.off) + 8 * b, 12 * b, 2, BF(L.g_a3.off), 4 * b));
    relu_b(BF(L.g_a3.off), 4 * b, BF(L.a3.off), 4 * b, 4 * b, 2);
    RUN(conv_b(4, BF(L.p2.off), 2 * b, BF(L.g_a3.off), 4 * b, 2, BF(L.g_p2.off), 2 * b));
    // encoder level 2
    k_avgpool_bwd_add<<<gs(M0 / 4 * 2 * b), 256, 0, s>>>(BF(L.g_p2.off), 2 * b, 2 * b, N, h1, w1, BF(L.g_cat2.off) + 4 * b, 6 * b);
    relu_b(BF(L.g_cat2.off) + 4 * b, 6 * b, BF(L.cat2.off) + 4 * b, 6 * b, 2 * b, 1);
    RUN(conv_b(3, BF(L.a2.off), 2 * b, BF(L.g_cat2.off) + 4 * b, 6 * b, 1, BF(L.g_a2.off), 2 * b));
    relu_b(BF(L.g_a2.off), 2 * b, BF(L.a2.off), 2 * b, 2 * b, 1);
    RUN(conv_b(2, BF(L.p1.off), b, BF(L.g_a2.off), 2 * b, 1, BF(L.g_p1.off), b));
    // encoder level 1
    k_avgpool_bwd_add<<<gs(M0 * b), 256, 0, s>>>(BF(L.g_p1.off), b, b, N, H, W, BF(L.g_cat1.off) + 2 * b, 3 * b);
    relu_b(BF(L.g_cat1.off) + 2 * b, 3 * b, BF(L.cat1.off) + 2 * b, 3 * b, b, 0);
    RUN(conv_b(1, BF(L.a1.off), b, BF(L.g_cat1.off) + 2 * b, 3 * b, 0, BF(L.g_a1.off), b));
    relu_b(BF(L.g_a1.off), b, BF(L.a1.off), b, b, 0);
    RUN(conv_b(0, BF(L.x0.off), 16, BF(L.g_a1.off), b, 0, nullptr, 0));
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

#undef BF

// Warm start of a batched solve: images of one shape go through the network
// together, up to kWarmGroupPixels pixels per forward (small images leave most
// SMs idle in the deep levels when run one at a time).
constexpr long long kWarmGroupPixels = 4200000;

int warm_group_size(int H, int W) {
    const long long n = kWarmGroupPixels / ((long long)H * W);
    return n < 1 ? 1 : (n > 64 ? 64 : (int)n);
}

// Workspace of one grouped forward over n images of HxW: the gathered inputs
// (I and Phi 3HW floats, t HW floats, A 3 floats per image; none for n = 1)
// followed by the network's own workspace.  0: a shape the network does not take.
struct WarmGather {
    size_t I, Phi, t, A, net;
};
static WarmGather warm_gather(int n, int H, int W) {
    const size_t HW = (size_t)H * W;
    WarmGather g{};
    size_t o = 0;
    if (n > 1) {
        g.I = o; o = align_up(o + (size_t)n * 3 * HW * sizeof(float));
        g.Phi = o; o = align_up(o + (size_t)n * 3 * HW * sizeof(float));
        g.t = o; o = align_up(o + (size_t)n * HW * sizeof(float));
        g.A = o; o = align_up(o + (size_t)n * 3 * sizeof(float));
    }
    g.net = o;
    return g;
}

size_t warm_net_bytes(int base, int n, int H, int W) {
    if (n < 1 || !unet_shape_ok(base, n, H, W)) return 0;
    return warm_gather(n, H, W).net + net_layout(base, n, H, W, false).total;
}

// u0[k] = net(I[k], t[k], A[k], Phi[k]) / lam[k] for n images of one shape in
// one forward, queued on s.  nws: warm_net_bytes(base, n, H, W) bytes, 256-byte
// aligned.  Every image's result equals its own single-image forward (the
// kernels work per pixel, per row segment or per image).
int warm_u0_group(const float *params, int base, int n, const float *const *I, const float *const *t,
                  const float *const *A, const float *const *phi, const float *const *lam, float *const *u0, int H,
                  int W, void *nws, size_t nws_bytes, cudaStream_t s) {
    if (n < 1 || !unet_shape_ok(base, n, H, W)) return DH_EINVAL;
    const WarmGather g = warm_gather(n, H, W);
    const NetLayout NL = net_layout(base, n, H, W, false);
    if (!nws || ((uintptr_t)nws % kAlign) || nws_bytes < g.net + NL.total) return DH_EWORKSPACE;
    char *ws = (char *)nws;
    const size_t HW = (size_t)H * W;
    const float *gI = I[0], *gPhi = phi[0], *gt = t[0], *gA = A[0];
    if (n > 1) {  // gather the group's inputs into contiguous N x ... arrays
        float *dI = reinterpret_cast<float *>(ws + g.I), *dPhi = reinterpret_cast<float *>(ws + g.Phi);
        float *dt = reinterpret_cast<float *>(ws + g.t), *dA = reinterpret_cast<float *>(ws + g.A);
        for (int k = 0; k < n; ++k) {
            DH_CUDA_TRY(cudaMemcpyAsync(dI + (size_t)k * 3 * HW, I[k], 3 * HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
            DH_CUDA_TRY(cudaMemcpyAsync(dPhi + (size_t)k * 3 * HW, phi[k], 3 * HW * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s));
            DH_CUDA_TRY(cudaMemcpyAsync(dt + (size_t)k * HW, t[k], HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
            DH_CUDA_TRY(cudaMemcpyAsync(dA + 3 * k, A[k], 3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
        gI = dI;
        gPhi = dPhi;
        gt = dt;
        gA = dA;
    }
    char *nw = ws + g.net;
    RUN(net_forward(params, base, gI, gt, gA, gPhi, n, H, W, nw, NL, false, s));
    const float *y = reinterpret_cast<const float *>(nw + NL.y);
    for (int k = 0; k < n; ++k)
        k_warm_start<<<gs(3 * HW), 256, 0, s>>>(y + (size_t)k * 3 * HW, lam[k], HW, u0[k]);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

}  // namespace dh

using namespace dh;

extern "C" {

size_t dh_unet_param_count(int base) {
    if (base != 16 && base != 32) return 0;
    return param_layout(base).total;
}

size_t dh_unet_workspace_bytes(int base, int N, int H, int W, int train) {
    if (!unet_shape_ok(base, N, H, W)) return 0;
    return net_layout(base, N, H, W, train != 0).total;
}

int dh_unet_init(float *params, int base, unsigned long long seed, void *stream) {
    if (!params || dh_unet_param_count(base) == 0) return DH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const ParamLayout P = param_layout(base);
    const auto convs = unet_convs(base);
    DH_CUDA_TRY(cudaMemsetAsync(params, 0, P.total * sizeof(float), s));
    for (size_t k = 0; k < convs.size(); ++k) {
        const size_t n = (size_t)convs[k].cout * 9 * convs[k].cin;
        const int fan_in = 9 * (k == 0 ? 10 : convs[k].cin);
        k_init_normal<<<gs(n), 256, 0, s>>>(params + P.w[k], n, sqrtf(2.f / fan_in), seed * 131 + k);
    }
    // a small head: the untrained network returns about the analytic guess y = Phi
    k_init_normal<<<1, 256, 0, s>>>(params + P.hw, 3 * (size_t)base, 0.01f * sqrtf(1.f / base), seed * 131 + 99);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int dh_unet_forward(const float *params, int base, const float *I, const float *t, const float *A,
                    const float *Phi, int N, int H, int W, float *y, void *workspace, size_t workspace_bytes,
                    void *stream) {
    if (!params || !I || !t || !A || !Phi || !y || !unet_shape_ok(base, N, H, W)) return DH_EINVAL;
    const NetLayout L = net_layout(base, N, H, W, false);
    if (!workspace || ((uintptr_t)workspace % kAlign) || workspace_bytes < L.total) return DH_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int rc = net_forward(params, base, I, t, A, Phi, N, H, W, ws, L, false, s);
    if (rc) return rc;
    DH_CUDA_TRY(cudaMemcpyAsync(y, ws + L.y, (size_t)3 * N * H * W * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return DH_OK;
}

int dh_unet_backward(const float *params, int base, const float *I, const float *t, const float *A,
                     const float *Phi, const float *target, int N, int H, int W, float *grads, float *loss,
                     void *workspace, size_t workspace_bytes, void *stream) {
    if (!params || !I || !t || !A || !Phi || !target || !grads || !loss || !unet_shape_ok(base, N, H, W))
        return DH_EINVAL;
    const NetLayout L = net_layout(base, N, H, W, true);
    if (!workspace || ((uintptr_t)workspace % kAlign) || workspace_bytes < L.total) return DH_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int rc = net_forward(params, base, I, t, A, Phi, N, H, W, ws, L, true, s);
    if (rc) return rc;
    return net_backward(params, base, target, N, H, W, ws, L, grads, loss, s);
}

int dh_unet_adam(float *params, const float *grads, float *m, float *v, size_t n, float lr, float beta1,
                 float beta2, float eps, int step, void *stream) {
    if (!params || !grads || !m || !v || n == 0 || step < 1 || !(lr > 0.f)) return DH_EINVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<gs(n), 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, lr, beta1, beta2, eps, c1, c2);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int dh_warm_start(const float *y, const float *lam, int H, int W, float *u0, void *stream) {
    if (!y || !lam || !u0 || !shape_ok(H, W)) return DH_EINVAL;
    const size_t HW = (size_t)H * W;
    k_warm_start<<<gs(3 * HW), 256, 0, (cudaStream_t)stream>>>(y, lam, HW, u0);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int dh_warm_target(const float *u, const float *lam, int H, int W, float *y, void *stream) {
    if (!u || !lam || !y || !shape_ok(H, W)) return DH_EINVAL;
    const size_t HW = (size_t)H * W;
    k_warm_target<<<gs(3 * HW), 256, 0, (cudaStream_t)stream>>>(u, lam, HW, y);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int dh_conv3x3_forward(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *bias, int Cout,
                       int relu, void *y, int ldy, void *stream) {
    if (!x || !w || !y || C % 16 || Cout % 8 || ldx < C || ldy < Cout || ldx % 8 || ldy % 2 || N < 1 || H < 1 || W < 1)
        return DH_EINVAL;
    return conv_fwd((const bf16 *)x, ldx, C, N, H, W, (const bf16 *)w, bias, Cout, relu != 0, (bf16 *)y, ldy,
                    (cudaStream_t)stream);
}

int dh_conv3x3_backward_weights(const void *x, int ldx, int C, const void *dy, int lddy, int Cout, int N, int H, int W,
                                float *dw, float *db, float *scratch, size_t scratch_bytes, void *stream) {
    if (!x || !dy || !dw || !db || !scratch || C % 8 || Cout % 8 || ldx % 8 || lddy % 8 || N < 1 || H < 1 || W < 1 ||
        256 % Cout)
        return DH_EINVAL;
    return conv_wgrad((const bf16 *)x, ldx, C, (const bf16 *)dy, lddy, Cout, N, H, W, dw, db, scratch, scratch_bytes,
                      (cudaStream_t)stream);
}

// Front end, network warm start u0 = y / lambda, then the fixed-point loop.
int dh_dehaze_warm(const float *params, int base, const float *I, int H, int W, const dh_params *p, float *J,
                   float *u, float *t, float *A, void *workspace, size_t workspace_bytes, void *net_workspace,
                   size_t net_workspace_bytes, void *stream, dh_report *report) {
    if (!params || !I || !J || !u || !t || !A || !p || !shape_ok(H, W) || !unet_shape_ok(base, 1, H, W))
        return DH_EINVAL;
    if (dh_workspace_bytes(H, W, p) == 0) return DH_EINVAL;
    const WsLayout WL = ws_layout(H, W, sweep_depth(p), sweep_tile_h(sweep_depth(p)), refine_bytes(H, W, p));
    if (!workspace || ((uintptr_t)workspace % kAlign) || workspace_bytes < WL.total) return DH_EWORKSPACE;
    const NetLayout NL = net_layout(base, 1, H, W, false);
    if (!net_workspace || ((uintptr_t)net_workspace % kAlign) || net_workspace_bytes < NL.total) return DH_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    cudaEvent_t e0 = nullptr, e1 = nullptr, la = nullptr, lb = nullptr;
    if (report) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventCreate(&la);
        cudaEventCreate(&lb);
        cudaEventRecord(e0, s);
    }
    float *dc = (float *)(ws + WL.dc), *lam = (float *)(ws + WL.lam), *phi = (float *)(ws + WL.phi);
    RUN(launch_dark_channel(I, H, W, p->patch, nullptr, dc, s));
    RUN(launch_select_A(I, dc, H, W, p->topk_permille, A, nullptr, ws, WL, s));
    RUN(launch_transmission(I, H, W, p, A, nullptr, t, lam, phi, nullptr, nullptr, ws + WL.refine, s));
    RUN(launch_phin(phi, H, W, (float2 *)(ws + WL.phin_part), (SolveState *)(ws + WL.state), s));
    char *nws = (char *)net_workspace;
    RUN(net_forward(params, base, I, t, A, phi, 1, H, W, nws, NL, false, s));
    k_warm_start<<<gs((size_t)3 * H * W), 256, 0, s>>>(reinterpret_cast<const float *>(nws + NL.y), lam,
                                                      (size_t)H * W, u);
    int launches = 0;
    RUN(run_solve(u, phi, lam, H, W, p, nullptr, ws, WL, s, J, la, lb, &launches));
    DH_CUDA_TRY(cudaGetLastError());
    if (!report) return DH_OK;
    std::memset(report, 0, sizeof(*report));
    cudaEventRecord(e1, s);
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&report->ms, e0, e1);
    cudaEventElapsedTime(&report->ms_loop, la, lb);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(la);
    cudaEventDestroy(lb);
    cudaGetLastError();
    SolveState st;
    SelectState sel;
    RUN(read_solve_state(ws, WL, &st));
    DH_CUDA_TRY(cudaMemcpy(&sel, ws + WL.sel, sizeof(sel), cudaMemcpyDeviceToHost));
    DH_CUDA_TRY(cudaMemcpy(report->A, A, 3 * sizeof(float), cudaMemcpyDeviceToHost));
    report->status = st.status;
    report->n_iter = st.n_final;
    for (int c = 0; c < 3; ++c) report->rho[c] = st.rho[c];
    report->a_index = sel.best;
    report->launches = launches + (p->use_graph ? st.n_final + 1 : 0) + 19 + 2 * 14 + 12;
    return report->status;
}

}  // extern "C"
