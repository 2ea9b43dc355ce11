// 3x3 convolution (zero padding, bias, optional ReLU) as an implicit GEMM on
// the 5th-generation tensor cores: tcgen05.mma (kind::f16, bf16 operands,
// fp32 accumulators in tensor memory), issued by one thread per CTA.
//
//   y[p][co] = bias[co] + sum_{tap, ci} x[p + tap][ci] * w[co][tap][ci]
//
// GEMM view: M = pixels (128 per CTA), N = output channels (NT per CTA),
// K = 9 taps x C channels, walked in k-blocks of one tap and 32 channels.
// Each k-block's operands are staged in shared memory by cp.async (16-byte
// copies, zero-filled outside the image and past C) in the K-major layout
// with the 64-byte swizzle: a 64-byte row per pixel / per output channel,
// 16-byte chunk j of row r stored at chunk j ^ ((r >> 1) & 3).  A ring of
// STAGES k-blocks keeps the loads ahead of the MMAs; each k-block's MMAs
// (two K = 16 steps) are committed to that stage's mbarrier, which frees the
// stage for the k-block STAGES ahead.  The epilogue reads the accumulators
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = pixels), adds the
// bias, applies ReLU, rounds to bf16 and stores.  The same kernel computes
// the data gradient (x = dy, w flipped and transposed).
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace dh {

int encode_tiled(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                 const cuuint64_t *strides, const cuuint32_t *box);
int encode_tiled_sw(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                    const cuuint64_t *strides, const cuuint32_t *box, CUtensorMapSwizzle swizzle);

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTcBM = 128;             // pixels per CTA = MMA M = TMEM lanes
constexpr int kTcBK = 32;              // channels per k-block (64-byte rows)
constexpr uint32_t kTcSmemBudget = 104 * 1024;  // two CTAs per SM (one's epilogue hides under the other's loop)
constexpr long long kTcWaitCycles = 4000000000LL;  // about 2 s

template <int NT>
struct TcPlan {
    static constexpr uint32_t A_BYTES = kTcBM * 64;
    static constexpr uint32_t B_BYTES = NT * 64;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;  // multiple of 1024 (NT % 16 == 0)
    static constexpr int STAGES = (int)(kTcSmemBudget / STAGE) < 16 ? (int)(kTcSmemBudget / STAGE) : 16;
    static constexpr uint32_t SMEM = STAGES * STAGE + 1024;  // + alignment slack
    static constexpr uint32_t TMEM_COLS = NT <= 32 ? 32 : NT <= 64 ? 64 : NT <= 128 ? 128 : 256;
};

// --- PTX wrappers (sm_100 family ISA) ---------------------------------------

__device__ __forceinline__ void cp_async_16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (stride byte offset), leading byte offset unused (1),
// descriptor version 1.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrives on the mbarrier once every MMA this thread issued so far is done.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// The load and its wait are one asm statement: the destination registers are
// written asynchronously, and with the wait in a statement of its own the
// compiler was free to schedule their first uses between the two.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

template <int NT>
__global__ void __launch_bounds__(128, 2)
k_conv3x3_tc(const bf16 *__restrict__ x, int ldx, int C, int Nimg, int H, int W, const bf16 *__restrict__ w,
             const float *__restrict__ bias, int Cout, int relu, bf16 *__restrict__ y, int ldy, int *err) {
    using P = TcPlan<NT>;
    constexpr int S = P::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t mma_bar[S];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = H * W, M = Nimg * HW;
    const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * NT;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(P::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&mma_bar[s], 1);
        mbar_init(&done_bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // this thread's A row: pixel m0 + tid
    const int p = m0 + tid;
    const bool pin = p < M;
    const int pn = pin ? p / HW : 0, prem = pin ? p - pn * HW : 0;
    const int py = prem / W, px = prem - py * W;
    const int KC = (C + kTcBK - 1) / kTcBK, KB = 9 * KC;
    const uint32_t sbase = smem_addr(smem);

    auto load = [&](int kb, int stage) {
        const int tap = kb / KC, c0 = (kb - tap * KC) * kTcBK;
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        const uint32_t As = sbase + stage * P::STAGE, Bs = As + P::A_BYTES;
        const bool ok = pin && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const bf16 *src = ok ? x + ((size_t)(pn * H + yy) * W + xx) * ldx + c0 : x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool v = ok && c0 + 8 * j < C;
            cp_async_16(As + tid * 64 + ((j ^ ((tid >> 1) & 3)) << 4), v ? src + 8 * j : x, v ? 16u : 0u);
        }
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) {
            const int idx = tid + i * 128, r = idx >> 2, j = idx & 3, co = n0 + r;
            const bool v = co < Cout && c0 + 8 * j < C;
            const bf16 *ws = v ? w + ((size_t)co * 9 + tap) * C + c0 + 8 * j : w;
            cp_async_16(Bs + r * 64 + ((j ^ ((r >> 1) & 3)) << 4), ws, v ? 16u : 0u);
        }
    };

    constexpr uint32_t IDESC = f16_idesc(kTcBM, NT);
    for (int s = 0; s < S - 1; ++s) {
        if (s < KB) load(s, s);
        cp_async_commit();
    }
    bool failed = false;
    for (int kb = 0; kb < KB; ++kb) {
        const int stage = kb % S;
        cp_async_wait<S - 2>();     // this thread's copies of k-block kb have landed
        fence_proxy_async_smem();   // ... and are visible to the tensor core's proxy
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const int c0 = (kb % KC) * kTcBK;
            const int ksteps = C - c0 >= 32 ? 2 : 1;  // C % 16 == 0
            const uint32_t As = sbase + stage * P::STAGE, Bs = As + P::A_BYTES;
            for (int k = 0; k < ksteps; ++k)
                tc_mma(tmem, sw64_desc(As + 32 * k), sw64_desc(Bs + 32 * k), IDESC, (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&mma_bar[stage]);
        }
        // refill the stage that k-block kb-1 used once its MMAs are done
        const int kn = kb + S - 1;
        if (kn < KB) {
            const int sn = kn % S;
            if (kn >= S && !mbar_wait_bounded(&mma_bar[sn], ((kn / S) - 1) & 1, kTcWaitCycles)) failed = true;
            load(kn, sn);
        }
        cp_async_commit();
        if (__syncthreads_or(failed)) break;
    }
    if (tid == 0) tc_commit(&done_bar);
    if (!mbar_wait_bounded(&done_bar, 0, kTcWaitCycles)) failed = true;
    cp_async_wait<0>();
    if (failed && err) atomicExch(err, DH_ETIMEOUT);
    tc_fence_after();

    // epilogue: warp w reads TMEM lanes 32w..32w+31, i.e. pixels m0 + 32w + lane
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < NT; c += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
        const int col = n0 + c;
        if (row < M && col < Cout && !failed) {
            uint32_t packed[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float v0 = __uint_as_float(r[2 * j]) + (bias ? __ldg(bias + col + 2 * j) : 0.f);
                float v1 = __uint_as_float(r[2 * j + 1]) + (bias ? __ldg(bias + col + 2 * j + 1) : 0.f);
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                packed[j] = *reinterpret_cast<const uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)row * ldy + col);
            dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::TMEM_COLS)
                     : "memory");
}

// TMA-fed variant for images whose rows fill 128-pixel segments well: a tile
// is a 128-pixel segment of one image row (N tile as above).  For each k-block
// (tap, 32 channels) one TMA box brings the A tile - the segment's pixels
// shifted by the tap, zero filled outside the image and past C - and one the
// weights (NT output channels x 32 input channels of that tap), both with the
// 64-byte swizzle, i.e. the K-major layout the descriptors above read.  One
// thread issues the loads into a ring of stages, another the MMAs; a "full"
// mbarrier per stage (TMA transaction bytes) and an "empty" one (tcgen05.commit)
// order them, so no block barrier sits in the k loop.
template <int NT>
__global__ void __launch_bounds__(128, 2)
k_conv3x3_tma(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw, int C, int H, int W,
              int segs, const float *__restrict__ bias, int Cout, int relu, bf16 *__restrict__ y, int ldy, int *err) {
    using P = TcPlan<NT>;
    constexpr int S = P::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = blockIdx.x;
    const int seg = t % segs, row = t / segs, n = row / H, yy = row - n * H, x0 = seg * 128;
    const int n0 = blockIdx.y * NT;
    const int KC = (C + kTcBK - 1) / kTcBK, KB = 9 * KC;
    const uint32_t sbase = smem_addr(smem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(P::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done_bar, 1);
        fence_mbar_init();
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {  // loads
        int kb = 0;
        for (; kb < KB; ++kb) {
            const int s = kb % S;
            if (kb >= S && !mbar_wait_bounded(&empty[s], (uint32_t)((kb / S) - 1) & 1u, kTcWaitCycles)) {
                s_fail = 1;
                break;
            }
            const int tap = kb / KC, c0 = (kb - tap * KC) * kTcBK;
            unsigned char *As = smem + s * P::STAGE;
            mbar_arrive_expect_tx(&full[s], P::STAGE);
            tma_load_4d(smem_addr(As), &tmx, &full[s], c0, x0 + tap % 3 - 1, yy + tap / 3 - 1, n);
            tma_load_2d(As + P::A_BYTES, &tmw, &full[s], tap * C + c0, n0);
        }
        s_issued = kb;
    } else if (tid == 32) {  // MMAs
        constexpr uint32_t IDESC = f16_idesc(kTcBM, NT);
        int kb = 0;
        for (; kb < KB; ++kb) {
            const int s = kb % S;
            if (!mbar_wait_bounded(&full[s], (uint32_t)(kb / S) & 1u, kTcWaitCycles)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const int c0 = (kb % KC) * kTcBK;
            const int ksteps = C - c0 >= 32 ? 2 : 1;  // C % 16 == 0
            const uint32_t As = sbase + s * P::STAGE, Bs = As + P::A_BYTES;
            for (int k = 0; k < ksteps; ++k)
                tc_mma(tmem, sw64_desc(As + 32 * k), sw64_desc(Bs + 32 * k), IDESC, (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[s]);  // the stage is free once these MMAs are done
        }
        s_consumed = kb;
        tc_commit(&done_bar);  // every MMA issued above
    }
    bool failed = !mbar_wait_bounded(&done_bar, 0, kTcWaitCycles);
    __syncthreads();
    failed = __syncthreads_or(failed || s_fail);
    if (failed) {
        // loads issued but never consumed land before the shared memory goes away
        if (tid == 0) {
            for (int kb = s_consumed; kb < s_issued; ++kb)
                mbar_wait_bounded(&full[kb % S], (uint32_t)(kb / S) & 1u, kTcWaitCycles);
            if (err) atomicExch(err, DH_ETIMEOUT);
        }
        __syncthreads();
    }
    tc_fence_after();

    // epilogue: warp w reads TMEM lanes 32w..32w+31 = pixels x0 + 32w + lane of the segment
    const int px = x0 + warp * 32 + lane;
    const size_t orow = (size_t)row * W + px;
#pragma unroll 1
    for (int c = 0; c < NT; c += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
        const int col = n0 + c;
        if (px < W && col < Cout && !failed) {
            uint32_t packed[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float v0 = __uint_as_float(r[2 * j]) + (bias ? __ldg(bias + col + 2 * j) : 0.f);
                float v1 = __uint_as_float(r[2 * j + 1]) + (bias ? __ldg(bias + col + 2 * j + 1) : 0.f);
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                packed[j] = *reinterpret_cast<const uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(y + orow * ldy + col);
            dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::TMEM_COLS)
                     : "memory");
}

// Input and weight maps of the TMA-fed kernel: x as (channel, x, y, image)
// with 32-channel x 128-pixel boxes, w ([cout][tap][cin]) as (tap*C + cin,
// cout) with 32 x NT boxes; both with the 64-byte swizzle.
static int encode_tc_maps(CUtensorMap *mx, CUtensorMap *mw, const bf16 *x, int ldx, int C, int N, int H, int W,
                          const bf16 *w, int Cout, int NT) {
    const cuuint64_t pitch = (cuuint64_t)ldx * sizeof(bf16);
    const cuuint64_t xd[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t xs[3] = {pitch, pitch * (cuuint64_t)W, pitch * (cuuint64_t)W * (cuuint64_t)H};
    const cuuint32_t xb[4] = {32, 128, 1, 1};
    int rc = encode_tiled_sw(mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, x, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_64B);
    if (rc) return rc;
    const cuuint64_t wd[2] = {(cuuint64_t)9 * C, (cuuint64_t)Cout};
    const cuuint64_t ws[1] = {(cuuint64_t)9 * C * sizeof(bf16)};
    const cuuint32_t wb[2] = {32, (cuuint32_t)NT};
    return encode_tiled_sw(mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, w, wd, ws, wb, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Whether the TMA-fed kernel serves this layer: rows that fill at least 3/4
// of their 128-pixel segments, 16-byte aligned activations and weights.
static bool tma_conv_ok(const void *x, const void *w, int W) {
    const int segs = (W + 127) / 128;
    return 4 * W >= 3 * 128 * segs && ((uintptr_t)x % 16) == 0 && ((uintptr_t)w % 16) == 0;
}

template <int NT>
int launch_tc_tma(const bf16 *x, int ldx, int C, int N, int H, int W, const bf16 *w, const float *b, int Cout,
                  bool relu, bf16 *y, int ldy, int *err, cudaStream_t s) {
    using P = TcPlan<NT>;
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return DH_ECUDA;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            DH_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3_tma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)P::SMEM));
            attr_set[dev] = true;
        }
    }
    CUtensorMap mx, mw;
    const int rc = encode_tc_maps(&mx, &mw, x, ldx, C, N, H, W, w, Cout, NT);
    if (rc) return rc;
    const int segs = (W + 127) / 128;
    dim3 grid((unsigned)(N * H * segs), (Cout + NT - 1) / NT);
    k_conv3x3_tma<NT><<<grid, 128, P::SMEM, s>>>(mx, mw, C, H, W, segs, b, Cout, relu ? 1 : 0, y, ldy, err);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

template <int NT>
int launch_tc(const bf16 *x, int ldx, int C, int N, int H, int W, const bf16 *w, const float *b, int Cout, bool relu,
              bf16 *y, int ldy, int *err, cudaStream_t s) {
    using P = TcPlan<NT>;
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return DH_ECUDA;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            DH_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)P::SMEM));
            attr_set[dev] = true;
        }
    }
    const int M = N * H * W;
    dim3 grid((M + kTcBM - 1) / kTcBM, (Cout + NT - 1) / NT);
    k_conv3x3_tc<NT><<<grid, 128, P::SMEM, s>>>(x, ldx, C, N, H, W, w, b, Cout, relu ? 1 : 0, y, ldy, err);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

// ---------------------------------------------------------------- weight gradient
// dw[co][tap][ci] = sum_p dy[p][co] * x[p + tap][ci] on the tensor cores: a GEMM
// with M = 128 output channels, N = NT input channels of one tap and K =
// pixels, walked in k-blocks of one 32-pixel row segment.  The activations are
// NHWC, so both operands come MN-major (channels contiguous): TMA loads
// 32-channel x 32-pixel boxes with the 64-byte swizzle (one 64-byte row per
// pixel, 8-pixel groups 512 bytes apart, each 32-channel box 2048 bytes after
// the previous one) and the MMA reads them with its transpose bits set.  The
// tap's shift is applied to the boxes' pixel coordinates (zero filled outside
// the image), never to the channel coordinate.  One thread loads, one issues
// the MMAs, on full/empty mbarriers; each CTA sums one split of the k-blocks
// and writes its partial, which a second pass sums over the splits in order.
constexpr int kWgBK = 32;  // pixels per k-block

template <int NT>
struct WgPlan {
    static constexpr uint32_t A_BYTES = 4 * 2048;               // 128 output channels
    static constexpr uint32_t B_BYTES = (NT / 32) * 2048;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = (int)(kTcSmemBudget / STAGE) < 8 ? (int)(kTcSmemBudget / STAGE) : 8;
    static constexpr uint32_t SMEM = STAGES * STAGE + 1024;
    static constexpr uint32_t TMEM_COLS = NT;
};

// Shared-memory descriptor of an MN-major operand with the 64-byte swizzle:
// leading byte offset = distance between 32-element blocks along M/N, stride
// byte offset = distance between 8-row groups along K.
__device__ __forceinline__ uint64_t sw64_mn_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

template <int NT>
__global__ void __launch_bounds__(128, 1)
k_wgrad_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmdy, int C, int Cout, int H,
           int W, int nci, int kb_per_split, int total_kb, float *__restrict__ part, int *err) {
    using P = WgPlan<NT>;
    constexpr int S = P::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int co0 = blockIdx.x * 128;
    const int tap = blockIdx.y / nci, ci0 = (blockIdx.y - tap * nci) * NT;
    const int dyt = tap / 3 - 1, dxt = tap % 3 - 1;
    const int split = blockIdx.z;
    const int kb0 = split * kb_per_split, kb1 = min(total_kb, kb0 + kb_per_split), nkb = max(0, kb1 - kb0);
    const int segs = (W + kWgBK - 1) / kWgBK;
    const int na = min(4, (Cout - co0 + 31) / 32);  // 32-channel boxes of dy inside Cout
    const uint32_t tx = (uint32_t)na * 2048 + P::B_BYTES;
    const uint32_t sbase = smem_addr(smem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(P::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the A boxes past Cout are never loaded: zero them once in every stage
    for (int st = 0; st < S; ++st)
        for (int e = tid; e < (4 - na) * 2048 / 16; e += 128)
            *reinterpret_cast<uint4 *>(smem + st * P::STAGE + na * 2048 + e * 16) = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(&done_bar, 1);
        fence_mbar_init();
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {  // loads
        int k = 0;
        for (; k < nkb; ++k) {
            const int st = k % S;
            if (k >= S && !mbar_wait_bounded(&empty[st], (uint32_t)((k / S) - 1) & 1u, kTcWaitCycles)) {
                s_fail = 1;
                break;
            }
            const int kb = kb0 + k;
            const int row = kb / segs, seg = kb - row * segs, n = row / H, y = row - n * H, x0 = seg * kWgBK;
            unsigned char *As = smem + st * P::STAGE, *Bs = As + P::A_BYTES;
            mbar_arrive_expect_tx(&full[st], tx);
            for (int a = 0; a < na; ++a) tma_load_4d(smem_addr(As + a * 2048), &tmdy, &full[st], co0 + 32 * a, x0, y, n);
#pragma unroll
            for (int b = 0; b < NT / 32; ++b)
                tma_load_4d(smem_addr(Bs + b * 2048), &tmx, &full[st], ci0 + 32 * b, x0 + dxt, y + dyt, n);
        }
        s_issued = k;
    } else if (tid == 32) {  // MMAs: D[co][ci] += A[co][p] B[ci][p], both MN-major
        constexpr uint32_t IDESC = f16_idesc(kTcBM, NT) | (1u << 15) | (1u << 16);
        int k = 0;
        for (; k < nkb; ++k) {
            const int st = k % S;
            if (!mbar_wait_bounded(&full[st], (uint32_t)(k / S) & 1u, kTcWaitCycles)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t As = sbase + st * P::STAGE, Bs = As + P::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < kWgBK / 16; ++kk)  // 16 pixels = two 8-row groups per MMA
                tc_mma(tmem, sw64_mn_desc(As + kk * 1024, 2048, 512), sw64_mn_desc(Bs + kk * 1024, 2048, 512), IDESC,
                       (k > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[st]);
        }
        s_consumed = k;
        tc_commit(&done_bar);
    }
    bool failed = !mbar_wait_bounded(&done_bar, 0, kTcWaitCycles);
    __syncthreads();
    failed = __syncthreads_or(failed || s_fail);
    if (failed) {
        if (tid == 0) {
            for (int k = s_consumed; k < s_issued; ++k)
                mbar_wait_bounded(&full[k % S], (uint32_t)(k / S) & 1u, kTcWaitCycles);
            if (err) atomicExch(err, DH_ETIMEOUT);
        }
        __syncthreads();
    }
    tc_fence_after();

    // epilogue: warp w reads TMEM lanes 32w..32w+31 = output channels co0 + 32w + lane
    const int co = co0 + warp * 32 + lane;
    float *dst = part + (((size_t)split * Cout + co) * 9 + tap) * C + ci0;
#pragma unroll 1
    for (int c = 0; c < NT; c += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
        if (co < Cout && !failed) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (ci0 + c + j < C) dst[c + j] = nkb > 0 ? __uint_as_float(r[j]) : 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::TMEM_COLS)
                     : "memory");
}

template <int NT>
int launch_wgrad_tc(const bf16 *x, int ldx, int C, const bf16 *dy, int lddy, int Cout, int N, int H, int W,
                    float *part, int splits, int *err, cudaStream_t s) {
    using P = WgPlan<NT>;
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return DH_ECUDA;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            DH_CUDA_TRY(cudaFuncSetAttribute(k_wgrad_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)P::SMEM));
            attr_set[dev] = true;
        }
    }
    CUtensorMap mx, mdy;
    const cuuint32_t box[4] = {32, (cuuint32_t)kWgBK, 1, 1};
    {
        const cuuint64_t pitch = (cuuint64_t)ldx * sizeof(bf16);
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
        const cuuint64_t strides[3] = {pitch, pitch * (cuuint64_t)W, pitch * (cuuint64_t)W * (cuuint64_t)H};
        const int rc = encode_tiled_sw(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, x, dims, strides, box,
                                       CU_TENSOR_MAP_SWIZZLE_64B);
        if (rc) return rc;
    }
    {
        const cuuint64_t pitch = (cuuint64_t)lddy * sizeof(bf16);
        const cuuint64_t dims[4] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
        const cuuint64_t strides[3] = {pitch, pitch * (cuuint64_t)W, pitch * (cuuint64_t)W * (cuuint64_t)H};
        const int rc = encode_tiled_sw(&mdy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, dy, dims, strides, box,
                                       CU_TENSOR_MAP_SWIZZLE_64B);
        if (rc) return rc;
    }
    const int total_kb = N * H * ((W + kWgBK - 1) / kWgBK);
    const int kbps = (total_kb + splits - 1) / splits;
    const int nci = (C + NT - 1) / NT;
    dim3 grid((Cout + 127) / 128, 9 * nci, splits);
    k_wgrad_tc<NT><<<grid, 128, P::SMEM, s>>>(mx, mdy, C, Cout, H, W, nci, kbps, total_kb, part, err);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

}  // namespace

// Weight gradient on the tensor cores into part[split][co][tap][ci] (fp32),
// `splits` pixel splits; DH_EINVAL (nothing queued) when the layer is not one
// it takes (C, Cout multiples of 16, 16-byte aligned pitches and bases).
int conv3x3_wgrad_tc(const void *x, int ldx, int C, const void *dy, int lddy, int Cout, int N, int H, int W,
                     float *part, int splits, int *err, cudaStream_t s) {
    if (C % 16 || Cout % 16 || ldx % 8 || lddy % 8 || ((uintptr_t)x % 16) || ((uintptr_t)dy % 16) || splits < 1)
        return DH_EINVAL;
    const bf16 *X = (const bf16 *)x, *D = (const bf16 *)dy;
    if (C <= 32) return launch_wgrad_tc<32>(X, ldx, C, D, lddy, Cout, N, H, W, part, splits, err, s);
    if (C <= 64) return launch_wgrad_tc<64>(X, ldx, C, D, lddy, Cout, N, H, W, part, splits, err, s);
    if (C <= 128) return launch_wgrad_tc<128>(X, ldx, C, D, lddy, Cout, N, H, W, part, splits, err, s);
    return launch_wgrad_tc<256>(X, ldx, C, D, lddy, Cout, N, H, W, part, splits, err, s);
}

namespace {

// ---------------------------------------------------------------- shallow layers
// Layers with few channels (C <= 96 in, <= 96 out) are bound by reading their
// input, which the general kernel above stages once per tap.  Here a tile is
// a 128-pixel segment of one image row; its three input rows with a one-pixel
// margin (3 x 130 pixels x C) are loaded once by TMA and each of the nine taps
// is the same staging viewed through a shifted descriptor.  Below 64 channels
// the halo comes one 8-channel chunk at a time (box: 8 channels x 130 pixels x
// 3 rows = 6240 bytes, zero filled outside the image, each chunk at a 128-byte
// aligned 6272-byte slot), so that chunk q of pixel p of halo row r sits at
// q*6272 + (r*130 + p)*16 bytes: the non-swizzled K-major layout ("core
// matrices" of 8 rows x 16 bytes), in which the M = 128 rows of a tap starting
// at any pixel are core matrices 128 bytes apart (stride byte offset) and the
// two chunks of a K = 16 step are 6272 bytes apart (leading byte offset).  From
// 64 channels, channels 0-63 come in one box with the 128-byte swizzle (a
// 128-byte row per pixel; the swizzle follows the address bits, so a tap's
// descriptor simply starts at its first pixel's row), the rest in 8-channel
// chunks as above: 2 + 4 boxes per tile for 96 channels instead of 12 (the
// 16-byte rows of the chunk boxes are what limits TMA there).  For 32 input and
// 96 output channels the halo is staged by all threads with 16-byte cp.async
// copies instead (eight warps).  All the weights stay in shared memory for the
// CTA's lifetime ([tap][chunk][cout] 16-byte rows).  CTAs are persistent over
// the tiles with two TMEM accumulators and two halo stages (three for the wide
// staging where shared memory allows): the epilogue of tile i runs while the
// MMAs of tile i+1 and the loads of the following tiles proceed.  With the wide
// staging (one CTA per SM) the warps specialise: one warp loads halos as stages
// free up, one issues each tile's MMAs as its halo lands and its accumulator
// frees up, and four run the epilogues, all ordered by mbarriers (1.3-1.4x the
// single-thread hand-off with a block barrier per tile, which the 16/32-channel
// layers, three CTAs per SM, keep).
template <int C, int CO>
struct HaloPlan {
    static constexpr int QC = C / 8;                         // 8-channel chunks
    static constexpr uint32_t W_BYTES = 9u * QC * CO * 16;
    // "wide" staging (64 or more input channels): channels 0-63 of the three
    // rows come in one TMA box with the 128-byte swizzle (one 128-byte row per
    // pixel, 390 rows); the remaining channels, and all of them below 64, in
    // 8-channel boxes of the non-swizzled core-matrix layout
    static constexpr bool WIDE = C >= 64;
    static constexpr int CW = WIDE ? 64 : 0;                 // channels in the swizzled box
    static constexpr int QN = (C - CW) / 8;                  // 8-channel boxes
    static constexpr uint32_t SW_BYTES = WIDE ? (390u * 128 + 1023) / 1024 * 1024 : 0;
    static constexpr uint32_t BOX_BYTES = 3u * 130 * 16;     // one chunk of the three rows
    static constexpr uint32_t CHUNK_BYTES = (BOX_BYTES + 127) / 128 * 128;  // its slot (TMA: 128-byte aligned)
    static constexpr uint32_t TX_BYTES = (WIDE ? 390u * 128 : 0) + QN * BOX_BYTES;  // bytes a tile's loads deliver
    static constexpr uint32_t HALO_BYTES = SW_BYTES + QN * CHUNK_BYTES;
    static constexpr uint32_t W_OFF = 0;
    static constexpr uint32_t H_OFF = (W_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t H_STRIDE = (HALO_BYTES + 1023) / 1024 * 1024;
    // halo stages: three for the wide staging where they fit (the load of tile
    // i+3 then has two tiles' time to land), else two
    static constexpr int NST = (WIDE && H_OFF + 3 * H_STRIDE + 1024 <= 232448u) ? 3 : 2;
    static constexpr uint32_t SMEM = H_OFF + NST * H_STRIDE + 1024;
    static constexpr uint32_t ACC_COLS = CO <= 32 ? 32 : CO <= 64 ? 64 : 128;  // one accumulator
    static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
    static constexpr bool CP_ASYNC = !WIDE && CO >= 96;      // staging by cp.async instead of TMA
    // threads: 8 warps when all threads stage by cp.async (two warps per TMEM lane
    // quadrant in the epilogue, each with half of the output channels); with the
    // wide staging 4 epilogue warps, a load warp and an MMA warp; else 4 warps
    static constexpr int NTHR = CP_ASYNC ? 256 : (WIDE ? 192 : 128);
    static constexpr int NH = CP_ASYNC ? 2 : 1;               // epilogue warps per lane quadrant
    static_assert(C % 16 == 0 && CO % 16 == 0 && CO <= 128, "channel counts");
    static_assert((CO / NH) % 16 == 0, "each epilogue warp takes whole 16-column loads");
};

// K-major, 128-byte swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart).
// The swizzle follows the shared-memory address bits, so a start address
// anywhere on a 128-byte row boundary of a 1024-byte aligned region reads the
// rows from there on (the base offset field stays 0).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// K-major, no swizzle: leading byte offset = K-direction core-matrix stride,
// stride byte offset = M/N-direction core-matrix stride.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;  // layout type 0: no swizzle
}

template <int C, int CO>
__global__ void __launch_bounds__(HaloPlan<C, CO>::NTHR)
k_conv3x3_halo(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
               const bf16 *__restrict__ x, int ldx, int Nimg, int H, int W,
               const bf16 *__restrict__ w, const float *__restrict__ bias, int relu, bf16 *__restrict__ y, int ldy,
               int *err) {
    using P = HaloPlan<C, CO>;
    constexpr int QC = P::QC;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t tma_bar[P::NST], mma_bar[2], stage_free[P::NST], acc_free[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float s_bias[CO];
    __shared__ volatile int s_fail;
    __shared__ int s_issued, s_landed, s_mmas;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = (W + 127) / 128;
    const int T = Nimg * H * segs;
    const int G = gridDim.x;
    const int nt = (int)blockIdx.x < T ? (T - 1 - (int)blockIdx.x) / G + 1 : 0;  // tiles blockIdx.x + i*G
    const uint32_t sbase = smem_addr(smem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(P::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < P::NST; ++k) {
            mbar_init(&tma_bar[k], 1);
            mbar_init(&stage_free[k], 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&mma_bar[k], 1);
            mbar_init(&acc_free[k], 4);
        }
        fence_mbar_init();
        s_fail = 0;
        s_issued = 0;
        s_landed = 0;
        s_mmas = 0;
    }
    constexpr int NTHR = P::NTHR;
    for (int c = tid; c < CO; c += NTHR) s_bias[c] = bias ? __ldg(bias + c) : 0.f;
    // weights [co][tap][ci] -> shared [tap][chunk][co] 16-byte rows
    for (int e = tid; e < 9 * QC * CO; e += NTHR) {
        const int co = e % CO, rest = e / CO, q = rest % QC, tap = rest / QC;
        cp_async_16(sbase + P::W_OFF + (uint32_t)e * 16, w + ((size_t)co * 9 + tap) * C + 8 * q, 16u);
    }
    cp_async_commit();
    cp_async_wait<0>();
    fence_proxy_async_smem();  // the weights, written by cp.async, are read by the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // the thread that issues the loads (the MMAs) counts them, so that a CTA
    // that gives up can still let everything in flight finish
    int n_load = 0, n_load_done = 0, n_mma = 0;
    auto issue = [&](int i) {  // the halo of tile i into stage i % NST
        const int t = (int)blockIdx.x + i * G;
        const int seg = t % segs, row = t / segs, n = row / H, yy = row - n * H;
        const uint32_t hb = sbase + P::H_OFF + (uint32_t)(i % P::NST) * P::H_STRIDE;
        uint64_t *bar = &tma_bar[i % P::NST];
        mbar_arrive_expect_tx(bar, P::TX_BYTES);
        if constexpr (P::WIDE) tma_load_4d(hb, &tmw, bar, 0, seg * 128 - 1, yy - 1, n);
#pragma unroll
        for (int q = 0; q < P::QN; ++q)
            tma_load_4d(hb + P::SW_BYTES + (uint32_t)q * P::CHUNK_BYTES, &tmx, bar, P::CW + 8 * q,
                        seg * 128 - 1, yy - 1, n);
        ++n_load;
    };
    constexpr uint32_t IDESC = f16_idesc(kTcBM, CO);
    auto mmas = [&](int i) {  // the nine taps of tile i (stage i % NST) into accumulator i & 1
        const uint32_t hb = sbase + P::H_OFF + (uint32_t)(i % P::NST) * P::H_STRIDE;
        const uint32_t acc = tmem + (uint32_t)(i & 1) * P::ACC_COLS;
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;  // halo row, start pixel
            const int rowoff = dy * 130 + dx;      // first halo row (pixel) of the tap's 128 rows
            if constexpr (P::WIDE) {
                for (int kk = 0; kk < 4; ++kk) {  // channels 16kk .. 16kk+15 of the swizzled box
                    const uint32_t a = hb + (uint32_t)rowoff * 128 + 32 * kk;
                    const uint32_t b = sbase + P::W_OFF + (uint32_t)((tap * QC + 2 * kk) * CO * 16);
                    tc_mma(acc, sw128_desc(a), kmajor_desc(b, CO * 16, 128), IDESC, (tap > 0 || kk > 0) ? 1u : 0u);
                }
            }
            for (int kk = 0; kk < P::QN / 2; ++kk) {
                const uint32_t a = hb + P::SW_BYTES + (uint32_t)(2 * kk) * P::CHUNK_BYTES + (uint32_t)(rowoff * 16);
                const uint32_t b = sbase + P::W_OFF + (uint32_t)((tap * QC + P::CW / 8 + 2 * kk) * CO * 16);
                tc_mma(acc, kmajor_desc(a, P::CHUNK_BYTES, 128), kmajor_desc(b, CO * 16, 128), IDESC,
                       (tap > 0 || P::WIDE || kk > 0) ? 1u : 0u);
            }
        }
        tc_commit(&mma_bar[i & 1]);
        ++n_mma;
    };
    // all threads: the halo of tile i into stage i & 1 by cp.async (zero fill
    // outside the image), one commit group per tile.  A halo row is 130 pixels
    // x QC chunks; consecutive threads take consecutive chunks (of a pixel,
    // then of the next pixel), and each thread advances its (pixel, chunk) by
    // the thread count without dividing, from a per-row base pointer.
    auto stage = [&](int i) {
        const int t = (int)blockIdx.x + i * G;
        const int seg = t % segs, row = t / segs, n = row / H, yy = row - n * H;
        const uint32_t hb = sbase + P::H_OFF + (uint32_t)(i & 1) * P::H_STRIDE;
        const int gx0 = seg * 128 - 1;
        constexpr int PER_ROW = 130 * QC, DP = NTHR / QC, DQ = NTHR % QC;
        const int p0 = tid / QC, q0 = tid - p0 * QC;
#pragma unroll 1
        for (int r = 0; r < 3; ++r) {
            const int gy = yy + r - 1;
            const bool rowok = gy >= 0 && gy < H;
            const bf16 *rowbase = x + (size_t)(n * H + (rowok ? gy : 0)) * W * ldx;
            const uint32_t rdst = hb + (uint32_t)(r * 130) * 16;
            int p = p0, q = q0;
            for (int e = tid; e < PER_ROW; e += NTHR) {
                const int gx = gx0 + p;
                const bool ok = rowok && gx >= 0 && gx < W;
                const bf16 *src = ok ? rowbase + gx * ldx + 8 * q : x;
                cp_async_16(rdst + (uint32_t)q * P::CHUNK_BYTES + (uint32_t)p * 16, src, ok ? 16u : 0u);
                p += DP;
                q += DQ;
                if (q >= QC) {
                    q -= QC;
                    ++p;
                }
            }
        }
        cp_async_commit();
    };
    // tile i's halo has landed (thread 0)
    auto landed = [&](int i) {
        const bool ok = mbar_wait_bounded(&tma_bar[i % P::NST], (uint32_t)(i / P::NST) & 1u, kTcWaitCycles);
        if (ok) ++n_load_done;
        return ok;
    };

    // epilogue of tile i: TMEM lane = pixel of the segment; warp w reads lane
    // quadrant w % 4 (the only one it can access) and the output channels of
    // half w / 4 (eight warps with cp.async staging, four otherwise)
    auto epilogue = [&](int i, bool skip) {
        const int t = (int)blockIdx.x + i * G;
        const int seg = t % segs, row = t / segs;
        const int quad = warp & 3, half = warp >> 2;
        const int px = seg * 128 + quad * 32 + lane;
        const uint32_t acc = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(i & 1) * P::ACC_COLS;
#pragma unroll
        for (int cc = 0; cc < CO / P::NH; cc += 16) {
            const int c = half * (CO / P::NH) + cc;
            uint32_t r[16];
            tmem_ld16(acc + (uint32_t)c, r);
            if (px < W && !skip) {
                uint32_t packed[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v0 = __uint_as_float(r[2 * j]) + s_bias[c + 2 * j];
                    float v1 = __uint_as_float(r[2 * j + 1]) + s_bias[c + 2 * j + 1];
                    if (relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                    packed[j] = *reinterpret_cast<const uint32_t *>(&h2);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(y + ((size_t)row * W + px) * ldy + c);
                dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    };

    bool failed = false;
    if constexpr (P::CP_ASYNC) {
        // two commit groups whatever nt is (an empty one when there is no
        // tile 1), so that waiting for all but the newest one always means
        // that tile 0 has landed
        if (nt > 0) stage(0);
        if (nt > 1) stage(1);
        else cp_async_commit();
        if (nt > 0) {
            cp_async_wait<1>();
            fence_proxy_async_smem();  // generic-proxy copies, read by the MMAs
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                mmas(0);
            }
        }
        for (int i = 0; i < nt; ++i) {
            // the next tile's MMAs run while this tile's epilogue does
            if (i + 1 < nt) {
                cp_async_wait<0>();
                fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0 && !failed) {
                    tc_fence_after();
                    mmas(i + 1);
                }
            }
            // tile i's MMAs are done: its accumulator is ready and its stage is free
            if (!failed && !mbar_wait_bounded(&mma_bar[i & 1], (uint32_t)(i >> 1) & 1u, kTcWaitCycles)) failed = true;
            tc_fence_after();
            if (!failed && i + 2 < nt) stage(i + 2);
            epilogue(i, failed);
            tc_fence_before();
            if (__syncthreads_or(failed)) {  // accumulator i & 1 is free for tile i+2 once all pass here
                failed = true;
                break;
            }
        }
        cp_async_wait<0>();
        if (failed && tid == 0) {
            // let every MMA thread 0 issued finish (bounded) before the shared
            // and tensor memory go away
            if (n_mma > 0) mbar_wait_bounded(&mma_bar[(n_mma - 1) & 1], (uint32_t)((n_mma - 1) >> 1) & 1u, kTcWaitCycles);
            if (err) atomicExch(err, DH_ETIMEOUT);
        }
    } else if constexpr (!P::WIDE) {
        // 8-channel boxes, three CTAs per SM: thread 0 issues the loads and the
        // MMAs; the next tile's MMAs go in right behind the current ones, then
        // the stage the current tile's MMAs release is refilled
        if (tid == 0 && nt > 0) {
            for (int k = 0; k < P::NST && k < nt; ++k) issue(k);
            if (landed(0)) {
                tc_fence_after();
                mmas(0);
            } else {
                failed = true;
            }
        }
        for (int i = 0; i < nt; ++i) {
            if (tid == 0 && !failed && i + 1 < nt) {
                if (landed(i + 1)) {
                    tc_fence_after();
                    mmas(i + 1);
                } else {
                    failed = true;
                }
            }
            if (!failed && !mbar_wait_bounded(&mma_bar[i & 1], (uint32_t)(i >> 1) & 1u, kTcWaitCycles)) failed = true;
            tc_fence_after();
            if (!failed && tid == 0 && i + P::NST < nt) issue(i + P::NST);
            epilogue(i, failed);
            tc_fence_before();
            if (__syncthreads_or(failed)) {  // accumulator i & 1 is free for tile i+2 once all pass here
                failed = true;
                break;
            }
        }
        if (failed && tid == 0) {
            for (int k = n_load_done; k < n_load; ++k)
                mbar_wait_bounded(&tma_bar[k % P::NST], (uint32_t)(k / P::NST) & 1u, kTcWaitCycles);
            if (n_mma > 0) mbar_wait_bounded(&mma_bar[(n_mma - 1) & 1], (uint32_t)((n_mma - 1) >> 1) & 1u, kTcWaitCycles);
            if (err) atomicExch(err, DH_ETIMEOUT);
        }
    } else {
        // Warp roles: warps 0-3 run the epilogues, lane 0 of warp 4 the halo
        // loads, lane 0 of warp 5 the MMAs, ordered by mbarriers alone (no
        // block barrier in the loop):
        //   tma_bar[s]    the halo of the tile in stage s has landed (TMA bytes)
        //   stage_free[s] the MMAs that read stage s are done (tcgen05.commit)
        //   mma_bar[a]    accumulator a holds its tile's sums (tcgen05.commit)
        //   acc_free[a]   the four epilogue warps have read accumulator a
        // Each barrier is waited for at most one phase behind its last use,
        // so no wait can mistake an older phase for the one it wants.
        if (warp == 4) {
            if (lane == 0) {
                for (int i = 0; i < nt && !s_fail; ++i) {
                    const int st = i % P::NST;
                    if (i >= P::NST &&
                        !mbar_wait_bounded(&stage_free[st], (uint32_t)(i / P::NST - 1) & 1u, kTcWaitCycles)) {
                        s_fail = 1;
                        break;
                    }
                    issue(i);
                }
                s_issued = n_load;
            }
        } else if (warp == 5) {
            if (lane == 0) {
                for (int i = 0; i < nt && !s_fail; ++i) {
                    const int st = i % P::NST, a = i & 1;
                    if (!landed(i) ||
                        (i >= 2 && !mbar_wait_bounded(&acc_free[a], (uint32_t)((i >> 1) - 1) & 1u, kTcWaitCycles))) {
                        s_fail = 1;
                        break;
                    }
                    tc_fence_after();
                    mmas(i);                  // commits to mma_bar[a]
                    tc_commit(&stage_free[st]);  // the same MMAs free the halo stage
                }
                s_landed = n_load_done;
                s_mmas = n_mma;
            }
        } else {
            for (int i = 0; i < nt; ++i) {
                const bool ok = mbar_wait_bounded(&mma_bar[i & 1], (uint32_t)(i >> 1) & 1u, kTcWaitCycles);
                if (__any_sync(0xffffffffu, !ok)) {
                    if (lane == 0) s_fail = 1;
                    break;
                }
                tc_fence_after();
                epilogue(i, false);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_free[i & 1]);
            }
        }
        __syncthreads();
        failed = s_fail != 0;
        if (failed && tid == 0) {
            // let every load and MMA issued finish (bounded) before the shared
            // and tensor memory go away
            for (int k = s_landed; k < s_issued; ++k)
                mbar_wait_bounded(&tma_bar[k % P::NST], (uint32_t)(k / P::NST) & 1u, kTcWaitCycles);
            if (s_mmas > 0) mbar_wait_bounded(&mma_bar[(s_mmas - 1) & 1], (uint32_t)((s_mmas - 1) >> 1) & 1u, kTcWaitCycles);
            if (err) atomicExch(err, DH_ETIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::TMEM_COLS)
                     : "memory");
}

// The halo kernel's input map: bf16 NHWC activations with a pixel pitch of
// ldx elements (C of them used), as a 4D tensor (channel, x, y, image) whose
// box is 8 channels x 130 pixels x 3 rows of one image.
static int encode_halo_map(CUtensorMap *m, const bf16 *x, int ldx, int C, int N, int H, int W) {
    const cuuint64_t pitch = (cuuint64_t)ldx * sizeof(bf16);
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {pitch, pitch * (cuuint64_t)W, pitch * (cuuint64_t)W * (cuuint64_t)H};
    const cuuint32_t box[4] = {8, 130, 3, 1};
    return encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, x, dims, strides, box);
}

template <int C, int CO>
int launch_halo(const bf16 *x, int ldx, int N, int H, int W, const bf16 *w, const float *b, bool relu, bf16 *y,
                int ldy, int *err, cudaStream_t s) {
    using P = HaloPlan<C, CO>;
    if ((uintptr_t)x % 16) return DH_EINVAL;  // TMA and cp.async need a 16-byte aligned base
    CUtensorMap map, wmap;
    std::memset(&map, 0, sizeof(map));
    std::memset(&wmap, 0, sizeof(wmap));
    if (!P::CP_ASYNC && P::QN > 0) {
        const int rc = encode_halo_map(&map, x, ldx, C, N, H, W);
        if (rc) return rc;
    }
    if (P::WIDE) {
        const cuuint64_t pitch = (cuuint64_t)ldx * sizeof(bf16);
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
        const cuuint64_t strides[3] = {pitch, pitch * (cuuint64_t)W, pitch * (cuuint64_t)W * (cuuint64_t)H};
        const cuuint32_t box[4] = {64, 130, 3, 1};
        const int rc = encode_tiled_sw(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, x, dims, strides, box,
                                       CU_TENSOR_MAP_SWIZZLE_128B);
        if (rc) return rc;
    }
    static std::mutex mu;
    static int grid_cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return DH_ECUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (!grid_cache[dev]) {
        DH_CUDA_TRY(cudaFuncSetAttribute(k_conv3x3_halo<C, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P::SMEM));
        // CTAs per SM as shared memory and tensor memory allow (the CTAs are
        // independent: a grid larger than what is resident is still correct)
        int smem_sm = 0, sms = 0;
        DH_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int per_sm = smem_sm / (int)(P::SMEM + 2048);  // + static shared memory and the per-CTA reserve
        if (per_sm > (int)(512 / P::TMEM_COLS)) per_sm = 512 / P::TMEM_COLS;
        if (per_sm > 8) per_sm = 8;
        if (per_sm < 1) per_sm = 1;
        grid_cache[dev] = per_sm * sms;
    }
    const long long T = (long long)N * H * ((W + 127) / 128);
    const int grid = (int)(T < grid_cache[dev] ? T : grid_cache[dev]);
    k_conv3x3_halo<C, CO><<<grid, P::NTHR, P::SMEM, s>>>(map, wmap, x, ldx, N, H, W, w, b, relu ? 1 : 0, y, ldy,
                                                         err);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

}  // namespace

// Shallow-layer kernel for the channel pairs it is built for; DH_EINVAL
// (nothing queued) for any other.
int conv3x3_halo(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *b, int Cout,
                 bool relu, void *y, int ldy, int *err, cudaStream_t s) {
    if (ldx % 8 || ldy % 8) return DH_EINVAL;
    const bf16 *X = (const bf16 *)x, *Wt = (const bf16 *)w;
    bf16 *Y = (bf16 *)y;
#define DH_HALO(c, co) \
    if (C == c && Cout == co) return launch_halo<c, co>(X, ldx, N, H, W, Wt, b, relu, Y, ldy, err, s);
    DH_HALO(16, 32)
    DH_HALO(32, 32)
    DH_HALO(96, 32)
    DH_HALO(32, 64)
    DH_HALO(64, 64)
    DH_HALO(64, 32)
    DH_HALO(32, 96)
#undef DH_HALO
    return DH_EINVAL;
}

namespace {
}  // namespace

// Tensor-core (tcgen05) 3x3 convolution; C % 16 == 0, Cout % 16 == 0, ldx and
// ldy multiples of 8 (16-byte rows).  N tile: the smallest of 32, 64, 96,
// 128, 192, 256 that holds Cout, else 256-wide tiles.
int conv3x3_tc(const void *x, int ldx, int C, int N, int H, int W, const void *w, const float *b, int Cout, bool relu,
               void *y, int ldy, int *err, cudaStream_t s) {
    if (C % 16 || Cout % 16 || ldx % 8 || ldy % 8) return DH_EINVAL;
    const bf16 *X = (const bf16 *)x, *Wt = (const bf16 *)w;
    bf16 *Y = (bf16 *)y;
    if (tma_conv_ok(x, w, W)) {
        if (Cout <= 32) return launch_tc_tma<32>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
        if (Cout <= 64) return launch_tc_tma<64>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
        if (Cout <= 96) return launch_tc_tma<96>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
        if (Cout <= 128) return launch_tc_tma<128>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
        if (Cout <= 192) return launch_tc_tma<192>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
        return launch_tc_tma<256>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    }
    if (Cout <= 32) return launch_tc<32>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    if (Cout <= 64) return launch_tc<64>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    if (Cout <= 96) return launch_tc<96>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    if (Cout <= 128) return launch_tc<128>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    if (Cout <= 192) return launch_tc<192>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
    return launch_tc<256>(X, ldx, C, N, H, W, Wt, b, Cout, relu, Y, ldy, err, s);
}

}  // namespace dh
