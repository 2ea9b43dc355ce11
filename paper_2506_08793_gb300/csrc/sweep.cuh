// Device code shared by the single-image and batched sweep kernels: the
// face flux, packed float32 pair arithmetic, iterate storage types, the row
// walk that evaluates one fixed-point update (App. A-A, A-B), the residual
// reductions and the end-of-iteration decision.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "tma.cuh"

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
// Every rounding step is spelled out (__f*_rn, fmaf) so that no kernel
// variant's contraction choices change the result: all variants agree bit for bit.
template <bool EDGE>
__device__ __forceinline__ float face_flux(float a, float b, float eps) {
    if (!EDGE) return a;  // ablation: D == 1
    const float s = fmaf(a, a, __fmul_rn(b, b));
    return __fmul_rn(a, rcp_approx(__fadd_rn(sqrt_approx(s), eps)));
}

__device__ __forceinline__ float half_diff(float p, float m) { return __fmul_rn(0.5f, __fsub_rn(p, m)); }

// 5-tap symmetric Gaussian: w2 (v-2 + v+2) + w1 (v-1 + v+1) + w0 v0
__device__ __forceinline__ float gauss5(float vm2, float vm1, float v0, float vp1, float vp2, float wg0, float wg1,
                                        float wg2) {
    return fmaf(wg2, __fadd_rn(vm2, vp2), fmaf(wg1, __fadd_rn(vm1, vp1), __fmul_rn(wg0, v0)));
}

__device__ __forceinline__ int ld_state_int(const int *p) { return __ldcg(p); }

// stop_status' value for "the residual meets tol" (internal; reported as DH_OK)
constexpr int kStatusConverged = 101;

// Reduces the per-tile partials of the launch (last CTA only), decides whether
// to stop, advances the state and sets the graph's while condition.  Every
// thread of the CTA keeps U partial loads per channel in flight; the sums are
// merged in a fixed order (thread stride, then lanes, then warps).  Thread 0
// loads the state fields it decides with before the partials, so that their
// latency overlaps the reduction; it returns the index of the next iterate
// (n + 1 when the loop goes on, n when it stops; other threads: unspecified).
// A multi-iteration launch sets the while condition only at its last
// iteration (last_in_launch); a caller whose arrival was an acquire-release
// atomic skips the opening fence (acquired), and one that publishes the state
// with a release store itself skips the closing fence (fence = false).
template <int U = 8>  // partial loads per channel in flight per thread
static __device__ int finish_iteration(const SolveDesc *d, SolveState *st, bool last_in_launch = true,
                                       bool fence = true, bool acquired = false) {
    __shared__ float2 wsum[3][32];
    __shared__ float sq[3];
    const int tid = threadIdx.x, nt = blockDim.x, w = tid >> 5, lane = tid & 31, nw = nt >> 5;
    if (!acquired) fence_acq_rel_gpu();  // the partials of every CTA that arrived before this one
    int n = 0, cur = 0, err = 0, max_iter = 0;
    float phin2[3] = {0.f, 0.f, 0.f}, tol = 0.f;
    if (tid == 0) {
        n = ld_state_int(&st->n);
        cur = ld_state_int(&st->cur);
        err = ld_state_int(&st->err);
        for (int c = 0; c < 3; ++c) phin2[c] = __ldcg(&st->phin2[c]);
        tol = d->tol;
        max_iter = d->max_iter;
    }
    const int nblk = d->nblk;
    const float2 *part = d->part;
    float s[3] = {0.f, 0.f, 0.f}, cc[3] = {0.f, 0.f, 0.f};
    for (int b0 = tid; b0 < nblk; b0 += U * nt) {
        float2 p[3][U];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int b = b0 + j * nt;
                p[c][j] = b < nblk ? __ldcg(part + (size_t)c * nblk + b) : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < U; ++j) neumaier_merge(s[c], cc[c], p[c][j].x, p[c][j].y);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[c], off);
            const float c2 = __shfl_down_sync(0xffffffffu, cc[c], off);
            neumaier_merge(s[c], cc[c], s2, c2);
        }
        if (lane == 0) wsum[c][w] = make_float2(s[c], cc[c]);
    }
    __syncthreads();
    if (tid < 3) {
        float a = wsum[tid][0].x, b = wsum[tid][0].y;
        for (int k = 1; k < nw; ++k) neumaier_merge(a, b, wsum[tid][k].x, wsum[tid][k].y);
        sq[tid] = a + b;
    }
    __syncthreads();
    if (tid != 0) return 0;
    float *rho_hist = d->rho_hist;
    float worst = 0.f;
    bool finite = true;
    float rho[3];
    for (int c = 0; c < 3; ++c) {
        const float pn = phin2[c];
        rho[c] = pn > 0.f ? sqrtf(sq[c] / pn) : sqrtf(sq[c]);
        if (!isfinite(rho[c])) finite = false;
        else worst = fmaxf(worst, rho[c]);
        if (rho_hist) rho_hist[3 * n + c] = rho[c];
    }
    const bool conv = finite && worst <= tol;
    // a 16-bit phase ends once its residual falls by less than 2 % over
    // kStallWindow iterations (the storage quantum has been reached)
    bool stall = false;
    if (d->phase_stop && finite) {
        const int slot = n % kStallWindow;
        if (n - ld_state_int(&st->phase_start) >= kStallWindow && worst > 0.98f * __ldcg(&st->rmax[slot])) stall = true;
        st->rmax[slot] = worst;
    }
    unsigned cont = 1;
    int next = n + 1;
    if (err || conv || !finite || n >= max_iter || stall) {
        st->done = 1;
        st->n_final = n;
        st->status = err ? err
                         : (!finite ? DH_ENONFINITE
                                    : (conv ? DH_OK : (n >= max_iter ? DH_WNOCONV : kStatusSwitch)));
        for (int c = 0; c < 3; ++c) st->rho[c] = rho[c];
        cont = 0;
        next = n;
    } else {
        st->n = n + 1;
        st->cur = cur ^ 1;
    }
    st->arrive = 0;
    if (fence) __threadfence();
    // the condition was cleared when the launch began: only a launch that goes
    // on after its last iteration sets it
    if (d->use_cond && cont && last_in_launch) cudaGraphSetConditional(d->cond, 1u);
    return next;
}

// ---------------------------------------------------------------- deferred decisions
// The multi-iteration float32 sweep with a third iterate buffer: the last CTA
// at the grid barrier of iteration n lets iteration n + 1 start at once and
// reduces the residual of u^n while the others sweep; the decision on u^n is
// read at the next barrier.  Iteration n + 1 writes u^{n+2} into the buffer
// that holds neither u^n nor u^{n+1}, so u^n is still there when that decision
// stops the loop at n (one sweep is then spent in vain).  The partials of
// iteration n go to part + (n & 1) * 3 * nblk, so those being reduced are
// never overwritten by the iteration running meanwhile.  The last iteration of
// a launch decides at once (a launch leaves no decision pending).

// sq[c] = the residual's sum of squares of channel c over the nblk tile
// partials at `part` (layout [3][nblk]), in a fixed order; every thread of
// the CTA takes part; sq (shared) is valid for all of them on return.
template <int U>
static __device__ void block_residual_sq(const float2 *part, int nblk, float *sq) {
    __shared__ float2 wsum[3][32];
    const int tid = threadIdx.x, nt = blockDim.x, w = tid >> 5, lane = tid & 31, nw = nt >> 5;
    float s[3] = {0.f, 0.f, 0.f}, cc[3] = {0.f, 0.f, 0.f};
    for (int b0 = tid; b0 < nblk; b0 += U * nt) {
        float2 p[3][U];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int b = b0 + j * nt;
                p[c][j] = b < nblk ? __ldcg(part + (size_t)c * nblk + b) : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < U; ++j) neumaier_merge(s[c], cc[c], p[c][j].x, p[c][j].y);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[c], off);
            const float c2 = __shfl_down_sync(0xffffffffu, cc[c], off);
            neumaier_merge(s[c], cc[c], s2, c2);
        }
        if (lane == 0) wsum[c][w] = make_float2(s[c], cc[c]);
    }
    __syncthreads();
    if (tid < 3) {
        float a = wsum[tid][0].x, b = wsum[tid][0].y;
        for (int k = 1; k < nw; ++k) neumaier_merge(a, b, wsum[tid][k].x, wsum[tid][k].y);
        sq[tid] = a + b;
    }
    __syncthreads();
}

// The stop rule on u^n from its sums of squares (thread 0): residual per
// channel, finiteness, tolerance, max_iter, a sweep's error.  Returns the
// status to stop with, or 0 to go on.
__device__ __forceinline__ int stop_status(const SolveDesc *d, const SolveState *st, int n, const float *sq,
                                           const float *phin2, float *rho) {
    float worst = 0.f;
    bool finite = true;
    for (int c = 0; c < 3; ++c) {
        const float pn = phin2[c];
        rho[c] = pn > 0.f ? sqrtf(sq[c] / pn) : sqrtf(sq[c]);
        if (!isfinite(rho[c])) finite = false;
        else worst = fmaxf(worst, rho[c]);
        if (d->rho_hist) d->rho_hist[3 * n + c] = rho[c];
    }
    const int err = ld_state_int(&st->err);
    if (err) return err;
    if (!finite) return DH_ENONFINITE;
    if (worst <= d->tol) return kStatusConverged;
    if (n >= d->max_iter) return DH_WNOCONV;
    return 0;
}

// Grid barrier of the deferring sweep, last CTA (every thread).  partn: the
// partials of the iteration just finished (the residual of u^n).  Returns 0
// when the loop stops here, 1 when it goes on with no decision pending (the
// launch's last iteration, decided at once), 2 when it goes on and the caller
// must reduce partn with defer_reduce after releasing the others.
template <int U>
static __device__ int defer_barrier(const SolveDesc *d, SolveState *st, bool last_in_launch, const float2 *partn) {
    __shared__ int s_mode;
    __shared__ float sq[3];
    int n = 0, cur = 0, cprev = 0;
    float phin2[3] = {0.f, 0.f, 0.f};
    if (threadIdx.x == 0) {
        n = ld_state_int(&st->n);
        cur = ld_state_int(&st->cur);
        cprev = ld_state_int(&st->cprev);
        for (int c = 0; c < 3; ++c) phin2[c] = __ldcg(&st->phin2[c]);
        int mode;
        if (ld_state_int(&st->pend) && ld_state_int(&st->dstop)) {
            // the decision on u^{n-1} stops the loop: u^{n-1} is still in cprev
            const int status = ld_state_int(&st->dstatus);
            st->done = 1;
            st->n = st->n_final = n - 1;
            st->status = status == kStatusConverged ? DH_OK : status;
            for (int c = 0; c < 3; ++c) st->rho[c] = __ldcg(&st->drho[c]);
            st->cur = cprev;
            st->pend = 0;
            mode = 0;
        } else if (last_in_launch) {
            mode = 1;
        } else {  // go on with u^{n+1}; u^n stays in cur until its decision is read
            st->cprev = cur;
            st->cur = 3 - cur - cprev;
            st->n = n + 1;
            st->pend = 1;
            mode = 2;
        }
        st->arrive = 0;
        s_mode = mode;
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode != 1) return mode;
    block_residual_sq<U>(partn, d->nblk, sq);
    if (threadIdx.x != 0) return 1;
    float rho[3];
    const int status = stop_status(d, st, n, sq, phin2, rho);
    st->pend = 0;
    if (status) {
        st->done = 1;
        st->n_final = n;
        st->status = status == kStatusConverged ? DH_OK : status;
        for (int c = 0; c < 3; ++c) st->rho[c] = rho[c];
        return 0;
    }
    st->cprev = cur;
    st->cur = 3 - cur - cprev;
    st->n = n + 1;
    if (d->use_cond) cudaGraphSetConditional(d->cond, 1u);  // the launch ends, the loop goes on
    return 1;
}

// The deferred half (every thread of the CTA that returned 2 from
// defer_barrier, after the release): the stop rule on u^{n_done} from partn,
// published for the next barrier in st->dstop / dstatus / drho.
template <int U>
static __device__ void defer_reduce(const SolveDesc *d, SolveState *st, int n_done, const float2 *partn) {
    __shared__ float sq[3];
    float phin2[3] = {0.f, 0.f, 0.f};
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) phin2[c] = __ldcg(&st->phin2[c]);
    block_residual_sq<U>(partn, d->nblk, sq);
    if (threadIdx.x == 0) {
        float rho[3];
        const int status = stop_status(d, st, n_done, sq, phin2, rho);
        st->dstatus = status;
        for (int c = 0; c < 3; ++c) st->drho[c] = rho[c];
        st->dstop = status != 0;
    }
}

// The loop ends unless a launch's last CTA sets the condition back to 1, so a
// launch that failed to count its CTAs cannot spin forever.  CTA (0,0,0)
// clears it before it arrives, hence before the last CTA decides.
__device__ __forceinline__ void clear_condition(const SolveDesc *d) {
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) {
        atomicAdd(&d->st->launches, 1u);
        if (d->use_cond) {
            cudaGraphSetConditional(d->cond, 0);
            __threadfence();
        }
    }
}

// Counts this CTA in and lets the last one finish the iteration.
__device__ __forceinline__ void arrive_and_finish(const SolveDesc *d, SolveState *st, int *s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        *s_last = prev == total - 1u;
    }
    __syncthreads();
    if (*s_last) finish_iteration(d, st);
}

// Deterministic block reduction of a (sum, compensation) pair; thread 0 gets it.
template <int NW>
__device__ __forceinline__ float2 block_pair_sum(float rs, float rc, float2 *red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 16; off; off >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, rs, off);
        const float c2 = __shfl_down_sync(0xffffffffu, rc, off);
        neumaier_merge(rs, rc, s2, c2);
    }
    if (lane == 0) red[w] = make_float2(rs, rc);
    __syncthreads();
    float a = red[0].x, b = red[0].y;
#pragma unroll
    for (int k = 1; k < NW; ++k) neumaier_merge(a, b, red[k].x, red[k].y);
    return make_float2(a, b);
}

// Packed float32 pairs (Blackwell f32x2 ALU ops).  Each lane of a pair is an
// IEEE round-to-nearest operation, the same as the scalar __f*_rn / fmaf.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// face_flux on two faces at once (same rounding as the scalar form)
template <bool EDGE>
__device__ __forceinline__ float2 face_flux2(float2 a, float2 b, float2 eps2) {
    if (!EDGE) return a;
    const float2 s = fma2(a, a, mul2(b, b));
    const float2 q = add2(make_float2(sqrt_approx(s.x), sqrt_approx(s.y)), eps2);
    return mul2(a, make_float2(rcp_approx(q.x), rcp_approx(q.y)));
}

// Iterate storage: float, or bf16 / f16 converted to float on load and
// rounded to nearest-even on store.  HALO = columns of tile halo on each side
// as loaded by TMA (a 16-bit TMA row must start on a multiple of 8 columns).
template <class T>
struct Store;
template <>
struct Store<float> {
    static constexpr int HALO = 4;
    static constexpr int TMA_TYPE = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    __device__ static void read12(const float *p, float *v) {  // 16-byte aligned
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *reinterpret_cast<const float4 *>(p + 4);
        const float4 c = *reinterpret_cast<const float4 *>(p + 8);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
        v[6] = b.z; v[7] = b.w; v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
    }
    __device__ static void write4(float *p, float a, float b, float c, float d) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
    __device__ static float get(const float *p) { return *p; }
    __device__ static void put(float *p, float v) { *p = v; }
};
template <>
struct Store<__nv_bfloat16> {
    static constexpr int HALO = 8;
    static constexpr int TMA_TYPE = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    __device__ static void w2(unsigned w, float &lo, float &hi) {
        lo = __uint_as_float(w << 16);
        hi = __uint_as_float(w & 0xffff0000u);
    }
    __device__ static void read12(const __nv_bfloat16 *p, float *v) {  // 8-byte aligned
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        const uint2 b = *reinterpret_cast<const uint2 *>(p + 4);
        const uint2 c = *reinterpret_cast<const uint2 *>(p + 8);
        w2(a.x, v[0], v[1]); w2(a.y, v[2], v[3]); w2(b.x, v[4], v[5]);
        w2(b.y, v[6], v[7]); w2(c.x, v[8], v[9]); w2(c.y, v[10], v[11]);
    }
    __device__ static void write4(__nv_bfloat16 *p, float a, float b, float c, float d) {
        const __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
        uint2 q;
        q.x = *reinterpret_cast<const unsigned *>(&x);
        q.y = *reinterpret_cast<const unsigned *>(&y);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    __device__ static float get(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static void put(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Store<__half> {
    static constexpr int HALO = 8;
    static constexpr int TMA_TYPE = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    __device__ static void w2(unsigned w, float &lo, float &hi) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        lo = f.x;
        hi = f.y;
    }
    __device__ static void read12(const __half *p, float *v) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        const uint2 b = *reinterpret_cast<const uint2 *>(p + 4);
        const uint2 c = *reinterpret_cast<const uint2 *>(p + 8);
        w2(a.x, v[0], v[1]); w2(a.y, v[2], v[3]); w2(b.x, v[4], v[5]);
        w2(b.y, v[6], v[7]); w2(c.x, v[8], v[9]); w2(c.y, v[10], v[11]);
    }
    __device__ static void write4(__half *p, float a, float b, float c, float d) {
        const __half2 x = __floats2half2_rn(a, b), y = __floats2half2_rn(c, d);
        uint2 q;
        q.x = *reinterpret_cast<const unsigned *>(&x);
        q.y = *reinterpret_cast<const unsigned *>(&y);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    __device__ static float get(const __half *p) { return __half2float(*p); }
    __device__ static void put(__half *p, float v) { *p = __float2half_rn(v); }
};

// One row of u for a lane, as the pairs the stencil needs: odd pairs
// o0 = (x-1, x), o1 = (x+1, x+2), o2 = (x+3, x+4) and even pairs
// e1 = (x, x+1), e2 = (x+2, x+3).
struct RowU {
    float2 o0, e1, o1, e2, o2;
};

// One warp's walk over tile rows [r0, r0+R) for its lane's 4 columns.
// `s` is the u^n tile in shared memory: row stride SW floats, tile row ty at
// smem row ty+2, the lane's first column at smem column 4*lane+4.  Every x-
// and y-face flux and every horizontally filtered row is computed once and
// kept in rolling registers; arithmetic runs on float32 pairs.
// pl(ty, ph, la) supplies Phi and lambda for the row; sink(ty, nu, F)
// consumes u^{n+1} and F.
template <int R, int SW, class T, bool EDGE, class PL, class SINK>
__device__ __forceinline__ void walk_rows(const T *__restrict__ s, int r0, int lane, float eps, float tau,
                                          float wg0, float wg1, float wg2, PL pl, SINK sink) {
    const int sc = 4 * lane + (Store<T>::HALO - 4);  // smem column of x-4
    const float2 W0 = make_float2(wg0, wg0), W1 = make_float2(wg1, wg1), W2 = make_float2(wg2, wg2);
    const float2 E2 = make_float2(eps, eps), HALF = make_float2(0.5f, 0.5f), TAU = make_float2(tau, tau);
    RowU uu[4];       // u at tile rows r0-1+k (mod 4)
    float2 gh[5][2];  // horizontal Gaussian at tile rows r0-2+k (mod 5), columns (x, x+1), (x+2, x+3)
    float2 fyu[2];    // y-face fluxes above the current row

    auto gauss = [&](float2 m2, float2 m1, float2 c0, float2 p1, float2 p2) {
        return fma2(W2, add2(m2, p2), fma2(W1, add2(m1, p1), mul2(W0, c0)));
    };
    auto load_row = [&](int tr, RowU &u, float2 *g) {
        float v[12];  // columns x-4 .. x+7
        Store<T>::read12(s + (tr + 2) * SW + sc, v);
        const float2 e0 = make_float2(v[2], v[3]), e3 = make_float2(v[8], v[9]);
        u.o0 = make_float2(v[3], v[4]);
        u.e1 = make_float2(v[4], v[5]);
        u.o1 = make_float2(v[5], v[6]);
        u.e2 = make_float2(v[6], v[7]);
        u.o2 = make_float2(v[7], v[8]);
        g[0] = gauss(e0, u.o0, u.e1, u.o1, u.e2);
        g[1] = gauss(u.e1, u.o1, u.e2, u.o2, e3);
    };
    // y-face fluxes below row `a` (between a and b), tangential difference on row a
    auto yfaces = [&](const RowU &a, const RowU &b, float2 *f) {
        f[0] = face_flux2<EDGE>(sub2(b.e1, a.e1), mul2(HALF, sub2(a.o1, a.o0)), E2);
        f[1] = face_flux2<EDGE>(sub2(b.e2, a.e2), mul2(HALF, sub2(a.o2, a.o1)), E2);
    };

    {
        RowU dummy;
        load_row(r0 - 2, dummy, gh[0]);
        load_row(r0 - 1, uu[0], gh[1]);
        load_row(r0, uu[1], gh[2]);
        load_row(r0 + 1, uu[2], gh[3]);
        yfaces(uu[0], uu[1], fyu);  // y-face at r0 - 1/2
    }

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ty = r0 + i;
        const RowU &um = uu[(i + 0) & 3];
        const RowU &u0 = uu[(i + 1) & 3];
        const RowU &up = uu[(i + 2) & 3];
        load_row(ty + 2, uu[(i + 3) & 3], gh[(i + 4) % 5]);
        const float2 *g_m2 = gh[(i + 0) % 5], *g_m1 = gh[(i + 1) % 5], *g_0 = gh[(i + 2) % 5];
        const float2 *g_p1 = gh[(i + 3) % 5], *g_p2 = gh[(i + 4) % 5];
        float ph[4], la[4];
        pl(ty, ph, la);
        // x-faces (x-1/2, x+1/2), (x+3/2, x+5/2) and x+7/2; tangential difference at the left cell
        const float2 fxA = face_flux2<EDGE>(sub2(u0.e1, u0.o0), mul2(HALF, sub2(up.o0, um.o0)), E2);
        const float2 fxB = face_flux2<EDGE>(sub2(u0.e2, u0.o1), mul2(HALF, sub2(up.o1, um.o1)), E2);
        const float fx4 = face_flux<EDGE>(__fsub_rn(u0.o2.y, u0.o2.x), half_diff(up.o2.x, um.o2.x), eps);
        float2 fyd[2];
        yfaces(u0, up, fyd);
        // the negated divergence -div(D grad u), by swapping the operands of
        // every difference (exact: round-to-nearest is odd-symmetric)
        const float2 ndxA = make_float2(__fsub_rn(fxA.x, fxA.y), __fsub_rn(fxA.y, fxB.x));
        const float2 ndxB = make_float2(__fsub_rn(fxB.x, fxB.y), __fsub_rn(fxB.y, fx4));
        const float2 ndvA = add2(ndxA, sub2(fyu[0], fyd[0]));
        const float2 ndvB = add2(ndxB, sub2(fyu[1], fyd[1]));
        const float2 GA = gauss(g_m2[0], g_m1[0], g_0[0], g_p1[0], g_p2[0]);
        const float2 GB = gauss(g_m2[1], g_m1[1], g_0[1], g_p1[1], g_p2[1]);
        // F = Phi - (lambda G - div): the same roundings as (div - lambda G) + Phi
        const float2 FA = sub2(make_float2(ph[0], ph[1]), fma2(make_float2(la[0], la[1]), GA, ndvA));
        const float2 FB = sub2(make_float2(ph[2], ph[3]), fma2(make_float2(la[2], la[3]), GB, ndvB));
        const float2 nA = fma2(TAU, FA, u0.e1);
        const float2 nB = fma2(TAU, FB, u0.e2);
        fyu[0] = fyd[0];
        fyu[1] = fyd[1];
        const float nu[4] = {nA.x, nA.y, nB.x, nB.y};
        const float F[4] = {FA.x, FA.y, FB.x, FB.y};
        sink(ty, nu, F);
    }
}


// Reflecting boundary on a staged tile: the cells one or two rows / columns
// outside the image (zero-filled by TMA) take the value of their half-sample
// reflection, which always lies inside the image and inside the tile.  Only
// the (at most four) border rows and columns of the tile are visited: rows with
// gy in {-2, -1, H, H+1} over all columns whose gx is inside the image or is
// itself such a border column (corners), then border columns over the rows
// inside the image.  Tile row r is image row ry0 + r, column q image column
// cx0 + q.  The sources are never written, so one pass in any order suffices.
template <class T>
__device__ __forceinline__ void reflect_border(T *s, int stride, int ncols, int nrows, int cx0, int ry0, int H,
                                               int W) {
    // the border rows / columns, one byte each (tiles are under 256 cells a
    // side), packed in a register rather than a local-memory array
    unsigned rows = 0, cols = 0;
    int nr = 0, nc = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int g = k < 2 ? k - 2 : H + k - 2;
        const int r = g - ry0;
        if (r >= 0 && r < nrows && (g < 0 || g >= H)) rows |= (unsigned)r << (8 * nr++);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int g = k < 2 ? k - 2 : W + k - 2;
        const int q = g - cx0;
        if (q >= 0 && q < ncols && (g < 0 || g >= W)) cols |= (unsigned)q << (8 * nc++);
    }
    const int nrow_cells = nr * ncols, total = nrow_cells + nc * nrows;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int r, q;
        if (e < nrow_cells) {
            const int k = e / ncols;
            r = (int)((rows >> (8 * k)) & 0xffu);
            q = e - k * ncols;
            const int gx = cx0 + q;
            const bool fx = gx == -2 || gx == -1 || gx == W || gx == W + 1;
            if (!(fx || (gx >= 0 && gx < W))) continue;
        } else {
            const int e2 = e - nrow_cells, k = e2 / nrows;
            q = (int)((cols >> (8 * k)) & 0xffu);
            r = e2 - k * nrows;
            const int gy = ry0 + r;
            if (gy < 0 || gy >= H) continue;  // rows outside were done above (corners included)
        }
        const int sy = reflect_idx(ry0 + r, H) - ry0, sx = reflect_idx(cx0 + q, W) - cx0;
        s[r * stride + q] = s[sy * stride + sx];
    }
}

// Shared-memory plan of the TMA sweep: per stage the u^n tile with its halo,
// the Phi tile and the lambda tile, each 1024-byte aligned.
template <int TH, bool PL_SMEM, class T>
struct TmaPlan {
    static constexpr int SW = kTW + 2 * Store<T>::HALO;
    static constexpr int SH = TH + 4;
    static constexpr uint32_t U_BYTES = SH * SW * sizeof(T);
    static constexpr uint32_t P_BYTES = PL_SMEM ? TH * kTW * 4 : 0;
    static constexpr uint32_t U_OFF = 0;
    static constexpr uint32_t PHI_OFF = (U_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t LAM_OFF = PHI_OFF + P_BYTES;
    static constexpr uint32_t STAGE = (LAM_OFF + P_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t TX = U_BYTES + 2 * P_BYTES;
};

constexpr long long kWaitLimitCycles = 4000000000LL;  // about 2 s at 2 GHz

}  // namespace dh
