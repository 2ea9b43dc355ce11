// Shared host/device helpers of the GB300 dehazing library: workspace layout,
// solver state, reflection, compensated sums and error plumbing.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dehaze.h"

namespace dh {

constexpr int kMaxDim = 32768;
constexpr long long kMaxPixels = 1LL << 28;
constexpr size_t kAlign = 256;

// ---------------------------------------------------------------- sweep tiling
// One CTA owns a TW x TH tile of one channel.  Each thread owns 4 adjacent
// columns and walks R rows; a warp covers the 128 columns of the tile.
constexpr int kTW = 128;
// The two-iteration sweep writes 120 output columns per tile (its first
// iteration covers the 128 columns around them); a sweep of depth K writes
// 128 - 8(K-1), the narrowest 104 (K = 4).
constexpr int kTW2 = 120;
constexpr int kTWmin = kTW - 8 * 3;

// ---------------------------------------------------------------- device state
// Iteration state of one image, in the workspace.
constexpr int kStallWindow = 16;  // residual-stall test of a 16-bit phase: iterations compared

struct SolveState {
    unsigned arrive;   // CTAs of the current sweep launch that have finished
    int n;             // index of the current iterate u^n
    int cur;           // buffer (0 = caller's u, 1 and 2 = workspace) holding u^n
    int done;          // 1 once the loop has stopped
    int status;        // DH_OK / DH_WNOCONV / DH_ENONFINITE
    int n_final;       // n of the returned iterate
    float rho[3];      // residual of u^n_final
    float phin2[3];    // ||Phi^c||^2
    int err;           // error raised inside a sweep (DH_ETIMEOUT), 0 if none
    int phase_start;   // first n of the current precision phase
    int depth;         // sweeps per launch of the current loop (SolveDesc::depth)
    int tb2;           // temporally blocked sweep: 1 while two iterations per tile load are taken
    float rmax[kStallWindow];  // max_c rho_n of the last iterations (ring)
    // Grid-barrier generation of the multi-iteration sweep, alone in its
    // 128-byte line so that the CTAs polling it do not contend with the
    // arrivals and state updates above.  Never reset: kernels read it first.
    unsigned gen;
    unsigned launches;  // sweep launches since the last reset (counted by CTA 0 of each)
    int pad_gen[30];
    // Item counters of the multi-iteration sweep (iteration n uses work[n & 1]),
    // in their own line: every CTA takes its items from them.
    unsigned work[2];
    int pad_work[30];
    // Deferred decision of the multi-iteration float32 sweep (three iterate
    // buffers): the iteration after n starts before the residual of u^n is
    // reduced; u^{n-1} stays in buffer cprev until that decision is known.
    int cprev;         // buffer holding u^{n-1} (3-buffer rotation)
    int pend;          // 1: the decision on u^{n-1} is being reduced
    int dstop;         // that decision: 1 = stop at n - 1
    int dstatus;       // its status when it stops
    float drho[3];     // its residual
};
static_assert(offsetof(SolveState, gen) % 128 == 0 && offsetof(SolveState, work) % 128 == 0,
              "the barrier generation and the item counters each start a 128-byte line");

// status a 16-bit phase ends with when its residual stalls (internal)
constexpr int kStatusSwitch = 100;

// Everything the loop kernels need; written to the workspace by one tiny
// kernel per call so that a cached CUDA graph can be relaunched unchanged.
struct SolveDesc {
    void *u[3];          // iterate buffers, float or 16-bit (storage); u[2]: third float buffer or null
    const float *phi;
    const float *lam;
    float *rho_hist;     // [3*(max_iter+1)] or nullptr
    float2 *part;        // per-CTA (sum, compensation) of sum F^2, [3][nblk][depth]
    SolveState *st;
    unsigned long long cond;  // cudaGraphConditionalHandle of the while node
    int use_cond;
    int vec;             // W % 4 == 0 and every plane 16-byte aligned
    int storage;         // element type of u[]: 0 float, 1 bf16, 2 f16
    int phase_stop;      // 1: stop this phase when the residual stalls
    int dirichlet;       // 1: u = 0 outside the image, else reflecting boundary
    int defer;           // 1: u[2] is set, the multi-iteration float32 sweep may defer its decisions
    int H, W;
    int max_iter;
    int depth;           // iterations per launch of the multi-iteration sweep (1 otherwise)
    int nblk;            // residual partials per channel (one per tile)
    float tol, tau, eps;
    float wg0, wg1, wg2; // Gaussian weights at offsets 0, +-1, +-2
};

// State of the atmospheric-light selection.
struct SelectState {
    unsigned prefix;   // key bits fixed so far
    unsigned krem;     // rank still to find among keys with that prefix
    unsigned key;      // the k-th largest key (after the 4 passes)
    unsigned take;     // number of keys equal to `key` that are selected
    int cutoff;        // largest index of a selected equal key
    int best;          // chosen pixel
    int clamped;
    int pad;
    double best_sum;
};

struct WsLayout {
    size_t state, desc, sel, hist, blk, phin_part, part, dc, lam, phi, ub, uc, refine, total;
    int nblk_sweep, nblk_dcp, nblk_sel, depth, tile_h;
};

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int sweep_tile_h(int depth);
int sweep_depth(const dh_params *p);
int dcp_blocks(int H, int W);
constexpr int kSelBlocks = 1024;

// Layout of the caller's workspace for an HxW image.
// Scratch of the front-end refinements (multiscale dark channel, guided
// filter) for these parameters; 0 when both are off.
size_t refine_bytes(int H, int W, const dh_params *p);

// third: a third float32 iterate buffer (uc) for the single-image sweep's
// deferred decisions (the batched solve has none).
static inline WsLayout ws_layout(int H, int W, int depth, int tile_h, size_t refine = 0, bool third = true) {
    WsLayout L;
    const size_t N = (size_t)H * W;
    L.depth = depth;
    L.tile_h = tile_h;
    // tiles of the narrowest tiling any sweep uses (128 columns, or down to
    // 104 for the temporally blocked sweeps) and the shortest (tile_h rows)
    L.nblk_sweep = ((W + kTWmin - 1) / kTWmin) * ((H + tile_h - 1) / tile_h);
    L.nblk_dcp = dcp_blocks(H, W);
    L.nblk_sel = kSelBlocks;
    size_t o = 0;
    L.state = o; o = align_up(o + sizeof(SolveState));
    L.desc = o; o = align_up(o + 2 * sizeof(SolveDesc));  // one per precision phase
    L.sel = o; o = align_up(o + sizeof(SelectState));
    L.hist = o; o = align_up(o + 256 * sizeof(unsigned));
    L.blk = o; o = align_up(o + (size_t)kSelBlocks * 16);
    L.phin_part = o; o = align_up(o + (size_t)3 * L.nblk_dcp * sizeof(float2));
    L.part = o; o = align_up(o + (size_t)3 * L.nblk_sweep * depth * sizeof(float2));
    L.dc = o; o = align_up(o + N * sizeof(float));
    L.lam = o; o = align_up(o + N * sizeof(float));
    L.phi = o; o = align_up(o + 3 * N * sizeof(float));
    L.ub = o; o = align_up(o + 3 * N * sizeof(float) + kAlign);  // f32 buffer, or two 16-bit ones
    L.uc = third ? o : 0; o = third ? align_up(o + 3 * N * sizeof(float)) : o;
    L.refine = o; o = align_up(o + refine);
    L.total = o;
    return L;
}

static inline bool shape_ok(int H, int W) {
    return H >= 1 && W >= 1 && H <= kMaxDim && W <= kMaxDim && (long long)H * W <= kMaxPixels;
}

// ---------------------------------------------------------------- device helpers
// Half-sample symmetric extension with period 2n (scipy.ndimage 'reflect').
__device__ __forceinline__ int reflect_idx(int i, int n) {
    if (i >= 0 && i < n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// Neumaier step: (s, c) += v, with the rounding error of the add kept in c.
__device__ __forceinline__ void neumaier_add(float &s, float &c, float v) {
    const float t = s + v;
    const float big = fabsf(s) >= fabsf(v) ? s : v;
    const float small = fabsf(s) >= fabsf(v) ? v : s;
    c += (big - t) + small;
    s = t;
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void neumaier_merge(float &s, float &c, float s2, float c2) {
    neumaier_add(s, c, s2);
    c += c2;
}

// Order-preserving map from float bits to unsigned (larger float => larger key).
__device__ __forceinline__ unsigned float_key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

}  // namespace dh

// Host-side error plumbing.
#define DH_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return dh::cuda_fail(e_);    \
    } while (0)

namespace dh {
int cuda_fail(cudaError_t e);
}
