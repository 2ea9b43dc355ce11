// Fixed-point solver of App. A-A for -div(D(grad u) grad u) + lambda G(u) = Phi
// (Sec. II-A), one sweep kernel per iteration:
//   F(u) = div(D grad u) - lambda G(u) + Phi,  u <- u + tau F(u)
// with the flux-form stencil of App. A-B-1 and the 5x5 Gaussian of App. A-B-2,
// plus the per-iteration residual, the stop decision and the loop engine.
#include <cmath>
#include <mutex>
#include <vector>

#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "sweep_kernels.cuh"

namespace dh {

// ------------------------------------------------------------ small kernels

// Writes the loop descriptor; `reset` starts a new solve, otherwise the
// iteration state (n, history) carries over into the next precision phase.
__global__ void k_set_desc(SolveDesc *dst, SolveDesc v, int reset) {
    *dst = v;
    SolveState *st = v.st;
    st->depth = v.depth;
    st->work[0] = st->work[1] = 0u;
    st->pend = 0;
    st->dstop = 0;
    if (!reset) return;
    st->cprev = 2;
    st->arrive = 0;
    st->n = 0;
    st->cur = 0;
    st->done = 0;
    st->status = 0;
    st->n_final = 0;
    st->err = 0;
    st->phase_start = 0;
    st->tb2 = 1;
    st->launches = 0;
}

// J = clamp(u^n, 0, 1) and u^n as float32 into u_out (skipped when u^n is
// already there: float storage, buffer 0).
template <class T>
__global__ void k_output(const SolveDesc *__restrict__ d, float *J, float *u_out) {
    const int cur = __ldcg(&d->st->cur);
    const size_t n3 = (size_t)3 * d->H * d->W;
    const T *src = static_cast<const T *>(d->u[cur]);
    const bool copy = u_out && (sizeof(T) != sizeof(float) || cur != 0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const float v = Store<T>::get(src + i);
        if (copy) u_out[i] = v;
        if (J) J[i] = fminf(fmaxf(v, 0.f), 1.f);
    }
}

template <class Tin, class Tout>
__global__ void k_convert(const Tin *__restrict__ src, Tout *__restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        Store<Tout>::put(dst + i, Store<Tin>::get(src + i));
}

// End of a 16-bit phase: its iterate u^n (in d->u[cur]) becomes float32 in `dst`.
template <class T>
__global__ void k_phase_convert(const SolveDesc *__restrict__ d, float *dst) {
    const int cur = __ldcg(&d->st->cur);
    const size_t n3 = (size_t)3 * d->H * d->W;
    const T *src = static_cast<const T *>(d->u[cur]);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = Store<T>::get(src + i);
}

// Hands the state to the float32 phase: the iterate now sits in buffer 0; a
// stalled phase continues from the same n, any other outcome stays final.
__global__ void k_phase_state(SolveState *st) {
    st->cur = 0;
    st->cprev = 2;
    st->pend = 0;
    st->arrive = 0;
    if (st->status == kStatusSwitch) {
        st->done = 0;
        st->status = 0;
        st->phase_start = st->n;
    }
}

// ------------------------------------------------------------ configuration

// Sweep variants.  tma = 0: generic kernel, one CTA per (tile, channel);
// tma = 1: persistent TMA kernel with `stages` items in flight per CTA.
struct SweepCfg {
    int R, NW, stages, tma;  // tma: 0 generic, 1 TMA (u, Phi, lambda), 2 TMA (u) + vector loads, 3 streams
    bool edge;
    int minb = 0;            // resident CTAs per SM the registers must allow (0: 16 warps' worth)
    int multi = 0;           // 1: cooperative launch of kItersPerLaunch iterations (tma == 1 only)
    int th() const { return R * NW; }
};

// Iterations one launch of a multi-iteration sweep runs at most; the graph's
// while loop relaunches it until the stop rule holds.
constexpr int kItersPerLaunch = 64;

constexpr int kMinTileH = 16;  // smallest tile height any variant uses

int sweep_depth(const dh_params *) { return 4; }  // residual levels per tile (temporally blocked sweeps)
int sweep_tile_h(int) { return kMinTileH; }

template <class T>
constexpr int storage_kind() {
    return sizeof(T) == 4 ? 0 : (Store<T>::TMA_TYPE == CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 ? 1 : 2);
}
template <class T>
static SweepFn sweep_fn(int R, int NW, bool edge) {
    return sweep_generic_fn(storage_kind<T>(), R, NW, edge);
}
template <class T>
static SweepTmaFn sweep_tma_fn(int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    return sweep_tma_fn_kind(storage_kind<T>(), R, NW, stages, tma, edge, minb, multi);
}

// Segment height (a multiple of the 20-row unroll) that minimises the waves of
// (channel, strip, segment) tasks over `warps` resident warps.
static int stream_segment(int H, int ntx, int warps) {
    int best_seg = kStreamUnroll, best_cost = 0x7fffffff;
    const int max_n = (H + kStreamUnroll - 1) / kStreamUnroll;
    for (int n = 1; n <= max_n; ++n) {
        const int seg = kStreamUnroll * ((H + kStreamUnroll * n - 1) / (kStreamUnroll * n));
        const int nseg = (H + seg - 1) / seg;
        const long long tasks = 3LL * ntx * nseg;
        const long long waves = (tasks + warps - 1) / warps;
        const long long cost = waves * (seg + 4);
        if (cost < best_cost || (cost == best_cost && seg > best_seg)) {
            best_cost = (int)cost;
            best_seg = seg;
        }
    }
    return best_seg;
}

static uint32_t tma_smem_bytes(int th, int stages, int tma, int esize) {
    const uint32_t SW = kTW + (esize == 4 ? 8 : 16), SH = th + 4;
    const uint32_t ub = SH * SW * esize, pb = tma == 1 ? th * kTW * 4 : 0;
    const uint32_t phi_off = (ub + 1023) / 1024 * 1024;
    const uint32_t stage = (phi_off + 2 * pb + 1023) / 1024 * 1024;
    return stages * stage + 1024;
}

// Sweep variants the tuner chooses from (index = dh_params.sweep_variant).
// tma: 0 generic gather, 1 TMA tiles with Phi/lambda staged, 2 TMA u tile with
// Phi/lambda vector loads, 3 per-warp row streams (R = ring slots).
static const SweepCfg kVariants[] = {
    {6, 4, 1, 1, true, 0, 1},  // 0: library default: 24-row tiles, multi-iteration launches
    {8, 4, 1, 1, true},  {8, 4, 2, 1, true},  {4, 8, 2, 1, true},  {4, 8, 1, 1, true},
    {8, 4, 1, 2, true},  {8, 4, 2, 2, true},  {4, 8, 1, 2, true},  {16, 4, 1, 2, true},
    {8, 8, 1, 2, true},  {16, 2, 2, 2, true}, {8, 4, 1, 3, true},  {8, 8, 1, 3, true},
    {16, 4, 1, 3, true}, {8, 2, 1, 3, true},  {8, 4, 1, 0, true},  {16, 4, 1, 0, true},
    {8, 8, 1, 0, true},
    {6, 4, 1, 1, true},  {4, 4, 1, 1, true},  {16, 2, 1, 1, true}, {12, 2, 1, 1, true},
    {8, 4, 1, 1, true, 5}, {6, 4, 1, 1, true, 5}, {4, 4, 1, 1, true, 6},
    // 25-28: multi-iteration cooperative launches
    {8, 4, 1, 1, true, 0, 1}, {6, 4, 1, 1, true, 5, 1}, {4, 4, 1, 1, true, 6, 1}, {6, 4, 1, 1, true, 0, 1},
    // 29-30: 16-row tiles, two stages (the next item's tiles land while this one is computed)
    {4, 4, 2, 1, true}, {4, 4, 2, 1, true, 0, 1},
    // 31-32: two iterations per tile load (120 x 16 / 120 x 24 output tiles), multi-iteration launches
    {4, 4, 1, 4, true, 0, 1}, {6, 4, 1, 4, true, 0, 1},
    // 33-35: one producer warp + NW compute warps, two stages, Phi/lambda staged, no block
    // barrier inside an iteration (tma 5), multi-iteration launches
    {4, 8, 2, 5, true, 2, 1}, {6, 4, 2, 5, true, 2, 1}, {8, 4, 2, 5, true, 2, 1},
    // 36-38: K iterations per tile load (tma 7, stages = K): 112 x 16, 112 x 24 and 104 x 16 output tiles
    {4, 4, 3, 7, true, 3, 1}, {6, 4, 3, 7, true, 2, 1}, {4, 4, 4, 7, true, 2, 1},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
constexpr int kTb2Variant = 31;  // the two-iteration sweep with 120 x 16 tiles
constexpr int kTb3Variant = 36;  // depth 3, 112 x 16 output tiles
constexpr int kTb4Variant = 38;  // depth 4, 104 x 16 output tiles

int sweep_variant_count() { return kNumVariants; }
bool sweep_variant_usable(int v, int W, bool aligned) {
    if (v < 1 || v >= kNumVariants) return false;
    return kVariants[v].tma == 0 || (aligned && W % 4 == 0);
}

// Per-device table of tuned variants by image shape and storage (dh_tune).
struct TuneEntry {
    int dev, H, W, storage, variant;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tuned;

void tune_set(int dev, int H, int W, int storage, int variant) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : g_tuned)
        if (e.dev == dev && e.H == H && e.W == W && e.storage == storage) {
            e.variant = variant;
            return;
        }
    g_tuned.push_back({dev, H, W, storage, variant});
}

int tune_get(int dev, int H, int W, int storage) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : g_tuned)
        if (e.dev == dev && e.H == H && e.W == W && e.storage == storage) return e.variant;
    return 0;
}

// Variant for this call: an explicit dh_params.sweep_variant, else the tuned
// entry for (device, shape, storage), else DH_SWEEP="R,NW,STAGES,TMA" from the
// environment (for experiments), else the default.
static SweepCfg pick_cfg(const dh_params *p, bool tma_ok, bool is16, int H, int W) {
    const bool edge = !(p->variant & DH_VAR_NO_EDGE);
    SweepCfg c = kVariants[0];
    c.edge = edge;
    if (is16) {  // 16-bit storage: 32-row tiles, multi-iteration launches (variant 1: single-iteration)
        if (tma_ok && p->sweep_variant != 1) c = SweepCfg{8, 4, 1, 1, edge, 0, 1};
        else c = SweepCfg{8, 4, 1, tma_ok ? 1 : 0, edge};
        return c;
    }
    if (!tma_ok) c.tma = 0;
    int v = p->sweep_variant;
    if (v <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) v = tune_get(dev, H, W, p->storage);
        // tb_depth: iterations per tile load requested by the caller
        const int t = v > 0 && v < kNumVariants ? kVariants[v].tma : 0;
        const int depth = t == 4 ? 2 : (t == 7 ? kVariants[v].stages : 1);
        if (p->tb_depth == 2 && depth != 2) v = kTb2Variant;
        if (p->tb_depth == 3 && depth != 3) v = kTb3Variant;
        if (p->tb_depth == 4 && depth != 4) v = kTb4Variant;
        if (p->tb_depth == 1 && depth != 1) v = 0;
    }
    if (p->boundary == DH_BOUNDARY_ZERO && v > 0 && v < kNumVariants && kVariants[v].tma == 3) v = 0;
    if (v > 0 && v < kNumVariants && (kVariants[v].tma == 0 || tma_ok)) {
        c = kVariants[v];
        c.edge = edge;
        return c;
    }
    if (const char *e = std::getenv("DH_SWEEP")) {  // "R,NW,STAGES,TMA[,MULTI[,MINB]]"
        int r, nw, st, t, mu = 0, mb = 0;
        if (std::sscanf(e, "%d,%d,%d,%d,%d,%d", &r, &nw, &st, &t, &mu, &mb) >= 4) {
            c.R = r;
            c.NW = nw;
            c.stages = st;
            c.minb = mb;
            c.tma = tma_ok ? t : 0;
            if (c.tma == 3 && p->boundary == DH_BOUNDARY_ZERO) c.tma = 1;
            c.multi = c.tma == 1 ? (mu != 0) : ((c.tma == 4 || c.tma == 5 || c.tma == 6 || c.tma == 7) ? 1 : 0);
        }
    }
    if (!c.tma && !sweep_fn<float>(c.R, c.NW, c.edge)) { c.R = 8; c.NW = 4; }
    if (!c.tma) c.stages = 1;
    if (c.tma != 1 && c.tma != 4 && c.tma != 5 && c.tma != 6 && c.tma != 7) c.multi = 0;
    if (c.tma == 0) c.minb = 0;
    return c;
}

// ------------------------------------------------------------ tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_enc_mu;

static int encode_map(CUtensorMap *m, CUtensorMapDataType dt, int esize, const void *base, int rank, int W, int H,
                      int C, int boxW, int boxH);

int encode_f32_map(CUtensorMap *m, const void *base, int rank, int W, int H, int C, int boxW, int boxH) {
    return encode_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, rank, W, H, C, boxW, boxH);
}

static int encode_map(CUtensorMap *m, CUtensorMapDataType dt, int esize, const void *base, int rank, int W, int H,
                      int C, int boxW, int boxH) {
    {
        std::lock_guard<std::mutex> lk(g_enc_mu);
        if (!g_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cuda_fail(e);
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
    }
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)C};
    cuuint64_t strides[2] = {(cuuint64_t)W * esize, (cuuint64_t)W * H * esize};
    cuuint32_t box[3] = {(cuuint32_t)boxW, (cuuint32_t)boxH, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(m, dt, rank, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DH_OK : DH_EINVAL;
}

// ------------------------------------------------------------ graph cache

struct GraphKey {
    int dev;
    const void *desc;
    const void *ptrs[5];
    int H, W, R, NW, stages, tma, edge, storage, minb, multi;
    bool operator==(const GraphKey &o) const {
        return dev == o.dev && desc == o.desc && std::memcmp(ptrs, o.ptrs, sizeof(ptrs)) == 0 && H == o.H &&
               W == o.W && R == o.R && NW == o.NW && stages == o.stages && tma == o.tma && edge == o.edge &&
               storage == o.storage && minb == o.minb && multi == o.multi;
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

struct LaunchSpec {
    void *func;
    dim3 grid, block;
    unsigned smem;
    void **args;
    int coop = 0;  // cooperative launch (all CTAs resident at once)
};

// A graph holding one while node whose body is the sweep kernel; the sweep's
// last CTA keeps the condition at 1 while the loop has to go on.
static int get_loop_graph(const GraphKey &key, const LaunchSpec &ls, GraphEntry *out) {
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
        kp.func = ls.func;
        kp.gridDim = ls.grid;
        kp.blockDim = ls.block;
        kp.sharedMemBytes = ls.smem;
        kp.kernelParams = ls.args;
        cudaGraphNode_t kn;
        err = cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp);
        if (err == cudaSuccess && ls.coop) {
            cudaLaunchAttributeValue av = {};
            av.cooperative = 1;
            err = cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeCooperative, &av);
        }
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

// Resident CTAs per SM x SMs for a persistent kernel (cached per device/kernel).
static int persistent_grid(void *func, int block, unsigned smem) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, void *>, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &e : cache)
        if (e.first.first == dev && e.first.second == func) return e.second;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, block, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const int g = per_sm * sms;
    cache.push_back({{dev, func}, g});
    return g;
}

// ------------------------------------------------------------ the solve loop

// Queues one precision phase of the fixed-point loop: descriptor `v` (its
// u[0]/u[1] hold element type T) written to desc_dev, then the sweep kernel
// repeated in a graph while loop (or from the host).
template <class T>
static int queue_loop(SolveDesc v, SolveDesc *desc_dev, bool reset, const dh_params *p, const WsLayout &L,
                      cudaStream_t s, int *launches) {
    const int H = v.H, W = v.W;
    constexpr int esize = (int)sizeof(T);
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const bool aligned = a16(v.u[0]) && a16(v.u[1]) && a16(v.phi) && a16(v.lam) && (!v.defer || a16(v.u[2]));
    // float4 Phi/lambda loads need W % 4; TMA rows of T need W * esize % 16
    v.vec = (W % 4 == 0) && aligned;
    const bool tma_ok = v.vec && (W * esize) % 16 == 0;
    v.storage = esize == 4 ? 0 : (Store<T>::TMA_TYPE == CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 ? 1 : 2);
    const SweepCfg cfg = pick_cfg(p, tma_ok, esize != 4, H, W);
    const int ntx = (W + kTW - 1) / kTW;
    CUtensorMap maps[5];
    const SolveDesc *dptr = desc_dev;
    int seg = 0;
    void *args_tma[5] = {&maps[0], &maps[1], &maps[2], &maps[3], (void *)&dptr};
    // k_sweep_tma: u buffers 0, 1, 2 (the third only with deferred decisions), Phi, lambda
    void *args_tma3[6] = {&maps[0], &maps[1], &maps[4], &maps[2], &maps[3], (void *)&dptr};
    void *args_stream[6] = {&maps[0], &maps[1], &maps[2], &maps[3], (void *)&dptr, (void *)&seg};
    void *args_gen[1] = {(void *)&dptr};
    LaunchSpec ls;
    if (cfg.tma == 3 && esize == 4) {
        // per-warp row streams over (channel, 128-column strip, segment) tasks
        int rc = encode_f32_map(&maps[0], v.u[0], 3, W, H, 3, kTW + 8, 1);
        if (!rc) rc = encode_f32_map(&maps[1], v.u[1], 3, W, H, 3, kTW + 8, 1);
        if (!rc) rc = encode_f32_map(&maps[2], v.phi, 3, W, H, 3, kTW, 1);
        if (!rc) rc = encode_f32_map(&maps[3], v.lam, 2, W, H, 1, kTW, 1);
        if (rc) return rc;
        SweepStreamFn fn = sweep_stream_fn(cfg.NW, cfg.R, cfg.edge);
        if (!fn) return DH_EINVAL;
        const unsigned smem = cfg.NW * cfg.R * kRowBytes + 1024;
        const int gmax = persistent_grid((void *)fn, cfg.NW * 32, smem);
        if (gmax <= 0) return DH_ECUDA;
        seg = stream_segment(H, ntx, gmax * cfg.NW);
        v.nblk = ntx * ((H + seg - 1) / seg);
        if (v.nblk > L.nblk_sweep) return DH_EINVAL;
        const int g = (3 * v.nblk + cfg.NW - 1) / cfg.NW;
        ls = LaunchSpec{(void *)fn, dim3(g < gmax ? g : gmax), dim3(cfg.NW * 32), smem, args_stream};
    } else if (cfg.tma == 4 && esize == 4) {
        // two iterations per tile load: 120 x TH output tiles
        const int TH = cfg.th();
        if (TH < kMinTileH) return DH_EINVAL;
        v.nblk = ((W + kTW2 - 1) / kTW2) * ((H + TH - 1) / TH);
        if (v.nblk > L.nblk_sweep || L.depth < 2) return DH_EINVAL;
        int rc = encode_f32_map(&maps[0], v.u[0], 3, W, H, 3, kTW + 8, TH + 8);
        if (!rc) rc = encode_f32_map(&maps[1], v.u[1], 3, W, H, 3, kTW + 8, TH + 8);
        if (!rc) rc = encode_f32_map(&maps[2], v.phi, 3, W, H, 3, kTW, TH + 4);
        if (!rc) rc = encode_f32_map(&maps[3], v.lam, 2, W, H, 1, kTW, TH + 4);
        if (rc) return rc;
        SweepTmaFn fn = sweep_tb2_fn(cfg.R, cfg.NW, cfg.edge);
        const unsigned smem = tb2_smem_bytes(cfg.R, cfg.NW);
        if (!fn || !smem) return DH_EINVAL;
        const int gmax = persistent_grid((void *)fn, cfg.NW * 32, smem);
        if (gmax <= 0) return DH_ECUDA;
        const int items = 3 * v.nblk;
        ls = LaunchSpec{(void *)fn, dim3(items < gmax ? items : gmax), dim3(cfg.NW * 32), smem, args_tma};
        ls.coop = 1;
        v.depth = kItersPerLaunch;
    } else if (cfg.tma == 7 && esize == 4) {
        // K = cfg.stages iterations per tile load: (128 - 8(K-1)) x TH output tiles
        const int K = cfg.stages, TH = cfg.th(), WO = kTW - 8 * (K - 1);
        if (TH < kMinTileH || K < 2 || K > 4) return DH_EINVAL;
        v.nblk = ((W + WO - 1) / WO) * ((H + TH - 1) / TH);
        if (v.nblk > L.nblk_sweep || L.depth < K) return DH_EINVAL;
        int rc = encode_f32_map(&maps[0], v.u[0], 3, W, H, 3, kTW + 8, TH + 4 * K);
        if (!rc) rc = encode_f32_map(&maps[1], v.u[1], 3, W, H, 3, kTW + 8, TH + 4 * K);
        if (!rc) rc = encode_f32_map(&maps[2], v.phi, 3, W, H, 3, kTW, TH + 4 * (K - 1));
        if (!rc) rc = encode_f32_map(&maps[3], v.lam, 2, W, H, 1, kTW, TH + 4 * (K - 1));
        if (rc) return rc;
        SweepTmaFn fn = sweep_tbk_fn(K, cfg.R, cfg.NW, cfg.edge);
        const unsigned smem = tbk_smem_bytes(K, cfg.R, cfg.NW);
        if (!fn || !smem) return DH_EINVAL;
        const int gmax = persistent_grid((void *)fn, cfg.NW * 32, smem);
        if (gmax <= 0) return DH_ECUDA;
        const int items = 3 * v.nblk;
        ls = LaunchSpec{(void *)fn, dim3(items < gmax ? items : gmax), dim3(cfg.NW * 32), smem, args_tma};
        ls.coop = 1;
        v.depth = kItersPerLaunch;
    } else if ((cfg.tma == 5 || cfg.tma == 6) && esize == 4) {
        // one producer warp and NW compute warps per CTA
        const int TH = cfg.th();
        if (TH < kMinTileH) return DH_EINVAL;
        v.nblk = ntx * ((H + TH - 1) / TH);
        if (v.nblk > L.nblk_sweep) return DH_EINVAL;
        int rc = encode_f32_map(&maps[0], v.u[0], 3, W, H, 3, kTW + 8, TH + 4);
        if (!rc) rc = encode_f32_map(&maps[1], v.u[1], 3, W, H, 3, kTW + 8, TH + 4);
        if (!rc) rc = encode_f32_map(&maps[2], v.phi, 3, W, H, 3, kTW, TH);
        if (!rc) rc = encode_f32_map(&maps[3], v.lam, 2, W, H, 1, kTW, TH);
        if (rc) return rc;
        SweepTmaFn fn = sweep_ws_fn(0, cfg.R, cfg.NW, cfg.stages, cfg.tma == 5, cfg.edge, cfg.minb, 1);
        if (!fn) return DH_EINVAL;
        const unsigned smem = tma_smem_bytes(TH, cfg.stages, cfg.tma == 5 ? 1 : 2, esize);
        const int block = (cfg.NW + 1) * 32;
        const int gmax = persistent_grid((void *)fn, block, smem);
        if (gmax <= 0) return DH_ECUDA;
        const int items = 3 * v.nblk;
        ls = LaunchSpec{(void *)fn, dim3(items < gmax ? items : gmax), dim3(block), smem, args_tma};
        ls.coop = 1;
        v.depth = kItersPerLaunch;
    } else if (cfg.tma == 1 || cfg.tma == 2) {
        const int TH = cfg.th();
        if (TH < kMinTileH) return DH_EINVAL;
        v.nblk = ntx * ((H + TH - 1) / TH);
        if (v.nblk > L.nblk_sweep) return DH_EINVAL;  // workspace sized for another tiling
        const int halo = Store<T>::HALO;
        const CUtensorMapDataType dt = (CUtensorMapDataType)Store<T>::TMA_TYPE;
        int rc = encode_map(&maps[0], dt, esize, v.u[0], 3, W, H, 3, kTW + 2 * halo, TH + 4);
        if (!rc) rc = encode_map(&maps[1], dt, esize, v.u[1], 3, W, H, 3, kTW + 2 * halo, TH + 4);
        if (!rc) rc = encode_f32_map(&maps[2], v.phi, 3, W, H, 3, kTW, TH);
        if (!rc) rc = encode_f32_map(&maps[3], v.lam, 2, W, H, 1, kTW, TH);
        if (!rc && v.defer) rc = encode_map(&maps[4], dt, esize, v.u[2], 3, W, H, 3, kTW + 2 * halo, TH + 4);
        if (!v.defer) maps[4] = maps[1];  // never read
        if (rc) return rc;
        SweepTmaFn fn = sweep_tma_fn<T>(cfg.R, cfg.NW, cfg.stages, cfg.tma, cfg.edge, cfg.minb, cfg.multi);
        if (!fn) return DH_EINVAL;
        const unsigned smem = tma_smem_bytes(TH, cfg.stages, cfg.tma, esize);
        const int gmax = persistent_grid((void *)fn, cfg.NW * 32, smem);
        if (gmax <= 0) return DH_ECUDA;
        const int items = 3 * v.nblk;
        ls = LaunchSpec{(void *)fn, dim3(items < gmax ? items : gmax), dim3(cfg.NW * 32), smem, args_tma3};
        if (cfg.multi) {
            ls.coop = 1;
            v.depth = kItersPerLaunch;
        }
    } else {
        const int TH = cfg.th();
        if (TH < kMinTileH) return DH_EINVAL;
        const int nty = (H + TH - 1) / TH;
        v.nblk = ntx * nty;
        if (v.nblk > L.nblk_sweep) return DH_EINVAL;
        SweepFn fn = sweep_fn<T>(cfg.R, cfg.NW, cfg.edge);
        if (!fn) return DH_EINVAL;
        ls = LaunchSpec{(void *)fn, dim3(ntx, nty, 3), dim3(cfg.NW * 32), 0, args_gen};
    }
    if (p->use_graph) {
        int dev = 0;
        DH_CUDA_TRY(cudaGetDevice(&dev));
        GraphKey key{dev, desc_dev, {v.u[0], v.u[1], v.phi, v.lam, v.u[2]}, H, W, cfg.R, cfg.NW, cfg.stages, cfg.tma,
                     cfg.edge ? 1 : 0, v.storage, cfg.minb, cfg.multi};
        GraphEntry ge;
        int rc = get_loop_graph(key, ls, &ge);
        if (rc != DH_OK) return rc;
        v.cond = ge.cond;
        v.use_cond = 1;
        k_set_desc<<<1, 1, 0, s>>>(desc_dev, v, reset ? 1 : 0);
        DH_CUDA_TRY(cudaGetLastError());
        DH_CUDA_TRY(cudaGraphLaunch(ge.exec, s));
    } else {
        v.use_cond = 0;
        k_set_desc<<<1, 1, 0, s>>>(desc_dev, v, reset ? 1 : 0);
        // every launch runs v.depth sweeps at most; finished ones exit at once
        const int nl = (p->max_iter + 1 + v.depth - 1) / v.depth;
        for (int n = 0; n < nl; ++n) {
            if (ls.coop)
                DH_CUDA_TRY(cudaLaunchCooperativeKernel(ls.func, ls.grid, ls.block, ls.args, ls.smem, s));
            else
                DH_CUDA_TRY(cudaLaunchKernel(ls.func, ls.grid, ls.block, ls.args, ls.smem, s));
        }
        if (launches) *launches += nl;
    }
    if (launches) *launches += 1;  // k_set_desc
    return DH_OK;
}

static int grid_for(size_t n) { return (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16); }

// The fixed-point loop from the caller's u (holding u^0, float32) to u^n
// (float32 in the caller's u) and optionally J.  st->phin2 must be set.
// Storage: float32 iterates ping-pong between the caller's u and the
// workspace buffer; 16-bit iterates between two halves of that buffer, and
// the switched forms finish with a float32 phase from the converted iterate.
int run_solve(float *u_caller, const float *phi, const float *lam, int H, int W, const dh_params *p,
              float *rho_hist, char *ws, const WsLayout &L, cudaStream_t s, float *J,
              cudaEvent_t loop_begin, cudaEvent_t loop_end, int *launches) {
    SolveDesc *desc1 = (SolveDesc *)(ws + L.desc);
    SolveDesc *desc2 = desc1 + 1;
    SolveDesc v = {};
    v.phi = phi;
    v.lam = lam;
    v.rho_hist = rho_hist;
    v.part = (float2 *)(ws + L.part);
    v.st = (SolveState *)(ws + L.state);
    v.H = H;
    v.W = W;
    v.max_iter = p->max_iter;
    v.depth = 1;
    v.tol = p->tol;
    v.tau = p->tau;
    v.eps = p->eps;
    v.dirichlet = p->boundary == DH_BOUNDARY_ZERO;
    {  // App. A-B-2: normalised 5-tap Gaussian, sigma = p->sigma
        double w[3];
        for (int k = 0; k <= 2; ++k) w[k] = exp(-(double)(k * k) / (2.0 * (double)p->sigma * p->sigma));
        const double sum = w[0] + 2.0 * (w[1] + w[2]);
        v.wg0 = (float)(w[0] / sum);
        v.wg1 = (float)(w[1] / sum);
        v.wg2 = (float)(w[2] / sum);
    }
    const size_t n3 = (size_t)3 * H * W;
    char *ub = ws + L.ub;
    float *ub32 = (float *)ub;
    const int storage = p->storage;
    const bool is16 = storage != DH_STORE_F32;
    const bool bf = storage == DH_STORE_BF16 || storage == DH_STORE_BF16_F32;
    const bool switched = storage == DH_STORE_BF16_F32 || storage == DH_STORE_F16_F32;
    int rc = DH_OK;
    if (loop_begin) DH_CUDA_TRY(cudaEventRecord(loop_begin, s));
    float *uc32 = L.uc ? (float *)(ws + L.uc) : nullptr;  // third float32 buffer (deferred decisions)
    if (!is16) {
        v.u[0] = u_caller;
        v.u[1] = ub32;
        v.u[2] = uc32;
        v.defer = uc32 != nullptr;
        v.phase_stop = 0;
        rc = queue_loop<float>(v, desc1, true, p, L, s, launches);
        if (rc) return rc;
        if (loop_end) DH_CUDA_TRY(cudaEventRecord(loop_end, s));
        k_output<float><<<grid_for(n3), 256, 0, s>>>(desc1, J, u_caller);
    } else {
        void *b0 = ub;
        void *b1 = ub + align_up(n3 * 2);
        v.u[0] = b0;
        v.u[1] = b1;
        v.phase_stop = switched ? 1 : 0;
        if (bf) {
            k_convert<float, __nv_bfloat16><<<grid_for(n3), 256, 0, s>>>(u_caller, (__nv_bfloat16 *)b0, n3);
            rc = queue_loop<__nv_bfloat16>(v, desc1, true, p, L, s, launches);
        } else {
            k_convert<float, __half><<<grid_for(n3), 256, 0, s>>>(u_caller, (__half *)b0, n3);
            rc = queue_loop<__half>(v, desc1, true, p, L, s, launches);
        }
        if (rc) return rc;
        if (launches) *launches += 1;
        if (switched) {
            if (bf)
                k_phase_convert<__nv_bfloat16><<<grid_for(n3), 256, 0, s>>>(desc1, u_caller);
            else
                k_phase_convert<__half><<<grid_for(n3), 256, 0, s>>>(desc1, u_caller);
            k_phase_state<<<1, 1, 0, s>>>(v.st);
            SolveDesc v2 = v;
            v2.u[0] = u_caller;
            v2.u[1] = ub32;
            v2.u[2] = uc32;
            v2.defer = uc32 != nullptr;
            v2.phase_stop = 0;
            rc = queue_loop<float>(v2, desc2, false, p, L, s, launches);
            if (rc) return rc;
            if (loop_end) DH_CUDA_TRY(cudaEventRecord(loop_end, s));
            k_output<float><<<grid_for(n3), 256, 0, s>>>(desc2, J, u_caller);
            if (launches) *launches += 2;
        } else {
            if (loop_end) DH_CUDA_TRY(cudaEventRecord(loop_end, s));
            if (bf)
                k_output<__nv_bfloat16><<<grid_for(n3), 256, 0, s>>>(desc1, J, u_caller);
            else
                k_output<__half><<<grid_for(n3), 256, 0, s>>>(desc1, J, u_caller);
        }
    }
    if (launches) *launches += 1;  // k_output
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int launch_output_f32(const SolveDesc *desc_dev, float *J, float *u, size_t n3, cudaStream_t s) {
    k_output<float><<<grid_for(n3), 256, 0, s>>>(desc_dev, J, u);
    DH_CUDA_TRY(cudaGetLastError());
    return DH_OK;
}

int read_solve_state(const char *ws, const WsLayout &L, SolveState *out) {
    DH_CUDA_TRY(cudaMemcpy(out, ws + L.state, sizeof(SolveState), cudaMemcpyDeviceToHost));
    return DH_OK;
}

}  // namespace dh
