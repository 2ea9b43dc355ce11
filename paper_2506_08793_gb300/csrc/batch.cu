// Batched dehazing of images of uneven sizes.  The front end runs per image;
// the fixed-point loops of all images share one CUDA graph while loop whose
// body is a single persistent sweep launch over the (tile, channel) items of
// every image that is still iterating.  Each image stops on its own residual
// (App. A-A, stop rule as in the single-image path); the launch's last CTA
// compacts the list of active images and ends the loop when it is empty.
#include <cstring>
#include <mutex>
#include <vector>

#include "sweep.cuh"

namespace dh {

int launch_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out, cudaStream_t s);
int launch_transmission(const float *I, int H, int W, const dh_params *p, const float *A, float *td, float *t,
                        float *lam, float *phi, float *u0, float2 *phin_part, void *scratch, cudaStream_t s);
int launch_phin_final(const float2 *part, int H, int W, SolveState *st, cudaStream_t s);
int launch_select_A(const float *I, const float *dc, int H, int W, int permille, float *A,
                    long long *index_out, char *ws, const WsLayout &L, cudaStream_t s);
int launch_output_f32(const SolveDesc *desc_dev, float *J, float *u, size_t n3, cudaStream_t s);
int encode_f32_map(CUtensorMap *m, const void *base, int rank, int W, int H, int C, int boxW, int boxH);
int encode_tiled(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                 const cuuint64_t *strides, const cuuint32_t *box);
int sweep_tile_h(int depth);
int warm_group_size(int H, int W);
size_t warm_net_bytes(int base, int n, int H, int W);
int warm_u0_group(const float *params, int base, int n, const float *const *I, const float *const *t,
                  const float *const *A, const float *const *phi, const float *const *lam, float *const *u0, int H,
                  int W, void *nws, size_t nws_bytes, cudaStream_t s);

// The warm-start network of dh_dehaze_batch_warm and the workspace of its forwards.
struct WarmNet {
    const float *params;
    int base;
    void *ws;
    size_t ws_bytes;
};
constexpr int kWarmForwardLaunches = 36;  // weight packing (14), input packing, 14 convolutions, 3 pools,
                                          // 3 upsamplings, head; plus u0 = y / lambda per image

// Same-shape images of a batch in order of first appearance, cut into groups
// of at most warm_group_size(H, W) images: one network forward per group.
static std::vector<std::vector<int>> warm_groups(int n, const dh_image *imgs) {
    std::vector<std::vector<int>> shapes, out;
    for (int i = 0; i < n; ++i) {
        bool placed = false;
        for (auto &g : shapes)
            if (imgs[g[0]].H == imgs[i].H && imgs[g[0]].W == imgs[i].W) {
                g.push_back(i);
                placed = true;
                break;
            }
        if (!placed) shapes.push_back({i});
    }
    for (auto &g : shapes) {
        const int cap = warm_group_size(imgs[g[0]].H, imgs[g[0]].W);
        for (size_t k = 0; k < g.size(); k += cap)
            out.emplace_back(g.begin() + k, g.begin() + (k + cap < g.size() ? k + cap : g.size()));
    }
    return out;
}

constexpr int kMaxBatch = 256;
constexpr int kBR = 6, kBNW = 4, kBTH = kBR * kBNW;  // 128 x 24 tiles, 4 warps, 5 CTAs per SM
constexpr int kBChunk = 3;  // items a CTA takes at a time: the three channels of one tile

// Per-image loop data in device memory.
struct __align__(128) BImg {
    CUtensorMap tm[4];  // u buffer 0, u buffer 1, Phi, lambda (when tma)
    SolveDesc d;        // per-image descriptor (use_cond = 0: the batch owns the loop)
    int ntx, items, tma, pad;
};

struct BatchHdr {
    BImg *imgs;
    int nimg;
    int nactive;
    int iter;          // loop iterations so far (odd ones walk the items in reverse)
    unsigned arrive;
    unsigned work;     // chunks handed out in the current launch beyond the first G
    int use_cond;
    unsigned long long cond;
    int active[kMaxBatch];
    int prefix[kMaxBatch + 1];  // items before each active image
};

struct BatchLayout {
    size_t hdr, imgs, img0, total;
    std::vector<size_t> off;  // per-image workspace offsets
};

static WsLayout img_layout(int H, int W, const dh_params *p) {
    return ws_layout(H, W, 1, sweep_tile_h(1), refine_bytes(H, W, p), false);
}

static BatchLayout batch_layout(int n, const dh_image *im, const dh_params *p) {
    BatchLayout B;
    size_t o = 0;
    B.hdr = o; o = align_up(o + sizeof(BatchHdr));
    B.imgs = o; o = align_up(o + (size_t)n * sizeof(BImg));
    B.img0 = o;
    for (int i = 0; i < n; ++i) {
        B.off.push_back(o);
        o = align_up(o + img_layout(im[i].H, im[i].W, p).total);
    }
    B.total = o;
    return B;
}

// Host -> device copy of a few BImg records through kernel parameters (no
// staging allocation), plus the reset of each image's iteration state.
constexpr int kPutChunk = 4;
struct PutChunk {
    BImg rec[kPutChunk];
};

__global__ void k_batch_put(BImg *dst, const __grid_constant__ PutChunk ch, int count, int reset) {
    const int words = (int)(sizeof(BImg) / 4);
    for (int r = 0; r < count; ++r) {
        const unsigned *src = reinterpret_cast<const unsigned *>(&ch.rec[r]);
        unsigned *d = reinterpret_cast<unsigned *>(dst + r);
        for (int k = threadIdx.x; k < words; k += blockDim.x) d[k] = src[k];
    }
    __syncthreads();
    if (reset && threadIdx.x < count) {
        SolveState *st = ch.rec[threadIdx.x].d.st;
        st->arrive = 0;
        st->n = 0;
        st->cur = 0;
        st->done = 0;
        st->status = 0;
        st->n_final = 0;
        st->err = 0;
        st->phase_start = 0;
    }
    __threadfence();
    tensormap_release();
}

__global__ void k_batch_init(BatchHdr *h, BImg *imgs, int n, int use_cond, unsigned long long cond) {
    if (threadIdx.x != 0) return;
    h->imgs = imgs;
    h->nimg = n;
    h->nactive = n;
    h->iter = 0;
    h->arrive = 0;
    h->work = 0;
    h->use_cond = use_cond;
    h->cond = cond;
    int acc = 0, k = 0;
    for (int i = 0; i < n; ++i) {
        if (__ldcg(&imgs[i].d.st->done)) continue;  // finished in an earlier precision phase
        h->active[k] = i;
        h->prefix[k] = acc;
        acc += imgs[i].items;
        ++k;
    }
    h->prefix[k] = acc;
    h->nactive = k;
}

// 16-bit iterate storage: u0 (float32) into the first iterate buffer
template <class T>
__global__ void k_b_to16(const float *__restrict__ src, T *__restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        Store<T>::put(dst + i, src[i]);
}

// End of an image's 16-bit loop: u^n (in d->u[cur]) as float32 into u_out and,
// when J is given, J = clamp(u^n, 0, 1).
template <class T>
__global__ void k_b_from16(const SolveDesc *__restrict__ d, float *u_out, float *J) {
    const int cur = __ldcg(&d->st->cur);
    const size_t n3 = (size_t)3 * d->H * d->W;
    const T *src = static_cast<const T *>(d->u[cur]);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const float v = Store<T>::get(src + i);
        u_out[i] = v;
        if (J) J[i] = fminf(fmaxf(v, 0.f), 1.f);
    }
}

// Hands an image to the float32 phase: its iterate now sits in buffer 0; a
// stalled 16-bit phase continues from the same n, any other outcome is final.
__global__ void k_b_handoff(SolveState *st) {
    st->cur = 0;
    st->arrive = 0;
    if (st->status == kStatusSwitch) {
        st->done = 0;
        st->status = 0;
        st->phase_start = st->n;
    }
}


// Tile t of an image, numbered down the columns of tiles (t = column * nty +
// row): consecutive tiles of a CTA's run are vertical neighbours, so the halo
// rows a tile loads were loaded or written by the tile just before it and are
// still in L2.
__device__ __forceinline__ void tile_origin(const BImg *im, int tile, int &x0, int &y0) {
    const int nty = (im->d.H + kBTH - 1) / kBTH;
    const int tx = tile / nty;
    x0 = tx * kTW;
    y0 = (tile - tx * nty) * kBTH;
}

// T: storage of the iterates (float, or bf16 / fp16 with float arithmetic)
template <bool EDGE, class T>
__global__ void __launch_bounds__(kBNW * 32, 5)
k_sweep_batch(BatchHdr *__restrict__ hb) {
    using P = TmaPlan<kBTH, true, T>;
    constexpr int SW = P::SW, SH = P::SH, HALO = Store<T>::HALO;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sb = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float2 red[kBNW];
    __shared__ int s_last, s_img_last;
    __shared__ int s_active[kMaxBatch];
    __shared__ int s_prefix[kMaxBatch + 1];
    __shared__ int s_cur[kMaxBatch];  // buffer holding u^n of each active image (fixed for the launch)

    if (hb->use_cond && (blockIdx.x | threadIdx.x) == 0) {
        cudaGraphSetConditional(hb->cond, 0);  // the last CTA sets it back while images remain
        __threadfence();
    }
    const int nact = __ldcg(&hb->nactive);
    for (int k = threadIdx.x; k < nact; k += blockDim.x) s_active[k] = __ldcg(&hb->active[k]);
    for (int k = threadIdx.x; k <= nact; k += blockDim.x) s_prefix[k] = __ldcg(&hb->prefix[k]);
    __syncthreads();
    for (int k = threadIdx.x; k < nact; k += blockDim.x) s_cur[k] = __ldcg(&hb->imgs[s_active[k]].d.st->cur);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int total = s_prefix[nact];
    BImg *imgs = hb->imgs;
    T *s = reinterpret_cast<T *>(sb + P::U_OFF);
    float *sphi = reinterpret_cast<float *>(sb + P::PHI_OFF);
    float *slam = reinterpret_cast<float *>(sb + P::LAM_OFF);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    // item -> (active slot, image, tile, channel)
    auto locate = [&](int item, int &slot, int &img, int &tile, int &c) {
        int lo = 0, hi = nact - 1;  // last k with prefix[k] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_prefix[mid] <= item) lo = mid; else hi = mid - 1;
        }
        slot = lo;
        img = s_active[lo];
        const int j = item - s_prefix[lo];
        tile = j / 3;
        c = j - 3 * tile;
    };
    // Items in walk order: position q -> item (odd loop iterations walk
    // backwards, starting on the tiles touched last).  The positions are
    // handed out in chunks of kBChunk (one tile's three channels; the next
    // chunk is the tile below): chunk blockIdx.x first, then G + the values of
    // a counter the grid shares for the launch, so that CTAs that run faster
    // take more chunks and all finish at about the same time.  Thread 0 takes
    // the next chunk while the first item of the current one is walked and
    // publishes each next position in s_next before the walk's closing
    // barrier.  Consecutive items of a CTA mostly belong to one image: one
    // tensor-map acquire and one arrival atomic per image change.
    const bool rev = (__ldcg(&hb->iter) & 1) != 0;
    const int G = gridDim.x, nch = (total + kBChunk - 1) / kBChunk;
    auto item_of = [&](int q) { return rev ? total - 1 - q : q; };
    // thread 0, TMA images only: load an item's tiles.  (No L2 prefetch of the
    // next item: the next tile down a column arrives as this tile's halo;
    // prefetching one item ahead cost 7 % on the 64-image batch.)
    // The maps were written on the device (k_batch_put): acquire them for the
    // tensor-map proxy when the image changes from the previous use by this CTA.
    __shared__ int s_acq_img, s_arr_cnt, s_next;  // thread 0's state, kept out of the walk's registers
    if (threadIdx.x == 0) {
        s_acq_img = -1;
        s_arr_cnt = 0;  // finished items of the current image not yet counted
    }
    auto maps = [&](int item, int &img, int &slot, int &tile, int &c, int &x0, int &y0) -> const BImg * {
        locate(item, slot, img, tile, c);
        const BImg *im = imgs + img;
        if (!im->tma) return nullptr;
        tile_origin(im, tile, x0, y0);
        if (img != s_acq_img) {
            tensormap_acquire(&im->tm[s_cur[slot]]);
            tensormap_acquire(&im->tm[2]);
            tensormap_acquire(&im->tm[3]);
            s_acq_img = img;
        }
        return im;
    };
    auto issue = [&](int item) {  // returns the item's image
        int img, slot, tile, c, x0 = 0, y0 = 0;
        const BImg *im = maps(item, img, slot, tile, c, x0, y0);
        if (!im) return img;
        mbar_arrive_expect_tx(&bar, P::TX);
        tma_load_3d(sb + P::U_OFF, &im->tm[s_cur[slot]], &bar, x0 - HALO, y0 - 2, c);
        tma_load_3d(sb + P::PHI_OFF, &im->tm[2], &bar, x0, y0, c);
        tma_load_2d(sb + P::LAM_OFF, &im->tm[3], &bar, x0, y0);
        return img;
    };
    int q = (int)blockIdx.x < nch ? (int)blockIdx.x * kBChunk : total;  // current position (every thread)
    int cn = nch;  // (thread 0) the chunk after the current one
    if (threadIdx.x == 0 && q < total) issue(item_of(q));

    // An image whose last item of this iteration a CTA has just finished is
    // finished (residual, stop rule) by that CTA at its next barrier, so the
    // arrival atomic's round trip overlaps the next tile's load.
    if (threadIdx.x == 0) s_img_last = -1;
    auto finish_pending = [&]() {  // all threads, right after a barrier
        const int fin = s_img_last;
        if (fin >= 0) {
            finish_iteration(&imgs[fin].d, imgs[fin].d.st);
            __syncthreads();
            if (threadIdx.x == 0) s_img_last = -1;
        }
    };

    int kt = 0;  // TMA items waited for so far (barrier phase)
    bool failed = false;
    while (q < total) {
        const int item = item_of(q);
        int slot, img, tile, c;
        locate(item, slot, img, tile, c);
        BImg *im = imgs + img;
        const SolveDesc *d = &im->d;
        SolveState *st = d->st;
        const int H = d->H, W = d->W;
        const size_t N = (size_t)H * W;
        int x0, y0;
        tile_origin(im, tile, x0, y0);
        const int cur = s_cur[slot];
        if (im->tma) {
            const bool ok = mbar_wait_bounded(&bar, kt & 1, kWaitLimitCycles);
            ++kt;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            finish_pending();
            if (!d->dirichlet && (x0 == 0 || y0 == 0 || x0 + kTW + 2 > W || y0 + kBTH + 2 > H)) {
                reflect_border(s, SW, SW, SH, x0 - HALO, y0 - 2, H, W);
                fence_proxy_async_smem();
            }
        } else {
            __syncthreads();
            finish_pending();
            // gather the tile with the reflecting boundary (W % 4 != 0 or unaligned image)
            const T *u = static_cast<const T *>(d->u[cur]) + c * N;
            for (int e = threadIdx.x; e < SH * SW; e += kBNW * 32) {
                const int r = e / SW, q = e - r * SW;
                const int yy = y0 - 2 + r, xx = x0 - HALO + q;
                if (!d->dirichlet)
                    s[e] = u[(size_t)reflect_idx(yy, H) * W + reflect_idx(xx, W)];
                else if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                    s[e] = u[(size_t)yy * W + xx];
                else
                    Store<T>::put(s + e, 0.f);
            }
            for (int e = threadIdx.x; e < kBTH * kTW; e += kBNW * 32) {
                const int r = e / kTW, q = e - r * kTW;
                const int y = y0 + r, x = x0 + q;
                const bool in = y < H && x < W;
                sphi[e] = in ? d->phi[c * N + (size_t)y * W + x] : 0.f;
                slam[e] = in ? d->lam[(size_t)y * W + x] : 0.f;
            }
            fence_proxy_async_smem();
        }
        __syncthreads();
        // first item of a chunk: take the next one (its value is needed only
        // after this chunk's last walk)
        if (threadIdx.x == 0 && q % kBChunk == 0) cn = G + (int)atomicAdd(&hb->work, 1u);

        T *__restrict__ un = static_cast<T *>(d->u[cur ^ 1]) + c * N;
        const int x = x0 + 4 * lane;
        const bool vec = im->tma != 0;  // aligned planes, W % 4 == 0 (W % 8 == 0 for 16-bit storage)
        float2 facc = make_float2(0.f, 0.f);  // this lane's sum of F^2 over the item, in pairs
        auto pl = [&](int ty, float *ph, float *la) {
            const float4 p4 = *reinterpret_cast<const float4 *>(sphi + ty * kTW + 4 * lane);
            const float4 l4 = *reinterpret_cast<const float4 *>(slam + ty * kTW + 4 * lane);
            ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
            la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
        };
        auto sink = [&](int ty, const float *nu, const float *F) {
            const int y = y0 + ty;
            if (y >= H || x >= W) return;
            const size_t ro = (size_t)y * W;
            if (x + 3 < W) {
                const float2 fa = make_float2(F[0], F[1]), fb = make_float2(F[2], F[3]);
                facc = fma2(fb, fb, fma2(fa, fa, facc));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x + j < W) facc.x = fmaf(F[j], F[j], facc.x);
            }
            if (vec) {
                Store<T>::write4(un + ro + x, nu[0], nu[1], nu[2], nu[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x + j < W) Store<T>::put(un + ro + x + j, nu[j]);
            }
        };
        walk_rows<kBR, SW, T, EDGE>(s, w * kBR, lane, d->eps, d->tau, d->wg0, d->wg1, d->wg2, pl, sink);

        if (threadIdx.x == 0) {  // the position after q: within the chunk, else the next chunk's first
            int qn = q + 1;
            if (qn % kBChunk == 0 || qn >= total) qn = cn < nch ? cn * kBChunk : total;
            s_next = qn;
        }
        const float2 tot = block_pair_sum<kBNW>(facc.x + facc.y, 0.f, red);  // every thread is past its walk
        const int qnext = s_next;  // rewritten only after the next item's first barrier
        if (threadIdx.x == 0) {
            int next_img = -1;
            if (qnext < total) {  // the stage is free: start the next load first
                fence_proxy_async_smem();
                next_img = issue(item_of(qnext));
            }
            d->part[(size_t)c * d->nblk + tile] = tot;
            const unsigned cnt = (unsigned)++s_arr_cnt;
            if (next_img != img) {  // the run leaves this image: count its items
                __threadfence();
                const unsigned prev = atomicAdd(&st->arrive, cnt);
                if (prev + cnt == (unsigned)im->items) s_img_last = img;  // read after the next barrier
                s_arr_cnt = 0;
            }
        }
        q = qnext;
    }
    __syncthreads();
    finish_pending();
    if (failed) {
        if (threadIdx.x == 0) {
            mbar_wait_bounded(&bar, kt & 1, kWaitLimitCycles);  // the load already issued
            for (int k = 0; k < nact; ++k) atomicCAS(&imgs[s_active[k]].d.st->err, 0, DH_ETIMEOUT);
        }
    }
    // last CTA: compact the active list, keep the loop going while it is not
    // empty.  The arrival is an acquire-release atomic (it publishes this CTA's
    // work; the last arrival sees everyone's).  The images' states are read by
    // all threads at once, then thread 0 scans the flags in shared memory.
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atom_add_acq_rel_gpu(&hb->arrive, 1u);
        s_last = prev == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last) {
        const int nimg = hb->nimg;
        int *s_keep = s_active, *s_items = s_prefix;  // free again: reused for the compaction
        for (int i = threadIdx.x; i < nimg; i += blockDim.x) {
            SolveState *st = imgs[i].d.st;
            int keep = 0;
            if (!__ldcg(&st->done)) {
                const int err = __ldcg(&st->err);
                if (err) {  // a bounded wait gave up: this image stops with the error
                    st->done = 1;
                    st->status = err;
                    st->n_final = __ldcg(&st->n);
                } else {
                    keep = 1;
                }
            }
            s_keep[i] = keep;
            s_items[i] = keep ? imgs[i].items : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = 0, acc = 0;
            for (int i = 0; i < nimg; ++i) {
                if (!s_keep[i]) continue;
                hb->active[k] = i;
                hb->prefix[k] = acc;
                acc += s_items[i];
                ++k;
            }
            hb->prefix[k] = acc;
            hb->nactive = k;
            hb->iter = hb->iter + 1;
            hb->arrive = 0;
            hb->work = 0;
            __threadfence();
            if (hb->use_cond && k > 0) cudaGraphSetConditional(hb->cond, 1);
        }
    }
}

// ------------------------------------------------------------ host

// storage kind: 0 float32, 1 bf16, 2 fp16
static void *batch_fn(bool edge, int kind) {
    if (kind == 1) return edge ? (void *)k_sweep_batch<true, __nv_bfloat16> : (void *)k_sweep_batch<false, __nv_bfloat16>;
    if (kind == 2) return edge ? (void *)k_sweep_batch<true, __half> : (void *)k_sweep_batch<false, __half>;
    return edge ? (void *)k_sweep_batch<true, float> : (void *)k_sweep_batch<false, float>;
}
static unsigned batch_smem(int kind) {
    return (kind ? TmaPlan<kBTH, true, __half>::STAGE : TmaPlan<kBTH, true, float>::STAGE) + 1024;
}


struct BatchGraph {
    int dev;
    const void *hdr;
    int grid;
    int edge;
    int kind;
    cudaGraphExec_t exec;
    cudaGraphConditionalHandle cond;
};
static std::mutex g_bmu;
static std::vector<BatchGraph> g_bcache;

static int batch_graph(int dev, BatchHdr *hdr, int grid, bool edge, int kind, unsigned smem, BatchGraph *out) {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto &e : g_bcache)
        if (e.dev == dev && e.hdr == hdr && e.grid == grid && e.edge == (edge ? 1 : 0) && e.kind == kind) {
            *out = e;
            return DH_OK;
        }
    cudaGraph_t g = nullptr;
    DH_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t wn;
    if (err == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        err = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &cp);
    }
    if (err == cudaSuccess) {
        cudaKernelNodeParams kp = {};
        void *args[] = {(void *)&hdr};
        kp.func = batch_fn(edge, kind);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(kBNW * 32);
        kp.sharedMemBytes = smem;
        kp.kernelParams = args;
        cudaGraphNode_t kn;
        err = cudaGraphAddKernelNode(&kn, cp.conditional.phGraph_out[0], nullptr, 0, &kp);
    }
    cudaGraphExec_t exec = nullptr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return cuda_fail(err);
    if (g_bcache.size() >= 8) {
        cudaGraphExecDestroy(g_bcache.front().exec);
        g_bcache.erase(g_bcache.begin());
    }
    BatchGraph e{dev, hdr, grid, edge ? 1 : 0, kind, exec, h};
    g_bcache.push_back(e);
    *out = e;
    return DH_OK;
}

static bool image_ok(const dh_image &m) {
    return m.I && m.J && m.u && m.t && m.A && shape_ok(m.H, m.W);
}

}  // namespace dh

using namespace dh;

extern "C" {

size_t dh_batch_workspace_bytes(int n, const dh_image *imgs, const dh_params *p) {
    if (n < 1 || n > kMaxBatch || !imgs || !p) return 0;
    for (int i = 0; i < n; ++i)
        if (!shape_ok(imgs[i].H, imgs[i].W)) return 0;
    if (dh_workspace_bytes(1, 1, p) == 0) return 0;
    return batch_layout(n, imgs, p).total;
}

// The batched solve; with `warm`, each image's u0 is the network's prediction
// (dh_dehaze_batch_warm), else the caller's u0 or Phi.
static int batch_run(int n, const dh_image *imgs, const dh_params *p, void *workspace, size_t workspace_bytes,
                     void *stream, dh_report *reports, const WarmNet *warm) {
    if (n < 1 || n > kMaxBatch || !imgs || !p) return DH_EINVAL;
    if (dh_workspace_bytes(1, 1, p) == 0) return DH_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!image_ok(imgs[i])) return DH_EINVAL;
    const BatchLayout B = batch_layout(n, imgs, p);
    if (!workspace || ((uintptr_t)workspace % kAlign) || workspace_bytes < B.total) return DH_EWORKSPACE;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (reports) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    // iterate storage: float32, 16-bit (bf16 / fp16), or 16-bit until the
    // residual stalls and float32 from the same n (as in the single-image path)
    const int storage = p->storage;
    const bool bf = storage == DH_STORE_BF16 || storage == DH_STORE_BF16_F32;
    const bool switched = storage == DH_STORE_BF16_F32 || storage == DH_STORE_F16_F32;
    const int kind1 = storage == DH_STORE_F32 ? 0 : (bf ? 1 : 2);
    auto grid_for_n = [](size_t m) { return (int)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096); };
    std::vector<BImg> recs(n);
    // the two iterate buffers of image i for storage `kind`, and their tensor maps
    auto set_iterates = [&](BImg &r, int i, int kind) -> int {
        const dh_image &m = imgs[i];
        char *iw = ws + B.off[i];
        const WsLayout L = img_layout(m.H, m.W, p);
        const size_t n3 = (size_t)3 * m.H * m.W;
        SolveDesc &d = r.d;
        if (kind == 0) {
            d.u[0] = m.u;
            d.u[1] = iw + L.ub;
        } else {
            d.u[0] = iw + L.ub;
            d.u[1] = iw + L.ub + align_up(n3 * 2);
        }
        auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
        // TMA rows start on 16-byte boundaries: W % 4 == 0 for float32, W % 8 == 0 for 16 bits
        r.tma = (m.W % (kind ? 8 : 4) == 0) && a16(d.u[0]) && a16(d.u[1]) && a16(d.phi) && a16(d.lam);
        if (!r.tma) return DH_OK;
        int e = DH_OK;
        if (kind == 0) {
            e = encode_f32_map(&r.tm[0], d.u[0], 3, m.W, m.H, 3, kTW + 8, kBTH + 4);
            if (!e) e = encode_f32_map(&r.tm[1], d.u[1], 3, m.W, m.H, 3, kTW + 8, kBTH + 4);
        } else {
            const cuuint64_t dims[3] = {(cuuint64_t)m.W, (cuuint64_t)m.H, 3};
            const cuuint64_t strides[2] = {(cuuint64_t)m.W * 2, (cuuint64_t)m.W * m.H * 2};
            const cuuint32_t box[3] = {kTW + 16, kBTH + 4, 1};
            const CUtensorMapDataType dt = kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
            e = encode_tiled(&r.tm[0], dt, 3, d.u[0], dims, strides, box);
            if (!e) e = encode_tiled(&r.tm[1], dt, 3, d.u[1], dims, strides, box);
        }
        if (!e) e = encode_f32_map(&r.tm[2], d.phi, 3, m.W, m.H, 3, kTW, kBTH);
        if (!e) e = encode_f32_map(&r.tm[3], d.lam, 2, m.W, m.H, 1, kTW, kBTH);
        return e;
    };
    // front end per image (Sec. II-D, II-A)
    int total_items = 0;
    for (int i = 0; i < n; ++i) {
        const dh_image &m = imgs[i];
        char *iw = ws + B.off[i];
        const WsLayout L = img_layout(m.H, m.W, p);
        float *dc = (float *)(iw + L.dc), *lam = (float *)(iw + L.lam), *phi = (float *)(iw + L.phi);
        int rc = launch_dark_channel(m.I, m.H, m.W, p->patch, nullptr, dc, s);
        if (!rc) rc = launch_select_A(m.I, dc, m.H, m.W, p->topk_permille, m.A, nullptr, iw, L, s);
        if (!rc) rc = launch_transmission(m.I, m.H, m.W, p, m.A, nullptr, m.t, lam, phi,
                                          (m.u0 || warm) ? nullptr : m.u, (float2 *)(iw + L.phin_part),
                                          iw + L.refine, s);
        if (rc) return rc;
        if (m.u0) {
            DH_CUDA_TRY(cudaMemcpyAsync(m.u, m.u0, (size_t)3 * m.H * m.W * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
        rc = launch_phin_final((const float2 *)(iw + L.phin_part), m.H, m.W, (SolveState *)(iw + L.state), s);
        if (rc) return rc;
        BImg &r = recs[i];
        std::memset(&r, 0, sizeof(r));
        SolveDesc &d = r.d;
        d.phi = phi;
        d.lam = lam;
        d.part = (float2 *)(iw + L.part);
        d.st = (SolveState *)(iw + L.state);
        d.H = m.H;
        d.W = m.W;
        d.max_iter = p->max_iter;
        d.depth = 1;
        d.tol = p->tol;
        d.tau = p->tau;
        d.eps = p->eps;
        d.dirichlet = p->boundary == DH_BOUNDARY_ZERO;
        double wgt[3];
        for (int k = 0; k <= 2; ++k) wgt[k] = exp(-(double)(k * k) / (2.0 * (double)p->sigma * p->sigma));
        const double sum = wgt[0] + 2.0 * (wgt[1] + wgt[2]);
        d.wg0 = (float)(wgt[0] / sum);
        d.wg1 = (float)(wgt[1] / sum);
        d.wg2 = (float)(wgt[2] / sum);
        r.ntx = (m.W + kTW - 1) / kTW;
        d.nblk = r.ntx * ((m.H + kBTH - 1) / kBTH);
        r.items = 3 * d.nblk;
        total_items += r.items;
        d.phase_stop = switched ? 1 : 0;
        const int rc2 = set_iterates(r, i, kind1);
        if (rc2) return rc2;
    }
    // warm start: u0 = net(I, t, A, Phi) / lambda into each image's u, one network
    // forward per group of same-shape images (the network's workspace is reused
    // group after group)
    int warm_launches = 0;
    if (warm) {
        for (const auto &g : warm_groups(n, imgs)) {
            const int cnt = (int)g.size();
            std::vector<const float *> I(cnt), t(cnt), A(cnt), phi(cnt), lam(cnt);
            std::vector<float *> u0(cnt);
            for (int k = 0; k < cnt; ++k) {
                const dh_image &m = imgs[g[k]];
                I[k] = m.I;
                t[k] = m.t;
                A[k] = m.A;
                phi[k] = recs[g[k]].d.phi;
                lam[k] = recs[g[k]].d.lam;
                u0[k] = m.u;
            }
            const int rc = warm_u0_group(warm->params, warm->base, cnt, I.data(), t.data(), A.data(), phi.data(),
                                         lam.data(), u0.data(), imgs[g[0]].H, imgs[g[0]].W, warm->ws, warm->ws_bytes,
                                         s);
            if (rc) return rc;
            warm_launches += kWarmForwardLaunches + cnt;
        }
    }
    if (kind1) {  // u0 (float32 in u) into each image's first 16-bit buffer
        for (int i = 0; i < n; ++i) {
            const size_t n3 = (size_t)3 * imgs[i].H * imgs[i].W;
            if (kind1 == 1)
                k_b_to16<__nv_bfloat16><<<grid_for_n(n3), 256, 0, s>>>(imgs[i].u, (__nv_bfloat16 *)recs[i].d.u[0], n3);
            else
                k_b_to16<__half><<<grid_for_n(n3), 256, 0, s>>>(imgs[i].u, (__half *)recs[i].d.u[0], n3);
        }
    }
    BImg *dimgs = (BImg *)(ws + B.imgs);
    auto put = [&](int reset) {
        for (int i = 0; i < n; i += kPutChunk) {
            PutChunk ch;
            const int cnt = n - i < kPutChunk ? n - i : kPutChunk;
            for (int k = 0; k < cnt; ++k) ch.rec[k] = recs[i + k];
            k_batch_put<<<1, 128, 0, s>>>(dimgs + i, ch, cnt, reset);
        }
    };
    put(1);
    DH_CUDA_TRY(cudaGetLastError());
    // the batched loop over the images still iterating, for storage `kind`
    const bool edge = !(p->variant & DH_VAR_NO_EDGE);
    BatchHdr *hdr = (BatchHdr *)(ws + B.hdr);
    int dev = 0, sms = 0, launches = 0;
    DH_CUDA_TRY(cudaGetDevice(&dev));
    DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto run_loop = [&](int kind) -> int {
        const unsigned smem = batch_smem(kind);
        void *fn = batch_fn(edge, kind);
        int per_sm = 0;
        DH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBNW * 32, smem));
        // every CTA resident at once (the chunks come from a counter, so any
        // grid size works; the multiple of 3 is kept from the earlier
        // one-CTA-per-channel assignment and costs nothing)
        int grid = total_items < per_sm * sms ? total_items : per_sm * sms;
        grid = grid < 3 ? 3 : grid - grid % 3;
        if (p->use_graph) {
            BatchGraph bg{};
            const int rc = batch_graph(dev, hdr, grid, edge, kind, smem, &bg);
            if (rc) return rc;
            k_batch_init<<<1, 32, 0, s>>>(hdr, dimgs, n, 1, bg.cond);
            DH_CUDA_TRY(cudaGraphLaunch(bg.exec, s));
        } else {
            k_batch_init<<<1, 32, 0, s>>>(hdr, dimgs, n, 0, 0);
            void *args[] = {(void *)&hdr};
            for (int it = 0; it <= p->max_iter; ++it)
                DH_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kBNW * 32), args, smem, s));
            launches += p->max_iter + 1;
        }
        return DH_OK;
    };
    int rc = run_loop(kind1);
    if (rc) return rc;
    if (kind1 && switched) {
        // each image's 16-bit iterate becomes float32 in its u; the stalled ones
        // continue in float32 from the same n, the others are final
        for (int i = 0; i < n; ++i) {
            if (kind1 == 1)
                k_b_from16<__nv_bfloat16><<<grid_for_n((size_t)3 * imgs[i].H * imgs[i].W), 256, 0, s>>>(&dimgs[i].d, imgs[i].u, nullptr);
            else
                k_b_from16<__half><<<grid_for_n((size_t)3 * imgs[i].H * imgs[i].W), 256, 0, s>>>(&dimgs[i].d, imgs[i].u, nullptr);
            k_b_handoff<<<1, 1, 0, s>>>(recs[i].d.st);
            recs[i].d.phase_stop = 0;
            rc = set_iterates(recs[i], i, 0);
            if (rc) return rc;
        }
        put(0);
        rc = run_loop(0);
        if (rc) return rc;
    }
    for (int i = 0; i < n; ++i) {
        const size_t n3 = (size_t)3 * imgs[i].H * imgs[i].W;
        if (kind1 && !switched) {
            if (kind1 == 1)
                k_b_from16<__nv_bfloat16><<<grid_for_n(n3), 256, 0, s>>>(&dimgs[i].d, imgs[i].u, imgs[i].J);
            else
                k_b_from16<__half><<<grid_for_n(n3), 256, 0, s>>>(&dimgs[i].d, imgs[i].u, imgs[i].J);
        } else {
            rc = launch_output_f32(&dimgs[i].d, imgs[i].J, imgs[i].u, n3, s);
            if (rc) return rc;
        }
    }
    DH_CUDA_TRY(cudaGetLastError());
    if (!reports) return DH_OK;
    float ms = 0.f;
    cudaEventRecord(e1, s);
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    int worst = DH_OK, max_n = 0;
    for (int i = 0; i < n; ++i) {
        SolveState st;
        SelectState sel;
        const WsLayout L = img_layout(imgs[i].H, imgs[i].W, p);
        DH_CUDA_TRY(cudaMemcpy(&st, ws + B.off[i] + L.state, sizeof(st), cudaMemcpyDeviceToHost));
        DH_CUDA_TRY(cudaMemcpy(&sel, ws + B.off[i] + L.sel, sizeof(sel), cudaMemcpyDeviceToHost));
        dh_report &r = reports[i];
        std::memset(&r, 0, sizeof(r));
        r.status = st.status;
        if (r.status == DH_OK && sel.clamped) r.status = DH_WDEGENERATE;
        r.n_iter = st.n_final;
        for (int c = 0; c < 3; ++c) r.rho[c] = st.rho[c];
        DH_CUDA_TRY(cudaMemcpy(r.A, imgs[i].A, 3 * sizeof(float), cudaMemcpyDeviceToHost));
        r.a_index = sel.best;
        r.ms = ms;  // the whole batch
        r.launches = 18 + 1;  // front end + output of this image
        if (st.n_final > max_n) max_n = st.n_final;
        if (r.status < 0 && worst >= 0) worst = r.status;
        else if (worst == DH_OK && r.status > 0) worst = r.status;
    }
    reports[0].launches += (p->use_graph ? max_n + 1 : launches) + 1 + (n + kPutChunk - 1) / kPutChunk + warm_launches;
    return worst;
}

int dh_dehaze_batch(int n, const dh_image *imgs, const dh_params *p, void *workspace, size_t workspace_bytes,
                    void *stream, dh_report *reports) {
    return batch_run(n, imgs, p, workspace, workspace_bytes, stream, reports, nullptr);
}

size_t dh_batch_net_workspace_bytes(int base, int n, const dh_image *imgs) {
    if (n < 1 || n > kMaxBatch || !imgs) return 0;
    for (int i = 0; i < n; ++i)
        if (!shape_ok(imgs[i].H, imgs[i].W)) return 0;
    size_t most = 0;
    for (const auto &g : warm_groups(n, imgs)) {
        const size_t b = warm_net_bytes(base, (int)g.size(), imgs[g[0]].H, imgs[g[0]].W);
        if (b == 0) return 0;
        if (b > most) most = b;
    }
    return most;
}

int dh_dehaze_batch_warm(const float *params, int base, int n, const dh_image *imgs, const dh_params *p,
                         void *workspace, size_t workspace_bytes, void *net_workspace, size_t net_workspace_bytes,
                         void *stream, dh_report *reports) {
    if (!params || n < 1 || n > kMaxBatch || !imgs) return DH_EINVAL;
    for (int i = 0; i < n; ++i)
        if (imgs[i].u0 || !shape_ok(imgs[i].H, imgs[i].W) || warm_net_bytes(base, 1, imgs[i].H, imgs[i].W) == 0)
            return DH_EINVAL;
    const size_t need = dh_batch_net_workspace_bytes(base, n, imgs);
    if (!net_workspace || ((uintptr_t)net_workspace % kAlign) || net_workspace_bytes < need) return DH_EWORKSPACE;
    const WarmNet w{params, base, net_workspace, net_workspace_bytes};
    return batch_run(n, imgs, p, workspace, workspace_bytes, stream, reports, &w);
}

}  // extern "C"
