// Sweep kernel templates (App. A-A fixed-point update with the App. A-B
// stencil): the generic gather kernel, the TMA tile kernel (one or many
// iterations per launch), the two-iterations-per-load kernel and the per-warp
// row-stream kernel.  They are instantiated in the sweep_inst_*.cu files, a few
// variants per translation unit, and reached through the dispatch functions
// declared at the end.
#pragma once

#include "sweep.cuh"

namespace dh {

// Generic sweep (any W, any alignment): one CTA per (tile, channel), tile of
// u^n gathered with the reflecting boundary by plain loads.
template <int R, int NW, class T, bool EDGE>
__global__ void __launch_bounds__(NW * 32)
k_sweep(const SolveDesc *__restrict__ d) {
    constexpr int TH = R * NW;
    constexpr int SW = kTW + 8;
    constexpr int SH = TH + 4;
    __shared__ __align__(16) float s[SH * SW];
    __shared__ float2 red[NW];
    __shared__ int s_last;

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    const int H = d->H, W = d->W;
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * TH;
    const int cur = __ldcg(&st->cur);
    const size_t N = (size_t)H * W;
    const T *__restrict__ u = static_cast<const T *>(d->u[cur]) + c * N;
    T *__restrict__ un = static_cast<T *>(d->u[cur ^ 1]) + c * N;
    const float *__restrict__ phi = d->phi + c * N;
    const float *__restrict__ lam = d->lam;

    const bool dirichlet = d->dirichlet != 0;
    for (int e = threadIdx.x; e < SH * SW; e += NW * 32) {
        const int r = e / SW, q = e - r * SW;
        const int yy = y0 - 2 + r, xx = x0 - 4 + q;
        if (dirichlet) {
            s[e] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? Store<T>::get(u + (size_t)yy * W + xx) : 0.f;
        } else {
            s[e] = Store<T>::get(u + (size_t)reflect_idx(yy, H) * W + reflect_idx(xx, W));
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = x0 + 4 * lane;
    const bool vec = d->vec != 0;
    float rs = 0.f, rc = 0.f;
    auto pl = [&](int ty, float *ph, float *la) {
        const int y = y0 + ty;
#pragma unroll
        for (int j = 0; j < 4; ++j) ph[j] = la[j] = 0.f;
        if (y >= H) return;
        const size_t ro = (size_t)y * W;
        if (vec) {
            if (x < W) {
                const float4 p4 = __ldg(reinterpret_cast<const float4 *>(phi + ro + x));
                const float4 l4 = __ldg(reinterpret_cast<const float4 *>(lam + ro + x));
                ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < W) { ph[j] = __ldg(phi + ro + x + j); la[j] = __ldg(lam + ro + x + j); }
        }
    };
    auto sink = [&](int ty, const float *nu, const float *F) {
        const int y = y0 + ty;
        if (y >= H) return;
        const size_t ro = (size_t)y * W;
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x + j < W) q = fmaf(F[j], F[j], q);
        neumaier_add(rs, rc, q);
        if (vec) {
            if (x < W) Store<T>::write4(un + ro + x, nu[0], nu[1], nu[2], nu[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < W) Store<T>::put(un + ro + x + j, nu[j]);
        }
    };
    walk_rows<R, SW, float, EDGE>(s, w * R, lane, d->eps, d->tau, d->wg0, d->wg1, d->wg2, pl, sink);

    const float2 tot = block_pair_sum<NW>(rs, rc, red);
    if (threadIdx.x == 0)
        d->part[(size_t)c * d->nblk + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    arrive_and_finish(d, st, &s_last);
}

// TMA sweep (W % 4 == 0, 16-byte aligned planes): persistent CTAs walk the
// (tile, channel) items; one thread streams each item's u^n tile (with halo)
// into shared memory by TMA, STAGES items ahead, together with the Phi and
// lambda tiles when PL_SMEM (otherwise the walk reads those with vector
// loads); the border halo is reflected in shared memory afterwards.  Each
// item's tiles are first pulled into L2 one item before their load is issued.
// Odd iterations walk the items in reverse order, so that an iteration starts
// on the tiles the previous one touched last (still in L2).
//
// MULTI: a cooperative launch runs up to d->depth iterations.  Between two
// iterations the CTAs meet at a grid barrier (an acquire-release arrival
// count) whose last arrival reduces the residual and decides
// (finish_iteration), then bumps st->gen; the others wait for the bump
// (bounded, DH_ETIMEOUT).  With one stage, a CTA's first two items are static
// and the others come from a grid-wide counter (DYN).  With float32 iterates
// and a third buffer the decision is deferred (defer_barrier): the last CTA
// bumps st->gen at once and reduces while the next iteration runs.  The
// u^{n+1} tiles that the next iteration loads by TMA were written by generic
// stores of other CTAs: the writers fence them to the async proxy before
// arriving and the issuing thread fences again after the barrier.
template <int R, int NW, int STAGES, bool PL_SMEM, class T, bool EDGE, int MINB = 0, bool MULTI = false>
__global__ void __launch_bounds__(NW * 32, MINB > 0 ? MINB : 16 / NW)
k_sweep_tma(const __grid_constant__ CUtensorMap tm_ua, const __grid_constant__ CUtensorMap tm_ub,
            const __grid_constant__ CUtensorMap tm_uc, const __grid_constant__ CUtensorMap tm_phi,
            const __grid_constant__ CUtensorMap tm_lam, const SolveDesc *__restrict__ d) {
    constexpr int TH = R * NW;
    constexpr int HALO = Store<T>::HALO;
    using P = TmaPlan<TH, PL_SMEM, T>;
    constexpr int SW = P::SW, SH = P::SH;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base (the launch adds 1 KiB of slack)
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ float2 red[NW];
    __shared__ int s_last, s_timeout, s_next;
    constexpr bool DYN = MULTI && STAGES == 1;  // items from a grid-wide counter
    // deferred decisions (float32 iterates, a third buffer): see defer_barrier
    constexpr bool DEFER = DYN && sizeof(T) == 4;
    constexpr int UR = MINB >= 6 ? 8 : 11;  // partial loads per channel in flight in the reduction

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    unsigned gen = 0;
    if (MULTI) gen = ld_acquire_gpu(&st->gen);  // before this CTA can arrive anywhere
    const int H = d->H, W = d->W;
    const size_t N = (size_t)H * W;
    const int ntx = (W + kTW - 1) / kTW, nty = (H + TH - 1) / TH;
    const int ntiles = ntx * nty, nitems = 3 * ntiles;
    const int G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float eps = d->eps, tau = d->tau, wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;
    const bool dirichlet = d->dirichlet != 0;
    const float *__restrict__ phi_all = d->phi;
    const float *__restrict__ glam = d->lam;
    float2 *__restrict__ part = d->part;
    const int nblk = d->nblk;
    const int iters = MULTI ? d->depth : 1;
    const bool defer = DEFER && d->defer != 0 && d->phase_stop == 0;
    const bool ahead2 = nitems >= 6 * G;  // DYN: take items two ahead (see the item loop)
    int k = 0;  // items this CTA has started in the launch (stage and parity)
    bool failed = false;
    for (int it = 0; it < iters; ++it) {
        const int cur = __ldcg(&st->cur);
        const int n_it = __ldcg(&st->n);
        const bool rev = (n_it & 1) != 0;
        // u^n is read from buffer cur; u^{n+1} goes to the other one, or with
        // deferred decisions to the one holding neither u^n nor u^{n-1}
        const int wb = defer ? 3 - cur - __ldcg(&st->cprev) : cur ^ 1;
        const CUtensorMap *tm_u = cur == 0 ? &tm_ua : (cur == 1 ? &tm_ub : &tm_uc);
        T *__restrict__ ubase = static_cast<T *>(d->u[wb]);
        float2 *__restrict__ partn = defer ? part + (size_t)(n_it & 1) * 3 * nblk : part;
        // position q in the iteration's walk order -> item (odd iterations walk backwards)
        auto item_of = [&](int q) { return rev ? nitems - 1 - q : q; };
        auto tile_xy = [&](int item, int &c, int &x0, int &y0) {
            const int tile = item / 3;
            c = item - 3 * tile;
            x0 = (tile % ntx) * kTW;
            y0 = (tile / ntx) * TH;
            return tile;
        };
        auto issue = [&](int q, int stage) {
            int c, x0, y0;
            tile_xy(item_of(q), c, x0, y0);
            unsigned char *sb = smem + stage * P::STAGE;
            mbar_arrive_expect_tx(&bar[stage], P::TX);
            tma_load_3d(sb + P::U_OFF, tm_u, &bar[stage], x0 - HALO, y0 - 2, c);
            if (PL_SMEM) {
                tma_load_3d(sb + P::PHI_OFF, &tm_phi, &bar[stage], x0, y0, c);
                tma_load_2d(sb + P::LAM_OFF, &tm_lam, &bar[stage], x0, y0);
            }
        };
        auto prefetch = [&](int q) {
            int c, x0, y0;
            tile_xy(item_of(q), c, x0, y0);
            tma_prefetch_3d(tm_u, x0 - HALO, y0 - 2, c);
            tma_prefetch_3d(&tm_phi, x0, y0, c);
            tma_prefetch_2d(&tm_lam, x0, y0);
        };
        // Walk positions of this CTA: blockIdx.x, then (DYN) positions from a
        // counter the grid shares for this iteration, so that CTAs that run
        // faster take more items and all reach the grid barrier at about the
        // same time; otherwise blockIdx.x + jG.  With many items per CTA
        // (ahead2) the second position is blockIdx.x + G and thread 0 takes
        // the one two items ahead (2G + counter) while the current one is
        // walked, so the next item can be pulled into L2 first; with few, it
        // takes only the next one (G + counter), which leaves at most one
        // item queued per CTA when the counter runs out.  The next position
        // is published in s_next before the walk's closing barrier.
        unsigned *ctr = &st->work[n_it & 1];
        int q = (int)blockIdx.x;           // current position (every thread)
        int qn = ahead2 ? q + G : nitems;  // next position (thread 0)
        int j = 0;                // items of this CTA in this iteration
        if (threadIdx.x == 0) {
            if (MULTI && it > 0) fence_proxy_async_global();
            for (int jj = 0; jj < STAGES && q + jj * G < nitems; ++jj) issue(q + jj * G, (k + jj) % STAGES);
        }
        for (; q < nitems; ++j, ++k) {
            const int stage = k % STAGES;
            const uint32_t parity = (k / STAGES) & 1;
            int c, x0, y0;
            const int tile = tile_xy(item_of(q), c, x0, y0);
            unsigned char *sb = smem + stage * P::STAGE;
            T *s = reinterpret_cast<T *>(sb + P::U_OFF);
            const float *sphi = reinterpret_cast<const float *>(sb + P::PHI_OFF);
            const float *slam = reinterpret_cast<const float *>(sb + P::LAM_OFF);
            if (threadIdx.x == 0) {
                if (DYN) {
                    if (ahead2 && qn < nitems) prefetch(qn);
                } else if (q + STAGES * G < nitems) {
                    prefetch(q + STAGES * G);
                }
            }

            const bool ok = mbar_wait_bounded(&bar[stage], parity, kWaitLimitCycles);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            // reflect the halo cells that fall outside the image (TMA filled zeros,
            // which is already the Dirichlet boundary); interior tiles need no
            // barrier here: the one above already ordered the landed tile
            if (!dirichlet && (x0 == 0 || y0 == 0 || x0 + kTW + 2 > W || y0 + TH + 2 > H)) {
                reflect_border(s, SW, SW, SH, x0 - HALO, y0 - 2, H, W);
                fence_proxy_async_smem();  // these writes precede the stage's next TMA load
                __syncthreads();
            }

            // (DYN, thread 0) the position after the next one, taken here so that
            // no block barrier waits for the atomic before the walk's closing one
            int qa = nitems;
            if (DYN && threadIdx.x == 0) {
                if (!ahead2) qn = G + (int)atomicAdd(ctr, 1u);
                else if (qn < nitems) qa = 2 * G + (int)atomicAdd(ctr, 1u);
            }

            T *__restrict__ un = ubase + c * N;
            const int x = x0 + 4 * lane;
            // this lane's sum of F^2 over the item, in pairs (the lanes' sums are
            // then merged with compensation in a fixed order)
            float2 facc = make_float2(0.f, 0.f);
            const float *__restrict__ gphi = phi_all + c * N;
            auto pl = [&](int ty, float *ph, float *la) {
                float4 p4, l4;
                if (PL_SMEM) {
                    p4 = *reinterpret_cast<const float4 *>(sphi + ty * kTW + 4 * lane);
                    l4 = *reinterpret_cast<const float4 *>(slam + ty * kTW + 4 * lane);
                } else {
                    const int y = y0 + ty;
                    p4 = l4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (y < H && x < W) {
                        p4 = __ldg(reinterpret_cast<const float4 *>(gphi + (size_t)y * W + x));
                        l4 = __ldg(reinterpret_cast<const float4 *>(glam + (size_t)y * W + x));
                    }
                }
                ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
            };
            auto sink = [&](int ty, const float *nu, const float *F) {
                const int y = y0 + ty;
                if (y >= H || x >= W) return;  // W % 4 == 0: x < W covers all 4 columns
                const float2 fa = make_float2(F[0], F[1]), fb = make_float2(F[2], F[3]);
                facc = fma2(fb, fb, fma2(fa, fa, facc));
                Store<T>::write4(un + (size_t)y * W + x, nu[0], nu[1], nu[2], nu[3]);
            };
            walk_rows<R, SW, T, EDGE>(s, w * R, lane, eps, tau, wg0, wg1, wg2, pl, sink);

            // every thread is past its walk once block_pair_sum's barrier is
            // passed, so the stage can be refilled; red[] and s_next are
            // rewritten only after the next item's wait barrier, which every
            // reader of them reaches first
            if (DYN && threadIdx.x == 0) s_next = qn;
            const float2 tot = block_pair_sum<NW>(facc.x + facc.y, 0.f, red);
            const int qnext = DYN ? s_next : q + G;
            if (threadIdx.x == 0) {
                partn[(size_t)c * nblk + tile] = tot;
                const int qi = DYN ? qn : q + STAGES * G;  // the position whose load goes into this stage
                if (qi < nitems) {
                    fence_proxy_async_smem();
                    issue(qi, stage);
                }
                if (DYN && ahead2) qn = qa;
            }
            q = qnext;
        }
        if (failed) {
            // let every load already issued land (bounded) before going on
            for (int jj = 0; jj < STAGES && q + jj * G < nitems; ++jj) {
                const int kk = k + jj;
                mbar_wait_bounded(&bar[kk % STAGES], (kk / STAGES) & 1, kWaitLimitCycles);
            }
            if (threadIdx.x == 0) atomicCAS(&st->err, 0, DH_ETIMEOUT);
        }
        if (!MULTI) break;

        // grid barrier; the last CTA to arrive finishes the iteration (the
        // arrival is an acquire-release atomic: it publishes this CTA's
        // partials and u^{n+1} tiles, and the last arrival sees everyone's)
        fence_proxy_async_global();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned prev = atom_add_acq_rel_gpu(&st->arrive, 1u);
            s_last = prev == (unsigned)G - 1u;
            s_timeout = 0;
        }
        __syncthreads();
        if (s_last) {
            if (defer) {
                const int mode = defer_barrier<UR>(d, st, it == iters - 1, partn);
                if (threadIdx.x == 0) {
                    st->work[0] = st->work[1] = 0u;  // every CTA is past its last take of this iteration
                    st_release_gpu(&st->gen, gen + 1u);
                }
                if (mode == 2) defer_reduce<UR>(d, st, n_it, partn);  // while the others sweep
            } else {
                const int next = finish_iteration<UR>(d, st, it == iters - 1, false, true);
                if (threadIdx.x == 0) {
                    // the counter of the next iteration was last used two iterations ago
                    if (DYN) st->work[next & 1] = 0u;
                    st_release_gpu(&st->gen, gen + 1u);
                }
            }
        } else if (threadIdx.x == 0) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&st->gen) == gen) {
                if (clock64() - t0 > kWaitLimitCycles) {
                    s_timeout = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        ++gen;
        __syncthreads();
        if (s_timeout) {  // another CTA never arrived: give up, report
            if (threadIdx.x == 0) {
                atomicCAS(&st->err, 0, DH_ETIMEOUT);
                st->status = DH_ETIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (__ldcg(&st->done) || failed) return;
    }
    if (!MULTI) arrive_and_finish(d, st, &s_last);
}

// ---------------------------------------------------------------- two iterations per tile load
// Temporally blocked sweep (float iterates, W % 4 == 0, 16-byte aligned
// planes).  An item is a 120 x TH output tile of one channel.  TMA loads u^n
// on the output tile plus a 4-cell ring (136 x (TH+8)), Phi and lambda on the
// tile plus a (2-row, 4-column) ring (128 x (TH+4)).  Step 1 walks the 128 x
// (TH+4) region around the tile and keeps u^{n+1} in shared memory; after the
// border ring is reflected, step 2 walks the tile from it and writes u^{n+2}.
// The residual of step 1 over the tile is F(u^n) and that of step 2 is
// F(u^{n+1}), the same quantities one iteration at a time would give.  The
// last CTA at the grid barrier decides with both (finish_tb2): stop at n, or
// advance by two, or - when u^{n+1} is the iterate to return (its residual
// meets tol, or n+1 = max_iter) - switch the rest of the solve to one
// iteration per load (step 1 writing the tile to global memory), which
// recomputes u^{n+1} and stops there.
template <int R2, int NW>
struct Tb2Plan {
    static constexpr int TH = R2 * NW;
    static constexpr int R1 = R2 + 4 / NW;        // rows per warp in step 1 (TH + 4 rows)
    static constexpr int SW = kTW + 8;            // 136 floats per shared row
    static constexpr uint32_t U0_BYTES = (TH + 8) * SW * 4;
    static constexpr uint32_t PL_BYTES = (TH + 4) * kTW * 4;
    static constexpr uint32_t U1_BYTES = (TH + 4) * SW * 4;
    static constexpr uint32_t U0_OFF = 0;
    static constexpr uint32_t PHI_OFF = (U0_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t LAM_OFF = PHI_OFF + PL_BYTES;
    static constexpr uint32_t U1_OFF = (LAM_OFF + PL_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t SMEM = U1_OFF + U1_BYTES + 1024;  // + alignment slack
    static constexpr uint32_t TX = U0_BYTES + 2 * PL_BYTES;
    static_assert(4 % NW == 0, "the TH + 4 step-1 rows must split evenly over the warps");
};

// Last CTA of a two-iteration sweep: residuals of both levels, decision.
// Called after an acquire-release arrival; thread 0 loads the state it
// decides with before the partials and returns the next iterate's index (the
// caller publishes the state with a release store).  The while condition is
// set only by a launch that goes on after its last iteration.
static __device__ int finish_tb2(const SolveDesc *d, SolveState *st, bool last_in_launch) {
    constexpr int U = 6;
    __shared__ float2 wsum[6][32];
    __shared__ float sq[6];
    const int tid = threadIdx.x, nt = blockDim.x, w = tid >> 5, lane = tid & 31, nw = nt >> 5;
    int n = 0, two = 0, cur = 0, err = 0;
    float phin2[3] = {0.f, 0.f, 0.f};
    if (tid == 0) {
        n = ld_state_int(&st->n);
        two = ld_state_int(&st->tb2);
        cur = ld_state_int(&st->cur);
        err = ld_state_int(&st->err);
        for (int c = 0; c < 3; ++c) phin2[c] = __ldcg(&st->phin2[c]);
    }
    const int nblk = d->nblk;
    const float2 *part = d->part;
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, cc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b0 = tid; b0 < nblk; b0 += U * nt) {
        float2 pv[6][U];
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int b = b0 + j * nt;
                pv[k][j] = b < nblk ? __ldcg(part + (size_t)k * nblk + b) : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int j = 0; j < U; ++j) neumaier_merge(s[k], cc[k], pv[k][j].x, pv[k][j].y);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[k], off);
            const float c2 = __shfl_down_sync(0xffffffffu, cc[k], off);
            neumaier_merge(s[k], cc[k], s2, c2);
        }
        if (lane == 0) wsum[k][w] = make_float2(s[k], cc[k]);
    }
    __syncthreads();
    if (tid < 6) {
        float a = wsum[tid][0].x, b = wsum[tid][0].y;
        for (int k = 1; k < nw; ++k) neumaier_merge(a, b, wsum[tid][k].x, wsum[tid][k].y);
        sq[tid] = a + b;
    }
    __syncthreads();
    if (tid != 0) return 0;
    auto rho_of = [&](int lv, float *rho, float &worst) {
        bool finite = true;
        worst = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float pn = phin2[c], q = sq[3 * lv + c];
            rho[c] = pn > 0.f ? sqrtf(q / pn) : sqrtf(q);
            if (!isfinite(rho[c])) finite = false;
            else worst = fmaxf(worst, rho[c]);
        }
        return finite;
    };
    float rho0[3], w0;
    const bool fin0 = rho_of(0, rho0, w0);
    if (d->rho_hist)
        for (int c = 0; c < 3; ++c) d->rho_hist[3 * n + c] = rho0[c];
    const bool conv = fin0 && w0 <= d->tol;
    unsigned cont = 1;
    int next = n;
    if (err || conv || !fin0 || n >= d->max_iter) {
        st->done = 1;
        st->n_final = n;
        st->status = err ? err : (!fin0 ? DH_ENONFINITE : (conv ? DH_OK : DH_WNOCONV));
        for (int c = 0; c < 3; ++c) st->rho[c] = rho0[c];
        cont = 0;
    } else if (!two) {
        st->n = next = n + 1;
        st->cur = cur ^ 1;
    } else {
        float rho1[3], w1;
        const bool fin1 = rho_of(1, rho1, w1);
        if (!fin1 || w1 <= d->tol || n + 1 >= d->max_iter) {
            st->tb2 = 0;  // u^{n+1} may be the answer: redo it one iteration at a time
        } else {
            if (d->rho_hist)
                for (int c = 0; c < 3; ++c) d->rho_hist[3 * (n + 1) + c] = rho1[c];
            st->n = next = n + 2;
            st->cur = cur ^ 1;
        }
    }
    st->arrive = 0;
    if (d->use_cond && cont && last_in_launch) cudaGraphSetConditional(d->cond, 1u);
    return next;
}

template <int R2, int NW, bool EDGE, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
k_sweep_tb2(const __grid_constant__ CUtensorMap tm_ua, const __grid_constant__ CUtensorMap tm_ub,
            const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_lam,
            const SolveDesc *__restrict__ d) {
    using P = Tb2Plan<R2, NW>;
    constexpr int TH = P::TH, R1 = P::R1, SW = P::SW;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float2 red[2][NW];
    __shared__ int s_last, s_timeout, s_next;
    float *s0 = reinterpret_cast<float *>(smem + P::U0_OFF);
    const float *sphi = reinterpret_cast<const float *>(smem + P::PHI_OFF);
    const float *slam = reinterpret_cast<const float *>(smem + P::LAM_OFF);
    float *s1 = reinterpret_cast<float *>(smem + P::U1_OFF);

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    unsigned gen = ld_acquire_gpu(&st->gen);
    const int H = d->H, W = d->W;
    const size_t N = (size_t)H * W;
    const int ntx = (W + kTW2 - 1) / kTW2, nty = (H + TH - 1) / TH;
    const int nitems = 3 * ntx * nty;
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float eps = d->eps, tau = d->tau, wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;
    const bool dirichlet = d->dirichlet != 0;
    float2 *__restrict__ part = d->part;
    const int nblk = d->nblk;
    int k = 0;
    bool failed = false;
    const int iters = d->depth;
    for (int it = 0; it < iters; ++it) {
        const int cur = __ldcg(&st->cur);
        const int n_it = __ldcg(&st->n);
        const bool rev = (n_it & 1) != 0;
        const bool two = __ldcg(&st->tb2) != 0;
        const CUtensorMap *tm_u = cur ? &tm_ub : &tm_ua;
        float *__restrict__ uout = static_cast<float *>(d->u[cur ^ 1]);
        // position q in the iteration's walk order -> item (odd n walk backwards);
        // the positions are handed out as in k_sweep_tma: blockIdx.x, blockIdx.x
        // + G, then 2G + a counter the grid shares for the iteration
        auto item_at = [&](int q) { return rev ? nitems - 1 - q : q; };
        unsigned *ctr = &st->work[n_it & 1];
        auto tile_xy = [&](int item, int &c, int &x0, int &y0) {
            const int tile = item / 3;
            c = item - 3 * tile;
            x0 = (tile % ntx) * kTW2;
            y0 = (tile / ntx) * TH;
            return tile;
        };
        auto issue = [&](int j) {
            int c, x0, y0;
            tile_xy(item_at(j), c, x0, y0);
            mbar_arrive_expect_tx(&bar, P::TX);
            tma_load_3d(smem + P::U0_OFF, tm_u, &bar, x0 - 8, y0 - 4, c);
            tma_load_3d(smem + P::PHI_OFF, &tm_phi, &bar, x0 - 4, y0 - 2, c);
            tma_load_2d(smem + P::LAM_OFF, &tm_lam, &bar, x0 - 4, y0 - 2);
        };
        auto prefetch = [&](int j) {
            int c, x0, y0;
            tile_xy(item_at(j), c, x0, y0);
            tma_prefetch_3d(tm_u, x0 - 8, y0 - 4, c);
            tma_prefetch_3d(&tm_phi, x0 - 4, y0 - 2, c);
            tma_prefetch_2d(&tm_lam, x0 - 4, y0 - 2);
        };
        int q = (int)blockIdx.x;  // current position (every thread)
        int qn = q + G;           // next position (thread 0)
        if (threadIdx.x == 0) {
            if (it > 0) fence_proxy_async_global();
            if (q < nitems) issue(q);
        }
        for (; q < nitems; ++k) {
            int c, x0, y0;
            const int tile = tile_xy(item_at(q), c, x0, y0);
            if (threadIdx.x == 0 && qn < nitems) prefetch(qn);
            const bool ok = mbar_wait_bounded(&bar, k & 1, kWaitLimitCycles);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            // the reflecting boundary on the u^n tile (rows / columns 1-2 outside)
            if (!dirichlet && (x0 < 8 || y0 < 4 || x0 + kTW2 + 8 > W || y0 + TH + 4 > H)) {
                reflect_border(s0, SW, SW, TH + 8, x0 - 8, y0 - 4, H, W);
                fence_proxy_async_smem();  // these writes precede the next TMA load into this buffer
            }
            __syncthreads();
            // (thread 0) the position after the next one, taken here so that no
            // block barrier waits for the atomic before the end of step 1
            int qa = nitems;
            if (threadIdx.x == 0 && qn < nitems) qa = 2 * G + (int)atomicAdd(ctr, 1u);

            // step 1: region rows y0-2 .. y0+TH+1, columns x0-4 .. x0+123 (frame row t, column 4*lane + j)
            float rs0 = 0.f, rc0 = 0.f, rs1 = 0.f, rc1 = 0.f;
            {
                const int xo = x0 - 4 + 4 * lane;  // output column of this lane's first pixel
                const bool colin = lane >= 1 && lane <= 30 && xo < W;
                float *__restrict__ gout = uout + c * N;
                auto pl = [&](int t, float *ph, float *la) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(sphi + t * kTW + 4 * lane);
                    const float4 l4 = *reinterpret_cast<const float4 *>(slam + t * kTW + 4 * lane);
                    ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                    la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
                };
                auto sink = [&](int t, const float *nu, const float *F) {
                    const int yo = y0 - 2 + t;
                    const bool in = colin && t >= 2 && t < TH + 2 && yo < H;
                    if (in) {
                        float q = 0.f;
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) q = fmaf(F[jj], F[jj], q);
                        neumaier_add(rs0, rc0, q);
                    }
                    if (two) {
                        *reinterpret_cast<float4 *>(s1 + t * SW + 4 * lane) = make_float4(nu[0], nu[1], nu[2], nu[3]);
                    } else if (in) {
                        *reinterpret_cast<float4 *>(gout + (size_t)yo * W + xo) = make_float4(nu[0], nu[1], nu[2], nu[3]);
                    }
                };
                walk_rows<R1, SW, float, EDGE>(s0 + 0 * SW, w * R1, lane, eps, tau, wg0, wg1, wg2, pl, sink);
            }
            if (two) {
                __syncthreads();
                // boundary rule on u^{n+1} (shared rows y0-2.., columns x0-4..)
                if (x0 < 4 || y0 < 4 || x0 + kTW2 + 4 > W || y0 + TH + 4 > H) {
                    if (dirichlet) {
                        for (int e = threadIdx.x; e < (TH + 4) * kTW; e += NW * 32) {
                            const int r = e / kTW, q = e - r * kTW;
                            const int gy = y0 - 2 + r, gx = x0 - 4 + q;
                            if (gy < 0 || gy >= H || gx < 0 || gx >= W) s1[r * SW + q] = 0.f;
                        }
                    } else {
                        reflect_border(s1, SW, kTW, TH + 4, x0 - 4, y0 - 2, H, W);
                    }
                    __syncthreads();
                }
                // step 2: the tile (frame row t = output row y0 + t, column x0 + 4*lane + j)
                const int xo = x0 + 4 * lane;
                const bool colin = lane < 30 && xo < W;
                float *__restrict__ gout = uout + c * N;
                auto pl = [&](int t, float *ph, float *la) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(sphi + (t + 2) * kTW + 4 + 4 * lane);
                    const float4 l4 = *reinterpret_cast<const float4 *>(slam + (t + 2) * kTW + 4 + 4 * lane);
                    ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                    la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
                };
                auto sink = [&](int t, const float *nu, const float *F) {
                    const int yo = y0 + t;
                    if (!colin || yo >= H) return;
                    float q = 0.f;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) q = fmaf(F[jj], F[jj], q);
                    neumaier_add(rs1, rc1, q);
                    *reinterpret_cast<float4 *>(gout + (size_t)yo * W + xo) = make_float4(nu[0], nu[1], nu[2], nu[3]);
                };
                walk_rows<R2, SW, float, EDGE>(s1, w * R2, lane, eps, tau, wg0, wg1, wg2, pl, sink);
            }
            if (threadIdx.x == 0) s_next = qn;  // read after the barrier below
            const float2 t0 = block_pair_sum<NW>(rs0, rc0, red[0]);  // ends with a barrier
            const float2 t1 = block_pair_sum<NW>(rs1, rc1, red[1]);
            const int qnext = s_next;
            if (threadIdx.x == 0) {
                part[(size_t)c * nblk + tile] = t0;
                part[(size_t)(3 + c) * nblk + tile] = t1;
                if (qn < nitems) {
                    fence_proxy_async_smem();
                    issue(qn);
                }
                qn = qa;
            }
            __syncthreads();
            q = qnext;
        }
        if (failed) {
            if (q < nitems) mbar_wait_bounded(&bar, k & 1, kWaitLimitCycles);  // the load in flight
            if (threadIdx.x == 0) atomicCAS(&st->err, 0, DH_ETIMEOUT);
        }
        // grid barrier; the last CTA to arrive decides (an acquire-release
        // arrival: it publishes this CTA's tiles, the last one sees everyone's)
        fence_proxy_async_global();
        __syncthreads();
        if (threadIdx.x == 0) {
            s_last = atom_add_acq_rel_gpu(&st->arrive, 1u) == (unsigned)G - 1u;
            s_timeout = 0;
        }
        __syncthreads();
        if (s_last) {
            const int next = finish_tb2(d, st, it == iters - 1);
            if (threadIdx.x == 0) {
                st->work[next & 1] = 0u;  // every CTA is past its last take of this iteration
                st_release_gpu(&st->gen, gen + 1u);
            }
        } else if (threadIdx.x == 0) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&st->gen) == gen) {
                if (clock64() - t0 > kWaitLimitCycles) {
                    s_timeout = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        ++gen;
        __syncthreads();
        if (s_timeout) {
            if (threadIdx.x == 0) {
                atomicCAS(&st->err, 0, DH_ETIMEOUT);
                st->status = DH_ETIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (__ldcg(&st->done) || failed) return;
    }
}

// Streaming sweep (W % 4 == 0, 16-byte aligned planes).  Each warp owns
// segments of a 128-column strip of one channel (tasks) and walks their rows
// top to bottom.  Lane 0 streams rows into a per-warp ring of NSLOT row slots
// (u with a 4-column halo, Phi, lambda), one TMA load per array and row, one
// mbarrier per slot, refilling a slot as soon as the walk has consumed it.
// The vertical reflecting boundary is applied by loading the reflected row,
// the horizontal one by substituting the reflected columns in registers.
// Rows are unrolled in blocks of 20 (the period of the 4- and 5-row register
// rings), so a segment is a multiple of 20 rows.
constexpr int kStreamUnroll = 20;
constexpr uint32_t kRowU = (kTW + 8) * 4;     // 544 bytes
constexpr uint32_t kRowPhiOff = 640;          // 128-byte aligned offsets in a slot
constexpr uint32_t kRowLamOff = 1152;
constexpr uint32_t kRowBytes = 1664;

template <int NW, int NSLOT, bool EDGE>
__global__ void __launch_bounds__(NW * 32)
k_sweep_stream(const __grid_constant__ CUtensorMap tm_ua, const __grid_constant__ CUtensorMap tm_ub,
               const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_lam,
               const SolveDesc *__restrict__ d, int seg) {
    static_assert(NSLOT >= 4 && (NSLOT & (NSLOT - 1)) == 0, "NSLOT: power of two >= 4");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t bars[NW][NSLOT];
    __shared__ int s_last;

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    const int H = d->H, W = d->W;
    const int cur = __ldcg(&st->cur);
    const CUtensorMap *tm_u = cur ? &tm_ub : &tm_ua;
    float *__restrict__ ubase = static_cast<float *>(d->u[cur ^ 1]);
    const size_t N = (size_t)H * W;
    const int ntx = (W + kTW - 1) / kTW;
    const int nseg = (H + seg - 1) / seg;
    const int ntasks = 3 * ntx * nseg;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * NW + w, GW = gridDim.x * NW;
    const int mytasks = gw < ntasks ? (ntasks - 1 - gw) / GW + 1 : 0;
    const int P = seg + 4;  // stream positions per task: u rows y0-2 .. y0+seg+1
    const int total = mytasks * P;
    unsigned char *ring = smem + (size_t)w * NSLOT * kRowBytes;
    uint64_t *bar = bars[w];
    const float eps = d->eps, tau = d->tau, wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;
    float2 *__restrict__ part = d->part;
    const int nblk = d->nblk;

    if (lane == 0) {
        for (int k = 0; k < NSLOT; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // task k of this warp -> (channel, strip, segment)
    auto task_of = [&](int k, int &c, int &x0, int &y0, int &tile) {
        const int t = gw + k * GW;
        c = t % 3;
        const int r = t / 3;
        tile = r;
        x0 = (r % ntx) * kTW;
        y0 = (r / ntx) * seg;
    };
    // Lane 0's issue cursor: positions are issued strictly in order, one per
    // released slot, so the (task, row) of the next position is advanced
    // incrementally.
    int iss_pos = 0, iss_k = 0, iss_o = 0, iss_c = 0, iss_x0 = 0, iss_y0 = 0, iss_tile = 0;
    if (mytasks > 0) task_of(0, iss_c, iss_x0, iss_y0, iss_tile);
    auto issue_next = [&]() {  // lane 0 only
        if (iss_pos >= total) return;
        const int Y = reflect_idx(iss_y0 - 2 + iss_o, H);
        const bool pl = iss_o >= 2 && iss_o < seg + 2;
        const int slot = iss_pos & (NSLOT - 1);
        unsigned char *sb = ring + slot * kRowBytes;
        mbar_arrive_expect_tx(&bar[slot], kRowU + (pl ? 2 * kTW * 4 : 0));
        tma_load_3d(sb, tm_u, &bar[slot], iss_x0 - 4, Y, iss_c);
        if (pl) {
            tma_load_3d(sb + kRowPhiOff, &tm_phi, &bar[slot], iss_x0, Y, iss_c);
            tma_load_2d(sb + kRowLamOff, &tm_lam, &bar[slot], iss_x0, Y);
        }
        ++iss_pos;
        if (++iss_o == P) {
            iss_o = 0;
            if (++iss_k < mytasks) task_of(iss_k, iss_c, iss_x0, iss_y0, iss_tile);
        }
    };
    if (lane == 0)
        for (int k = 0; k < NSLOT; ++k) issue_next();

    bool failed = false;
    int waited = 0;  // positions [0, waited) have been waited for
    auto wait_pos = [&](int pos) -> const unsigned char * {
        const int slot = pos & (NSLOT - 1);
        const uint32_t parity = (uint32_t)((pos / NSLOT) & 1);
        const bool ok = mbar_wait_bounded(&bar[slot], parity, kWaitLimitCycles);
        if (__any_sync(0xffffffffu, !ok)) failed = true;
        waited = pos + 1;
        return ring + slot * kRowBytes;
    };
    // The walk is done with the oldest slot in use: refill it with the next position.
    auto release = [&]() {
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            issue_next();
        }
    };

    const float2 W0 = make_float2(wg0, wg0), W1 = make_float2(wg1, wg1), W2 = make_float2(wg2, wg2);
    const float2 E2 = make_float2(eps, eps), HALF = make_float2(0.5f, 0.5f), TAU = make_float2(tau, tau);
    const float2 MONE = make_float2(-1.f, -1.f);
    auto gauss = [&](float2 m2, float2 m1, float2 c0, float2 p1, float2 p2) {
        return fma2(W2, add2(m2, p2), fma2(W1, add2(m1, p1), mul2(W0, c0)));
    };

    for (int k = 0; k < mytasks && !failed; ++k) {
        int c, x0, y0, tile;
        task_of(k, c, x0, y0, tile);
        const int p0 = k * P;
        const int x = x0 + 4 * lane;
        const bool left = x == 0, right = x + 4 == W;
        auto load_row = [&](const unsigned char *sb, RowU &u, float2 *g) {
            const float *row = reinterpret_cast<const float *>(sb) + 4 * lane;
            float4 L = *reinterpret_cast<const float4 *>(row);
            const float4 C = *reinterpret_cast<const float4 *>(row + 4);
            float4 Rr = *reinterpret_cast<const float4 *>(row + 8);
            if (left) { L.z = C.y; L.w = C.x; }     // u(-2) = u(1), u(-1) = u(0)
            if (right) { Rr.x = C.w; Rr.y = C.z; }  // u(W) = u(W-1), u(W+1) = u(W-2)
            const float2 e0 = make_float2(L.z, L.w), e3 = make_float2(Rr.x, Rr.y);
            u.o0 = make_float2(L.w, C.x);
            u.e1 = make_float2(C.x, C.y);
            u.o1 = make_float2(C.y, C.z);
            u.e2 = make_float2(C.z, C.w);
            u.o2 = make_float2(C.w, Rr.x);
            g[0] = gauss(e0, u.o0, u.e1, u.o1, u.e2);
            g[1] = gauss(u.e1, u.o1, u.e2, u.o2, e3);
        };
        auto yfaces = [&](const RowU &a, const RowU &b, float2 *f) {
            f[0] = face_flux2<EDGE>(sub2(b.e1, a.e1), mul2(HALF, sub2(a.o1, a.o0)), E2);
            f[1] = face_flux2<EDGE>(sub2(b.e2, a.e2), mul2(HALF, sub2(a.o2, a.o1)), E2);
        };
        RowU uu[4];
        float2 gh[5][2];
        float2 fyu[2];
        {
            RowU dummy;
            load_row(wait_pos(p0 + 0), dummy, gh[0]);
            load_row(wait_pos(p0 + 1), uu[0], gh[1]);
            load_row(wait_pos(p0 + 2), uu[1], gh[2]);
            load_row(wait_pos(p0 + 3), uu[2], gh[3]);
            yfaces(uu[0], uu[1], fyu);
            release();  // rows y0-2, y0-1 carry no Phi/lambda: done with them
            release();
        }
        if (failed) break;
        float rs = 0.f, rc = 0.f;
        float *__restrict__ un = ubase + c * N;
        for (int m = 0; m < seg; m += kStreamUnroll) {
#pragma unroll
            for (int j = 0; j < kStreamUnroll; ++j) {
                const int i = m + j;
                const RowU &um = uu[(j + 0) & 3];
                const RowU &u0 = uu[(j + 1) & 3];
                const RowU &up = uu[(j + 2) & 3];
                load_row(wait_pos(p0 + 4 + i), uu[(j + 3) & 3], gh[(j + 4) % 5]);
                const unsigned char *sbo = ring + ((p0 + 2 + i) & (NSLOT - 1)) * kRowBytes;
                const float4 p4 = *reinterpret_cast<const float4 *>(sbo + kRowPhiOff + 16 * lane);
                const float4 l4 = *reinterpret_cast<const float4 *>(sbo + kRowLamOff + 16 * lane);
                const float2 *g_m2 = gh[(j + 0) % 5], *g_m1 = gh[(j + 1) % 5], *g_0 = gh[(j + 2) % 5];
                const float2 *g_p1 = gh[(j + 3) % 5], *g_p2 = gh[(j + 4) % 5];
                const float2 fxA = face_flux2<EDGE>(sub2(u0.e1, u0.o0), mul2(HALF, sub2(up.o0, um.o0)), E2);
                const float2 fxB = face_flux2<EDGE>(sub2(u0.e2, u0.o1), mul2(HALF, sub2(up.o1, um.o1)), E2);
                const float fx4 = face_flux<EDGE>(__fsub_rn(u0.o2.y, u0.o2.x), half_diff(up.o2.x, um.o2.x), eps);
                float2 fyd[2];
                yfaces(u0, up, fyd);
                const float2 dxA = make_float2(__fsub_rn(fxA.y, fxA.x), __fsub_rn(fxB.x, fxA.y));
                const float2 dxB = make_float2(__fsub_rn(fxB.y, fxB.x), __fsub_rn(fx4, fxB.y));
                const float2 dvA = add2(dxA, sub2(fyd[0], fyu[0]));
                const float2 dvB = add2(dxB, sub2(fyd[1], fyu[1]));
                const float2 GA = gauss(g_m2[0], g_m1[0], g_0[0], g_p1[0], g_p2[0]);
                const float2 GB = gauss(g_m2[1], g_m1[1], g_0[1], g_p1[1], g_p2[1]);
                const float2 FA = add2(fma2(mul2(MONE, make_float2(l4.x, l4.y)), GA, dvA), make_float2(p4.x, p4.y));
                const float2 FB = add2(fma2(mul2(MONE, make_float2(l4.z, l4.w)), GB, dvB), make_float2(p4.z, p4.w));
                const float2 nA = fma2(TAU, FA, u0.e1);
                const float2 nB = fma2(TAU, FB, u0.e2);
                fyu[0] = fyd[0];
                fyu[1] = fyd[1];
                const int y = y0 + i;
                if (y < H && x < W) {
                    const float2 q2 = fma2(FB, FB, mul2(FA, FA));
                    neumaier_add(rs, rc, __fadd_rn(q2.x, q2.y));
                    *reinterpret_cast<float4 *>(un + (size_t)y * W + x) = make_float4(nA.x, nA.y, nB.x, nB.y);
                }
                release();
            }
            if (failed) break;
        }
        if (failed) break;
        release();  // look-ahead rows of the segment's end
        release();
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, rs, off);
            const float c2 = __shfl_down_sync(0xffffffffu, rc, off);
            neumaier_merge(rs, rc, s2, c2);
        }
        if (lane == 0) part[(size_t)c * nblk + tile] = make_float2(rs, rc);
    }
    if (failed) {
        // let the loads this warp still has in flight land (bounded), then report
        const int issued = __shfl_sync(0xffffffffu, iss_pos, 0);
        for (int pos = waited; pos < issued; ++pos)
            mbar_wait_bounded(&bar[pos & (NSLOT - 1)], (uint32_t)((pos / NSLOT) & 1), kWaitLimitCycles);
        if (lane == 0) atomicCAS(&st->err, 0, DH_ETIMEOUT);
    }
    arrive_and_finish(d, st, &s_last);
}


// ---------------------------------------------------------------- K iterations per tile load
// Temporally blocked sweep of depth K (float iterates, W % 4 == 0, 16-byte
// aligned planes): the generalisation of k_sweep_tb2 to K = 2..4.  An item is
// a WO x TH output tile of one channel, WO = 128 - 8(K-1).  All K steps walk
// one frame of 128 columns: lane L owns global columns xf + 4L .. xf + 4L + 3,
// xf = x0 - 4(K-1).  TMA loads u^n on the frame with a 4-column / 2K-row ring
// (136 x (TH + 4K), starting at (x0 - 4K, y0 - 2K)) and Phi / lambda on the
// frame's 128 columns and the TH + 4(K-1) rows of step 1.  Step s (1..K) walks
// the frame rows y0 - 2(K-s) .. y0 + TH + 2(K-s) - 1 from the iterate of step
// s-1 (the TMA tile for s = 1, else a shared buffer in which the boundary rule
// has been applied) and writes u^{n+s} to the other shared buffer, or for s = K
// the output tile to global memory.  Lanes s-1 .. 32-s hold valid values after
// step s; the output lanes are K-1 .. 32-K.  The residual of step s over the
// output tile is F(u^{n+s-1}), the quantity one iteration at a time gives; the
// last CTA at the grid barrier decides with all K of them (finish_tbk): stop
// at n, advance by K, or, when some u^{n+l} with 0 < l < K is the iterate to
// return, switch the rest of the solve to one iteration per load (step 1 writes
// the output tile to global memory), which recomputes u^{n+1} .. and stops there.
template <int K, int RO, int NW>
struct TbkPlan {
    static constexpr int TH = RO * NW;
    static constexpr int WO = kTW - 8 * (K - 1);  // output columns
    static constexpr int SW = kTW + 8;             // 136 floats per shared row
    static constexpr int F1 = TH + 4 * (K - 1);    // frame rows of step 1
    static constexpr uint32_t U0_BYTES = (TH + 4 * K) * SW * 4;
    static constexpr uint32_t PL_BYTES = F1 * kTW * 4;
    static constexpr uint32_t BUF_BYTES = F1 * SW * 4;
    static constexpr uint32_t U0_OFF = 0;
    static constexpr uint32_t PHI_OFF = (U0_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t LAM_OFF = PHI_OFF + PL_BYTES;
    static constexpr uint32_t B0_OFF = (LAM_OFF + PL_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t B1_OFF = (B0_OFF + BUF_BYTES + 1023) / 1024 * 1024;
    static constexpr uint32_t SMEM = (K >= 3 ? B1_OFF + BUF_BYTES : B0_OFF + BUF_BYTES) + 1024;  // + alignment slack
    static constexpr uint32_t TX = U0_BYTES + 2 * PL_BYTES;
    static_assert(K >= 2 && K <= 4, "depth 2..4");
    static_assert((4 * (K - 1)) % NW == 0, "every step's frame rows must split evenly over the warps");
};

// Last CTA of a depth-K sweep: residuals of the K levels, decision.
// Called after an acquire-release arrival; thread 0 loads the state it
// decides with before the partials and returns the next iterate's index (the
// caller publishes the state with a release store).  The while condition is
// set only by a launch that goes on after its last iteration.
template <int K>
static __device__ int finish_tbk(const SolveDesc *d, SolveState *st, bool last_in_launch) {
    constexpr int L3 = 3 * K, U = K >= 4 ? 2 : 4;  // partial loads per level in flight per thread
    __shared__ float2 wsum[L3][32];
    __shared__ float sq[L3];
    const int tid = threadIdx.x, nt = blockDim.x, w = tid >> 5, lane = tid & 31, nw = nt >> 5;
    int n = 0, deep = 0, cur = 0, err = 0;
    float phin2[3] = {0.f, 0.f, 0.f};
    if (tid == 0) {
        n = ld_state_int(&st->n);
        deep = ld_state_int(&st->tb2);
        cur = ld_state_int(&st->cur);
        err = ld_state_int(&st->err);
        for (int c = 0; c < 3; ++c) phin2[c] = __ldcg(&st->phin2[c]);
    }
    const int nblk = d->nblk;
    const float2 *part = d->part;
    float s[L3], cc[L3];
#pragma unroll
    for (int q = 0; q < L3; ++q) s[q] = cc[q] = 0.f;
    for (int b0 = tid; b0 < nblk; b0 += U * nt) {
        float2 v[L3][U];
#pragma unroll
        for (int q = 0; q < L3; ++q)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int b = b0 + j * nt;
                v[q][j] = b < nblk ? __ldcg(part + (size_t)q * nblk + b) : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int q = 0; q < L3; ++q)
#pragma unroll
            for (int j = 0; j < U; ++j) neumaier_merge(s[q], cc[q], v[q][j].x, v[q][j].y);
    }
#pragma unroll
    for (int q = 0; q < L3; ++q) {
        for (int off = 16; off; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s[q], off);
            const float c2 = __shfl_down_sync(0xffffffffu, cc[q], off);
            neumaier_merge(s[q], cc[q], s2, c2);
        }
        if (lane == 0) wsum[q][w] = make_float2(s[q], cc[q]);
    }
    __syncthreads();
    if (tid < L3) {
        float a = wsum[tid][0].x, b = wsum[tid][0].y;
        for (int q = 1; q < nw; ++q) neumaier_merge(a, b, wsum[tid][q].x, wsum[tid][q].y);
        sq[tid] = a + b;
    }
    __syncthreads();
    if (tid != 0) return 0;
    auto rho_of = [&](int lv, float *rho, float &worst) {
        bool finite = true;
        worst = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float pn = phin2[c], q = sq[3 * lv + c];
            rho[c] = pn > 0.f ? sqrtf(q / pn) : sqrtf(q);
            if (!isfinite(rho[c])) finite = false;
            else worst = fmaxf(worst, rho[c]);
        }
        return finite;
    };
    float rho0[3], w0;
    const bool fin0 = rho_of(0, rho0, w0);
    if (d->rho_hist)
        for (int c = 0; c < 3; ++c) d->rho_hist[3 * n + c] = rho0[c];
    const bool conv = fin0 && w0 <= d->tol;
    unsigned cont = 1;
    int next = n;
    if (err || conv || !fin0 || n >= d->max_iter) {
        st->done = 1;
        st->n_final = n;
        st->status = err ? err : (!fin0 ? DH_ENONFINITE : (conv ? DH_OK : DH_WNOCONV));
        for (int c = 0; c < 3; ++c) st->rho[c] = rho0[c];
        cont = 0;
    } else if (!deep) {
        st->n = next = n + 1;
        st->cur = cur ^ 1;
    } else {
        // u^{n+l}, 0 < l < K, is the answer if its residual meets tol, is not
        // finite or n + l reaches max_iter: then redo it one iteration at a time
        bool redo = false;
        for (int l = 1; l < K && !redo; ++l) {
            float rl[3], wl;
            const bool fin = rho_of(l, rl, wl);
            redo = !fin || wl <= d->tol || n + l >= d->max_iter;
        }
        if (redo) {
            st->tb2 = 0;
        } else {
            if (d->rho_hist)
                for (int l = 1; l < K; ++l) {
                    float rl[3], wl;
                    rho_of(l, rl, wl);
                    for (int c = 0; c < 3; ++c) d->rho_hist[3 * (n + l) + c] = rl[c];
                }
            st->n = next = n + K;
            st->cur = cur ^ 1;
        }
    }
    st->arrive = 0;
    if (d->use_cond && cont && last_in_launch) cudaGraphSetConditional(d->cond, 1u);
    return next;
}

// Step S of a depth-K item: walks the step's frame rows from `src` (row 0 =
// global row y0 - 2(K-S+1) + 2 - 2 ... see TbkPlan), accumulates F over the
// output tile into (rs, rc), and writes u^{n+S} to `dst` (S < K, depth mode)
// or the output tile to global memory (S = K, or S = 1 one iteration at a time).
template <int K, int RO, int NW, int S, bool EDGE>
__device__ __forceinline__ void tbk_step(const float *src, float *dst, float *__restrict__ gout, const float *sphi,
                                         const float *slam, bool deep, int x0, int y0, int H, int W, int lane, int w,
                                         float eps, float tau, float wg0, float wg1, float wg2, float &rs, float &rc) {
    using P = TbkPlan<K, RO, NW>;
    constexpr int TH = P::TH, SW = P::SW;
    constexpr int R = RO + 4 * (K - S) / NW;  // rows per warp of this step
    constexpr int T0 = 2 * (K - S);           // first frame row of the output tile
    const int gx = x0 - 4 * (K - 1) + 4 * lane;
    const bool lane_out = lane >= K - 1 && lane <= 32 - K && gx < W;
    const bool to_global = S == K || !deep;
    auto pl = [&](int t, float *ph, float *la) {
        const int r = t + 2 * (S - 1);
        const float4 p4 = *reinterpret_cast<const float4 *>(sphi + r * kTW + 4 * lane);
        const float4 l4 = *reinterpret_cast<const float4 *>(slam + r * kTW + 4 * lane);
        ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
        la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
    };
    auto sink = [&](int t, const float *nu, const float *F) {
        const int gy = y0 - T0 + t;
        const bool in = lane_out && t >= T0 && t < T0 + TH && gy < H;
        if (in) {
            float q = 0.f;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) q = fmaf(F[jj], F[jj], q);
            neumaier_add(rs, rc, q);
        }
        if (!to_global) {
            *reinterpret_cast<float4 *>(dst + t * SW + 4 + 4 * lane) = make_float4(nu[0], nu[1], nu[2], nu[3]);
        } else if (in) {
            *reinterpret_cast<float4 *>(gout + (size_t)gy * W + gx) = make_float4(nu[0], nu[1], nu[2], nu[3]);
        }
    };
    walk_rows<R, SW, float, EDGE>(src, w * R, lane, eps, tau, wg0, wg1, wg2, pl, sink);
}

// The boundary rule on a shared iterate written by step s: its rows start at
// global row ry0, its columns at global column cx0 (= x0 - 4K); nrows rows.
template <int NW>
__device__ __forceinline__ void tbk_boundary(float *buf, int nrows, int cx0, int ry0, int H, int W, bool dirichlet) {
    constexpr int SW = kTW + 8;
    if (dirichlet) {
        for (int e = threadIdx.x; e < nrows * SW; e += NW * 32) {
            const int r = e / SW, q = e - r * SW;
            const int gy = ry0 + r, gx = cx0 + q;
            if (gy < 0 || gy >= H || gx < 0 || gx >= W) buf[e] = 0.f;
        }
    } else {
        reflect_border(buf, SW, SW, nrows, cx0, ry0, H, W);
    }
}

template <int K, int RO, int NW, bool EDGE, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
k_sweep_tbk(const __grid_constant__ CUtensorMap tm_ua, const __grid_constant__ CUtensorMap tm_ub,
            const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_lam,
            const SolveDesc *__restrict__ d) {
    using P = TbkPlan<K, RO, NW>;
    constexpr int TH = P::TH, WO = P::WO, SW = P::SW;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float2 red[K][NW];
    __shared__ int s_last, s_timeout, s_next;
    float *s0 = reinterpret_cast<float *>(smem + P::U0_OFF);
    const float *sphi = reinterpret_cast<const float *>(smem + P::PHI_OFF);
    const float *slam = reinterpret_cast<const float *>(smem + P::LAM_OFF);
    float *b0 = reinterpret_cast<float *>(smem + P::B0_OFF);
    float *b1 = reinterpret_cast<float *>(smem + (K >= 3 ? P::B1_OFF : P::B0_OFF));

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    unsigned gen = ld_acquire_gpu(&st->gen);
    const int H = d->H, W = d->W;
    const size_t N = (size_t)H * W;
    const int ntx = (W + WO - 1) / WO, nty = (H + TH - 1) / TH;
    const int nitems = 3 * ntx * nty;
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float eps = d->eps, tau = d->tau, wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;
    const bool dirichlet = d->dirichlet != 0;
    float2 *__restrict__ part = d->part;
    const int nblk = d->nblk;
    int k = 0;
    bool failed = false;
    const int iters = d->depth;
    for (int it = 0; it < iters; ++it) {
        const int cur = __ldcg(&st->cur);
        const int n_it = __ldcg(&st->n);
        const bool rev = (n_it & 1) != 0;
        const bool deep = __ldcg(&st->tb2) != 0;
        const CUtensorMap *tm_u = cur ? &tm_ub : &tm_ua;
        float *__restrict__ uout = static_cast<float *>(d->u[cur ^ 1]);
        // position q in the iteration's walk order -> item (odd n walk backwards);
        // the positions are handed out as in k_sweep_tma: blockIdx.x, blockIdx.x
        // + G, then 2G + a counter the grid shares for the iteration
        auto item_at = [&](int q) { return rev ? nitems - 1 - q : q; };
        unsigned *ctr = &st->work[n_it & 1];
        auto tile_xy = [&](int item, int &c, int &x0, int &y0) {
            const int tile = item / 3;
            c = item - 3 * tile;
            x0 = (tile % ntx) * WO;
            y0 = (tile / ntx) * TH;
            return tile;
        };
        auto issue = [&](int j) {
            int c, x0, y0;
            tile_xy(item_at(j), c, x0, y0);
            mbar_arrive_expect_tx(&bar, P::TX);
            tma_load_3d(smem + P::U0_OFF, tm_u, &bar, x0 - 4 * K, y0 - 2 * K, c);
            tma_load_3d(smem + P::PHI_OFF, &tm_phi, &bar, x0 - 4 * (K - 1), y0 - 2 * (K - 1), c);
            tma_load_2d(smem + P::LAM_OFF, &tm_lam, &bar, x0 - 4 * (K - 1), y0 - 2 * (K - 1));
        };
        auto prefetch = [&](int j) {
            int c, x0, y0;
            tile_xy(item_at(j), c, x0, y0);
            tma_prefetch_3d(tm_u, x0 - 4 * K, y0 - 2 * K, c);
            tma_prefetch_3d(&tm_phi, x0 - 4 * (K - 1), y0 - 2 * (K - 1), c);
            tma_prefetch_2d(&tm_lam, x0 - 4 * (K - 1), y0 - 2 * (K - 1));
        };
        int q = (int)blockIdx.x;  // current position (every thread)
        int qn = q + G;           // next position (thread 0)
        if (threadIdx.x == 0) {
            if (it > 0) fence_proxy_async_global();
            if (q < nitems) issue(q);
        }
        for (; q < nitems; ++k) {
            int c, x0, y0;
            const int tile = tile_xy(item_at(q), c, x0, y0);
            if (threadIdx.x == 0 && qn < nitems) prefetch(qn);
            const bool ok = mbar_wait_bounded(&bar, k & 1, kWaitLimitCycles);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const int cx0 = x0 - 4 * K;  // global column of shared column 0 (every buffer)
            const bool border = cx0 < 0 || y0 - 2 * K < 0 || cx0 + SW > W || y0 + TH + 2 * K > H;
            if (border && !dirichlet) {  // the reflecting boundary on the u^n tile
                reflect_border(s0, SW, SW, TH + 4 * K, cx0, y0 - 2 * K, H, W);
                fence_proxy_async_smem();  // these writes precede the next TMA load into this buffer
            }
            __syncthreads();
            // (thread 0) the position after the next one, taken here so that no
            // block barrier waits for the atomic before the end of step 1
            int qa = nitems;
            if (threadIdx.x == 0 && qn < nitems) qa = 2 * G + (int)atomicAdd(ctr, 1u);
            float rs[K], rc[K];
#pragma unroll
            for (int l = 0; l < K; ++l) rs[l] = rc[l] = 0.f;
            float *__restrict__ gout = uout + c * N;
            tbk_step<K, RO, NW, 1, EDGE>(s0, b0, gout, sphi, slam, deep, x0, y0, H, W, lane, w, eps, tau, wg0, wg1,
                                         wg2, rs[0], rc[0]);
            if (deep) {
                __syncthreads();
                if (border) {
                    tbk_boundary<NW>(b0, TH + 4 * (K - 1), cx0, y0 - 2 * (K - 1), H, W, dirichlet);
                    __syncthreads();
                }
                tbk_step<K, RO, NW, 2, EDGE>(b0, b1, gout, sphi, slam, deep, x0, y0, H, W, lane, w, eps, tau, wg0,
                                             wg1, wg2, rs[1], rc[1]);
                if constexpr (K >= 3) {
                    __syncthreads();
                    if (border) {
                        tbk_boundary<NW>(b1, TH + 4 * (K - 2), cx0, y0 - 2 * (K - 2), H, W, dirichlet);
                        __syncthreads();
                    }
                    tbk_step<K, RO, NW, 3, EDGE>(b1, b0, gout, sphi, slam, deep, x0, y0, H, W, lane, w, eps, tau,
                                                 wg0, wg1, wg2, rs[2], rc[2]);
                }
                if constexpr (K >= 4) {
                    __syncthreads();
                    if (border) {
                        tbk_boundary<NW>(b0, TH + 4 * (K - 3), cx0, y0 - 2 * (K - 3), H, W, dirichlet);
                        __syncthreads();
                    }
                    tbk_step<K, RO, NW, 4, EDGE>(b0, b1, gout, sphi, slam, deep, x0, y0, H, W, lane, w, eps, tau,
                                                 wg0, wg1, wg2, rs[3], rc[3]);
                }
            }
            if (threadIdx.x == 0) s_next = qn;  // read after the barriers below
            float2 tot[K];
#pragma unroll
            for (int l = 0; l < K; ++l) tot[l] = block_pair_sum<NW>(rs[l], rc[l], red[l]);  // each ends with a barrier
            const int qnext = s_next;
            if (threadIdx.x == 0) {
#pragma unroll
                for (int l = 0; l < K; ++l) part[(size_t)(3 * l + c) * nblk + tile] = tot[l];
                if (qn < nitems) {
                    fence_proxy_async_smem();
                    issue(qn);
                }
                qn = qa;
            }
            __syncthreads();
            q = qnext;
        }
        if (failed) {
            if (q < nitems) mbar_wait_bounded(&bar, k & 1, kWaitLimitCycles);  // the load in flight
            if (threadIdx.x == 0) atomicCAS(&st->err, 0, DH_ETIMEOUT);
        }
        // grid barrier; the last CTA to arrive decides (an acquire-release
        // arrival: it publishes this CTA's tiles, the last one sees everyone's)
        fence_proxy_async_global();
        __syncthreads();
        if (threadIdx.x == 0) {
            s_last = atom_add_acq_rel_gpu(&st->arrive, 1u) == (unsigned)G - 1u;
            s_timeout = 0;
        }
        __syncthreads();
        if (s_last) {
            const int next = finish_tbk<K>(d, st, it == iters - 1);
            if (threadIdx.x == 0) {
                st->work[next & 1] = 0u;  // every CTA is past its last take of this iteration
                st_release_gpu(&st->gen, gen + 1u);
            }
        } else if (threadIdx.x == 0) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&st->gen) == gen) {
                if (clock64() - t0 > kWaitLimitCycles) {
                    s_timeout = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        ++gen;
        __syncthreads();
        if (s_timeout) {
            if (threadIdx.x == 0) {
                atomicCAS(&st->err, 0, DH_ETIMEOUT);
                st->status = DH_ETIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (__ldcg(&st->done) || failed) return;
    }
}

// ---------------------------------------------------------------- warp-specialised TMA sweep
// Reflects the border halo cells (see reflect_border) in shared-memory rows
// [r0, r0 + nr) of a staged tile, by the 32 lanes of one warp: exactly the
// rows that warp's walk reads.  A cell another warp also reflects receives
// the same value from both; the sources lie inside the image and are never
// written.
template <class T>
__device__ __forceinline__ void reflect_rows_warp(T *s, int stride, int ncols, int r0, int nr, int cx0, int ry0,
                                                  int H, int W, int lane) {
    for (int r = r0; r < r0 + nr; ++r) {
        const int gy = ry0 + r;
        if (gy < -2 || gy > H + 1) continue;  // never read by a stored output
        if (gy < 0 || gy >= H) {
            const int sy = reflect_idx(gy, H) - ry0;
            for (int q = lane; q < ncols; q += 32) {
                const int gx = cx0 + q;
                if (gx < -2 || gx > W + 1) continue;
                s[r * stride + q] = s[sy * stride + reflect_idx(gx, W) - cx0];
            }
        } else if (lane < 4) {
            const int g = lane < 2 ? lane - 2 : W + lane - 2;  // -2, -1, W, W + 1
            const int q = g - cx0;
            if (q >= 0 && q < ncols) s[r * stride + q] = s[r * stride + reflect_idx(g, W) - cx0];
        }
    }
}

// TMA sweep with one producer warp and NW compute warps per CTA (W % 4 == 0,
// 16-byte aligned planes).  Persistent CTAs walk the (tile, channel) items as
// k_sweep_tma does.  Lane 0 of the producer warp loads each item's u^n tile
// (with halo) and, when PL_SMEM, its Phi and lambda tiles into a ring of
// STAGES stages by TMA (full[s] completes on the transaction bytes), pulls
// the item STAGES further on into L2, and refills a stage once all NW compute
// warps have released it (empty[s], NW arrivals); at that point it also merges
// the NW per-warp residual partials the warps left in the stage's slots, in
// warp order (the same order as block_pair_sum), into the item's partial.
// Compute warp w walks rows [w*R, w*R + R) of every item: it reflects the
// border cells its own walk reads, walks, reduces its residual over the warp,
// stores it in the slot and releases the stage.  No block barrier is taken
// inside an iteration, so a warp that finishes early goes on to the next
// staged item.  MULTI: as k_sweep_tma, up to d->depth iterations per
// cooperative launch with a grid barrier between them.
template <int R, int NW, int STAGES, bool PL_SMEM, class T, bool EDGE, int MINB, bool MULTI>
__global__ void __launch_bounds__((NW + 1) * 32, MINB)
k_sweep_ws(const __grid_constant__ CUtensorMap tm_ua, const __grid_constant__ CUtensorMap tm_ub,
           const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_lam,
           const SolveDesc *__restrict__ d) {
    constexpr int TH = R * NW;
    constexpr int HALO = Store<T>::HALO;
    using P = TmaPlan<TH, PL_SMEM, T>;
    constexpr int SW = P::SW, SH = P::SH;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_align1024(smem_raw);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    __shared__ float2 slot[STAGES][NW];
    __shared__ int s_last, s_timeout;
    __shared__ volatile int s_fail;

    SolveState *st = d->st;
    clear_condition(d);
    if (__ldcg(&st->done)) return;
    unsigned gen = 0;
    if (MULTI) gen = ld_acquire_gpu(&st->gen);  // before this CTA can arrive anywhere
    const int H = d->H, W = d->W;
    const size_t N = (size_t)H * W;
    const int ntx = (W + kTW - 1) / kTW, nty = (H + TH - 1) / TH;
    const int ntiles = ntx * nty, nitems = 3 * ntiles;
    const int G = gridDim.x;
    const int m = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / G + 1 : 0;  // items of this CTA

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], NW);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float eps = d->eps, tau = d->tau, wg0 = d->wg0, wg1 = d->wg1, wg2 = d->wg2;
    const bool dirichlet = d->dirichlet != 0;
    const float *__restrict__ phi_all = d->phi;
    const float *__restrict__ glam = d->lam;
    float2 *__restrict__ part = d->part;
    const int nblk = d->nblk;
    const int iters = MULTI ? d->depth : 1;
    int k = 0;        // ring position of this CTA's first item in the current iteration
    int issued = 0;   // producer: ring positions whose loads were issued
    for (int it = 0; it < iters; ++it) {
        const int cur = __ldcg(&st->cur);
        const bool rev = (__ldcg(&st->n) & 1) != 0;
        const CUtensorMap *tm_u = cur ? &tm_ub : &tm_ua;
        T *__restrict__ ubase = static_cast<T *>(d->u[cur ^ 1]);
        auto item_at = [&](int j) { return (int)blockIdx.x + (rev ? m - 1 - j : j) * G; };
        auto tile_xy = [&](int item, int &c, int &x0, int &y0) {
            const int tile = item / 3;
            c = item - 3 * tile;
            x0 = (tile % ntx) * kTW;
            y0 = (tile / ntx) * TH;
            return tile;
        };
        if (w == NW) {
            if (lane == 0) {
                // item j's partial from the NW slots of its stage, in warp order
                auto store_partial = [&](int j, int stage) {
                    int c, x0, y0;
                    const int tile = tile_xy(item_at(j), c, x0, y0);
                    float a = slot[stage][0].x, b = slot[stage][0].y;
#pragma unroll
                    for (int q = 1; q < NW; ++q) neumaier_merge(a, b, slot[stage][q].x, slot[stage][q].y);
                    part[(size_t)c * nblk + tile] = make_float2(a, b);
                };
                if (MULTI && it > 0) fence_proxy_async_global();
                for (int j = 0; j < m; ++j) {
                    const int kk = k + j, stage = kk % STAGES;
                    if (kk >= STAGES) {  // the stage held ring position kk - STAGES
                        if (!mbar_wait_bounded(&empty[stage], (uint32_t)((kk / STAGES) - 1) & 1u, kWaitLimitCycles)) {
                            s_fail = 1;
                            break;
                        }
                        if (j >= STAGES) store_partial(j - STAGES, stage);
                    }
                    if (s_fail) break;
                    int c, x0, y0;
                    tile_xy(item_at(j), c, x0, y0);
                    unsigned char *sb = smem + stage * P::STAGE;
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&full[stage], P::TX);
                    tma_load_3d(sb + P::U_OFF, tm_u, &full[stage], x0 - HALO, y0 - 2, c);
                    if (PL_SMEM) {
                        tma_load_3d(sb + P::PHI_OFF, &tm_phi, &full[stage], x0, y0, c);
                        tma_load_2d(sb + P::LAM_OFF, &tm_lam, &full[stage], x0, y0);
                    }
                    ++issued;
                    if (j + STAGES < m) {
                        int c2, x2, y2;
                        tile_xy(item_at(j + STAGES), c2, x2, y2);
                        tma_prefetch_3d(tm_u, x2 - HALO, y2 - 2, c2);
                        if (PL_SMEM) {
                            tma_prefetch_3d(&tm_phi, x2, y2, c2);
                            tma_prefetch_2d(&tm_lam, x2, y2);
                        }
                    }
                }
                // the partials of the last items (not yet waited for)
                for (int j = m > STAGES ? m - STAGES : 0; j < m && !s_fail; ++j) {
                    const int kk = k + j, stage = kk % STAGES;
                    if (!mbar_wait_bounded(&empty[stage], (uint32_t)(kk / STAGES) & 1u, kWaitLimitCycles)) {
                        s_fail = 1;
                        break;
                    }
                    store_partial(j, stage);
                }
            }
        } else {
            for (int j = 0; j < m; ++j) {
                const int kk = k + j, stage = kk % STAGES;
                const bool ok = mbar_wait_bounded(&full[stage], (uint32_t)(kk / STAGES) & 1u, kWaitLimitCycles);
                if (__any_sync(0xffffffffu, !ok)) {
                    if (lane == 0) s_fail = 1;
                    break;
                }
                if (s_fail) break;
                int c, x0, y0;
                tile_xy(item_at(j), c, x0, y0);
                unsigned char *sb = smem + stage * P::STAGE;
                T *s = reinterpret_cast<T *>(sb + P::U_OFF);
                const float *sphi = reinterpret_cast<const float *>(sb + P::PHI_OFF);
                const float *slam = reinterpret_cast<const float *>(sb + P::LAM_OFF);
                const bool border = !dirichlet && (x0 == 0 || y0 == 0 || x0 + kTW + 2 > W || y0 + TH + 2 > H);
                if (border) {
                    reflect_rows_warp(s, SW, SW, w * R, R + 4, x0 - HALO, y0 - 2, H, W, lane);
                    __syncwarp();
                }
                T *__restrict__ un = ubase + c * N;
                const int x = x0 + 4 * lane;
                float rs = 0.f, rc = 0.f;
                const float *__restrict__ gphi = phi_all + c * N;
                auto pl = [&](int ty, float *ph, float *la) {
                    float4 p4, l4;
                    if (PL_SMEM) {
                        p4 = *reinterpret_cast<const float4 *>(sphi + ty * kTW + 4 * lane);
                        l4 = *reinterpret_cast<const float4 *>(slam + ty * kTW + 4 * lane);
                    } else {
                        const int y = y0 + ty;
                        p4 = l4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (y < H && x < W) {
                            p4 = __ldg(reinterpret_cast<const float4 *>(gphi + (size_t)y * W + x));
                            l4 = __ldg(reinterpret_cast<const float4 *>(glam + (size_t)y * W + x));
                        }
                    }
                    ph[0] = p4.x; ph[1] = p4.y; ph[2] = p4.z; ph[3] = p4.w;
                    la[0] = l4.x; la[1] = l4.y; la[2] = l4.z; la[3] = l4.w;
                };
                auto sink = [&](int ty, const float *nu, const float *F) {
                    const int y = y0 + ty;
                    if (y >= H || x >= W) return;  // W % 4 == 0: x < W covers all 4 columns
                    float q = 0.f;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) q = fmaf(F[jj], F[jj], q);
                    neumaier_add(rs, rc, q);
                    Store<T>::write4(un + (size_t)y * W + x, nu[0], nu[1], nu[2], nu[3]);
                };
                walk_rows<R, SW, T, EDGE>(s, w * R, lane, eps, tau, wg0, wg1, wg2, pl, sink);
                for (int off = 16; off; off >>= 1) {
                    const float s2 = __shfl_down_sync(0xffffffffu, rs, off);
                    const float c2 = __shfl_down_sync(0xffffffffu, rc, off);
                    neumaier_merge(rs, rc, s2, c2);
                }
                if (lane == 0) slot[stage][w] = make_float2(rs, rc);
                if (border) fence_proxy_async_smem();  // the reflected cells precede the stage's next TMA load
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[stage]);
            }
        }
        k += m;
        __syncthreads();
        if (s_fail) {
            // let every load issued and not waited for land (bounded) before going on
            if (w == NW && lane == 0) {
                for (int q = issued > STAGES ? issued - STAGES : 0; q < issued; ++q)
                    mbar_wait_bounded(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, kWaitLimitCycles);
                atomicCAS(&st->err, 0, DH_ETIMEOUT);
            }
            __syncthreads();
            if (MULTI) {
                if (threadIdx.x == 0) {
                    st->status = DH_ETIMEOUT;
                    st->done = 1;
                }
                return;
            }
        }
        if (!MULTI) break;

        // grid barrier; the last CTA to arrive finishes the iteration
        fence_proxy_async_global();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&st->arrive, 1u);
            s_last = prev == (unsigned)G - 1u;
            s_timeout = 0;
        }
        __syncthreads();
        if (s_last) {
            finish_iteration(d, st);
            if (threadIdx.x == 0) {
                __threadfence();
                st_release_gpu(&st->gen, gen + 1u);
            }
        } else if (threadIdx.x == 0) {
            const long long t0 = clock64();
            while (ld_acquire_gpu(&st->gen) == gen) {
                if (clock64() - t0 > kWaitLimitCycles) {
                    s_timeout = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        ++gen;
        __syncthreads();
        if (s_timeout) {  // another CTA never arrived: give up, report
            if (threadIdx.x == 0) {
                atomicCAS(&st->err, 0, DH_ETIMEOUT);
                st->status = DH_ETIMEOUT;
                st->done = 1;
            }
            return;
        }
        if (__ldcg(&st->done)) return;
    }
    if (!MULTI) arrive_and_finish(d, st, &s_last);
}


typedef void (*SweepFn)(const SolveDesc *);
typedef void (*SweepTmaFn)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, const SolveDesc *);
typedef void (*SweepStreamFn)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, const SolveDesc *, int);

// Element type of the iterates: 0 float, 1 bf16, 2 f16.
// Each returns the matching kernel instance, or nullptr if none is built.
SweepFn sweep_generic_fn(int kind, int R, int NW, bool edge);
SweepTmaFn sweep_tma_fn_kind(int kind, int R, int NW, int stages, int tma, bool edge, int minb, int multi);
SweepTmaFn sweep_tma_f32_a(int R, int NW, int stages, int tma, bool edge, int minb, int multi);
SweepTmaFn sweep_tma_f32_b(int R, int NW, int stages, int tma, bool edge, int minb, int multi);
SweepTmaFn sweep_tma_f32_c(int R, int NW, int stages, int tma, bool edge, int minb, int multi);
SweepTmaFn sweep_tma_16(int kind, int R, int NW, int stages, int tma, bool edge, int minb, int multi);
SweepTmaFn sweep_tb2_fn(int R, int NW, bool edge);
uint32_t tb2_smem_bytes(int R, int NW);
SweepStreamFn sweep_stream_fn(int NW, int NSLOT, bool edge);
SweepTmaFn sweep_ws_fn(int kind, int R, int NW, int stages, int pl, bool edge, int minb, int multi);
SweepTmaFn sweep_tbk_fn(int K, int RO, int NW, bool edge);
uint32_t tbk_smem_bytes(int K, int RO, int NW);

// Instance selector shared by the sweep_inst_*.cu files.
#define DH_STX_T(T, r, nw, st, pls, mb, mu)                                                         \
    if (R == r && NW == nw && stages == st && tma == (pls ? 1 : 2) && minb == mb && multi == mu)     \
        return edge ? (SweepTmaFn)k_sweep_tma<r, nw, st, pls, T, true, mb, mu>                      \
                    : (SweepTmaFn)k_sweep_tma<r, nw, st, pls, T, false, mb, mu>;

}  // namespace dh
