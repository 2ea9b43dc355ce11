// C ABI entry points (include/dehaze.h): validation, workspace checks and the
// order in which the per-step kernels are queued.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace dh {

int launch_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out,
                        cudaStream_t s);
int launch_transmission(const float *I, int H, int W, const dh_params *p, const float *A, float *td,
                        float *t, float *lam, float *phi, float *u0, float2 *phin_part, void *scratch,
                        cudaStream_t s);
int launch_phin(const float *phi, int H, int W, float2 *part, SolveState *st, cudaStream_t s);
int launch_phin_final(const float2 *part, int H, int W, SolveState *st, cudaStream_t s);
int launch_select_A(const float *I, const float *dc, int H, int W, int permille, float *A,
                    long long *index_out, char *ws, const WsLayout &L, cudaStream_t s);
int run_solve(float *u_caller, const float *phi, const float *lam, int H, int W, const dh_params *p,
              float *rho_hist, char *ws, const WsLayout &L, cudaStream_t s, float *J,
              cudaEvent_t loop_begin, cudaEvent_t loop_end, int *launches);
int read_solve_state(const char *ws, const WsLayout &L, SolveState *out);
int sweep_variant_count();
bool sweep_variant_usable(int v, int W, bool aligned);
void tune_set(int dev, int H, int W, int storage, int variant);
int tune_get(int dev, int H, int W, int storage);

size_t semi_workspace_bytes(int H, int W);
int run_semi_implicit(float *u, float *u_lo, const float *Phi, const float *lam, int H, int W, const dh_params *p,
                      float step, int cg_iters, float *rho_hist, float *J, void *workspace, cudaStream_t s);
int read_semi_implicit(const void *workspace, cudaStream_t s, int *n_final, int *status, float rho[3]);

int cuda_fail(cudaError_t) {
    cudaGetLastError();  // clear a non-sticky error so the next call starts clean
    return DH_ECUDA;
}

static bool params_ok(const dh_params *p) {
    if (!p) return false;
    if (p->patch < 1 || p->patch > 31 || (p->patch & 1) == 0) return false;
    if (p->topk_permille < 1 || p->topk_permille > 1000) return false;
    if (!(p->omega >= 0.f && p->omega <= 1.f)) return false;
    if (!(p->t0 > 0.f && p->t0 <= 1.f)) return false;
    if (!(p->lambda0 >= 0.f) || !std::isfinite(p->lambda0)) return false;
    if (!std::isfinite(p->beta)) return false;
    if (!(p->eps > 0.f) || !std::isfinite(p->eps)) return false;
    if (!(p->sigma > 0.f) || !std::isfinite(p->sigma)) return false;
    if (p->radius != 2) return false;
    if (!(p->tau > 0.f) || !std::isfinite(p->tau)) return false;
    if (!(p->tol >= 0.f)) return false;
    if (p->max_iter < 0 || p->max_iter > 10000000) return false;
    if (p->tb_depth < 0 || p->tb_depth > 4) return false;
    if (p->storage < DH_STORE_F32 || p->storage > DH_STORE_F16_F32) return false;
    if (p->variant & ~(DH_VAR_NO_ADAPTIVE | DH_VAR_NO_EDGE | DH_VAR_NO_NONLOCAL)) return false;
    if (p->sweep_variant < 0 || p->sweep_variant >= sweep_variant_count()) return false;
    if (p->boundary != DH_BOUNDARY_REFLECT && p->boundary != DH_BOUNDARY_ZERO) return false;
    if (p->dc_scales != 1 && !(p->dc_scales == 3 && p->patch <= 15)) return false;
    if (p->gf_radius < 0 || p->gf_radius > 24) return false;
    if (p->gf_radius > 0 && (!(p->gf_eps > 0.f) || !std::isfinite(p->gf_eps))) return false;
    return true;
}

static WsLayout layout_for(int H, int W, const dh_params *p) {
    const int depth = sweep_depth(p);
    return ws_layout(H, W, depth, sweep_tile_h(depth), refine_bytes(H, W, p));
}

static int ws_ok(const void *ws, size_t bytes, const WsLayout &L) {
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || bytes < L.total) return DH_EWORKSPACE;
    return DH_OK;
}

// CUDA events around a whole call and around its fixed-point loop, recorded
// only when the caller asked for a report.
struct Timer {
    cudaEvent_t a = nullptr, b = nullptr, la = nullptr, lb = nullptr;
    bool on = false, loop = false;
    void start(cudaStream_t s, bool want) {
        if (!want) return;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
            cudaEventCreate(&la) != cudaSuccess || cudaEventCreate(&lb) != cudaSuccess)
            return;
        on = cudaEventRecord(a, s) == cudaSuccess;
    }
    cudaEvent_t loop_begin() {
        loop = on;
        return on ? la : nullptr;
    }
    cudaEvent_t loop_end() const { return on ? lb : nullptr; }
    void stop(cudaStream_t s, float *ms, float *ms_loop) {
        *ms = 0.f;
        *ms_loop = 0.f;
        if (on && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess) {
            cudaEventElapsedTime(ms, a, b);
            if (loop) cudaEventElapsedTime(ms_loop, la, lb);
        }
        cudaGetLastError();  // timing is best effort; leave no error behind
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (la) cudaEventDestroy(la);
        if (lb) cudaEventDestroy(lb);
    }
};

}  // namespace dh

using namespace dh;

extern "C" {

int dh_version(void) { return DH_VERSION; }

int dh_params_default(dh_params *p, int preset) {
    if (!p || (preset != DH_PRESET_PAPER && preset != DH_PRESET_STABLE)) return DH_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->patch = 15;
    p->topk_permille = 1;
    p->omega = 0.95f;
    p->t0 = 0.1f;
    p->lambda0 = 0.5f;
    p->beta = 3.0f;
    p->eps = preset == DH_PRESET_PAPER ? 1e-3f : 1.0f;
    p->sigma = 2.0f;
    p->radius = 2;
    p->tau = 0.2f;
    p->tol = 1e-4f;
    p->max_iter = 5000;
    p->tb_depth = 0;
    p->storage = DH_STORE_F32;
    p->variant = 0;
    p->use_graph = 1;
    p->sweep_variant = 0;
    p->boundary = DH_BOUNDARY_REFLECT;
    p->dc_scales = 1;
    p->gf_radius = 0;
    p->gf_eps = 1e-3f;
    return DH_OK;
}

const char *dh_strerror(int status) {
    switch (status) {
        case DH_OK: return "ok";
        case DH_WDEGENERATE: return "warning: a component of the atmospheric light was <= 0 and was clamped to 1e-6";
        case DH_WNOCONV: return "warning: max_iter reached with the residual above tol";
        case DH_EINVAL: return "invalid shape, pointer, alignment or parameter";
        case DH_ENONFINITE: return "non-finite residual; iteration stopped";
        case DH_EWORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case DH_ECUDA: return "CUDA runtime error (no usable GPU, or a launch failed)";
        case DH_ETIMEOUT: return "a bounded device-side wait ran out";
        default: return "unknown status";
    }
}

size_t dh_workspace_bytes(int H, int W, const dh_params *p) {
    dh_params d;
    if (!p) {
        dh_params_default(&d, DH_PRESET_PAPER);
        p = &d;
    }
    if (!shape_ok(H, W) || !params_ok(p)) return 0;
    return layout_for(H, W, p).total;
}

int dh_dark_channel(const float *I, int H, int W, int patch, const float *A, float *out, void *stream) {
    if (!I || !out || !shape_ok(H, W) || patch < 1 || patch > 31 || (patch & 1) == 0) return DH_EINVAL;
    return launch_dark_channel(I, H, W, patch, A, out, (cudaStream_t)stream);
}

int dh_atmospheric_light(const float *I, const float *dc, int H, int W, int topk_permille, float *A_out,
                         long long *index_out, void *workspace, size_t workspace_bytes, void *stream,
                         dh_report *report) {
    if (!I || !dc || !A_out || !shape_ok(H, W) || topk_permille < 1 || topk_permille > 1000)
        return DH_EINVAL;
    dh_params d;
    dh_params_default(&d, DH_PRESET_PAPER);
    const WsLayout L = layout_for(H, W, &d);
    int rc = ws_ok(workspace, workspace_bytes, L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    Timer tm;
    tm.start(s, report != nullptr);
    rc = launch_select_A(I, dc, H, W, topk_permille, A_out, index_out, (char *)workspace, L, s);
    if (rc || !report) return rc;
    std::memset(report, 0, sizeof(*report));
    tm.stop(s, &report->ms, &report->ms_loop);
    report->launches = 13;
    SelectState sel;
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    DH_CUDA_TRY(cudaMemcpy(&sel, (char *)workspace + L.sel, sizeof(sel), cudaMemcpyDeviceToHost));
    DH_CUDA_TRY(cudaMemcpy(report->A, A_out, 3 * sizeof(float), cudaMemcpyDeviceToHost));
    report->a_index = sel.best;
    report->status = sel.clamped ? DH_WDEGENERATE : DH_OK;
    return report->status;
}

int dh_transmission(const float *I, const float *A, int H, int W, const dh_params *p, float *td, float *t,
                    float *lam, float *Phi, void *stream) {
    if (!I || !A || !shape_ok(H, W) || !params_ok(p)) return DH_EINVAL;
    return launch_transmission(I, H, W, p, A, td, t, lam, Phi, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

int dh_transmission_ws(const float *I, const float *A, int H, int W, const dh_params *p, float *td, float *t,
                       float *lam, float *Phi, void *workspace, size_t workspace_bytes, void *stream) {
    if (!I || !A || !t || !lam || !Phi || !shape_ok(H, W) || !params_ok(p)) return DH_EINVAL;
    const WsLayout L = layout_for(H, W, p);
    const int rc = ws_ok(workspace, workspace_bytes, L);
    if (rc) return rc;
    return launch_transmission(I, H, W, p, A, td, t, lam, Phi, nullptr, nullptr, (char *)workspace + L.refine,
                               (cudaStream_t)stream);
}

static void fill_solve_report(dh_report *r, const SolveState &st, int launches, bool graph) {
    r->status = st.status;
    r->n_iter = st.n_final;
    for (int c = 0; c < 3; ++c) r->rho[c] = st.rho[c];
    r->launches = launches + (graph ? (int)st.launches : 0);  // sweep launches counted on the device
}

int dh_fixed_point(float *u, const float *Phi, const float *lam, int H, int W, const dh_params *p,
                   float *rho_hist, void *workspace, size_t workspace_bytes, void *stream,
                   dh_report *report) {
    if (!u || !Phi || !lam || !shape_ok(H, W) || !params_ok(p)) return DH_EINVAL;
    const WsLayout L = layout_for(H, W, p);
    int rc = ws_ok(workspace, workspace_bytes, L);
    if (rc) return rc;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    Timer tm;
    tm.start(s, report != nullptr);
    rc = launch_phin(Phi, H, W, (float2 *)(ws + L.phin_part), (SolveState *)(ws + L.state), s);
    if (rc) return rc;
    int launches = 2;  // ||Phi||^2 partials and final
    rc = run_solve(u, Phi, lam, H, W, p, rho_hist, ws, L, s, nullptr, tm.loop_begin(), tm.loop_end(),
                   &launches);
    if (rc || !report) return rc;
    std::memset(report, 0, sizeof(*report));
    tm.stop(s, &report->ms, &report->ms_loop);
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    SolveState st;
    rc = read_solve_state(ws, L, &st);
    if (rc) return rc;
    fill_solve_report(report, st, launches, p->use_graph != 0);
    report->a_index = -1;
    return report->status;
}

int dh_dehaze(const float *I, int H, int W, const dh_params *p, const float *u0, float *J, float *u,
              float *t, float *A, void *workspace, size_t workspace_bytes, void *stream,
              dh_report *report) {
    if (!I || !J || !u || !t || !A || !shape_ok(H, W) || !params_ok(p)) return DH_EINVAL;
    const WsLayout L = layout_for(H, W, p);
    int rc = ws_ok(workspace, workspace_bytes, L);
    if (rc) return rc;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    Timer tm;
    tm.start(s, report != nullptr);
    float *dc = (float *)(ws + L.dc);
    float *lam = (float *)(ws + L.lam);
    float *phi = (float *)(ws + L.phi);
    // Sec. II-D: dark channel of I, then A (DCP rule), then t, lambda, Phi
    rc = launch_dark_channel(I, H, W, p->patch, nullptr, dc, s);
    if (rc) return rc;
    rc = launch_select_A(I, dc, H, W, p->topk_permille, A, nullptr, ws, L, s);
    if (rc) return rc;
    rc = launch_transmission(I, H, W, p, A, nullptr, t, lam, phi, u0 ? nullptr : u,
                             (float2 *)(ws + L.phin_part), ws + L.refine, s);
    if (rc) return rc;
    if (u0) DH_CUDA_TRY(cudaMemcpyAsync(u, u0, (size_t)3 * H * W * sizeof(float), cudaMemcpyDeviceToDevice, s));
    rc = launch_phin_final((const float2 *)(ws + L.phin_part), H, W, (SolveState *)(ws + L.state), s);
    if (rc) return rc;
    // App. A-A fixed point, then J = clamp(u, 0, 1)
    int launches = 1 + 13 + 1 + 1;  // dark channel, A selection, transmission, ||Phi||^2
    rc = run_solve(u, phi, lam, H, W, p, nullptr, ws, L, s, J, tm.loop_begin(), tm.loop_end(), &launches);
    if (rc || !report) return rc;
    std::memset(report, 0, sizeof(*report));
    tm.stop(s, &report->ms, &report->ms_loop);
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    SolveState st;
    SelectState sel;
    rc = read_solve_state(ws, L, &st);
    if (rc) return rc;
    DH_CUDA_TRY(cudaMemcpy(&sel, ws + L.sel, sizeof(sel), cudaMemcpyDeviceToHost));
    DH_CUDA_TRY(cudaMemcpy(report->A, A, 3 * sizeof(float), cudaMemcpyDeviceToHost));
    fill_solve_report(report, st, launches, p->use_graph != 0);
    report->a_index = sel.best;
    if (report->status == DH_OK && sel.clamped) report->status = DH_WDEGENERATE;
    return report->status;
}

int dh_sweep_variants(void) { return sweep_variant_count(); }

int dh_tune_set(int H, int W, int storage, int variant) {
    if (!shape_ok(H, W) || variant < 0 || variant >= sweep_variant_count() || storage < 0 || storage > DH_STORE_F16_F32)
        return DH_EINVAL;
    int dev = 0;
    DH_CUDA_TRY(cudaGetDevice(&dev));
    tune_set(dev, H, W, storage, variant);
    return DH_OK;
}

int dh_tune_get(int H, int W, int storage) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return tune_get(dev, H, W, storage);
}

int dh_tune(const float *Phi, const float *lam, float *u_scratch, int H, int W, const dh_params *p, int iters,
            void *workspace, size_t workspace_bytes, void *stream, dh_tune_result *out) {
    if (!Phi || !lam || !u_scratch || !shape_ok(H, W) || !params_ok(p) || iters < 1 || iters > 100000 ||
        p->storage != DH_STORE_F32)
        return DH_EINVAL;
    const WsLayout L = layout_for(H, W, p);
    int rc = ws_ok(workspace, workspace_bytes, L);
    if (rc) return rc;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const bool aligned = a16(Phi) && a16(lam) && a16(u_scratch) && a16(ws + L.ub);
    dh_tune_result res;
    std::memset(&res, 0, sizeof(res));
    res.best = 0;
    float best = 3.4e38f;
    cudaEvent_t a, b;
    DH_CUDA_TRY(cudaEventCreate(&a));
    DH_CUDA_TRY(cudaEventCreate(&b));
    const size_t bytes = (size_t)3 * H * W * sizeof(float);
    rc = launch_phin(Phi, H, W, (float2 *)(ws + L.phin_part), (SolveState *)(ws + L.state), s);
    int vs[64], nv = 0;
    for (int v = 1; v < sweep_variant_count() && nv < 64; ++v)
        if (sweep_variant_usable(v, W, aligned)) vs[nv++] = v;
    float us_min[64];
    // two rounds over all variants, the faster time of each kept: a clock or
    // thermal drift during one round does not decide the winner
    for (int round = 0; round < 2 && !rc; ++round) {
        for (int i = 0; i < nv && !rc; ++i) {
            dh_params q = *p;
            q.sweep_variant = vs[i];
            q.tol = 0.f;
            q.max_iter = iters;
            q.use_graph = 1;
            float ms = 0.f;
            const int reps = round == 0 ? 2 : 1;  // the first run builds and warms the graph
            for (int rep = 0; rep < reps && !rc; ++rep) {
                if (cudaMemcpyAsync(u_scratch, Phi, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = DH_ECUDA; break; }
                rc = run_solve(u_scratch, Phi, lam, H, W, &q, nullptr, ws, L, s, nullptr, a, b, nullptr);
                if (!rc && rep == reps - 1) {
                    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
                        rc = DH_ECUDA;
                }
            }
            if (rc) break;
            const float us = 1e3f * ms / (iters + 1);
            us_min[i] = round == 0 || us < us_min[i] ? us : us_min[i];
        }
    }
    if (!rc) {
        for (int i = 0; i < nv; ++i) {
            res.variant[i] = vs[i];
            res.us_per_iter[i] = us_min[i];
            if (us_min[i] < best) {
                best = us_min[i];
                res.best = vs[i];
            }
        }
        res.count = nv;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc == DH_ECUDA ? cuda_fail(cudaGetLastError()) : rc;
    int dev = 0;
    DH_CUDA_TRY(cudaGetDevice(&dev));
    if (res.best > 0) tune_set(dev, H, W, DH_STORE_F32, res.best);
    if (out) *out = res;
    return DH_OK;
}

size_t dh_semi_implicit_workspace_bytes(int H, int W) {
    if (!shape_ok(H, W)) return 0;
    return semi_workspace_bytes(H, W);
}

int dh_semi_implicit(float *u, float *u_lo, const float *Phi, const float *lam, int H, int W, const dh_params *p,
                     float step, int cg_iters, float *rho_hist, float *J, void *workspace, size_t workspace_bytes,
                     void *stream, dh_report *report) {
    if (!u || !Phi || !lam || !shape_ok(H, W) || !params_ok(p)) return DH_EINVAL;
    if (!(step > 0.f) || !std::isfinite(step) || cg_iters < 1 || cg_iters > 10000) return DH_EINVAL;
    if (p->storage != DH_STORE_F32) return DH_EINVAL;
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < semi_workspace_bytes(H, W))
        return DH_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Timer tm;
    tm.start(s, report != nullptr);
    cudaEvent_t lb = tm.loop_begin();
    if (lb) DH_CUDA_TRY(cudaEventRecord(lb, s));
    int rc = run_semi_implicit(u, u_lo, Phi, lam, H, W, p, step, cg_iters, rho_hist, J, workspace, s);
    if (rc || !report) return rc;
    if (tm.loop_end()) DH_CUDA_TRY(cudaEventRecord(tm.loop_end(), s));
    std::memset(report, 0, sizeof(*report));
    tm.stop(s, &report->ms, &report->ms_loop);
    int n_final = 0, status = 0;
    float rho[3] = {0.f, 0.f, 0.f};
    rc = read_semi_implicit(workspace, s, &n_final, &status, rho);
    if (rc) return rc;
    report->status = status;
    report->n_iter = n_final;
    for (int c = 0; c < 3; ++c) report->rho[c] = rho[c];
    report->a_index = -1;
    report->launches = J ? 3 : 2;  // state reset + the cooperative solve (+ J)
    return report->status;
}

}  // extern "C"
