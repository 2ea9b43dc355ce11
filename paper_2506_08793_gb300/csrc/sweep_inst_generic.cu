// Instances of the generic gather sweep kernel (any width or alignment).
#include "sweep_kernels.cuh"

namespace dh {

template <class T>
static SweepFn generic_fn(int R, int NW, bool edge) {
#define DH_SW(r, nw) \
    if (R == r && NW == nw) return edge ? k_sweep<r, nw, T, true> : k_sweep<r, nw, T, false>;
    DH_SW(8, 4)
    if (sizeof(T) == 4) {
        DH_SW(16, 4)
        DH_SW(8, 8)
    }
#undef DH_SW
    return nullptr;
}

SweepFn sweep_generic_fn(int kind, int R, int NW, bool edge) {
    if (kind == 0) return generic_fn<float>(R, NW, edge);
    if (kind == 1) return generic_fn<__nv_bfloat16>(R, NW, edge);
    return generic_fn<__half>(R, NW, edge);
}

SweepTmaFn sweep_tma_fn_kind(int kind, int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    if (kind != 0) return sweep_tma_16(kind, R, NW, stages, tma, edge, minb, multi);
    SweepTmaFn f = sweep_tma_f32_a(R, NW, stages, tma, edge, minb, multi);
    if (!f) f = sweep_tma_f32_b(R, NW, stages, tma, edge, minb, multi);
    if (!f) f = sweep_tma_f32_c(R, NW, stages, tma, edge, minb, multi);
    return f;
}

}  // namespace dh
