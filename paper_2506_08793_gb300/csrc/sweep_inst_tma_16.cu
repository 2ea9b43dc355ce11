// Instances of the TMA sweep kernel for 16-bit iterates (bf16, f16).
#include "sweep_kernels.cuh"

namespace dh {

template <class T>
static SweepTmaFn tma16(int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    DH_STX_T(T, 8, 4, 1, true, 0, false)
    DH_STX_T(T, 6, 4, 1, true, 5, true)
    DH_STX_T(T, 8, 4, 1, true, 0, true)
    return nullptr;
}

SweepTmaFn sweep_tma_16(int kind, int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    return kind == 1 ? tma16<__nv_bfloat16>(R, NW, stages, tma, edge, minb, multi)
                     : tma16<__half>(R, NW, stages, tma, edge, minb, multi);
}

}  // namespace dh
