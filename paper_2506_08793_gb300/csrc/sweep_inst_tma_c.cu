// Instances of the TMA sweep kernel, float iterates (3 of 3).
#include "sweep_kernels.cuh"

namespace dh {

SweepTmaFn sweep_tma_f32_c(int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    DH_STX_T(float, 4, 8, 1, true, 0, false)
    DH_STX_T(float, 8, 4, 1, false, 0, false)
    DH_STX_T(float, 8, 4, 2, false, 0, false)
    DH_STX_T(float, 4, 8, 1, false, 0, false)
    DH_STX_T(float, 4, 8, 2, false, 0, false)
    DH_STX_T(float, 16, 4, 1, false, 0, false)
    DH_STX_T(float, 8, 8, 1, false, 0, false)
    DH_STX_T(float, 16, 2, 2, false, 0, false)
    return nullptr;
}

}  // namespace dh
