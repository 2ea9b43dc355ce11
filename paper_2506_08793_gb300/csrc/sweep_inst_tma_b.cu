// Instances of the TMA sweep kernel, float iterates (2 of 3).
#include "sweep_kernels.cuh"

namespace dh {

SweepTmaFn sweep_tma_f32_b(int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    DH_STX_T(float, 4, 4, 1, true, 0, false)
    DH_STX_T(float, 16, 2, 1, true, 0, false)
    DH_STX_T(float, 12, 2, 1, true, 0, false)
    DH_STX_T(float, 8, 4, 1, true, 5, false)
    DH_STX_T(float, 6, 4, 1, true, 5, false)
    DH_STX_T(float, 4, 4, 1, true, 6, false)
    DH_STX_T(float, 8, 4, 2, true, 0, false)
    DH_STX_T(float, 4, 8, 2, true, 0, false)
    return nullptr;
}

}  // namespace dh
