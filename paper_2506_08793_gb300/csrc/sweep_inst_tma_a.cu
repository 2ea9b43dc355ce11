// Instances of the TMA sweep kernel, float iterates (1 of 3).
#include "sweep_kernels.cuh"

namespace dh {

SweepTmaFn sweep_tma_f32_a(int R, int NW, int stages, int tma, bool edge, int minb, int multi) {
    DH_STX_T(float, 8, 4, 1, true, 0, false)
    DH_STX_T(float, 6, 4, 1, true, 5, true)
    DH_STX_T(float, 8, 4, 1, true, 0, true)
    DH_STX_T(float, 4, 4, 1, true, 6, true)
    DH_STX_T(float, 6, 4, 1, true, 0, true)
    DH_STX_T(float, 4, 4, 2, true, 0, true)
    DH_STX_T(float, 4, 4, 2, true, 0, false)
    DH_STX_T(float, 6, 4, 1, true, 0, false)
    return nullptr;
}

}  // namespace dh
