// Instances of the two-iterations-per-load sweep kernel.
#include "sweep_kernels.cuh"

namespace dh {

SweepTmaFn sweep_tb2_fn(int R, int NW, bool edge) {
#define DH_TB(r, nw, mb) \
    if (R == r && NW == nw) return edge ? (SweepTmaFn)k_sweep_tb2<r, nw, true, mb> : (SweepTmaFn)k_sweep_tb2<r, nw, false, mb>;
    DH_TB(4, 4, 4)
    DH_TB(6, 4, 3)
#undef DH_TB
    return nullptr;
}

uint32_t tb2_smem_bytes(int R, int NW) {
    if (R == 4 && NW == 4) return Tb2Plan<4, 4>::SMEM;
    if (R == 6 && NW == 4) return Tb2Plan<6, 4>::SMEM;
    return 0;
}

}  // namespace dh
