// Instances of the depth-K temporally blocked sweep kernel (K = 3, 4).
#include "sweep_kernels.cuh"

namespace dh {

SweepTmaFn sweep_tbk_fn(int K, int RO, int NW, bool edge) {
#define DH_TBK(k, ro, nw, mb)                                                                  \
    if (K == k && RO == ro && NW == nw)                                                        \
        return edge ? (SweepTmaFn)k_sweep_tbk<k, ro, nw, true, mb> : (SweepTmaFn)k_sweep_tbk<k, ro, nw, false, mb>;
    DH_TBK(3, 4, 4, 3)
    DH_TBK(3, 6, 4, 2)
    DH_TBK(4, 4, 4, 2)
#undef DH_TBK
    return nullptr;
}

uint32_t tbk_smem_bytes(int K, int RO, int NW) {
    if (K == 3 && RO == 4 && NW == 4) return TbkPlan<3, 4, 4>::SMEM;
    if (K == 3 && RO == 6 && NW == 4) return TbkPlan<3, 6, 4>::SMEM;
    if (K == 4 && RO == 4 && NW == 4) return TbkPlan<4, 4, 4>::SMEM;
    return 0;
}

}  // namespace dh
