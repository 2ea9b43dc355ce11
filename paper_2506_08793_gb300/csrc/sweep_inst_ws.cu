// Instances of the warp-specialised TMA sweep kernel (one producer warp, NW
// compute warps), float iterates, multi-iteration cooperative launches.
#include "sweep_kernels.cuh"

namespace dh {

#define DH_WSX(T, r, nw, st, pls, mb)                                                                   \
    if (R == r && NW == nw && stages == st && pl == pls && minb == mb)                                  \
        return edge ? (SweepTmaFn)k_sweep_ws<r, nw, st, pls, T, true, mb, true>                         \
                    : (SweepTmaFn)k_sweep_ws<r, nw, st, pls, T, false, mb, true>;

SweepTmaFn sweep_ws_fn(int kind, int R, int NW, int stages, int pl, bool edge, int minb, int multi) {
    if (kind != 0 || !multi) return nullptr;
    DH_WSX(float, 4, 8, 2, true, 2)
    DH_WSX(float, 6, 4, 2, true, 2)
    DH_WSX(float, 8, 4, 2, true, 2)
    return nullptr;
}

}  // namespace dh
