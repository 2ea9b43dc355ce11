// Instances of the per-warp row-stream sweep kernel.
#include "sweep_kernels.cuh"

namespace dh {

SweepStreamFn sweep_stream_fn(int NW, int NSLOT, bool edge) {
#define DH_SS(nw, ns) \
    if (NW == nw && NSLOT == ns) return edge ? k_sweep_stream<nw, ns, true> : k_sweep_stream<nw, ns, false>;
    DH_SS(4, 8)
    DH_SS(8, 8)
    DH_SS(4, 16)
    DH_SS(2, 8)
    DH_SS(8, 4)
#undef DH_SS
    return nullptr;
}

}  // namespace dh
