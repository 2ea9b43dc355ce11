// Atmospheric-light selection that allocates nothing and needs no workspace.
//
// Some callers cannot call cudaMalloc at all: a plug-in inside a host
// application that owns every device buffer and hands the plug-in only its
// inputs and outputs, or a real-time pipeline whose memory is fixed at start
// and whose frame loop may not allocate (allocation can block the device and
// can fail in the middle of a frame).  This entry point serves them: its
// scratch is a file-scope device array of fixed size, so the caller passes
// only the image, its dark channel and the outputs.
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace dh {

int launch_select_A(const float *I, const float *dc, int H, int W, int permille, float *A,
                    long long *index_out, char *ws, const WsLayout &L, cudaStream_t s);

// Selection state, the 256-bin radix histogram and kSelBlocks 16-byte
// per-block records.  Its size does not depend on the image.
constexpr size_t kNoAllocScratchBytes = 32768;
static __device__ __align__(256) unsigned char g_select_scratch[kNoAllocScratchBytes];

constexpr size_t kNaHist = align_up(sizeof(SelectState));
constexpr size_t kNaBlk = kNaHist + align_up(256 * sizeof(unsigned));
static_assert(kNaBlk + (size_t)kSelBlocks * 16 <= kNoAllocScratchBytes, "scratch too small");

}  // namespace dh

using namespace dh;

extern "C" int dh_atmospheric_light_noalloc(const float *I, const float *dc, int H, int W,
                                            int topk_permille, float *A_out, long long *index_out,
                                            void *stream) {
    if (!I || !dc || !A_out || !shape_ok(H, W) || topk_permille < 1 || topk_permille > 1000)
        return DH_EINVAL;
    // The array's device address, looked up on every call for the current
    // device and context (the host-side name is only a stand-in and must not
    // reach a kernel; an address kept from an earlier context would go stale
    // after a device reset).  The lookup allocates nothing.
    char *scratch = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&scratch, g_select_scratch);
    if (e != cudaSuccess || !scratch) return cuda_fail(e);
    WsLayout L = {};
    L.sel = 0;
    L.hist = kNaHist;
    L.blk = kNaBlk;
    // The selection clears its state and histogram itself before use, and
    // writes every per-block record before reading it.
    return launch_select_A(I, dc, H, W, topk_permille, A_out, index_out, scratch, L,
                           (cudaStream_t)stream);
}

// ---------------------------------------------------------------- bounded-wait self test
// A wait on an mbarrier that nothing ever completes, given up after
// limit_cycles: the same bounded wait every TMA / tensor-core stage uses.
namespace dh {
static __device__ int g_selftest_result;

__global__ void k_selftest_wait(int *out, long long limit_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected, none will come
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_cycles);
    if (threadIdx.x == 0) *out = ok ? DH_OK : DH_ETIMEOUT;
}
}  // namespace dh

extern "C" int dh_selftest_bounded_wait(long long limit_cycles, void *stream) {
    using namespace dh;
    if (limit_cycles < 1 || limit_cycles > 4000000000LL) return DH_EINVAL;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int *d = nullptr;
    DH_CUDA_TRY(cudaGetSymbolAddress((void **)&d, g_selftest_result));
    cudaStream_t s = (cudaStream_t)stream;
    k_selftest_wait<<<1, 32, 0, s>>>(d, limit_cycles);
    DH_CUDA_TRY(cudaGetLastError());
    int h = DH_ECUDA;
    DH_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    DH_CUDA_TRY(cudaStreamSynchronize(s));
    return h;
}
