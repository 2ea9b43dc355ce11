// Tensor maps for the kernels outside the single-image sweep (the batched
// sweep's 16-bit iterates, the convolutions' activations): the CUDA driver API's
// cuTensorMapEncodeTiled, looked up once at run time, with no interleave,
// 256-byte L2 promotion, zero fill outside the tensor, and no swizzle unless
// asked for.
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace dh {

int encode_tiled_sw(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                    const cuuint64_t *strides, const cuuint32_t *box, CUtensorMapSwizzle swizzle) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (rank < 1 || rank > 5) return DH_EINVAL;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            const cudaError_t e =
                cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return DH_ECUDA;
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
    }
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode(m, dt, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DH_OK : DH_EINVAL;
}

int encode_tiled(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const cuuint64_t *dims,
                 const cuuint64_t *strides, const cuuint32_t *box) {
    return encode_tiled_sw(m, dt, rank, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

}  // namespace dh
