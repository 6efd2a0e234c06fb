// Tensor-core Gram S = X^T X / n (tcgen05 + TMA), BF16 split and TF32 modes.
#include "internal.cuh"

namespace hpc {

size_t gram_tc_scratch_bytes(int, int64_t, int64_t, int) { return 0; }

cudaError_t gram_tc(const void*, int, int64_t, int64_t, float*, int64_t, int, void*, size_t, cudaStream_t, int*) {
    return cudaErrorNotSupported;
}

}  // namespace hpc
