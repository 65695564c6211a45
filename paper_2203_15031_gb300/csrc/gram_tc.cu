// Split-BF16 Gram on the tensor cores (SPMESL_MIXED).  Not built yet: the
// launcher reports "not supported" so the mixed path fails loudly.
#include <cuda_runtime.h>

#include "common.cuh"

namespace spmesl {

size_t gram_tc_ws_bytes(int n, int p) { return align_up((size_t)n * p * 4, 256); }

cudaError_t launch_gram_tc(const float*, int, int, int, int, float*, int, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace spmesl
