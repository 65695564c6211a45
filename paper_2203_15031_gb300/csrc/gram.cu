// Gram matrix S = X'X / n on the CUDA cores (FP64 and FP32 paths); the tile
// itself is in gram_device.cuh.  Only the t(t+1)/2 upper-triangular tiles are
// launched; each writes its mirror too.
#include <cuda_runtime.h>

#include <algorithm>

#include "gram_device.cuh"

namespace spmesl {

namespace {

template <typename T>
__global__ void column_mean_kernel(const T* __restrict__ X, int n, int p, int ldx, T* mu) {
    column_means<T>(X, n, p, ldx, mu, blockIdx.x * blockDim.x + threadIdx.x,
                    gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(256) gram_simt_kernel(const T* __restrict__ X, int n, int p,
                                                       int ldx, const T* __restrict__ mu,
                                                       T* __restrict__ S, int lds, T inv_n) {
    const int t = (p + GRAM_BM - 1) / GRAM_BM;
    int tm, tn;
    upper_tile(blockIdx.x, t, tm, tn);
    gram_tile<T>(X, n, p, ldx, mu, S, lds, inv_n, tm, tn);
}

template <typename T>
cudaError_t run_gram_simt(const T* X, int n, int p, int ldx, int center, T* S, int lds, void* ws,
                          cudaStream_t st) {
    T* mu = nullptr;
    if (center) {
        mu = reinterpret_cast<T*>(ws);
        column_mean_kernel<T><<<(p + 255) / 256, 256, 0, st>>>(X, n, p, ldx, mu);
    }
    const int t = (p + GRAM_BM - 1) / GRAM_BM;
    gram_simt_kernel<T><<<t * (t + 1) / 2, 256, 0, st>>>(X, n, p, ldx, mu, S, lds,
                                                        (T)(1.0 / (double)n));
    return cudaGetLastError();
}

}  // namespace

// Defined in gram_tc.cu (split-BF16 tensor-core path).
size_t gram_tc_ws_bytes(int n, int p);
cudaError_t launch_gram_tc(const float* X, int n, int p, int ldx, int center, float* S, int lds,
                           void* ws, cudaStream_t st);

size_t gram_ws_bytes(int n, int p, int precision) {
    if (precision == SPMESL_MIXED) return gram_tc_ws_bytes(n, p);
    return align_up((size_t)p * (size_t)elem_size(precision), 256);
}

cudaError_t launch_gram(const void* X, int n, int p, int ldx, int precision, int center, void* S,
                        int lds, void* ws, cudaStream_t st) {
    if (precision == SPMESL_FP64)
        return run_gram_simt<double>(static_cast<const double*>(X), n, p, ldx, center,
                                     static_cast<double*>(S), lds, ws, st);
    if (precision == SPMESL_FP32)
        return run_gram_simt<float>(static_cast<const float*>(X), n, p, ldx, center,
                                    static_cast<float*>(S), lds, ws, st);
    return launch_gram_tc(static_cast<const float*>(X), n, p, ldx, center, static_cast<float*>(S),
                          lds, ws, st);
}

}  // namespace spmesl
