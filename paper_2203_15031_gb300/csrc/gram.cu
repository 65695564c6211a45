// Gram matrix S = X'X / n on the CUDA cores (FP64 and FP32 paths).
//
// X is row-major n x p, so the k-th slice X[i, m0 .. m0+63] of both operand
// tiles is a contiguous row segment: every global load below is coalesced.
// Only tiles with tile_m <= tile_n are computed; each writes its tile and the
// mirrored tile through a shared-memory transpose, so both triangles of S are
// stored with row-contiguous writes.  Column centring (Section 2.2) subtracts
// the column means on the way into shared memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace spmesl {

namespace {

constexpr int BM = 64;       // output tile (BM x BM)
constexpr int BK = 16;       // rows of X per stage
constexpr int TM = 4;        // outputs per thread per dimension (16 x 16 threads)

template <typename T>
__global__ void column_mean_kernel(const T* __restrict__ X, int n, int p, int ldx, T* mu) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < p; c += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += (double)X[(size_t)i * ldx + c];
        mu[c] = (T)(acc / n);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gram_simt_kernel(const T* __restrict__ X, int n, int p,
                                                       int ldx, const T* __restrict__ mu,
                                                       T* __restrict__ S, int lds, T inv_n) {
    const int tm = blockIdx.y, tn = blockIdx.x;
    if (tm > tn) return;                      // symmetric: upper tiles only
    // operand tiles during the K loop, output staging tile afterwards
    constexpr size_t kOpBytes = 2 * sizeof(T) * BK * BM;
    constexpr size_t kOutBytes = sizeof(T) * BM * (BM + 1);
    __shared__ __align__(16) unsigned char raw[kOpBytes > kOutBytes ? kOpBytes : kOutBytes];
    T (*As)[BM] = reinterpret_cast<T (*)[BM]>(raw);
    T (*Bs)[BM] = reinterpret_cast<T (*)[BM]>(raw + sizeof(T) * BK * BM);
    T (*Cs)[BM + 1] = reinterpret_cast<T (*)[BM + 1]>(raw);
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = tm * BM, n0 = tn * BM;

    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);

    for (int i0 = 0; i0 < n; i0 += BK) {
        // 16 x 64 elements per operand tile, 256 threads: 4 each
#pragma unroll
        for (int q = 0; q < (BK * BM) / 256; ++q) {
            const int e = tid + q * 256;
            const int kk = e / BM, mm = e % BM;
            const int i = i0 + kk;
            T va = T(0), vb = T(0);
            if (i < n) {
                const int ca = m0 + mm, cb = n0 + mm;
                if (ca < p) va = X[(size_t)i * ldx + ca] - (mu ? mu[ca] : T(0));
                if (cb < p) vb = X[(size_t)i * ldx + cb] - (mu ? mu[cb] : T(0));
            }
            As[kk][mm] = va;
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TM];
#pragma unroll
            for (int t = 0; t < TM; ++t) {
                a[t] = As[kk][ty * TM + t];
                b[t] = Bs[kk][tx * TM + t];
            }
#pragma unroll
            for (int u = 0; u < TM; ++u)
#pragma unroll
                for (int v = 0; v < TM; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TM; ++v) Cs[ty * TM + u][tx * TM + v] = acc[u][v] * inv_n;
    __syncthreads();
    // tile (m0, n0): row-contiguous
    for (int e = tid; e < BM * BM; e += 256) {
        const int r = e / BM, c = e % BM;
        if (m0 + r < p && n0 + c < p) S[(size_t)(m0 + r) * lds + n0 + c] = Cs[r][c];
    }
    if (tm != tn) {
        // mirrored tile (n0, m0) = transpose
        for (int e = tid; e < BM * BM; e += 256) {
            const int r = e / BM, c = e % BM;
            if (n0 + r < p && m0 + c < p) S[(size_t)(n0 + r) * lds + m0 + c] = Cs[c][r];
        }
    }
}

template <typename T>
cudaError_t run_gram_simt(const T* X, int n, int p, int ldx, int center, T* S, int lds, void* ws,
                          cudaStream_t st) {
    T* mu = nullptr;
    if (center) {
        mu = reinterpret_cast<T*>(ws);
        column_mean_kernel<T><<<(p + 255) / 256, 256, 0, st>>>(X, n, p, ldx, mu);
    }
    const int tiles = (p + BM - 1) / BM;
    gram_simt_kernel<T><<<dim3(tiles, tiles), 256, 0, st>>>(X, n, p, ldx, mu, S, lds,
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
