#pragma once
// Gram tile on the CUDA cores (FP64 / FP32), shared by the single-fit and the
// batched Gram kernels.
//
// X is row-major n x p, so the k-th slice X[i, m0 .. m0+63] of both operand
// tiles is a contiguous row segment: every global load is coalesced.  A tile
// (tm, tn) with tm <= tn writes itself and its mirror through a shared-memory
// transpose, so both triangles of S are stored with row-contiguous writes.
// Column centring (Section 2.2) subtracts the column means on the way into
// shared memory.  Block shape: 256 threads.
#include <cuda_runtime.h>

#include "common.cuh"

namespace spmesl {

constexpr int GRAM_BM = 64;      // output tile (BM x BM)
constexpr int GRAM_BK = 16;      // rows of X per stage
constexpr int GRAM_TM = 4;       // outputs per thread per dimension (16 x 16 threads)

template <typename T>
__device__ void gram_tile(const T* __restrict__ X, int n, int p, int ldx, const T* __restrict__ mu,
                          T* __restrict__ S, int lds, T inv_n, int tm, int tn) {
    constexpr int BM = GRAM_BM, BK = GRAM_BK, TM = GRAM_TM;
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
    for (int e = tid; e < BM * BM; e += 256) {
        const int r = e / BM, c = e % BM;
        if (m0 + r < p && n0 + c < p) S[(size_t)(m0 + r) * lds + n0 + c] = Cs[r][c];
    }
    if (tm != tn) {
        for (int e = tid; e < BM * BM; e += 256) {
            const int r = e / BM, c = e % BM;
            if (n0 + r < p && m0 + c < p) S[(size_t)(n0 + r) * lds + m0 + c] = Cs[c][r];
        }
    }
    __syncthreads();     // the staging tile is reused by the next tile of a batched block
}

// Column means of X (for centring), one thread per column, FP64 accumulation.
template <typename T>
__device__ void column_means(const T* __restrict__ X, int n, int p, int ldx, T* __restrict__ mu,
                             int start, int stride) {
    for (int c = start; c < p; c += stride) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += (double)X[(size_t)i * ldx + c];
        mu[c] = (T)(acc / n);
    }
}

// Upper-triangular tile index -> (tm, tn), tm <= tn, for a t x t tile grid
// enumerated row by row: row tm holds t - tm tiles.
__device__ __forceinline__ void upper_tile(int idx, int t, int& tm, int& tn) {
    int row = 0, rem = idx;
    while (rem >= t - row) {
        rem -= t - row;
        ++row;
    }
    tm = row;
    tn = row + rem;
}

}  // namespace spmesl
