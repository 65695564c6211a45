#pragma once
// Split-BF16 Gram on the tensor cores: the pieces shared by the single-fit
// path (spmesl_gram with SPMESL_MIXED) and the batched one (spmesl_batch_*).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace spmesl {

constexpr int TC_BM = 128;            // accumulator rows = TMEM lanes
constexpr int TC_NPAD = 64;           // sample dimension padded to the K block
static_assert(TC_NPAD % 64 == 0, "split_transpose_tile64 takes 64 samples of the padded dimension");

__host__ __device__ inline int tc_pad_n(int n) { return (n + TC_NPAD - 1) / TC_NPAD * TC_NPAD; }

// Tiles of 128 rows x bn columns holding an entry with column >= row: row
// block tm keeps column blocks tn >= (128 tm) / bn.  Tiles are numbered row
// block by row block.
struct TileGrid {
    int tm_count, tn_count, bn;
    __host__ __device__ int first_tn(int tm) const { return (TC_BM * tm) / bn; }
    __host__ __device__ int count() const {
        int c = 0;
        for (int tm = 0; tm < tm_count; ++tm) c += tn_count - first_tn(tm);
        return c;
    }
    __device__ void coords(int idx, int& tm, int& tn) const {
        int r = 0;
        for (; r < tm_count - 1; ++r) {
            const int c = tn_count - first_tn(r);
            if (idx < c) break;
            idx -= c;
        }
        tm = r;
        tn = first_tn(r) + idx;
    }
};

inline TileGrid tc_tile_grid(int p, int bn) {
    return TileGrid{(p + TC_BM - 1) / TC_BM, (p + bn - 1) / bn, bn};
}

// One fit of the tensor-core Gram: TMA maps over its K-major operands
// XhT, XlT ([p][n_pad] bf16), its output and its first tile in the launch.
struct TcFit {
    CUtensorMap mh, ml;
    float* S;
    int p, n_pad, lds, tile_start;
    float inv_n;
    TileGrid g;
};

// Centre (optional), split into bf16 hi/lo and transpose a 32 x 32 block of
// X (rows i0.., columns c0..) into XhT, XlT ([p][n_pad]; rows n..n_pad-1 of
// the padded sample dimension are written as zeros).  Block shape 32 x 8.
__device__ __forceinline__ void split_transpose_tile(const float* __restrict__ X, int n, int p,
                                                     int ldx, const float* __restrict__ mu,
                                                     __nv_bfloat16* __restrict__ XhT,
                                                     __nv_bfloat16* __restrict__ XlT, int n_pad,
                                                     int i0, int c0) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, c = c0 + tx;
        float v = 0.f;
        if (i < n && c < p) v = X[(size_t)i * ldx + c] - (mu ? mu[c] : 0.f);
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int c = c0 + r, i = i0 + tx;
        if (c < p && i < n_pad) {
            const float v = tile[tx][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            XhT[(size_t)c * n_pad + i] = h;
            XlT[(size_t)c * n_pad + i] = l;
        }
    }
}

// The same for a block of 64 samples x 32 columns (block shape 32 x 8; i0 a
// multiple of 64, so with n_pad a multiple of 64 the block's samples are all
// below n_pad): lane tx writes samples i0 + 2 tx and i0 + 2 tx + 1 of a
// column as one 4-byte bf16 pair, so a warp stores 128 contiguous bytes.
// The tile is kept column-major (tile[column][sample], even stride), so the
// pair is one 8-byte shared-memory read.  Same values as
// split_transpose_tile.
__device__ __forceinline__ void split_transpose_tile64(const float* __restrict__ X, int n, int p,
                                                       int ldx, const float* __restrict__ mu,
                                                       __nv_bfloat16* __restrict__ XhT,
                                                       __nv_bfloat16* __restrict__ XlT, int n_pad,
                                                       int i0, int c0) {
    __shared__ __align__(16) float tile[32][66];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cl = c0 + tx;
    const float m = (mu && cl < p) ? mu[cl] : 0.f;
    for (int r = ty; r < 64; r += 8) {
        const int i = i0 + r;
        float v = 0.f;
        if (i < n && cl < p) v = X[(size_t)i * ldx + cl] - m;
        tile[tx][r] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int c = c0 + r, i = i0 + 2 * tx;
        if (c < p) {
            const float2 v = *reinterpret_cast<const float2*>(&tile[r][2 * tx]);
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v.x - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v.y - __bfloat162float(h1));
            *reinterpret_cast<__nv_bfloat162*>(XhT + (size_t)c * n_pad + i) = __halves2bfloat162(h0, h1);
            *reinterpret_cast<__nv_bfloat162*>(XlT + (size_t)c * n_pad + i) = __halves2bfloat162(l0, l1);
        }
    }
}

// Bytes of XhT + XlT for one fit (each 256-byte aligned).
inline size_t tc_operand_bytes(int n, int p) {
    return 2 * align_up((size_t)p * tc_pad_n(n) * 2, 256);
}

// Tile width of the batched launch.
constexpr int TC_BATCH_BN = 128;

// Fill f (host side) for a fit whose operands are at XhT / XlT and whose
// output is S (leading dimension lds).  False if the tensor maps could not be
// encoded.
bool tc_encode_fit(TcFit& f, const void* XhT, const void* XlT, int n, int p, float* S, int lds,
                   int tile_start, int bn);

// One persistent launch over the tiles of a batch: device table `fits`
// (tile_start ascending, every g.bn == TC_BATCH_BN) and the fit of each of
// the `n_tiles` tiles in `tile_fit`.
cudaError_t launch_gram_tc_batch(const TcFit* fits, const int* tile_fit, int n_tiles,
                                 cudaStream_t st);

}  // namespace spmesl
