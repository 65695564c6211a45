// Split-BF16 Gram S = X'X / n on the 5th-generation tensor cores
// (SPMESL_MIXED).
//
// X (FP32, n x p) is split as X = Xh + Xl with Xh = bf16(X) and
// Xl = bf16(X - Xh), and S ~ (Xh'Xh + Xh'Xl + Xl'Xh) / n with FP32
// accumulation (the dropped Xl'Xl term and the split residual are about
// 2^-17 of each product).  A first kernel centres (optional), splits and
// transposes X into K-major copies XhT, XlT ([p][n_pad] bf16, n_pad a
// multiple of 64, zero-padded), so both MMA operands are K-major rows.
//
// Main kernel: one CTA (4 warps) per 128 x 128 output tile with tile_m <=
// tile_n (S is symmetric; the tile and its mirror are both written).
//   - warp 0, one lane: TMA producer.  Per 64-wide K block it loads the four
//     128 x 64 bf16 operand tiles (Xh and Xl rows of tile_m and of tile_n)
//     with 128-byte swizzle into one of 3 shared-memory stages.
//   - warp 1, one lane: MMA issuer.  Per K block, 4 K-steps of 16, three
//     tcgen05.mma (hi*hi, hi*lo, lo*hi) into one 128 x 128 FP32 accumulator
//     in tensor memory; tcgen05.commit frees the stage.
//   - all 4 warps: epilogue.  Each warp reads its 32 accumulator lanes with
//     tcgen05.ld, scales by 1/n, stages the tile in shared memory and writes
//     the tile and its transpose with coalesced stores.
// Every wait on an mbarrier is bounded; on timeout the CTA stops issuing,
// writes NaN into its output tile (so the fit that reads S reports
// non-finite input) and still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gram_device.cuh"

namespace spmesl {

namespace {

constexpr int TC_TILE = 128;          // M = N = 128
constexpr int TC_KB = 64;             // K block (64 bf16 = one 128-byte swizzle row)
constexpr int TC_STAGES = 3;
constexpr int TC_OP_BYTES = TC_TILE * TC_KB * 2;       // 16 KB per operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_OP_BYTES;        // Ah, Al, Bh, Bl
constexpr int TC_TMEM_COLS = 128;
constexpr int TC_THREADS = 128;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s
// dynamic shared memory: stages + barriers + 1 KB for 1024-byte alignment
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 + 1024;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for an mbarrier phase; false on timeout.
__device__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity)) {
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stage buffers are 1024-aligned).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);        // start address
    d |= (unsigned long long)1 << 16;                           // leading byte offset (unused)
    d |= (unsigned long long)(1024 >> 4) << 32;                 // stride byte offset
    d |= (unsigned long long)1 << 46;                           // descriptor version
    d |= (unsigned long long)2 << 61;                           // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major,
// M = 128, N = 128.
constexpr unsigned kIdesc = (1u << 4)                  // D format F32
                            | (1u << 7)                // A format BF16
                            | (1u << 10)               // B format BF16
                            | ((unsigned)(TC_TILE >> 3) << 17)   // N >> 3
                            | ((unsigned)(TC_TILE >> 4) << 24);  // M >> 4

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a,
                                         unsigned long long b, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Centre (optional), split into bf16 hi/lo and transpose to [p][n_pad].
__global__ void split_transpose_kernel(const float* __restrict__ X, int n, int p, int ldx,
                                       const float* __restrict__ mu, __nv_bfloat16* __restrict__ XhT,
                                       __nv_bfloat16* __restrict__ XlT, int n_pad) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;            // 32 x 8
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

__global__ void tc_mean_kernel(const float* __restrict__ X, int n, int p, int ldx, float* mu) {
    column_means<float>(X, n, p, ldx, mu, blockIdx.x * blockDim.x + threadIdx.x,
                        gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap map_h,
                   const __grid_constant__ CUtensorMap map_l, int p, int n_pad, float inv_n,
                   float* __restrict__ S, int lds) {
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char* stages = smem;
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars[0..S): full, bars[S..2S): empty, bars[2S]: done
    volatile unsigned* tmem_slot = reinterpret_cast<volatile unsigned*>(bars + 2 * TC_STAGES + 1);
    volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* issued_slot = fail + 1;       // K blocks whose loads were issued
    volatile int* consumed_slot = fail + 2;     // K blocks whose loads the MMA issuer saw land

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = (p + TC_TILE - 1) / TC_TILE;
    int tm, tn;
    upper_tile(blockIdx.x, t, tm, tn);
    const int m0 = tm * TC_TILE, n0 = tn * TC_TILE;
    const int KT = n_pad / TC_KB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * TC_STAGES + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
        *fail = 0;
        *issued_slot = 0;
        *consumed_slot = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_h)));
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_l)));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(const_cast<unsigned*>(tmem_slot))),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kt = 0; kt < KT && !*fail; ++kt) {
            const int s = kt % TC_STAGES;
            if (kt >= TC_STAGES &&
                !mbar_wait(smem_u32(&bars[TC_STAGES + s]), ((kt / TC_STAGES) - 1) & 1)) {
                *fail = 1;
                break;
            }
            const unsigned full = smem_u32(&bars[s]);
            unsigned char* st = stages + (size_t)s * TC_STAGE_BYTES;
            mbar_expect_tx(full, TC_STAGE_BYTES);
            const int x = kt * TC_KB;
            tma_load_2d(smem_u32(st), &map_h, x, m0, full);
            tma_load_2d(smem_u32(st + TC_OP_BYTES), &map_l, x, m0, full);
            tma_load_2d(smem_u32(st + 2 * TC_OP_BYTES), &map_h, x, n0, full);
            tma_load_2d(smem_u32(st + 3 * TC_OP_BYTES), &map_l, x, n0, full);
            *issued_slot = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        unsigned acc = 0;
        int kt = 0;
        for (; kt < KT; ++kt) {
            const int s = kt % TC_STAGES;
            if (!mbar_wait(smem_u32(&bars[s]), (kt / TC_STAGES) & 1)) {
                *fail = 1;
                break;
            }
            *consumed_slot = kt + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned base = smem_u32(stages + (size_t)s * TC_STAGE_BYTES);
            const unsigned long long ah = smem_desc(base), al = smem_desc(base + TC_OP_BYTES);
            const unsigned long long bh = smem_desc(base + 2 * TC_OP_BYTES),
                                     bl = smem_desc(base + 3 * TC_OP_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_KB / 16; ++kk) {
                // advance 16 bf16 = 32 bytes along K inside the swizzled rows
                const unsigned long long off = (unsigned long long)((32 * kk) >> 4);
                mma_bf16(tmem, ah + off, bh + off, acc);
                acc = 1;
                mma_bf16(tmem, ah + off, bl + off, 1);
                mma_bf16(tmem, al + off, bh + off, 1);
            }
            mma_commit(smem_u32(&bars[TC_STAGES + s]));   // stage s free when these finish
        }
        mma_commit(smem_u32(&bars[2 * TC_STAGES]));       // accumulator ready
    }
    __syncwarp();

    // epilogue: wait for the accumulator (bounded)
    if (!mbar_wait(smem_u32(&bars[2 * TC_STAGES]), 0)) *fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool good = (*fail == 0);                          // same value in every thread
    if (!good && threadIdx.x == 0) {
        // let copies still in flight land before the stages are reused (bounded)
        const int issued = *issued_slot, consumed = *consumed_slot;
        for (int kt = consumed; kt < issued; ++kt)
            mbar_wait(smem_u32(&bars[kt % TC_STAGES]), (kt / TC_STAGES) & 1);
    }
    __syncthreads();
    float* stage_out = reinterpret_cast<float*>(stages);      // 128 x 129 floats, reuses stages
    const int row = warp * 32 + lane;
    for (int c = 0; c < TC_TILE; c += 16) {
        float v[16];
        if (good) {
            tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c, v);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) stage_out[row * (TC_TILE + 1) + c + i] = good ? v[i] * inv_n : v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    for (int e = threadIdx.x; e < TC_TILE * TC_TILE; e += TC_THREADS) {
        const int r = e / TC_TILE, c = e % TC_TILE;
        // on a diagonal tile (j, k) and (k, j) come out of different accumulation
        // orders; store the upper triangle's value in both so S is exactly symmetric
        const int rr = (tm == tn && c < r) ? c : r, cc = (tm == tn && c < r) ? r : c;
        if (m0 + r < p && n0 + c < p)
            S[(size_t)(m0 + r) * lds + n0 + c] = stage_out[rr * (TC_TILE + 1) + cc];
    }
    if (tm != tn) {
        for (int e = threadIdx.x; e < TC_TILE * TC_TILE; e += TC_THREADS) {
            const int r = e / TC_TILE, c = e % TC_TILE;     // mirror row r = col of the tile
            if (n0 + r < p && m0 + c < p)
                S[(size_t)(n0 + r) * lds + m0 + c] = stage_out[c * (TC_TILE + 1) + r];
        }
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS));
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(ptr);
    });
    return fn;
}

int pad_n(int n) { return (n + TC_KB - 1) / TC_KB * TC_KB; }

}  // namespace

size_t gram_tc_ws_bytes(int n, int p) {
    const size_t np = (size_t)pad_n(n);
    return align_up((size_t)p * 4, 256) + 2 * align_up((size_t)p * np * 2, 256);
}

cudaError_t launch_gram_tc(const float* X, int n, int p, int ldx, int center, float* S, int lds,
                           void* ws, cudaStream_t st) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int n_pad = pad_n(n);
    unsigned char* base = static_cast<unsigned char*>(ws);
    float* mu = reinterpret_cast<float*>(base);
    __nv_bfloat16* XhT = reinterpret_cast<__nv_bfloat16*>(base + align_up((size_t)p * 4, 256));
    __nv_bfloat16* XlT = reinterpret_cast<__nv_bfloat16*>(
        reinterpret_cast<unsigned char*>(XhT) + align_up((size_t)p * n_pad * 2, 256));
    if (center) tc_mean_kernel<<<(p + 255) / 256, 256, 0, st>>>(X, n, p, ldx, mu);
    split_transpose_kernel<<<dim3(n_pad / 32, (p + 31) / 32), dim3(32, 8), 0, st>>>(
        X, n, p, ldx, center ? mu : nullptr, XhT, XlT, n_pad);

    CUtensorMap mh, ml;
    const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)p};
    const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 2};
    const cuuint32_t box[2] = {TC_KB, TC_TILE};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, XhT, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (enc(&ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, XlT, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    const int t = (p + TC_TILE - 1) / TC_TILE;
    gram_tc_kernel<<<t * (t + 1) / 2, TC_THREADS, TC_SMEM, st>>>(mh, ml, p, n_pad,
                                                                 (float)(1.0 / (double)n), S, lds);
    return cudaGetLastError();
}

}  // namespace spmesl
