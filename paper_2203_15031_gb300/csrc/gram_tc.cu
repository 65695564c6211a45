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
// Main kernel: persistent, one CTA (10 warps) per SM, looping over the
// 128 x BN output tiles that hold at least one entry of the upper triangle
// (column >= row); each entry S_jk with k >= j is computed once and written
// to both S_jk and S_kj, so S is exactly symmetric.
//   - warp 0, one lane: TMA producer.  Per K block of KB bf16 it loads the
//     Xh and Xl rows of the tile's 128 rows and BN columns with KB*2-byte
//     swizzle into one of STAGES shared-memory stages.
//   - warp 1: owns the tensor memory (two BN-column FP32 accumulators); one
//     lane issues, per K block and per K step of 16, three tcgen05.mma
//     (hi*hi, hi*lo, lo*hi) and commits the stage back to the producer and,
//     after the last K block, the accumulator to the epilogue.
//   - warps 2-9: epilogue, one 32-lane quadrant of the accumulator and one
//     half of its columns each.  Per 32-column chunk: tcgen05.ld, scale by
//     1/n, store the mirror S_kj straight from registers (lanes run along a
//     row of S) and S_jk as 16-byte stores through a 32 x 32 swizzled
//     transpose in shared memory.  The accumulator is handed back once
//     read, so the epilogue of tile i runs under the MMAs of tile i+1.
// Every wait on an mbarrier is bounded and also ends when another role has
// failed; on failure the CTA stops issuing, writes NaN into the tile it was
// on and every later tile of its share (so the fit that reads S reports
// non-finite input), lets its copies and MMAs in flight land and still
// releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gram_device.cuh"
#include "gram_tc.cuh"

namespace spmesl {

namespace {

constexpr int TC_THREADS = 320;       // producer, MMA, 8 epilogue warps
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_EPI_WARP0 = 2;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s

template <int BN, int KB, int STAGES>
struct TcCfg {
    static_assert(BN == 128 || BN == 256, "BN");
    static_assert(KB == 32 || KB == 64, "KB");
    static constexpr int A_BYTES = TC_BM * KB * 2;          // one 128-row operand tile
    static constexpr int B_BYTES = BN * KB * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // Ah, Al, Bh, Bl
    static constexpr int TMEM_COLS = 2 * BN;                 // two accumulators
    static constexpr int EPI_FLOATS = 32 * 32;               // per epilogue warp
    // barriers: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], done
    static constexpr int NBARS = 2 * STAGES + 5;
    // + tensor-memory address, flags and the K-block ring, + 1024-byte alignment
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + TC_EPI_WARPS * EPI_FLOATS * 4 +
                                   NBARS * 8 + 64 + 1024;
    // smem descriptor: layout type (2 = 128-byte swizzle, 4 = 64-byte) and
    // the byte distance between 8-row groups
    static constexpr unsigned long long SWZ = KB == 64 ? 2ull : 4ull;
    static constexpr unsigned SBO = 8 * KB * 2;
    // instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = BN
    static constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                      ((unsigned)(BN >> 3) << 17) |
                                      ((unsigned)(TC_BM >> 4) << 24);
};

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

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// Bounded wait for an mbarrier phase; false on timeout or once another role
// has raised the failure flag (fail may be null).
__device__ bool mbar_wait(unsigned bar, unsigned parity, const volatile int* fail) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity)) {
        if ((fail && *fail) || global_ns() - t0 > TC_WAIT_NS) return false;
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

// Shared-memory matrix descriptor of a K-major swizzled operand whose rows
// are KB*2 bytes and whose 8-row groups are SBO bytes apart (buffers are
// 1024-byte aligned, so the swizzle phase starts at zero).
template <class C>
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);        // start address
    d |= (unsigned long long)1 << 16;                           // leading byte offset (unused)
    d |= (unsigned long long)(C::SBO >> 4) << 32;               // stride byte offset
    d |= (unsigned long long)1 << 46;                           // descriptor version
    d |= C::SWZ << 61;                                          // swizzle mode
    return d;
}

template <class C>
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a,
                                         unsigned long long b, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(C::IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Centre (optional), split into bf16 hi/lo and transpose to [p][n_pad].
__global__ void split_transpose_kernel(const float* __restrict__ X, int n, int p, int ldx,
                                       const float* __restrict__ mu, __nv_bfloat16* __restrict__ XhT,
                                       __nv_bfloat16* __restrict__ XlT, int n_pad) {
    split_transpose_tile(X, n, p, ldx, mu, XhT, XlT, n_pad, blockIdx.x * 32, blockIdx.y * 32);
}

__global__ void tc_mean_kernel(const float* __restrict__ X, int n, int p, int ldx, float* mu) {
    column_means<float>(X, n, p, ldx, mu, blockIdx.x * blockDim.x + threadIdx.x,
                        gridDim.x * blockDim.x);
}

// Where one tile's operands and output are.
struct TcJob {
    const CUtensorMap* mh;
    const CUtensorMap* ml;
    float* S;
    int lds, p, m0, n0, KT;
    float inv_n;
};

template <int KB>
__device__ __forceinline__ void make_job(const TcFit& f, int local, TcJob& j) {
    int tm, tn;
    f.g.coords(local, tm, tn);
    j.mh = &f.mh;
    j.ml = &f.ml;
    j.S = f.S;
    j.lds = f.lds;
    j.p = f.p;
    j.m0 = tm * TC_BM;
    j.n0 = tn * f.g.bn;
    j.KT = f.n_pad / KB;
    j.inv_n = f.inv_n;
}

// Tile source of one fit: the fit (and its tensor maps) in the kernel's
// parameter space.
struct TcOne {
    TcFit f;
    int n_tiles;
    static constexpr bool kTableMaps = false;
    __device__ int tiles() const { return n_tiles; }
    __device__ int fit_index(int) const { return 0; }
    __device__ const TcFit& fit_at(int) const { return f; }
};

// Tile source of a batch: a table of fits and the fit of every tile, in
// global memory.
struct TcMany {
    const TcFit* fits;
    const int* tile_fit;
    int n_tiles;
    static constexpr bool kTableMaps = true;
    __device__ int tiles() const { return n_tiles; }
    __device__ int fit_index(int tile) const { return __ldg(tile_fit + tile); }
    __device__ const TcFit& fit_at(int fi) const { return fits[fi]; }
};

// Slots of the per-tile K-block counts the producer hands to the MMA issuer
// (the producer runs at most STAGES K blocks, so at most STAGES tiles, ahead).
constexpr int TC_RING = 8;

template <int BN, int KB, int STAGES, class Src>
__global__ void __launch_bounds__(TC_THREADS, 1) gram_tc_kernel(const __grid_constant__ Src src) {
    using C = TcCfg<BN, KB, STAGES>;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char* stages = smem;
    float* epi = reinterpret_cast<float*>(smem + (size_t)STAGES * C::STAGE_BYTES);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(epi + TC_EPI_WARPS * C::EPI_FLOATS);
    unsigned long long* full = bars;
    unsigned long long* empty = bars + STAGES;
    unsigned long long* acc_full = bars + 2 * STAGES;
    unsigned long long* acc_empty = bars + 2 * STAGES + 2;
    unsigned long long* done = bars + 2 * STAGES + 4;
    volatile unsigned* tmem_slot = reinterpret_cast<volatile unsigned*>(bars + C::NBARS);
    volatile int* fail = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* issued_slot = fail + 1;       // K blocks whose loads were issued
    volatile int* consumed_slot = fail + 2;     // K blocks whose loads the MMA issuer saw land
    volatile int* kt_ring = fail + 4;           // K blocks of the CTA's i-th tile at [i % TC_RING]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = src.tiles();

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), TC_EPI_WARPS);   // one arrival per epilogue warp
        }
        mbar_init(smem_u32(done), 1);
        *fail = 0;
        *issued_slot = 0;
        *consumed_slot = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(const_cast<unsigned*>(tmem_slot))),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            int kb = 0;      // K blocks issued by this CTA over all its tiles
            const TcFit* last = nullptr;
            int fi_next = blockIdx.x < n_tiles ? src.fit_index(blockIdx.x) : 0;
            int li = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*fail; tile += gridDim.x, ++li) {
                const int fi = fi_next;
                // the next tile's fit is read while this tile's copies run
                if (tile + (int)gridDim.x < n_tiles) fi_next = src.fit_index(tile + gridDim.x);
                const TcFit& f = src.fit_at(fi);
                TcJob jb;
                make_job<KB>(f, tile - f.tile_start, jb);
                kt_ring[li % TC_RING] = jb.KT;      // published by the first expect_tx below
                if (Src::kTableMaps && &f != last) {
                    // maps written to global memory before the launch: order
                    // those writes before the copies that read the maps
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                     reinterpret_cast<unsigned long long>(jb.mh))
                                 : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                     reinterpret_cast<unsigned long long>(jb.ml))
                                 : "memory");
                    last = &f;
                }
                const int m0 = jb.m0, n0 = jb.n0;
                for (int kt = 0; kt < jb.KT; ++kt, ++kb) {
                    const int s = kb % STAGES;
                    if (kb >= STAGES &&
                        !mbar_wait(smem_u32(&empty[s]), ((kb / STAGES) - 1) & 1, fail)) {
                        *fail = 1;
                        break;
                    }
                    const unsigned fb = smem_u32(&full[s]);
                    unsigned char* st = stages + (size_t)s * C::STAGE_BYTES;
                    mbar_expect_tx(fb, C::STAGE_BYTES);
                    const int x = kt * KB;
                    tma_load_2d(smem_u32(st), jb.mh, x, m0, fb);
                    tma_load_2d(smem_u32(st + C::A_BYTES), jb.ml, x, m0, fb);
                    unsigned char* bh = st + 2 * C::A_BYTES;
                    unsigned char* bl = bh + C::B_BYTES;
#pragma unroll
                    for (int h = 0; h < BN / TC_BM; ++h) {
                        tma_load_2d(smem_u32(bh + h * C::A_BYTES), jb.mh, x, n0 + h * TC_BM, fb);
                        tma_load_2d(smem_u32(bl + h * C::A_BYTES), jb.ml, x, n0 + h * TC_BM, fb);
                    }
                    *issued_slot = kb + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            int kb = 0, local = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++local) {
                const int b = local & 1, u = local >> 1;
                if (u >= 1 && !mbar_wait(smem_u32(&acc_empty[b]), (u - 1) & 1, fail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned d = tmem + (unsigned)(b * BN);
                int KT = 1;                  // read once the tile's first K block has landed
                for (int kt = 0; kt < KT; ++kt, ++kb) {
                    const int s = kb % STAGES;
                    if (!mbar_wait(smem_u32(&full[s]), (kb / STAGES) & 1, fail)) {
                        ok = false;
                        break;
                    }
                    if (kt == 0) KT = kt_ring[local % TC_RING];
                    *consumed_slot = kb + 1;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned base = smem_u32(stages + (size_t)s * C::STAGE_BYTES);
                    const unsigned long long ah = smem_desc<C>(base),
                                             al = smem_desc<C>(base + C::A_BYTES);
                    const unsigned long long bh = smem_desc<C>(base + 2 * C::A_BYTES),
                                             bl = smem_desc<C>(base + 2 * C::A_BYTES + C::B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < KB / 16; ++kk) {
                        // advance 16 bf16 = 32 bytes along K inside the swizzled rows
                        const unsigned long long off = (unsigned long long)((32 * kk) >> 4);
                        mma_bf16<C>(d, ah + off, bh + off, (kt | kk) ? 1u : 0u);
                        mma_bf16<C>(d, ah + off, bl + off, 1u);
                        mma_bf16<C>(d, al + off, bh + off, 1u);
                    }
                    mma_commit(smem_u32(&empty[s]));       // stage s free when these finish
                }
                if (!ok) break;
                mma_commit(smem_u32(&acc_full[b]));        // accumulator b ready
            }
            if (!ok) *fail = 1;
            // every MMA issued above has finished once this commit arrives
            mma_commit(smem_u32(done));
            mbar_wait(smem_u32(done), 0, nullptr);
        }
    } else {
        // epilogue: 8 warps; warp w reads accumulator lanes 32 (w % 4) .. +31,
        // warps 2-5 the first half of the columns and warps 6-9 the second
        const int ew = warp - TC_EPI_WARP0;
        const int q = warp & 3, half = ew >> 2;
        // 32 x 32 floats, row j at 32 j, its 16-byte groups XOR-swizzled by j
        float4* buf = reinterpret_cast<float4*>(epi + ew * C::EPI_FLOATS);
        bool ok = true;
        int local = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++local) {
            TcJob jb;
            {
                const TcFit& f = src.fit_at(src.fit_index(tile));
                make_job<KB>(f, tile - f.tile_start, jb);
            }
            const int m0 = jb.m0 + 32 * q, n0 = jb.n0, p = jb.p, lds = jb.lds;
            float* __restrict__ S = jb.S;
            const float inv_n = jb.inv_n;
            const bool vec = (lds & 3) == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0;
            const int b = local & 1, u = local >> 1;
            if (ok) {
                int got = 0;
                if (lane == 0) got = mbar_wait(smem_u32(&acc_full[b]), u & 1, fail) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, got, 0) != 0;
                if (!ok && lane == 0) *fail = 1;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = m0 + lane;
            for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
                const int c0 = n0 + c;
                // chunk outside S or wholly below the diagonal
                if (m0 >= p || c0 >= p || c0 + 31 < m0) continue;
                float v[32];
                if (ok) {
                    tmem_ld32(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(b * BN + c), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] *= inv_n;
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = __int_as_float(0x7fc00000);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    buf[lane * 8 + (k ^ (lane & 7))] =
                        make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                __syncwarp();
                if (vec && c0 > m0 + 31 && c0 + 32 <= p && m0 + 32 <= p) {
                    // interior chunk, strictly above the diagonal: no predicates
                    float* dm = S + (size_t)c0 * lds + row;       // mirror S_kj, lanes along row k
#pragma unroll
                    for (int i = 0; i < 32; ++i) dm[(size_t)i * lds] = v[i];
                    const int g = lane & 7;                       // S_jk, 4 rows x 128 bytes per store
#pragma unroll
                    for (int jj = 0; jj < 32; jj += 4) {
                        const int j = jj + (lane >> 3);
                        *reinterpret_cast<float4*>(S + (size_t)(m0 + j) * lds + c0 + 4 * g) =
                            buf[j * 8 + (g ^ (j & 7))];
                    }
                } else {
                    // diagonal or ragged chunk: S_kj for k > j, S_jk for k >= j
                    if (row < p) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int col = c0 + i;
                            if (col < p && col > row) S[(size_t)col * lds + row] = v[i];
                        }
                    }
                    const int col = c0 + lane;
                    const float* bf = reinterpret_cast<const float*>(buf);
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) {
                        const int r = m0 + j;
                        if (r < p && col < p && col >= r)
                            S[(size_t)r * lds + col] = bf[(j * 8 + ((lane >> 2) ^ (j & 7))) * 4 + (lane & 3)];
                    }
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        }
    }
    __syncthreads();
    if (*fail && threadIdx.x == 0) {
        // let copies still in flight land before the CTA exits (bounded)
        const int issued = *issued_slot, consumed = *consumed_slot;
        for (int kb = consumed; kb < issued; ++kb)
            mbar_wait(smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::TMEM_COLS));
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

// Operand maps over XhT / XlT ([p][n_pad] bf16): boxes of KB x 128 rows.
template <int KB>
bool encode_maps(EncodeTiled enc, CUtensorMap& mh, CUtensorMap& ml, const void* XhT,
                 const void* XlT, int p, int n_pad) {
    const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)p};
    const cuuint64_t strides[1] = {(cuuint64_t)n_pad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KB, (cuuint32_t)TC_BM};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle swz = KB == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    return enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(XhT), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
           enc(&ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(XlT), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int TC_KB = 64;             // K block of every launch (128-byte swizzle)

bool fill_fit(EncodeTiled enc, TcFit& f, const void* XhT, const void* XlT, int n, int p, float* S,
              int lds, int tile_start, int bn) {
    f = TcFit{};
    f.n_pad = tc_pad_n(n);
    if (!encode_maps<TC_KB>(enc, f.mh, f.ml, XhT, XlT, p, f.n_pad)) return false;
    f.S = S;
    f.p = p;
    f.lds = lds;
    f.tile_start = tile_start;
    f.inv_n = (float)(1.0 / (double)n);
    f.g = tc_tile_grid(p, bn);
    return true;
}

int num_sms_now() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

template <int BN, int STAGES, class Src>
cudaError_t launch_src(const Src& src, int n_tiles, cudaStream_t st) {
    using C = TcCfg<BN, TC_KB, STAGES>;
    auto kern = gram_tc_kernel<BN, TC_KB, STAGES, Src>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const int sms = num_sms_now();
    if (sms <= 0) return cudaErrorInvalidDevice;
    if (n_tiles <= 0) return cudaSuccess;
    const int grid = n_tiles < sms ? n_tiles : sms;
    kern<<<grid, TC_THREADS, C::SMEM, st>>>(src);
    return cudaGetLastError();
}

}  // namespace

size_t gram_tc_ws_bytes(int n, int p) { return align_up((size_t)p * 4, 256) + tc_operand_bytes(n, p); }

cudaError_t launch_gram_tc(const float* X, int n, int p, int ldx, int center, float* S, int lds,
                           void* ws, cudaStream_t st) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int n_pad = tc_pad_n(n);
    unsigned char* base = static_cast<unsigned char*>(ws);
    float* mu = reinterpret_cast<float*>(base);
    __nv_bfloat16* XhT = reinterpret_cast<__nv_bfloat16*>(base + align_up((size_t)p * 4, 256));
    __nv_bfloat16* XlT = reinterpret_cast<__nv_bfloat16*>(
        reinterpret_cast<unsigned char*>(XhT) + align_up((size_t)p * n_pad * 2, 256));
    if (center) tc_mean_kernel<<<(p + 255) / 256, 256, 0, st>>>(X, n, p, ldx, mu);
    split_transpose_kernel<<<dim3(n_pad / 32, (p + 31) / 32), dim3(32, 8), 0, st>>>(
        X, n, p, ldx, center ? mu : nullptr, XhT, XlT, n_pad);
    // 128 x 256 tiles cut the operand traffic per flop by a quarter against
    // 128 x 128 and keep the MMA operand reads within shared-memory
    // bandwidth; two 96 KB stages of 128-byte-swizzled K blocks of 64 ran
    // faster than four 48 KB stages of 64-byte-swizzled blocks of 32.  Small
    // p keeps 128-column tiles for more tiles per SM.
    const int bn = p > 1024 ? 256 : 128;
    TcOne one;
    if (!fill_fit(enc, one.f, XhT, XlT, n, p, S, lds, 0, bn)) return cudaErrorInvalidValue;
    one.n_tiles = one.f.g.count();
    if (bn == 256) return launch_src<256, 2>(one, one.n_tiles, st);
    return launch_src<128, 3>(one, one.n_tiles, st);
}

bool tc_encode_fit(TcFit& f, const void* XhT, const void* XlT, int n, int p, float* S, int lds,
                   int tile_start, int bn) {
    EncodeTiled enc = encoder();
    return enc && fill_fit(enc, f, XhT, XlT, n, p, S, lds, tile_start, bn);
}

cudaError_t launch_gram_tc_batch(const TcFit* fits, const int* tile_fit, int n_tiles,
                                 cudaStream_t st) {
    static_assert(TC_BATCH_BN == 128, "the batched launch is instantiated for 128-column tiles");
    TcMany many{fits, tile_fit, n_tiles};
    return launch_src<128, 3>(many, n_tiles, st);
}

}  // namespace spmesl
