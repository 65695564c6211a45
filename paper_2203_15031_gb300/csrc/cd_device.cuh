#pragma once
// Device building blocks of the coordinate-descent fit, shared by the single-fit
// kernels (cd.cu) and the batched kernels (batch.cu).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "common.cuh"

namespace spmesl {

template <typename T>
struct CDArgs {
    const T* SC;
    T* BT;
    T* GT;
    const T* diag;       // S_kk of the working matrix (unstandardised update)
    double* sigma;       // working-scale sigma
    int* col_status;
    int* active;
    int* active_next;
    int* flag;
    FitCtrl* ctrl;
    int p, ldp, maxit;
    double lambda0, tol;
    int* ovf_list;       // columns handed from the lazy solver to the block (or eager) solver
    int* ovf_count;
    const int* order;    // queue order of the lazy solver (nullptr: 0..p-1)
    int n_queue;         // columns the lazy solver takes from its queue
    int ovf_supp;        // the lazy solver hands a column over when its support exceeds this
                         // at the start of an active-set phase (ACT_MAX with heavy-column
                         // routing, LAZY_CAP without)
    const float* chunk_max;   // per column j and 128-coordinate chunk c, max_k |S^C_jk| over
                              // the chunk (k != j), written by the standardisation pass; the
                              // first sweep's skip test starts from it (nullptr: scan all)
    unsigned* rows_moved;     // measurement (nullptr: off): bit k of row m is set when
                              // coordinate k moved in the m-th full sweep of any column
    int rows_words;           // 32-bit words per row of that bitmap
    double* hand;             // per column the last sigma step (sigma, F(sigma)) at a hand-over
                              // from the lazy to the block solver (nullptr: the block solver
                              // starts every column afresh)
};

// Full sweeps per column whose moved coordinates are recorded in the bitmap.
constexpr int ROWS_SWEEPS = 64;

// ctrl->rows_moved += the set bits of bits[0, nwords) (grid-stride).
__device__ __forceinline__ void count_rows_moved(const unsigned* __restrict__ bits, size_t nwords,
                                                 FitCtrl* ctrl, size_t tid, size_t nthr) {
    unsigned long long c = 0;
    for (size_t i = tid; i < nwords; i += nthr) c += __popc(bits[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&ctrl->rows_moved, c);
}

// Record that coordinate k moved in full sweep m (one thread calls it).
template <typename T>
__device__ __forceinline__ void note_row_moved(const CDArgs<T>& a, int m, int k) {
    if (a.rows_moved && m >= 0 && m < ROWS_SWEEPS)
        atomicOr(a.rows_moved + (size_t)m * a.rows_words + (k >> 5), 1u << (k & 31));
}

namespace {
// Order of a coordinate-descent queue: columns by decreasing heat (the count
// of off-diagonal standardised entries above lambda0, from standardize_row;
// counting sort, one block), so the longest column solves start first instead
// of in the tail of the launch.  Ties in any order: a column's result does not
// depend on when it runs.  With n_heavy, also the number of columns whose heat
// exceeds heavy_heat (< HEAT_BINS - 1): they lead the order and go to the
// block solver.
constexpr int HEAT_BINS = 64;
__global__ void __launch_bounds__(1024) order_by_heat_kernel(const int* __restrict__ heat, int n,
                                                          int* __restrict__ order,
                                                          int* __restrict__ n_heavy,
                                                          int heavy_heat) {
    __shared__ int bin[HEAT_BINS];
    const int t = threadIdx.x;
    if (t < HEAT_BINS) bin[t] = 0;
    __syncthreads();
    for (int i = t; i < n; i += blockDim.x) atomicAdd(&bin[min(heat[i], HEAT_BINS - 1)], 1);
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int h = HEAT_BINS - 1; h >= 0; --h) {
            const int c = bin[h];
            bin[h] = run;
            run += c;
            if (h == heavy_heat + 1 && n_heavy) *n_heavy = run;
        }
    }
    __syncthreads();
    for (int i = t; i < n; i += blockDim.x) order[atomicAdd(&bin[min(heat[i], HEAT_BINS - 1)], 1)] = i;
}
}  // namespace

template <typename T>
__device__ __forceinline__ T soft(T x, T lam) {
    // Soft_lambda(x) = sign(x) (|x| - lambda)_+   (Section 3.1)
    return x > lam ? x - lam : (x < -lam ? x + lam : T(0));
}

// The smallest float f >= x.  For a float m, m < x exactly when m < f, so a
// stop test of a float iterate against the FP64 tolerance needs no FP64
// arithmetic per test.
__device__ __forceinline__ float float_at_least(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

// md < tol for an iterate of the working precision T (float: against the
// float threshold tf of float_at_least(tol); double: directly).
template <typename T>
__device__ __forceinline__ bool below_tol(T md, double tol, float tf) {
    if constexpr (sizeof(T) == 4) return md < tf;
    else return (double)md < tol;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Ordered bits of a non-negative double (for atomicMax).
__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}

// dst[0..ldp) = src[0..ldp) with 16-byte vectors (one warp).
template <typename T>
__device__ __forceinline__ void warp_copy(T* __restrict__ dst, const T* __restrict__ src, int ldp) {
    using V = typename Vec16<T>::type;
    constexpr int N = Vec16<T>::N;
    const int lane = threadIdx.x & 31;
    for (int l = lane * N; l < ldp; l += 32 * N)
        *reinterpret_cast<V*>(dst + l) = *reinterpret_cast<const V*>(src + l);
}

template <typename T>
__device__ __forceinline__ void warp_zero(T* __restrict__ dst, int ldp) {
    using V = typename Vec16<T>::type;
    constexpr int N = Vec16<T>::N;
    const int lane = threadIdx.x & 31;
    V z;
    if constexpr (N == 4) z = make_float4(0.f, 0.f, 0.f, 0.f);
    else z = make_double2(0.0, 0.0);
    for (int l = lane * N; l < ldp; l += 32 * N) *reinterpret_cast<V*>(dst + l) = z;
}

// g[l] -= srow[l] * delta for l in [0, ldp): the column-j slice of the rank-1
// update G -= S_.k delta_k. (Proposition 2 on the covariance.)
template <typename T>
__device__ __forceinline__ void axpy_row(T* __restrict__ g, const T* __restrict__ srow, T delta,
                                         int ldp) {
    const int lane = threadIdx.x & 31;
    if constexpr (sizeof(T) == 4) {
        for (int l = lane * 4; l < ldp; l += 128) {
            const float4 s = __ldg(reinterpret_cast<const float4*>(srow + l));
            float4 v = *reinterpret_cast<float4*>(g + l);
            v.x = fmaf(-s.x, delta, v.x);
            v.y = fmaf(-s.y, delta, v.y);
            v.z = fmaf(-s.z, delta, v.z);
            v.w = fmaf(-s.w, delta, v.w);
            *reinterpret_cast<float4*>(g + l) = v;
        }
    } else {
        for (int l = lane * 2; l < ldp; l += 64) {
            const double2 s = __ldg(reinterpret_cast<const double2*>(srow + l));
            double2 v = *reinterpret_cast<double2*>(g + l);
            v.x = fma(-s.x, delta, v.x);
            v.y = fma(-s.y, delta, v.y);
            *reinterpret_cast<double2*>(g + l) = v;
        }
    }
}

// One cyclic ascending sweep over k != j for column j (Algorithm 1's inner
// loop, written on g = S_.j - S b).  Returns max |delta b| over the sweep
// (same value in every lane); `moves` counts coordinates that changed.
// Four consecutive elements starting at a 4-aligned index (16-byte or 2 x
// 16-byte shared-memory loads).
template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ src, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(src);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(src);
        const double2 q1 = *reinterpret_cast<const double2*>(src + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

// Each lane evaluates 4 consecutive coordinates, so one step of the warp
// covers a 128-coordinate chunk; the first coordinate whose update changes b
// is applied and the scan resumes right after it within the chunk.
constexpr int SCAN_V = 4;
constexpr int CHUNK = 32 * SCAN_V;

// Per-chunk summary kept between sweeps for the skip test (standardised
// working matrix only): after the chunk was last scanned, the largest |g_k|
// over its coordinates with b_k = 0, how many of its b_k were nonzero, and
// the running sum of |delta| and move count at that moment.
struct ChunkInfo {
    float maxabs;
    float dsum_at;
    unsigned moves_at;
    int nsupp;
};

// Scan state of one column solve (warp-uniform).
struct ColScan {
    ChunkInfo* ci;
    float dsum;          // running sum of the l1 size of every change of b_j so far: one
                         // move's |delta|, or an active-set phase's net change
    unsigned nmoves;     // number of those changes
    float bl1;           // lazy solver: an upper bound of ||b_j||_1 (0 elsewhere)
};

// A chunk with no support can be skipped when no coordinate in it can reach
// the threshold: each move delta_m at row m changes g_k by -S_km delta_m with
// |S_km| <= 1 (standardised), so |g_k| <= maxabs + sum|delta| since the chunk
// was scanned (and a change of several coefficients at once moves g_k by at
// most its l1 size).  The lazy solver forms g_k afresh from S rows at every
// scan: each of the two computations (then and now) is off by at most
// 384 * 2^-24 (1 + ||b||_1) (up to 256 support rows and 128 moves in a
// chunk, |S| <= 1), the last term below with ||b_then||_1 <=
// ||b_now||_1 + the change since.  The margins cover FP32 rounding of the standardised S
// (|S_km| <= 1 + 2^-22), of every g update (half an ulp of a value below
// lambda) and of the running sum (each of the dm additions since the scan is
// off by at most 2^-24 of the sum, which only grows); after 4096 moves the
// chunk is always rescanned.  A skipped coordinate therefore has
// |g_k| < lambda and b_k = 0, so it would not have moved: the sweep is the
// same as a full scan.  With `frozen` (a sweep that leaves the support's
// values as they are, see solve_column_lazy) a chunk holding support may be
// skipped too: maxabs covers the chunk's coordinates that were zero when it
// was scanned, and a coordinate that has left the support since then marks
// its chunk for a rescan (maxabs = infinity).
__device__ __forceinline__ bool chunk_skippable(const ChunkInfo& c, const ColScan& cs, float lam,
                                                bool frozen = false) {
    const unsigned dm = cs.nmoves - c.moves_at;
    if ((c.nsupp != 0 && !frozen) || dm > 4096u) return false;
    const float dd = cs.dsum - c.dsum_at;
    const float bound = c.maxabs + dd * (1.0f + 0x1p-10f) + cs.dsum * (float)(dm + 2u) * 0x1p-23f +
                        (float)dm * lam * 0x1p-20f + (1.0f + cs.bl1 + dd) * 0x1p-14f;
    return bound < lam;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

template <typename T, bool STD>
__device__ T sweep_column(int j, T* __restrict__ g, T* __restrict__ b, const CDArgs<T>& a, T lam,
                          unsigned long long& moves, ColScan& cs, int sweep_idx = -1) {
    const int lane = threadIdx.x & 31;
    const int p = a.p;
    const int ldp = a.ldp;
    T maxd = T(0);
    for (int cb = 0, ci = 0; cb < p; cb += CHUNK, ++ci) {
        if constexpr (STD) {
            if (chunk_skippable(cs.ci[ci], cs, (float)lam)) continue;
        }
        const int k0 = cb + lane * SCAN_V;
        int cursor = cb;
        for (;;) {
            T gv[SCAN_V], bv[SCAN_V], nbv[SCAN_V];
            if (k0 < ldp) {                   // ldp is a multiple of 32: the whole quad is in range
                load4<T>(g + k0, gv);
                load4<T>(b + k0, bv);
            } else {
#pragma unroll
                for (int t = 0; t < SCAN_V; ++t) gv[t] = bv[t] = T(0);
            }
            unsigned mvmask = 0u;
#pragma unroll
            for (int t = 0; t < SCAN_V; ++t) {
                const int k = k0 + t;
                nbv[t] = bv[t];
                if (k >= cursor && k < p && k != j) {
                    T nb;
                    if constexpr (STD) {
                        nb = soft<T>(gv[t] + bv[t], lam);                  // S_kk = 1
                    } else {
                        const T skk = a.diag[k];
                        nb = soft<T>(gv[t] + skk * bv[t], lam) / skk;      // Soft(c, lambda)/S_kk
                    }
                    nbv[t] = nb;
                    if (nb != bv[t]) mvmask |= 1u << t;
                }
            }
            const unsigned bal = __ballot_sync(FULL_MASK, mvmask != 0u);
            if (bal == 0u) break;
            const int f = __ffs(bal) - 1;
            const int tf = __ffs(__shfl_sync(FULL_MASK, mvmask, f)) - 1;
            T nb_sel = nbv[0], b_sel = bv[0];
#pragma unroll
            for (int t = 1; t < SCAN_V; ++t)
                if (t == tf) { nb_sel = nbv[t]; b_sel = bv[t]; }
            const T nbs = __shfl_sync(FULL_MASK, nb_sel, f);
            const T delta = nbs - __shfl_sync(FULL_MASK, b_sel, f);
            const int ks = cb + f * SCAN_V + tf;
            if (lane == 0) {
                b[ks] = nbs;
                note_row_moved(a, sweep_idx, ks);
            }
            maxd = fmax(maxd, fabs(delta));
            ++moves;
            cs.dsum += fabsf((float)delta);
            ++cs.nmoves;
            axpy_row<T>(g, a.SC + (size_t)ks * ldp, delta, ldp);
            __syncwarp();
            cursor = ks + 1;
            if (cursor >= cb + CHUNK) break;
        }
        if constexpr (STD) {
            // summary of the chunk as it leaves the scan
            float mx = 0.f;
            int ns = 0;
            if (k0 < ldp) {
                T gv[SCAN_V], bv[SCAN_V];
                load4<T>(g + k0, gv);
                load4<T>(b + k0, bv);
#pragma unroll
                for (int t = 0; t < SCAN_V; ++t) {
                    const int k = k0 + t;
                    if (k < p && k != j) {
                        if (bv[t] != T(0)) ++ns;
                        else mx = fmaxf(mx, fabsf((float)gv[t]));
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
                ns += __shfl_xor_sync(FULL_MASK, ns, o);
            }
            if (lane == 0) cs.ci[ci] = ChunkInfo{mx, cs.dsum, cs.nmoves, ns};
            __syncwarp();
        }
    }
    return maxd;
}

// Mark every chunk "must scan" (maxabs = infinity fails every skip test).
__device__ __forceinline__ void reset_chunks(ColScan& cs, int ldp) {
    const int nc = (ldp + CHUNK - 1) / CHUNK;
    for (int c = threadIdx.x & 31; c < nc; c += 32) cs.ci[c] = ChunkInfo{INFINITY, 0.f, 0u, 1};
    cs.dsum = 0.f;
    cs.nmoves = 0u;
    cs.bl1 = 0.f;
}

// Per-warp scratch for the support list used by the sigma update.
constexpr int SUPP_CAP = 128;

// Shared memory of one warp: g_j and b_j (ldp elements each), the support
// list and the chunk summaries.
__host__ __device__ constexpr int num_chunks(int ldp) { return (ldp + CHUNK - 1) / CHUNK; }

template <typename T>
__host__ __device__ constexpr size_t warp_smem_bytes(int ldp) {
    return 2 * (size_t)ldp * sizeof(T) + SUPP_CAP * sizeof(int) +
           (size_t)num_chunks(ldp) * sizeof(ChunkInfo);
}

// sigma_j^2 = S_jj - 2 b'S_.j + b'S b in FP64 over the support of b
// (Eq. (14) written on S).  Same value in every lane.
template <typename T>
__device__ double residual_quadratic_form(int j, const T* __restrict__ b, const CDArgs<T>& a,
                                          int* __restrict__ list) {
    const int lane = threadIdx.x & 31;
    const int p = a.p;
    // support of b in ascending order
    int ns = 0;
    for (int c0 = 0; c0 < p; c0 += 32) {
        const int k = c0 + lane;
        const bool nz = k < p && b[k] != T(0);
        const unsigned bal = __ballot_sync(FULL_MASK, nz);
        if (nz) {
            const int pos = ns + __popc(bal & ((1u << lane) - 1u));
            if (pos < SUPP_CAP) list[pos] = k;
        }
        ns += __popc(bal);
    }
    __syncwarp();
    double lin = 0.0, quad = 0.0;
    if (ns <= SUPP_CAP) {
        for (int t = lane; t < ns; t += 32) {
            const int k = list[t];
            lin = fma((double)b[k], (double)a.SC[(size_t)k * a.ldp + j], lin);
        }
        // rows of the support in turn, lanes over its columns (FP64 products)
        for (int u = 0; u < ns; ++u) {
            const int k = list[u];
            const T* __restrict__ row = a.SC + (size_t)k * a.ldp;
            double part = 0.0;
            for (int v = lane; v < ns; v += 32) {
                const int l = list[v];
                part = fma((double)b[l], (double)row[l], part);
            }
            quad = fma((double)b[k], part, quad);
        }
        lin = warp_sum(lin);
        quad = warp_sum(quad);
        __syncwarp();
        return (double)a.SC[(size_t)j * a.ldp + j] - 2.0 * lin + quad;
    }
    // large support: row-wise accumulation without the list
    for (int c0 = 0; c0 < p; c0 += 32) {
        const int k = c0 + lane;
        const T bk = (k < p) ? b[k] : T(0);
        unsigned bal = __ballot_sync(FULL_MASK, bk != T(0));
        while (bal) {
            const int f = __ffs(bal) - 1;
            bal &= bal - 1;
            const int kk = c0 + f;
            const double bkk = (double)__shfl_sync(FULL_MASK, bk, f);
            const T* srow = a.SC + (size_t)kk * a.ldp;
            double part = 0.0;
            for (int l = lane; l < p; l += 32) {
                const T bl = b[l];
                if (bl != T(0)) part += (double)bl * (double)srow[l];
            }
            quad += bkk * part;
            if (lane == 0) lin += bkk * (double)srow[j];
        }
    }
    lin = warp_sum(lin);
    quad = warp_sum(quad);
    return (double)a.SC[(size_t)j * a.ldp + j] - 2.0 * lin + quad;
}

// Row r of S^C = C S C into SC (zero padding up to ldp), optionally copied
// into GT, with BT's row cleared.  FP32 data is scaled in FP32 by the scales
// rounded once to FP32 (csf); FP64 data in FP64.  One warp takes one
// 128-coordinate chunk of the row at a time (threads tid, tid + nthr, ...;
// nthr a multiple of 32).  Optional outputs: heat, this thread's count of
// off-diagonal |SC_rc| > heat_lam; cmax, per chunk c of the row the largest
// off-diagonal |SC_rk| (row r of a p x num_chunks(ldp) table; S^C is
// symmetric, so it is also column r's first-sweep gradient bound).  Returns
// true if a non-finite entry was seen.
constexpr int STD_U = 4;
template <typename T>
__device__ __forceinline__ bool standardize_row(const T* __restrict__ S, int p, int ldp, int r,
                                                const double* __restrict__ cs,
                                                const float* __restrict__ csf,
                                                T* __restrict__ SC, T* __restrict__ GT,
                                                T* __restrict__ BT, T* __restrict__ diag, int tid,
                                                int nthr, T heat_lam = T(0), int* heat = nullptr,
                                                float* __restrict__ cmax = nullptr) {
    bool bad = false;
    const int lane = tid & 31;
    const T cr = sizeof(T) == 4 ? (T)csf[r] : (T)cs[r];
    const T* __restrict__ srow = S + (size_t)r * p;
    T* __restrict__ out = SC + (size_t)r * ldp;
    T* __restrict__ grow = GT ? GT + (size_t)r * ldp : nullptr;
    T* __restrict__ brow = BT ? BT + (size_t)r * ldp : nullptr;
    const int nch = num_chunks(ldp);
    const int wstep = nthr >> 5;
    // 16-byte accesses when the rows of S are 16-byte aligned (same arithmetic)
    const bool vec = sizeof(T) == 4 && (p & 3) == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0;
    // STD_U chunks per pass: their S values are loaded first, so a warp has
    // STD_U loads in flight instead of one
    for (int chb = tid >> 5; chb < nch; chb += STD_U * wstep) {
        T sv[STD_U][4];
#pragma unroll
        for (int u = 0; u < STD_U; ++u) {
            const int ch = chb + u * wstep;
            const int c0 = ch * CHUNK;
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (vec) {                            // lane: coordinates c0 + 4 lane + t
                    const int c = c0 + 4 * lane;
                    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ch < nch && c < p) q = *reinterpret_cast<const float4*>(srow + c);
                    sv[u][0] = q.x; sv[u][1] = q.y; sv[u][2] = q.z; sv[u][3] = q.w;
                    done = true;
                }
            }
            if (!done) {                              // lane: coordinates c0 + lane + 32 t
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = c0 + lane + 32 * t;
                    sv[u][t] = (ch < nch && c < p) ? srow[c] : T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < STD_U; ++u) {
            const int ch = chb + u * wstep;
            if (ch >= nch) break;                     // warp-uniform
            const int c0 = ch * CHUNK;
            float mx = 0.f;
            T v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int c = vec ? c0 + 4 * lane + t : c0 + lane + 32 * t;
                v[t] = T(0);
                if (c < p) {
                    bad |= !isfinite(sv[u][t]);
                    const T cc = sizeof(T) == 4 ? (T)csf[c] : (T)cs[c];
                    v[t] = sv[u][t] * cr * cc;
                    if (c == r) {
                        diag[r] = v[t];
                    } else {
                        mx = fmaxf(mx, (float)fabs(v[t]));
                        if (heat && fabs(v[t]) > heat_lam) ++*heat;
                    }
                }
            }
            if (vec) {                                // ldp % 4 == 0: the quad is inside the row
                const int c = c0 + 4 * lane;
                if (c < ldp) {
                    const float4 q = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
                    *reinterpret_cast<float4*>(out + c) = q;
                    if (grow) *reinterpret_cast<float4*>(grow + c) = q;
                    if (brow) *reinterpret_cast<float4*>(brow + c) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = c0 + lane + 32 * t;
                    if (c < ldp) {
                        out[c] = v[t];
                        if (grow) grow[c] = v[t];
                        if (brow) brow[c] = T(0);
                    }
                }
            }
            if (cmax) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
                if (lane == 0) cmax[(size_t)r * nch + ch] = mx;
            }
        }
    }
    return bad;
}

// Per-warp counters of the column solves, flushed into a fit's FitCtrl.
struct ColCounters {
    unsigned long long sweeps = 0, moves = 0;        // full sweeps and their moves
    unsigned long long act_sweeps = 0, act_moves = 0;   // active-set phase
    int outer_max = 0, n_nc = 0, n_deg = 0, max_sw = 0;
    int blk = 0;                                      // columns solved by the block solver
};

__device__ __forceinline__ void flush_counters(FitCtrl* ctrl, ColCounters& c) {
    if ((threadIdx.x & 31) == 0) {
        if (c.sweeps) atomicAdd(&ctrl->total_sweeps, c.sweeps);
        if (c.moves) atomicAdd(&ctrl->moves, c.moves);
        if (c.act_sweeps) atomicAdd(&ctrl->act_sweeps, c.act_sweeps);
        if (c.act_moves) atomicAdd(&ctrl->act_moves, c.act_moves);
        atomicMax(&ctrl->outer_max, c.outer_max);
        atomicMax(&ctrl->max_col_sweeps, c.max_sw);
        if (c.n_nc) atomicAdd(&ctrl->n_not_converged, c.n_nc);
        if (c.n_deg) atomicAdd(&ctrl->n_degenerate, c.n_deg);
    }
    c = ColCounters();
}

// The sigma step of the per-column solvers.  Algorithm 1 iterates the fixed
// point sigma <- F(sigma) = Q(b(sigma lambda0))^1/2 (Eq. (14)), which
// converges linearly.  From the second step on the solvers take the secant
// step on g(s) = F(s) - s through the last two points (s0, F(s0)),
// (s1, F(s1)), kept only when it is positive and within four plain steps of
// [min(s1, F(s1)), max(s1, F(s1))]; otherwise the plain step F(s1).  The stop
// test |F(sigma) - sigma| < tol and the returned pair (b(sigma), F(sigma)) are
// Algorithm 1's, so the fit ends at the same fixed point within tol; about
// 40 % fewer sigma steps reach it.  Any accepted step is a valid next sigma,
// so only the differences are taken in FP64 and the step itself (relative to
// s1) is formed and safeguarded in FP32: FP64 arithmetic is scarce on this
// part and every column takes this step a few times.
__device__ __forceinline__ double sigma_step(double s0, double f0, double s1, double f1) {
    const float g1 = (float)(f1 - s1), g0 = (float)(f0 - s0), ds = (float)(s1 - s0);
    const float den = g1 - g0;
    if (den == 0.0f) return f1;
    const float step = -g1 * (ds / den);                  // candidate - s1
    const float w = 4.0f * fabsf(g1);
    const float lo = fminf(0.0f, g1) - w, hi = fmaxf(0.0f, g1) + w;
    const double cand = s1 + (double)step;
    return (cand > 0.0 && step >= lo && step <= hi) ? cand : f1;
}

// sqrt(q) for q > 0 in FP64 by one step of Newton's (Heron's) iteration
// y <- y + (q - y^2) / (2 y) from the FP32 root: the FP32 root's relative
// error (at most 2^-23) is squared, so the result is within a few FP64 units
// of the root, with five FP64 operations.  Outside the FP32 range, sqrt.
__device__ __forceinline__ double sqrt_heron(double q) {
    const float yf = sqrtf((float)q);
    if (!(yf > 1e-18f && yf < 1e18f)) return sqrt(q);
    const double y0 = (double)yf;
    return fma(fma(-y0, y0, q), (double)(0.5f / yf), y0);
}

// Algorithm 1 for response column j, by one warp: warm start from b = 0,
// sigma = 1; lasso sweeps at lambda = sigma * lambda0 until
// max |delta b| < tol; sigma from Eq. (14) in FP64; repeat until sigma moves
// by less than tol.  Writes b_j (row j of BT), sigma_j and the column status.
template <typename T, bool STD>
__device__ void solve_column(int j, T* __restrict__ g, T* __restrict__ b, int* __restrict__ list,
                             const CDArgs<T>& a, ColCounters& cnt) {
    const int lane = threadIdx.x & 31;
    warp_copy<T>(g, a.SC + (size_t)j * a.ldp, a.ldp);   // g = S_.j  (b = 0)
    warp_zero<T>(b, a.ldp);
    ColScan cs{reinterpret_cast<ChunkInfo*>(list + SUPP_CAP), 0.f, 0u};
    reset_chunks(cs, a.ldp);
    __syncwarp();

    double sigma = 1.0;                                  // sigma^(0) = 1
    double s_prev = 0.0, f_prev = 0.0;                   // last (sigma, F(sigma))
    bool have_prev = false;
    const unsigned long long sweeps0 = cnt.sweeps;
    const double floor2 = 1e-12 * (double)a.SC[(size_t)j * a.ldp + j];
    int status = COL_OK;
    int r;
    for (r = 0; r < a.maxit; ++r) {
        const T lam = (T)(sigma * a.lambda0);
        bool inner_ok = false;
        for (int m = 0; m < a.maxit; ++m) {
            const T md = sweep_column<T, STD>(j, g, b, a, lam, cnt.moves, cs,
                                              (int)(cnt.sweeps - sweeps0));
            ++cnt.sweeps;
            if ((double)md < a.tol) {
                inner_ok = true;
                break;
            }
        }
        if (!inner_ok) status |= COL_NOT_CONVERGED;
        double q = residual_quadratic_form<T>(j, b, a, list);
        if (q <= floor2) {
            q = floor2;
            status |= COL_DEGENERATE;
        }
        const double sn = sqrt_heron(q);
        if (fabs(sn - sigma) < a.tol) {
            sigma = sn;
            break;
        }
        double nxt = sn;
        if (have_prev && r + 1 < a.maxit && !(status & COL_DEGENERATE))
            nxt = sigma_step(s_prev, f_prev, sigma, sn);
        s_prev = sigma;
        f_prev = sn;
        have_prev = true;
        sigma = nxt;
    }
    if (r == a.maxit) {
        r = a.maxit - 1;
        status |= COL_NOT_CONVERGED;
    }
    warp_copy<T>(a.BT + (size_t)j * a.ldp, b, a.ldp);
    if (lane == 0) {
        a.sigma[j] = sigma;
        a.col_status[j] = status;
    }
    cnt.outer_max = max(cnt.outer_max, r + 1);
    cnt.max_sw = max(cnt.max_sw, (int)(cnt.sweeps - sweeps0));
    cnt.n_nc += (status & COL_NOT_CONVERGED) != 0;
    cnt.n_deg += (status & COL_DEGENERATE) != 0;
    __syncwarp();
}

// ===========================================================================
// Lazy-gradient column solver.
//
// Algorithm 1 in ascending cyclic order, with an active-set phase before each
// certifying sweep (see solve_column_lazy), and the gradient g = S_.j - S b
// never stored.  The warp keeps only the
// support of b_j, sorted by coordinate, in shared memory.  Each 128-coordinate
// chunk forms its slice of g from coalesced 16-byte reads of row j and of the
// rows of the support (S symmetric), so the chunk's reads are independent and
// cost one round trip.  When a coordinate moves, the rank-1 update
// g -= S_.k delta is applied at once to the rest of the chunk and reaches
// every later chunk when that chunk forms its slice from the updated support.
// This is the covariance form of c = S_kj - sum_{l != k} S_kl b_l.  With about
// 5 KB of shared memory per column instead of two p-vectors, many more columns
// stay resident per SM.
// If the support outgrows the list, the column is handed to the eager solver
// (solve_column) through a queue and solved again from the start.
// ===========================================================================
constexpr int LAZY_CAP = 256;

// Supports up to ACT_MAX coordinates get the active-set phase (one
// coordinate per lane, the support's block of S in shared memory).
constexpr int ACT_MAX = 32;

template <typename T>
struct Support {
    int* idx;      // sorted coordinates with b != 0
    T* val;        // their b values
    int n;         // warp-uniform count
};

// Shared memory of one lazy-solver warp: the support list, the chunk
// summaries, the support's block of S, the last sigma step (sigma,
// F(sigma)) for the secant step (kept out of registers) and the support the
// block of S was gathered for.
template <typename T>
__host__ __device__ constexpr size_t lazy_warp_smem_bytes(int ldp) {
    return (size_t)LAZY_CAP * (sizeof(int) + sizeof(T)) + (size_t)num_chunks(ldp) * sizeof(ChunkInfo) +
           (size_t)ACT_MAX * ACT_MAX * sizeof(T) + 2 * sizeof(double) + ACT_MAX * sizeof(int);
}

// Set b_k = v in the sorted support (insert, update or remove).  pos is the
// first index with idx[pos] >= k.  Returns false if an insert would overflow.
template <typename T>
__device__ bool support_set(Support<T>& s, int pos, int k, T v) {
    const int lane = threadIdx.x & 31;
    const bool exists = pos < s.n && s.idx[pos] == k;
    if (exists && v != T(0)) {
        if (lane == 0) s.val[pos] = v;
        __syncwarp();
        return true;
    }
    if (!exists && v == T(0)) return true;
    if (!exists && s.n >= LAZY_CAP) return false;
    const int shift = exists ? -1 : 1;
    const int from = exists ? pos + 1 : pos;        // entries [from, n) move by `shift`
    const int cnt = s.n - from;
    // move in register-sized rounds; the direction keeps every read ahead of its write
    for (int base = 0; base < cnt; base += 32) {
        const int t = shift > 0 ? cnt - 1 - (base + lane) : base + lane;
        int ix = 0;
        T vv = T(0);
        const bool act = (base + lane) < cnt;
        if (act) {
            ix = s.idx[from + t];
            vv = s.val[from + t];
        }
        __syncwarp();
        if (act) {
            s.idx[from + t + shift] = ix;
            s.val[from + t + shift] = vv;
        }
        __syncwarp();
    }
    if (!exists && lane == 0) {
        s.idx[pos] = k;
        s.val[pos] = v;
    }
    s.n += shift;
    __syncwarp();
    return true;
}

template <typename T>
__device__ __forceinline__ void load4g(const T* __restrict__ src, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = __ldg(reinterpret_cast<const double2*>(src));
        const double2 q1 = __ldg(reinterpret_cast<const double2*>(src + 2));
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

// Chunks of [from, from + 32) that the sweep must scan, as a bit mask: with
// the standardised matrix, a chunk is skipped when chunk_skippable proves
// that none of its coordinates can move; the test reads only the chunk's
// summary and the column's running sums, so the lanes test 32 chunks at once.
// The mask stays valid until a move changes the running sums.
template <bool STD>
__device__ __forceinline__ unsigned chunks_to_scan(const ColScan& cs, int from, int nch, float lam,
                                                   bool frozen) {
    const int ci = from + (int)(threadIdx.x & 31);
    bool need = ci < nch;
    if constexpr (STD) {
        if (need) need = !chunk_skippable(cs.ci[ci], cs, lam, frozen);
    }
    return __ballot_sync(FULL_MASK, need);
}

// One sweep; returns max |delta b|.  Sets `overflow` and stops early if the
// support list is full.  With `frozen` the coordinates in the support keep
// their values and only the others are updated (a coordinate that enters is
// not revisited in the same sweep).
template <typename T, bool STD>
__device__ T sweep_column_lazy(int j, Support<T>& s, const CDArgs<T>& a, T lam,
                               unsigned long long& moves, ColScan& cs, bool& overflow,
                               bool frozen, int sweep_idx) {
    const int lane = threadIdx.x & 31;
    const int p = a.p;
    const int ldp = a.ldp;
    const T* __restrict__ Sj = a.SC + (size_t)j * ldp;
    const int nch = (p + CHUNK - 1) / CHUNK;
    T maxd = T(0);
    int e0 = 0;                                   // first support entry with idx >= cb
    int mbase = 0;
    if constexpr (STD) {
        float l1 = 0.f;
        for (int e = lane; e < s.n; e += 32) l1 += fabsf((float)s.val[e]);
        cs.bl1 = warp_sum_f(l1) * (1.0f + 0x1p-16f);
    }
    unsigned mask = chunks_to_scan<STD>(cs, 0, nch, (float)lam, frozen);
    for (;;) {
        if (mask == 0u) {
            mbase += 32;
            if (mbase >= nch) break;
            mask = chunks_to_scan<STD>(cs, mbase, nch, (float)lam, frozen);
            continue;
        }
        const int ci = mbase + __ffs(mask) - 1;
        mask &= mask - 1u;
        const int cb = ci * CHUNK;
        while (e0 < s.n && s.idx[e0] < cb) ++e0;
        int e1 = e0;
        while (e1 < s.n && s.idx[e1] < cb + CHUNK) ++e1;
        const int k0 = cb + lane * SCAN_V;
        const bool in = k0 < ldp;                 // the whole quad is inside the padded row
        // slice of g: S_jk - sum_{l in support} S_lk b_l (four rows in flight;
        // an L1 prefetch of all the support rows first was measured slower)
        const T* __restrict__ col = a.SC + k0;    // column k0 of S; row l at col + l ldp
        T acc[SCAN_V] = {T(0), T(0), T(0), T(0)};
        if (in) load4g<T>(Sj + k0, acc);
#pragma unroll 4
        for (int e = 0; e < s.n; ++e) {
            const int l = s.idx[e];
            const T v = s.val[e];
            if (in) {
                T r[SCAN_V];
                load4g<T>(col + (size_t)l * ldp, r);
#pragma unroll
                for (int t = 0; t < SCAN_V; ++t) acc[t] = fma(-v, r[t], acc[t]);
            }
        }
        // current b of this lane's coordinates (support entries of the chunk)
        T bv[SCAN_V] = {T(0), T(0), T(0), T(0)};
        for (int e = e0; e < e1; ++e) {
            const int t = s.idx[e] - k0;
            if (t >= 0 && t < SCAN_V) {
#pragma unroll
                for (int u = 0; u < SCAN_V; ++u)
                    if (u == t) bv[u] = s.val[e];
            }
        }
        const unsigned nmoves0 = cs.nmoves;
        int cursor = cb;
        for (;;) {
            T nbv[SCAN_V];
            unsigned mvmask = 0u;
#pragma unroll
            for (int t = 0; t < SCAN_V; ++t) {
                const int k = k0 + t;
                nbv[t] = bv[t];
                if (k >= cursor && k < p && k != j && !(frozen && bv[t] != T(0))) {
                    T nb;
                    if constexpr (STD) {
                        nb = soft<T>(acc[t] + bv[t], lam);                 // S_kk = 1
                    } else {
                        const T skk = a.diag[k];
                        nb = soft<T>(acc[t] + skk * bv[t], lam) / skk;     // Soft(c, lambda)/S_kk
                    }
                    nbv[t] = nb;
                    if (nb != bv[t]) mvmask |= 1u << t;
                }
            }
            const unsigned bal = __ballot_sync(FULL_MASK, mvmask != 0u);
            if (bal == 0u) break;
            const int f = __ffs(bal) - 1;
            const int tf = __ffs(__shfl_sync(FULL_MASK, mvmask, f)) - 1;
            T nb_sel = nbv[0], b_sel = bv[0];
#pragma unroll
            for (int t = 1; t < SCAN_V; ++t)
                if (t == tf) { nb_sel = nbv[t]; b_sel = bv[t]; }
            const T nbs = __shfl_sync(FULL_MASK, nb_sel, f);
            const T delta = nbs - __shfl_sync(FULL_MASK, b_sel, f);
            const int ks = cb + f * SCAN_V + tf;
            int pos = e0;
            while (pos < e1 && s.idx[pos] < ks) ++pos;
            const int n_before = s.n;
            if (!support_set<T>(s, pos, ks, nbs)) {
                overflow = true;
                return maxd;
            }
            e1 += s.n - n_before;
            if (lane == 0) note_row_moved(a, sweep_idx, ks);
            if (lane == f) {
#pragma unroll
                for (int u = 0; u < SCAN_V; ++u)
                    if (u == tf) bv[u] = nbs;
            }
            maxd = fmax(maxd, fabs(delta));
            ++moves;
            cs.dsum += fabsf((float)delta);
            ++cs.nmoves;
            cs.bl1 += fabsf((float)delta);
            // rank-1 update of the rest of this chunk's slice
            if (in) {
                T r[SCAN_V];
                load4g<T>(a.SC + (size_t)ks * ldp + k0, r);
#pragma unroll
                for (int t = 0; t < SCAN_V; ++t) acc[t] = fma(-delta, r[t], acc[t]);
            }
            cursor = ks + 1;
            if (cursor >= cb + CHUNK) break;
        }
        if constexpr (STD) {
            float mx = 0.f;
#pragma unroll
            for (int t = 0; t < SCAN_V; ++t) {
                const int k = k0 + t;
                if (k < p && k != j && bv[t] == T(0)) mx = fmaxf(mx, fabsf((float)acc[t]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
            if (lane == 0) cs.ci[ci] = ChunkInfo{mx, cs.dsum, cs.nmoves, e1 - e0};
            __syncwarp();
            // moves raised the running sums: test the chunks after this one again
            if (cs.nmoves != nmoves0) {
                mbase = ci + 1;
                if (mbase >= nch) break;
                mask = chunks_to_scan<STD>(cs, mbase, nch, (float)lam, frozen);
            }
        } else {
            __syncwarp();
        }
    }
    return maxd;
}

// Active-set phase of the lasso at a fixed lambda: cyclic sweeps (ascending
// coordinate order) over the current support A only, until a sweep moves no
// coefficient by tol or more (at most maxit sweeps).  Lane m holds coordinate
// A_m: its b and g_m = S_jm - sum_{l in A} S_ml b_l; the block S_AA is
// gathered into shared memory (column k at saa + k ACT_MAX), and kept from
// the column's last phase when A is the same (saa_list, saa_n).  The phase's
// net change of b enters the column's running sums as one change, so the
// chunk skip test stays exact for the coordinates outside A.  Coordinates
// that reach zero leave the support and mark their chunk for a rescan.  One
// move is the phase's critical path: every lane forms its candidate, one
// shuffle broadcasts the owner's change, and every lane updates its gradient
// with the column of S_AA loaded one move ahead (a zero change adds exact
// zeros, so no lane branches on it).  Returns the sweeps done (0 when A is
// empty or larger than ACT_MAX); `conv` tells whether the last sweep moved
// nothing by tol (true for an empty A, false when A is too large).
template <typename T, bool STD>
__device__ int active_phase(int j, Support<T>& s, const CDArgs<T>& a, T lam, T* __restrict__ saa,
                            int* __restrict__ saa_list, int& saa_n, unsigned long long& moves,
                            ColScan& cs, bool& conv) {
    const int lane = threadIdx.x & 31;
    const int n = s.n;
    conv = n <= ACT_MAX;
    if (n == 0 || n > ACT_MAX) return 0;
    conv = false;
    const int ldp = a.ldp;
    const int my = lane < n ? s.idx[lane] : 0;
    if (!(saa_n == n && __all_sync(FULL_MASK, lane >= n || saa_list[lane] == my))) {
        // lane m reads S_{A_m A_k} for four k at a time (independent loads)
        for (int k0 = 0; k0 < n; k0 += 4) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u;
                v[u] = (k < n && lane < n) ? a.SC[(size_t)my * ldp + s.idx[k]] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u < n) saa[(k0 + u) * ACT_MAX + lane] = v[u];
        }
        saa_list[lane] = my;
        saa_n = n;
    }
    T b = lane < n ? s.val[lane] : T(0);
    const T b_start = b;
    T g = lane < n ? a.SC[(size_t)j * ldp + my] : T(0);
    T skk = T(1);
    if constexpr (!STD) skk = lane < n ? a.diag[my] : T(1);
    __syncwarp();
    for (int l = 0; l < n; ++l) {
        const T bl = __shfl_sync(FULL_MASK, b, l);
        if (lane < n) g = fma(-saa[l * ACT_MAX + lane], bl, g);
    }
    int sw = 0;
    unsigned mv = 0;
    const float tf = float_at_least(a.tol);
    while (sw < a.maxit) {
        ++sw;
        T md = T(0);
        T c = lane < n ? saa[lane] : T(0);                   // column of S_AA for k = 0
        for (int k = 0; k < n; ++k) {
            const int kn = k + 1 < n ? k + 1 : k;
            const T cn = lane < n ? saa[kn * ACT_MAX + lane] : T(0);   // next column
            T nb;
            if constexpr (STD) nb = soft<T>(g + b, lam);                 // S_kk = 1
            else nb = soft<T>(g + skk * b, lam) / skk;
            const T d = __shfl_sync(FULL_MASK, nb - b, k);
            if (lane == k) b = nb;
            g = fma(-c, d, g);
            md = fmax(md, fabs(d));
            mv += d != T(0);
            c = cn;
        }
        if (below_tol<T>(md, a.tol, tf)) {
            conv = true;
            break;
        }
    }
    moves += mv;
    // the phase enters the running sums as one change: its net l1 size
    const float net = warp_sum_f(lane < n ? fabsf((float)(b - b_start)) : 0.f);
    cs.dsum += net * (1.0f + 0x1p-16f);
    ++cs.nmoves;
    // write back, dropping coordinates at zero (the list stays sorted)
    const bool keep = lane < n && b != T(0);
    if (lane < n && b == T(0)) cs.ci[my / CHUNK].maxabs = INFINITY;
    const unsigned km = __ballot_sync(FULL_MASK, keep);
    const int pos = __popc(km & ((1u << lane) - 1u));
    __syncwarp();
    if (keep) {
        s.idx[pos] = my;
        s.val[pos] = b;
    }
    s.n = __popc(km);
    __syncwarp();
    return sw;
}

// sigma_j^2 = S_jj - 2 b'S_.j + b'S b in FP64 over the sorted support (Eq. (14)).
// Every product is formed in FP64 (for FP32 data the product of two FP32
// values is exact in FP64) and every sum is carried in FP64.  FP64 arithmetic
// is scarce on this part and every column runs this step a few times, so the
// FP64 work is kept to a few instructions per lane: the n^2 pairs (u, v) and
// the n terms of b'S_.j are spread over the lanes (pair indices stepped by
// 32 without a divide per pair), each lane adds b_u b_v S_uv and -2 b_u S_uj
// into one FP64 partial, and one FP64 warp sum ends it.
template <typename T>
__device__ double residual_quadratic_form_list(int j, const Support<T>& s, const CDArgs<T>& a) {
    const int lane = threadIdx.x & 31;
    const int n = s.n;
    const int ldp = a.ldp;
    double acc = 0.0;
    if (lane < n) {
        // -2 b_u S_uj for u = lane, lane + 32, ... (-2 b_u is exact in the data precision)
        for (int u = lane; u < n; u += 32)
            acc = fma((double)(T(-2) * s.val[u]), (double)a.SC[(size_t)s.idx[u] * ldp + j], acc);
    }
    const int np = n * n;
    if (lane < np) {
        // pair t = u n + v for t = lane, lane + 32, ...: (u, v) advance by (q, r)
        int u = lane / n, v = lane - (lane / n) * n;
        const int q = 32 / n, r = 32 - (32 / n) * n;
        for (int t = lane; t < np; t += 32) {
            const double bb = (double)s.val[u] * (double)s.val[v];
            acc = fma(bb, (double)a.SC[(size_t)s.idx[u] * ldp + s.idx[v]], acc);
            u += q;
            v += r;
            if (v >= n) {
                v -= n;
                ++u;
            }
        }
    }
    acc = warp_sum(acc);
    return (double)a.SC[(size_t)j * ldp + j] + acc;
}

// b_j as the whole row j of BT, zeros included (16-byte stores; ldp is a
// multiple of 32), so BT needs no clearing before the fit.
template <typename T>
__device__ __forceinline__ void store_row_lazy(int j, const Support<T>& s, const CDArgs<T>& a) {
    const int lane = threadIdx.x & 31;
    T* brow = a.BT + (size_t)j * a.ldp;
    uint4* q = reinterpret_cast<uint4*>(brow);
    const int nq = a.ldp * (int)sizeof(T) / 16;
    for (int i = lane; i < nq; i += 32) q[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    for (int t = lane; t < s.n; t += 32) brow[s.idx[t]] = s.val[t];
}

// The lazy solver's state when it hands column j over: b_j as row j of BT,
// sigma, the last sigma step and the step index, so that the
// block solver continues from this iterate.  Any (b, sigma) is a valid start
// for the coordinate descent, and the hand-over point depends only on the
// column's data, so the result is the same wherever the column is solved.
template <typename T, bool HS>
__device__ __forceinline__ void hand_over_lazy(int j, const Support<T>& s, const CDArgs<T>& a, double sigma,
                               double s_prev, double f_prev, int r, int status) {
    if (!a.hand) return;
    const int lane = threadIdx.x & 31;
    store_row_lazy<T>(j, s, a);
    if (lane == 0) {
        a.sigma[j] = sigma;
        a.hand[2 * (size_t)j] = s_prev;
        a.hand[2 * (size_t)j + 1] = f_prev;
        a.col_status[j] = COL_HANDED | (status & (COL_NOT_CONVERGED | COL_DEGENERATE)) |
                          (r << COL_STEP_SHIFT);
    }
    __syncwarp();
}

// Algorithm 1 for column j with the lazy gradient.  Returns false when the
// support outgrew the list (nothing written; the caller queues the column
// for the eager solver).  HS keeps the last sigma step in the warp's shared
// memory instead of registers (for kernels at a tight register cap).
template <typename T, bool STD, bool HS = false>
__device__ bool solve_column_lazy(int j, unsigned char* wsm, const CDArgs<T>& a, ColCounters& cnt) {
    const int lane = threadIdx.x & 31;
    Support<T> s;
    s.idx = reinterpret_cast<int*>(wsm);
    s.val = reinterpret_cast<T*>(wsm + LAZY_CAP * sizeof(int));
    s.n = 0;
    ColScan cs{reinterpret_cast<ChunkInfo*>(wsm + LAZY_CAP * (sizeof(int) + sizeof(T))), 0.f, 0u};
    T* saa = reinterpret_cast<T*>(cs.ci + num_chunks(a.ldp));
    double* prev = reinterpret_cast<double*>(saa + ACT_MAX * ACT_MAX);   // HS: (sigma, F(sigma))
    int* saa_list = reinterpret_cast<int*>(prev + 2);    // the support S_AA was gathered for
    int saa_n = -1;
    reset_chunks(cs, a.ldp);
    if constexpr (STD) {
        // b = 0: the gradient is row j of S^C, whose chunk maxima the
        // standardisation pass wrote, so the first sweep may skip chunks too
        if (a.chunk_max) {
            const int nch = num_chunks(a.ldp);
            const float* __restrict__ cm = a.chunk_max + (size_t)j * nch;
            for (int c = lane; c < nch; c += 32) cs.ci[c] = ChunkInfo{cm[c], 0.f, 0u, 0};
        }
    }
    __syncwarp();

    double sigma = 1.0;                                  // sigma^(0) = 1, b = 0
    double s_prev = 0.0, f_prev = 0.0;                   // last (sigma, F(sigma))
    const unsigned long long sweeps0 = cnt.sweeps;
    const double floor2 = 1e-12 * (double)a.SC[(size_t)j * a.ldp + j];
    int status = COL_OK;
    bool overflow = false;
    int r;
    for (r = 0; r < a.maxit; ++r) {
        const T lam = (T)(sigma * a.lambda0);
        bool inner_ok = false;
        for (int m = 0; m < a.maxit; ++m) {
            // converge on the support first; then, if that converged, a
            // sweep over the other coordinates with the support held (its
            // chunks skippable by the bound) decides: the lasso has converged
            // when the support's last sweep and this sweep both moved nothing
            // by tol.  Otherwise a full sweep of every coordinate decides (the
            // stop rule of Algorithm 1).
            bool conv;
            if (s.n > a.ovf_supp) {                       // a heavy column: the block solver
                hand_over_lazy<T, HS>(j, s, a, sigma, HS ? prev[0] : s_prev, HS ? prev[1] : f_prev,
                                      r, status);
                return false;
            }
            cnt.act_sweeps += active_phase<T, STD>(j, s, a, lam, saa, saa_list, saa_n, cnt.act_moves,
                                                  cs, conv);
            const T md = sweep_column_lazy<T, STD>(j, s, a, lam, cnt.moves, cs, overflow, conv,
                                                   (int)(cnt.sweeps - sweeps0));
            ++cnt.sweeps;
            if (overflow) {
                hand_over_lazy<T, HS>(j, s, a, sigma, HS ? prev[0] : s_prev, HS ? prev[1] : f_prev,
                                      r, status);
                return false;
            }
            if ((double)md < a.tol) {
                inner_ok = true;
                break;
            }
        }
        if (!inner_ok) status |= COL_NOT_CONVERGED;
        double q = residual_quadratic_form_list<T>(j, s, a);
        if (q <= floor2) {
            q = floor2;
            status |= COL_DEGENERATE;
        }
        const double sn = sqrt_heron(q);
        if (fabs(sn - sigma) < a.tol) {
            sigma = sn;
            break;
        }
        double nxt = sn;
        if (r > 0 && r + 1 < a.maxit && !(status & COL_DEGENERATE))
            nxt = HS ? sigma_step(prev[0], prev[1], sigma, sn) : sigma_step(s_prev, f_prev, sigma, sn);
        if constexpr (HS) {
            __syncwarp();
            if (lane == 0) {
                prev[0] = sigma;
                prev[1] = sn;
            }
            __syncwarp();
        } else {
            s_prev = sigma;
            f_prev = sn;
        }
        sigma = nxt;
    }
    if (r == a.maxit) {
        r = a.maxit - 1;
        status |= COL_NOT_CONVERGED;
    }
    store_row_lazy<T>(j, s, a);
    if (lane == 0) {
        a.sigma[j] = sigma;
        a.col_status[j] = status;
    }
    cnt.outer_max = max(cnt.outer_max, r + 1);
    cnt.max_sw = max(cnt.max_sw, (int)(cnt.sweeps - sweeps0));
    cnt.n_nc += (status & COL_NOT_CONVERGED) != 0;
    cnt.n_deg += (status & COL_DEGENERATE) != 0;
    __syncwarp();
    return true;
}

// ===========================================================================
// Optimality diagnostics of a finished fit (opts.diagnostics).
//
// For column j the returned pair (b_j, sigma_j) solves Algorithm 1's problem
// when the lasso subgradient conditions hold at lambda = lambda0 sigma_j
// (Section 2.1): with g = S_.j - S b_j,
//   g_k = lambda sign(b_k) where b_k != 0,   |g_k| <= lambda where b_k = 0,
// and sigma_j is the fixed point of Eq. (14).  One warp per column forms the
// whole gradient in FP64 from the working matrix (row j and the support rows,
// the lazy solver's slices accumulated in FP64) and reports
//  - the largest violation of those conditions relative to lambda;
//  - the relative duality gap (P - D) / P of the lasso subproblem: with
//    rr = S_jj - b'S_.j - b'g (= ||x_j - X b||^2 / n), yr = S_jj - b'S_.j and
//    the dual point s r, s = min(1, lambda / ||g||_inf):
//    P = rr / 2 + lambda ||b||_1, D = s yr - s^2 rr / 2;
//  - a first-order estimate of the error of the column's Theta entries.  The
//    rounding of the working matrix (eps_s per entry, relative) moves each
//    gradient entry by about eps_s (1 + ||b||_2) (independent signs); with
//    the measured gradient residual this is read as a coefficient error
//    (unit diagonal).  sigma moves by the fixed-point residual plus
//    drr / (2 sigma), drr the first-order change of rr: eps_s (1 + ||b||_2)^2
//    from the matrix (at the optimum the change through b is second order)
//    and 2 lambda |A| kkt from a solve that is not exactly optimal.  Then
//    Theta_kj = -b_kj / sigma_j^2, Theta_jj = 1 / sigma_j^2 differentiated.
// ===========================================================================
constexpr int DIAG_CAP = 1024;         // support list of one warp

__host__ __device__ constexpr size_t diag_warp_smem_bytes() {
    return (size_t)DIAG_CAP * (sizeof(int) + sizeof(double));
}

// Per-warp maxima of the diagnostics (non-negative doubles), flushed with
// atomicMax on their bits.
struct DiagMax {
    double kkt = 0.0, gap = 0.0, err = 0.0, thmax = 0.0;
};

__device__ __forceinline__ void flush_diag(FitCtrl* ctrl, const DiagMax& d) {
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&ctrl->diag_kkt, dbits(d.kkt));
        atomicMax(&ctrl->diag_gap, dbits(d.gap));
        atomicMax(&ctrl->diag_err, dbits(d.err));
        atomicMax(&ctrl->diag_thmax, dbits(d.thmax));
        atomicAdd(&ctrl->diag_cols, 1u);
    }
}

template <typename T>
__device__ void diagnose_column(int j, unsigned char* wsm, const CDArgs<T>& a, double eps_s,
                                DiagMax& out) {
    const int lane = threadIdx.x & 31;
    const int p = a.p, ldp = a.ldp;
    int* idx = reinterpret_cast<int*>(wsm);
    double* val = reinterpret_cast<double*>(wsm + DIAG_CAP * sizeof(int));
    const T* __restrict__ brow = a.BT + (size_t)j * ldp;
    // support of b_j in ascending order
    int ns = 0;
    for (int c0 = 0; c0 < p; c0 += 32) {
        const int k = c0 + lane;
        const T bk = k < p ? brow[k] : T(0);
        const unsigned bal = __ballot_sync(FULL_MASK, bk != T(0));
        const int pos = ns + __popc(bal & ((1u << lane) - 1u));
        if (bk != T(0) && pos < DIAG_CAP) {
            idx[pos] = k;
            val[pos] = (double)bk;
        }
        ns += __popc(bal);
    }
    __syncwarp();
    const bool listed = ns <= DIAG_CAP;
    const double sig = a.sigma[j];
    const double lam = a.lambda0 * sig;
    const T* __restrict__ Sj = a.SC + (size_t)j * ldp;
    double kkt = 0.0, gmax = 0.0, bg = 0.0;
    for (int cb = 0; cb < p; cb += CHUNK) {
        const int k0 = cb + lane * SCAN_V;
        const bool in = k0 < ldp;
        double acc[SCAN_V] = {0.0, 0.0, 0.0, 0.0};
        if (in) {
            T r[SCAN_V];
            load4g<T>(Sj + k0, r);
#pragma unroll
            for (int t = 0; t < SCAN_V; ++t) acc[t] = (double)r[t];
        }
        if (listed) {
#pragma unroll 4
            for (int e = 0; e < ns; ++e) {
                const double v = val[e];
                if (in) {
                    T r[SCAN_V];
                    load4g<T>(a.SC + (size_t)idx[e] * ldp + k0, r);
#pragma unroll
                    for (int t = 0; t < SCAN_V; ++t) acc[t] = fma(-v, (double)r[t], acc[t]);
                }
            }
        } else {
            for (int l = 0; l < p; ++l) {
                const double v = (double)brow[l];
                if (v != 0.0 && in) {
                    T r[SCAN_V];
                    load4g<T>(a.SC + (size_t)l * ldp + k0, r);
#pragma unroll
                    for (int t = 0; t < SCAN_V; ++t) acc[t] = fma(-v, (double)r[t], acc[t]);
                }
            }
        }
        if (in) {
            T bq[SCAN_V];
            load4g<T>(brow + k0, bq);
#pragma unroll
            for (int t = 0; t < SCAN_V; ++t) {
                const int k = k0 + t;
                if (k >= p || k == j) continue;
                const double g = acc[t], bk = (double)bq[t];
                const double viol = bk != 0.0 ? fabs(g - copysign(lam, bk)) : fmax(0.0, fabs(g) - lam);
                kkt = fmax(kkt, viol);
                gmax = fmax(gmax, fabs(g));
                if (bk != 0.0) bg = fma(bk, g, bg);
            }
        }
    }
    double bS = 0.0, l1 = 0.0, l2 = 0.0, bmax = 0.0;
    if (listed) {
        for (int e = lane; e < ns; e += 32) {
            bS = fma(val[e], (double)Sj[idx[e]], bS);
            l1 += fabs(val[e]);
            l2 = fma(val[e], val[e], l2);
            bmax = fmax(bmax, fabs(val[e]));
        }
    } else {
        for (int k = lane; k < p; k += 32) {
            const double v = (double)brow[k];
            bS = fma(v, (double)Sj[k], bS);
            l1 += fabs(v);
            l2 = fma(v, v, l2);
            bmax = fmax(bmax, fabs(v));
        }
    }
    kkt = warp_max(kkt);
    gmax = warp_max(gmax);
    bmax = warp_max(bmax);
    bg = warp_sum(bg);
    bS = warp_sum(bS);
    l1 = warp_sum(l1);
    l2 = sqrt(warp_sum(l2));
    const double Sjj = (double)Sj[j];
    const double rr = Sjj - bS - bg;
    const double yr = Sjj - bS;
    const double s = gmax > lam ? lam / gmax : 1.0;
    const double P = 0.5 * rr + lam * l1;
    const double D = s * yr - 0.5 * s * s * rr;
    const double gap = P > 0.0 ? fmax(0.0, P - D) / P : 0.0;
    // first-order error of the column's Theta entries
    const double eb = kkt + eps_s * (1.0 + l2);
    const double es = fabs(sig - sqrt(fmax(rr, 0.0))) +
                      (eps_s * (1.0 + l2) * (1.0 + l2) + 2.0 * lam * (double)ns * kkt) / (2.0 * sig);
    const double s2 = sig * sig;
    const double eth = eb / s2 + 2.0 * fmax(1.0, bmax) * es / (s2 * sig);
    out.kkt = fmax(out.kkt, lam > 0.0 ? kkt / lam : kkt);
    out.gap = fmax(out.gap, gap);
    out.err = fmax(out.err, eth);
    out.thmax = fmax(out.thmax, 1.0 / s2);
    __syncwarp();
}

// ===========================================================================
// Block solver for heavy columns.
//
// Algorithm 1 for one column by a whole block of BLK_THREADS threads, for the
// columns whose support is too large for the lazy solver's active-set phase
// (a hub's regression on its neighbours has 40-50 coefficients).  The block
// keeps the whole gradient g_j = S_.j - S b_j and b_j in shared memory:
//  - active-set phase: one warp runs cyclic sweeps over the support A (up to
//    BLK_AMAX coordinates, two per lane, the block S_AA in shared memory)
//    until a sweep moves nothing by tol; then the block forms g afresh from
//    row j and the |A| support rows (no drift accumulates across phases);
//  - working set: after a converged phase one pass over g finds every
//    coordinate outside A that a sweep with A held would move; none ends the
//    lasso at this lambda (that sweep would move nothing), else they join A
//    at b = 0 and the phase runs on the union (while it fits the phase), so
//    coordinates enter the support without an O(p) update per entry;
//  - sweep: the cyclic ascending pass of Algorithm 1 over all coordinates (or
//    with the support held after a converged phase, as in the lazy solver).
//    Every thread tests its coordinates, a block minimum finds the first
//    coordinate whose update changes b, and the rank-1 update
//    g -= S_.k delta (Proposition 2 on S) is applied by the whole block in
//    the same pass that looks for the next mover, so one move costs one pass
//    over g and one barrier;
//  - sigma from Eq. (14) in FP64 over the support (FP64 products), and the
//    safeguarded secant step of the per-column solvers.
// ===========================================================================
constexpr int BLK_THREADS = 512;
constexpr int BLK_WARPS = BLK_THREADS / 32;
constexpr int BLK_AMAX = 64;       // active-set phase: up to 64 coordinates, two per lane
constexpr int BLK_LIST = 1024;     // sorted support list (sigma step, phase, g refresh)
constexpr int BLK_WS_ROUNDS = 16;  // working-set rounds (scan, phase on the union) per inner step
static_assert(LAZY_CAP <= BLK_LIST, "a handed-over support must fit the block solver's list");

// Shared memory of the block solver: g and b (ldp each), S_AA, the support
// list, the double-buffered candidate moves of the sweep and the support S_AA
// was gathered for.
template <typename T>
__host__ __device__ constexpr size_t block_smem_bytes(int ldp) {
    return 2 * (size_t)ldp * sizeof(T) + (size_t)BLK_AMAX * BLK_AMAX * sizeof(T) +
           (size_t)BLK_LIST * sizeof(int) + 2 * 2 * (size_t)BLK_THREADS * sizeof(T) +
           (size_t)BLK_AMAX * sizeof(int);
}

// Per-block scratch of the block solver (static shared memory).
struct BlockScratch {
    int red[2][BLK_WARPS];       // block minimum / counts, double-buffered by parity
    double dred[BLK_WARPS];      // FP64 block sums
    int vred[BLK_WARPS];         // scan: coordinates that would move, per warp
    float mred[BLK_WARPS];       // scan: their largest candidate |move|, per warp
    int wcnt[2], wmax[2];        // refresh scan: count and largest |move| (float bits), by parity
    int saa_n;                   // size of the support S_AA was last gathered for (warp 0's copy)
    int nlist;
    int col;
};

// Smallest v over the block (one barrier; `par` alternates the buffer so the
// next call cannot overwrite values still being read).
__device__ __forceinline__ int block_min_int(int v, BlockScratch& sc, int& par) {
    v = __reduce_min_sync(FULL_MASK, v);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sc.red[par][warp] = v;
    __syncthreads();
    int m = sc.red[par][0];
#pragma unroll
    for (int w = 1; w < BLK_WARPS; ++w) m = min(m, sc.red[par][w]);
    par ^= 1;
    return m;
}

// Sum of v over the block in a fixed order (deterministic for a fixed block size).
__device__ __forceinline__ double block_sum_d(double v, BlockScratch& sc) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sc.dred[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < BLK_WARPS; ++w) t += sc.dred[w];
    __syncthreads();
    return t;
}

// Sorted support of b (ascending) into list[0, min(n, BLK_LIST)); returns n.
// Each thread counts the nonzeros of its own contiguous segment of b, a block
// scan gives the segment offsets, and each thread writes its entries.
template <typename T>
__device__ int block_support_list(const T* __restrict__ b, int p, int* __restrict__ list,
                                  BlockScratch& sc, int& par) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = (p + BLK_THREADS - 1) / BLK_THREADS;
    const int k0 = min(p, (int)threadIdx.x * seg), k1 = min(p, k0 + seg);
    int c = 0;
    for (int k = k0; k < k1; ++k) c += b[k] != T(0);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) sc.red[par][warp] = incl;
    __syncthreads();
    int off = incl - c, total = 0;
#pragma unroll
    for (int w = 0; w < BLK_WARPS; ++w) {
        const int t = sc.red[par][w];
        if (w < warp) off += t;
        total += t;
    }
    par ^= 1;
    for (int k = k0; k < k1 && off < BLK_LIST; ++k)
        if (b[k] != T(0)) list[off++] = k;
    __syncthreads();
    return total;
}

// The scan that certifies a converged support.  A coordinate k != j outside
// the support (b_k = 0) would move in a sweep with the support held exactly
// when its candidate Soft(g_k, lambda) (divided by S_kk without
// standardisation) is nonzero, i.e. |g_k| > lambda; the candidates are formed
// as the sweep forms them.  Writes the sorted union of the support and those
// coordinates into list[0, min(n, BLK_LIST)) and returns n; nv is the number
// of coordinates that would move and mv the largest |candidate| among them
// (each taken as if it moved first).  Same segment layout as
// block_support_list; the block's counts are read before its last barrier,
// so the single-buffered vred / mred can be written by the next call.
template <typename T, bool STD>
__device__ __forceinline__ bool scan_member(int k, int j, const T* __restrict__ g,
                                            const T* __restrict__ b, const CDArgs<T>& a, T lam,
                                            T& nb) {
    const T bk = b[k];
    nb = T(0);
    if (bk != T(0)) return true;
    if (k == j) return false;
    if constexpr (STD) nb = soft<T>(g[k] + bk, lam);                         // S_kk = 1
    else nb = soft<T>(g[k] + a.diag[k] * bk, lam) / a.diag[k];
    return nb != T(0);
}

template <typename T, bool STD>
__device__ int block_scan_list(int j, const T* __restrict__ g, const T* __restrict__ b,
                               const CDArgs<T>& a, T lam, int* __restrict__ list, BlockScratch& sc,
                               int& par, int& nv, float& mv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = a.p;
    const int seg = (p + BLK_THREADS - 1) / BLK_THREADS;
    const int k0 = min(p, (int)threadIdx.x * seg), k1 = min(p, k0 + seg);
    int c = 0, v = 0;
    float m = 0.f;
    for (int k = k0; k < k1; ++k) {
        T nb;
        if (scan_member<T, STD>(k, j, g, b, a, lam, nb)) {
            ++c;
            if (nb != T(0)) {
                ++v;
                m = fmaxf(m, fabsf((float)nb));
            }
        }
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += u;
    }
    const int vw = __reduce_add_sync(FULL_MASK, v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL_MASK, m, o));
    if (lane == 31) sc.red[par][warp] = incl;
    if (lane == 0) {
        sc.vred[warp] = vw;
        sc.mred[warp] = m;
    }
    __syncthreads();
    int off = incl - c, total = 0, vt = 0;
    float mt = 0.f;
#pragma unroll
    for (int w = 0; w < BLK_WARPS; ++w) {
        const int t = sc.red[par][w];
        if (w < warp) off += t;
        total += t;
        vt += sc.vred[w];
        mt = fmaxf(mt, sc.mred[w]);
    }
    par ^= 1;
    for (int k = k0; k < k1 && off < BLK_LIST; ++k) {
        T nb;
        if (scan_member<T, STD>(k, j, g, b, a, lam, nb)) list[off++] = k;
    }
    __syncthreads();
    nv = vt;
    mv = mt;
    return total;
}

// Whether k is one of the sorted list[0, n) (binary search).
__device__ __forceinline__ bool list_contains(const int* __restrict__ list, int n, int k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (list[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && list[lo] == k;
}

// The scan of a converged support, folded into the gradient refresh: while
// g is formed, every coordinate k != j outside list[0, n) with b_k = 0 whose
// candidate Soft(g_k, lambda) (divided by S_kk without standardisation) is
// nonzero, i.e. which a sweep with the support held would move, is counted
// into sc.wcnt[wp] and, while there is room, appended to vlist (in no
// particular order); sc.wmax[wp] keeps the largest |candidate| (as the bits
// of a non-negative float).  Thread 0 clears the other parity's pair for
// the next scan: that pair was last read before a barrier that every thread
// has passed since.
struct RefreshScan {
    int* vlist;
    int vcap;
    int wp;
};

// g = S_.j - sum_{l in A} S_.l b_l over the whole row (block-wide), A = list[0, n).
// A thread takes QG of its quads at once and reads R support rows for each, so
// QG * R independent loads are in flight; the products are accumulated in
// the order of the list.  With `scan` the refresh also scans (RefreshScan).
template <typename T, bool STD>
__device__ void block_form_gradient(int j, T* __restrict__ g, const T* __restrict__ b,
                                    const int* __restrict__ list, int n, const CDArgs<T>& a,
                                    bool scan, T lam, BlockScratch& sc, RefreshScan ws) {
    constexpr int QG = sizeof(T) == 4 ? 2 : 1, R = 4;
    const int ldp = a.ldp;
    const T* __restrict__ Sj = a.SC + (size_t)j * ldp;
    if (scan) {
        if (threadIdx.x == 0) {
            sc.wcnt[ws.wp ^ 1] = 0;
            sc.wmax[ws.wp ^ 1] = 0;
        }
    }
    for (int q0 = threadIdx.x; 4 * q0 < ldp; q0 += QG * BLK_THREADS) {
        T acc[QG][4];
#pragma unroll
        for (int u = 0; u < QG; ++u) {
            const int k0 = 4 * (q0 + u * BLK_THREADS);
            if (k0 < ldp) load4g<T>(Sj + k0, acc[u]);
        }
        int e = 0;
        for (; e + R <= n; e += R) {
            T r[R][QG][4];
#pragma unroll
            for (int v = 0; v < R; ++v) {
                const T* __restrict__ row = a.SC + (size_t)list[e + v] * ldp;
#pragma unroll
                for (int u = 0; u < QG; ++u) {
                    const int k0 = 4 * (q0 + u * BLK_THREADS);
                    if (k0 < ldp) load4g<T>(row + k0, r[v][u]);
                }
            }
#pragma unroll
            for (int v = 0; v < R; ++v) {
                const T bv = b[list[e + v]];
#pragma unroll
                for (int u = 0; u < QG; ++u)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[u][t] = fma(-bv, r[v][u][t], acc[u][t]);
            }
        }
        for (; e < n; ++e) {
            const T* __restrict__ row = a.SC + (size_t)list[e] * ldp;
            const T bv = b[list[e]];
#pragma unroll
            for (int u = 0; u < QG; ++u) {
                const int k0 = 4 * (q0 + u * BLK_THREADS);
                if (k0 < ldp) {
                    T r[4];
                    load4g<T>(row + k0, r);
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[u][t] = fma(-bv, r[t], acc[u][t]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < QG; ++u) {
            const int k0 = 4 * (q0 + u * BLK_THREADS);
            if (k0 < ldp)
#pragma unroll
                for (int t = 0; t < 4; ++t) g[k0 + t] = acc[u][t];
        }
        if (scan) {
#pragma unroll
            for (int u = 0; u < QG; ++u) {
                const int k0 = 4 * (q0 + u * BLK_THREADS);
                if (k0 < a.p) {
                    T bq[4];
                    load4<T>(b + k0, bq);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int k = k0 + t;
                        if (k < a.p && k != j && bq[t] == T(0)) {
                            T nb;
                            if constexpr (STD) nb = soft<T>(acc[u][t] + bq[t], lam);     // S_kk = 1
                            else nb = soft<T>(acc[u][t] + a.diag[k] * bq[t], lam) / a.diag[k];
                            if (nb != T(0) && !list_contains(list, n, k)) {
                                const int slot = atomicAdd(&sc.wcnt[ws.wp], 1);
                                if (slot < ws.vcap) ws.vlist[slot] = k;
                                atomicMax(&sc.wmax[ws.wp], __float_as_int(fabsf((float)nb)));
                            }
                        }
                    }
                }
            }
        }
    }
}

// The sorted union of list[0, n) (sorted) and vlist[0, nv) (distinct, not in
// the list, in any order) into u[0, n + nv), by warp 0 (n + nv <= BLK_AMAX):
// an entry's place is the number of entries of both lists below it.
__device__ inline void warp_union(const int* __restrict__ list, int n, const int* __restrict__ vlist,
                           int nv, int* __restrict__ u) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h;
        int x = INT_MAX, cv = 0;
        if (e < n) x = list[e];
        int y = INT_MAX, ry = 0;
        if (e < nv) y = vlist[e];
        for (int t = 0; t < nv; ++t) {
            const int w = vlist[t];
            cv += w < x;
            ry += w < y;
        }
        if (e < n) u[e + cv] = x;
        if (e < nv) {
            int lo = 0, hi = n;                       // entries of the list below y
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (list[mid] < y) lo = mid + 1;
                else hi = mid;
            }
            u[ry + lo] = y;
        }
    }
    __syncwarp();
}

// Active-set phase of the block solver, run by warp 0 on A = list[0, n),
// n <= BLK_AMAX: lane m holds coordinates A_m and A_{m+32}.  Reads and writes
// b for the coordinates of A; g is formed afresh by the caller afterwards.
// Returns the sweeps done; conv tells whether the last one moved nothing by tol.
// One move is the critical path of the phase: every lane forms the candidate
// of its slot, the owner's change is broadcast by one shuffle, and every lane
// updates its two gradients with the column of S_AA loaded one move ahead.  A
// zero change adds exact zeros, so no lane branches on it.
template <typename T, bool STD>
__device__ int block_active_phase(int j, T* __restrict__ b, const int* __restrict__ list, int n,
                                  const CDArgs<T>& a, T lam, T* __restrict__ saa,
                                  int* __restrict__ saa_list, int& saa_n,
                                  unsigned long long& moves, bool& conv) {
    const int lane = threadIdx.x & 31;
    const int ldp = a.ldp;
    const int m0 = lane, m1 = lane + 32;
    // S_AA, zero outside the n x n block so the idle slots stay finite; kept
    // from the last phase when the support is the same (saa_list, saa_n)
    const bool same = saa_n == n &&
                      __all_sync(FULL_MASK, (m0 >= n || saa_list[m0] == list[m0]) &&
                                                (m1 >= n || saa_list[m1] == list[m1]));
    if (!same) {
        const int l0 = m0 < n ? list[m0] : 0, l1 = m1 < n ? list[m1] : 0;
        for (int k0 = 0; k0 < BLK_AMAX; k0 += 8) {
            T v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u;
                const T* __restrict__ row = a.SC + (size_t)(k < n ? list[k] : 0) * ldp;
                v0[u] = (k < n && m0 < n) ? row[l0] : T(0);
                v1[u] = (k < n && m1 < n) ? row[l1] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                saa[(k0 + u) * BLK_AMAX + m0] = v0[u];
                saa[(k0 + u) * BLK_AMAX + m1] = v1[u];
            }
        }
        if (m0 < n) saa_list[m0] = list[m0];
        if (m1 < n) saa_list[m1] = list[m1];
        saa_n = n;
        __syncwarp();
    }
    const bool h0 = m0 < n, h1 = m1 < n;
    T b0 = h0 ? b[list[m0]] : T(0), b1 = h1 ? b[list[m1]] : T(0);
    T g0 = h0 ? a.SC[(size_t)j * ldp + list[m0]] : T(0);
    T g1 = h1 ? a.SC[(size_t)j * ldp + list[m1]] : T(0);
    T s0 = T(1), s1 = T(1);
    if constexpr (!STD) {
        if (h0) s0 = a.diag[list[m0]];
        if (h1) s1 = a.diag[list[m1]];
    }
    __syncwarp();
    for (int l = 0; l < n; ++l) {
        const T bl = __shfl_sync(FULL_MASK, l < 32 ? b0 : b1, l & 31);
        g0 = fma(-saa[l * BLK_AMAX + m0], bl, g0);
        g1 = fma(-saa[l * BLK_AMAX + m1], bl, g1);
    }
    conv = false;
    int sw = 0;
    unsigned mv = 0;
    const float tf = float_at_least(a.tol);
    while (sw < a.maxit) {
        ++sw;
        T md = T(0);
        T c0 = saa[m0], c1 = saa[m1];                     // column of S_AA for k = 0
        for (int k = 0; k < n; ++k) {
            const int kn = k + 1 < n ? k + 1 : k;
            const T n0 = saa[kn * BLK_AMAX + m0], n1 = saa[kn * BLK_AMAX + m1];   // next column
            const bool hi = k >= 32;
            const T gk = hi ? g1 : g0, bk = hi ? b1 : b0;
            T nb;
            if constexpr (STD) {
                nb = soft<T>(gk + bk, lam);                          // S_kk = 1
            } else {
                const T sk = hi ? s1 : s0;
                nb = soft<T>(gk + sk * bk, lam) / sk;
            }
            const T d = __shfl_sync(FULL_MASK, nb - bk, k & 31);
            if (lane == (k & 31)) {
                if (hi) b1 = nb;
                else b0 = nb;
            }
            g0 = fma(-c0, d, g0);
            g1 = fma(-c1, d, g1);
            md = fmax(md, fabs(d));
            mv += d != T(0);
            c0 = n0;
            c1 = n1;
        }
        if (below_tol<T>(md, a.tol, tf)) {
            conv = true;
            break;
        }
    }
    moves += mv;
    if (h0) b[list[m0]] = b0;
    if (h1) b[list[m1]] = b1;
    return sw;
}

// One sweep of the block solver (cyclic ascending, k != j; with `frozen` the
// coordinates of the support keep their values).  Returns max |delta b|.
// cand holds the candidate moves (new b, delta) of every thread, two buffers.
template <typename T, bool STD>
__device__ T block_sweep(int j, T* __restrict__ g, T* __restrict__ b, const CDArgs<T>& a, T lam,
                         bool frozen, T* __restrict__ cand, unsigned long long& moves,
                         BlockScratch& sc, int& par, int sweep_idx) {
    const int tid = threadIdx.x;
    const int p = a.p, ldp = a.ldp;
    T maxd = T(0);
    int ks = -1;                      // the move of the last pass, applied in this pass
    T delta = T(0);
    for (;;) {
        const T* __restrict__ srow = a.SC + (size_t)(ks < 0 ? 0 : ks) * ldp;
        T* __restrict__ cb = cand + (size_t)par * 2 * BLK_THREADS;
        int kmin = INT_MAX;
        // the thread's quads q0, q0 + BLK_THREADS, ... in groups of G, the
        // group's S-row loads issued together
        constexpr int G = sizeof(T) == 4 ? 4 : 2;
        for (int q0 = tid; 4 * q0 < ldp; q0 += G * BLK_THREADS) {
            T r[G][4];
            if (ks >= 0) {
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int k0 = 4 * (q0 + u * BLK_THREADS);
                    if (k0 < ldp) load4g<T>(srow + k0, r[u]);
                }
            }
#pragma unroll
          for (int u = 0; u < G; ++u) {
            const int k0 = 4 * (q0 + u * BLK_THREADS);
            if (k0 >= ldp) break;
            T gv[4];
            load4<T>(g + k0, gv);
            if (ks >= 0) {            // rank-1 update g -= S_.ks delta (Proposition 2)
#pragma unroll
                for (int t = 0; t < 4; ++t) gv[t] = fma(-delta, r[u][t], gv[t]);
#pragma unroll
                for (int t = 0; t < 4; ++t) g[k0 + t] = gv[t];
            }
            if (kmin == INT_MAX && k0 + 3 > ks && k0 < p) {
                T bv[4];
                load4<T>(b + k0, bv);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int k = k0 + t;
                    if (kmin == INT_MAX && k > ks && k < p && k != j && !(frozen && bv[t] != T(0))) {
                        T nb;
                        if constexpr (STD) {
                            nb = soft<T>(gv[t] + bv[t], lam);                 // S_kk = 1
                        } else {
                            const T skk = a.diag[k];
                            nb = soft<T>(gv[t] + skk * bv[t], lam) / skk;     // Soft(c, lambda)/S_kk
                        }
                        if (nb != bv[t]) {
                            kmin = k;
                            cb[tid] = nb;
                            cb[BLK_THREADS + tid] = nb - bv[t];
                        }
                    }
                }
            }
          }
        }
        const int kb = block_min_int(kmin, sc, par);    // barrier: g updated, candidates visible
        if (kb == INT_MAX) break;
        const int owner = (kb >> 2) % BLK_THREADS;      // the thread whose quads hold kb
        delta = cb[BLK_THREADS + owner];
        if (tid == owner) {
            b[kb] = cb[owner];
            note_row_moved(a, sweep_idx, kb);
        }
        maxd = fmax(maxd, fabs(delta));
        ++moves;
        ks = kb;
    }
    return maxd;
}

// sigma_j^2 = S_jj - 2 b'S_.j + b'S b in FP64 over the support list (block-wide),
// FP64 products; a support longer than the list takes the rows from b itself.
template <typename T>
__device__ __noinline__ double block_quadratic_form(int j, const T* __restrict__ b, const int* __restrict__ list,
                                       int n, const CDArgs<T>& a, BlockScratch& sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ldp = a.ldp, p = a.p;
    double lin = 0.0, quad = 0.0;
    if (n <= BLK_LIST) {
        for (int u = warp; u < n; u += BLK_WARPS) {
            const int ku = list[u];
            const T* __restrict__ row = a.SC + (size_t)ku * ldp;
            double part = 0.0;
            for (int v = lane; v < n; v += 32) {
                const int kv = list[v];
                part = fma((double)b[kv], (double)row[kv], part);
            }
            quad = fma((double)b[ku], part, quad);
            if (lane == 0) lin = fma((double)b[ku], (double)row[j], lin);
        }
    } else {
        for (int u = warp; u < p; u += BLK_WARPS) {
            const T bu = b[u];
            if (bu == T(0)) continue;
            const T* __restrict__ row = a.SC + (size_t)u * ldp;
            double part = 0.0;
            for (int v = lane; v < p; v += 32)
                if (b[v] != T(0)) part = fma((double)b[v], (double)row[v], part);
            quad = fma((double)bu, part, quad);
            if (lane == 0) lin = fma((double)bu, (double)row[j], lin);
        }
    }
    lin = block_sum_d(lin, sc);
    quad = block_sum_d(quad, sc);
    return (double)a.SC[(size_t)j * ldp + j] - 2.0 * lin + quad;
}

// sigma_j^2 = S_jj - 2 b'S_.j + b'S b (Eq. (14)) in FP64 from the block
// S_AA in shared memory, when the support lies in the list A it was
// gathered for (A = saa_list[0, na), sorted; saa[k BLK_AMAX + m] = S_{A_k A_m}):
// b is zero on A outside the support, and the zero terms add nothing.
// Returns false (nothing computed) when some support coordinate is not in A.
// The products are formed in FP64, warp w taking the rows k = w, w + 16, ...
// of S_AA and each lane two of its entries; one fixed-order block sum.
template <typename T>
__device__ __noinline__ bool block_quadratic_form_saa(int j, const T* __restrict__ b, int nsupp,
                                         const int* __restrict__ saa_list, int na,
                                         const T* __restrict__ saa, const CDArgs<T>& a,
                                         BlockScratch& sc, double& q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tid = threadIdx.x;
    if (na <= 0 || na > BLK_AMAX || nsupp > na) return false;
    const int inA = __syncthreads_count(tid < na && b[saa_list[tid]] != T(0));
    if (inA != nsupp) return false;
    const int v0 = lane, v1 = lane + 32;
    const double bv0 = v0 < na ? (double)b[saa_list[v0]] : 0.0;
    const double bv1 = v1 < na ? (double)b[saa_list[v1]] : 0.0;
    double acc = 0.0;
    for (int k = warp; k < na; k += BLK_WARPS) {
        const int ak = saa_list[k];
        const double bk = (double)b[ak];
        double t = v0 < na ? bv0 * (double)saa[k * BLK_AMAX + v0] : 0.0;
        if (v1 < na) t = fma(bv1, (double)saa[k * BLK_AMAX + v1], t);
        acc = fma(bk, t, acc);                              // b_k sum_m S_km b_m
        if (lane == 0) acc = fma(-2.0 * bk, (double)a.SC[(size_t)ak * a.ldp + j], acc);
    }
    acc = block_sum_d(acc, sc);
    q = (double)a.SC[(size_t)j * a.ldp + j] + acc;
    return true;
}

// Algorithm 1 for column j by the whole block (see above).  Writes b_j (the
// whole row j of BT), sigma_j and the column status.  Counters are kept
// identically by every thread; the caller flushes thread 0's.
template <typename T, bool STD>
__device__ void solve_column_block(int j, unsigned char* smem, const CDArgs<T>& a,
                                   ColCounters& cnt, BlockScratch& sc) {
    const int tid = threadIdx.x;
    const int ldp = a.ldp;
    T* g = reinterpret_cast<T*>(smem);
    T* b = g + ldp;
    T* saa = b + ldp;
    int* list = reinterpret_cast<int*>(saa + BLK_AMAX * BLK_AMAX);
    T* cand = reinterpret_cast<T*>(list + BLK_LIST);
    int* saa_list = reinterpret_cast<int*>(cand + 2 * 2 * BLK_THREADS);   // support of S_AA
    // the candidate buffers are idle between sweeps: the working set's union
    // and the refresh scan's coordinates live there
    int* ubuf = reinterpret_cast<int*>(cand);
    int* vlist = ubuf + BLK_AMAX;
    int saa_n = -1;                                       // warp 0: no S_AA gathered yet
    int par = 0;
    int wp = 0;                                           // parity of the refresh scan's counters
    // a column the lazy solver handed over continues from its iterate
    const int st0 = a.hand ? a.col_status[j] : COL_OK;
    const bool warm = (st0 & COL_HANDED) != 0;
    {
        const T* __restrict__ Sj = a.SC + (size_t)j * ldp;
        const T* __restrict__ brow = a.BT + (size_t)j * ldp;
        for (int k = tid; k < ldp; k += BLK_THREADS) {
            g[k] = Sj[k];                                 // g = S_.j  (b = 0)
            b[k] = warm ? brow[k] : T(0);
        }
        if (tid == 0) {
            sc.wcnt[0] = sc.wcnt[1] = 0;
            sc.wmax[0] = sc.wmax[1] = 0;
            sc.saa_n = -1;
        }
    }
    __syncthreads();
    double sigma = 1.0;                                   // sigma^(0) = 1
    double s_prev = 0.0, f_prev = 0.0;                    // last (sigma, F(sigma))
    int status = COL_OK;
    int r0 = 0;
    bool stale = false;                                   // g is not yet S_.j - S b
    if (warm) {
        sigma = a.sigma[j];
        s_prev = a.hand[2 * (size_t)j];
        f_prev = a.hand[2 * (size_t)j + 1];
        status = st0 & (COL_NOT_CONVERGED | COL_DEGENERATE);
        r0 = st0 >> COL_STEP_SHIFT;
        stale = true;
    }
    const unsigned long long sweeps0 = cnt.sweeps;
    const double floor2 = 1e-12 * (double)a.SC[(size_t)j * ldp + j];
    int r;
    for (r = r0; r < a.maxit; ++r) {
        const T lam = (T)(sigma * a.lambda0);
        bool inner_ok = false;
        int rounds = 0;              // working-set rounds at this lambda
        bool uni = false;            // ubuf[0, nu) holds the union for the next phase
        int nu = 0;
        for (int m = 0; m < a.maxit; ++m) {
            // converge on the support first (when it fits the phase), then a
            // sweep with the support held decides; otherwise a full sweep
            // decides (Algorithm 1's stop), as in the lazy solver
            int n = uni ? nu : block_support_list<T>(b, a.p, list, sc, par);
            const int* plist = uni ? ubuf : list;
            bool conv = n == 0;
            const bool phase = n > 0 && n <= BLK_AMAX;
            if (phase) {
                int sw = 0;
                bool c = false;
                if (tid < 32) sw = block_active_phase<T, STD>(j, b, plist, n, a, lam, saa, saa_list,
                                                              saa_n, cnt.act_moves, c);
                if (tid == 0) {
                    sc.red[par][0] = sw;
                    sc.red[par][1] = c ? 1 : 0;
                    sc.saa_n = saa_n;
                }
                __syncthreads();
                sw = sc.red[par][0];
                conv = sc.red[par][1] != 0;
                par ^= 1;
                cnt.act_sweeps += sw;
            }
            // Working set: with the support converged, one scan of every
            // coordinate finds those that a sweep with the support held
            // would move.  None: that sweep would move nothing
            // (max |delta| = 0), so the lasso at this lambda is solved.
            // Otherwise, while their union with the support fits the phase
            // and one of them would move by tol or more, they join the next
            // phase's coordinates at b = 0, instead of the sweep moving them
            // one at a time with an O(p) update each.  Else the sweep decides.
            // After a phase the scan runs inside the gradient refresh.
            const bool ws = conv && rounds < BLK_WS_ROUNDS;
            bool scanned = false;
            int nv = 0;
            float mv = 0.f;
            // a handed-over support (at most LAZY_CAP entries) fits the list
            if (phase || stale) {
                if (uni) n = block_support_list<T>(b, a.p, list, sc, par);   // the support
                scanned = ws && n <= BLK_AMAX;
                block_form_gradient<T, STD>(j, g, b, list, n, a, scanned, lam, sc,
                                            RefreshScan{vlist, BLK_AMAX, wp});
                __syncthreads();
                if (scanned) {
                    nv = sc.wcnt[wp];
                    mv = __int_as_float(sc.wmax[wp]);
                    wp ^= 1;
                }
                stale = false;
            }
            uni = false;
            if (ws && n <= BLK_AMAX) {
                if (!scanned) {
                    // no refresh (b = 0, g = S_.j): a scan of its own, the union into ubuf
                    nu = block_scan_list<T, STD>(j, g, b, a, lam, ubuf, sc, par, nv, mv);
                }
                ++cnt.sweeps;
                if (nv == 0) {
                    inner_ok = true;
                    break;
                }
                if (scanned) nu = n + nv;
                if (nu <= BLK_AMAX && (double)mv >= a.tol) {
                    if (scanned && tid < 32) warp_union(list, n, vlist, nv, ubuf);
                    __syncthreads();
                    uni = true;
                    ++rounds;
                    continue;
                }
            }
            const T md = block_sweep<T, STD>(j, g, b, a, lam, conv, cand, cnt.moves, sc, par,
                                             (int)(cnt.sweeps - sweeps0));
            ++cnt.sweeps;
            if ((double)md < a.tol) {
                inner_ok = true;
                break;
            }
        }
        if (!inner_ok) status |= COL_NOT_CONVERGED;
        const int n = block_support_list<T>(b, a.p, list, sc, par);
        double q;
        if (!block_quadratic_form_saa<T>(j, b, n, saa_list, sc.saa_n, saa, a, sc, q))
            q = block_quadratic_form<T>(j, b, list, n, a, sc);
        if (q <= floor2) {
            q = floor2;
            status |= COL_DEGENERATE;
        }
        const double sn = sqrt_heron(q);
        if (fabs(sn - sigma) < a.tol) {
            sigma = sn;
            break;
        }
        double nxt = sn;
        if (r > 0 && r + 1 < a.maxit && !(status & COL_DEGENERATE))
            nxt = sigma_step(s_prev, f_prev, sigma, sn);
        s_prev = sigma;
        f_prev = sn;
        sigma = nxt;
    }
    if (r == a.maxit) {
        r = a.maxit - 1;
        status |= COL_NOT_CONVERGED;
    }
    // b_j into row j of BT (the whole row, zeros included)
    T* brow = a.BT + (size_t)j * ldp;
    for (int k = tid; k < ldp; k += BLK_THREADS) brow[k] = b[k];
    if (tid == 0) {
        a.sigma[j] = sigma;
        a.col_status[j] = status;
    }
    cnt.outer_max = max(cnt.outer_max, r + 1);
    cnt.max_sw = max(cnt.max_sw, (int)(cnt.sweeps - sweeps0));
    cnt.n_nc += (status & COL_NOT_CONVERGED) != 0;
    cnt.n_deg += (status & COL_DEGENERATE) != 0;
    ++cnt.blk;
    __syncthreads();
}

__device__ __forceinline__ void flush_counters_block(FitCtrl* ctrl, ColCounters& c) {
    if (threadIdx.x == 0) {
        if (c.blk) atomicAdd(&ctrl->block_cols, c.blk);
        if (c.sweeps) atomicAdd(&ctrl->total_sweeps, c.sweeps);
        if (c.moves) atomicAdd(&ctrl->moves, c.moves);
        if (c.act_sweeps) atomicAdd(&ctrl->act_sweeps, c.act_sweeps);
        if (c.act_moves) atomicAdd(&ctrl->act_moves, c.act_moves);
        atomicMax(&ctrl->outer_max, c.outer_max);
        atomicMax(&ctrl->max_col_sweeps, c.max_sw);
        if (c.n_nc) atomicAdd(&ctrl->n_not_converged, c.n_nc);
        if (c.n_deg) atomicAdd(&ctrl->n_degenerate, c.n_deg);
    }
    c = ColCounters();
}

// Theta (Eq. (4), Eq. (9), Proposition 1) over pairs of TS x TS tiles: the
// tile of rows j0.., columns k0.. (j0 <= k0) and its mirror.  Omega_1 = -B D
// on the working scale, min-magnitude symmetrisation (for j < k a tie keeps
// omega_jk) and Omega^o = C Omega C.  Both coefficient tiles are read once
// into shared memory, and every entry of both Theta tiles is written, both
// entries of a pair with the same value, so Theta is exactly symmetric and
// needs no clearing beforehand.  Blocks of the first
// tile row also write sigma in the original scale; nonzero coefficients are
// counted into ctrl->nnz.  Block shape 32 x 8.  TS = 64 for FP32
// coefficients, 32 for FP64 (static shared memory).
template <typename T>
__host__ __device__ constexpr int theta_ts() { return sizeof(T) == 4 ? 64 : 32; }

// Tile pairs of a p x p Theta.
template <typename T>
__host__ __device__ inline int theta_pairs(int p) {
    const int t = (p + theta_ts<T>() - 1) / theta_ts<T>();
    return t * (t + 1) / 2;
}

template <typename T>
__device__ void theta_pair(const T* __restrict__ BT, int p, int ldp,
                           const double* __restrict__ sigma, const double* __restrict__ cs,
                           double* __restrict__ Theta, double* __restrict__ sigma_out,
                           FitCtrl* ctrl, int pair) {
    constexpr int TS = theta_ts<T>();
    __shared__ T tA[TS][TS + 1];    // tA[kk][jj] = BT[k0+kk][j0+jj] = b_jk
    __shared__ T tB[TS][TS + 1];    // tB[jj][kk] = BT[j0+jj][k0+kk] = b_kj
    // 1/sigma^2 and c for the pair's rows and columns: FP64 divisions are
    // expensive on this part, so each block does 2 TS of them
    __shared__ double inv_j[TS], inv_k[TS], c_j[TS], c_k[TS];
    const int t = (p + TS - 1) / TS;
    int a = 0, rem = pair;
    while (rem >= t - a) {
        rem -= t - a;
        ++a;
    }
    const int j0 = a * TS, k0 = (a + rem) * TS;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int lin = ty * 32 + tx;
    if (lin < 2 * TS) {
        const bool col = lin < TS;
        const int i = col ? k0 + lin : j0 + lin - TS;
        double inv = 0.0, c = 0.0;
        if (i < p) {
            const double s = sigma[i];
            inv = 1.0 / (s * s);
            c = cs[i];
        }
        if (col) { inv_k[lin] = inv; c_k[lin] = c; }
        else { inv_j[lin - TS] = inv; c_j[lin - TS] = c; }
    }
    if constexpr (sizeof(T) == 4) {
        // 16-byte reads: 16 lanes per 64-float row; columns p..ldp-1 of B are
        // zero, quads past the padded row are not read
        const int q = 4 * (tx & 15);
        for (int r = 2 * ty + (tx >> 4); r < TS; r += 16) {
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (k0 + r < p && j0 + q < ldp) va = *reinterpret_cast<const float4*>(BT + (size_t)(k0 + r) * ldp + j0 + q);
            if (j0 + r < p && k0 + q < ldp) vb = *reinterpret_cast<const float4*>(BT + (size_t)(j0 + r) * ldp + k0 + q);
            tA[r][q] = va.x; tA[r][q + 1] = va.y; tA[r][q + 2] = va.z; tA[r][q + 3] = va.w;
            tB[r][q] = vb.x; tB[r][q + 1] = vb.y; tB[r][q + 2] = vb.z; tB[r][q + 3] = vb.w;
        }
    } else {
        for (int r = ty; r < TS; r += 8)
            for (int q = tx; q < TS; q += 32) {
                tA[r][q] = (k0 + r < p && j0 + q < p) ? BT[(size_t)(k0 + r) * ldp + j0 + q] : T(0);
                tB[r][q] = (j0 + r < p && k0 + q < p) ? BT[(size_t)(j0 + r) * ldp + k0 + q] : T(0);
            }
    }
    __syncthreads();
    // Theta_jk for j = j0 + jj, k = k0 + kk
    auto value = [&](int jj, int kk) -> double {
        const int j = j0 + jj, k = k0 + kk;
        // the scale (c_j c_k) is formed before it multiplies, so the value
        // does not depend on which of the pair computes it
        if (j == k) return inv_k[kk] * (c_j[jj] * c_k[kk]);
        const T bjk = tA[kk][jj];      // coefficient of x_j in regression k
        const T bkj = tB[jj][kk];      // coefficient of x_k in regression j
        if (bjk == T(0) && bkj == T(0)) return 0.0;   // both candidates are zero
        const double ojk = -(double)bjk * inv_k[kk];  // Omega_1[j][k]
        const double okj = -(double)bkj * inv_j[jj];  // Omega_1[k][j]
        double out;
        if (j < k) out = fabs(ojk) > fabs(okj) ? okj : ojk;
        else out = fabs(okj) > fabs(ojk) ? ojk : okj;  // pair (k, j) with k < j
        return out * (c_j[jj] * c_k[kk]);
    };
    // Every entry of the tile and of its mirror is written (Theta needs no
    // clearing first), each row segment by consecutive lanes.  Both entries
    // of a pair come from the same value(jj, kk), so Theta is exactly
    // symmetric; a diagonal tile is its own mirror and is written once.
    unsigned long long nnz = 0;
    for (int jj = ty; jj < TS; jj += 8) {
        const int j = j0 + jj;
        if (j >= p) break;
        for (int kk = tx; kk < TS; kk += 32) {
            const int k = k0 + kk;
            if (k >= p) break;
            nnz += (j != k && tB[jj][kk] != T(0)) + (j0 != k0 && tA[kk][jj] != T(0));
            Theta[(size_t)j * p + k] = value(jj, kk);
        }
    }
    if (j0 != k0) {
        for (int kk = ty; kk < TS; kk += 8) {
            const int k = k0 + kk;
            if (k >= p) break;
            for (int jj = tx; jj < TS; jj += 32) {
                const int j = j0 + jj;
                if (j >= p) break;
                Theta[(size_t)k * p + j] = value(jj, kk);
            }
        }
    }
    if (j0 == 0 && lin < TS && k0 + lin < p) sigma_out[k0 + lin] = sigma[k0 + lin] / cs[k0 + lin];
    // one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(FULL_MASK, nnz, o);
    if (tx == 0 && nnz) atomicAdd(&ctrl->nnz, nnz);
}

}  // namespace spmesl
