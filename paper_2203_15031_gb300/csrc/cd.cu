// Coordinate descent for SPMESL on the covariance matrix (sm_103a).
//
// Layout in HBM (one fit; see common.cuh FitLayout):
//   SC  p x ldp  working covariance (S^C = C S C when standardising), rows
//                zero-padded to ldp = roundup(p, 32) elements
//   BT  p x ldp  row j = coefficients b_.j of regression j (B transposed)
//   GT  p x ldp  row j = gradient g_j = S_.j - S b_j (joint rule only)
// S is symmetric, so column k of S (needed by the rank-1 update) is row k of
// SC: every S access below is a contiguous, 16-byte-vector, coalesced row read.
//
// One warp owns one column j at a time and keeps g_j and b_j in shared
// memory.  A sweep is the cyclic ascending pass over k (Algorithm 1): the
// warp evaluates 32 consecutive coordinates at once, finds the first one whose
// soft-threshold update changes b_kj (ballot), applies it, performs the
// rank-1 update g_j -= S_.k * delta and restarts the scan right after k.
// Coordinates that do not move change nothing, so skipping over them is
// exactly the sequential order of Algorithm 1 and of the per-column view of
// Proposition 2 (Theorem 1: PCD iterates equal the per-column CD iterates).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cd_device.cuh"

namespace spmesl {

// ---------------------------------------------------------------------------
// Per-column rule (Algorithms 1-2): every warp takes the next unsolved column
// and runs the whole scaled lasso for it; no grid-wide synchronisation.
// ---------------------------------------------------------------------------
// Eager gradient (g_j and b_j in shared memory).  With from_queue the warps
// take the columns the lazy solver handed over instead of 0..p-1.
template <typename T, bool STD>
__global__ void __launch_bounds__(512) cd_column_kernel(CDArgs<T> a, int from_queue) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T* g = reinterpret_cast<T*>(smem_raw + (size_t)warp * warp_smem_bytes<T>(a.ldp));
    T* b = g + a.ldp;
    int* list = reinterpret_cast<int*>(b + a.ldp);
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    const int nq = from_queue ? *reinterpret_cast<volatile int*>(a.ovf_count) : 0;
    ColCounters cnt;
    for (;;) {
        int j = 0;
        if (from_queue) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&ctrl->ovf_next, 1);
            t = __shfl_sync(FULL_MASK, t, 0);
            if (t >= nq) break;
            j = a.ovf_list[t];
        } else {
            if (lane == 0) j = atomicAdd(&ctrl->next_col, 1);
            j = __shfl_sync(FULL_MASK, j, 0);
            if (j >= a.p) break;
        }
        solve_column<T, STD>(j, g, b, list, a, cnt);
    }
    flush_counters(ctrl, cnt);
}

// Lazy gradient (sorted support in shared memory); columns whose support
// outgrows the list go to the queue for cd_column_kernel.
template <typename T, bool STD>
__global__ void __launch_bounds__(256, 3) cd_column_lazy_kernel(CDArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)warp * lazy_warp_smem_bytes<T>(a.ldp);
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    // the first n_heavy columns of the order belong to the block solver
    const int q0 = *reinterpret_cast<volatile int*>(&ctrl->n_heavy);
    ColCounters cnt;
    for (;;) {
        int j = 0;
        if (lane == 0) {
            const int q = q0 + atomicAdd(&ctrl->next_col, 1);
            j = q >= a.n_queue ? a.p : (a.order ? a.order[q] : q);
        }
        j = __shfl_sync(FULL_MASK, j, 0);
        if (j >= a.p) break;
        if (!solve_column_lazy<T, STD, true>(j, wsm, a, cnt) && lane == 0)
            a.ovf_list[atomicAdd(a.ovf_count, 1)] = j;
        __syncwarp();
    }
    flush_counters(ctrl, cnt);
}

// Block solver (one block per column, see solve_column_block): the heavy
// columns at the head of the heat order (from_overflow = 0, launched beside
// the lazy kernel) or the columns the lazy solver handed over (from_overflow
// = 1, after it).
template <typename T, bool STD>
__global__ void __launch_bounds__(BLK_THREADS, 1) cd_column_block_kernel(CDArgs<T> a,
                                                                      int from_overflow) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockScratch sc;
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    const int nq = from_overflow ? *reinterpret_cast<volatile int*>(a.ovf_count)
                                 : *reinterpret_cast<volatile int*>(&ctrl->n_heavy);
    int* next = from_overflow ? &ctrl->ovf_next : &ctrl->heavy_next;
    ColCounters cnt;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(next, 1);
            sc.col = t < nq ? (from_overflow ? a.ovf_list[t] : a.order[t]) : -1;
        }
        __syncthreads();
        const int j = sc.col;
        __syncthreads();
        if (j < 0) break;
        solve_column_block<T, STD>(j, smem_raw, a, cnt, sc);
    }
    flush_counters_block(ctrl, cnt);
}

__global__ void rows_count_kernel(const unsigned* __restrict__ bits, size_t nwords, FitCtrl* ctrl) {
    count_rows_moved(bits, nwords, ctrl, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                     (size_t)gridDim.x * blockDim.x);
}

// Optimality diagnostics of columns [j0, j1): one warp per column
// (diagnose_column), 4 warps a block, grid-stride over the columns.
constexpr int DIAG_WARPS = 4;
template <typename T>
__global__ void __launch_bounds__(32 * DIAG_WARPS) cd_diag_kernel(CDArgs<T> a, double eps, int j0,
                                                                  int j1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)warp * diag_warp_smem_bytes();
    if (*reinterpret_cast<volatile int*>(&a.ctrl->err) != 0) return;
    DiagMax d;
    for (int j = j0 + blockIdx.x * DIAG_WARPS + warp; j < j1; j += gridDim.x * DIAG_WARPS)
        diagnose_column<T>(j, wsm, a, eps, d);
    flush_diag(a.ctrl, d);
}

// A caller's estimate in the original scale onto the working scale of the
// workspace (spmesl_diagnose): BT[k][j] = b^C_jk = b_jk c_k / c_j (the
// inverse of the map of Proposition 1's proof) and sigma^C_k = sigma_k c_k.
template <typename T>
__global__ void load_estimate_kernel(const double* __restrict__ B, const double* __restrict__ sig,
                                     int p, int ldp, const double* __restrict__ cs,
                                     T* __restrict__ BT, double* __restrict__ sigma_w) {
    const size_t total = (size_t)p * p;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / p), k = (int)(i - (size_t)j * p);   // B[j][k] = b_jk
        BT[(size_t)k * ldp + j] = j == k ? T(0) : (T)(B[i] * cs[k] / cs[j]);
        if (j == 0) sigma_w[k] = sig[k] * cs[k];
    }
}

// ---------------------------------------------------------------------------
// Joint rule (Algorithm 3): all active columns sweep together; a sweep ends at
// a grid barrier where max_{active j} ||b_j,next - b_j,cur||_inf is tested.
// After the joint lasso converges every active column updates sigma, columns
// whose sigma moved by less than tol are retired, and the active index vector
// is compacted in order.  Launched cooperatively so the barrier cannot wait
// on a block that is not resident; every wait is bounded.
// ---------------------------------------------------------------------------
__device__ bool grid_sync(FitCtrl* c) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &c->bar_gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            c->bar_count = 0u;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g0) {
                __nanosleep(40);
                if (global_ns() - t0 > SPIN_LIMIT_NS) {
                    set_error(c, DEV_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        ok = (*reinterpret_cast<volatile int*>(&c->err) == 0);
    }
    __syncthreads();
    return ok != 0;
}

// Ordered compaction of active[0..nc) by flag (one block).  Returns the count.
__device__ int compact_active(int* active, int* active_next, const int* flag, int nc) {
    __shared__ int wcount[32];
    __shared__ int woff[32];
    __shared__ int total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int base = 0;
    for (int c0 = 0; c0 < nc; c0 += blockDim.x) {
        const int t = c0 + threadIdx.x;
        const bool keep = t < nc && flag[t] != 0;
        const unsigned bal = __ballot_sync(FULL_MASK, keep);
        const int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            const int v = lane < nw ? wcount[lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= o) incl += u;
            }
            woff[lane] = incl - v;
            if (lane == 31) total = incl;
        }
        __syncthreads();
        if (keep) active_next[base + woff[warp] + pre] = active[t];
        base += total;
        __syncthreads();
    }
    for (int t = threadIdx.x; t < base; t += blockDim.x) active[t] = active_next[t];
    __syncthreads();
    return base;
}

template <typename T, bool STD>
__global__ void __launch_bounds__(512) cd_joint_kernel(CDArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int gw = blockIdx.x * W + warp;
    const int TW = gridDim.x * W;
    T* g = reinterpret_cast<T*>(smem_raw + (size_t)warp * warp_smem_bytes<T>(a.ldp));
    T* b = g + a.ldp;
    int* list = reinterpret_cast<int*>(b + a.ldp);
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;

    unsigned long long moves = 0;
    unsigned long long gs = 0;        // global sweep counter (same in every block)
    double gmax = 0.0;
    int r;
    for (r = 0; r < a.maxit; ++r) {
        const int nc = *reinterpret_cast<volatile int*>(&ctrl->n_active);
        if (nc == 0) break;
        const bool resident = nc <= TW;
        if (resident && gw < nc) {
            const int j = a.active[gw];
            warp_copy<T>(g, a.GT + (size_t)j * a.ldp, a.ldp);
            warp_copy<T>(b, a.BT + (size_t)j * a.ldp, a.ldp);
            __syncwarp();
        }
        bool inner_ok = false;
        for (int m = 0; m < a.maxit; ++m, ++gs) {
            const int slot = (int)(gs % 3);
            if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->sweep_max[(gs + 1) % 3] = 0ull;
            T wmax = T(0);
            for (int t = gw; t < nc; t += TW) {
                const int j = a.active[t];
                if (!resident) {
                    warp_copy<T>(g, a.GT + (size_t)j * a.ldp, a.ldp);
                    warp_copy<T>(b, a.BT + (size_t)j * a.ldp, a.ldp);
                    __syncwarp();
                }
                const T lam = (T)(a.sigma[j] * a.lambda0);
                // no summaries carried between joint sweeps: every chunk is scanned
                ColScan cs{reinterpret_cast<ChunkInfo*>(list + SUPP_CAP), 0.f, 0u};
                reset_chunks(cs, a.ldp);
                __syncwarp();
                wmax = fmax(wmax, sweep_column<T, STD>(j, g, b, a, lam, moves, cs, (int)gs));
                if (!resident) {
                    warp_copy<T>(a.GT + (size_t)j * a.ldp, g, a.ldp);
                    warp_copy<T>(a.BT + (size_t)j * a.ldp, b, a.ldp);
                    __syncwarp();
                }
            }
            if (lane == 0 && wmax > T(0)) atomicMax(&ctrl->sweep_max[slot], dbits((double)wmax));
            if (!grid_sync(ctrl)) return;
            gmax = __longlong_as_double(
                (long long)*reinterpret_cast<volatile unsigned long long*>(&ctrl->sweep_max[slot]));
            if (gmax < a.tol) {
                inner_ok = true;
                ++gs;
                break;
            }
        }
        if (!inner_ok && blockIdx.x == 0 && threadIdx.x == 0) ctrl->inner_cap_hit = 1;

        // sigma update of every active column (Algorithm 3), FP64.
        for (int t = gw; t < nc; t += TW) {
            const int j = a.active[t];
            if (resident) {
                warp_copy<T>(a.GT + (size_t)j * a.ldp, g, a.ldp);
                warp_copy<T>(a.BT + (size_t)j * a.ldp, b, a.ldp);
            } else {
                warp_copy<T>(b, a.BT + (size_t)j * a.ldp, a.ldp);
            }
            __syncwarp();
            double q = residual_quadratic_form<T>(j, b, a, list);
            const double floor2 = 1e-12 * (double)a.SC[(size_t)j * a.ldp + j];
            if (q <= floor2) {
                q = floor2;
                if (lane == 0 && !(atomicOr(&a.col_status[j], COL_DEGENERATE) & COL_DEGENERATE))
                    atomicAdd(&ctrl->n_degenerate, 1);
            }
            const double sn = sqrt(q);
            if (lane == 0) {
                a.flag[t] = fabs(sn - a.sigma[j]) >= a.tol ? 1 : 0;
                a.sigma[j] = sn;
            }
            __syncwarp();
        }
        if (!grid_sync(ctrl)) return;
        if (blockIdx.x == 0) {
            const int nn = compact_active(a.active, a.active_next, a.flag, nc);
            if (threadIdx.x == 0) ctrl->n_active = nn;
        }
        if (!grid_sync(ctrl)) return;
    }
    if (lane == 0) atomicAdd(&ctrl->moves, moves);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->total_sweeps = gs;
        ctrl->max_col_sweeps = (int)gs;
        ctrl->outer_max = r < a.maxit ? r : a.maxit;
        ctrl->max_db_bits = dbits(gmax);
        const int left = *reinterpret_cast<volatile int*>(&ctrl->n_active);
        if (left > 0) ctrl->n_not_converged = left;
    }
}

// ---------------------------------------------------------------------------
// Preparation: C = diag(S_jj^-1/2), S^C = C S C into the padded SC, the
// diagonal of the working matrix, and the starting state of Algorithm 3
// (B = 0, G = S, sigma = 1, I = (1..p)).  Non-finite input or S_jj <= 0 sets
// DEV_ERR_NONFINITE and the fit kernels then do nothing.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void prep_diag_kernel(const T* __restrict__ S, int p, int standardize, double* cs,
                                 float* csf, double* sigma, int* active, int* col_status,
                                 FitCtrl* ctrl) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x) {
        const double d = (double)S[(size_t)j * p + j];
        if (!(d > 0.0) || !isfinite(d)) set_error(ctrl, DEV_ERR_NONFINITE);
        const double c = standardize ? 1.0 / sqrt(d) : 1.0;
        cs[j] = c;
        csf[j] = (float)c;
        sigma[j] = 1.0;
        active[j] = j;
        col_status[j] = COL_OK;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->n_active = p;
}

// One block per row of S^C (grid-stride over rows).
// With heat: per column, the count of off-diagonal standardised entries above
// heat_lam (see order_by_heat_kernel).
template <typename T>
__global__ void prep_matrix_kernel(const T* __restrict__ S, int p, int ldp, const double* cs,
                                   const float* csf, T* SC, T* GT, T* diag, int init_g,
                                   FitCtrl* ctrl, T heat_lam, int* heat, float* cmax) {
    bool bad = false;
    for (int r = blockIdx.x; r < p; r += gridDim.x) {
        int cnt = 0;
        bad |= standardize_row<T>(S, p, ldp, r, cs, csf, SC, init_g ? GT : nullptr, nullptr,
                                  diag, threadIdx.x, blockDim.x, heat_lam, heat ? &cnt : nullptr,
                                  cmax);
        if (cnt) atomicAdd(&heat[r], cnt);
    }
    if (bad) set_error(ctrl, DEV_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Theta: Omega_1 = -B D on the working scale (Eq. (4)), min-magnitude
// symmetrisation (Eq. (9); for j < k the tie keeps omega_jk) and
// Omega^o = C Omega C (Proposition 1), over pairs of mirrored output tiles
// whose coefficient tiles are read once into shared memory.  Also writes
// sigma in the original scale and counts nonzero b.
// ---------------------------------------------------------------------------
// Theta for one fit: one block per tile pair (see theta_pair).
template <typename T>
__global__ void theta_kernel(const T* __restrict__ BT, int p, int ldp,
                             const double* __restrict__ sigma, const double* __restrict__ cs,
                             double* __restrict__ Theta, double* __restrict__ sigma_out,
                             FitCtrl* ctrl) {
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    theta_pair<T>(BT, p, ldp, sigma, cs, Theta, sigma_out, ctrl, blockIdx.x);
}

// One regression r (spmesl_scaled_lasso): beta over the other columns in
// order, in the original scale (b^o_k = b^C_k c_k / c_r, proof of
// Proposition 1), sigma^o = sigma^C / c_r, nonzero coefficients counted.
template <typename T>
__global__ void lasso_export_kernel(const T* __restrict__ BT, int p, int ldp, int r,
                                    const double* __restrict__ sigma,
                                    const double* __restrict__ cs, double* __restrict__ beta,
                                    double* __restrict__ sigma_out, FitCtrl* ctrl) {
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const T* brow = BT + (size_t)r * ldp;
    bool nz = false;
    if (k < p && k != r) {
        const T b = brow[k];
        nz = b != T(0);
        beta[k < r ? k : k - 1] = (double)b * cs[k] / cs[r];
    }
    const unsigned cnt = __popc(__ballot_sync(FULL_MASK, nz));
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctrl->nnz, (unsigned long long)cnt);
    if (k == 0) sigma_out[0] = sigma[r] / cs[r];
}

// B[j][k] = b_jk in the original scale: b^o_jk = b^C_jk c_j / c_k.
template <typename T>
__global__ void export_b_kernel(const T* __restrict__ BT, int p, int ldp, const double* cs,
                                double* __restrict__ B) {
    __shared__ T tile[32][33];
    const int j0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int rr = ty; rr < 32; rr += 8) {
        const int k = k0 + rr, j = j0 + tx;
        tile[rr][tx] = (k < p && j < p) ? BT[(size_t)k * ldp + j] : T(0);
    }
    __syncthreads();
    const int k = k0 + tx;
    for (int rr = ty; rr < 32; rr += 8) {
        const int j = j0 + rr;
        if (j < p && k < p) B[(size_t)j * p + k] = (double)tile[tx][rr] * cs[j] / cs[k];
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int g_num_sms = 0;
static int g_max_smem_block = 0;
static int g_max_smem_sm = 0;

static cudaError_t device_limits() {
    if (g_num_sms) return cudaSuccess;
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&g_max_smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&g_max_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return cudaGetLastError();
}

// Shared memory a block may take (leave room for the small static arrays).
static size_t smem_budget() { return (size_t)g_max_smem_block - 1024; }

int max_p_for(int precision) {
    // one warp of the eager solver needs warp_smem_bytes(ldp) of shared
    // memory and one block of the block solver block_smem_bytes(ldp); the
    // opt-in block limit on GB300 is 227 KB.
    const size_t budget = 232448 - 1024;
    int p = 32;
    if (precision == SPMESL_FP64) {
        while (warp_smem_bytes<double>(p + 32) <= budget && block_smem_bytes<double>(p + 32) <= budget)
            p += 32;
    } else {
        while (warp_smem_bytes<float>(p + 32) <= budget && block_smem_bytes<float>(p + 32) <= budget)
            p += 32;
    }
    return p;
}

// Side stream and fork/join events of the calling thread on the current
// device, for the block solver's launch over the heavy columns beside the lazy
// launch.  One set per thread and device, so the fork/join records of fits
// issued from different threads cannot interleave; they live as long as the
// process.
namespace {
struct SideRes {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxSideDevices = 64;
}  // namespace

static cudaError_t side_resources(SideRes** out) {
    thread_local SideRes res[kMaxSideDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxSideDevices) return cudaErrorInvalidDevice;
    SideRes& r = res[dev];
    if (!r.s) {
        if ((e = cudaStreamCreateWithFlags(&r.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&r.join, cudaEventDisableTiming)) != cudaSuccess)
            return e;
    }
    *out = &r;
    return cudaSuccess;
}

// ctrl->n_heavy = 1 when the one column of a single regression is heavy.
__global__ void heavy_flag_kernel(const int* __restrict__ heat, int* __restrict__ n_heavy,
                                  int heavy_heat) {
    if (threadIdx.x == 0) *n_heavy = heat[0] > heavy_heat ? 1 : 0;
}

// Persistent grid of the block solver for this size.
template <typename T, bool STD>
static cudaError_t block_launch_shape(int ldp, size_t& smem, int& grid) {
    auto bk = cd_column_block_kernel<T, STD>;
    smem = block_smem_bytes<T>(ldp);
    if (smem > smem_budget()) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk, BLK_THREADS, smem)) !=
        cudaSuccess)
        return e;
    grid = g_num_sms * std::max(1, std::min(per_sm, 2));
    return cudaSuccess;
}

template <typename T>
static cudaError_t launch_diag(const CDArgs<T>& a, double eps, int j0, int j1, cudaStream_t st) {
    const size_t sm = diag_warp_smem_bytes() * DIAG_WARPS;
    auto k = cd_diag_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int cols = j1 - j0;
    const int grid = std::max(1, std::min((cols + DIAG_WARPS - 1) / DIAG_WARPS, g_num_sms * 4));
    k<<<grid, 32 * DIAG_WARPS, sm, st>>>(a, eps, j0, j1);
    return cudaGetLastError();
}

template <typename T, bool STD>
static cudaError_t run_fit(const FitLaunch& f, const FitLayout& L, cudaStream_t st) {
    cudaError_t e = device_limits();
    if (e != cudaSuccess) return e;
    unsigned char* ws = f.ws;
    FitCtrl* ctrl = reinterpret_cast<FitCtrl*>(ws + L.ctrl);
    CDArgs<T> a;
    a.SC = reinterpret_cast<const T*>(ws + L.SC);
    a.BT = reinterpret_cast<T*>(ws + L.BT);
    a.GT = reinterpret_cast<T*>(ws + L.GT);
    a.diag = reinterpret_cast<const T*>(ws + L.diag);
    a.sigma = reinterpret_cast<double*>(ws + L.sigma);
    a.col_status = reinterpret_cast<int*>(ws + L.col_status);
    a.active = reinterpret_cast<int*>(ws + L.active);
    a.active_next = reinterpret_cast<int*>(ws + L.active_next);
    a.flag = reinterpret_cast<int*>(ws + L.flag);
    a.ctrl = ctrl;
    a.p = f.p;
    a.ldp = L.ldp;
    a.maxit = f.maxit;
    a.lambda0 = f.lambda0;
    a.tol = f.tol;
    a.ovf_list = a.flag;            // the column rule does not use the flag array
    a.ovf_count = &ctrl->ovf_count;
    a.order = nullptr;
    a.n_queue = f.p;
    a.chunk_max = nullptr;
    a.rows_moved = f.count_rows ? reinterpret_cast<unsigned*>(ws + L.rows) : nullptr;
    a.rows_words = rows_words(f.p);
    // the hand-over record of the column rule lives in the joint rule's G matrix
    a.hand = reinterpret_cast<double*>(ws + L.GT);
    const bool single = f.response_col >= 0;    // one regression: lazy column rule
    const bool joint = !single && f.inner_rule == SPMESL_INNER_JOINT;
    // Lazy launch shape (warps per block, blocks per SM).
    const bool lazy = single || (!joint && f.gradient != SPMESL_GRADIENT_EAGER);
    // AUTO: heavy columns (heat above heavy_heat, in fits of at least
    // heavy_min_p columns) go to the block solver beside the lazy launch, and
    // the lazy solver hands over a column whose support outgrows its
    // active-set phase; LAZY: the lazy solver keeps every column its list can
    // hold.  Heat overstates the support of small fits, whose slices are cheap
    // anyway, so the routing by heat is kept to large fits.
    const bool route = lazy && f.gradient == SPMESL_GRADIENT_AUTO;
    a.ovf_supp = route ? handover_of(f.handover) : LAZY_CAP;
    auto lk = cd_column_lazy_kernel<T, STD>;
    const size_t lper = lazy_warp_smem_bytes<T>(L.ldp);
    int LW = f.warps_per_block > 0 ? f.warps_per_block : 8;
    LW = std::max(1, std::min({LW, 8, (int)(smem_budget() / lper)}));
    const size_t lsm = lper * LW;
    int lper_sm = 1;
    if (lazy) {
        if ((e = cudaFuncSetAttribute(lk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)lsm)) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lper_sm, lk, 32 * LW, lsm)) !=
            cudaSuccess)
            return e;
        lper_sm = std::max(lper_sm, 1);
    }
    // The lazy queue takes the columns heaviest first (standardised matrix)
    // when there are more columns than resident warps or when heavy columns
    // are routed.  The active index vectors are the joint rule's; the column
    // rule lends them to the heat counts and the order.
    const int hheat = heavy_heat_of(f.heavy_heat);
    const bool heavy = route && f.standardize && f.p >= heavy_min_p_of(f.heavy_min_p);
    const bool ordered = !single && lazy && f.standardize &&
                         (heavy || f.p > g_num_sms * lper_sm * LW);
    int* heat = (ordered || (single && heavy)) ? a.active_next : nullptr;
    // first-sweep chunk maxima (standardised lazy solves)
    float* cmax = (lazy && f.standardize) ? reinterpret_cast<float*>(ws + L.cmax) : nullptr;
    a.chunk_max = cmax;

    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(FitCtrl), st)) != cudaSuccess) return e;
    if (heat && (e = cudaMemsetAsync(heat, 0, sizeof(int) * (size_t)f.p, st)) != cudaSuccess)
        return e;
    // the joint rule keeps B in memory from B = 0; the column solvers write
    // every row of B whole
    if (joint &&
        (e = cudaMemsetAsync(ws + L.BT, 0, (size_t)f.p * L.ldp * sizeof(T), st)) != cudaSuccess)
        return e;
    if (a.rows_moved &&
        (e = cudaMemsetAsync(a.rows_moved, 0, rows_bitmap_bytes(f.p), st)) != cudaSuccess)
        return e;
    const int pb = 256;
    prep_diag_kernel<T><<<(f.p + pb - 1) / pb, pb, 0, st>>>(
        reinterpret_cast<const T*>(f.S), f.p, f.standardize, reinterpret_cast<double*>(ws + L.cs),
        reinterpret_cast<float*>(ws + L.csf), a.sigma, a.active, a.col_status, ctrl);
    {
        const int grid = std::min(f.p, g_num_sms * 8);
        prep_matrix_kernel<T><<<grid, pb, 0, st>>>(
            reinterpret_cast<const T*>(f.S), f.p, L.ldp, reinterpret_cast<double*>(ws + L.cs),
            reinterpret_cast<const float*>(ws + L.csf), reinterpret_cast<T*>(ws + L.SC), a.GT,
            reinterpret_cast<T*>(ws + L.diag), joint ? 1 : 0, ctrl, (T)f.lambda0, heat, cmax);
    }
    if (ordered) {
        order_by_heat_kernel<<<1, 1024, 0, st>>>(heat, f.p, a.active, heavy ? &ctrl->n_heavy : nullptr,
                                                 hheat);
        a.order = a.active;
    }
    if (single) {
        // a queue of one column: active[j] = j after prep_diag_kernel
        a.order = a.active + f.response_col;
        a.n_queue = 1;
        if (heavy) heavy_flag_kernel<<<1, 32, 0, st>>>(heat + f.response_col, &ctrl->n_heavy, hheat);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // warps per block: spread columns over the SMs, bounded by shared memory
    const size_t per_warp = warp_smem_bytes<T>(L.ldp);
    int wmax = (int)std::min<size_t>(16, smem_budget() / per_warp);
    if (wmax < 1) return cudaErrorInvalidValue;
    // Automatic shape: one block per SM holding ceil(p / #SM) warps, but
    // shared memory capped at about half of the SM so the rest of the unified
    // L1 keeps the few S rows a long-running column re-reads every sweep.
    const bool auto_shape = f.warps_per_block <= 0;
    int W = (f.p + g_num_sms - 1) / g_num_sms;
    if (auto_shape) W = std::min(W, (int)std::max<size_t>(1, (smem_budget() / 2) / per_warp));
    else W = f.warps_per_block;
    W = std::max(1, std::min(W, wmax));
    const size_t smem = per_warp * W;
    const int threads = 32 * W;

    if (f.phase_events) cudaEventRecord(f.phase_events[0], st);
    if (!joint) {
        if (lazy) {
            size_t bsm = 0;
            int bgrid = 0;
            if ((e = block_launch_shape<T, STD>(L.ldp, bsm, bgrid)) != cudaSuccess) return e;
            auto bk = cd_column_block_kernel<T, STD>;
            SideRes* side = nullptr;
            if (heavy) {
                // heavy columns on the block solver, beside the lazy launch
                if ((e = side_resources(&side)) != cudaSuccess) return e;
                if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(side->s, side->fork, 0)) != cudaSuccess)
                    return e;
                bk<<<single ? 1 : bgrid, BLK_THREADS, bsm, side->s>>>(a, 0);
                if ((e = cudaEventRecord(side->join, side->s)) != cudaSuccess) return e;
            }
            // lazy gradient: small shared-memory footprint, many columns per SM
            if (single) {
                lk<<<1, 32, lper, st>>>(a);          // one warp for the one column
            } else {
                const int lgrid = std::min((f.p + LW - 1) / LW, g_num_sms * lper_sm);
                lk<<<lgrid, 32 * LW, lsm, st>>>(a);
            }
            // the columns the lazy solver handed over
            bk<<<single ? 1 : bgrid, BLK_THREADS, bsm, st>>>(a, 1);
            if (heavy && (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess) return e;
        } else {
            // eager gradient for every column
            auto kern = cd_column_kernel<T, STD>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess)
                return e;
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) !=
                cudaSuccess)
                return e;
            per_sm = auto_shape ? 1 : std::max(per_sm, 1);
            const int grid = std::min((f.p + W - 1) / W, g_num_sms * per_sm);
            kern<<<grid, threads, smem, st>>>(a, 0);
        }
    } else {
        auto kern = cd_joint_kernel<T, STD>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) !=
            cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int grid = std::min((f.p + W - 1) / W, g_num_sms * per_sm);
        void* args[] = {&a};
        if ((e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args,
                                             smem, st)) != cudaSuccess)
            return e;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (f.phase_events) cudaEventRecord(f.phase_events[1], st);
    if (a.rows_moved)
        rows_count_kernel<<<g_num_sms, 256, 0, st>>>(a.rows_moved, rows_bitmap_bytes(f.p) / 4, ctrl);
    if (f.diagnostics) {
        const int j0 = single ? f.response_col : 0, j1 = single ? f.response_col + 1 : f.p;
        if ((e = launch_diag<T>(a, f.diag_eps, j0, j1, st)) != cudaSuccess) return e;
    }

    if (single) {
        lasso_export_kernel<T><<<(f.p + 255) / 256, 256, 0, st>>>(
            a.BT, f.p, L.ldp, f.response_col, a.sigma, reinterpret_cast<const double*>(ws + L.cs),
            f.beta_out, f.sigma_out, ctrl);
        if (f.phase_events) cudaEventRecord(f.phase_events[2], st);
        return cudaGetLastError();
    }
    theta_kernel<T><<<theta_pairs<T>(f.p), dim3(32, 8), 0, st>>>(a.BT, f.p, L.ldp, a.sigma,
                                       reinterpret_cast<const double*>(ws + L.cs), f.Theta,
                                       f.sigma_out, ctrl);
    if (f.phase_events) cudaEventRecord(f.phase_events[2], st);
    return cudaGetLastError();
}

cudaError_t launch_fit(const FitLaunch& f, cudaStream_t st) {
    const FitLayout L = fit_layout(f.p, f.precision);
    if (f.precision == SPMESL_FP64) {
        return f.standardize ? run_fit<double, true>(f, L, st) : run_fit<double, false>(f, L, st);
    }
    return f.standardize ? run_fit<float, true>(f, L, st) : run_fit<float, false>(f, L, st);
}

template <typename T>
static cudaError_t run_diagnose(const void* S, int p, int standardize, double lambda0,
                                const double* B, const double* sigma, double eps,
                                unsigned char* ws, const FitLayout& L, cudaStream_t st) {
    cudaError_t e = device_limits();
    if (e != cudaSuccess) return e;
    FitCtrl* ctrl = reinterpret_cast<FitCtrl*>(ws + L.ctrl);
    double* cs = reinterpret_cast<double*>(ws + L.cs);
    CDArgs<T> a{};
    a.SC = reinterpret_cast<const T*>(ws + L.SC);
    a.BT = reinterpret_cast<T*>(ws + L.BT);
    a.diag = reinterpret_cast<const T*>(ws + L.diag);
    a.sigma = reinterpret_cast<double*>(ws + L.sigma);
    a.ctrl = ctrl;
    a.p = p;
    a.ldp = L.ldp;
    a.lambda0 = lambda0;
    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(FitCtrl), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + L.BT, 0, (size_t)p * L.ldp * sizeof(T), st)) != cudaSuccess)
        return e;
    const int pb = 256;
    prep_diag_kernel<T><<<(p + pb - 1) / pb, pb, 0, st>>>(
        reinterpret_cast<const T*>(S), p, standardize, cs, reinterpret_cast<float*>(ws + L.csf),
        a.sigma, reinterpret_cast<int*>(ws + L.active), reinterpret_cast<int*>(ws + L.col_status),
        ctrl);
    prep_matrix_kernel<T><<<std::min(p, g_num_sms * 8), pb, 0, st>>>(
        reinterpret_cast<const T*>(S), p, L.ldp, cs, reinterpret_cast<const float*>(ws + L.csf),
        reinterpret_cast<T*>(ws + L.SC), nullptr, reinterpret_cast<T*>(ws + L.diag), 0, ctrl, T(0),
        nullptr, nullptr);
    const size_t total = (size_t)p * p;
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)g_num_sms * 16);
    load_estimate_kernel<T><<<grid, 256, 0, st>>>(B, sigma, p, L.ldp, cs, a.BT, a.sigma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_diag<T>(a, eps, 0, p, st);
}

cudaError_t launch_diagnose(const void* S, int p, int precision, int standardize,
                            double lambda0, const double* B, const double* sigma, double eps,
                            unsigned char* ws, cudaStream_t st) {
    const FitLayout L = fit_layout(p, precision);
    if (precision == SPMESL_FP64)
        return run_diagnose<double>(S, p, standardize, lambda0, B, sigma, eps, ws, L, st);
    return run_diagnose<float>(S, p, standardize, lambda0, B, sigma, eps, ws, L, st);
}

cudaError_t launch_export_B(const unsigned char* ws, int p, int precision, double* B,
                            cudaStream_t st) {
    const FitLayout L = fit_layout(p, precision);
    dim3 tb(32, 8), tg((p + 31) / 32, (p + 31) / 32);
    const double* cs = reinterpret_cast<const double*>(ws + L.cs);
    if (precision == SPMESL_FP64)
        export_b_kernel<double><<<tg, tb, 0, st>>>(reinterpret_cast<const double*>(ws + L.BT), p,
                                                   L.ldp, cs, B);
    else
        export_b_kernel<float><<<tg, tb, 0, st>>>(reinterpret_cast<const float*>(ws + L.BT), p,
                                                  L.ldp, cs, B);
    return cudaGetLastError();
}

}  // namespace spmesl
