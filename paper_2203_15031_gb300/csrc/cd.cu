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
};

template <typename T>
__device__ __forceinline__ T soft(T x, T lam) {
    // Soft_lambda(x) = sign(x) (|x| - lambda)_+   (Section 3.1)
    return x > lam ? x - lam : (x < -lam ? x + lam : T(0));
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
// covers 128 coordinates; the first coordinate whose update changes b is
// applied and the scan resumes right after it.
constexpr int SCAN_V = 4;

template <typename T, bool STD>
__device__ T sweep_column(int j, T* __restrict__ g, T* __restrict__ b, const CDArgs<T>& a, T lam,
                          unsigned long long& moves) {
    const int lane = threadIdx.x & 31;
    const int p = a.p;
    const int ldp = a.ldp;
    T maxd = T(0);
    int cursor = 0;
    while (cursor < p) {
        const int base = cursor & ~(SCAN_V - 1);
        const int k0 = base + lane * SCAN_V;
        T gv[SCAN_V], bv[SCAN_V], nbv[SCAN_V];
        if (k0 < ldp) {                       // ldp is a multiple of 32: the whole quad is in range
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
        if (bal == 0u) {
            cursor = base + 32 * SCAN_V;
            continue;
        }
        const int f = __ffs(bal) - 1;
        const int tf = __ffs(__shfl_sync(FULL_MASK, mvmask, f)) - 1;
        T nb_sel = nbv[0], b_sel = bv[0];
#pragma unroll
        for (int t = 1; t < SCAN_V; ++t)
            if (t == tf) { nb_sel = nbv[t]; b_sel = bv[t]; }
        const T nbs = __shfl_sync(FULL_MASK, nb_sel, f);
        const T delta = nbs - __shfl_sync(FULL_MASK, b_sel, f);
        const int ks = base + f * SCAN_V + tf;
        if (lane == 0) b[ks] = nbs;
        maxd = fmax(maxd, fabs(delta));
        ++moves;
        axpy_row<T>(g, a.SC + (size_t)ks * ldp, delta, ldp);
        __syncwarp();
        cursor = ks + 1;
    }
    return maxd;
}

// sigma_j^2 = S_jj - 2 b'S_.j + b'S b in FP64 over the support of b
// (Eq. (14) written on S).  Same value in every lane.
// Per-warp scratch for the support list used by the sigma update.
constexpr int SUPP_CAP = 128;

// Shared memory of one warp: g_j and b_j (ldp elements each) and the list.
template <typename T>
__host__ __device__ constexpr size_t warp_smem_bytes(int ldp) {
    return 2 * (size_t)ldp * sizeof(T) + SUPP_CAP * sizeof(int);
}

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
            lin += (double)b[k] * (double)a.SC[(size_t)k * a.ldp + j];
        }
        for (int t = lane; t < ns * ns; t += 32) {
            const int k = list[t / ns], l = list[t % ns];
            quad += (double)b[k] * (double)b[l] * (double)a.SC[(size_t)k * a.ldp + l];
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

// ---------------------------------------------------------------------------
// Per-column rule (Algorithms 1-2): every warp takes the next unsolved column
// and runs the whole scaled lasso for it; no grid-wide synchronisation.
// ---------------------------------------------------------------------------
template <typename T, bool STD>
__global__ void __launch_bounds__(512) cd_column_kernel(CDArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T* g = reinterpret_cast<T*>(smem_raw + (size_t)warp * warp_smem_bytes<T>(a.ldp));
    T* b = g + a.ldp;
    int* list = reinterpret_cast<int*>(b + a.ldp);
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;

    unsigned long long sweeps = 0, moves = 0;
    int outer_max = 0, n_nc = 0, n_deg = 0, max_sw = 0;
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(&ctrl->next_col, 1);
        j = __shfl_sync(FULL_MASK, j, 0);
        if (j >= a.p) break;

        warp_copy<T>(g, a.SC + (size_t)j * a.ldp, a.ldp);   // g = S_.j  (b = 0)
        warp_zero<T>(b, a.ldp);
        __syncwarp();

        double sigma = 1.0;                                  // sigma^(0) = 1
        const unsigned long long sweeps0 = sweeps;
        const double floor2 = 1e-12 * (double)a.SC[(size_t)j * a.ldp + j];
        int status = COL_OK;
        int r;
        for (r = 0; r < a.maxit; ++r) {
            const T lam = (T)(sigma * a.lambda0);
            bool inner_ok = false;
            for (int m = 0; m < a.maxit; ++m) {
                const T md = sweep_column<T, STD>(j, g, b, a, lam, moves);
                ++sweeps;
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
            const double sn = sqrt(q);
            const double ds = fabs(sn - sigma);
            sigma = sn;
            if (ds < a.tol) break;
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
        outer_max = max(outer_max, r + 1);
        max_sw = max(max_sw, (int)(sweeps - sweeps0));
        n_nc += (status & COL_NOT_CONVERGED) != 0;
        n_deg += (status & COL_DEGENERATE) != 0;
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&ctrl->total_sweeps, sweeps);
        atomicAdd(&ctrl->moves, moves);
        atomicMax(&ctrl->outer_max, outer_max);
        atomicMax(&ctrl->max_col_sweeps, max_sw);
        if (n_nc) atomicAdd(&ctrl->n_not_converged, n_nc);
        if (n_deg) atomicAdd(&ctrl->n_degenerate, n_deg);
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
                wmax = fmax(wmax, sweep_column<T, STD>(j, g, b, a, lam, moves));
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
                                 double* sigma, int* active, int* col_status, FitCtrl* ctrl) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x) {
        const double d = (double)S[(size_t)j * p + j];
        if (!(d > 0.0) || !isfinite(d)) set_error(ctrl, DEV_ERR_NONFINITE);
        cs[j] = standardize ? 1.0 / sqrt(d) : 1.0;
        sigma[j] = 1.0;
        active[j] = j;
        col_status[j] = COL_OK;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->n_active = p;
}

template <typename T>
__global__ void prep_matrix_kernel(const T* __restrict__ S, int p, int ldp, const double* cs,
                                   T* SC, T* GT, T* diag, int init_g, FitCtrl* ctrl) {
    const size_t total = (size_t)p * ldp;
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / ldp), c = (int)(i % ldp);
        T v = T(0);
        if (c < p) {
            const T s = S[(size_t)r * p + c];
            bad |= !isfinite((double)s);
            v = (T)((double)s * cs[r] * cs[c]);
            if (c == r) diag[r] = v;
        }
        SC[i] = v;
        if (init_g) GT[i] = v;
    }
    if (bad) set_error(ctrl, DEV_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Theta: Omega_1 = -B D on the working scale (Eq. (4)), min-magnitude
// symmetrisation (Eq. (9); for j < k the tie keeps omega_jk) and
// Omega^o = C Omega C (Proposition 1).  32x32 output tiles; the transposed
// coefficient tile goes through shared memory so both reads are coalesced.
// Also writes sigma in the original scale and counts nonzero b.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void theta_kernel(const T* __restrict__ BT, int p, int ldp,
                             const double* __restrict__ sigma, const double* __restrict__ cs,
                             double* __restrict__ Theta, double* __restrict__ sigma_out,
                             FitCtrl* ctrl) {
    __shared__ T tileA[32][33];   // tileA[kk][jj] = BT[k0+kk][j0+jj] = b_{j,k}
    // 1/sigma^2 and c for the tile's 32 columns k and 32 rows j: FP64
    // divisions are expensive on this part, so each block does 64 of them
    // instead of one per element
    __shared__ double inv_k[32], inv_j[32], c_k[32], c_j[32];
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    const int j0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    if (ty < 2) {
        const int i = (ty == 0 ? k0 : j0) + tx;
        double inv = 0.0, c = 0.0;
        if (i < p) {
            const double s = sigma[i];
            inv = 1.0 / (s * s);
            c = cs[i];
        }
        if (ty == 0) { inv_k[tx] = inv; c_k[tx] = c; }
        else { inv_j[tx] = inv; c_j[tx] = c; }
    }
    for (int rr = ty; rr < 32; rr += 8) {
        const int k = k0 + rr, j = j0 + tx;
        tileA[rr][tx] = (k < p && j < p) ? BT[(size_t)k * ldp + j] : T(0);
    }
    __syncthreads();
    unsigned long long nnz = 0;
    const int k = k0 + tx;
    for (int rr = ty; rr < 32; rr += 8) {
        const int j = j0 + rr;
        if (j >= p || k >= p) continue;
        double out;
        if (j == k) {
            out = inv_k[tx];
        } else {
            const T bjk = tileA[tx][rr];                       // coefficient of x_j in regression k
            const T bkj = BT[(size_t)j * ldp + k];             // coefficient of x_k in regression j
            nnz += (bkj != T(0));
            if (bjk == T(0) && bkj == T(0)) {
                out = 0.0;                                     // both candidates are zero
            } else {
                const double ojk = -(double)bjk * inv_k[tx];   // Omega_1[j][k]
                const double okj = -(double)bkj * inv_j[rr];   // Omega_1[k][j]
                if (j < k) out = fabs(ojk) > fabs(okj) ? okj : ojk;
                else out = fabs(okj) > fabs(ojk) ? ojk : okj;  // pair (k, j) with k < j
                out *= c_j[rr] * c_k[tx];
            }
        }
        if (j == k) out *= c_j[rr] * c_k[tx];
        // the scale (c_j c_k) is formed before it multiplies, so (j, k) and
        // (k, j) get bit-identical values and the result is exactly symmetric
        Theta[(size_t)j * p + k] = out;
    }
    if (blockIdx.y == 0 && ty == 0 && k < p) sigma_out[k] = sigma[k] / cs[k];
    // one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(FULL_MASK, nnz, o);
    if (tx == 0 && nnz) atomicAdd(&ctrl->nnz, nnz);
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
    // one warp needs g and b: 2 * ldp * s bytes; the opt-in block limit on
    // GB300 is 227 KB.
    const size_t budget = 232448 - 1024 - SUPP_CAP * sizeof(int);
    const size_t s = (size_t)elem_size(precision);
    int p = (int)(budget / (2 * s));
    return p / 32 * 32;
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
    const bool joint = f.inner_rule == SPMESL_INNER_JOINT;

    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(FitCtrl), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + L.BT, 0, (size_t)f.p * L.ldp * sizeof(T), st)) != cudaSuccess)
        return e;
    const int pb = 256;
    prep_diag_kernel<T><<<(f.p + pb - 1) / pb, pb, 0, st>>>(
        reinterpret_cast<const T*>(f.S), f.p, f.standardize, reinterpret_cast<double*>(ws + L.cs),
        a.sigma, a.active, a.col_status, ctrl);
    {
        const size_t total = (size_t)f.p * L.ldp;
        int grid = (int)std::min<size_t>((total + pb - 1) / pb, (size_t)g_num_sms * 16);
        prep_matrix_kernel<T><<<grid, pb, 0, st>>>(
            reinterpret_cast<const T*>(f.S), f.p, L.ldp, reinterpret_cast<double*>(ws + L.cs),
            reinterpret_cast<T*>(ws + L.SC), a.GT, reinterpret_cast<T*>(ws + L.diag), joint ? 1 : 0,
            ctrl);
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
        kern<<<grid, threads, smem, st>>>(a);
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

    dim3 tb(32, 8), tg((f.p + 31) / 32, (f.p + 31) / 32);
    theta_kernel<T><<<tg, tb, 0, st>>>(a.BT, f.p, L.ldp, a.sigma,
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
