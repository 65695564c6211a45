#pragma once
// Device building blocks of the coordinate-descent fit, shared by the single-fit
// kernels (cd.cu) and the batched kernels (batch.cu).
#include <cuda_runtime.h>
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

// Per-warp counters of the column solves, flushed into a fit's FitCtrl.
struct ColCounters {
    unsigned long long sweeps = 0, moves = 0;
    int outer_max = 0, n_nc = 0, n_deg = 0, max_sw = 0;
};

__device__ __forceinline__ void flush_counters(FitCtrl* ctrl, ColCounters& c) {
    if ((threadIdx.x & 31) == 0) {
        if (c.sweeps) atomicAdd(&ctrl->total_sweeps, c.sweeps);
        if (c.moves) atomicAdd(&ctrl->moves, c.moves);
        atomicMax(&ctrl->outer_max, c.outer_max);
        atomicMax(&ctrl->max_col_sweeps, c.max_sw);
        if (c.n_nc) atomicAdd(&ctrl->n_not_converged, c.n_nc);
        if (c.n_deg) atomicAdd(&ctrl->n_degenerate, c.n_deg);
    }
    c = ColCounters();
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
    __syncwarp();

    double sigma = 1.0;                                  // sigma^(0) = 1
    const unsigned long long sweeps0 = cnt.sweeps;
    const double floor2 = 1e-12 * (double)a.SC[(size_t)j * a.ldp + j];
    int status = COL_OK;
    int r;
    for (r = 0; r < a.maxit; ++r) {
        const T lam = (T)(sigma * a.lambda0);
        bool inner_ok = false;
        for (int m = 0; m < a.maxit; ++m) {
            const T md = sweep_column<T, STD>(j, g, b, a, lam, cnt.moves);
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
    cnt.outer_max = max(cnt.outer_max, r + 1);
    cnt.max_sw = max(cnt.max_sw, (int)(cnt.sweeps - sweeps0));
    cnt.n_nc += (status & COL_NOT_CONVERGED) != 0;
    cnt.n_deg += (status & COL_DEGENERATE) != 0;
    __syncwarp();
}

// One 32 x 32 tile (rows j0.., columns k0..) of Theta: Omega_1 = -B D on the
// working scale (Eq. (4)), min-magnitude symmetrisation (Eq. (9); for j < k a
// tie keeps omega_jk) and Omega^o = C Omega C (Proposition 1).  The
// transposed coefficient tile goes through shared memory so both reads are
// coalesced.  Blocks of the tile row j0 = 0 also write sigma in the original
// scale; nonzero coefficients are counted into ctrl->nnz.  Block shape 32 x 8.
template <typename T>
__device__ void theta_tile(const T* __restrict__ BT, int p, int ldp,
                          const double* __restrict__ sigma, const double* __restrict__ cs,
                          double* __restrict__ Theta, double* __restrict__ sigma_out,
                          FitCtrl* ctrl, int j0, int k0) {
    __shared__ T tileA[32][33];   // tileA[kk][jj] = BT[k0+kk][j0+jj] = b_{j,k}
    // 1/sigma^2 and c for the tile's 32 columns k and 32 rows j: FP64
    // divisions are expensive on this part, so each block does 64 of them
    // instead of one per element
    __shared__ double inv_k[32], inv_j[32], c_k[32], c_j[32];
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
    if (j0 == 0 && ty == 0 && k < p) sigma_out[k] = sigma[k] / cs[k];
    // one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(FULL_MASK, nnz, o);
    if (tx == 0 && nnz) atomicAdd(&ctrl->nnz, nnz);
}

}  // namespace spmesl
