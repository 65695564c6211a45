// Coordinate descent for SPMESL in the residual form, without the Gram
// matrix (sm_103a).  Algorithm 3 keeps the residual matrix E = X - X B and
// forms each coordinate's gradient from the data (a_kj = x_k' e_j / n), and
// Proposition 2 updates E by a rank-1 term after every move; this file runs
// that form per column, with the cyclic ascending order and the per-column
// stopping rule of Algorithm 1.
//
// Layout in HBM (see res_layout):
//   W   ldn x ldp  W[i][k] = w_k[i], the scaled data, rows past n and columns
//                  past p zero
//   Wt  p x ldn    Wt[k][i] = w_k[i] (the same values, transposed)
//   BT  p x ldp    row j = coefficients b_.j of regression j
// with w_k = (x_k - mu_k) c_k / sqrt(n), c_k = s_kk^-1/2 when standardising
// (else 1), so that w_k' w_l = S^C_kl: the working matrix of the covariance
// form is never formed.  Memory is O(n p) for the data plus the p x p
// coefficients; the covariance form needs three p x p matrices besides S.
//
// One warp solves one column j at a time and keeps its residual
// r_j = w_j - W b_j (n values) in shared memory, with the sorted support of
// b_j and per-chunk summaries.  The gradient of coordinate k is
// g_kj = w_k' r_j, the same quantity S^C_kj - S^C_k. b_j that the covariance
// form keeps.  A sweep walks 128-coordinate chunks: the chunk's slice of g_j
// is W[:, chunk]' r_j (n coalesced 512-byte row reads, r_j broadcast from
// shared memory), the first coordinate that moves is found by ballot, its
// move updates r_j -= w_k delta from row k of Wt, and the slice is formed
// again from the new r_j.  sigma_j^2 = ||r_j||^2 (Eq. (14)) is formed in FP64
// from a residual recomputed from the data, which also removes the rounding
// drift of the running r_j.  No active-set phase: the iterates are those of
// plain cyclic sweeps (Algorithm 1).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cd_device.cuh"

namespace spmesl {
namespace {

constexpr int RES_MAX_N = 16384;   // the skip margins below assume n <= 2^14

template <typename T>
struct ResArgs {
    const T* W;
    const T* Wt;
    T* BT;
    const T* diag;       // ||w_k||^2 (unstandardised update)
    double* sigma;       // working-scale sigma
    int* col_status;
    FitCtrl* ctrl;
    int n, ldn, p, ldp, maxit;
    double lambda0, tol;
};

// Upper bounds on ||r_j|| (warp-uniform): rb now, rmax over the solve so far.
struct ResNorm {
    float rb, rmax;
};

template <typename T>
__host__ __device__ constexpr size_t res_warp_smem_bytes(int ldn, int ldp) {
    return (size_t)ldn * sizeof(T) + (size_t)LAZY_CAP * (sizeof(int) + sizeof(T)) +
           (size_t)num_chunks(ldp) * sizeof(ChunkInfo);
}

template <typename T>
__device__ __forceinline__ void lds4(const T* __restrict__ src, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(src);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(src);
        const double2 q1 = *reinterpret_cast<const double2*>(src + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}

// acc[t] = sum_i W[i][k0 + t] r[i] over i < n4 (a multiple of 4; rows of W
// and entries of r past n are zero).  Two interleaved partial sums.
template <typename T>
__device__ __forceinline__ void slice_dot(const T* __restrict__ W, int ldp, int n4, int k0,
                                          const T* __restrict__ r, T (&acc)[SCAN_V]) {
    T a0[SCAN_V] = {T(0), T(0), T(0), T(0)}, a1[SCAN_V] = {T(0), T(0), T(0), T(0)};
    const T* w = W + k0;
#pragma unroll 2
    for (int i = 0; i < n4; i += 4) {
        T rv[4];
        lds4<T>(r + i, rv);
        T z0[SCAN_V], z1[SCAN_V], z2[SCAN_V], z3[SCAN_V];
        load4g<T>(w + (size_t)i * ldp, z0);
        load4g<T>(w + (size_t)(i + 1) * ldp, z1);
        load4g<T>(w + (size_t)(i + 2) * ldp, z2);
        load4g<T>(w + (size_t)(i + 3) * ldp, z3);
#pragma unroll
        for (int t = 0; t < SCAN_V; ++t) {
            a0[t] = fma(z0[t], rv[0], a0[t]);
            a1[t] = fma(z1[t], rv[1], a1[t]);
            a0[t] = fma(z2[t], rv[2], a0[t]);
            a1[t] = fma(z3[t], rv[3], a1[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < SCAN_V; ++t) acc[t] = a0[t] + a1[t];
}

// Chunks of [from, from + 32) that the sweep must scan (standardised data).
// A chunk with no support is skipped when none of its coordinates can reach
// the threshold.  Since the chunk was scanned, each move delta_m changed the
// exact dot w_k' r by at most |delta_m| ||w_k|| ||w_m|| <= |delta_m| (1 + 2^-21)
// plus the rounding of the r update (2^-24 ||r||), and each residual
// recomputation was entered as a move of size ||r_new - r_old||; each of the
// two computed dots (then and now) is within n 2^-24 ||r|| of the exact one
// (Cauchy-Schwarz, ||w_k|| <= 1 + 2^-22).  With rmax bounding ||r|| over the
// solve, the margins below cover these terms, the rounding of the running
// sum (as in chunk_skippable) and of the bound itself.  A skipped coordinate
// would therefore have computed |g_k| < lambda with b_k = 0 and not moved:
// the sweep is the same as a full scan.
template <bool STD>
__device__ __forceinline__ unsigned res_chunks_to_scan(const ColScan& cs, int from, int nch,
                                                       float lam, float rmax, int n) {
    const int ci = from + (int)(threadIdx.x & 31);
    bool need = ci < nch;
    if constexpr (STD) {
        if (need) {
            const ChunkInfo c = cs.ci[ci];
            const unsigned dm = cs.nmoves - c.moves_at;
            if (c.nsupp == 0 && dm <= 4096u) {
                const float bound = c.maxabs * (1.0f + 0x1p-22f) +
                                    (cs.dsum - c.dsum_at) * (1.0f + 0x1p-10f) +
                                    cs.dsum * (float)(dm + 2u) * 0x1p-23f +
                                    rmax * (float)(n + (int)dm + 2) * 0x1p-22f + lam * 0x1p-20f;
                need = !(bound < lam);
            }
        }
    }
    return __ballot_sync(FULL_MASK, need);
}

// One sweep over all coordinates of column j; returns max |delta b|.  Sets
// `overflow` and stops if the support list is full (the move is not applied).
template <typename T, bool STD>
__device__ T sweep_residual(int j, Support<T>& s, T* __restrict__ r, const ResArgs<T>& a, T lam,
                            unsigned long long& moves, ColScan& cs, ResNorm& rn, bool& overflow) {
    const int lane = threadIdx.x & 31;
    const int p = a.p, ldp = a.ldp;
    const int n4 = (a.n + 3) & ~3;
    const int nch = (p + CHUNK - 1) / CHUNK;
    T maxd = T(0);
    int e0 = 0;
    int mbase = 0;
    unsigned mask = res_chunks_to_scan<STD>(cs, 0, nch, (float)lam, rn.rmax, a.n);
    for (;;) {
        if (mask == 0u) {
            mbase += 32;
            if (mbase >= nch) break;
            mask = res_chunks_to_scan<STD>(cs, mbase, nch, (float)lam, rn.rmax, a.n);
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
        T acc[SCAN_V] = {T(0), T(0), T(0), T(0)};
        if (in) slice_dot<T>(a.W, ldp, n4, k0, r, acc);
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
                if (k >= cursor && k < p && k != j) {
                    T nb;
                    if constexpr (STD) {
                        nb = soft<T>(acc[t] + bv[t], lam);                 // ||w_k||^2 = 1
                    } else {
                        const T dk = a.diag[k];
                        nb = soft<T>(acc[t] + dk * bv[t], lam) / dk;       // Soft(c, lambda)/S_kk
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
            if (lane == f) {
#pragma unroll
                for (int u = 0; u < SCAN_V; ++u)
                    if (u == tf) bv[u] = nbs;
            }
            maxd = fmax(maxd, fabs(delta));
            ++moves;
            cs.dsum += fabsf((float)delta);
            ++cs.nmoves;
            rn.rb = (rn.rb + fabsf((float)delta)) * (1.0f + 0x1p-19f);
            rn.rmax = fmaxf(rn.rmax, rn.rb);
            // Proposition 2: r_j -= w_k delta (row k of Wt)
            const T* wk = a.Wt + (size_t)ks * a.ldn;
            for (int i = lane; i < a.n; i += 32) r[i] = fma(-delta, wk[i], r[i]);
            __syncwarp();
            cursor = ks + 1;
            if (cursor >= cb + CHUNK) break;
            // the slice again from the new residual (every lane, so that the
            // chunk summary below refers to one residual)
            if (in) slice_dot<T>(a.W, ldp, n4, k0, r, acc);
        }
        if constexpr (STD) {
            // the summary must describe the residual after the chunk's last
            // move: a move at the chunk's end left the slice one move behind
            if (cursor >= cb + CHUNK && cs.nmoves != nmoves0 && in)
                slice_dot<T>(a.W, ldp, n4, k0, r, acc);
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
            if (cs.nmoves != nmoves0) {
                mbase = ci + 1;
                if (mbase >= nch) break;
                mask = res_chunks_to_scan<STD>(cs, mbase, nch, (float)lam, rn.rmax, a.n);
            }
        } else {
            __syncwarp();
        }
    }
    return maxd;
}

// r_j = w_j - sum_{k in support} w_k b_k recomputed from the data in the data
// precision (lanes over samples), sigma_j^2 = ||r_j||^2 summed in FP64
// (Eq. (14): ||x_j - X b_j||^2 / n on the working scale), and in `dr` the
// distance between the new and the running residual.
template <typename T>
__device__ double residual_reset(int j, const Support<T>& s, T* __restrict__ r,
                                 const ResArgs<T>& a, double& dr) {
    const int lane = threadIdx.x & 31;
    const T* wj = a.Wt + (size_t)j * a.ldn;
    double q = 0.0, d2 = 0.0;
    for (int i = lane; i < a.n; i += 32) {
        T v = wj[i];
#pragma unroll 4
        for (int e = 0; e < s.n; ++e) v = fma(-s.val[e], a.Wt[(size_t)s.idx[e] * a.ldn + i], v);
        const double dv = (double)v;
        q = fma(dv, dv, q);
        const double dd = dv - (double)r[i];
        d2 = fma(dd, dd, d2);
        r[i] = v;
    }
    q = warp_sum(q);
    d2 = warp_sum(d2);
    __syncwarp();
    dr = sqrt(d2);
    return q;
}

// Algorithm 1 for column j in the residual form.
template <typename T, bool STD>
__device__ void solve_column_residual(int j, unsigned char* wsm, const ResArgs<T>& a,
                                      ColCounters& cnt) {
    const int lane = threadIdx.x & 31;
    T* r = reinterpret_cast<T*>(wsm);
    Support<T> s;
    s.idx = reinterpret_cast<int*>(wsm + (size_t)a.ldn * sizeof(T));
    s.val = reinterpret_cast<T*>(s.idx + LAZY_CAP);
    s.n = 0;
    ColScan cs{reinterpret_cast<ChunkInfo*>(s.val + LAZY_CAP), 0.f, 0u};
    reset_chunks(cs, a.ldp);
    // r_j = w_j (b = 0); rows of Wt are zero past n
    const T* wj = a.Wt + (size_t)j * a.ldn;
    double q0 = 0.0;
    for (int i = lane; i < a.ldn; i += 32) {
        const T v = wj[i];
        r[i] = v;
        q0 = fma((double)v, (double)v, q0);
    }
    q0 = warp_sum(q0);
    __syncwarp();
    ResNorm rn;
    rn.rb = (float)sqrt(q0) * (1.0f + 0x1p-20f);
    rn.rmax = rn.rb;

    double sigma = 1.0;                                  // sigma^(0) = 1, b = 0
    const unsigned long long sweeps0 = cnt.sweeps;
    const double floor2 = 1e-12 * q0;                    // S_jj of the working matrix
    int status = COL_OK;
    bool overflow = false;
    int it;
    for (it = 0; it < a.maxit; ++it) {
        const T lam = (T)(sigma * a.lambda0);
        bool inner_ok = false;
        for (int m = 0; m < a.maxit; ++m) {
            const T md = sweep_residual<T, STD>(j, s, r, a, lam, cnt.moves, cs, rn, overflow);
            ++cnt.sweeps;
            if (overflow) break;
            if ((double)md < a.tol) {
                inner_ok = true;
                break;
            }
        }
        if (overflow) {
            status |= COL_NOT_CONVERGED;          // support above the list's capacity
            break;
        }
        if (!inner_ok) status |= COL_NOT_CONVERGED;
        double dr;
        double q = residual_reset<T>(j, s, r, a, dr);
        // the recomputed residual moved r by dr: one move of that size for the
        // skip bound
        cs.dsum += (float)dr * (1.0f + 0x1p-8f);
        ++cs.nmoves;
        rn.rb = (float)sqrt(q) * (1.0f + 0x1p-20f);
        rn.rmax = fmaxf(rn.rmax, rn.rb);
        if (q <= floor2) {
            q = floor2;
            status |= COL_DEGENERATE;
        }
        const double sn = sqrt(q);
        const double ds = fabs(sn - sigma);
        sigma = sn;
        if (ds < a.tol) break;
    }
    if (it == a.maxit) {
        it = a.maxit - 1;
        status |= COL_NOT_CONVERGED;
    }
    T* brow = a.BT + (size_t)j * a.ldp;
    for (int t = lane; t < s.n; t += 32) brow[s.idx[t]] = s.val[t];
    if (lane == 0) {
        a.sigma[j] = sigma;
        a.col_status[j] = status;
    }
    cnt.outer_max = max(cnt.outer_max, it + 1);
    cnt.max_sw = max(cnt.max_sw, (int)(cnt.sweeps - sweeps0));
    cnt.n_nc += (status & COL_NOT_CONVERGED) != 0;
    cnt.n_deg += (status & COL_DEGENERATE) != 0;
    __syncwarp();
}

template <typename T, bool STD>
__global__ void __launch_bounds__(256) cd_residual_kernel(ResArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)warp * res_warp_smem_bytes<T>(a.ldn, a.ldp);
    FitCtrl* ctrl = a.ctrl;
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    ColCounters cnt;
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(&ctrl->next_col, 1);
        j = __shfl_sync(FULL_MASK, j, 0);
        if (j >= a.p) break;
        solve_column_residual<T, STD>(j, wsm, a, cnt);
    }
    flush_counters(ctrl, cnt);
}

// Per column k (one thread): mu_k (0 without centring), s_kk = ||x_k - mu_k||^2 / n
// in FP64, c_k = s_kk^-1/2 when standardising (else 1), the factor
// c_k / sqrt(n) that makes w_k, the working diagonal ||w_k||^2 = c_k^2 s_kk,
// and the starting sigma = 1.  Non-finite data or s_kk <= 0 sets
// DEV_ERR_NONFINITE.  Threads run along k, so every read of X is coalesced.
template <typename T>
__global__ void res_stats_kernel(const T* __restrict__ X, int n, int p, int ldx, int center,
                                 int standardize, double* __restrict__ cs,
                                 double* __restrict__ mu, double* __restrict__ wscale,
                                 T* __restrict__ diag, double* __restrict__ sigma,
                                 int* __restrict__ col_status, FitCtrl* ctrl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p) return;
    double m = 0.0;
    if (center) {
        for (int i = 0; i < n; ++i) m += (double)X[(size_t)i * ldx + k];
        m /= (double)n;
    }
    double ss = 0.0;
    for (int i = 0; i < n; ++i) {
        const double d = (double)X[(size_t)i * ldx + k] - m;
        ss = fma(d, d, ss);
    }
    const double skk = ss / (double)n;
    if (!(skk > 0.0) || !isfinite(skk) || !isfinite(m)) set_error(ctrl, DEV_ERR_NONFINITE);
    const double c = standardize ? 1.0 / sqrt(skk) : 1.0;
    cs[k] = c;
    mu[k] = m;
    wscale[k] = c / sqrt((double)n);
    diag[k] = (T)(c * c * skk);
    sigma[k] = 1.0;
    col_status[k] = COL_OK;
}

// W[i][k] and Wt[k][i] = (x_ik - mu_k) c_k / sqrt(n), formed in FP64 and
// rounded once, over 32 x 32 tiles of (sample, column) that cover the padded
// extents (ldn rows of W, ldn entries of each row of Wt, ldp columns of W),
// with zeros in the padding.  The transpose goes through shared memory so
// that both stores are coalesced.
template <typename T>
__global__ void res_build_kernel(const T* __restrict__ X, int n, int p, int ldx,
                                 const double* __restrict__ mu,
                                 const double* __restrict__ wscale, T* __restrict__ W, int ldp,
                                 T* __restrict__ Wt, int ldn, FitCtrl* ctrl) {
    __shared__ T tile[32][33];
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;      // 32 x 8
    const int k = k0 + tx;
    double m = 0.0, sc = 0.0;
    if (k < p) {
        m = mu[k];
        sc = wscale[k];
    }
    for (int rr = ty; rr < 32; rr += 8) {
        const int i = i0 + rr;
        T v = T(0);
        if (i < n && k < p) v = (T)(((double)X[(size_t)i * ldx + k] - m) * sc);
        tile[rr][tx] = v;
        if (i < ldn && k < ldp) W[(size_t)i * ldp + k] = v;
    }
    __syncthreads();
    const int i = i0 + tx;
    for (int rr = ty; rr < 32; rr += 8) {
        const int kk = k0 + rr;
        if (kk < p && i < ldn) Wt[(size_t)kk * ldn + i] = tile[tx][rr];
    }
}

template <typename T>
__global__ void res_theta_kernel(const T* __restrict__ BT, int p, int ldp,
                                 const double* __restrict__ sigma, const double* __restrict__ cs,
                                 double* __restrict__ Theta, double* __restrict__ sigma_out,
                                 FitCtrl* ctrl) {
    if (*reinterpret_cast<volatile int*>(&ctrl->err) != 0) return;
    theta_pair<T>(BT, p, ldp, sigma, cs, Theta, sigma_out, ctrl, blockIdx.x);
}

template <typename T, bool STD>
cudaError_t run_residual(const ResLaunch& f, const ResLayout& L, cudaStream_t st) {
    int dev = 0, nsm = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    unsigned char* ws = f.ws;
    FitCtrl* ctrl = reinterpret_cast<FitCtrl*>(ws + L.ctrl);
    ResArgs<T> a;
    a.W = reinterpret_cast<const T*>(ws + L.W);
    a.Wt = reinterpret_cast<const T*>(ws + L.Wt);
    a.BT = reinterpret_cast<T*>(ws + L.BT);
    a.diag = reinterpret_cast<const T*>(ws + L.diag);
    a.sigma = reinterpret_cast<double*>(ws + L.sigma);
    a.col_status = reinterpret_cast<int*>(ws + L.col_status);
    a.ctrl = ctrl;
    a.n = f.n;
    a.ldn = L.ldn;
    a.p = f.p;
    a.ldp = L.ldp;
    a.maxit = f.maxit;
    a.lambda0 = f.lambda0;
    a.tol = f.tol;
    double* cs = reinterpret_cast<double*>(ws + L.cs);

    const size_t per = res_warp_smem_bytes<T>(L.ldn, L.ldp);
    const size_t budget = (size_t)smem_optin - 1024;
    if (per > budget) return cudaErrorInvalidValue;
    int LW = f.warps_per_block > 0 ? f.warps_per_block : 8;
    LW = std::max(1, std::min({LW, 8, (int)(budget / per)}));
    const size_t smem = per * LW;
    auto kern = cd_residual_kernel<T, STD>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * LW, smem)) !=
        cudaSuccess)
        return e;
    per_sm = std::max(per_sm, 1);

    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(FitCtrl), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + L.BT, 0, (size_t)f.p * L.ldp * sizeof(T), st)) != cudaSuccess)
        return e;
    const T* X = static_cast<const T*>(f.X);
    res_stats_kernel<T><<<(f.p + 127) / 128, 128, 0, st>>>(
        X, f.n, f.p, f.ldx, f.center, f.standardize, cs, reinterpret_cast<double*>(ws + L.mu),
        reinterpret_cast<double*>(ws + L.wscale), reinterpret_cast<T*>(ws + L.diag), a.sigma,
        a.col_status, ctrl);
    {
        dim3 grid((L.ldp + 31) / 32, (L.ldn + 31) / 32);
        res_build_kernel<T><<<grid, dim3(32, 8), 0, st>>>(
            X, f.n, f.p, f.ldx, reinterpret_cast<const double*>(ws + L.mu),
            reinterpret_cast<const double*>(ws + L.wscale), reinterpret_cast<T*>(ws + L.W), L.ldp,
            reinterpret_cast<T*>(ws + L.Wt), L.ldn, ctrl);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (f.phase_events) cudaEventRecord(f.phase_events[0], st);
    const int grid = std::min((f.p + LW - 1) / LW, nsm * per_sm);
    kern<<<grid, 32 * LW, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (f.phase_events) cudaEventRecord(f.phase_events[1], st);
    res_theta_kernel<T><<<theta_pairs<T>(f.p), dim3(32, 8), 0, st>>>(
        a.BT, f.p, L.ldp, a.sigma, cs, f.Theta, f.sigma_out, ctrl);
    if (f.phase_events) cudaEventRecord(f.phase_events[2], st);
    return cudaGetLastError();
}

}  // namespace

bool residual_sizes_ok(int n, int p, int precision) {
    if (n < 1 || n > RES_MAX_N || p < 2) return false;
    const ResLayout L = res_layout(n, p, precision);
    const size_t per = precision == SPMESL_FP64 ? res_warp_smem_bytes<double>(L.ldn, L.ldp)
                                                : res_warp_smem_bytes<float>(L.ldn, L.ldp);
    return per <= 232448 - 1024;
}

cudaError_t launch_fit_residual(const ResLaunch& f, cudaStream_t st) {
    const ResLayout L = res_layout(f.n, f.p, f.precision);
    if (f.precision == SPMESL_FP64)
        return f.standardize ? run_residual<double, true>(f, L, st)
                             : run_residual<double, false>(f, L, st);
    return f.standardize ? run_residual<float, true>(f, L, st)
                         : run_residual<float, false>(f, L, st);
}

}  // namespace spmesl
