// Internal definitions shared by the libspmesl translation units.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "spmesl.h"

namespace spmesl {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Column status bits written by the fit kernels (a column may carry both).
constexpr int COL_OK = 0;
constexpr int COL_NOT_CONVERGED = 1;
constexpr int COL_DEGENERATE = 2;
// Set by the lazy solver when it hands a column to the block solver; the bits
// from COL_STEP_SHIFT up hold the sigma step it was in.
constexpr int COL_HANDED = 4;
constexpr int COL_STEP_SHIFT = 8;

// Device-side error codes stored in FitCtrl::err (0 = none).
constexpr int DEV_ERR_NONFINITE = 1;
constexpr int DEV_ERR_TIMEOUT = 2;

// Upper bound of any bounded spin wait (ns of %globaltimer).
constexpr unsigned long long SPIN_LIMIT_NS = 4000000000ull;

// Control block at the start of a fit workspace.  Zeroed before every fit.
struct FitCtrl {
    unsigned int bar_count;       // grid barrier arrivals
    unsigned int bar_gen;         // grid barrier generation
    int err;                      // DEV_ERR_* (first error wins)
    int n_active;                 // joint rule: active columns of the current outer iteration
    int next_col;                 // column rule: dynamic work counter
    int outer_max;                // max sigma iterations over columns (joint: global)
    int n_not_converged;
    int n_degenerate;
    unsigned long long sweep_max[3];   // joint rule: max|delta| per sweep, as ordered bits
    unsigned long long total_sweeps;   // sum over columns (joint: global sweep count)
    unsigned long long moves;          // coordinate updates that changed b
    unsigned long long max_db_bits;    // joint rule: max|delta| of the last sweep (double bits)
    unsigned long long nnz;            // nonzero b at exit
    int inner_cap_hit;                 // joint rule: inner cap reached in some outer iteration
    int max_col_sweeps;                // largest per-column sweep count
    int ovf_count;                     // columns handed from the lazy to the block (eager) solver
    int ovf_next;                      // that solver's position in the queue
    int n_heavy;                       // heavy columns: the first n_heavy of the heat order
    int heavy_next;                    // block solver's position among them
    int block_cols;                    // columns solved by the block solver
    int pad[1];
    unsigned long long act_sweeps;     // lazy solver: sweeps over the support only
    unsigned long long act_moves;      // moves in those sweeps
    // optimality diagnostics (opts.diagnostics): maxima over the columns of
    // the relative subgradient violation, the relative duality gap, the
    // first-order Theta error estimate and 1/sigma^2 (bits of non-negative
    // doubles), and the columns checked
    unsigned long long diag_kkt, diag_gap, diag_err, diag_thmax;
    unsigned int diag_cols;
    unsigned int pad2;
    unsigned long long rows_moved;     // measurement (opts.count_rows): distinct coordinates
                                       // moved per full-sweep index, summed over the indices
};
static_assert(sizeof(FitCtrl) <= 256, "FitCtrl must fit its 256-byte slot");

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int elem_size(int precision) { return precision == SPMESL_FP64 ? 8 : 4; }

// Leading dimension of the per-column p-vectors in the workspace: a multiple
// of 32 elements, so every row starts on a 128-byte (FP32) or 256-byte (FP64)
// boundary and 16-byte vector loads never straddle a row.
inline int padded_ld(int p) { return (p + 31) / 32 * 32; }

// Byte offsets of the fit workspace (see spmesl_fit_workspace_bytes).
struct FitLayout {
    int ldp;
    size_t ctrl, cs, csf, sigma, col_status, active, active_next, flag, diag, cmax, rows, SC, BT,
        GT, total;
};

// 128-coordinate chunks of a padded row (the lazy solver's scan unit).
inline int row_chunks(int ldp) { return (ldp + 127) / 128; }

// Bitmap of the coordinates moved per full-sweep index (opts.count_rows):
// 64 rows of ceil(p / 32) words.
__host__ __device__ inline int rows_words(int p) { return (p + 31) / 32; }
__host__ __device__ inline size_t rows_bitmap_bytes(int p) { return (size_t)64 * rows_words(p) * 4; }

inline FitLayout fit_layout(int p, int precision) {
    FitLayout L{};
    const size_t s = (size_t)elem_size(precision);
    L.ldp = padded_ld(p);
    const size_t mat = align_up((size_t)p * (size_t)L.ldp * s, 256);
    size_t off = 0;
    L.ctrl = off;        off += 256;
    L.cs = off;          off += align_up((size_t)p * 8, 256);
    L.csf = off;         off += align_up((size_t)p * 4, 256);
    L.sigma = off;       off += align_up((size_t)p * 8, 256);
    L.col_status = off;  off += align_up((size_t)p * 4, 256);
    L.active = off;      off += align_up((size_t)p * 4, 256);
    L.active_next = off; off += align_up((size_t)p * 4, 256);
    L.flag = off;        off += align_up((size_t)p * 4, 256);
    L.diag = off;        off += align_up((size_t)p * s, 256);
    L.cmax = off;        off += align_up((size_t)p * row_chunks(L.ldp) * 4, 256);
    L.rows = off;        off += align_up(rows_bitmap_bytes(p), 256);
    L.SC = off;          off += mat;
    L.BT = off;          off += mat;
    L.GT = off;          off += mat;
    L.total = off;
    return L;
}

// Byte offsets of the residual-form workspace (spmesl_fit_residual): the
// control block first (spmesl_fit_result reads it there), then the per-column
// vectors, the scaled data W (ldn x ldp) and its transpose Wt (p x ldn), and
// the coefficients BT (p x ldp).
struct ResLayout {
    int ldn, ldp;
    size_t ctrl, cs, sigma, col_status, mu, wscale, diag, W, Wt, BT, total;
};

inline ResLayout res_layout(int n, int p, int precision) {
    ResLayout L{};
    const size_t s = (size_t)elem_size(precision);
    L.ldn = padded_ld(n);
    L.ldp = padded_ld(p);
    size_t off = 0;
    L.ctrl = off;        off += 256;
    L.cs = off;          off += align_up((size_t)p * 8, 256);
    L.sigma = off;       off += align_up((size_t)p * 8, 256);
    L.col_status = off;  off += align_up((size_t)p * 4, 256);
    L.mu = off;          off += align_up((size_t)p * 8, 256);
    L.wscale = off;      off += align_up((size_t)p * 8, 256);
    L.diag = off;        off += align_up((size_t)p * s, 256);
    L.W = off;           off += align_up((size_t)L.ldn * L.ldp * s, 256);
    L.Wt = off;          off += align_up((size_t)p * L.ldn * s, 256);
    L.BT = off;          off += align_up((size_t)p * L.ldp * s, 256);
    L.total = off;
    return L;
}

// 16-byte vector of T.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Record the first device-side error.
__device__ __forceinline__ void set_error(FitCtrl* c, int code) { atomicCAS(&c->err, 0, code); }

}  // namespace spmesl

// Launchers implemented in the .cu files (host side, stream-ordered).
namespace spmesl {
// Heavy-column routing limits of spmesl_opts with the defaults applied.
inline int heavy_heat_of(int v) { return v <= 0 ? 32 : (v > 62 ? 62 : v); }
inline int heavy_min_p_of(int v) { return v == 0 ? 4096 : (v < 0 ? 0x7fffffff : v); }
inline int handover_of(int v) { return v <= 0 ? 32 : (v > 256 ? 256 : v); }

cudaError_t launch_gram(const void* X, int n, int p, int ldx, int precision, int center, void* S,
                        int lds, void* ws, cudaStream_t st);
size_t gram_ws_bytes(int n, int p, int precision);

struct FitLaunch {
    const void* S;       // input covariance (p x p, ld p)
    int p;
    double lambda0, tol;
    int maxit;
    int precision, standardize, inner_rule, warps_per_block;
    double* Theta;
    double* sigma_out;
    unsigned char* ws;   // workspace base
    cudaEvent_t* phase_events;   // nullptr, or 3 events: before CD, after CD, after Theta
    int gradient;                // spmesl_gradient (column rule only)
    int heavy_heat = 32;         // heat above which a column goes to the block solver
    int heavy_min_p = 4096;      // ... in fits of at least this size (< 0: never)
    int diagnostics = 0;         // 1: optimality diagnostics after the coordinate descent
    int count_rows = 0;          // 1: count the distinct coordinates moved per sweep index
    int handover = 0;            // support above which the lazy solver hands a column over
    double diag_eps = 0.0;       // rounding bound of the working matrix (see diag_eps_for)
    // >= 0: solve only this column (one scaled-lasso regression, lazy column
    // rule) and write its coefficients to beta_out (the p - 1 other columns in
    // order, original scale) and its sigma to sigma_out[0] instead of Theta
    int response_col = -1;
    double* beta_out = nullptr;
};
cudaError_t launch_fit(const FitLaunch& f, cudaStream_t st);
// Diagnostics of a given (B, sigma) in the original scale against S (spmesl_diagnose).
cudaError_t launch_diagnose(const void* S, int p, int precision, int standardize,
                            double lambda0, const double* B, const double* sigma, double eps,
                            unsigned char* ws, cudaStream_t st);
// Typical rounding of an entry of a working matrix built in `precision` from
// n samples, relative to sqrt(S_jj S_kk): two roundings of the
// standardisation, the accumulation of the Gram over n terms (sqrt(n) unit
// roundoffs, the usual size of a sum of independent roundings), and for
// SPMESL_MIXED the 3-term split-BF16 products (each within 3 * 2^-18 of the
// exact product: hi and lo of a factor keep 16 bits, lo * lo is dropped),
// averaged over the n products (/ sqrt(n)).  An estimate, not a bound.
inline double diag_eps_for(int precision, int n) {
    const double u = precision == SPMESL_FP64 ? 0x1p-53 : 0x1p-24;
    const double rn = sqrt((double)(n > 1 ? n : 1));
    double e = u * (2.0 + rn);
    if (precision == SPMESL_MIXED) e += 3.0 * 0x1p-18 / rn;
    return e;
}
// One fit in the residual form (residual.cu): X n x p (ld ldx) on the device.
struct ResLaunch {
    const void* X;
    int n, p, ldx;
    double lambda0, tol;
    int maxit;
    int precision, standardize, center, warps_per_block;
    double* Theta;
    double* sigma_out;
    unsigned char* ws;
    cudaEvent_t* phase_events;   // nullptr, or 3 events: before CD, after CD, after Theta
};
cudaError_t launch_fit_residual(const ResLaunch& f, cudaStream_t st);
bool residual_sizes_ok(int n, int p, int precision);
cudaError_t launch_export_B(const unsigned char* ws, int p, int precision, double* B,
                            cudaStream_t st);
void fill_diagnostics(const FitCtrl& c, spmesl_stats* stats);
int max_p_for(int precision);

// When true on the calling thread, spmesl_batch_create stages its descriptor
// table in ordinary host memory instead of pinned memory (the serving worker
// sets it: releasing pinned memory can synchronise the whole device).
extern thread_local bool g_batch_pageable_staging;
}  // namespace spmesl
