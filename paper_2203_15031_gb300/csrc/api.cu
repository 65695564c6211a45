// C ABI of libspmesl (declared in include/spmesl.h): argument validation,
// workspace layout, stream-ordered launches and status reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <array>
#include <mutex>
#include <unordered_map>

#include "common.cuh"

using namespace spmesl;

namespace {

constexpr int kVersion = 1 * 10000 + 1 * 100 + 0;

bool valid_precision(int prec) {
    return prec == SPMESL_FP64 || prec == SPMESL_FP32 || prec == SPMESL_MIXED;
}

spmesl_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SPMESL_OK;
    if (e == cudaErrorMemoryAllocation) return SPMESL_ENOMEM;
    if (e == cudaErrorInvalidValue) return SPMESL_EINVAL;
    return SPMESL_ECUDA;
}

// Standard normal quantile: Newton's method on Phi(x) = erfc(-x/sqrt 2)/2,
// started from the logistic approximation and safeguarded by bisection.
double normal_quantile(double u) {
    if (!(u > 0.0 && u < 1.0)) return NAN;
    double lo = -40.0, hi = 40.0;
    double x = log(u / (1.0 - u)) / 1.702;      // logistic approximation of the probit
    if (!(x > lo && x < hi)) x = 0.0;
    for (int it = 0; it < 200; ++it) {
        const double F = 0.5 * erfc(-x / sqrt(2.0));
        const double f = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
        if (F < u) lo = x; else hi = x;
        double nx = (f > 0.0) ? x - (F - u) / f : 0.5 * (lo + hi);
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (fabs(nx - x) <= 1e-15 * (1.0 + fabs(x))) return nx;
        x = nx;
    }
    return x;
}

// L_n(t) = n^{-1/2} Phi^{-1}(1 - t)  (Section 2.3)
double L_n(double n, double t) { return normal_quantile(1.0 - t) / sqrt(n); }

// Root of k = L_1^4(k/p) + 2 L_1^2(k/p) by bisection (Section 2.3).
double pb_root(int p) {
    double lo = 1e-9 * p, hi = 0.5 * p;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double L = L_n(1.0, mid / p);
        const double h = mid - (L * L * L * L + 2.0 * L * L);
        if (h < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// Phase-timing events of the last fit recorded in a workspace
// (record_phase_times), keyed by the workspace address.
std::mutex g_phase_mu;
std::unordered_map<const void*, std::array<cudaEvent_t, 3>> g_phase_events;

cudaEvent_t* phase_events_for(const void* ws) {
    std::lock_guard<std::mutex> lk(g_phase_mu);
    auto it = g_phase_events.find(ws);
    if (it == g_phase_events.end()) {
        std::array<cudaEvent_t, 3> ev{};
        for (auto& x : ev)
            if (cudaEventCreate(&x) != cudaSuccess) return nullptr;
        it = g_phase_events.emplace(ws, ev).first;
    }
    return it->second.data();
}

void read_phase_times(const void* ws, spmesl_stats* stats) {
    std::lock_guard<std::mutex> lk(g_phase_mu);
    auto it = g_phase_events.find(ws);
    if (it == g_phase_events.end() || !stats) return;
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, it->second[0], it->second[1]) == cudaSuccess) stats->ms_cd = a;
    if (cudaEventElapsedTime(&b, it->second[1], it->second[2]) == cudaSuccess) stats->ms_theta = b;
    cudaGetLastError();
}

double from_bits(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

}  // namespace

namespace spmesl {
// The diagnostics of a control block into the stats (when they were computed).
void fill_diagnostics(const FitCtrl& c, spmesl_stats* stats) {
    if (c.diag_cols == 0 || !stats) return;
    stats->diagnostics = 1;
    stats->kkt_viol = from_bits(c.diag_kkt);
    stats->dual_gap = from_bits(c.diag_gap);
    const double th = from_bits(c.diag_thmax);
    stats->err_est = th > 0.0 ? from_bits(c.diag_err) / th : NAN;
}
}  // namespace spmesl

namespace {

spmesl_opts resolve_opts(const spmesl_opts* o) {
    spmesl_opts d;
    spmesl_default_opts(&d);
    return o ? *o : d;
}

// Workspace of spmesl_scaled_lasso: Z = [X y] (n x (p+1)), its Gram, the
// Gram's scratch and the fit workspace of the (p+1)-column problem.
struct LassoLayout {
    size_t Z, S, gram, fit, total;
};

LassoLayout lasso_layout(int n, int p, int precision) {
    const size_t s = (size_t)elem_size(precision);
    const int q = p + 1;
    LassoLayout L{};
    size_t off = 0;
    L.Z = off;    off += align_up((size_t)n * q * s, 256);
    L.S = off;    off += align_up((size_t)q * q * s, 256);
    L.gram = off; off += align_up(gram_ws_bytes(n, q, precision), 256);
    L.fit = off;  off += fit_layout(q, precision).total;
    L.total = off;
    return L;
}

template <typename T>
__global__ void augment_kernel(const T* __restrict__ X, const T* __restrict__ y, int n, int p,
                               T* __restrict__ Z) {
    const int q = p + 1;
    const size_t total = (size_t)n * q;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / q;
        const int c = (int)(i - r * q);
        Z[i] = c < p ? X[r * p + c] : y[r];
    }
}

}  // namespace

extern "C" {

void spmesl_default_opts(spmesl_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = SPMESL_FP32;
    o->standardize = 1;
    o->center = 0;
    o->lambda_rule = SPMESL_LAMBDA_GIVEN;
    o->inner_rule = SPMESL_INNER_COLUMN;
    o->warps_per_block = 0;
}

const char* spmesl_status_string(int s) {
    switch (s) {
        case SPMESL_OK: return "ok";
        case SPMESL_NOT_CONVERGED: return "iteration cap reached (last iterate returned)";
        case SPMESL_EINVAL: return "invalid argument";
        case SPMESL_ENOMEM: return "out of memory or workspace too small";
        case SPMESL_ENONFINITE: return "non-finite input or non-positive variance";
        case SPMESL_EDEGENERATE: return "sigma reached its floor (degenerate fit)";
        case SPMESL_ETIMEOUT: return "bounded device-side wait ran out";
        case SPMESL_ECUDA: return "CUDA runtime error";
        case SPMESL_EBUSY: return "busy";
        case SPMESL_ENOTFOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

int spmesl_version(void) { return kVersion; }

double spmesl_lambda(int rule, int n, int p) {
    if (n < 1 || p < 2) return NAN;
    switch (rule) {
        case SPMESL_LAMBDA_UNIV: return sqrt(2.0 * log((double)p) / n);
        case SPMESL_LAMBDA_UNIV_PM1: return p > 2 ? sqrt(2.0 * log((double)p - 1.0) / n) : NAN;
        case SPMESL_LAMBDA_UB: return sqrt(4.0 * log((double)p) / n);
        case SPMESL_LAMBDA_PB: return sqrt(2.0) * L_n((double)n, pb_root(p) / p);
        default: return NAN;
    }
}

int spmesl_max_p(int precision) {
    if (!valid_precision(precision)) return 0;
    return max_p_for(precision);
}

size_t spmesl_gram_workspace_bytes(int n, int p, int precision) {
    if (n < 1 || p < 1 || !valid_precision(precision)) return 0;
    return gram_ws_bytes(n, p, precision);
}

spmesl_status spmesl_gram(const void* X, int n, int p, int ldx, int precision, int center, void* S,
                          int lds, void* workspace, size_t ws_bytes, void* stream) {
    if (!X || !S || n < 1 || p < 1 || ldx < p || lds < p || !valid_precision(precision))
        return SPMESL_EINVAL;
    const size_t need = gram_ws_bytes(n, p, precision);
    if (need > 0 && (!workspace || ws_bytes < need)) return SPMESL_EINVAL;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return SPMESL_EINVAL;
    return from_cuda(launch_gram(X, n, p, ldx, precision, center, S, lds, workspace,
                                 static_cast<cudaStream_t>(stream)));
}

size_t spmesl_fit_workspace_bytes(int p, int precision) {
    if (p < 2 || !valid_precision(precision)) return 0;
    return fit_layout(p, precision).total;
}

spmesl_status spmesl_fit(const void* S, int n, int p, double lambda0, double tol, int maxit,
                         const spmesl_opts* opts, double* Theta, double* sigma,
                         spmesl_stats* stats, void* workspace, size_t ws_bytes, void* stream) {
    const spmesl_opts o = resolve_opts(opts);
    if (!S || !Theta || !sigma || !workspace || p < 2 || maxit < 1 || !(tol > 0.0) ||
        !valid_precision(o.precision))
        return SPMESL_EINVAL;
    if (o.inner_rule != SPMESL_INNER_JOINT && o.inner_rule != SPMESL_INNER_COLUMN)
        return SPMESL_EINVAL;
    if (o.gradient < SPMESL_GRADIENT_AUTO || o.gradient > SPMESL_GRADIENT_LAZY) return SPMESL_EINVAL;
    if (p > max_p_for(o.precision)) return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    if (ws_bytes < fit_layout(p, o.precision).total) return SPMESL_EINVAL;
    double lam = lambda0;
    if (o.lambda_rule != SPMESL_LAMBDA_GIVEN) {
        lam = spmesl_lambda(o.lambda_rule, n, p);
    }
    if (!(lam > 0.0) || !isfinite(lam)) return SPMESL_EINVAL;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    FitLaunch f;
    f.S = S;
    f.p = p;
    f.lambda0 = lam;
    f.tol = tol;
    f.maxit = maxit;
    f.precision = o.precision;
    f.standardize = o.standardize ? 1 : 0;
    f.inner_rule = o.inner_rule;
    f.warps_per_block = o.warps_per_block;
    f.gradient = o.gradient;
    f.heavy_heat = o.heavy_heat;
    f.heavy_min_p = o.heavy_min_p;
    f.diagnostics = o.diagnostics ? 1 : 0;
    f.diag_eps = diag_eps_for(o.precision, n);
    f.count_rows = o.count_rows ? 1 : 0;
    f.handover = o.handover;
    f.Theta = Theta;
    f.sigma_out = sigma;
    f.ws = static_cast<unsigned char*>(workspace);
    f.phase_events = o.record_phase_times ? phase_events_for(workspace) : nullptr;
    cudaError_t e = launch_fit(f, st);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return from_cuda(e);
    }
    if (!stats) return SPMESL_OK;
    cudaEventRecord(e1, st);
    spmesl_status rs = spmesl_fit_result(workspace, p, o.precision, stats, stream);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->ms_fit = ms;
    stats->lambda0 = lam;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rs;
}

size_t spmesl_fit_residual_workspace_bytes(int n, int p, int precision) {
    if (!valid_precision(precision) || !residual_sizes_ok(n, p, precision)) return 0;
    return res_layout(n, p, precision).total;
}

spmesl_status spmesl_fit_residual(const void* X, int n, int p, int ldx, double lambda0,
                                  double tol, int maxit, const spmesl_opts* opts, double* Theta,
                                  double* sigma, spmesl_stats* stats, void* workspace,
                                  size_t ws_bytes, void* stream) {
    const spmesl_opts o = resolve_opts(opts);
    if (!X || !Theta || !sigma || !workspace || p < 2 || n < 1 || ldx < p || maxit < 1 ||
        !(tol > 0.0) || !valid_precision(o.precision))
        return SPMESL_EINVAL;
    if (o.inner_rule != SPMESL_INNER_COLUMN) return SPMESL_EINVAL;
    if (!residual_sizes_ok(n, p, o.precision)) return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    if (ws_bytes < res_layout(n, p, o.precision).total) return SPMESL_EINVAL;
    double lam = lambda0;
    if (o.lambda_rule != SPMESL_LAMBDA_GIVEN) lam = spmesl_lambda(o.lambda_rule, n, p);
    if (!(lam > 0.0) || !isfinite(lam)) return SPMESL_EINVAL;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    ResLaunch f;
    f.X = X;
    f.n = n;
    f.p = p;
    f.ldx = ldx;
    f.lambda0 = lam;
    f.tol = tol;
    f.maxit = maxit;
    f.precision = o.precision;
    f.standardize = o.standardize ? 1 : 0;
    f.center = o.center ? 1 : 0;
    f.warps_per_block = o.warps_per_block;
    f.Theta = Theta;
    f.sigma_out = sigma;
    f.ws = static_cast<unsigned char*>(workspace);
    f.phase_events = o.record_phase_times ? phase_events_for(workspace) : nullptr;
    cudaError_t e = launch_fit_residual(f, st);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return from_cuda(e);
    }
    if (!stats) return SPMESL_OK;
    cudaEventRecord(e1, st);
    spmesl_status rs = spmesl_fit_result(workspace, p, o.precision, stats, stream);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->ms_fit = ms;
    stats->lambda0 = lam;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rs;
}

size_t spmesl_scaled_lasso_workspace_bytes(int n, int p, int precision) {
    if (n < 1 || p < 1 || !valid_precision(precision)) return 0;
    return lasso_layout(n, p, precision).total;
}

spmesl_status spmesl_scaled_lasso(const void* X, const void* y, int n, int p, double lambda0,
                                  double tol, int maxit, const spmesl_opts* opts, double* beta,
                                  double* sigma, spmesl_stats* stats, void* workspace,
                                  size_t ws_bytes, void* stream) {
    const spmesl_opts o = resolve_opts(opts);
    if (!X || !y || !beta || !sigma || !workspace || n < 1 || p < 1 || maxit < 1 ||
        !(tol > 0.0) || !valid_precision(o.precision))
        return SPMESL_EINVAL;
    if (p + 1 > max_p_for(o.precision)) return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    const LassoLayout L = lasso_layout(n, p, o.precision);
    if (ws_bytes < L.total) return SPMESL_EINVAL;
    double lam = lambda0;
    if (o.lambda_rule != SPMESL_LAMBDA_GIVEN) lam = spmesl_lambda(o.lambda_rule, n, p);
    if (!(lam > 0.0) || !isfinite(lam)) return SPMESL_EINVAL;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    const int q = p + 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    const size_t total = (size_t)n * q;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    if (o.precision == SPMESL_FP64)
        augment_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(X),
                                                     static_cast<const double*>(y), n, p,
                                                     reinterpret_cast<double*>(ws + L.Z));
    else
        augment_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(X),
                                                    static_cast<const float*>(y), n, p,
                                                    reinterpret_cast<float*>(ws + L.Z));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_gram(ws + L.Z, n, q, q, o.precision, o.center, ws + L.S, q, ws + L.gram, st);
    if (e == cudaSuccess) {
        FitLaunch f;
        f.S = ws + L.S;
        f.p = q;
        f.lambda0 = lam;
        f.tol = tol;
        f.maxit = maxit;
        f.precision = o.precision;
        f.standardize = o.standardize ? 1 : 0;
        f.inner_rule = SPMESL_INNER_COLUMN;
        f.warps_per_block = 0;
        f.gradient = SPMESL_GRADIENT_AUTO;
        f.heavy_heat = o.heavy_heat;
        f.heavy_min_p = o.heavy_min_p;
        f.diagnostics = o.diagnostics ? 1 : 0;
        f.diag_eps = diag_eps_for(o.precision, n);
        f.handover = o.handover;
        f.Theta = nullptr;
        f.sigma_out = sigma;
        f.ws = ws + L.fit;
        f.phase_events = nullptr;
        f.response_col = p;
        f.beta_out = beta;
        e = launch_fit(f, st);
    }
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return from_cuda(e);
    }
    if (!stats) return SPMESL_OK;
    cudaEventRecord(e1, st);
    spmesl_status rs = spmesl_fit_result(ws + L.fit, q, o.precision, stats, stream);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->ms_total = ms;
    stats->lambda0 = lam;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rs;
}

spmesl_status spmesl_fit_result(const void* workspace, int p, int precision, spmesl_stats* stats,
                                void* stream) {
    if (!workspace || p < 2 || !valid_precision(precision)) return SPMESL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FitCtrl c;
    cudaError_t e = cudaMemcpyAsync(&c, workspace, sizeof(FitCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    spmesl_status s = SPMESL_OK;
    if (c.err == DEV_ERR_NONFINITE) s = SPMESL_ENONFINITE;
    else if (c.err == DEV_ERR_TIMEOUT) s = SPMESL_ETIMEOUT;
    else if (c.n_degenerate > 0) s = SPMESL_EDEGENERATE;
    else if (c.n_not_converged > 0 || c.inner_cap_hit) s = SPMESL_NOT_CONVERGED;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->status = s;
        stats->outer_iters = c.outer_max;
        stats->inner_sweeps = (int64_t)c.total_sweeps;
        stats->moves = (int64_t)c.moves;
        stats->active_sweeps = (int64_t)c.act_sweeps;
        stats->active_moves = (int64_t)c.act_moves;
        stats->nnz_B = (int64_t)c.nnz;
        stats->n_not_converged = c.n_not_converged;
        stats->n_degenerate = c.n_degenerate;
        double md;
        memcpy(&md, &c.max_db_bits, sizeof(md));
        stats->max_db = md;
        stats->max_col_sweeps = c.max_col_sweeps;
        stats->max_col_outer = c.outer_max;
        stats->block_columns = c.block_cols;
        stats->rows_moved = (int64_t)c.rows_moved;
        fill_diagnostics(c, stats);
        read_phase_times(workspace, stats);
    }
    return s;
}

spmesl_status spmesl_fit_coefficients(const void* workspace, int p, int precision, double* B,
                                      void* stream) {
    if (!workspace || !B || p < 2 || !valid_precision(precision)) return SPMESL_EINVAL;
    return from_cuda(launch_export_B(static_cast<const unsigned char*>(workspace), p, precision, B,
                                     static_cast<cudaStream_t>(stream)));
}

spmesl_status spmesl_diagnose(const void* S, int n, int p, double lambda0, const double* B,
                              const double* sigma, const spmesl_opts* opts, spmesl_stats* stats,
                              void* workspace, size_t ws_bytes, void* stream) {
    const spmesl_opts o = resolve_opts(opts);
    if (!S || !B || !sigma || !stats || !workspace || p < 2 || !valid_precision(o.precision))
        return SPMESL_EINVAL;
    if (p > max_p_for(o.precision)) return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    if (ws_bytes < fit_layout(p, o.precision).total) return SPMESL_EINVAL;
    double lam = lambda0;
    if (o.lambda_rule != SPMESL_LAMBDA_GIVEN) lam = spmesl_lambda(o.lambda_rule, n, p);
    if (!(lam > 0.0) || !isfinite(lam)) return SPMESL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_diagnose(S, p, o.precision, o.standardize ? 1 : 0, lam, B, sigma,
                                    diag_eps_for(o.precision, n),
                                    static_cast<unsigned char*>(workspace), st);
    if (e != cudaSuccess) return from_cuda(e);
    FitCtrl c;
    e = cudaMemcpyAsync(&c, workspace, sizeof(FitCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    memset(stats, 0, sizeof(*stats));
    stats->lambda0 = lam;
    if (c.err == DEV_ERR_NONFINITE) {
        stats->status = SPMESL_ENONFINITE;
        return SPMESL_ENONFINITE;
    }
    fill_diagnostics(c, stats);
    stats->status = SPMESL_OK;
    return SPMESL_OK;
}

size_t spmesl_solve_workspace_bytes(int n, int p, int precision) {
    if (n < 1 || p < 2 || !valid_precision(precision)) return 0;
    const size_t s = (size_t)elem_size(precision);
    size_t off = 0;
    off += align_up((size_t)n * p * s, 256);                 // X
    off += align_up((size_t)p * p * s, 256);                 // S
    off += align_up((size_t)p * p * 8, 256);                 // Theta
    off += align_up((size_t)p * 8, 256);                     // sigma
    off += align_up(gram_ws_bytes(n, p, precision), 256);    // Gram scratch
    off += fit_layout(p, precision).total;                   // fit workspace
    return off;
}

spmesl_status spmesl_solve(const void* X_host, int n, int p, double lambda0, double tol,
                           int maxit, const spmesl_opts* opts, double* Theta_host,
                           double* sigma_host, spmesl_stats* stats, void* workspace,
                           size_t ws_bytes, void* stream) {
    const spmesl_opts o = resolve_opts(opts);
    if (!X_host || !Theta_host || !sigma_host || !workspace || n < 1 || p < 2 ||
        !valid_precision(o.precision))
        return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    if (ws_bytes < spmesl_solve_workspace_bytes(n, p, o.precision)) return SPMESL_EINVAL;
    const size_t s = (size_t)elem_size(o.precision);
    unsigned char* base = static_cast<unsigned char*>(workspace);
    size_t off = 0;
    void* dX = base + off;       off += align_up((size_t)n * p * s, 256);
    void* dS = base + off;       off += align_up((size_t)p * p * s, 256);
    double* dT = reinterpret_cast<double*>(base + off); off += align_up((size_t)p * p * 8, 256);
    double* dsg = reinterpret_cast<double*>(base + off); off += align_up((size_t)p * 8, 256);
    const size_t gws = gram_ws_bytes(n, p, o.precision);
    void* dG = base + off;       off += align_up(gws, 256);
    void* dF = base + off;
    const size_t fws = fit_layout(p, o.precision).total;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (stats)
        for (auto& x : ev) cudaEventCreate(&x);
    cudaError_t e = cudaMemcpyAsync(dX, X_host, (size_t)n * p * s, cudaMemcpyHostToDevice, st);
    if (stats) cudaEventRecord(ev[0], st);
    spmesl_status rs = SPMESL_OK;
    if (e == cudaSuccess) rs = spmesl_gram(dX, n, p, p, o.precision, o.center, dS, p, dG, gws, stream);
    if (stats) cudaEventRecord(ev[1], st);
    if (e == cudaSuccess && rs == SPMESL_OK)
        rs = spmesl_fit(dS, n, p, lambda0, tol, maxit, &o, dT, dsg, nullptr, dF, fws, stream);
    if (stats) cudaEventRecord(ev[2], st);
    if (e == cudaSuccess && rs == SPMESL_OK)
        e = cudaMemcpyAsync(Theta_host, dT, (size_t)p * p * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rs == SPMESL_OK)
        e = cudaMemcpyAsync(sigma_host, dsg, (size_t)p * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rs == SPMESL_OK) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && rs == SPMESL_OK) {
        rs = spmesl_fit_result(dF, p, o.precision, stats, stream);
        if (stats) {
            cudaEventElapsedTime(&stats->ms_gram, ev[0], ev[1]);
            cudaEventElapsedTime(&stats->ms_fit, ev[1], ev[2]);
            stats->lambda0 = o.lambda_rule == SPMESL_LAMBDA_GIVEN ? lambda0
                                                                  : spmesl_lambda(o.lambda_rule, n, p);
        }
    }
    if (stats)
        for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return from_cuda(e);
    return rs;
}

}  // extern "C"
