// Support-recovery and estimation-error measures of an estimate against the
// true precision matrix (Section 4.2): TP, FP, TN, FN over the pairs j < k
// (an entry counts as an edge when it is not exactly zero), and the Frobenius
// norm of the difference over all entries.  SEN, SPE, FDR, MISR and MCC follow
// from the counts.
//
// One pass over both matrices: a fixed grid of blocks walks the rows, each
// block reduces its counts and its sum of squared differences (FP64) into
// one slot of the workspace; a single block then adds the slots in a fixed
// order, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"

namespace spmesl {
namespace {

constexpr int MT_BLOCKS = 608;
constexpr int MT_THREADS = 256;

struct MetricSlot {
    unsigned long long tp, fp, tn, fn;
    double sq;
};

__global__ void __launch_bounds__(MT_THREADS) metrics_kernel(const double* __restrict__ A,
                                                           const double* __restrict__ B, int p,
                                                           MetricSlot* __restrict__ slots) {
    unsigned long long tp = 0, fp = 0, tn = 0, fn = 0;
    double sq = 0.0;
    for (int j = blockIdx.x; j < p; j += gridDim.x) {
        const double* a = A + (size_t)j * p;
        const double* b = B + (size_t)j * p;
        for (int k = threadIdx.x; k < p; k += blockDim.x) {
            const double x = a[k], y = b[k];
            const double d = x - y;
            sq = fma(d, d, sq);
            if (k > j) {
                const bool e = x != 0.0, t = y != 0.0;
                tp += e && t;
                fp += e && !t;
                tn += !e && !t;
                fn += !e && t;
            }
        }
    }
    __shared__ unsigned long long s_tp[MT_THREADS / 32], s_fp[MT_THREADS / 32],
        s_tn[MT_THREADS / 32], s_fn[MT_THREADS / 32];
    __shared__ double s_sq[MT_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        tp += __shfl_xor_sync(FULL_MASK, tp, o);
        fp += __shfl_xor_sync(FULL_MASK, fp, o);
        tn += __shfl_xor_sync(FULL_MASK, tn, o);
        fn += __shfl_xor_sync(FULL_MASK, fn, o);
        sq += __shfl_xor_sync(FULL_MASK, sq, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_tp[w] = tp;
        s_fp[w] = fp;
        s_tn[w] = tn;
        s_fn[w] = fn;
        s_sq[w] = sq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        MetricSlot m{0, 0, 0, 0, 0.0};
        for (int i = 0; i < MT_THREADS / 32; ++i) {
            m.tp += s_tp[i];
            m.fp += s_fp[i];
            m.tn += s_tn[i];
            m.fn += s_fn[i];
            m.sq += s_sq[i];
        }
        slots[blockIdx.x] = m;
    }
}

__global__ void metrics_sum_kernel(const MetricSlot* __restrict__ slots, int n,
                                   MetricSlot* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    MetricSlot m{0, 0, 0, 0, 0.0};
    for (int i = 0; i < n; ++i) {
        m.tp += slots[i].tp;
        m.fp += slots[i].fp;
        m.tn += slots[i].tn;
        m.fn += slots[i].fn;
        m.sq += slots[i].sq;
    }
    *out = m;
}

double ratio(double a, double b) { return b > 0.0 ? a / b : NAN; }

}  // namespace
}  // namespace spmesl

using namespace spmesl;

extern "C" {

size_t spmesl_metrics_workspace_bytes(void) {
    return align_up(sizeof(MetricSlot) * (MT_BLOCKS + 1), 256);
}

spmesl_status spmesl_support_metrics(const double* Theta_hat, const double* Theta_true, int p,
                                     spmesl_metrics* out, void* workspace, size_t ws_bytes,
                                     void* stream) {
    if (!Theta_hat || !Theta_true || !out || !workspace || p < 2) return SPMESL_EINVAL;
    if (ws_bytes < spmesl_metrics_workspace_bytes()) return SPMESL_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPMESL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MetricSlot* slots = static_cast<MetricSlot*>(workspace);
    const int grid = p < MT_BLOCKS ? p : MT_BLOCKS;
    metrics_kernel<<<grid, MT_THREADS, 0, st>>>(Theta_hat, Theta_true, p, slots);
    metrics_sum_kernel<<<1, 32, 0, st>>>(slots, grid, slots + MT_BLOCKS);
    MetricSlot m;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&m, slots + MT_BLOCKS, sizeof(m), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SPMESL_ECUDA;
    memset(out, 0, sizeof(*out));
    out->tp = (int64_t)m.tp;
    out->fp = (int64_t)m.fp;
    out->tn = (int64_t)m.tn;
    out->fn = (int64_t)m.fn;
    out->n_edges_hat = (int64_t)(m.tp + m.fp);
    out->n_edges_true = (int64_t)(m.tp + m.fn);
    out->frobenius = sqrt(m.sq);
    const double tp = (double)m.tp, fp = (double)m.fp, tn = (double)m.tn, fn = (double)m.fn;
    out->sen = ratio(tp, tp + fn);
    out->spe = ratio(tn, tn + fp);
    out->fdr = ratio(fp, tp + fp);
    out->misr = (fp + fn) / ((double)p * (p - 1) / 2.0);
    out->mcc = ratio(tp * tn - fp * fn, sqrt((tp + fp) * (tp + fn) * (tn + fp) * (tn + fn)));
    return SPMESL_OK;
}

}  // extern "C"
