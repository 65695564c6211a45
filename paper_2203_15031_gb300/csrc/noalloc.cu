// spmesl_fit_noalloc: the fit of spmesl_fit for callers that may not allocate
// device memory at all.
//
// Some callers cannot call cudaMalloc or hand over a workspace: a plugin
// hosted by an application whose own pool owns every byte of device memory
// and gives its extensions none; real-time or certified code that forbids
// allocation once it has started; a latency-critical loop that must never
// change the process's device-memory footprint.  For them the fit's scratch
// (standardised S, coefficients, gradients, control block) lives in one
// file-scope __device__ array of kScratchBytes (64 MiB).  The array belongs
// to this library's module: the CUDA runtime loads the module (and commits
// the 64 MiB on the device) when the first call on that device looks up the
// array's address, and the device then holds it until the process exits.
// So that first call changes the device-memory footprint; make it at
// start-up, before memory is tight.  If the device cannot hold the array the
// call returns SPMESL_ENOMEM.
//
// Host code cannot pass the array's name to a kernel (on the host it is only
// a stand-in symbol, not a device address), so the first call on each device
// looks the device address up with cudaGetSymbolAddress, with that device
// current, and keeps it; later calls reuse it.  Make that first call on a
// device before any stream capture begins.
//
// All calls share the one array and it keeps whatever the last call left in
// it: every fit clears its control block and coefficient matrix before it
// starts.  Two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on the array; issue them on one stream or
// order them.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_fit_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_fit_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_fit_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" spmesl_status spmesl_fit_noalloc(const void* S, int n, int p, double lambda0,
                                            double tol, int maxit, const spmesl_opts* opts,
                                            double* Theta, double* sigma, spmesl_stats* stats,
                                            void* stream) {
    spmesl_opts o;
    if (opts) o = *opts;
    else spmesl_default_opts(&o);
    if (o.precision != SPMESL_FP64 && o.precision != SPMESL_FP32 && o.precision != SPMESL_MIXED)
        return SPMESL_EINVAL;
    if (p < 2) return SPMESL_EINVAL;
    // the fit must fit in the fixed scratch
    if (spmesl::fit_layout(p, o.precision).total > kScratchBytes) return SPMESL_ENOMEM;
    o.record_phase_times = 0;           // timing events are not created here
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e == cudaErrorMemoryAllocation) return SPMESL_ENOMEM;   // no room for the array
    if (e != cudaSuccess) return SPMESL_ECUDA;
    spmesl_status s = spmesl_fit(S, n, p, lambda0, tol, maxit, &o, Theta, sigma, nullptr, scratch,
                                 kScratchBytes, stream);
    if (s != SPMESL_OK || !stats) return s;
    s = spmesl_fit_result(scratch, p, o.precision, stats, stream);
    // the penalty level the fit used (the rule's value unless it was given)
    stats->lambda0 = o.lambda_rule == SPMESL_LAMBDA_GIVEN ? lambda0
                                                          : spmesl_lambda(o.lambda_rule, n, p);
    return s;
}
