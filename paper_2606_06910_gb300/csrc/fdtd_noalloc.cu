// fdtd_misfit_noalloc: the FP64 data-misfit reduction of fdtd_misfit for
// callers that cannot allocate device memory.
//
// Some callers have no device memory to spare for scratch: a process whose
// device memory is owned by another allocator with a fixed budget (a training
// framework's caching allocator, a serving runtime's preallocated arena), or a
// latency-critical loop where cudaMalloc, which may synchronise the device, is
// not allowed.  This entry point allocates nothing: its scratch is the
// file-scope array below, reserved on every GPU that loads the library until
// the process exits.
//
// The array's name in host code is a host-side stand-in, not a device address,
// so every call looks the device address up with cudaGetSymbolAddress on the
// caller's current device and passes it to the kernels.  The lookup is a
// host-side query; the first one on a device also loads the library's device
// code there (the set-up of that device).  Looking it up on every call, rather
// than caching it, keeps the address right after a context teardown
// (cudaDeviceReset) reloads the module.  All calls on a device share the
// array; the kernels overwrite every partial they later read, so nothing has
// to start at zero, but calls that overlap on the GPU (concurrent streams)
// race on it.
#include "fdtd_internal.cuh"

namespace fdtd {
cudaError_t launch_misfit_flat(const float *tr, const float *dobs, float *resid, long long n, int nblocks,
                               double *part, double *out, cudaStream_t s);
}

namespace {

constexpr int kMaxBlocks = 4096;                       // partial sums
constexpr long long kPerBlock = 65536;                 // values per partial
static_assert((long long)kMaxBlocks * kPerBlock == FDTD_NOALLOC_MISFIT_MAX, "limit mismatch");

// kMaxBlocks partial sums followed by the result (33 KB)
__device__ __align__(256) double g_misfit_scratch[kMaxBlocks + 32];

// Device address of the scratch array on the current device.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_misfit_scratch);
    if (e != cudaSuccess)
        return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" int fdtd_misfit_noalloc(const float *traces_dev, const float *dobs_dev, long long n, float *resid_dev,
                                   double *out_host, void *stream)
{
    if (!traces_dev || !dobs_dev || !out_host)
        return FDTD_EINVAL;
    if (n < 1 || n > FDTD_NOALLOC_MISFIT_MAX)
        return FDTD_EINVAL;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess)
        return FDTD_ECUDA;
    const int nblocks = (int)((n + kPerBlock - 1) / kPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (fdtd::launch_misfit_flat(traces_dev, dobs_dev, resid_dev, n, nblocks, scratch, scratch + kMaxBlocks, s) !=
        cudaSuccess)
        return FDTD_ECUDA;
    if (cudaMemcpyAsync(out_host, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FDTD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return FDTD_ECUDA;
    return FDTD_OK;
}
