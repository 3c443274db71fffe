// noalloc.cu -- hsvd_solve_pointwise_noalloc: the pointwise solver with its
// scratch in a fixed device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory: code that runs while the
// caching allocator of a host framework owns the device, real-time or
// safety-critical callers that forbid allocation after start-up, and callers
// on memory-capped contexts.  For them this entry point allocates nothing:
// its scratch (the accumulated transformation W and two status words) lives
// in `g_noalloc_scratch`, a file-scope device array of a fixed, modest size
// that every GPU which loads the library keeps until the process exits.
#include <mutex>

#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

// W of up to HSVD_NOALLOC_MAX_N + 1 bordered columns, then the status words
constexpr int64_t kNoallocMaxPad = HSVD_NOALLOC_MAX_N + (HSVD_NOALLOC_MAX_N & 1);
constexpr int64_t kScratchDoubles = kNoallocMaxPad * kNoallocMaxPad + 8;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per
// device; the host-side name of the array is not a device address).
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace hsvd

using namespace hsvd;

extern "C" int hsvd_solve_pointwise_noalloc(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J,
                                            double tol, int max_sweeps, int sort, double *sigma, double *U,
                                            int64_t ldu, double *V, int64_t ldv, int *sweeps, void *stream) {
    if (!G || !J || !sigma || n < 1 || m < n || ldg < m) return HSVD_ERR_ARG;
    if (n > HSVD_NOALLOC_MAX_N || !pointwise_fits(m, n)) return HSVD_ERR_ARG;
    if ((U && ldu < m) || (V && ldv < n) || max_sweeps < 0 || !(tol == tol)) return HSVD_ERR_ARG;
    if (!all_device({G, J, sigma, U, V})) return HSVD_ERR_ARG;
    if (max_sweeps == 0) max_sweeps = 30;
    if (!(tol > 0.0)) tol = (double)n * 0x1p-53;
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return HSVD_ERR_CUDA;
    const int64_t n_pad = n + (n & 1);
    double *W = scratch;
    int *out = reinterpret_cast<int *>(scratch + n_pad * n_pad);
    long long *rot = reinterpret_cast<long long *>(scratch + n_pad * n_pad + 2);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the kernel writes every scratch word it later reads (W = I first, the
    // status words last), so nothing has to be cleared between calls
    if (launch_pointwise(G, ldg, (int)m, (int)n, J, tol, 0.0, max_sweeps, sort ? 1 : 0, W, sigma, U, ldu, V, ldv,
                         out, rot, st) != cudaSuccess)
        return HSVD_ERR_CUDA;
    int h_out[2] = {0, 0};
    if (cudaMemcpyAsync(h_out, out, sizeof h_out, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HSVD_ERR_CUDA;
    if (sweeps) *sweeps = h_out[1];
    return h_out[0];
}
