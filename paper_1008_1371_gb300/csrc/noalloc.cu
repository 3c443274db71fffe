// noalloc.cu -- hsvd_solve_pointwise_noalloc: the pointwise solver with its
// scratch in a fixed device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory: code that runs while the
// caching allocator of a host framework owns the device, real-time or
// safety-critical callers that forbid allocation after start-up, and callers
// on memory-capped contexts.  For them this entry point allocates nothing:
// its scratch lives in `g_noalloc_scratch`, a file-scope device array of a
// fixed, modest size that every GPU which loads the library keeps until the
// process exits.  The array holds, for n_pad = n rounded up to even:
//   [0, n_pad^2)            doubles: the accumulated transformation W
//   kStatusOff (n_pad^2)    three ints: status, sweeps, stop rule
//   kRotOff (n_pad^2 + 2)   one 64-bit integer: the rotation count
#include <cuda.h>

#include <mutex>

#include "hsvd_internal.cuh"

namespace hsvd {
namespace {

constexpr int64_t kNoallocMaxPad = HSVD_NOALLOC_MAX_N + (HSVD_NOALLOC_MAX_N & 1);
constexpr int64_t status_off(int64_t n_pad) { return n_pad * n_pad; }  // in doubles
constexpr int64_t rot_off(int64_t n_pad) { return n_pad * n_pad + 2; }  // in doubles
constexpr int64_t kScratchDoubles = kNoallocMaxPad * kNoallocMaxPad + 4;
// three ints fit the two doubles before the rotation count, and the count
// fits the array at the largest n
static_assert(3 * sizeof(int) <= 2 * sizeof(double), "status words overrun the rotation count");
static_assert(rot_off(kNoallocMaxPad) + 1 <= kScratchDoubles, "scratch array too small");
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;  // the context the address belongs to (0: unknown)
    double *ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Identity of the current context, 0 if it cannot be read.  A device reset
// (cudaDeviceReset) ends the context and reloads the module with the array
// at a possibly different address; the new context has a new identity.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array in the current device's context.  The
// host-side name of the array is not a device address; the address is looked
// up (cudaGetSymbolAddress, which allocates nothing) with the device current,
// once per device and context, and again after a device reset.
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    ScratchAddr &s = g_scratch[dev];
    if (!s.ptr || ctx == 0 || s.ctx_id != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        s.ptr = static_cast<double *>(p);
        s.ctx_id = ctx;
    }
    *out = s.ptr;
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
    int *out = reinterpret_cast<int *>(scratch + status_off(n_pad));
    long long *rot = reinterpret_cast<long long *>(scratch + rot_off(n_pad));
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
