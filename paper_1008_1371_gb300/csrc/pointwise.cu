// pointwise.cu -- the pointwise one-sided hyperbolic Jacobi method (Sec. 2,
// Alg. 4.5) for one factor small enough to live in one SM's shared memory:
// one CTA of 1024 threads runs pw_solve (pw_core.cuh) with G in shared memory
// and W in global memory.
#include "pw_core.cuh"

namespace hsvd {
namespace {

constexpr int kThreads = 1024;

__global__ void __launch_bounds__(kThreads, 1)
k_pointwise(const double *__restrict__ G, int64_t ldg, int m, int n, const int8_t *__restrict__ J,
            int m_pad, int n_pad, double tol, double tstop, int max_sweeps, int sort, double *__restrict__ W,
            double *__restrict__ sigma, double *__restrict__ U, int64_t ldu, double *__restrict__ V,
            int64_t ldv, int *__restrict__ out, long long *__restrict__ rot_out) {
    extern __shared__ __align__(16) double smem[];
    __shared__ PwScalars sc;
    PwArrays sh;
    sh.G = smem;
    sh.W = W;
    sh.d = sh.G + (size_t)m_pad * n_pad;
    sh.pos = reinterpret_cast<int *>(sh.d + n_pad);
    sh.newpos = sh.pos + n_pad;
    sh.sg = sh.newpos + n_pad;
    pw_solve<kThreads>(G, ldg, m, n, J, m_pad, n_pad, tol, tstop, max_sweeps, sort, sh, sc, sigma, U, ldu, V,
                       ldv, &out[0], &out[1], rot_out, &out[2], 0);
}

}  // namespace

size_t pointwise_smem_bytes(int64_t m_pad, int64_t n_pad) {
    return (size_t)m_pad * n_pad * sizeof(double) + pw_aux_bytes(n_pad);
}

bool pointwise_fits(int64_t m, int64_t n) {
    const int64_t n_pad = n + (n & 1);
    return n_pad <= 2048 && pointwise_smem_bytes(pw_rows_pad(m, n), n_pad) <= 200 * 1024;
}

cudaError_t launch_pointwise(const double *G, int64_t ldg, int m, int n, const int8_t *J,
                             double tol, double tstop, int max_sweeps, int sort, double *Wws, double *sigma,
                             double *U, int64_t ldu, double *V, int64_t ldv, int *dev_out,
                             long long *dev_rot, cudaStream_t st) {
    const int n_pad = n + (n & 1);
    const int m_pad = pw_rows_pad(m, n);
    const size_t smem = pointwise_smem_bytes(m_pad, n_pad);
    cudaError_t e = cudaFuncSetAttribute(k_pointwise, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_pointwise<<<1, kThreads, smem, st>>>(G, ldg, m, n, J, m_pad, n_pad, tol, tstop, max_sweeps, sort, Wws,
                                           sigma, U, ldu, V, ldv, dev_out, dev_rot);
    return cudaGetLastError();
}

}  // namespace hsvd
