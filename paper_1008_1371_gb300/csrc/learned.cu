// learned.cu -- the learned form of the blocked method: a small MLP predicts,
// from the previous sweep's record of a block-pair visit, whether that visit
// will need a rotation (its pivot block fails the test of Eq. 2.3); visits
// predicted to pass are skipped.  The plain full sweep stays the judge: a
// masked sweep that rotates nothing is followed by a full sweep, and only a
// full sweep without rotations ends the iteration (Sec. 2 stopping rule), so
// the result never depends on the network.
//
// Network: 8 features -> 64 (ReLU) -> 64 (ReLU) -> 1 (logit), weights rounded
// to BF16, FP32 accumulation.  The same forward code serves inference in the
// solver and the training kernels (forward + backward, then Adam).
//
// Parameter vector (FP32 master copy, kMlpParams floats):
//   W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3.
//
// Features of a visit v (pair of block columns I, J) for sweep k, from the
// record r[v] the inner solve wrote at v's last computed visit:
//   f0 = log2(max scaled |a_ij| over the I x J block / tol) / 64
//   f1 = log2(Frobenius norm of the scaled I x J block) / 64
//   f2 = inner rotations applied / b^2
//   f3 = k / max_sweeps
//   f4 = fraction of (i in I, j in J) with opposite signs (hyperbolic pairs)
//   f5 = log2(mean d over I / mean d over J) / 64
//   f6 = |I - J| / nb
//   f7 = 1 if v was skipped in sweep k - 1, else 0
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "hsvd_internal.cuh"

namespace hsvd {

namespace {

constexpr int kF = 8, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;
static_assert(kParams == HSVD_MLP_PARAMS, "parameter count");

constexpr int kTrainSamples = 64;  // samples per CTA of the training kernel
constexpr int kTrainThreads = 256;

__device__ __forceinline__ float bf16_round(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// weights rounded to BF16 (biases stay FP32) into shared memory
__device__ void load_params(const float *__restrict__ p, float *__restrict__ sp) {
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
        const bool is_w = (i < kOffB1) || (i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3);
        sp[i] = is_w ? bf16_round(p[i]) : p[i];
    }
}

// forward pass of one sample; h1, h2 receive the post-ReLU activations
__device__ __forceinline__ float mlp_forward(const float *__restrict__ sp, const float *__restrict__ x, float *h1,
                                             float *h2) {
    for (int j = 0; j < kH; ++j) {
        float a = sp[kOffB1 + j];
#pragma unroll
        for (int i = 0; i < kF; ++i) a = fmaf(sp[kOffW1 + j * kF + i], x[i], a);
        h1[j] = fmaxf(a, 0.0f);
    }
    for (int j = 0; j < kH; ++j) {
        float a = sp[kOffB2 + j];
        for (int i = 0; i < kH; ++i) a = fmaf(sp[kOffW2 + j * kH + i], h1[i], a);
        h2[j] = fmaxf(a, 0.0f);
    }
    float z = sp[kOffB3];
    for (int i = 0; i < kH; ++i) z = fmaf(sp[kOffW3 + i], h2[i], z);
    return z;
}

__global__ void __launch_bounds__(128) k_mlp_infer(const float *__restrict__ params, const float *__restrict__ X,
                                                   int n, float *__restrict__ logits, int8_t *__restrict__ skip,
                                                   float logit_tau) {
    __shared__ float sp[kParams];
    load_params(params, sp);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kF], h1[kH], h2[kH];
#pragma unroll
    for (int i = 0; i < kF; ++i) x[i] = X[(size_t)s * kF + i];
    const float z = mlp_forward(sp, x, h1, h2);
    if (logits) logits[s] = z;
    if (skip) skip[s] = z < logit_tau ? 1 : 0;
}

// Gradient of the mean binary cross-entropy with logits over n samples,
// L = mean(softplus(z) - y z), per CTA of kTrainSamples samples: partial
// sums over the CTA's samples in a fixed order (deterministic).
__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad_partial(const float *__restrict__ params,
                                                                    const float *__restrict__ X,
                                                                    const float *__restrict__ y, int n,
                                                                    float *__restrict__ gpart,
                                                                    float *__restrict__ lpart) {
    extern __shared__ float sm[];
    float *sp = sm;                                  // kParams
    float *xs = sp + kParams;                        // [S][kF]
    float *h1 = xs + kTrainSamples * kF;             // [S][kH]
    float *h2 = h1 + kTrainSamples * kH;             // [S][kH]
    float *d2 = h2 + kTrainSamples * kH;             // [S][kH]  dL/d(pre-activation 2)
    float *d1 = d2 + kTrainSamples * kH;             // [S][kH]  dL/d(pre-activation 1)
    float *dz = d1 + kTrainSamples * kH;             // [S]
    float *ls = dz + kTrainSamples;                  // [S]
    load_params(params, sp);
    const int s0 = blockIdx.x * kTrainSamples;
    const int ns = min(kTrainSamples, n - s0);
    for (int e = threadIdx.x; e < kTrainSamples * kF; e += blockDim.x) {
        const int s = e / kF;
        xs[e] = s < ns ? X[(size_t)(s0 + s) * kF + e % kF] : 0.0f;
    }
    __syncthreads();
    const float inv_n = 1.0f / (float)n;
    if (threadIdx.x < kTrainSamples) {
        const int s = threadIdx.x;
        float hh1[kH], hh2[kH];
        const float z = mlp_forward(sp, xs + s * kF, hh1, hh2);
        for (int j = 0; j < kH; ++j) {
            h1[s * kH + j] = hh1[j];
            h2[s * kH + j] = hh2[j];
        }
        if (s < ns) {
            const float yy = y[s0 + s];
            const float p = 1.0f / (1.0f + expf(-z));
            dz[s] = (p - yy) * inv_n;
            // softplus(z) - y z, written stably
            ls[s] = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - yy * z;
        } else {
            dz[s] = 0.0f;
            ls[s] = 0.0f;
        }
        for (int j = 0; j < kH; ++j) d2[s * kH + j] = hh2[j] > 0.0f ? dz[s] * sp[kOffW3 + j] : 0.0f;
        for (int i = 0; i < kH; ++i) {
            float a = 0.0f;
            for (int j = 0; j < kH; ++j) a = fmaf(sp[kOffW2 + j * kH + i], d2[s * kH + j], a);
            d1[s * kH + i] = hh1[i] > 0.0f ? a : 0.0f;
        }
    }
    __syncthreads();
    float *g = gpart + (size_t)blockIdx.x * kParams;
    for (int q = threadIdx.x; q < kParams; q += blockDim.x) {
        float a = 0.0f;
        if (q < kOffB1) {
            const int j = q / kF, i = q % kF;
            for (int s = 0; s < kTrainSamples; ++s) a = fmaf(d1[s * kH + j], xs[s * kF + i], a);
        } else if (q < kOffW2) {
            const int j = q - kOffB1;
            for (int s = 0; s < kTrainSamples; ++s) a += d1[s * kH + j];
        } else if (q < kOffB2) {
            const int j = (q - kOffW2) / kH, i = (q - kOffW2) % kH;
            for (int s = 0; s < kTrainSamples; ++s) a = fmaf(d2[s * kH + j], h1[s * kH + i], a);
        } else if (q < kOffW3) {
            const int j = q - kOffB2;
            for (int s = 0; s < kTrainSamples; ++s) a += d2[s * kH + j];
        } else if (q < kOffB3) {
            const int i = q - kOffW3;
            for (int s = 0; s < kTrainSamples; ++s) a = fmaf(dz[s], h2[s * kH + i], a);
        } else {
            for (int s = 0; s < kTrainSamples; ++s) a += dz[s];
        }
        g[q] = a;
    }
    if (threadIdx.x == 0) {
        float l = 0.0f;
        for (int s = 0; s < kTrainSamples; ++s) l += ls[s];
        lpart[blockIdx.x] = l * inv_n;
    }
}

// sum of the CTA partials, in CTA order
__global__ void k_mlp_grad_reduce(const float *__restrict__ gpart, const float *__restrict__ lpart, int nblk,
                                  float *__restrict__ grad, float *__restrict__ loss) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kParams) {
        float a = 0.0f;
        for (int b = 0; b < nblk; ++b) a += gpart[(size_t)b * kParams + q];
        grad[q] = a;
    }
    if (q == 0 && loss) {
        float l = 0.0f;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = l;
    }
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int t, float lr, float b1, float b2, float eps) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kParams) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float mh = mq / (1.0f - powf(b1, (float)t));
    const float vh = vq / (1.0f - powf(b2, (float)t));
    p[q] -= lr * mh / (sqrtf(vh) + eps);
}

// features of every visit (see the file comment); tab holds the first
// columns (I b, J b) of each visit, trace the inner solve's records
__global__ void k_features(const float *__restrict__ trace, const int8_t *__restrict__ prev_skip,
                           const int *__restrict__ tab, int nvis, int b, int nb, int sweep, int max_sweeps,
                           double tol, float *__restrict__ X) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvis) return;
    const float *r = trace + (size_t)v * HSVD_TRACE_FIELDS;
    const float tiny = 1e-30f;
    const float bi = (float)(tab[2 * v] / b), bj = (float)(tab[2 * v + 1] / b);
    float *x = X + (size_t)v * kF;
    x[0] = log2f(fmaxf(r[0], tiny) / (float)tol) * (1.0f / 64.0f);
    x[1] = log2f(fmaxf(r[1], tiny)) * (1.0f / 64.0f);
    x[2] = r[2] / (float)(b * b);
    x[3] = (float)sweep / (float)max_sweeps;
    x[4] = r[5];
    x[5] = log2f(fmaxf(r[3], tiny) / fmaxf(r[4], tiny)) * (1.0f / 64.0f);
    x[6] = fabsf(bi - bj) / (float)nb;
    x[7] = prev_skip ? (float)prev_skip[v] : 0.0f;
}

// training rows (8 features, label = the visit rotated in this sweep)
__global__ void k_export(const float *__restrict__ X, const float *__restrict__ trace, int nvis,
                         float *__restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvis) return;
#pragma unroll
    for (int i = 0; i < kF; ++i) out[(size_t)v * (kF + 1) + i] = X[(size_t)v * kF + i];
    out[(size_t)v * (kF + 1) + kF] = trace[(size_t)v * HSVD_TRACE_FIELDS + 2] > 0.0f ? 1.0f : 0.0f;
}

// the visit table of a masked sweep under the pair schedule: a skipped visit's
// entry becomes (-1, -1), which the Gram and inner-solve kernels treat as "no
// visit"; *kept counts the visits that stay
__global__ void k_mask_table(const int *__restrict__ outer, const int8_t *__restrict__ skip, int nvis,
                             int *__restrict__ tab, int *__restrict__ kept) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const bool keep = v < nvis && !skip[v];
    if (v < nvis) {
        tab[2 * v] = keep ? outer[2 * v] : -1;
        tab[2 * v + 1] = keep ? outer[2 * v + 1] : -1;
    }
    const unsigned n = __popc(__ballot_sync(0xffffffffu, keep));
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(kept, (int)n);
}

size_t grad_smem() {
    return sizeof(float) * (kParams + kTrainSamples * kF + 4 * kTrainSamples * kH + 2 * kTrainSamples);
}

}  // namespace

cudaError_t launch_features(const float *trace, const int8_t *prev_skip, const int *tab, int nvis, int b, int nb,
                            int sweep, int max_sweeps, double tol, float *X, cudaStream_t st) {
    k_features<<<(nvis + 127) / 128, 128, 0, st>>>(trace, prev_skip, tab, nvis, b, nb, sweep, max_sweeps, tol, X);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const float *params, const float *X, int n, float *logits, int8_t *skip,
                             float logit_tau, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_mlp_infer<<<(n + 127) / 128, 128, 0, st>>>(params, X, n, logits, skip, logit_tau);
    return cudaGetLastError();
}

cudaError_t launch_mask_table(const int *outer, const int8_t *skip, int nvis, int *tab, int *kept, cudaStream_t st) {
    k_mask_table<<<(nvis + 127) / 128, 128, 0, st>>>(outer, skip, nvis, tab, kept);
    return cudaGetLastError();
}

cudaError_t launch_export(const float *X, const float *trace, int nvis, float *out, cudaStream_t st) {
    k_export<<<(nvis + 127) / 128, 128, 0, st>>>(X, trace, nvis, out);
    return cudaGetLastError();
}

int mlp_grad_blocks(int n) { return (n + kTrainSamples - 1) / kTrainSamples; }

cudaError_t launch_mlp_grad(const float *params, const float *X, const float *y, int n, float *gpart, float *lpart,
                            float *grad, float *loss, cudaStream_t st) {
    const int nblk = mlp_grad_blocks(n);
    const size_t smem = grad_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_grad_partial<<<nblk, kTrainThreads, smem, st>>>(params, X, y, n, gpart, lpart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_grad_reduce<<<(kParams + 255) / 256, 256, 0, st>>>(gpart, lpart, nblk, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *m, float *v, const float *g, int t, float lr, float b1, float b2, float eps,
                        cudaStream_t st) {
    k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(p, m, v, g, t, lr, b1, b2, eps);
    return cudaGetLastError();
}

}  // namespace hsvd

using namespace hsvd;

extern "C" {

int hsvd_mlp_forward(const float *params, const float *X, int64_t n, float *logits, void *stream) {
    if (!params || !X || !logits || n < 0 || n > (1 << 30)) return HSVD_ERR_ARG;
    if (!all_device({params, X, logits})) return HSVD_ERR_ARG;
    return launch_mlp_infer(params, X, (int)n, logits, nullptr, 0.0f, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? HSVD_OK
               : HSVD_ERR_CUDA;
}

int hsvd_mlp_grad(const float *params, const float *X, const float *y, int64_t n, float *grad, float *loss,
                  void *stream) {
    if (!params || !X || !y || !grad || n < 1 || n > (1 << 26)) return HSVD_ERR_ARG;
    if (!all_device({params, X, y, grad, loss})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblk = mlp_grad_blocks((int)n);
    float *gpart = nullptr, *lpart = nullptr;
    if (cudaMallocAsync((void **)&gpart, sizeof(float) * (size_t)nblk * HSVD_MLP_PARAMS, st) != cudaSuccess)
        return HSVD_ERR_NOMEM;
    if (cudaMallocAsync((void **)&lpart, sizeof(float) * (size_t)nblk, st) != cudaSuccess) {
        cudaFreeAsync(gpart, st);
        return HSVD_ERR_NOMEM;
    }
    const cudaError_t e = launch_mlp_grad(params, X, y, (int)n, gpart, lpart, grad, loss, st);
    cudaFreeAsync(gpart, st);
    cudaFreeAsync(lpart, st);
    return e == cudaSuccess ? HSVD_OK : HSVD_ERR_CUDA;
}

int hsvd_mlp_adam(float *params, float *m, float *v, const float *grad, int t, float lr, float beta1, float beta2,
                  float eps, void *stream) {
    if (!params || !m || !v || !grad || t < 1 || !(lr > 0.0f)) return HSVD_ERR_ARG;
    if (!all_device({params, m, v, grad})) return HSVD_ERR_ARG;
    return launch_adam(params, m, v, grad, t, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? HSVD_OK
               : HSVD_ERR_CUDA;
}

}  // extern "C"
