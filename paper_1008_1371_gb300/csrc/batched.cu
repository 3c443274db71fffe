// batched.cu -- the batched form: many independent factors (sizes mixed) in
// one persistent launch, each solved by the pointwise one-sided hyperbolic
// Jacobi method (Sec. 2, Alg. 4.5; the per-factor body is pw_solve).
//
// Work distribution.  The host sorts the factors by (group width, n), both
// decreasing, and the kernel's CTAs (1024 threads, or 512 with twice the
// registers a thread, one per SM, launched once and captured in a CUDA graph)
// take them from one atomic counter: the largest
// first, so the long factors start early and the short ones fill the tail.
// A CTA starts as one group of 1024 threads.  When the next factor in the
// queue asks for a narrower group, the CTA splits into two groups of 512
// (each with half the shared memory and its own named barrier), and a 512
// group splits again into two groups of 256; every group then takes factors
// from the same counter on its own.  The queue order makes the widths
// non-increasing, so a group never has to grow back.
//
// Residency.  In its group's shared memory a factor keeps G and W when both
// fit, otherwise G only (W then in a per-group slot of a global workspace,
// L2-resident), otherwise neither.
//
// The autotuner (host, tune_widths) picks the group width per size bucket by
// timing each width on a sample of that bucket's factors for two sweeps, and
// caches the choice per device and bucket layout.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pw_core.cuh"

namespace hsvd {
namespace {

constexpr int kBarriers = 7;  // 1 (1024) + 2 (512) + 4 (256)

struct BTask {
    const double *G;
    const int8_t *J;
    double *sigma, *U, *V;
    int64_t ldg, ldu, ldv;
    double tol;
    int m, n, idx, width;
};

struct BArgs {
    const BTask *tasks;
    int count;
    int *counter;
    int max_sweeps, sort;
    double tstop;        // tangent threshold of the early stop, 0 = off
    double *ws;          // grid x ws_stride doubles
    int64_t ws_stride;   // doubles per CTA
    int *res;            // 3 per factor: status, sweeps, stop rule
    long long *rot;      // per factor
    int *where;          // per factor: 0 G and W shared, 1 G shared, 2 global
};

__device__ __forceinline__ int bar_id(int width, int g) { return width == 1024 ? 0 : (width == 512 ? 1 + g : 3 + g); }

template <int NT>
__device__ void solve_task(const BArgs &A, int k, int g, unsigned char *sm, size_t budget, double *wsg,
                           PwScalars *sc) {
    const BTask t = A.tasks[k];
    const int n_pad = t.n + (t.n & 1), m_pad = pw_rows_pad(t.m, t.n);
    const size_t gb = (size_t)m_pad * n_pad * sizeof(double), wb = (size_t)n_pad * n_pad * sizeof(double);
    const size_t ab = pw_aux_bytes(n_pad);
    PwArrays a;
    unsigned char *aux;
    int where;
    if (gb + wb + ab <= budget) {
        a.G = reinterpret_cast<double *>(sm);
        a.W = a.G + (size_t)m_pad * n_pad;
        aux = sm + gb + wb;
        where = 0;
    } else if (gb + ab <= budget) {
        a.G = reinterpret_cast<double *>(sm);
        a.W = wsg;
        aux = sm + gb;
        where = 1;
    } else {
        a.G = wsg;
        a.W = wsg + (size_t)m_pad * n_pad;
        aux = sm;
        where = 2;
    }
    a.d = reinterpret_cast<double *>(aux);
    a.pos = reinterpret_cast<int *>(a.d + n_pad);
    a.newpos = a.pos + n_pad;
    a.sg = a.newpos + n_pad;
    const int bar = bar_id(NT, g);
    int *res = A.res + 3 * (size_t)t.idx;
    pw_solve<NT>(t.G, t.ldg, t.m, t.n, t.J, m_pad, n_pad, t.tol, A.tstop, A.max_sweeps, A.sort, a, sc[bar], t.sigma,
                 t.U, t.ldu, t.V, t.ldv, &res[0], &res[1], &A.rot[t.idx], &res[2], bar);
    if ((threadIdx.x & (NT - 1)) == 0) A.where[t.idx] = where;
}

// Group g of width NT: solves factors from the queue, starting with factor k
// (k < 0: take one from the counter first).
template <int NT>
__device__ void group_loop(const BArgs &A, int k, int g, unsigned char *sm, size_t budget, double *wsg,
                           int64_t wsg_len, PwScalars *sc, int *fetch) {
    const int bar = bar_id(NT, g);
    const int tid = threadIdx.x & (NT - 1);
    for (;;) {
        if (k < 0) {
            if (tid == 0) fetch[bar] = atomicAdd(A.counter, 1);
            grp_sync<NT>(bar);
            k = fetch[bar];
            grp_sync<NT>(bar);
        }
        if (k >= A.count) return;
        if constexpr (NT > 256) {
            if (A.tasks[k].width < NT) {
                const int sub = tid / (NT / 2);
                group_loop<NT / 2>(A, sub == 0 ? k : -1, 2 * g + sub, sm + sub * (budget / 2), budget / 2,
                                   wsg + sub * (wsg_len / 2), wsg_len / 2, sc, fetch);
                return;
            }
        }
        solve_task<NT>(A, k, g, sm, budget, wsg, sc);
        k = -1;
    }
}

// CTA threads: 1024 (64 registers a thread) or 512 (128: the per-thread
// state of pw_solve without spills)
template <int CTA>
__global__ void __launch_bounds__(CTA, 1) k_batched(BArgs A, int smem_budget) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PwScalars sc[kBarriers];
    __shared__ int fetch[kBarriers];
    group_loop<CTA>(A, -1, 0, smem, (size_t)smem_budget, A.ws + (size_t)blockIdx.x * A.ws_stride, A.ws_stride, sc,
                    fetch);
}

// ------------------------------------------------------------------ host side

constexpr int kSmemBudget = 220 * 1024;  // one CTA per SM
const int kBucketEdges[] = {16, 40, 72, 128, 192, 1 << 30};
constexpr int kBuckets = 5;

int bucket_of(int64_t n) {
    for (int b = 0; b < kBuckets; ++b)
        if (n < kBucketEdges[b + 1]) return b;
    return kBuckets - 1;
}

size_t need_bytes(int64_t m, int64_t n) {
    const int64_t n_pad = n + (n & 1), m_pad = pw_rows_pad(m, n);
    return (size_t)(m_pad * n_pad + n_pad * n_pad) * sizeof(double);
}

// workspace doubles per CTA: a group of width w owns w/cta of the slot, and
// must hold G and W of any factor it may take
int64_t ws_stride_for(const std::vector<BTask> &tasks, int cta) {
    size_t s = 0;
    for (const BTask &t : tasks) s = std::max(s, need_bytes(t.m, t.n) * (size_t)(cta / t.width));
    return (int64_t)((s / sizeof(double) + 31) / 32 * 32);
}

struct Launch {
    int grid = 0;
    cudaError_t err = cudaSuccess;
};

// Runs the persistent kernel over `tasks` (already in queue order) as one
// captured graph: counter reset + the launch.
cudaError_t run_batch(const std::vector<BTask> &tasks, int max_sweeps, int sort, double tstop, bool use_graph,
                      int grid, int cta, int *res, long long *rot, int *where, cudaStream_t st, float *ms) {
    const int count = (int)tasks.size();
    const int64_t stride = ws_stride_for(tasks, cta);
    void (*kern)(BArgs, int) = cta == 512 ? k_batched<512> : k_batched<1024>;
    BTask *d_tasks = nullptr;
    int *d_counter = nullptr;
    double *d_ws = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_tasks, sizeof(BTask) * (size_t)count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_counter, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_ws, sizeof(double) * (size_t)grid * stride + 64, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(BTask) * (size_t)count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
    BArgs A;
    A.tasks = d_tasks;
    A.count = count;
    A.counter = d_counter;
    A.max_sweeps = max_sweeps;
    A.sort = sort;
    A.tstop = tstop;
    A.ws = d_ws;
    A.ws_stride = stride;
    A.res = res;
    A.rot = rot;
    A.where = where;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess && ms) {
        e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && use_graph) {
        // the memset and the launch form the graph; a stream that is itself
        // being captured gets the two nodes directly
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e == cudaSuccess && cs != cudaStreamCaptureStatusNone) use_graph = false;
    }
    if (e == cudaSuccess && use_graph) {
        cudaStream_t cap = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(d_counter, 0, sizeof(int), cap);
            kern<<<grid, cta, kSmemBudget, cap>>>(A, kSmemBudget);
            const cudaError_t le = cudaGetLastError();
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (cap) cudaStreamDestroy(cap);
        if (e == cudaSuccess && ms) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess && ms) e = cudaEventRecord(e1, st);
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
        if (e == cudaSuccess && ms) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            kern<<<grid, cta, kSmemBudget, st>>>(A, kSmemBudget);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && ms) e = cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess && ms) {
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_tasks) cudaFreeAsync(d_tasks, st);
    if (d_counter) cudaFreeAsync(d_counter, st);
    if (d_ws) cudaFreeAsync(d_ws, st);
    return e;
}

// queue order: width decreasing, then n decreasing, then input order
void order_tasks(std::vector<BTask> &tasks) {
    std::stable_sort(tasks.begin(), tasks.end(), [](const BTask &a, const BTask &b) {
        if (a.width != b.width) return a.width > b.width;
        return a.n > b.n;
    });
}

std::mutex g_tune_mu;
std::map<long long, std::vector<int>> g_tune_cache;  // (device, CTA, bucket mask) -> width per bucket

// Picks the group width of every size bucket present: each candidate width is
// timed on up to (SMs x 1024 / width) factors of the bucket, two sweeps each,
// and scored by sum(m n^2) / time.
long long tune_key(int dev, int cta, long long mask) { return ((long long)dev << 32) | ((long long)cta << 16) | mask; }

cudaError_t tune_widths(const std::vector<BTask> &all, int grid, int cta, int *res, long long *rot, int *where,
                        cudaStream_t st, std::vector<int> &width, float *ms_total) {
    width.assign(kBuckets, cta);
    int dev = 0;
    cudaGetDevice(&dev);
    long long mask = 0;
    for (const BTask &t : all) mask |= 1LL << bucket_of(t.n);
    const long long key = tune_key(dev, cta, mask);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            width = it->second;
            return cudaSuccess;
        }
    }
    for (int b = 0; b < kBuckets; ++b) {
        if (!(mask & (1LL << b))) continue;
        std::vector<BTask> members;
        for (const BTask &t : all)
            if (bucket_of(t.n) == b) members.push_back(t);
        double best = -1.0;
        for (int w : {1024, 512, 256}) {
            if (w > cta) continue;
            const size_t want = (size_t)grid * (cta / w);
            std::vector<BTask> sample;
            const size_t stepk = std::max<size_t>(1, members.size() / want);
            for (size_t i = 0; i < members.size() && sample.size() < want; i += stepk) sample.push_back(members[i]);
            double work = 0.0;
            for (BTask &t : sample) {
                t.width = w;
                work += (double)t.m * t.n * t.n;
            }
            order_tasks(sample);
            float ms = 0.f;
            const cudaError_t e = run_batch(sample, 2, 1, 0.0, false, grid, cta, res, rot, where, st, &ms);
            if (e != cudaSuccess) return e;
            if (ms_total) *ms_total += ms;
            const double score = work / std::max(ms, 1e-3f);
            if (score > best) {
                best = score;
                width[b] = w;
            }
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = width;
    return cudaSuccess;
}

}  // namespace
}  // namespace hsvd

using namespace hsvd;

extern "C" {

void hsvd_default_batch_opts(hsvd_batch_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->tol = 0.0;
    o->max_sweeps = 30;
    o->sort = 1;
    o->group_width = 0;
    o->use_graph = 1;
}

int hsvd_solve_batched_ex(int64_t count, const double *const *G, const int64_t *m, const int64_t *n,
                          const int64_t *ldg, const int8_t *const *J, double *const *sigma, double *const *U,
                          double *const *V, int *sweeps, int *status, const hsvd_batch_opts *opts,
                          hsvd_batch_info *info, void *stream) {
    hsvd_batch_opts o;
    if (opts) o = *opts;
    else hsvd_default_batch_opts(&o);
    if (count < 0 || (count > 0 && (!G || !m || !n || !ldg || !J || !sigma))) return HSVD_ERR_ARG;
    if (o.max_sweeps <= 0) o.max_sweeps = 30;
    if (o.group_width != 0 && o.group_width != 256 && o.group_width != 512 && o.group_width != 1024)
        return HSVD_ERR_ARG;
    if (o.cta_threads != 0 && o.cta_threads != 512 && o.cta_threads != 1024) return HSVD_ERR_ARG;
    const int cta = o.cta_threads ? o.cta_threads : 1024;
    if (o.group_width > cta) return HSVD_ERR_ARG;
    if (o.reserved) return HSVD_ERR_ARG;
    if (o.tstop < 0.0) o.tstop = HSVD_TSTOP_PAPER;
    if (!(o.tstop >= 0.0 && o.tstop <= 1.0)) return HSVD_ERR_ARG;
    if (info) memset(info, 0, sizeof *info);
    if (count == 0) return HSVD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // host arrays: stage through device copies, one copy per matrix
    const bool host = !is_device_ptr(G[0]);
    std::vector<BTask> tasks((size_t)count);
    size_t g_off = 0, j_off = 0, s_off = 0, u_off = 0, v_off = 0;
    for (int64_t k = 0; k < count; ++k) {
        if (n[k] < 1 || m[k] < n[k] || ldg[k] < m[k] || n[k] > 2048 || m[k] > 4096) return HSVD_ERR_ARG;
        if (!G[k] || !J[k] || !sigma[k]) return HSVD_ERR_ARG;
        // all of one kind: host arrays are staged, device arrays used in place
        if (is_device_ptr(G[k]) == host || is_device_ptr(J[k]) == host || is_device_ptr(sigma[k]) == host)
            return HSVD_ERR_ARG;
        if ((U && U[k] && is_device_ptr(U[k]) == host) || (V && V[k] && is_device_ptr(V[k]) == host))
            return HSVD_ERR_ARG;
        if (need_bytes(m[k], n[k]) > (size_t)1 << 30) return HSVD_ERR_ARG;
        BTask &t = tasks[(size_t)k];
        t.m = (int)m[k];
        t.n = (int)n[k];
        t.idx = (int)k;
        t.ldg = host ? m[k] : ldg[k];
        t.ldu = m[k];
        t.ldv = n[k];
        t.tol = o.tol > 0.0 ? o.tol : (double)n[k] * 0x1p-53;
        g_off += (size_t)(m[k] * n[k]);
        j_off += (size_t)n[k];
        s_off += (size_t)n[k];
        if (U && U[k]) u_off += (size_t)(m[k] * n[k]);
        if (V && V[k]) v_off += (size_t)(n[k] * n[k]);
    }
    int rc = HSVD_OK;
    double *dG = nullptr, *dS = nullptr, *dU = nullptr, *dV = nullptr;
    int8_t *dJ = nullptr;
    int *d_res = nullptr, *d_where = nullptr;
    long long *d_rot = nullptr;
    auto fail = [&](int code) {
        if (rc == HSVD_OK) rc = code;
    };
    if (cudaMallocAsync((void **)&d_res, sizeof(int) * 3 * (size_t)count, st) != cudaSuccess ||
        cudaMallocAsync((void **)&d_where, sizeof(int) * (size_t)count, st) != cudaSuccess ||
        cudaMallocAsync((void **)&d_rot, sizeof(long long) * (size_t)count, st) != cudaSuccess)
        fail(HSVD_ERR_NOMEM);
    if (rc == HSVD_OK && host) {
        if (cudaMallocAsync((void **)&dG, sizeof(double) * g_off + 16, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dJ, j_off + 16, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dS, sizeof(double) * s_off + 16, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dU, sizeof(double) * u_off + 16, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dV, sizeof(double) * v_off + 16, st) != cudaSuccess)
            fail(HSVD_ERR_NOMEM);
    }
    size_t go = 0, jo = 0, so = 0, uo = 0, vo = 0;
    for (int64_t k = 0; k < count && rc == HSVD_OK; ++k) {
        BTask &t = tasks[(size_t)k];
        if (host) {
            t.G = dG + go;
            t.J = dJ + jo;
            t.sigma = dS + so;
            t.U = (U && U[k]) ? dU + uo : nullptr;
            t.V = (V && V[k]) ? dV + vo : nullptr;
            if (cudaMemcpy2DAsync(dG + go, sizeof(double) * m[k], G[k], sizeof(double) * ldg[k], sizeof(double) * m[k],
                                  n[k], cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(dJ + jo, J[k], n[k], cudaMemcpyHostToDevice, st) != cudaSuccess)
                fail(HSVD_ERR_CUDA);
            go += (size_t)(m[k] * n[k]);
            jo += (size_t)n[k];
            so += (size_t)n[k];
            if (t.U) uo += (size_t)(m[k] * n[k]);
            if (t.V) vo += (size_t)(n[k] * n[k]);
        } else {
            t.G = G[k];
            t.J = J[k];
            t.sigma = sigma[k];
            t.U = U ? U[k] : nullptr;
            t.V = V ? V[k] : nullptr;
        }
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(sms, count);
    std::vector<int> width(kBuckets, o.group_width ? o.group_width : cta);
    float ms_tune = 0.f;
    int tuned = 0;
    if (rc == HSVD_OK && o.group_width == 0) {
        std::vector<int> w;
        const bool cached = [&] {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            long long mask = 0;
            for (const BTask &t : tasks) mask |= 1LL << bucket_of(t.n);
            return g_tune_cache.count(tune_key(dev, cta, mask)) > 0;
        }();
        if (tune_widths(tasks, sms, cta, d_res, d_rot, d_where, st, w, &ms_tune) != cudaSuccess) fail(HSVD_ERR_CUDA);
        else width = w;
        tuned = cached ? 2 : 1;
    }
    for (BTask &t : tasks) t.width = width[(size_t)bucket_of(t.n)];
    order_tasks(tasks);
    float ms = 0.f;
    if (rc == HSVD_OK &&
        run_batch(tasks, o.max_sweeps, o.sort ? 1 : 0, o.tstop, o.use_graph != 0, grid, cta, d_res, d_rot, d_where,
                  st, &ms) != cudaSuccess)
        fail(HSVD_ERR_CUDA);
    std::vector<int> h_res(3 * (size_t)count, 0), h_where((size_t)count, 0);
    std::vector<long long> h_rot((size_t)count, 0);
    if (rc == HSVD_OK &&
        (cudaMemcpyAsync(h_res.data(), d_res, sizeof(int) * 3 * (size_t)count, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(h_where.data(), d_where, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(h_rot.data(), d_rot, sizeof(long long) * (size_t)count, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess))
        fail(HSVD_ERR_CUDA);
    if (rc == HSVD_OK && host) {
        // results back, one copy per array
        size_t so2 = 0, uo2 = 0, vo2 = 0;
        for (int64_t k = 0; k < count && rc == HSVD_OK; ++k) {
            if (cudaMemcpyAsync(sigma[k], dS + so2, sizeof(double) * n[k], cudaMemcpyDeviceToHost, st) != cudaSuccess)
                fail(HSVD_ERR_CUDA);
            so2 += (size_t)n[k];
            if (U && U[k]) {
                if (cudaMemcpyAsync(U[k], dU + uo2, sizeof(double) * m[k] * n[k], cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
                    fail(HSVD_ERR_CUDA);
                uo2 += (size_t)(m[k] * n[k]);
            }
            if (V && V[k]) {
                if (cudaMemcpyAsync(V[k], dV + vo2, sizeof(double) * n[k] * n[k], cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
                    fail(HSVD_ERR_CUDA);
                vo2 += (size_t)(n[k] * n[k]);
            }
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) fail(HSVD_ERR_CUDA);
    int worst = HSVD_OK;
    if (rc == HSVD_OK) {
        for (int64_t k = 0; k < count; ++k) {
            const int s_k = h_res[3 * (size_t)k];
            if (status) status[k] = s_k;
            if (sweeps) sweeps[k] = h_res[3 * (size_t)k + 1];
            if (s_k < 0 && worst >= 0) worst = s_k;
            else if (s_k == HSVD_NOT_CONVERGED && worst == HSVD_OK) worst = s_k;
        }
        if (info) {
            info->grid = grid;
            info->cta_threads = cta;
            info->tuned = tuned;
            for (int b = 0; b < 5; ++b) info->bucket_width[b] = width[(size_t)b];
            info->ms_kernel = ms;
            info->ms_tune = ms_tune;
            info->kernel_launches = 1;
            for (int64_t k = 0; k < count; ++k) {
                info->rotations += h_rot[(size_t)k];
                info->max_sweeps_run = std::max(info->max_sweeps_run, h_res[3 * (size_t)k + 1]);
                info->tangent_stops += h_res[3 * (size_t)k + 2] == HSVD_STOP_TANGENT;
                info->resident[std::min(2, std::max(0, h_where[(size_t)k]))] += 1;
            }
        }
    }
    if (d_res) cudaFreeAsync(d_res, st);
    if (d_where) cudaFreeAsync(d_where, st);
    if (d_rot) cudaFreeAsync(d_rot, st);
    if (dG) cudaFreeAsync(dG, st);
    if (dJ) cudaFreeAsync(dJ, st);
    if (dS) cudaFreeAsync(dS, st);
    if (dU) cudaFreeAsync(dU, st);
    if (dV) cudaFreeAsync(dV, st);
    if (host) cudaStreamSynchronize(st);
    return rc != HSVD_OK ? rc : worst;
}

int hsvd_solve_batched(int64_t count, const double *const *G, const int64_t *m, const int64_t *n, const int64_t *ldg,
                       const int8_t *const *J, double tol, int max_sweeps, double *const *sigma, double *const *U,
                       double *const *V, int *sweeps, int *status, void *stream) {
    hsvd_batch_opts o;
    hsvd_default_batch_opts(&o);
    o.tol = tol;
    o.max_sweeps = max_sweeps;
    return hsvd_solve_batched_ex(count, G, m, n, ldg, J, sigma, U, V, sweeps, status, &o, nullptr, stream);
}

}  // extern "C"
