// api.cu -- the C ABI (include/hsvd.h): argument checks, host/device staging,
// workspace, and the sweep driver of the blocked method (Alg. 4.1 on the host:
// one CUDA graph per sweep, one synchronisation per sweep to read the
// convergence counter).
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <math.h>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hsvd_internal.cuh"

namespace hsvd {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool all_device(std::initializer_list<const void *> ps) {
    for (const void *p : ps)
        if (p && !is_device_ptr(p)) return false;
    return true;
}

}  // namespace hsvd

using namespace hsvd;

namespace {

// Modified modulus pairs on r indices (Sec. 2), closed form: step s holds the
// pairs (a, b), a < b, with a + b = (r - 1 + s) mod r (mod r), plus
// (c/2, c/2 + r/2) for even residue c; slots ordered by a.
void fill_modulus(int r, int nsteps, int *pairs) {
    const int h = r / 2;
    for (int s = 0; s < nsteps; ++s)
        for (int k = 0; k < h; ++k) {
            int a, b;
            modulus_pair(r, s, k, a, b);
            pairs[2 * (s * h + k)] = a;
            pairs[2 * (s * h + k) + 1] = b;
        }
}

// Cross pass over the off-diagonal block of a 2h x 2h pivot block: step s
// pairs (k, h + (k + s) mod h).
void fill_cross(int h, int *pairs) {
    for (int s = 0; s < h; ++s)
        for (int k = 0; k < h; ++k) {
            pairs[2 * (s * h + k)] = k;
            pairs[2 * (s * h + k) + 1] = h + (k + s) % h;
        }
}

struct Ws {
    std::vector<void *> ptrs;
    cudaStream_t st;
    explicit Ws(cudaStream_t s) : st(s) {}
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, count * sizeof(T) + 16, st) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Ws() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

int64_t round_up(int64_t x, int64_t k) { return (x + k - 1) / k * k; }

// Block width when none is given.  Measured on graded factors (FP64, pair
// schedule, whole HSVD): n = 512: b = 16/32/64 take 36.1/33.6/47.0 ms; n = 1024:
// 122.3/126.0/153.6 ms; n = 1536: 311/334/360 ms; n = 2048: 685/734/821 ms.
int choose_block(int64_t n) {
    if (n >= 1024 && n <= 2048) return 16;
    if (n >= 512) return 32;
    return 16;
}

struct SweepStats {
    int sweeps = 0;
    long long rotations = 0, pair_updates = 0, launches = 0;
    double ms_gram = 0, ms_solve = 0, ms_update = 0, ms_other = 0;
    double ms_host_graph = 0;  // host wall time capturing and instantiating sweep graphs
    long long pair_visits = 0, trace_rows = 0;
    int masked_sweeps = 0, judge_sweeps = 0;
    int stop_rule = HSVD_STOP_NONE;
};

// CUDA events recorded as graph nodes around every kernel of a sweep when
// profiling: ev[4 s + 0..3] bracket Gram / solve / update of step s, the last
// two bracket the reordering.
struct SweepEvents {
    std::vector<cudaEvent_t> ev;
    ~SweepEvents() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    bool create(size_t count) {
        ev.assign(count, nullptr);
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return false;
        return true;
    }
    cudaError_t record(size_t i, cudaStream_t st) {  // inside a stream capture
        return ev.empty() ? cudaSuccess : cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
    }
    cudaError_t record_now(size_t i, cudaStream_t st) {  // outside a capture
        return ev.empty() ? cudaSuccess : cudaEventRecord(ev[i], st);
    }
    float between(size_t a, size_t b) const {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return ms;
    }
};

struct GraphGuard {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int *h_cnt = nullptr;
    int *h_tab = nullptr;
    ~GraphGuard() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (h_cnt) cudaFreeHost(h_cnt);
        if (h_tab) cudaFreeHost(h_tab);
    }
};

// Streams and events with which a sweep of the pair schedule is captured:
// one stream per visit slot, one event per block column (its last writer),
// and the fork and join events of the capture.
constexpr int kRing = 3;
constexpr int64_t kMaxNodes = 1536;
struct DagStreams {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> col, join;
    cudaEvent_t fork = nullptr;
    bool create(int nstreams, int ncols) {
        streams.assign((size_t)nstreams, nullptr);
        join.assign((size_t)nstreams, nullptr);
        col.assign((size_t)ncols, nullptr);
        for (auto &x : streams)
            if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return false;
        for (auto *v : {&join, &col})
            for (auto &e : *v)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
        return cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    }
    ~DagStreams() {
        for (auto x : streams)
            if (x) cudaStreamDestroy(x);
        for (auto *v : {&join, &col})
            for (auto e : *v)
                if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
};

#define CKR(expr)                                   \
    do {                                            \
        if ((expr) != cudaSuccess) return HSVD_ERR_CUDA; \
    } while (0)

// A named range on the timeline of a profiler that reads NVTX (a no-op
// without one): the solve, each sweep, the front and back ends.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Blocked method on device arrays (Sec. 5; host loop of Alg. 4.1).
int solve_blocked_core(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma,
                       double *U, int64_t ldu, double *V, int64_t ldv, const hsvd_opts &o, double tol, int b,
                       SweepStats &stats, cudaStream_t st) {
    const int nn = 2 * b;
    const int64_t n_pad = round_up(n, nn);
    const int64_t m_pad = round_up(m + (n_pad - n), 64);
    const int64_t ldw = round_up(n_pad, 64);
    const int nb = (int)(n_pad / b);
    const int npairs = nb / 2;
    const int nsplit = gram_nsplit(m_pad, npairs);
    // The pair schedule runs visits of up to kRing consecutive steps at once:
    // every visit slot (Gram partials, W_P, flags) exists once per step of the
    // ring.  The step schedule needs one per pair.  Measured (graded factors,
    // FP64): 9.5% faster at n = 1024, b = 32, 2.4% at n = 2048; split precision
    // at Haar 4096: 1.1% faster (1426 against 1442 ms per HSVD).  Automatic
    // choice takes it unless the call profiles its kernels one by one.
    const bool pair_sched =
        o.schedule == HSVD_SCHEDULE_PAIRS || (o.schedule == HSVD_SCHEDULE_AUTO && !o.profile);
    const int nslot = pair_sched ? kRing * npairs : npairs;
    GraphGuard gg;
    DagStreams dag;
    Ws ws(st);
    double *Gw = ws.get<double>(m_pad * n_pad), *Gt = ws.get<double>(m_pad * n_pad);
    double *Ww = ws.get<double>(ldw * n_pad), *Wt = ws.get<double>(ldw * n_pad);
    int *perm = ws.get<int>(n_pad), *perm_t = ws.get<int>(n_pad), *newpos = ws.get<int>(n_pad);
    int8_t *sgn = ws.get<int8_t>(n_pad), *sgn_t = ws.get<int8_t>(n_pad);
    double *d = ws.get<double>(n_pad);
    // Gram partials: a step with np active pairs uses gram_nsplit(m_pad, np) row splits
    // (the pair schedule launches one pair at a time with the full step's split)
    int64_t part_items = (int64_t)nslot * nsplit;
    for (int np = 1; np <= npairs; ++np)
        part_items = std::max<int64_t>(part_items, (int64_t)np * gram_nsplit(m_pad, np));
    double *part = ws.get<double>((size_t)part_items * 3 * b * b);
    double *Wp = ws.get<double>((size_t)nslot * nn * nn);
    int *rotated = ws.get<int>(nslot);
    // counters: [0] status (int), [2..3] rotations (u64), [4..5] updated pairs (u64),
    // [6] a rotation of the sweep had |t| > tstop (the (11)_2 code of Eq. 4.2),
    // [7] visits kept by the skip mask of a masked sweep
    int *cnt = ws.get<int>(8);
    int *d_tab_outer = ws.get<int>((size_t)nb * npairs * 2);
    int *d_tab_full = ws.get<int>((size_t)nn * b * 2 + ring_table_ints(b));
    int *d_tab_cross = ws.get<int>((size_t)b * b * 2);
    if (!Gw || !Gt || !Ww || !Wt || !perm || !perm_t || !newpos || !sgn || !sgn_t || !d || !part || !Wp ||
        !rotated || !cnt || !d_tab_outer || !d_tab_full || !d_tab_cross)
        return HSVD_ERR_NOMEM;
    // split-precision products: full 2b x 2b Gram partials, W' slices, exponents
    const bool prec = o.precision == HSVD_PRECISION_BF16X8;
    const int ksplit_x = prec ? precision_gram_ksplit(m_pad) : 0;
    double *part_x = prec ? ws.get<double>((size_t)nslot * ksplit_x * nn * nn) : nullptr;
    uint16_t *wsl = prec ? ws.get<uint16_t>(precision_wsl_elems(nslot)) : nullptr;
    int *wexp = prec ? ws.get<int>((size_t)nslot * 2 * nn) : nullptr;
    int *dexp = prec ? ws.get<int>((size_t)nslot * nn) : nullptr;
    if (prec && (!part_x || !wsl || !wexp || !dexp)) return HSVD_ERR_NOMEM;
    unsigned long long *rot_ctr = reinterpret_cast<unsigned long long *>(cnt + 2);
    unsigned long long *upd_ctr = reinterpret_cast<unsigned long long *>(cnt + 4);
    const bool tangent_stop = o.tstop > 0.0;
    int *tbig = tangent_stop ? cnt + 6 : nullptr;
    // pair tables: outer over nb block columns as first-column indices
    std::vector<int> outer((size_t)nb * npairs * 2);
    fill_modulus(nb, nb, outer.data());
    for (auto &v : outer) v *= b;
    {
        std::vector<int> full((size_t)nn * b * 2 + ring_table_ints(b)), cross((size_t)b * b * 2);
        fill_modulus(nn, nn, full.data());
        if (!fill_ring(b, full.data() + (size_t)nn * b * 2)) return HSVD_ERR_ARG;
        fill_cross(b, cross.data());
        CKR(cudaMemcpyAsync(d_tab_outer, outer.data(), outer.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CKR(cudaMemcpyAsync(d_tab_full, full.data(), full.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CKR(cudaMemcpyAsync(d_tab_cross, cross.data(), cross.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CKR(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    CKR(cudaMallocHost(&gg.h_cnt, 8 * sizeof(int)));
    int *h_cnt = gg.h_cnt;
    CKR(cudaMemsetAsync(cnt, 0, 8 * sizeof(int), st));
    CKR(launch_load_pad(G, ldg, m, n, J, Gw, m_pad, n_pad, Ww, ldw, perm, sgn, cnt, st));
    CKR(launch_reorder(Gw, Gt, m_pad, Ww, Wt, ldw, n_pad, perm, perm_t, sgn, sgn_t, d, newpos, o.sort, st));
    CKR(cudaMemcpyAsync(h_cnt, cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (h_cnt[0] != 0) return h_cnt[0];

    const int reorder_kernels = o.sort ? 3 : 2;
    stats.launches += 1 + reorder_kernels;
    SweepEvents evs;
    if (o.profile && !evs.create((size_t)nb * 4 + 4)) return HSVD_ERR_CUDA;
    const size_t evr = (size_t)nb * 4;

    // learned form and training export: one record per block-pair visit
    const int nvis = nb * npairs;
    const bool learned = o.skip_model != nullptr, export_rows = o.trace_out != nullptr;
    float *trace = nullptr, *X = nullptr, *params = nullptr;
    int8_t *skip = nullptr, *prev_skip = nullptr;
    int *d_visit = nullptr, *d_tab_mask = nullptr, *d_visit_mask = nullptr;
    int *h_tab = nullptr, *h_vis = nullptr;
    int8_t *h_skip = nullptr;
    if (learned || export_rows) {
        trace = ws.get<float>((size_t)nvis * HSVD_TRACE_FIELDS);
        X = ws.get<float>((size_t)nvis * HSVD_MLP_FEATURES);
        d_visit = ws.get<int>(nvis);
        prev_skip = ws.get<int8_t>(nvis);
        if (!trace || !X || !d_visit || !prev_skip) return HSVD_ERR_NOMEM;
        std::vector<int> ident((size_t)nvis);
        for (int v = 0; v < nvis; ++v) ident[(size_t)v] = v;
        CKR(cudaMemcpyAsync(d_visit, ident.data(), sizeof(int) * nvis, cudaMemcpyHostToDevice, st));
        CKR(cudaMemsetAsync(trace, 0, sizeof(float) * nvis * HSVD_TRACE_FIELDS, st));
        CKR(cudaMemsetAsync(prev_skip, 0, nvis, st));
        CKR(cudaStreamSynchronize(st));
    }
    if (learned) {
        params = ws.get<float>(HSVD_MLP_PARAMS);
        skip = ws.get<int8_t>(nvis);
        d_tab_mask = ws.get<int>((size_t)nvis * 2);
        d_visit_mask = ws.get<int>(nvis);
        if (!params || !skip || !d_tab_mask || !d_visit_mask) return HSVD_ERR_NOMEM;
        CKR(cudaMemcpyAsync(params, o.skip_model, sizeof(float) * HSVD_MLP_PARAMS, cudaMemcpyDefault, st));
        CKR(cudaMallocHost(&gg.h_tab, sizeof(int) * (size_t)nvis * 3 + nvis));
        h_tab = gg.h_tab;
        h_vis = h_tab + (size_t)nvis * 2;
        h_skip = reinterpret_cast<int8_t *>(h_vis + nvis);
    }
    const std::vector<int> &outer_host = outer;
    const double tau = o.skip_tau > 0.0 ? o.skip_tau : 0.5;
    const float logit_tau = (float)log(tau / (1.0 - tau));

    // One sweep as a graph: for every step s with nact[s] > 0 pairs, whose first
    // columns are tab + off[s] and visit indices vis + off[s]: Gram, inner
    // solve, update; then the reordering and the read-back of the counters.
    auto capture = [&](const int *tab, const int *vis, const std::vector<int> &nact, const std::vector<int> &off,
                       cudaGraph_t *graph, long long *launches) -> cudaError_t {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        long long nl = 0;
        e = cudaMemsetAsync(cnt + 2, 0, 5 * sizeof(int), st);
        for (int s = 0; s < nb && e == cudaSuccess; ++s) {
            const int np = nact[(size_t)s];
            if (np == 0) continue;
            const int *col0 = tab + off[(size_t)s] * 2;
            const int *vs = vis ? vis + off[(size_t)s] : nullptr;
            const int ns = gram_nsplit(m_pad, np);
            const int mode = (o.inner_mode == HSVD_INNER_FULL) ? 0 : (s == 0 ? 2 : 1);
            e = evs.record(4 * s, st);
            if (e == cudaSuccess)
                e = prec ? launch_gram_x(Gw, m_pad, m_pad, np, col0, part_x, cnt, st)
                         : launch_gram(Gw, m_pad, m_pad, b, np, col0, ns, part, st);
            if (e == cudaSuccess) e = evs.record(4 * s + 1, st);
            if (e == cudaSuccess)
                e = prec ? launch_solve(b, np, part_x, ksplit_x, nullptr, sgn, col0, nullptr, tol, mode,
                                        o.inner_max_passes, d_tab_full, d_tab_cross, Wp, rotated, rot_ctr, cnt, st,
                                        1, dexp, vs, vs ? trace : nullptr, o.tstop, tbig)
                         : launch_solve(b, np, part, ns, nullptr, sgn, col0, nullptr, tol, mode,
                                        o.inner_max_passes, d_tab_full, d_tab_cross, Wp, rotated, rot_ctr, cnt, st,
                                        0, nullptr, vs, vs ? trace : nullptr, o.tstop, tbig);
            if (e == cudaSuccess) e = evs.record(4 * s + 2, st);
            if (e == cudaSuccess && prec) e = launch_wprep_x(np, Wp, dexp, rotated, wsl, wexp, upd_ctr, st);
            if (e == cudaSuccess)
                e = prec ? launch_update_x(Gw, m_pad, m_pad, Ww, ldw, ldw, np, col0, wsl, wexp, dexp, rotated, cnt,
                                           st)
                         : launch_update(Gw, m_pad, m_pad, Ww, ldw, ldw, b, np, col0, Wp, rotated, upd_ctr, st);
            if (e == cudaSuccess) e = evs.record(4 * s + 3, st);
            nl += prec ? 4 : 3;
        }
        if (e == cudaSuccess) e = evs.record(evr, st);
        if (e == cudaSuccess)
            e = launch_reorder(Gw, Gt, m_pad, Ww, Wt, ldw, n_pad, perm, perm_t, sgn, sgn_t, d, newpos, o.sort, st);
        if (e == cudaSuccess) e = evs.record(evr + 1, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
        const cudaError_t e2 = cudaStreamEndCapture(st, graph);
        *launches = nl + reorder_kernels;
        return e != cudaSuccess ? e : e2;
    };

    // One sweep as a dependency graph of visits (the pair schedule): a group of
    // up to `grp` consecutive visits of step s runs Gram, inner solve and update
    // on the stream of its first slot (s mod kRing, k), after the updates that
    // last wrote its block columns.  Those are its only inputs; the slot's
    // stream orders the reuse of the slot's buffers kRing steps later.  The
    // group size keeps the graph near kMaxNodes kernel nodes per sweep: the
    // GPU dispatches graph nodes at a bounded rate (about 2 us per node
    // measured), which would otherwise bound the sweep.  From n = 4096 a
    // visit's kernels take hundreds of microseconds and twice the nodes
    // (smaller groups, more overlap) measured faster (Haar 4096, split
    // precision: 1263 against 1275 ms; 11 visits per group: 1344 ms).
    const int kpv = prec ? 4 : 3;  // kernels per visit
    const int64_t max_nodes = n_pad >= 4096 ? 2 * kMaxNodes : kMaxNodes;
    const int grp = (int)std::min<int64_t>(npairs, std::max<int64_t>(1, ((int64_t)nb * npairs * kpv + max_nodes - 1) /
                                                                          max_nodes));
    auto capture_pairs = [&](const int *tab, const int *vis, const std::vector<int> &nact,
                             const std::vector<int> &off, const int *tab_host, cudaGraph_t *graph,
                             long long *launches) -> cudaError_t {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        long long nl = 0;
        e = cudaMemsetAsync(cnt + 2, 0, 5 * sizeof(int), st);
        if (e == cudaSuccess) e = cudaEventRecord(dag.fork, st);
        for (size_t i = 0; i < dag.streams.size() && e == cudaSuccess; ++i)
            e = cudaStreamWaitEvent(dag.streams[i], dag.fork, 0);
        std::vector<char> written((size_t)nb, 0);
        for (int s = 0; s < nb && e == cudaSuccess; ++s) {
            const int mode = (o.inner_mode == HSVD_INNER_FULL) ? 0 : (s == 0 ? 2 : 1);
            for (int k = 0; k < nact[(size_t)s] && e == cudaSuccess; k += grp) {
                const int np = std::min(grp, nact[(size_t)s] - k);
                const int v = off[(size_t)s] + k;
                const int slot = (s % kRing) * npairs + k;
                cudaStream_t ss = dag.streams[(size_t)slot];
                for (int i = 0; i < 2 * np && e == cudaSuccess; ++i) {
                    const int c = tab_host[2 * v + i] / b;
                    if (written[(size_t)c]) e = cudaStreamWaitEvent(ss, dag.col[(size_t)c], 0);
                }
                const int *c0 = tab + 2 * v;
                const int *vs = vis ? vis + v : nullptr;
                double *wp = Wp + (size_t)slot * nn * nn;
                int *rot = rotated + slot;
                if (prec) {
                    double *px = part_x + (size_t)slot * ksplit_x * nn * nn;
                    int *dx = dexp + (size_t)slot * nn;
                    uint16_t *wl = wsl + precision_wsl_elems(1) * slot;
                    int *we = wexp + (size_t)slot * 2 * nn;
                    if (e == cudaSuccess) e = launch_gram_x(Gw, m_pad, m_pad, np, c0, px, cnt, ss);
                    if (e == cudaSuccess)
                        e = launch_solve(b, np, px, ksplit_x, nullptr, sgn, c0, nullptr, tol, mode,
                                         o.inner_max_passes, d_tab_full, d_tab_cross, wp, rot, rot_ctr, cnt, ss, 1, dx,
                                         vs, vs ? trace : nullptr, o.tstop, tbig);
                    if (e == cudaSuccess) e = launch_wprep_x(np, wp, dx, rot, wl, we, upd_ctr, ss);
                    if (e == cudaSuccess)
                        e = launch_update_x(Gw, m_pad, m_pad, Ww, ldw, ldw, np, c0, wl, we, dx, rot, cnt, ss);
                    nl += 4;
                } else {
                    double *pt = part + (size_t)slot * nsplit * 3 * b * b;
                    if (e == cudaSuccess) e = launch_gram(Gw, m_pad, m_pad, b, np, c0, nsplit, pt, ss);
                    if (e == cudaSuccess)
                        e = launch_solve(b, np, pt, nsplit, nullptr, sgn, c0, nullptr, tol, mode,
                                         o.inner_max_passes, d_tab_full, d_tab_cross, wp, rot, rot_ctr, cnt, ss, 0,
                                         nullptr, vs, vs ? trace : nullptr, o.tstop, tbig);
                    if (e == cudaSuccess)
                        e = launch_update(Gw, m_pad, m_pad, Ww, ldw, ldw, b, np, c0, wp, rot, upd_ctr, ss);
                    nl += 3;
                }
                for (int i = 0; i < 2 * np && e == cudaSuccess; ++i) {
                    const int c = tab_host[2 * v + i] / b;
                    e = cudaEventRecord(dag.col[(size_t)c], ss);
                    written[(size_t)c] = 1;
                }
            }
        }
        for (size_t i = 0; i < dag.streams.size() && e == cudaSuccess; ++i) {
            e = cudaEventRecord(dag.join[i], dag.streams[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, dag.join[i], 0);
        }
        if (e == cudaSuccess) e = evs.record(evr, st);
        if (e == cudaSuccess)
            e = launch_reorder(Gw, Gt, m_pad, Ww, Wt, ldw, n_pad, perm, perm_t, sgn, sgn_t, d, newpos, o.sort, st);
        if (e == cudaSuccess) e = evs.record(evr + 1, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
        const cudaError_t e2 = cudaStreamEndCapture(st, graph);
        *launches = nl + reorder_kernels;
        return e != cudaSuccess ? e : e2;
    };

    std::vector<int> full_n((size_t)nb, npairs), full_off((size_t)nb);
    for (int s = 0; s < nb; ++s) full_off[(size_t)s] = s * npairs;
    long long full_launches = 0;
    // host time of graph capture and instantiation (reported in the info record)
    using Clock = std::chrono::steady_clock;
    auto ms_since = [](Clock::time_point t0) {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    };
    const Clock::time_point tg0 = Clock::now();
    if (pair_sched) {
        if (!dag.create(nslot, nb)) return HSVD_ERR_CUDA;
        if (capture_pairs(d_tab_outer, d_visit, full_n, full_off, outer.data(), &gg.graph, &full_launches) !=
            cudaSuccess)
            return HSVD_ERR_CUDA;
    } else if (capture(d_tab_outer, d_visit, full_n, full_off, &gg.graph, &full_launches) != cudaSuccess) {
        return HSVD_ERR_CUDA;
    }
    CKR(cudaGraphInstantiate(&gg.exec, gg.graph, 0));
    stats.ms_host_graph += ms_since(tg0);
    // profiling spans every step, skipped ones included (they record nothing)
    auto add_profile = [&](const std::vector<int> &nact, bool steps) {
        if (!o.profile) return;
        if (!steps) {  // visits overlap: only the sweep's total
            stats.ms_other += evs.between(evr + 2, evr + 3);
            return;
        }
        for (int s = 0; s < nb; ++s) {
            if (nact[(size_t)s] == 0) continue;
            stats.ms_gram += evs.between(4 * s, 4 * s + 1);
            stats.ms_solve += evs.between(4 * s + 1, 4 * s + 2);
            stats.ms_update += evs.between(4 * s + 2, 4 * s + 3);
        }
        stats.ms_other += evs.between(evr, evr + 1);
    };

    // masked sweeps under the pair schedule (FP64 products) keep the mask on the
    // device and reuse one graph; otherwise the host compacts the visit table
    const bool mask_on_device = learned && pair_sched && !prec;
    GraphGuard gm;
    long long mask_launches = 0;
    int status = HSVD_NOT_CONVERGED, sweep;
    bool judge_next = false;  // the next sweep must be a full one
    for (sweep = 1; sweep <= o.max_sweeps; ++sweep) {
        Range sweep_range("hsvd sweep");
        const bool masked = learned && sweep >= 2 && !judge_next;
        if ((masked || export_rows) && sweep >= 2) {
            CKR(launch_features(trace, masked ? prev_skip : nullptr, d_tab_outer, nvis, b, nb, sweep, o.max_sweeps,
                                tol, X, st));
            stats.launches += 1;
        }
        unsigned long long rots, upds;
        if (masked && mask_on_device) {
            // the mask stays on the device: one graph over every visit, skipped
            // visits reduced to empty kernels by the (-1, -1) table entries
            CKR(launch_mlp_infer(params, X, nvis, nullptr, skip, logit_tau, st));
            CKR(cudaMemsetAsync(cnt + 7, 0, sizeof(int), st));
            CKR(launch_mask_table(d_tab_outer, skip, nvis, d_tab_mask, cnt + 7, st));
            CKR(cudaMemcpyAsync(prev_skip, skip, nvis, cudaMemcpyDeviceToDevice, st));
            stats.launches += 2;
            if (!gm.exec) {
                const Clock::time_point t0 = Clock::now();
                if (capture_pairs(d_tab_mask, d_visit, full_n, full_off, outer.data(), &gm.graph, &mask_launches) !=
                    cudaSuccess)
                    return HSVD_ERR_CUDA;
                CKR(cudaGraphInstantiate(&gm.exec, gm.graph, 0));
                stats.ms_host_graph += ms_since(t0);
            }
            CKR(evs.record_now(evr + 2, st));
            CKR(cudaGraphLaunch(gm.exec, st));
            CKR(evs.record_now(evr + 3, st));
            CKR(cudaStreamSynchronize(st));
            stats.launches += mask_launches;
            stats.pair_visits += h_cnt[7];
            stats.masked_sweeps += 1;
            add_profile(full_n, false);
        } else if (masked) {
            CKR(launch_mlp_infer(params, X, nvis, nullptr, skip, logit_tau, st));
            CKR(cudaMemcpyAsync(h_skip, skip, nvis, cudaMemcpyDeviceToHost, st));
            CKR(cudaMemcpyAsync(prev_skip, skip, nvis, cudaMemcpyDeviceToDevice, st));
            CKR(cudaStreamSynchronize(st));
            stats.launches += 1;
            std::vector<int> nact((size_t)nb, 0), off((size_t)nb, 0);
            int cur = 0;
            for (int s = 0; s < nb; ++s) {
                off[(size_t)s] = cur;
                for (int k = 0; k < npairs; ++k) {
                    const int v = s * npairs + k;
                    if (h_skip[v]) continue;
                    h_tab[2 * cur] = outer_host[2 * (size_t)v];
                    h_tab[2 * cur + 1] = outer_host[2 * (size_t)v + 1];
                    h_vis[cur] = v;
                    ++cur;
                }
                nact[(size_t)s] = cur - off[(size_t)s];
            }
            stats.pair_visits += cur;
            stats.masked_sweeps += 1;
            CKR(cudaMemcpyAsync(d_tab_mask, h_tab, sizeof(int) * 2 * (size_t)std::max(cur, 1), cudaMemcpyHostToDevice,
                                st));
            CKR(cudaMemcpyAsync(d_visit_mask, h_vis, sizeof(int) * (size_t)std::max(cur, 1), cudaMemcpyHostToDevice,
                                st));
            GraphGuard mg;
            long long ml = 0;
            const Clock::time_point t0 = Clock::now();
            if (capture(d_tab_mask, d_visit_mask, nact, off, &mg.graph, &ml) != cudaSuccess) return HSVD_ERR_CUDA;
            CKR(cudaGraphInstantiate(&mg.exec, mg.graph, 0));
            stats.ms_host_graph += ms_since(t0);
            CKR(cudaGraphLaunch(mg.exec, st));
            CKR(cudaStreamSynchronize(st));
            stats.launches += ml;
            add_profile(nact, true);
        } else {
            if (learned && judge_next) stats.judge_sweeps += 1;
            CKR(evs.record_now(evr + 2, st));
            CKR(cudaGraphLaunch(gg.exec, st));
            CKR(evs.record_now(evr + 3, st));
            CKR(cudaStreamSynchronize(st));
            stats.launches += full_launches;
            stats.pair_visits += nvis;
            add_profile(full_n, !pair_sched);
            if (learned) CKR(cudaMemsetAsync(prev_skip, 0, nvis, st));
        }
        memcpy(&rots, h_cnt + 2, sizeof rots);
        memcpy(&upds, h_cnt + 4, sizeof upds);
        stats.rotations += (long long)rots;
        stats.pair_updates += (long long)upds;
        stats.sweeps = sweep;
        if (h_cnt[0] != 0) { status = h_cnt[0]; break; }
        if (export_rows && sweep >= 2 && stats.trace_rows + nvis <= o.trace_cap) {
            CKR(launch_export(X, trace, nvis, o.trace_out + (size_t)stats.trace_rows * (HSVD_MLP_FEATURES + 1), st));
            stats.trace_rows += nvis;
            stats.launches += 1;
        }
        // Eq. 4.2 reduced over the sweep: (00)_2 no rotation, (01)_2 every
        // tangent <= tstop, (11)_2 otherwise
        const bool small_tangents = tangent_stop && h_cnt[6] == 0;
        if (rots == 0 || small_tangents) {
            if (masked) {
                judge_next = true;  // a masked sweep never ends the iteration
                continue;
            }
            status = HSVD_OK;
            stats.stop_rule = rots == 0 ? HSVD_STOP_ORTHO : HSVD_STOP_TANGENT;
            break;
        }
        judge_next = false;
    }
    if (sweep > o.max_sweeps) sweep = o.max_sweeps;
    if (status == HSVD_OK || status == HSVD_NOT_CONVERGED) {
        CKR(cudaMemsetAsync(cnt, 0, sizeof(int), st));
        CKR(launch_finalize(Gw, m_pad, Ww, ldw, perm, n_pad, m, n, sigma, U, ldu, V, ldv, cnt, st));
        stats.launches += 1;
        CKR(cudaMemcpyAsync(h_cnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        if (h_cnt[0] != 0) status = h_cnt[0];
    }
    return status;
}

int solve_blocked(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma, double *U,
                  int64_t ldu, double *V, int64_t ldv, const hsvd_opts &o, double tol, int b, hsvd_info *info,
                  cudaStream_t st) {
    SweepStats stats;
    const int rc = solve_blocked_core(G, m, n, ldg, J, sigma, U, ldu, V, ldv, o, tol, b, stats, st);
    if (info) {
        info->sweeps = stats.sweeps;
        info->method = HSVD_METHOD_BLOCKED;
        info->block_w = b;
        info->rotations = stats.rotations;
        info->pair_updates = stats.pair_updates;
        info->kernel_launches = stats.launches;
        info->ms_gram = stats.ms_gram;
        info->ms_solve = stats.ms_solve;
        info->ms_update = stats.ms_update;
        info->ms_other = stats.ms_other;
        info->ms_host_graph = stats.ms_host_graph;
        info->pair_visits = stats.pair_visits;
        info->masked_sweeps = stats.masked_sweeps;
        info->judge_sweeps = stats.judge_sweeps;
        info->trace_rows = stats.trace_rows;
        info->stop_rule = rc == HSVD_OK ? stats.stop_rule : HSVD_STOP_NONE;
    }
    return rc;
}

int solve_pointwise(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma, double *U,
                    int64_t ldu, double *V, int64_t ldv, const hsvd_opts &o, double tol, hsvd_info *info,
                    cudaStream_t st) {
    const int64_t n_pad = n + (n & 1);
    Ws ws(st);
    double *W = ws.get<double>(n_pad * n_pad);
    int *out = ws.get<int>(4);
    long long *rot = ws.get<long long>(1);
    int h_out[4] = {0, 0, 0, 0};
    long long h_rot = 0;
    if (!W || !out || !rot) return HSVD_ERR_NOMEM;
    SweepEvents evs;
    if (o.profile && !evs.create(2)) return HSVD_ERR_CUDA;
    CKR(evs.record(0, st));
    CKR(launch_pointwise(G, ldg, (int)m, (int)n, J, tol, o.tstop, o.max_sweeps, o.sort, W, sigma, U, ldu, V, ldv, out,
                         rot, st));
    CKR(evs.record(1, st));
    CKR(cudaMemcpyAsync(h_out, out, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaMemcpyAsync(&h_rot, rot, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (info) {
        info->sweeps = h_out[1];
        info->method = HSVD_METHOD_POINTWISE;
        info->block_w = 1;
        info->rotations = h_rot;
        info->pair_updates = 0;
        info->kernel_launches = 1;
        info->stop_rule = h_out[2];
        if (o.profile) info->ms_solve = evs.between(0, 1);
    }
    return h_out[0];
}

// Shortening (Sec. 1): G = Q R, the HSVD of R (n x n) by the chosen method,
// U = Q [U_R; 0].  V and sigma are R's.
int solve_shortened(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma, double *U,
                    int64_t ldu, double *V, int64_t ldv, const hsvd_opts &o, double tol, int method, int b,
                    hsvd_info *info, cudaStream_t st) {
    Range range("hsvd shortened solve");
    Ws ws(st);
    double *A = ws.get<double>((size_t)m * n);  // QR in place on a copy: G is read-only
    double *R = ws.get<double>((size_t)n * n);
    double *UR = U ? ws.get<double>((size_t)n * n) : nullptr;
    double *qws = ws.get<double>(qr_workspace_doubles(n));
    if (!A || !R || (U && !UR) || !qws) return HSVD_ERR_NOMEM;
    long long nl = 0;
    CKR(cudaMemcpy2DAsync(A, sizeof(double) * m, G, sizeof(double) * ldg, sizeof(double) * m, n,
                          cudaMemcpyDeviceToDevice, st));
    CKR(qr_factor(A, m, m, n, qws, st, &nl));
    CKR(qr_extract_r(A, m, n, R, n, st));
    nl += 1;
    const int rc = method == HSVD_METHOD_POINTWISE
                       ? solve_pointwise(R, n, n, n, J, sigma, UR, n, V, ldv, o, tol, info, st)
                       : solve_blocked(R, n, n, n, J, sigma, UR, n, V, ldv, o, tol, b, info, st);
    if ((rc == HSVD_OK || rc == HSVD_NOT_CONVERGED) && U) {
        CKR(qr_embed_u(UR, n, m, n, U, ldu, st));
        CKR(qr_apply_q(A, m, m, n, qws, U, ldu, st, &nl));
        nl += 1;
    }
    CKR(cudaStreamSynchronize(st));
    if (info) {
        info->shortened = 1;
        info->kernel_launches += nl;
    }
    return rc;
}

// A wide factor (m < n, Sec. 1): the hyperbolic QR of G^T (hypqr.cu) gives the
// square F = C R^T with signature Jh_1, whose HSVD F V_F = U Sigma gives
// V = T^T [V_F; 0]: G V = U Sigma and V^T J V = Jh_1.
int solve_wide(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma, double *U,
               int64_t ldu, double *V, int64_t ldv, const hsvd_opts *opts_in, hsvd_info *info, void *stream) {
    Range range("hsvd wide solve");
    hsvd_opts o;
    if (opts_in) o = *opts_in;
    else hsvd_default_opts(&o);
    auto fail = [&](int rc) {
        if (info) info->status = rc;
        return rc;
    };
    if (!G || !J || !sigma || m < 1 || n <= m || ldg < m || n > ((int64_t)1 << 24)) return fail(HSVD_ERR_ARG);
    if ((U && ldu < m) || (V && ldv < n)) return fail(HSVD_ERR_ARG);
    const bool dev = is_device_ptr(G);
    const void *arrs[5] = {J, sigma, U, V, o.jout};
    for (int i = 0; i < 5; ++i)
        if (arrs[i] && is_device_ptr(arrs[i]) != dev) return fail(HSVD_ERR_ARG);
    cudaStream_t user = static_cast<cudaStream_t>(stream), st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(HSVD_ERR_CUDA);
    int rc = HSVD_OK;
    long long nl = 0;
    {
        Ws ws(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev, user) != cudaSuccess || cudaStreamWaitEvent(st, ev, 0) != cudaSuccess)
            rc = HSVD_ERR_CUDA;
        HypQr hq = {};
        hq.A = ws.get<double>((size_t)n * m);
        hq.C = ws.get<double>((size_t)m * m);
        hq.Vr = ws.get<double>((size_t)n * m);
        hq.z = ws.get<double>((size_t)n);
        hq.beta = ws.get<double>((size_t)m);
        hq.cperm = ws.get<int>((size_t)m);
        hq.rswap = ws.get<int>((size_t)m);
        hq.drows = ws.get<int>(4);
        hq.s = ws.get<int8_t>((size_t)n);
        hq.bsize = ws.get<int8_t>((size_t)m);
        hq.state = ws.get<unsigned char>(hypqr_state_bytes());
        hq.mx = ws.get<unsigned char>(hypqr_mx_bytes(m));
        double *F = ws.get<double>((size_t)m * m);
        int8_t *Jh1 = ws.get<int8_t>((size_t)m);
        double *VF = V ? ws.get<double>((size_t)m * m) : nullptr;
        const double *g = G;
        const int8_t *j = J;
        double *s = sigma, *u = U, *v = V;
        int64_t lg = ldg, lu = ldu, lv = ldv;
        if (!dev) {  // host arrays: staged through device memory
            double *dG = ws.get<double>((size_t)m * n);
            int8_t *dJ = ws.get<int8_t>((size_t)n);
            s = ws.get<double>((size_t)m);
            u = U ? ws.get<double>((size_t)m * m) : nullptr;
            v = V ? ws.get<double>((size_t)n * m) : nullptr;
            lg = m;
            lu = m;
            lv = n;
            if (!dG || !dJ || !s || (U && !u) || (V && !v)) rc = HSVD_ERR_NOMEM;
            else if (cudaMemcpy2DAsync(dG, sizeof(double) * m, G, sizeof(double) * ldg, sizeof(double) * m, n,
                                       cudaMemcpyHostToDevice, st) != cudaSuccess ||
                     cudaMemcpyAsync(dJ, J, (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = HSVD_ERR_CUDA;
            g = dG;
            j = dJ;
        }
        if (rc == HSVD_OK && (!hq.A || !hq.C || !hq.Vr || !hq.z || !hq.beta || !hq.cperm || !hq.rswap ||
                              !hq.drows || !hq.s || !hq.bsize || !hq.state || !hq.mx || !F || !Jh1 || (V && !VF)))
            rc = HSVD_ERR_NOMEM;
        if (rc == HSVD_OK) rc = hypqr_factor(g, m, n, lg, j, hq, F, st, &nl);
        if (rc == HSVD_OK) {
            if (cudaMemcpyAsync(Jh1, hq.s, (size_t)m, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = HSVD_ERR_CUDA;
        }
        if (rc == HSVD_OK) {
            // the square F with the signature Jh_1, on the internal stream
            hsvd_opts o2 = o;
            o2.jout = nullptr;
            rc = hsvd_solve_ex(F, m, m, m, Jh1, s, u, lu, VF, m, &o2, info, st);
        }
        if ((rc == HSVD_OK || rc == HSVD_NOT_CONVERGED) && V &&
            hypqr_apply_tt(hq, m, n, VF, v, lv, st, &nl) != HSVD_OK)
            rc = HSVD_ERR_CUDA;
        if ((rc == HSVD_OK || rc == HSVD_NOT_CONVERGED) && o.jout &&
            cudaMemcpyAsync(o.jout, Jh1, (size_t)m, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
            rc = HSVD_ERR_CUDA;
        if (!dev && (rc == HSVD_OK || rc == HSVD_NOT_CONVERGED)) {
            if (cudaMemcpyAsync(sigma, s, sizeof(double) * m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                (U && cudaMemcpy2DAsync(U, sizeof(double) * ldu, u, sizeof(double) * m, sizeof(double) * m, m,
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
                (V && cudaMemcpy2DAsync(V, sizeof(double) * ldv, v, sizeof(double) * n, sizeof(double) * n, m,
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess))
                rc = HSVD_ERR_CUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess && rc >= 0) rc = HSVD_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc >= 0) rc = HSVD_ERR_CUDA;
    if (ev) cudaEventDestroy(ev);
    cudaStreamDestroy(st);
    if (info) {
        info->kernel_launches += nl;
        info->shortened = 2;
        info->status = rc;
    }
    return rc;
}

int validate(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, const double *sigma, int64_t ldu,
             const double *U, int64_t ldv, const double *V) {
    if (!G || !J || !sigma) return HSVD_ERR_ARG;
    if (n < 1 || m < n || ldg < m) return HSVD_ERR_ARG;
    if (n > (int64_t)1 << 24 || m > (int64_t)1 << 31) return HSVD_ERR_ARG;
    if (U && ldu < m) return HSVD_ERR_ARG;
    if (V && ldv < n) return HSVD_ERR_ARG;
    return HSVD_OK;
}

}  // namespace

extern "C" {

void hsvd_default_opts(hsvd_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->tol = 0.0;
    o->max_sweeps = 30;
    o->method = HSVD_METHOD_AUTO;
    o->block_w = 0;
    o->inner_mode = HSVD_INNER_ORIENTED;
    o->inner_max_passes = 8;
    o->sort = HSVD_SORT_AUTO;
}

const char *hsvd_status_string(int s) {
    switch (s) {
        case HSVD_OK: return "HSVD_OK";
        case HSVD_NOT_CONVERGED: return "HSVD_NOT_CONVERGED";
        case HSVD_ERR_ARG: return "HSVD_ERR_ARG";
        case HSVD_ERR_RANK: return "HSVD_ERR_RANK";
        case HSVD_ERR_NONFINITE: return "HSVD_ERR_NONFINITE";
        case HSVD_ERR_CUDA: return "HSVD_ERR_CUDA";
        case HSVD_ERR_NOMEM: return "HSVD_ERR_NOMEM";
        default: return "HSVD_UNKNOWN_STATUS";
    }
}

int hsvd_modulus_pairs(int r, int nsteps, int *pairs) {
    if (r < 2 || (r & 1) || r > 65536 || nsteps < 0 || (!pairs && nsteps > 0)) return HSVD_ERR_ARG;
    fill_modulus(r, nsteps, pairs);
    return HSVD_OK;
}

int hsvd_ring_table(int b, int *tab) {
    if ((b != 16 && b != 32 && b != 64) || !tab) return HSVD_ERR_ARG;
    return fill_ring(b, tab) ? HSVD_OK : HSVD_ERR_ARG;
}

int hsvd_solve_ex(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double *sigma, double *U,
                  int64_t ldu, double *V, int64_t ldv, const hsvd_opts *opts_in, hsvd_info *info, void *stream) {
    Range range("hsvd_solve_ex");
    hsvd_opts o;
    if (opts_in) o = *opts_in;
    else hsvd_default_opts(&o);
    if (info) memset(info, 0, sizeof *info);
    if (G && m >= 1 && n > m) return solve_wide(G, m, n, ldg, J, sigma, U, ldu, V, ldv, opts_in, info, stream);
    int rc = validate(G, m, n, ldg, J, sigma, ldu, U, ldv, V);
    if (rc == HSVD_OK) {
        for (int i = 0; i < 2; ++i)
            if (o.reserved[i]) rc = HSVD_ERR_ARG;
        if (o.schedule < HSVD_SCHEDULE_AUTO || o.schedule > HSVD_SCHEDULE_PAIRS) rc = HSVD_ERR_ARG;
        if (o.shorten < HSVD_SHORTEN_AUTO || o.shorten > HSVD_SHORTEN_ALWAYS) rc = HSVD_ERR_ARG;
        if (o.tstop < 0.0) o.tstop = HSVD_TSTOP_PAPER;
        if (!(o.tstop >= 0.0 && o.tstop <= 1.0)) rc = HSVD_ERR_ARG;
        if (o.max_sweeps <= 0) o.max_sweeps = 30;
        if (o.inner_max_passes <= 0) o.inner_max_passes = 8;
        if (o.method < HSVD_METHOD_AUTO || o.method > HSVD_METHOD_BLOCKED) rc = HSVD_ERR_ARG;
        if (o.block_w != 0 && o.block_w != 16 && o.block_w != 32 && o.block_w != 64) rc = HSVD_ERR_ARG;
        if (o.inner_mode != HSVD_INNER_ORIENTED && o.inner_mode != HSVD_INNER_FULL) rc = HSVD_ERR_ARG;
        if (o.sort != 0 && o.sort != 1 && o.sort != HSVD_SORT_AUTO) rc = HSVD_ERR_ARG;
        if (o.precision != HSVD_PRECISION_FP64 && o.precision != HSVD_PRECISION_BF16X8) rc = HSVD_ERR_ARG;
        if (o.precision == HSVD_PRECISION_BF16X8 &&
            (o.method == HSVD_METHOD_POINTWISE || (o.block_w != 0 && o.block_w != 64)))
            rc = HSVD_ERR_ARG;
        if (!(o.tol == o.tol)) rc = HSVD_ERR_ARG;
    }
    if (rc != HSVD_OK) {
        if (info) info->status = rc;
        return rc;
    }
    const double tol = (o.tol > 0.0) ? o.tol : (double)n * 0x1p-53;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    const bool dev = is_device_ptr(G);
    // all arrays of one call are of one kind
    const void *arrs[5] = {J, sigma, U, V, nullptr};
    for (int i = 0; i < 4; ++i)
        if (arrs[i] && is_device_ptr(arrs[i]) != dev) {
            if (info) info->status = HSVD_ERR_ARG;
            return HSVD_ERR_ARG;
        }
    // a tall factor is shortened first; the method is then chosen for the square R
    const bool shorten =
        m > n && (o.shorten == HSVD_SHORTEN_ALWAYS || (o.shorten == HSVD_SHORTEN_AUTO && 4 * m >= 5 * n));
    const int64_t m_eff = shorten ? n : m;
    // the one-CTA pointwise solve is the faster method only for narrow factors
    // (measured, N(0,1) square factors: n = 16: 1.07 ms against 2.39 ms blocked
    // with b = 16; n = 32: 3.27 against 2.91 ms; n = 128: 53.8 against 8.5 ms)
    int method = o.method;
    if (method == HSVD_METHOD_AUTO)
        method = (n < 32 && pointwise_fits(m_eff, n) && o.precision == HSVD_PRECISION_FP64) ? HSVD_METHOD_POINTWISE
                                                                                             : HSVD_METHOD_BLOCKED;
    // diagonal sorting pays for the pointwise method (Sec. 5, Table 5.3) and for
    // the split-precision form (measured: Haar 4096, 2269 -> 2085 ms; Haar 1024,
    // 211 -> 197 ms), but costs sweeps in the FP64 blocked one (graded 1024:
    // 14 sweeps sorted, 11 unsorted); the learned form needs unsorted sweeps
    if (o.sort == HSVD_SORT_AUTO)
        o.sort = (method == HSVD_METHOD_POINTWISE ||
                  (o.precision == HSVD_PRECISION_BF16X8 && !o.skip_model && !o.trace_out))
                     ? 1
                     : 0;
    // the learned form and the trace export follow block-pair visits across
    // sweeps: blocked method without column reordering
    if ((o.skip_model || o.trace_out) && (method != HSVD_METHOD_BLOCKED || o.sort != 0 ||
                                          (o.trace_out && o.trace_cap < 1) || !(o.skip_tau < 1.0))) {
        if (info) info->status = HSVD_ERR_ARG;
        return HSVD_ERR_ARG;
    }
    if (method == HSVD_METHOD_POINTWISE && !pointwise_fits(m_eff, n)) {
        if (info) info->status = HSVD_ERR_ARG;
        return HSVD_ERR_ARG;
    }
    const int b = o.block_w ? o.block_w : (o.precision == HSVD_PRECISION_BF16X8 ? 64 : choose_block(n));
    double *dG = nullptr, *dS = nullptr, *dU = nullptr, *dV = nullptr;
    int8_t *dJ = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        if (info) info->status = HSVD_ERR_CUDA;
        return HSVD_ERR_CUDA;
    }
    // order after the work already queued on the caller's stream
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, user) != cudaSuccess || cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
        rc = HSVD_ERR_CUDA;
        goto done;
    }
    if (!dev) {
        // host arrays: stage through device memory on the internal stream
        if (cudaMallocAsync((void **)&dG, sizeof(double) * m * n, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dJ, n, st) != cudaSuccess ||
            cudaMallocAsync((void **)&dS, sizeof(double) * n, st) != cudaSuccess ||
            (U && cudaMallocAsync((void **)&dU, sizeof(double) * m * n, st) != cudaSuccess) ||
            (V && cudaMallocAsync((void **)&dV, sizeof(double) * n * n, st) != cudaSuccess)) {
            rc = HSVD_ERR_NOMEM;
            goto done;
        }
        if (cudaMemcpy2DAsync(dG, sizeof(double) * m, G, sizeof(double) * ldg, sizeof(double) * m, n,
                              cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(dJ, J, n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = HSVD_ERR_CUDA;
            goto done;
        }
    }
    {
        const double *g = dev ? G : dG;
        const int8_t *j = dev ? J : dJ;
        double *s = dev ? sigma : dS;
        double *u = dev ? U : dU;
        double *v = dev ? V : dV;
        const int64_t lg = dev ? ldg : m, lu = dev ? ldu : m, lv = dev ? ldv : n;
        if (shorten)
            rc = solve_shortened(g, m, n, lg, j, s, u, lu, v, lv, o, tol, method, b, info, st);
        else if (method == HSVD_METHOD_POINTWISE)
            rc = solve_pointwise(g, m, n, lg, j, s, u, lu, v, lv, o, tol, info, st);
        else
            rc = solve_blocked(g, m, n, lg, j, s, u, lu, v, lv, o, tol, b, info, st);
    }
    if (!dev && (rc == HSVD_OK || rc == HSVD_NOT_CONVERGED)) {
        if (cudaMemcpyAsync(sigma, dS, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (U && cudaMemcpy2DAsync(U, sizeof(double) * ldu, dU, sizeof(double) * m, sizeof(double) * m, n,
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            (V && cudaMemcpy2DAsync(V, sizeof(double) * ldv, dV, sizeof(double) * n, sizeof(double) * n, n,
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess))
            rc = HSVD_ERR_CUDA;
    }
done:
    if (dG) cudaFreeAsync(dG, st);
    if (dJ) cudaFreeAsync(dJ, st);
    if (dS) cudaFreeAsync(dS, st);
    if (dU) cudaFreeAsync(dU, st);
    if (dV) cudaFreeAsync(dV, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc >= 0) rc = HSVD_ERR_CUDA;
    if (ev) cudaEventDestroy(ev);
    cudaStreamDestroy(st);
    if (info) info->status = rc;
    return rc;
}

int hsvd_solve(const double *G, int64_t m, int64_t n, int64_t ldg, const int8_t *J, double tol, int max_sweeps,
               double *sigma, double *U, int64_t ldu, double *V, int64_t ldv, int *sweeps, void *stream) {
    hsvd_opts o;
    hsvd_default_opts(&o);
    o.tol = tol;
    o.max_sweeps = max_sweeps;
    hsvd_info info;
    const int rc = hsvd_solve_ex(G, m, n, ldg, J, sigma, U, ldu, V, ldv, &o, &info, stream);
    if (sweeps) *sweeps = info.sweeps;
    return rc;
}

int hsvd_diag_wait_timeout(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *d = nullptr, h = -1;
    if (cudaMallocAsync((void **)&d, sizeof(int), st) != cudaSuccess) return HSVD_ERR_NOMEM;
    int rc = HSVD_OK;
    if (launch_diag_wait(4096, d, st) != cudaSuccess ||
        cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        rc = HSVD_ERR_CUDA;
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
    if (rc == HSVD_OK && h != 1) rc = HSVD_ERR_CUDA;  // the wait must have given up
    return rc;
}

int hsvd_sym_factor(const double *M, int64_t n, int64_t ldm, double *G, int64_t ldg, int8_t *J, int64_t *rank,
                    void *stream) {
    Range range("hsvd_sym_factor");
    if (!M || !G || !J || n < 1 || n > ((int64_t)1 << 20) || ldm < n || ldg < n) return HSVD_ERR_ARG;
    if (!is_device_ptr(M) || !is_device_ptr(G) || !is_device_ptr(J)) return HSVD_ERR_ARG;
    return ldl_factor(M, n, ldm, G, ldg, J, static_cast<cudaStream_t>(stream), nullptr, rank);
}

namespace {
__global__ void k_sym_lambda(const double *__restrict__ sigma, const int8_t *__restrict__ J, int64_t n,
                             double *__restrict__ lambda) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) lambda[j] = sigma[j] * sigma[j] * (double)J[j];
}
// X (n x (n - r), ldx) <- [0; I_(n-r)]
__global__ void k_sym_null_init(double *__restrict__ X, int64_t ldx, int64_t n, int64_t r) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * (n - r)) return;
    const int64_t i = e % n, c = e / n;
    X[i + c * ldx] = (i == r + c) ? 1.0 : 0.0;
}
}  // namespace

int hsvd_sym_eig(const double *M, int64_t n, int64_t ldm, double *lambda, double *U, int64_t ldu,
                 const hsvd_opts *opts, hsvd_info *info, void *stream) {
    if (info) memset(info, 0, sizeof *info);
    if (!M || !lambda || n < 1 || n > ((int64_t)1 << 20) || ldm < n || (U && ldu < n)) return HSVD_ERR_ARG;
    if (!is_device_ptr(M) || !is_device_ptr(lambda) || (U && !is_device_ptr(U))) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = HSVD_OK;
    long long nl = 0;
    int64_t r = 0;
    {
        Ws ws(st);
        double *G = ws.get<double>((size_t)n * n), *sigma = ws.get<double>((size_t)n);
        int8_t *J = ws.get<int8_t>((size_t)n);
        if (!G || !sigma || !J) rc = HSVD_ERR_NOMEM;
        if (rc == HSVD_OK) rc = ldl_factor(M, n, ldm, G, n, J, st, &nl, &r);
        // eigenvalues past the rank of a singular M are zero; the HSVD of the
        // n x r factor gives the others
        if (rc == HSVD_OK && cudaMemsetAsync(lambda, 0, sizeof(double) * n, st) != cudaSuccess) rc = HSVD_ERR_CUDA;
        if (rc == HSVD_OK && r > 0) {
            rc = hsvd_solve_ex(G, n, r, n, J, sigma, U, ldu, nullptr, r, opts, info, stream);
            if (rc == HSVD_OK || rc == HSVD_NOT_CONVERGED) {
                k_sym_lambda<<<(unsigned)((r + 255) / 256), 256, 0, st>>>(sigma, J, r, lambda);
                if (cudaGetLastError() != cudaSuccess) rc = HSVD_ERR_CUDA;
                nl += 1;
            }
        }
        // eigenvectors of the zero eigenvalues: the orthogonal complement of
        // range(U_r) = range(G_r), the last n - r columns of the full Q of a QR
        // of U_r
        if ((rc == HSVD_OK || rc == HSVD_NOT_CONVERGED) && U && r < n) {
            double *A = ws.get<double>((size_t)n * (r > 0 ? r : 1));
            double *qws = ws.get<double>(qr_workspace_doubles(r > 0 ? r : 1));
            if (!A || !qws) {
                rc = HSVD_ERR_NOMEM;
            } else {
                double *Un = U + r * ldu;
                const int64_t tot = n * (n - r);
                k_sym_null_init<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Un, ldu, n, r);  // [0; I_(n-r)]
                nl += 1;
                if (cudaGetLastError() != cudaSuccess)
                    rc = HSVD_ERR_CUDA;
                else if (r > 0 &&
                         (cudaMemcpy2DAsync(A, sizeof(double) * n, U, sizeof(double) * ldu, sizeof(double) * n, r,
                                            cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                          qr_factor(A, n, n, r, qws, st, &nl) != cudaSuccess ||
                          qr_apply_q(A, n, n, r, qws, Un, ldu, st, &nl, n - r) != cudaSuccess))
                    rc = HSVD_ERR_CUDA;
                if (cudaStreamSynchronize(st) != cudaSuccess && rc >= 0) rc = HSVD_ERR_CUDA;
            }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess && rc >= 0) rc = HSVD_ERR_CUDA;
    }
    cudaStreamSynchronize(st);
    if (info) {
        info->kernel_launches += nl;
        info->status = rc;
    }
    return rc;
}

int hsvd_shorten_qr(const double *G, int64_t m, int64_t n, int64_t ldg, double *R, int64_t ldr, double *Q,
                    int64_t ldq, void *stream) {
    if (!G || !R || n < 1 || m < n || ldg < m || ldr < n || (Q && ldq < m)) return HSVD_ERR_ARG;
    if (n > (int64_t)1 << 24 || m > (int64_t)1 << 31) return HSVD_ERR_ARG;
    if (!all_device({G, R, Q})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = HSVD_OK;
    {
        Ws ws(st);
        double *A = ws.get<double>((size_t)m * n);
        double *qws = ws.get<double>(qr_workspace_doubles(n));
        double *I = Q ? ws.get<double>((size_t)n * n) : nullptr;
        long long nl = 0;
        if (!A || !qws || (Q && !I)) {
            rc = HSVD_ERR_NOMEM;
        } else if (cudaMemcpy2DAsync(A, sizeof(double) * m, G, sizeof(double) * ldg, sizeof(double) * m, n,
                                     cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                   qr_factor(A, m, m, n, qws, st, &nl) != cudaSuccess ||
                   qr_extract_r(A, m, n, R, ldr, st) != cudaSuccess) {
            rc = HSVD_ERR_CUDA;
        } else if (Q) {
            // Q = Q [I; 0]: the identity embedded, then the reflectors applied
            std::vector<double> eye((size_t)n * n, 0.0);
            for (int64_t i = 0; i < n; ++i) eye[(size_t)(i + i * n)] = 1.0;
            if (cudaMemcpyAsync(I, eye.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                qr_embed_u(I, n, m, n, Q, ldq, st) != cudaSuccess ||
                qr_apply_q(A, m, m, n, qws, Q, ldq, st, &nl) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = HSVD_ERR_CUDA;
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == HSVD_OK) rc = HSVD_ERR_CUDA;
    return rc;
}

int hsvd_pivot_gram(const double *G, int64_t rows, int64_t ldg, int b, int npairs, const int *col0, double *A,
                    void *stream) {
    if (!G || !col0 || !A || npairs < 1 || rows < 1 || (rows % 64) || ldg < rows) return HSVD_ERR_ARG;
    if (b != 16 && b != 32 && b != 64) return HSVD_ERR_ARG;
    if (!all_device({G, col0, A})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nsplit = gram_nsplit(rows, npairs);
    double *part = nullptr;
    if (cudaMallocAsync((void **)&part, sizeof(double) * npairs * 3 * nsplit * b * b, st) != cudaSuccess)
        return HSVD_ERR_NOMEM;
    int rc = HSVD_OK;
    if (launch_gram(G, rows, ldg, b, npairs, col0, nsplit, part, st) != cudaSuccess ||
        launch_assemble(b, npairs, part, nsplit, A, st) != cudaSuccess)
        rc = HSVD_ERR_CUDA;
    cudaFreeAsync(part, st);
    return rc;
}

int hsvd_pivot_solve(int b, int npairs, double *A, const int8_t *sgn, double tol, int mode, int max_passes, double *W,
                     int *rotated, int *status_dev, void *stream) {
    if (!A || !sgn || !W || !rotated || npairs < 1 || !(tol > 0.0)) return HSVD_ERR_ARG;
    if (b != 16 && b != 32 && b != 64) return HSVD_ERR_ARG;
    if (mode < 0 || mode > 2 || (mode == 0 && max_passes < 1)) return HSVD_ERR_ARG;
    if (!all_device({A, sgn, W, rotated, status_dev})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nn = 2 * b;
    std::vector<int> full((size_t)nn * b * 2 + ring_table_ints(b)), cross((size_t)b * b * 2);
    fill_modulus(nn, nn, full.data());
    if (!fill_ring(b, full.data() + (size_t)nn * b * 2)) return HSVD_ERR_ARG;
    fill_cross(b, cross.data());
    int *dt = nullptr;
    if (cudaMallocAsync((void **)&dt, sizeof(int) * (full.size() + cross.size()), st) != cudaSuccess)
        return HSVD_ERR_NOMEM;
    int rc = HSVD_OK;
    if (cudaMemcpyAsync(dt, full.data(), full.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dt + full.size(), cross.data(), cross.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        launch_solve(b, npairs, nullptr, 0, A, nullptr, nullptr, sgn, tol, mode, mode == 0 ? max_passes : 1, dt,
                     dt + full.size(), W, rotated, nullptr, status_dev, st) != cudaSuccess)
        rc = HSVD_ERR_CUDA;
    // the host tables must outlive the asynchronous copies
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = HSVD_ERR_CUDA;
    cudaFreeAsync(dt, st);
    return rc;
}

int hsvd_pivot_update(double *X, int64_t rows, int64_t ldx, int b, int npairs, const int *col0, const double *W,
                      const int *rotated, void *stream) {
    if (!X || !col0 || !W || !rotated || npairs < 1 || rows < 1 || (rows % 32) || ldx < rows) return HSVD_ERR_ARG;
    if (b != 16 && b != 32 && b != 64) return HSVD_ERR_ARG;
    if (!all_device({X, col0, W, rotated})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return launch_update(X, rows, ldx, nullptr, 0, 0, b, npairs, col0, W, rotated, nullptr, st) == cudaSuccess
               ? HSVD_OK
               : HSVD_ERR_CUDA;
}

int hsvd_pivot_gram_x(const double *G, int64_t rows, int64_t ldg, int npairs, const int *col0, double *A,
                      void *stream) {
    if (!G || !col0 || !A || npairs < 1 || rows < 1 || ldg < rows) return HSVD_ERR_ARG;
    if (!all_device({G, col0, A})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ks = precision_gram_ksplit(rows);
    double *part = nullptr;
    int *status = nullptr;
    if (cudaMallocAsync((void **)&part, sizeof(double) * (size_t)npairs * ks * 128 * 128, st) != cudaSuccess)
        return HSVD_ERR_NOMEM;
    if (cudaMallocAsync((void **)&status, sizeof(int), st) != cudaSuccess) {
        cudaFreeAsync(part, st);
        return HSVD_ERR_NOMEM;
    }
    int rc = HSVD_OK, h = 0;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
        launch_gram_x(G, rows, ldg, npairs, col0, part, status, st) != cudaSuccess ||
        launch_assemble_x(npairs, part, ks, A, st) != cudaSuccess ||
        cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        rc = HSVD_ERR_CUDA;
    if (rc == HSVD_OK && h) rc = h;
    cudaFreeAsync(part, st);
    cudaFreeAsync(status, st);
    return rc;
}

int hsvd_pivot_update_x(double *X, int64_t rows, int64_t ldx, int npairs, const int *col0, const double *W,
                        const int *rotated, const int *dexp, void *stream) {
    if (!X || !col0 || !W || !rotated || npairs < 1 || rows < 1 || ldx < rows) return HSVD_ERR_ARG;
    if (!all_device({X, col0, W, rotated, dexp})) return HSVD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint16_t *wsl = nullptr;
    int *wexp = nullptr, *dz = nullptr, *status = nullptr;
    int rc = HSVD_OK, h = 0;
    if (cudaMallocAsync((void **)&wsl, sizeof(uint16_t) * precision_wsl_elems(npairs), st) != cudaSuccess ||
        cudaMallocAsync((void **)&wexp, sizeof(int) * (size_t)npairs * 256, st) != cudaSuccess ||
        cudaMallocAsync((void **)&dz, sizeof(int) * (size_t)npairs * 128, st) != cudaSuccess ||
        cudaMallocAsync((void **)&status, sizeof(int), st) != cudaSuccess)
        rc = HSVD_ERR_NOMEM;
    if (rc == HSVD_OK) {
        const int *dk = dexp;
        if (!dk && cudaMemsetAsync(dz, 0, sizeof(int) * (size_t)npairs * 128, st) != cudaSuccess) rc = HSVD_ERR_CUDA;
        if (!dk) dk = dz;
        if (rc == HSVD_OK &&
            (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
             launch_wprep_x(npairs, W, dk, rotated, wsl, wexp, nullptr, st) != cudaSuccess ||
             launch_update_x(X, rows, ldx, nullptr, 0, 0, npairs, col0, wsl, wexp, dk, rotated, status, st) !=
                 cudaSuccess ||
             cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = HSVD_ERR_CUDA;
        if (rc == HSVD_OK && h) rc = h;
    }
    if (wsl) cudaFreeAsync(wsl, st);
    if (wexp) cudaFreeAsync(wexp, st);
    if (dz) cudaFreeAsync(dz, st);
    if (status) cudaFreeAsync(status, st);
    return rc;
}

}  // extern "C"
