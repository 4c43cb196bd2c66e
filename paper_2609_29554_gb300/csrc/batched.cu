// Batched LU and solve of many independent, unevenly sized instances.
//
// Instances are sorted by size and spread over up to 32 library-owned streams
// (greedy, by n^3), each with its own workspace, so that the latency-bound
// panels of small instances run side by side: the cooperative panel kernel of
// an instance takes about one SM per 32 rows.  Every residue GEMM of an
// instance covers all moduli and digit groups in one launch.  With
// opts->graph set, the whole batch (fork, per-stream instance sequences,
// join) is captured into a CUDA graph on the second call with the same batch
// description (sizes and pointers) and replayed from the third call on: the
// first call warms the workspaces and the back-end autotuner, so nothing
// inside the capture allocates or waits for the host.
#include <string.h>

#include <algorithm>
#include <functional>
#include <numeric>
#include <vector>

#include "ozlu_handle.h"

namespace ozlu {
namespace {

constexpr int NSUB = MAX_SUB;

int ensure_subs(ozlu_handle* h) {
    if (!h->fork && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) return OZLU_ERR_CUDA;
    for (int k = 0; k < NSUB; ++k) {
        if (h->sub[k]) continue;
        ozlu_handle* s = new ozlu_handle();
        s->device = h->device;
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return OZLU_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&h->join[k], cudaEventDisableTiming) != cudaSuccess) return OZLU_ERR_CUDA;
        h->sub[k] = s;
    }
    return OZLU_OK;
}

// every option field is part of a graph's key (a graph replays one configuration)
void append_opts(std::vector<long long>& key, const ozlu_opts& o) {
    const int* w = reinterpret_cast<const int*>(&o);
    for (size_t i = 0; i < sizeof(ozlu_opts) / sizeof(int); ++i) key.push_back(w[i]);
}

// greedy assignment of instances (largest first) to the least-loaded stream
std::vector<std::vector<int>> assign(int count, const int* n) {
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    std::vector<std::vector<int>> lists(NSUB);
    std::vector<double> load(NSUB, 0.0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[k].push_back(i);
        load[k] += (double)n[i] * n[i] * n[i] + 1e6;  // + fixed cost per instance
    }
    return lists;
}

// fork from `root` onto the sub-streams, issue the instances round-robin
// (one instance per stream in turn, so that a full launch queue never holds
// one stream's work alone), then join every forked stream back into `root`
int fork_join(ozlu_handle* h, cudaStream_t root, const std::vector<std::vector<int>>& lists,
              const std::function<int(ozlu_handle*, int)>& work) {
    if (cudaEventRecord(h->fork, root) != cudaSuccess) return OZLU_ERR_CUDA;
    size_t rounds = 0;
    for (int k = 0; k < NSUB; ++k) {
        if (lists[k].empty()) continue;
        ozlu_handle* s = h->sub[k];
        if (cudaStreamWaitEvent(s->stream, h->fork, 0) != cudaSuccess) return OZLU_ERR_CUDA;
        s->capturing = h->capturing;
        s->timing = h->timing && !h->capturing;
        rounds = std::max(rounds, lists[k].size());
    }
    int rc = OZLU_OK;
    for (size_t r = 0; r < rounds && !rc; ++r)
        for (int k = 0; k < NSUB && !rc; ++k)
            if (r < lists[k].size()) rc = work(h->sub[k], lists[k][r]);
    for (int k = 0; k < NSUB; ++k) {  // join all, also after an error (a capture needs it)
        if (lists[k].empty()) continue;
        ozlu_handle* s = h->sub[k];
        s->phase(-1);
        if (cudaEventRecord(h->join[k], s->stream) != cudaSuccess ||
            cudaStreamWaitEvent(root, h->join[k], 0) != cudaSuccess)
            rc = rc ? rc : OZLU_ERR_CUDA;
    }
    return rc;
}

// the work counters of the sub-handles (launches, operations, bytes)
ozlu_stats sub_counters(ozlu_handle* h) {
    ozlu_stats c;
    memset(&c, 0, sizeof c);
    for (int k = 0; k < NSUB; ++k) {
        if (!h->sub[k]) continue;
        const ozlu_stats& s = h->sub[k]->stats;
        c.gemm_launches += s.gemm_launches;
        c.crt_launches += s.crt_launches;
        c.panel_launches += s.panel_launches;
        c.launches += s.launches;
        c.gemm_ops += s.gemm_ops;
        c.crt_bytes += s.crt_bytes;
        c.convert_bytes += s.convert_bytes;
    }
    return c;
}

// eager, capture or replay, keyed by the batch description; a replay adds
// the counters the captured call recorded, so the statistics count the
// kernels a replay runs.  The capture runs on a library-owned stream (the
// caller's stream may be the legacy default stream, which cannot capture);
// the graph is then launched on the caller's stream.
int run_batched(ozlu_handle* h, const std::vector<long long>& key, bool graph,
                const std::function<int(cudaStream_t)>& issue_on) {
    auto issue = [&]() { return issue_on(h->stream); };
    if (!graph) return issue();
    auto g = h->graphs.find(key);
    if (g != h->graphs.end()) {
        if (!g->second.exec) {  // capture failed before: stay eager
            h->stats.graph_status = g->second.status;
            return issue();
        }
        if (cudaGraphLaunch(g->second.exec, h->stream) != cudaSuccess) return OZLU_ERR_CUDA;
        h->stats.graph_status = 2;
        const ozlu_stats& d = g->second.work;
        ozlu_stats& s = h->stats;
        s.gemm_launches += d.gemm_launches;
        s.crt_launches += d.crt_launches;
        s.panel_launches += d.panel_launches;
        s.launches += d.launches;
        s.gemm_ops += d.gemm_ops;
        s.crt_bytes += d.crt_bytes;
        s.convert_bytes += d.convert_bytes;
        return OZLU_OK;
    }
    if (h->warm[key] == 0) {
        const int rc = issue();
        if (!rc) h->warm[key] = 1;
        h->stats.graph_status = 0;
        return rc;
    }
    auto fail = [&](cudaError_t e) -> int {
        cudaGetLastError();
        h->graphs[key] = {nullptr, {}, -(int)e};
        h->stats.graph_status = -(int)e;
        return issue();
    };
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(cudaErrorUnknown);
    cudaGraph_t gr = nullptr;
    const cudaError_t be = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
    if (be != cudaSuccess) return fail(be);
    const ozlu_stats before = sub_counters(h);
    h->capturing = true;
    const int rc = issue_on(h->cap_stream);
    h->capturing = false;
    ozlu_stats work = sub_counters(h);
    work.gemm_launches -= before.gemm_launches;
    work.crt_launches -= before.crt_launches;
    work.panel_launches -= before.panel_launches;
    work.launches -= before.launches;
    work.gemm_ops -= before.gemm_ops;
    work.crt_bytes -= before.crt_bytes;
    work.convert_bytes -= before.convert_bytes;
    const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &gr);
    if (rc || ce != cudaSuccess || !gr) {
        if (gr) cudaGraphDestroy(gr);
        if (rc) {
            cudaGetLastError();
            return rc;
        }
        return fail(ce != cudaSuccess ? ce : cudaErrorUnknown);  // not capturable: run eagerly
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) return fail(ie);
    h->graphs[key] = {ex, work, 1};
    h->stats.graph_status = 1;
    return cudaGraphLaunch(ex, h->stream) == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

}  // namespace
}  // namespace ozlu

using namespace ozlu;

extern "C" int ozlu_getrf_batched(ozlu_handle* h, int nc, int p, int count, const int* n, double* const* A,
                                  const long long* lda, int* const* ipiv, int* info, int nb,
                                  const ozlu_opts* opts) {
    if (!h) return -1;
    if (nc < 2 || nc > 4) return -2;
    if (p == 0) p = 53 * nc;
    if (p < 1 || p > 53 * nc) return -3;
    if (count < 0) return -4;
    if (count == 0) return OZLU_OK;
    if (!n) return -5;
    if (!A) return -6;
    if (!lda) return -7;
    if (!ipiv) return -8;
    if (!info || !is_device_ptr(info)) return -9;
    if (nb < 0) return -10;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 0) return -5;
        if (n[i] && (!A[i] || !is_device_ptr(A[i]))) return -6;
        if (lda[i] < (n[i] > 1 ? n[i] : 1)) return -7;
        if (n[i] && (!ipiv[i] || !is_device_ptr(ipiv[i]))) return -8;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    int rc = ensure_subs(h);
    if (rc) return rc;
    ozlu_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    std::vector<long long> key{1, nc, p, count, nb, (long long)info};
    append_opts(key, o);
    for (int i = 0; i < count; ++i) {
        key.push_back(n[i]);
        key.push_back((long long)A[i]);
        key.push_back(lda[i]);
        key.push_back((long long)ipiv[i]);
    }
    // nb = 0: each instance takes the measured panel width of its size class
    // (tuned on the first call, one representative instance per class)
    std::vector<int> nbs(count, nb);
    if (nb == 0) {
        for (int i = 0; i < count; ++i) {
            if (n[i] == 0) { nbs[i] = 1; continue; }
            if ((rc = tune_nb(h, nc, p, n[i], A[i], lda[i], &o, &nbs[i]))) return rc;
        }
    }
    const auto lists = assign(count, n);
    // concurrent instances take fewer SMs per panel (32 rows per block at least;
    // 256 TD instances: 576 ms against 643 ms with 16); a single instance keeps 16
    for (int k = 0; k < NSUB; ++k) h->sub[k]->coop_min_rows = count > 1 ? 32 : 16;
    auto issue = [&](cudaStream_t root) -> int {
        return fork_join(h, root, lists, [&](ozlu_handle* s, int i) -> int {
            return getrf_one(s, nc, p, n[i], A[i], lda[i], ipiv[i], nbs[i], info + i, &o);
        });
    };
    return run_batched(h, key, o.graph != 0, issue);
}

extern "C" int ozlu_getrs_batched(ozlu_handle* h, int nc, int p, int count, const int* n, int nrhs,
                                  const double* const* LU, const long long* lda, const int* const* ipiv,
                                  double* const* B, const long long* ldb, const ozlu_opts* opts) {
    if (!h) return -1;
    if (nc < 2 || nc > 4) return -2;
    if (p == 0) p = 53 * nc;
    if (p < 1 || p > 53 * nc) return -3;
    if (count < 0) return -4;
    if (count == 0 || nrhs == 0) return OZLU_OK;
    if (!n) return -5;
    if (nrhs < 0) return -6;
    if (!LU || !lda || !ipiv || !B || !ldb) return -7;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 0) return -5;
        if (n[i] && (!is_device_ptr(LU[i]) || !is_device_ptr(ipiv[i]) || !is_device_ptr(B[i]))) return -7;
        if (lda[i] < (n[i] > 1 ? n[i] : 1) || ldb[i] < (n[i] > 1 ? n[i] : 1)) return -7;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    int rc = ensure_subs(h);
    if (rc) return rc;
    ozlu_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    std::vector<long long> key{2, nc, p, count, nrhs};
    append_opts(key, o);
    for (int i = 0; i < count; ++i) {
        key.push_back(n[i]);
        key.push_back((long long)LU[i]);
        key.push_back((long long)B[i]);
        key.push_back((long long)ipiv[i]);
    }
    const auto lists = assign(count, n);
    auto issue = [&](cudaStream_t root) -> int {
        return fork_join(h, root, lists, [&](ozlu_handle* s, int i) -> int {
            if (n[i] == 0) return (int)OZLU_OK;
            return getrs_one(s, nc, p, n[i], nrhs, LU[i], lda[i], ipiv[i], B[i], ldb[i], &o);
        });
    };
    return run_batched(h, key, o.graph != 0, issue);
}
