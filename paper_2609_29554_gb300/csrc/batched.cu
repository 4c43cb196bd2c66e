// Batched LU and solve of many independent, unevenly sized instances.
//
// Instances are sorted by size and spread over up to 8 library-owned streams
// (greedy, by n^3), each with its own workspace, so that the latency-bound
// panels of small instances run side by side: the cooperative panel kernel of
// an instance takes about one SM per 16 rows.  Every residue GEMM of an
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

constexpr int NSUB = 8;

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

// fork onto the sub-streams, run `work(k, list)` on each, join back
int fork_join(ozlu_handle* h, const std::vector<std::vector<int>>& lists,
              const std::function<int(ozlu_handle*, const std::vector<int>&)>& work) {
    if (cudaEventRecord(h->fork, h->stream) != cudaSuccess) return OZLU_ERR_CUDA;
    int rc = OZLU_OK;
    for (int k = 0; k < NSUB; ++k) {
        if (lists[k].empty()) continue;
        ozlu_handle* s = h->sub[k];
        if (cudaStreamWaitEvent(s->stream, h->fork, 0) != cudaSuccess) return OZLU_ERR_CUDA;
        s->capturing = h->capturing;
        s->timing = false;
        rc = work(s, lists[k]);
        if (rc) break;
        if (cudaEventRecord(h->join[k], s->stream) != cudaSuccess) return OZLU_ERR_CUDA;
        if (cudaStreamWaitEvent(h->stream, h->join[k], 0) != cudaSuccess) return OZLU_ERR_CUDA;
    }
    return rc;
}

// eager, capture or replay, keyed by the batch description
int run_batched(ozlu_handle* h, const std::vector<long long>& key, bool graph,
                const std::function<int()>& issue) {
    if (!graph) return issue();
    auto g = h->graphs.find(key);
    if (g != h->graphs.end())
        return cudaGraphLaunch(g->second, h->stream) == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
    if (h->warm[key] == 0) {
        const int rc = issue();
        if (!rc) h->warm[key] = 1;
        return rc;
    }
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return issue();
    }
    h->capturing = true;
    const int rc = issue();
    h->capturing = false;
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &gr);
    if (rc || ce != cudaSuccess || !gr) {
        cudaGetLastError();
        if (gr) cudaGraphDestroy(gr);
        return rc ? rc : issue();  // capture not possible here: run eagerly
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        return issue();
    }
    h->graphs[key] = ex;
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
    if (nb == 0) nb = 128;
    if (nb < 1) return -10;
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
    std::vector<long long> key{1, nc, p, count, nb, o.backend, o.nslice, o.extra_groups, o.g_ex, o.native,
                               (long long)info};
    for (int i = 0; i < count; ++i) {
        key.push_back(n[i]);
        key.push_back((long long)A[i]);
        key.push_back(lda[i]);
        key.push_back((long long)ipiv[i]);
    }
    const auto lists = assign(count, n);
    auto issue = [&]() -> int {
        return fork_join(h, lists, [&](ozlu_handle* s, const std::vector<int>& list) -> int {
            for (int i : list) {
                const int r = getrf_one(s, nc, p, n[i], A[i], lda[i], ipiv[i], nb, info + i, &o);
                if (r) return r;
                s->count(1);
            }
            return (int)OZLU_OK;
        });
    };
    rc = run_batched(h, key, o.graph != 0, issue);
    long long launches = 0;
    for (int k = 0; k < NSUB; ++k)
        if (h->sub[k]) launches += h->sub[k]->stats.launches;
    h->stats.launches = launches;
    return rc;
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
    std::vector<long long> key{2, nc, p, count, nrhs, o.backend, o.nslice, o.extra_groups, o.g_ex};
    for (int i = 0; i < count; ++i) {
        key.push_back(n[i]);
        key.push_back((long long)LU[i]);
        key.push_back((long long)B[i]);
        key.push_back((long long)ipiv[i]);
    }
    const auto lists = assign(count, n);
    auto issue = [&]() -> int {
        return fork_join(h, lists, [&](ozlu_handle* s, const std::vector<int>& list) -> int {
            for (int i : list) {
                if (n[i] == 0) continue;
                const int r = getrs_one(s, nc, p, n[i], nrhs, LU[i], lda[i], ipiv[i], B[i], ldb[i], &o);
                if (r) return r;
            }
            return (int)OZLU_OK;
        });
    };
    return run_batched(h, key, o.graph != 0, issue);
}
