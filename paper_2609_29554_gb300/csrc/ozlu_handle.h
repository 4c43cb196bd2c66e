// The handle: stream, device workspace, plan cache, last-GEMM layout, timers.
#pragma once

#include <map>
#include <tuple>
#include <utility>
#include <vector>

#include "ozlu_internal.h"

namespace ozlu {

struct Workspace {
    void* base = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes);
    void release();
};

struct PlanEntry {
    Plan plan;
    DevTable table;
};

// byte offsets of the last ozlu_gemm's intermediates inside the workspace
struct GemmLayout {
    int m = 0, n = 0, k = 0, Mpad = 0, Npad = 0, Kpad = 0, N = 0, S = 0, G = 0, backend = 0;
    size_t mu = 0, nu = 0, ra = 0, rb = 0, t = 0;
};

}  // namespace ozlu

constexpr int MAX_SUB = 32;  // library streams of the batched driver

struct ozlu_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    ozlu::Workspace ws;     // GEMM intermediates
    ozlu::Workspace stage;  // host-argument staging
    ozlu::Workspace tune_ws;  // scratch output of the back-end autotuner
    // shape key -> (back-end, slice count) chosen by the autotuner
    std::map<std::tuple<int, int, int, int, int, int>, std::pair<int, int>> tuned;
    std::map<std::tuple<int, int, int, int>, int> tuned_nb;  // (nc, p, log2 n, backend) -> nb
    ozlu::Workspace nb_ws;  // scratch copy of A for the panel-width autotuner
    std::map<std::tuple<int, int, int, int, int, int>, ozlu::PlanEntry> plans;
    ozlu::GemmLayout last;
    int* dev_err = nullptr;  // device error word of the tensor-core GEMMs
    // second stream of the GEMM's conversion: B's exponents and residues run
    // beside A's (fork / join events on the handle's stream)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    bool timing = false;
    ozlu_stats stats = {};
    void* lu_scratch = nullptr;  // pivot-search scratch of ozlu_getrf
    void* coop_scratch = nullptr;  // grid-barrier and candidate slots of the panel kernel
    size_t coop_bytes = 0;
    int coop_min_rows = 16;  // rows per block of the panel kernel at least (32 on batched sub-streams)
    // phase timing: (phase, start, end) event triples resolved in ozlu_get_stats
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    int open_phase = -1;
    cudaEvent_t open_ev = nullptr;
    void phase(int ph);     // close the open phase (if any) and open ph (-1: none)
    void resolve_times();
    void count(long long launches) { stats.launches += launches; }
    bool capturing = false;  // inside a CUDA-graph capture: no host synchronisation
    // batched driver: sub-handles with their own streams and workspaces, fork/join
    // events, and instantiated graphs keyed by the batch description
    ozlu_handle* sub[MAX_SUB] = {};
    cudaStream_t cap_stream = nullptr;  // graph captures run here
    cudaEvent_t fork = nullptr, join[MAX_SUB] = {};
    struct Graph {
        cudaGraphExec_t exec;  // null: capture failed, the batch runs eagerly
        ozlu_stats work;       // counters of the captured call, added on each replay
        int status;            // graph_status of ozlu_stats
    };
    std::map<std::vector<long long>, Graph> graphs;
    std::map<std::vector<long long>, int> warm;
    // p-bit calls: options (modulus table, slice count) and the device tables
    // of extended-table plans, keyed by (p, K, S)
    ozlu_opts mp_opts = {};
    struct ExtPlan {
        ozlu::Plan plan;
        void* dev = nullptr;
        ozlu::ExtDev view;
    };
    std::map<std::tuple<int, int, int>, ExtPlan> ext_plans;
};

enum { PH_CONVERT = 0, PH_GEMM = 1, PH_CRT = 2, PH_PANEL = 3, PH_OTHER = 4, PH_TRSM = 5 };

namespace ozlu {
int getrf_one(ozlu_handle* h, int nc, int p, int n, double* A, long long lda, int* ipiv, int nb, int* info_out,
              const ozlu_opts* opts);
int tune_nb(ozlu_handle* h, int nc, int p, int n, const double* A, long long lda, const ozlu_opts* opts,
            int* nb_out);
int getrs_one(ozlu_handle* h, int nc, int p, int n, int nrhs, const double* LU, long long lda, const int* ipiv,
              double* B, long long ldb, const ozlu_opts* opts);
int gemm_device(ozlu_handle* h, int nc, int p, int m, int n, int k, int alpha, const double* A,
                long long lda, const double* B, long long ldb, int beta, double* C,
                long long ldc, const ozlu_opts* opts);
bool is_device_ptr(const void* p);
int* err_word(ozlu_handle* h);
int mp_gemm_device(ozlu_handle* h, int p, int m, int n, int k, int alpha, const ozlu_mp_matrix& A,
                   const ozlu_mp_matrix& B, int beta, const ozlu_mp_matrix& C);
int clear_err_word(ozlu_handle* h);
// the handle's second stream, forked from s (made by the first call outside a
// graph capture); s itself when there is none
cudaStream_t side_fork(ozlu_handle* h, cudaStream_t s);
// s waits for the work issued on `side` (nothing when side is s); false on a
// CUDA error
bool side_join(ozlu_handle* h, cudaStream_t s, cudaStream_t side);
int cuda_rc(cudaError_t e);
}  // namespace ozlu
