// Internal declarations shared by the translation units of libqbx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qbx.h"

namespace qbx {

// ---------------------------------------------------------------- errors

void set_error(const std::string &msg);

struct Error {
    int code;
    std::string msg;
};

#define QBX_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw ::qbx::Error{e_ == cudaErrorMemoryAllocation ? QBX_ERR_OOM : QBX_ERR_CUDA,  \
                               std::string(#expr) + ": " + cudaGetErrorString(e_)};           \
    } while (0)

#define QBX_LAUNCH_CHECK() QBX_CUDA_TRY(cudaGetLastError())

template <class T>
T *dalloc(size_t n)
{
    void *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();  // an allocation failure must not surface again at the next launch check
        throw ::qbx::Error{e == cudaErrorMemoryAllocation ? QBX_ERR_OOM : QBX_ERR_CUDA,
                           "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes: " + cudaGetErrorString(e)};
    }
    return static_cast<T *>(p);
}

inline void dfree(void *p)
{
    if (p) cudaFree(p);
}

inline unsigned nblocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- kinds and constants

enum { KSRC = 0, KCTR = 1, KTGT = 2 };
enum { LU = 0, LV = 1, LWC = 2, LWF = 3, LXC = 4, LXF = 5, NLIST = 6 };

constexpr int PMAX = 20;   // highest FMM order
constexpr int QMAX = 16;   // highest QBX order

__host__ __device__ constexpr int ntri(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ constexpr int tri(int n, int m) { return n * (n + 1) / 2 + m; }

}  // namespace qbx

// ---------------------------------------------------------------- handles

struct qbx_tree {
    int64_t nb = 0, nlev = 0, np[3] = {0, 0, 0}, n_overfull = 0;
    int n_max = 0, max_depth = 0;
    double tf = 0.0;
    unsigned flags = 0;  // QBX_TREE_LINF_TCR, QBX_TREE_LEVEL_RESTRICT
    double root_c[3] = {0, 0, 0}, root_h = 0.0;
    std::vector<int> level_start;  // host copy, nlev + 1
    // device box arrays
    int *level = nullptr;
    int64_t *ic = nullptr;   // 3 per box
    double *cen = nullptr;   // 3 per box
    double *hw = nullptr;    // |b|
    int *parent = nullptr;
    int *child = nullptr;    // 8 per box
    int *nsrc_sub = nullptr, *ntgt_sub = nullptr;
    // particles: owner in input order, perm (sorted position -> input index), CSR over boxes
    int *owner[3] = {nullptr, nullptr, nullptr};
    int *perm[3] = {nullptr, nullptr, nullptr};
    int *own_start[3] = {nullptr, nullptr, nullptr};
    // geometry in sorted order, SoA
    double *sxyz = nullptr, *cxyz = nullptr, *cr = nullptr, *txyz = nullptr;
    int *ctr_box = nullptr;   // owning box of each sorted center
    int *tgt_box = nullptr;   // owning box of each sorted target
    int *ctr_rank = nullptr;  // input center index -> sorted position
    // forest of several problems (qbx_build_forest): the boxes of level l are
    // lvl_boxes[level_start[l] .. level_start[l+1]); plain trees keep lvl_boxes == nullptr and
    // number their boxes by level
    int *lvl_boxes = nullptr;
    int nprob = 1;
    std::vector<int64_t> prob_off;  // 4 x (nprob + 1) prefix sums: boxes, sources, centers, targets
};

struct qbx_workspace;

struct qbx_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct qbx_lists {
    const qbx_tree *tree = nullptr;
    int *start[qbx::NLIST] = {};
    int *idx[qbx::NLIST] = {};
    int64_t nnz[qbx::NLIST] = {};
    qbx_workspace *ws = nullptr;
    int tile_m2l_kc = 0;                     // List 2 tensor-core K chunk (0: library default)
    int tile_wfar_w = 0;                     // List 3 far tensor-core K chunk cap (0: library default)
    long long wait_limit = 0;                // tensor-core pipeline wait limit in clock cycles (0: default)
    int probe_step = -1;                     // failure-path probe step of the tensor-core pipelines (-1: off)
    bool prof = false;                       // record stage events in qbx_eval
    bool prof_valid = false;                 // the events hold a finished profiled evaluation
    cudaEvent_t ev[QBX_NSTAGES + 1] = {};
};

namespace qbx {
// records stage event i when profiling is on
inline void stage_mark(qbx_lists *L, int i, cudaStream_t st)
{
    if (L->prof) QBX_CUDA_TRY(cudaEventRecord(L->ev[i], st));
}
}  // namespace qbx

namespace qbx {
void build_tree(qbx_tree *T, const double *sxyz, const double *cxyz, const double *cr, const double *txyz,
                cudaStream_t st);
void build_lists(qbx_lists *L, cudaStream_t st);
void eval(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu,
          const double *nrm, const int *tgt_ctr, const qbx_eval_opts *o, double *pot, cudaStream_t st);
void free_workspace(qbx_workspace *ws);
void prep_sources(const int *perm, int64_t ns, const double *w, const double *sigma, const double *mu,
                  const double *nrm, double *sq, double *sd, int *flags, cudaStream_t st);
void eval_order_sweep(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu,
                      const double *nrm, const int *tgt_ctr, const qbx_eval_opts *o, double *partial, cudaStream_t st);
void exclusive_scan(const int *in, int *out, int64_t n, int base_offset, int *total_dev, cudaStream_t st);
void free_tree(qbx_tree *T);
void free_lists(qbx_lists *L);
void build_forest(int n, const qbx_tree *const *trees, const qbx_lists *const *lists, qbx_tree *F, qbx_lists *FL,
                  cudaStream_t st);
void free_graph(qbx_graph *g);
void capture_eval(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu,
                  const double *nrm, const int *tgt_ctr, const qbx_eval_opts *o, double *pot, cudaStream_t st,
                  qbx_graph *g);
void sort_pairs_by_key(int *keys, int *vals, int64_t n, int key_bits, cudaStream_t st);
void list_counts(const qbx_lists *L, int64_t *counts_host, cudaStream_t st);
// argument checks shared by the evaluation entry points (throws Error{QBX_ERR_INVALID_ARG, ...})
void check_eval_args(const qbx_tree *T, const qbx_lists *L, const double *w, const double *mu, const double *nrm,
                     const int32_t *tgt_ctr, const qbx_eval_opts *o, const double *pot);
}  // namespace qbx
