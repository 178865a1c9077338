// Batched problems: a forest is the concatenation of independently built trees and their
// interaction lists.  Box, particle and list indices of problem i are shifted by the sizes of
// problems 0..i-1; the lists never cross problems, so every stage of the evaluation (Algorithm 4,
// Stages 2-9) runs over all problems in one launch (level-synchronous stages over the union of
// each level), and one evaluation can be captured as one CUDA graph (qbx_graph_*).
#include <algorithm>

#include "qbx_internal.cuh"

namespace qbx {

// dst[i] = src[i] + add (negative entries kept as they are when keep_negative)
__global__ void k_copy_shift(int *dst, const int *src, int64_t n, int add, bool keep_negative)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = src[i];
    dst[i] = (keep_negative && v < 0) ? v : v + add;
}

static void shift(int *dst, const int *src, int64_t n, int add, bool keep_negative, cudaStream_t st)
{
    if (n <= 0) return;
    k_copy_shift<<<nblocks(n, 256), 256, 0, st>>>(dst, src, n, add, keep_negative);
    QBX_LAUNCH_CHECK();
}

template <class T>
static void copy(T *dst, const T *src, int64_t n, cudaStream_t st)
{
    if (n > 0) QBX_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
}

static void set_int(int *dst, int v, cudaStream_t st)
{
    QBX_CUDA_TRY(cudaMemcpyAsync(dst, &v, sizeof(int), cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaStreamSynchronize(st));  // v lives on this stack frame
}

void build_forest(int n, const qbx_tree *const *trees, const qbx_lists *const *lists, qbx_tree *F, qbx_lists *FL,
                  cudaStream_t st)
{
    // sizes and offsets
    F->nprob = n;
    F->prob_off.assign(4 * (n + 1), 0);
    int64_t nb = 0, np[3] = {0, 0, 0}, nnz[NLIST] = {};
    int nlev = 0;
    for (int i = 0; i < n; ++i) {
        const qbx_tree *T = trees[i];
        F->prob_off[0 * (n + 1) + i] = nb;
        for (int k = 0; k < 3; ++k) F->prob_off[(k + 1) * (n + 1) + i] = np[k];
        nb += T->nb;
        for (int k = 0; k < 3; ++k) np[k] += T->np[k];
        for (int l = 0; l < NLIST; ++l) nnz[l] += lists[i]->nnz[l];
        nlev = std::max<int>(nlev, (int)T->nlev);
        F->n_overfull += T->n_overfull;
        F->n_max = std::max(F->n_max, T->n_max);
        F->max_depth = std::max(F->max_depth, T->max_depth);
    }
    F->prob_off[0 * (n + 1) + n] = nb;
    for (int k = 0; k < 3; ++k) F->prob_off[(k + 1) * (n + 1) + n] = np[k];
    if (nb >= (int64_t(1) << 31) || np[0] + np[1] + np[2] >= (int64_t(1) << 31))
        throw Error{QBX_ERR_INVALID_ARG, "forest too large for 32-bit indices"};
    for (int l = 0; l < NLIST; ++l)
        if (nnz[l] >= (int64_t(1) << 31)) throw Error{QBX_ERR_INVALID_ARG, "forest lists too large"};
    F->nb = nb;
    F->nlev = nlev;
    for (int k = 0; k < 3; ++k) F->np[k] = np[k];
    F->tf = trees[0]->tf;
    F->flags = trees[0]->flags;
    for (int d = 0; d < 3; ++d) F->root_c[d] = trees[0]->root_c[d];
    F->root_h = trees[0]->root_h;

    // box arrays
    F->level = dalloc<int>(nb);
    F->ic = dalloc<int64_t>(3 * nb);
    F->cen = dalloc<double>(3 * nb);
    F->hw = dalloc<double>(nb);
    F->parent = dalloc<int>(nb);
    F->child = dalloc<int>(8 * nb);
    F->nsrc_sub = dalloc<int>(nb);
    F->ntgt_sub = dalloc<int>(nb);
    for (int k = 0; k < 3; ++k) {
        F->owner[k] = dalloc<int>(np[k]);
        F->perm[k] = dalloc<int>(np[k]);
        F->own_start[k] = dalloc<int>(nb + 1);
    }
    F->sxyz = dalloc<double>(3 * np[KSRC]);
    F->cxyz = dalloc<double>(3 * np[KCTR]);
    F->cr = dalloc<double>(np[KCTR]);
    F->txyz = dalloc<double>(3 * np[KTGT]);
    F->ctr_box = dalloc<int>(np[KCTR]);
    F->tgt_box = dalloc<int>(np[KTGT]);
    F->ctr_rank = dalloc<int>(np[KCTR]);
    for (int l = 0; l < NLIST; ++l) {
        FL->start[l] = dalloc<int>(nb + 1);
        FL->idx[l] = dalloc<int>(nnz[l]);
        FL->nnz[l] = nnz[l];
    }

    std::vector<int64_t> eoff(NLIST, 0);
    for (int i = 0; i < n; ++i) {
        const qbx_tree *T = trees[i];
        const qbx_lists *L = lists[i];
        const int64_t b0 = F->prob_off[i], tb = T->nb;
        const int ob = (int)b0;
        int64_t o[3];
        for (int k = 0; k < 3; ++k) o[k] = F->prob_off[(k + 1) * (n + 1) + i];
        copy(F->level + b0, T->level, tb, st);
        copy(F->ic + 3 * b0, T->ic, 3 * tb, st);
        copy(F->cen + 3 * b0, T->cen, 3 * tb, st);
        copy(F->hw + b0, T->hw, tb, st);
        copy(F->nsrc_sub + b0, T->nsrc_sub, tb, st);
        copy(F->ntgt_sub + b0, T->ntgt_sub, tb, st);
        shift(F->parent + b0, T->parent, tb, ob, true, st);
        shift(F->child + 8 * b0, T->child, 8 * tb, ob, true, st);
        for (int k = 0; k < 3; ++k) {
            shift(F->owner[k] + o[k], T->owner[k], T->np[k], ob, false, st);
            shift(F->perm[k] + o[k], T->perm[k], T->np[k], (int)o[k], false, st);
            shift(F->own_start[k] + b0, T->own_start[k], tb, (int)o[k], false, st);
        }
        for (int d = 0; d < 3; ++d) {
            copy(F->sxyz + d * np[KSRC] + o[KSRC], T->sxyz + d * T->np[KSRC], T->np[KSRC], st);
            copy(F->cxyz + d * np[KCTR] + o[KCTR], T->cxyz + d * T->np[KCTR], T->np[KCTR], st);
            copy(F->txyz + d * np[KTGT] + o[KTGT], T->txyz + d * T->np[KTGT], T->np[KTGT], st);
        }
        copy(F->cr + o[KCTR], T->cr, T->np[KCTR], st);
        shift(F->ctr_box + o[KCTR], T->ctr_box, T->np[KCTR], ob, false, st);
        shift(F->tgt_box + o[KTGT], T->tgt_box, T->np[KTGT], ob, false, st);
        shift(F->ctr_rank + o[KCTR], T->ctr_rank, T->np[KCTR], (int)o[KCTR], false, st);
        for (int l = 0; l < NLIST; ++l) {
            shift(FL->start[l] + b0, L->start[l], tb, (int)eoff[l], false, st);
            shift(FL->idx[l] + eoff[l], L->idx[l], L->nnz[l], ob, false, st);
            eoff[l] += L->nnz[l];
        }
    }
    for (int k = 0; k < 3; ++k) set_int(F->own_start[k] + nb, (int)np[k], st);
    for (int l = 0; l < NLIST; ++l) set_int(FL->start[l] + nb, (int)nnz[l], st);

    // boxes grouped by level across problems
    std::vector<int> lb;
    lb.reserve(nb);
    F->level_start.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        F->level_start[l] = (int)lb.size();
        for (int i = 0; i < n; ++i) {
            const qbx_tree *T = trees[i];
            if (l >= T->nlev) continue;
            for (int b = T->level_start[l]; b < T->level_start[l + 1]; ++b) lb.push_back((int)F->prob_off[i] + b);
        }
    }
    F->level_start[nlev] = (int)lb.size();
    F->lvl_boxes = dalloc<int>(nb);
    QBX_CUDA_TRY(cudaMemcpyAsync(F->lvl_boxes, lb.data(), lb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace qbx

// ---------------------------------------------------------------- captured evaluation

namespace qbx {

void free_graph(qbx_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// Runs one evaluation eagerly (argument checks, workspace and plan set-up), then captures a
// second one on `st` and instantiates it.
void capture_eval(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu,
                  const double *nrm, const int *tgt_ctr, const qbx_eval_opts *o, double *pot, cudaStream_t st,
                  qbx_graph *g)
{
    eval(T, L, w, sigma, mu, nrm, tgt_ctr, o, pot, st);
    QBX_CUDA_TRY(cudaStreamSynchronize(st));
    const bool prof = L->prof;
    L->prof = false;  // no event records inside the graph
    QBX_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        eval(T, L, w, sigma, mu, nrm, tgt_ctr, o, pot, st);
    } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(st, &junk);
        if (junk) cudaGraphDestroy(junk);
        cudaGetLastError();
        L->prof = prof;
        throw;
    }
    L->prof = prof;
    QBX_CUDA_TRY(cudaStreamEndCapture(st, &g->graph));
    QBX_CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
}

}  // namespace qbx
