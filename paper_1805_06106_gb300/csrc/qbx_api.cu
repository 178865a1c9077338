// extern "C" entry points declared in include/qbx.h: argument checks, handle
// lifetime and error reporting around the tree, list and evaluation drivers.
#include <cmath>
#include <cstring>
#include <new>

#include "qbx_internal.cuh"

namespace qbx {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

template <class F>
static int guarded(F &&f)
{
    try {
        g_err.clear();
        return f();
    } catch (const Error &e) {
        g_err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return QBX_ERR_OOM;
    } catch (...) {
        g_err = "unexpected exception";
        return QBX_ERR_CUDA;
    }
}

void free_tree(qbx_tree *T)
{
    if (!T) return;
    dfree(T->lvl_boxes);
    dfree(T->level); dfree(T->ic); dfree(T->cen); dfree(T->hw); dfree(T->parent); dfree(T->child);
    dfree(T->nsrc_sub); dfree(T->ntgt_sub);
    for (int k = 0; k < 3; ++k) { dfree(T->owner[k]); dfree(T->perm[k]); dfree(T->own_start[k]); }
    dfree(T->sxyz); dfree(T->cxyz); dfree(T->cr); dfree(T->txyz);
    dfree(T->ctr_box); dfree(T->tgt_box); dfree(T->ctr_rank);
    delete T;
}

void free_lists(qbx_lists *L)
{
    if (!L) return;
    for (int l = 0; l < NLIST; ++l) { dfree(L->start[l]); dfree(L->idx[l]); }
    for (int i = 0; i <= QBX_NSTAGES; ++i)
        if (L->ev[i]) cudaEventDestroy(L->ev[i]);
    free_workspace(L->ws);
    delete L;
}

}  // namespace qbx

namespace qbx {
void check_eval_args(const qbx_tree *T, const qbx_lists *L, const double *w, const double *mu, const double *nrm,
                     const int32_t *tgt_ctr, const qbx_eval_opts *o, const double *pot)
{
    if (!T || !L || !o || L->tree != T) throw Error{QBX_ERR_INVALID_ARG, "tree/lists/opts mismatch or NULL"};
    if (T->np[0] && !w) throw Error{QBX_ERR_INVALID_ARG, "src_w is NULL"};
    if (mu && !nrm) throw Error{QBX_ERR_INVALID_ARG, "mu given without normals"};
    if (T->np[2] && (!tgt_ctr || !pot)) throw Error{QBX_ERR_INVALID_ARG, "tgt_ctr/pot is NULL"};
    const int base = o->precision & 0xF, only = o->precision & ~0xF;
    if (base != QBX_FP64 && base != QBX_M2L_FP32 && base != QBX_M2L_3XTF32)
        throw Error{QBX_ERR_INVALID_ARG, "precision mode not available"};
    if (only != 0 && (base == QBX_FP64 || (only != QBX_MIXED_M2L_ONLY && only != QBX_MIXED_M2QBXL_ONLY)))
        throw Error{QBX_ERR_INVALID_ARG, "stage selection needs QBX_M2L_FP32 or QBX_M2L_3XTF32 and one stage"};
    if (o->p_qbx < 0 || o->p_qbx > QMAX) throw Error{QBX_ERR_INVALID_ARG, "p_qbx out of range"};
    if (o->p_fmm < 0 || o->p_fmm > PMAX) throw Error{QBX_ERR_INVALID_ARG, "p_fmm out of range"};
    if (!o->p_qbx_per_ctr && !o->p_fmm_per_box && o->p_qbx > o->p_fmm)
        throw Error{QBX_ERR_INVALID_ARG, "p_qbx > p_fmm"};
}
}  // namespace qbx

using namespace qbx;

extern "C" {

int qbx_build_tree(const double *src_xyz_dev, int64_t n_src, const double *ctr_xyz_dev, const double *ctr_r_dev,
                   int64_t n_ctr, const double *tgt_xyz_dev, int64_t n_tgt, const qbx_tree_opts *opts,
                   qbx_tree **out, void *stream)
{
    return guarded([&]() -> int {
        if (!out) throw Error{QBX_ERR_INVALID_ARG, "out is NULL"};
        *out = nullptr;
        if (!opts) throw Error{QBX_ERR_INVALID_ARG, "opts is NULL"};
        if (n_src < 0 || n_ctr < 0 || n_tgt < 0 || n_src + n_ctr + n_tgt < 1)
            throw Error{QBX_ERR_INVALID_ARG, "particle counts must be >= 0 with at least one particle"};
        if (n_src + n_ctr + n_tgt >= (int64_t(1) << 31)) throw Error{QBX_ERR_INVALID_ARG, "too many particles"};
        if ((n_src && !src_xyz_dev) || (n_ctr && (!ctr_xyz_dev || !ctr_r_dev)) || (n_tgt && !tgt_xyz_dev))
            throw Error{QBX_ERR_INVALID_ARG, "NULL particle array"};
        if (opts->n_max < 1 || !(opts->t_f >= 0.0) || !std::isfinite(opts->t_f) ||
            (opts->flags & ~(unsigned)(QBX_TREE_LINF_TCR | QBX_TREE_LEVEL_RESTRICT)) != 0 ||
            opts->max_depth < 1)
            throw Error{QBX_ERR_INVALID_ARG, "bad tree options"};
        if (opts->max_depth > 50) throw Error{QBX_ERR_DEPTH, "max_depth > 50"};
        qbx_tree *T = new qbx_tree();
        T->np[0] = n_src;
        T->np[1] = n_ctr;
        T->np[2] = n_tgt;
        T->n_max = opts->n_max;
        T->max_depth = opts->max_depth;
        T->tf = opts->t_f;
        T->flags = opts->flags;
        try {
            build_tree(T, src_xyz_dev, ctr_xyz_dev, ctr_r_dev, tgt_xyz_dev, (cudaStream_t)stream);
        } catch (...) {
            free_tree(T);
            throw;
        }
        *out = T;
        return QBX_OK;
    });
}

int qbx_tree_query(const qbx_tree *T, qbx_tree_info *info)
{
    return guarded([&]() -> int {
        if (!T || !info) throw Error{QBX_ERR_INVALID_ARG, "NULL argument"};
        info->n_boxes = T->nb;
        info->n_levels = T->nlev;
        info->n_src = T->np[0];
        info->n_ctr = T->np[1];
        info->n_tgt = T->np[2];
        info->n_overfull = T->n_overfull;
        for (int d = 0; d < 3; ++d) info->root_center[d] = T->root_c[d];
        info->root_radius = T->root_h;
        return QBX_OK;
    });
}

int qbx_tree_export(const qbx_tree *T, int32_t *level, int64_t *coords, int32_t *parent, int32_t *child,
                    int32_t *src_owner, int32_t *ctr_owner, int32_t *tgt_owner, void *stream)
{
    return guarded([&]() -> int {
        if (!T) throw Error{QBX_ERR_INVALID_ARG, "tree is NULL"};
        cudaStream_t st = (cudaStream_t)stream;
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            if (dst && bytes) QBX_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
        };
        cp(level, T->level, T->nb * sizeof(int));
        cp(coords, T->ic, 3 * T->nb * sizeof(int64_t));
        cp(parent, T->parent, T->nb * sizeof(int));
        cp(child, T->child, 8 * T->nb * sizeof(int));
        cp(src_owner, T->owner[0], T->np[0] * sizeof(int));
        cp(ctr_owner, T->owner[1], T->np[1] * sizeof(int));
        cp(tgt_owner, T->owner[2], T->np[2] * sizeof(int));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        return QBX_OK;
    });
}

void qbx_tree_free(qbx_tree *T) { free_tree(T); }

int qbx_build_lists(const qbx_tree *T, qbx_lists **out, void *stream)
{
    return guarded([&]() -> int {
        if (!T || !out) throw Error{QBX_ERR_INVALID_ARG, "NULL argument"};
        *out = nullptr;
        if (T->lvl_boxes) throw Error{QBX_ERR_INVALID_ARG, "a forest gets its lists from qbx_build_forest"};
        qbx_lists *L = new qbx_lists();
        L->tree = T;
        try {
            build_lists(L, (cudaStream_t)stream);
        } catch (...) {
            free_lists(L);
            throw;
        }
        *out = L;
        return QBX_OK;
    });
}

int qbx_lists_nnz(const qbx_lists *L, int which, int64_t *nnz)
{
    return guarded([&]() -> int {
        if (!L || !nnz || which < 0 || which >= NLIST) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        *nnz = L->nnz[which];
        return QBX_OK;
    });
}

int qbx_lists_export(const qbx_lists *L, int which, int32_t *start, int32_t *idx, void *stream)
{
    return guarded([&]() -> int {
        if (!L || which < 0 || which >= NLIST) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        if (start)
            QBX_CUDA_TRY(cudaMemcpyAsync(start, L->start[which], (L->tree->nb + 1) * sizeof(int),
                                         cudaMemcpyDeviceToDevice, st));
        if (idx && L->nnz[which])
            QBX_CUDA_TRY(cudaMemcpyAsync(idx, L->idx[which], L->nnz[which] * sizeof(int), cudaMemcpyDeviceToDevice, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        return QBX_OK;
    });
}

void qbx_lists_free(qbx_lists *L) { free_lists(L); }

int qbx_eval(const qbx_tree *T, const qbx_lists *L, const double *w, const double *sigma, const double *mu,
             const double *nrm, const int32_t *tgt_ctr, const qbx_eval_opts *o, double *pot, void *stream)
{
    return guarded([&]() -> int {
        check_eval_args(T, L, w, mu, nrm, tgt_ctr, o, pot);
        eval(T, const_cast<qbx_lists *>(L), w, sigma, mu, nrm, tgt_ctr, o, pot, (cudaStream_t)stream);
        return QBX_OK;
    });
}

int qbx_build_forest(int n, const qbx_tree *const *trees, const qbx_lists *const *lists, qbx_tree **forest_out,
                     qbx_lists **lists_out, void *stream)
{
    return guarded([&]() -> int {
        if (!forest_out || !lists_out || !trees || !lists || n < 1)
            throw Error{QBX_ERR_INVALID_ARG, "bad forest arguments"};
        *forest_out = nullptr;
        *lists_out = nullptr;
        for (int i = 0; i < n; ++i) {
            if (!trees[i] || !lists[i] || lists[i]->tree != trees[i])
                throw Error{QBX_ERR_INVALID_ARG, "tree/lists mismatch or NULL in the forest"};
            if (trees[i]->lvl_boxes) throw Error{QBX_ERR_INVALID_ARG, "a forest cannot contain a forest"};
        }
        qbx_tree *F = new qbx_tree();
        qbx_lists *FL = new qbx_lists();
        FL->tree = F;
        try {
            build_forest(n, trees, lists, F, FL, (cudaStream_t)stream);
        } catch (...) {
            free_lists(FL);
            free_tree(F);
            throw;
        }
        *forest_out = F;
        *lists_out = FL;
        return QBX_OK;
    });
}

int qbx_forest_problems(const qbx_tree *T, int *n_host)
{
    return guarded([&]() -> int {
        if (!T || !n_host) throw Error{QBX_ERR_INVALID_ARG, "NULL argument"};
        *n_host = T->nprob;
        return QBX_OK;
    });
}

int qbx_forest_offsets(const qbx_tree *T, int64_t *off_host)
{
    return guarded([&]() -> int {
        if (!T || !off_host) throw Error{QBX_ERR_INVALID_ARG, "NULL argument"};
        if (!T->lvl_boxes) {
            const int64_t v[8] = {0, T->nb, 0, T->np[0], 0, T->np[1], 0, T->np[2]};
            for (int i = 0; i < 8; ++i) off_host[i] = v[i];
        } else {
            for (size_t i = 0; i < T->prob_off.size(); ++i) off_host[i] = T->prob_off[i];
        }
        return QBX_OK;
    });
}

int qbx_graph_create(const qbx_tree *T, const qbx_lists *L, const double *w, const double *sigma, const double *mu,
                     const double *nrm, const int32_t *tgt_ctr, const qbx_eval_opts *o, double *pot, qbx_graph **out,
                     void *stream)
{
    return guarded([&]() -> int {
        if (!out) throw Error{QBX_ERR_INVALID_ARG, "out is NULL"};
        *out = nullptr;
        if (!stream) throw Error{QBX_ERR_INVALID_ARG, "graph capture needs a non-default stream"};
        check_eval_args(T, L, w, mu, nrm, tgt_ctr, o, pot);
        qbx_graph *g = new qbx_graph();
        try {
            capture_eval(T, const_cast<qbx_lists *>(L), w, sigma, mu, nrm, tgt_ctr, o, pot, (cudaStream_t)stream, g);
        } catch (...) {
            free_graph(g);
            throw;
        }
        *out = g;
        return QBX_OK;
    });
}

int qbx_graph_launch(qbx_graph *g, void *stream)
{
    return guarded([&]() -> int {
        if (!g || !g->exec) throw Error{QBX_ERR_INVALID_ARG, "graph is NULL"};
        QBX_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
        return QBX_OK;
    });
}

void qbx_graph_free(qbx_graph *g) { free_graph(g); }

int qbx_lists_set_tiles(qbx_lists *L, int m2l_kchunk, int m2qbxl_kchunk)
{
    return guarded([&]() -> int {
        if (!L) throw Error{QBX_ERR_INVALID_ARG, "lists is NULL"};
        if (m2l_kchunk != 0 && m2l_kchunk != 16 && m2l_kchunk != 32)
            throw Error{QBX_ERR_INVALID_ARG, "m2l_kchunk must be 0, 16 or 32"};
        if (m2qbxl_kchunk != 0 && (m2qbxl_kchunk < 16 || m2qbxl_kchunk > 128 || m2qbxl_kchunk % 8))
            throw Error{QBX_ERR_INVALID_ARG, "m2qbxl_kchunk must be 0 or a multiple of 8 in [16, 128]"};
        L->tile_m2l_kc = m2l_kchunk;
        L->tile_wfar_w = m2qbxl_kchunk;
        return QBX_OK;
    });
}

int qbx_lists_set_wait(qbx_lists *L, long long limit_cycles, int probe_step)
{
    return guarded([&]() -> int {
        if (!L || limit_cycles < 0 || probe_step < -1) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        L->wait_limit = limit_cycles;
        L->probe_step = probe_step;
        return QBX_OK;
    });
}

int qbx_profile(qbx_lists *L, int enable)
{
    return guarded([&]() -> int {
        if (!L) throw Error{QBX_ERR_INVALID_ARG, "lists is NULL"};
        if (enable && !L->ev[0])
            for (int i = 0; i <= QBX_NSTAGES; ++i) QBX_CUDA_TRY(cudaEventCreate(&L->ev[i]));
        L->prof = enable != 0;
        L->prof_valid = false;
        return QBX_OK;
    });
}

int qbx_profile_read(const qbx_lists *L, double *ms)
{
    return guarded([&]() -> int {
        if (!L || !ms) throw Error{QBX_ERR_INVALID_ARG, "NULL argument"};
        if (!L->prof_valid) throw Error{QBX_ERR_INVALID_ARG, "no profiled evaluation to read"};
        QBX_CUDA_TRY(cudaEventSynchronize(L->ev[QBX_NSTAGES]));
        for (int i = 0; i < QBX_NSTAGES; ++i) {
            float t = 0.f;
            QBX_CUDA_TRY(cudaEventElapsedTime(&t, L->ev[i], L->ev[i + 1]));
            ms[i] = t;
        }
        return QBX_OK;
    });
}

int qbx_eval_order_sweep(const qbx_tree *T, const qbx_lists *L, const double *w, const double *sigma,
                         const double *mu, const double *nrm, const int32_t *tgt_ctr, const qbx_eval_opts *o,
                         double *partial, void *stream)
{
    return guarded([&]() -> int {
        if (!o || o->p_qbx_per_ctr) throw Error{QBX_ERR_INVALID_ARG, "order sweep needs a fixed p_qbx"};
        int rc = qbx_eval(T, L, w, sigma, mu, nrm, tgt_ctr, o, partial, stream);
        if (rc != QBX_OK) throw Error{rc, g_err};
        eval_order_sweep(T, const_cast<qbx_lists *>(L), w, sigma, mu, nrm, tgt_ctr, o, partial, (cudaStream_t)stream);
        return QBX_OK;
    });
}

int qbx_lists_cost(const qbx_lists *L, int p_qbx, int p_fmm, qbx_cost *cost, void *stream)
{
    return guarded([&]() -> int {
        if (!L || !cost || p_qbx < 0 || p_fmm < 0) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        const qbx_tree *T = L->tree;
        list_counts(L, cost->count, (cudaStream_t)stream);
        const double q2 = (double)p_qbx * p_qbx, p3 = (double)p_fmm * p_fmm * p_fmm, p2 = (double)p_fmm * p_fmm;
        const double per_entry[NLIST] = {q2, p3, q2, p3, q2, p2};  // U, V, W-close, W-far, X-close, X-far
        for (int l = 0; l < NLIST; ++l) cost->ops[l] = per_entry[l] * (double)cost->count[l];
        cost->ops_stages = (double)T->np[KSRC] * p2 + (double)T->nb * p3 + 8.0 * (double)T->nb * p3 +
                           (double)T->np[KCTR] * p3 + (double)T->np[KTGT] * q2;
        double tot = 0.0;
        for (int l = 0; l < NLIST; ++l) tot += cost->ops[l];
        cost->ops_total = tot + cost->ops_stages;
        return QBX_OK;
    });
}

const char *qbx_last_error(void) { return g_err.c_str(); }

}  // extern "C"
