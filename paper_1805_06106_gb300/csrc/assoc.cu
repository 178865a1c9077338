// Target association (Section 3.4, Algorithm 3) on the built tree, from the point of view of the
// targets: one thread per target searches the tree from the root for the boxes whose closed cube
// meets a query cube around the target.
//   Stage 1: sources within the largest danger radius; the target is endangered if some source s
//            has |t - s| <= r_danger(s); the nearest source (lowest input index among equals) gives
//            the preferred side sign((t - s*) . n(s*)).
//   Stage 2: centers within the largest association radius r_c (1 + eps), owned by any box (centers
//            may sit in non-leaf boxes); the closest center on the preferred side with
//            |t - c| <= r_c (1 + eps) wins, ties to the lowest input index.
//   Stage 3: endangered targets left without a center are flagged.
// The result is the set the paper's source- and center-centric area queries (Algorithm 5) produce:
// every source or center inside a query cube lies in a box that meets the cube, and so do all of
// that box's ancestors.  Distances are sqrt(dx^2 + dy^2 + dz^2) with explicitly rounded operations,
// so the comparisons agree bit for bit with a CPU evaluation of the same expressions.
#include "qbx_internal.cuh"

namespace qbx {

constexpr int ASSOC_STACK = 512;

__device__ __forceinline__ double rn_dist(double x0, double x1, double x2, double y0, double y1, double y2)
{
    const double dx = __dsub_rn(x0, y0), dy = __dsub_rn(x1, y1), dz = __dsub_rn(x2, y2);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// largest value of a non-negative array (IEEE doubles of one sign order like their bit patterns)
__global__ void k_max_nonneg(int64_t n, const double *v, const int *perm, double scale, unsigned long long *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, __dmul_rn(v[perm ? perm[i] : i], scale));
    for (int off = 16; off >= 1; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

struct AssocArgs {
    int64_t nt, ns, nc;
    const int *tperm, *sperm, *cperm;           // sorted position -> input index
    const double *txyz, *sxyz, *cxyz, *cr;      // sorted geometry of the tree
    const double *cen, *hw;
    const int *child, *own_src, *own_ctr;
    const double *rdanger;                      // input order
    const double *snrm;                         // (3, ns) input order, or null: no side preference
    const signed char *cside;                   // input order
    double eps;
    const unsigned long long *rmax;             // [0] danger, [1] association radius bound (as bits)
    int *tgt_ctr;
    signed char *flagged;
    int *err;
};

__device__ __forceinline__ bool meets(const AssocArgs &a, int b, double x, double y, double z, double r)
{
    const double e = __dadd_rn(r, a.hw[b]);
    return fabs(__dsub_rn(x, a.cen[3 * b])) <= e && fabs(__dsub_rn(y, a.cen[3 * b + 1])) <= e &&
           fabs(__dsub_rn(z, a.cen[3 * b + 2])) <= e;
}

__global__ void k_assoc(AssocArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nt) return;
    const double x = a.txyz[i], y = a.txyz[a.nt + i], z = a.txyz[2 * a.nt + i];
    const int ti = a.tperm[i];
    int stack[ASSOC_STACK];
    // Stage 1: endangerment and the nearest source
    const double R1 = __longlong_as_double((long long)a.rmax[0]);
    bool endangered = false;
    double dbest = INFINITY;
    int sbest = -1, sslot = -1;  // nearest source: input index and sorted slot
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int b = stack[--sp];
        if (!meets(a, b, x, y, z, R1)) continue;
        bool leaf = true;
        for (int o = 0; o < 8; ++o) {
            const int ch = a.child[8 * b + o];
            if (ch < 0) continue;
            leaf = false;
            if (sp < ASSOC_STACK) stack[sp++] = ch;
            else atomicOr(a.err, 1);
        }
        if (!leaf) continue;
        for (int j = a.own_src[b]; j < a.own_src[b + 1]; ++j) {
            const int sj = a.sperm[j];
            const double d = rn_dist(x, y, z, a.sxyz[j], a.sxyz[a.ns + j], a.sxyz[2 * a.ns + j]);
            if (d <= a.rdanger[sj]) endangered = true;
            if (d < dbest || (d == dbest && sj < sbest)) {
                dbest = d;
                sbest = sj;
                sslot = j;
            }
        }
    }
    a.tgt_ctr[ti] = -1;
    a.flagged[ti] = 0;
    if (!endangered) return;
    // preferred side: sign of (t - s*) . n(s*), summed as ((dx nx + dy ny) + dz nz)
    int side = 0;
    if (a.snrm) {
        const double dx = __dsub_rn(x, a.sxyz[sslot]), dy = __dsub_rn(y, a.sxyz[a.ns + sslot]),
                     dz = __dsub_rn(z, a.sxyz[2 * a.ns + sslot]);
        const double dot = __dadd_rn(__dadd_rn(__dmul_rn(dx, a.snrm[sbest]), __dmul_rn(dy, a.snrm[a.ns + sbest])),
                                     __dmul_rn(dz, a.snrm[2 * a.ns + sbest]));
        side = dot > 0.0 ? 1 : -1;
    }
    // Stage 2: the closest admissible center, owned by any box that meets the query cube
    const double R2 = __longlong_as_double((long long)a.rmax[1]);
    const double f = __dadd_rn(1.0, a.eps);
    double cbest = INFINITY;
    int cidx = -1;
    sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int b = stack[--sp];
        if (!meets(a, b, x, y, z, R2)) continue;
        for (int o = 0; o < 8; ++o) {
            const int ch = a.child[8 * b + o];
            if (ch < 0) continue;
            if (sp < ASSOC_STACK) stack[sp++] = ch;
            else atomicOr(a.err, 1);
        }
        for (int k = a.own_ctr[b]; k < a.own_ctr[b + 1]; ++k) {
            const int ck = a.cperm[k];
            if (a.snrm && a.cside[ck] != side) continue;
            const double d = rn_dist(x, y, z, a.cxyz[k], a.cxyz[a.nc + k], a.cxyz[2 * a.nc + k]);
            if (d <= __dmul_rn(a.cr[k], f) && (d < cbest || (d == cbest && ck < cidx))) {
                cbest = d;
                cidx = ck;
            }
        }
    }
    // Stage 3
    a.tgt_ctr[ti] = cidx;
    a.flagged[ti] = cidx < 0 ? 1 : 0;
}


// ---------------------------------------------------------------- refinement marks (Section 3)

// Algorithms 1 and 2 mark elements for bisection from per-point tests over a tree of the sources
// and centers; one thread per query point searches the tree from the root for the boxes whose
// closed cube meets the query cube (padded by a relative 1e-12 against rounding in the box test;
// the distance test itself is exact in the same expression as a CPU evaluation):
//   which 0 (Algorithm 1): query = center i, radius (1 - eps) r_i, hit = a source strictly
//           inside; marks the element that spawned the center (sources live in leaves);
//   which 1 (Algorithm 2): query = source j of element k, radius 0.375 eta_k (0.5 (3/4) eta_k),
//           hit = a center at most that far, owned by any box (centers may sit above the leaves);
//           marks element k.
struct RefineArgs {
    int which;
    int64_t nq, ns, nc, n_elem;
    const int *qperm;                           // sorted query slot -> input index
    const double *qxyz;                         // sorted query points
    const double *qr;                           // which 0: sorted center radii
    const double *sxyz, *cxyz;
    const double *cen, *hw;
    const int *child, *own_src, *own_ctr;
    const int *elem;                            // input order: element of each query point
    const double *eta;                          // which 1: eta per element
    double eps;
    unsigned char *mark;
    int *err;                                   // 1: stack overflow, 2: element index out of range
};

__global__ void k_refine_marks(RefineArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nq) return;
    const int e = a.elem[a.qperm[i]];
    if (e < 0 || e >= a.n_elem) {
        atomicOr(a.err, 2);
        return;
    }
    if (a.mark[e]) return;  // already marked by another point of the element (a benign read)
    const double x = a.qxyz[i], y = a.qxyz[a.nq + i], z = a.qxyz[2 * a.nq + i];
    const double R = a.which == 0 ? __dmul_rn(__dsub_rn(1.0, a.eps), a.qr[i]) : __dmul_rn(0.375, a.eta[e]);
    int stack[ASSOC_STACK];
    int sp = 0;
    stack[sp++] = 0;
    bool hit = false;
    while (sp > 0 && !hit) {
        const int b = stack[--sp];
        const double ext = __dmul_rn(__dadd_rn(R, a.hw[b]), 1.0 + 1e-12);
        if (!(fabs(__dsub_rn(x, a.cen[3 * b])) <= ext && fabs(__dsub_rn(y, a.cen[3 * b + 1])) <= ext &&
              fabs(__dsub_rn(z, a.cen[3 * b + 2])) <= ext))
            continue;
        bool leaf = true;
        for (int o = 0; o < 8; ++o) {
            const int ch = a.child[8 * b + o];
            if (ch < 0) continue;
            leaf = false;
            if (sp < ASSOC_STACK) stack[sp++] = ch;
            else atomicOr(a.err, 1);
        }
        if (a.which == 0) {
            if (!leaf) continue;
            for (int j = a.own_src[b]; j < a.own_src[b + 1] && !hit; ++j)
                hit = rn_dist(x, y, z, a.sxyz[j], a.sxyz[a.ns + j], a.sxyz[2 * a.ns + j]) < R;
        } else {
            for (int k = a.own_ctr[b]; k < a.own_ctr[b + 1] && !hit; ++k)
                hit = rn_dist(x, y, z, a.cxyz[k], a.cxyz[a.nc + k], a.cxyz[2 * a.nc + k]) <= R;
        }
    }
    if (hit) a.mark[e] = 1;
}
}  // namespace qbx

using namespace qbx;

extern "C" int qbx_assoc_targets(const qbx_tree *T, const double *rdanger, const double *src_n,
                                 const int8_t *ctr_side, double eps, int32_t *tgt_ctr, int8_t *flagged, void *stream)
{
    try {
        set_error("");
        if (!T || !tgt_ctr || !flagged || (T->np[KSRC] && !rdanger) || (src_n && !ctr_side && T->np[KCTR]) ||
            !(eps >= 0.0) || T->nprob != 1)
            throw Error{QBX_ERR_INVALID_ARG, "bad argument (NULL array, eps < 0, or a forest)"};
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t nt = T->np[KTGT];
        if (nt == 0) return QBX_OK;
        unsigned long long *rmax = dalloc<unsigned long long>(2);
        int *err = dalloc<int>(1);
        try {
            QBX_CUDA_TRY(cudaMemsetAsync(rmax, 0, 2 * sizeof(unsigned long long), st));
            QBX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
            if (T->np[KSRC])
                k_max_nonneg<<<152, 256, 0, st>>>(T->np[KSRC], rdanger, nullptr, 1.0, rmax);
            if (T->np[KCTR])
                k_max_nonneg<<<152, 256, 0, st>>>(T->np[KCTR], T->cr, nullptr, 1.0 + eps, rmax + 1);
            QBX_LAUNCH_CHECK();
            AssocArgs a{nt,       T->np[KSRC], T->np[KCTR], T->perm[KTGT], T->perm[KSRC], T->perm[KCTR],
                        T->txyz,  T->sxyz,     T->cxyz,     T->cr,         T->cen,        T->hw,
                        T->child, T->own_start[KSRC], T->own_start[KCTR], rdanger, src_n,
                        reinterpret_cast<const signed char *>(ctr_side), eps, rmax, tgt_ctr,
                        reinterpret_cast<signed char *>(flagged), err};
            k_assoc<<<nblocks(nt, 128), 128, 0, st>>>(a);
            QBX_LAUNCH_CHECK();
            int e = 0;
            QBX_CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            if (e) throw Error{QBX_ERR_CUDA, "target association: traversal stack overflow"};
        } catch (...) {
            dfree(rmax);
            dfree(err);
            throw;
        }
        dfree(rmax);
        dfree(err);
        return QBX_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected exception");
        return QBX_ERR_CUDA;
    }
}

extern "C" int qbx_refine_marks(const qbx_tree *T, int which, const int32_t *elem, const double *elem_eta,
                                int64_t n_elem, double eps, uint8_t *marks, void *stream)
{
    try {
        set_error("");
        if (!T || !elem || !marks || n_elem < 0 || T->nprob != 1 || (which != QBX_REFINE_INTERFERING &&
                                                                     which != QBX_REFINE_QUAD_RES))
            throw Error{QBX_ERR_INVALID_ARG, "bad argument (NULL array, which, n_elem < 0, or a forest)"};
        if (which == QBX_REFINE_INTERFERING && !(eps >= 0.0 && eps < 1.0))
            throw Error{QBX_ERR_INVALID_ARG, "eps must lie in [0, 1)"};
        if (which == QBX_REFINE_QUAD_RES && !elem_eta) throw Error{QBX_ERR_INVALID_ARG, "elem_eta is NULL"};
        cudaStream_t st = (cudaStream_t)stream;
        if (n_elem == 0) return QBX_OK;
        QBX_CUDA_TRY(cudaMemsetAsync(marks, 0, (size_t)n_elem, st));
        const bool q_is_ctr = which == QBX_REFINE_INTERFERING;
        const int64_t nq = q_is_ctr ? T->np[KCTR] : T->np[KSRC];
        if (nq == 0) return QBX_OK;
        int *err = dalloc<int>(1);
        try {
            QBX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
            RefineArgs a{which,        nq,       T->np[KSRC],  T->np[KCTR],
                         n_elem,       q_is_ctr ? T->perm[KCTR] : T->perm[KSRC],
                         q_is_ctr ? T->cxyz : T->sxyz,          T->cr,
                         T->sxyz,      T->cxyz,  T->cen,       T->hw,
                         T->child,     T->own_start[KSRC], T->own_start[KCTR], elem, elem_eta, eps,
                         reinterpret_cast<unsigned char *>(marks), err};
            k_refine_marks<<<nblocks(nq, 128), 128, 0, st>>>(a);
            QBX_LAUNCH_CHECK();
            int e = 0;
            QBX_CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            if (e & 2) throw Error{QBX_ERR_INVALID_ARG, "element index out of range"};
            if (e & 1) throw Error{QBX_ERR_CUDA, "refinement marks: traversal stack overflow"};
        } catch (...) {
            dfree(err);
            throw;
        }
        dfree(err);
        return QBX_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected exception");
        return QBX_ERR_CUDA;
    }
}
