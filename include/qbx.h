/*
 * qbx.h - C ABI of the GB300 GIGAQBX library (3D Laplace single- and double-layer
 * potentials by quadrature by expansion, accelerated by the GIGAQBX FMM of
 * Wala & Kloeckner, "A Fast Algorithm for Quadrature by Expansion in Three
 * Dimensions", arXiv 1805.06106).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are device pointers (CUDA global memory) owned by the
 *     caller; host pointers are marked *_host.  Point arrays are structure-of-arrays
 *     (3, N) float64: x[0..N), y[0..N), z[0..N).
 *   - Every call that takes a `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) enqueues its device work on that stream.  Calls that
 *     return sizes or host data synchronize that stream before returning.
 *   - Return value 0 on success, a negative QBX_ERR_* code otherwise; nothing is
 *     printed and nothing aborts.  qbx_last_error() returns a message for the last
 *     failure on the calling thread.  After an error no output is guaranteed.
 *   - Handles (qbx_tree, qbx_lists) are owned by the library and released only by
 *     the matching *_free call.  A tree keeps its own sorted copy of the geometry,
 *     taken when it is built: rebuild the tree if the geometry changes.
 *     Densities may change freely between qbx_eval calls.
 */
#ifndef QBX_H
#define QBX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QBX_OK 0
#define QBX_ERR_INVALID_ARG (-1) /* NaN/Inf input, radius <= 0, bad order, bad index, mu without normals */
#define QBX_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define QBX_ERR_OOM (-3)         /* device allocation failed */
#define QBX_ERR_DEPTH (-4)       /* max_depth beyond what exact dyadic box geometry allows (> 50) */
#define QBX_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */

/* qbx_eval_opts.precision */
#define QBX_FP64 0         /* every stage in FP64 */
#define QBX_M2L_FP32 1     /* List 2 M2L and List 3-far M2QBXL in FP32; the rest FP64 */
#define QBX_M2L_3XTF32 2   /* the same two stages as split-TF32 tensor-core products, FP32 accumulation */
/* OR'ed into QBX_M2L_FP32 or QBX_M2L_3XTF32 to reduce the precision of one of the two stages only,
   so that the error of each reduced-precision stage can be measured on its own: */
#define QBX_MIXED_M2L_ONLY 0x10     /* List 2 M2L reduced; List 3-far M2QBXL stays FP64 */
#define QBX_MIXED_M2QBXL_ONLY 0x20  /* List 3-far M2QBXL reduced; List 2 M2L stays FP64 */

/* list identifiers for qbx_lists_nnz / qbx_lists_export (Section 5.2.3-5.2.4) */
#define QBX_LIST_U 0      /* List 1 */
#define QBX_LIST_V 1      /* List 2 */
#define QBX_LIST_WCLOSE 2 /* List 3 close */
#define QBX_LIST_WFAR 3   /* List 3 far */
#define QBX_LIST_XCLOSE 4 /* List 4 close */
#define QBX_LIST_XFAR 5   /* List 4 far */

typedef struct qbx_tree qbx_tree;
typedef struct qbx_lists qbx_lists;
typedef struct qbx_graph qbx_graph;

/* qbx_tree_opts.flags: tree variants (both off = the method of Section 5.2) */
#define QBX_TREE_LINF_TCR 1u       /* box-shaped TCR of the two-dimensional method (Table l2-comparison) */
#define QBX_TREE_LEVEL_RESTRICT 2u /* adjacent leaves differ by at most one level (Section 5.3, Remark
                                      "Effect of level-restriction on List 3 complexity") */

typedef struct {
    int n_max;       /* split boxes owning more than n_max particles (Algorithm 4, Stage 1); >= 1 */
    double t_f;      /* target confinement factor t_f (Section 5.2.2); >= 0 */
    int max_depth;   /* deepest level created; 0 < max_depth <= 50 */
    unsigned flags;  /* 0 or an OR of QBX_TREE_LINF_TCR, QBX_TREE_LEVEL_RESTRICT */
} qbx_tree_opts;

typedef struct {
    int64_t n_boxes, n_levels, n_src, n_ctr, n_tgt;
    int64_t n_overfull;      /* leaves left above n_max because max_depth was reached */
    double root_center[3];
    double root_radius;      /* l-infinity radius |root| */
} qbx_tree_info;

/*
 * Octree with target confinement (Algorithm 4 Stage 1; Section 5.2.1-5.2.2).
 * The root is centered at the midpoint of the bounding box of all points and
 * expansion balls, rounded to a multiple of R/8, R the smallest power of two at
 * least 1.25 x the largest half extent.  A box owning more than n_max particles
 * (sources + centers + targets) splits if some particle can move: points go to the
 * octant "coordinate >= box center", a center goes to its octant child only if its
 * ball lies inside the child's TCR, B2(sqrt(3)|child|(1+t_f)).  Only non-empty
 * children are made.  Boxes are numbered by (level, Morton code).
 * Variants (opts->flags):
 *   QBX_TREE_LINF_TCR: the TCR of a box is the cube of l-infinity radius |b|(1+t_f) about its
 *     center (the region of the two-dimensional method that Table l2-comparison compares with),
 *     both for where a center goes and in the relation a < TCR(b) of the lists, which then
 *     measures the l-infinity distance to that cube;
 *   QBX_TREE_LEVEL_RESTRICT: after Stage 1 the tree is made level-restricted in rounds; a round
 *     splits every leaf that touches (closed cubes meet) a leaf two or more levels finer, moving
 *     its particles by the Stage 1 rule, until a round splits nothing (a leaf none of whose
 *     particles can move stays a leaf).
 *   src_xyz_dev (3,n_src), ctr_xyz_dev (3,n_ctr), ctr_r_dev (n_ctr, > 0), tgt_xyz_dev (3,n_tgt):
 *   device arrays, read during the call only.  n_* >= 0, n_src + n_ctr + n_tgt >= 1.
 *   out: receives a new handle.
 * Errors: QBX_ERR_INVALID_ARG (non-finite coordinate, radius <= 0, bad options),
 * QBX_ERR_DEPTH, QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_build_tree(const double *src_xyz_dev, int64_t n_src, const double *ctr_xyz_dev, const double *ctr_r_dev,
                   int64_t n_ctr, const double *tgt_xyz_dev, int64_t n_tgt, const qbx_tree_opts *opts,
                   qbx_tree **out, void *stream);

/* Sizes of a built tree (host struct). */
int qbx_tree_query(const qbx_tree *tree, qbx_tree_info *info_host);

/*
 * Copy the tree into caller arrays (device pointers, sizes from qbx_tree_query):
 * level[n_boxes], coords[3*n_boxes] (integer box coordinates at the box's level,
 * interleaved x,y,z), parent[n_boxes] (-1 for the root), child[8*n_boxes] (octant
 * o = x_bit | y_bit<<1 | z_bit<<2, -1 = none), and the owning box of every source,
 * center and target in input order.  Any pointer may be NULL to skip that array.
 */
int qbx_tree_export(const qbx_tree *tree, int32_t *level_dev, int64_t *coords_dev, int32_t *parent_dev,
                    int32_t *child_dev, int32_t *src_owner_dev, int32_t *ctr_owner_dev, int32_t *tgt_owner_dev,
                    void *stream);

void qbx_tree_free(qbx_tree *tree);

/*
 * Interaction lists U (List 1), V (List 2), W-close/W-far (List 3 close/far),
 * X-close/X-far (List 4 close/far) of Section 5.2.3-5.2.4, as CSR over boxes with
 * each box's entries in ascending box order.  Lists U and W are made for boxes owning
 * a center or a target, lists V and X for those boxes and their ancestors; boxes whose
 * subtree holds no source appear in no list; k-colleagues exclude the box itself.
 * The handle keeps a pointer to `tree`: free the lists before the tree.
 * Errors: QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_build_lists(const qbx_tree *tree, qbx_lists **out, void *stream);

/* Number of entries of list `which` (QBX_LIST_*). */
int qbx_lists_nnz(const qbx_lists *lists, int which, int64_t *nnz_host);

/* Copy list `which` as start[n_boxes+1], idx[nnz] (device pointers). */
int qbx_lists_export(const qbx_lists *lists, int which, int32_t *start_dev, int32_t *idx_dev, void *stream);

void qbx_lists_free(qbx_lists *lists);

/*
 * Target association (Section 3.4, Algorithm 3): decides which targets of the tree need QBX and
 * associates each of them with an expansion center.  A target t is endangered if some source s has
 * |t - s| <= r_danger(s) (the danger zone eta_k / 2 of the source's element); an endangered target is
 * associated with the closest center c with |t - c| <= r_c (1 + eps), ties to the lowest center index;
 * with a side preference (src_n given) only centers on t's preferred side qualify, the side of
 * (t - s*) . n(s*) for the source s* nearest to t (positive: ctr_side +1, otherwise -1).  Endangered
 * targets without such a center are flagged.  The search runs from each target's point of view over
 * the boxes of the tree that meet a cube around it (the sets Algorithm 5's area queries return).
 *   src_danger_r_dev [n_src] (> 0), src_n_dev (3, n_src) or NULL (no side preference),
 *   ctr_side_dev [n_ctr] (+1 / -1; required with src_n), eps >= 0;
 *   tgt_ctr_dev [n_tgt] out: center index or -1; flagged_dev [n_tgt] out: 1 for endangered targets
 *   left without a center, else 0.  All arrays in input order.  Not for forests.
 * Every target of the tree is associated: build the tree with the targets to associate (points
 * with their own centers known beforehand are simply left out).
 * Errors: QBX_ERR_INVALID_ARG, QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_assoc_targets(const qbx_tree *tree, const double *src_danger_r_dev, const double *src_n_dev,
                      const int8_t *ctr_side_dev, double eps, int32_t *tgt_ctr_dev, int8_t *flagged_dev,
                      void *stream);

typedef struct {
    /* interaction counts per list (index QBX_LIST_*), n_t = QBX centers owned by the target box,
     * n_s = sources owned by the source box (its whole subtree for List 4 far):
     * U, W-close, X-close: sum over entries of n_s n_t;  V: entries;  W-far: sum of n_t;
     * X-far: sum of n_s.  Exact integers. */
    int64_t count[6];
    double ops[6];      /* modeled operations per list: count x p_qbx^2 (U, W-close, X-close),
                           x p_fmm^3 (V, W-far), x p_fmm^2 (X-far) */
    double ops_stages;  /* the stage terms no list carries: N_S p_fmm^2 + N_B p_fmm^3 (Stage 2),
                           8 N_B p_fmm^3 (Stage 7), N_C p_fmm^3 (Stage 8), N_T p_qbx^2 (Stage 9) */
    double ops_total;   /* ops[0] + ... + ops[5] + ops_stages, summed in that order */
} qbx_cost;

/*
 * Modeled operation counts of one evaluation (Section 6.3): the per-entry costs of Table
 * ilist-operation-counts over the built lists, plus the remaining stage costs of Table
 * complexity-analysis, for orders p_qbx and p_fmm.  The counts are reduced on the device
 * (integer sums); the call synchronizes `stream`.
 *   cost_host: host struct, overwritten.
 * Errors: QBX_ERR_INVALID_ARG (NULL handle or output, negative order), QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_lists_cost(const qbx_lists *lists, int p_qbx, int p_fmm, qbx_cost *cost_host, void *stream);

typedef struct {
    int p_qbx;                   /* QBX order, 0 <= p_qbx <= 16; with p_qbx_per_ctr: the largest entry allowed */
    int p_fmm;                    /* FMM order, 0 <= p_fmm <= 20: the order of every multipole expansion, and of
                                     every box's local expansion unless p_fmm_per_box is given */
    const int8_t *p_qbx_per_ctr;  /* optional device array [n_ctr], per-center QBX order in [0, p_qbx] */
    const int8_t *p_fmm_per_box;  /* optional device array [n_boxes], order in [0, p_fmm] of each box's local
                                     expansion (List 2 M2L and List 4 far P2L outputs, L2L, L2QBXL, L2P);
                                     multipoles always have the order p_fmm */
    int precision;                /* QBX_FP64, QBX_M2L_FP32 or QBX_M2L_3XTF32 (the latter two optionally
                                     OR QBX_MIXED_M2L_ONLY or QBX_MIXED_M2QBXL_ONLY) */
} qbx_eval_opts;

/*
 * Element marks of the geometry processing (Section 3): the tests by which Algorithm 1
 * (stage-1 refinement: expansion balls disturbed by source geometry, Section 3.2) and
 * Algorithm 2 (stage-2 refinement: quadrature resolution near centers, Section 3.3) choose the
 * elements to bisect, evaluated over `tree`, a tree of the sources and the expansion centers
 * (targets are not needed).  Each query point searches the boxes of the tree that meet a cube
 * around it (the area queries of Appendix A):
 *   which = QBX_REFINE_INTERFERING (Algorithm 1): for every center c_i, the element elem_dev[i]
 *     that spawned it is marked if some source s has |c_i - s| < (1 - eps) r_i; eps is the
 *     disturbance tolerance (0.025 in the paper; 0 <= eps < 1) that keeps the source point
 *     below the center out of the test.  elem_dev[n_ctr] in input center order; elem_eta unused.
 *   which = QBX_REFINE_QUAD_RES (Algorithm 2): for every source s_j, its element k = elem_dev[j]
 *     is marked if some center c has |c - s_j| <= 0.5 (3/4) eta_k; elem_dev[n_src] in input source
 *     order, elem_eta_dev[n_elem] the elements' resolution measure eta_k (eq. stretch-factor).
 *   marks_dev[n_elem] out: 1 for marked elements, 0 otherwise.
 * Distances are sqrt(dx^2 + dy^2 + dz^2) with correctly rounded operations in that order.  The
 * bisection itself and the loop until nothing is marked belong to the caller, who owns the mesh.
 * Not for forests.
 * Errors: QBX_ERR_INVALID_ARG (NULL array, bad `which` or eps, element index outside [0, n_elem)),
 * QBX_ERR_OOM, QBX_ERR_CUDA.
 */
#define QBX_REFINE_INTERFERING 0
#define QBX_REFINE_QUAD_RES 1
int qbx_refine_marks(const qbx_tree *tree, int which, const int32_t *elem_dev, const double *elem_eta_dev,
                     int64_t n_elem, double eps, uint8_t *marks_dev, void *stream);

/*
 * GIGAQBX FMM evaluation (Algorithm 4, Stages 2-9) of
 *     pot[t] = S[sigma](t) + D[mu](t),
 *     S[sigma](x) = int G(x,y) sigma(y) dS(y),  D[mu](x) = int d/dn(y) G(x,y) mu(y) dS(y),
 *     G(x,y) = 1/(4 pi |x-y|)                                   (eq. laplace-fs-green)
 * discretised by the source quadrature: charges w sigma and dipoles w mu n at the
 * sources.  A target t with tgt_ctr[t] = c >= 0 is evaluated through the order-p_qbx
 * QBX local expansion at center c (eqs. qbxcoeff, qbxlocal); tgt_ctr[t] = -1 marks a
 * conventional (point) target.
 *   src_w_dev[n_src]   quadrature weight x area element (> 0)
 *   sigma_dev[n_src]   single-layer density, or NULL for none
 *   mu_dev[n_src]      double-layer density, or NULL for none
 *   src_n_dev (3,n_src) unit outward normals; required iff mu_dev != NULL
 *   tgt_ctr_dev[n_tgt] center index or -1
 *   pot_dev[n_tgt]     output, overwritten
 * All arrays are in the input order given to qbx_build_tree.  The first call with a
 * given (orders, precision) allocates the library's workspace; later calls allocate
 * nothing and may be captured in a CUDA graph.
 * Precision: QBX_FP64; QBX_M2L_FP32 or QBX_M2L_3XTF32 reduce List 2 M2L and List 3-far M2QBXL
 * (Stages 4 and 5(b)); OR'ed with QBX_MIXED_M2L_ONLY or QBX_MIXED_M2QBXL_ONLY they reduce only
 * that stage and keep the other in FP64.
 * Errors: QBX_ERR_INVALID_ARG (orders out of range, p_qbx > p_fmm for fixed orders,
 * mu without normals, tgt_ctr out of range, a stage selection without a reduced mode or with
 * both stages), QBX_ERR_TIMEOUT (a bounded wait of a tensor-core pipeline gave up),
 * QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_eval(const qbx_tree *tree, const qbx_lists *lists, const double *src_w_dev, const double *sigma_dev,
             const double *mu_dev, const double *src_n_dev, const int32_t *tgt_ctr_dev,
             const qbx_eval_opts *opts, double *pot_dev, void *stream);

/*
 * Order sweep of the QBX expansions (generates the order-versus-error data the learned
 * orders are trained on).  Runs qbx_eval with `opts`, then writes, for every target t and
 * every QBX order q = 0..p_qbx (fixed orders only), the potential with each QBX local
 * truncated at order q:
 *     partial_dev[q * n_tgt + t] = 1/(4 pi) sum_{k <= q} sum_l A_k^l R_k^l((c - t)/r_c)
 * The coefficients of order k do not depend on the truncation order (they are produced by
 * the same P2QBXL, M2QBXL and L2QBXL sums), so column q equals a qbx_eval at p_qbx = q
 * with the same p_fmm.  Point targets get their potential in every column.
 *   partial_dev: device array of (p_qbx + 1) * n_tgt doubles, overwritten.
 * Errors: as qbx_eval; QBX_ERR_INVALID_ARG if per-center orders are given.
 */
int qbx_eval_order_sweep(const qbx_tree *tree, const qbx_lists *lists, const double *src_w_dev,
                         const double *sigma_dev, const double *mu_dev, const double *src_n_dev,
                         const int32_t *tgt_ctr_dev, const qbx_eval_opts *opts, double *partial_dev, void *stream);

/* ------------------------------------------------------------------------------------------
 * Learned expansion orders.  Not in the paper: a small network picks per-center QBX orders and
 * per-box FMM orders that the fixed-order evaluation (its acceptance check and fallback) would accept
 * within a tolerance.  Training data are order sweeps of the method itself
 * (qbx_eval_order_sweep and qbx_eval at several p_fmm); the network is trained by the kernels
 * below.  All pointers are device pointers unless marked _host.
 * ------------------------------------------------------------------------------------------ */

/* Number of floats of the network's parameter vector: W1[64][4], b1[64], W2[64][64], b2[64],
 * W3[2][64], b3[2] (4 -> 64 -> 64 -> 2, tanh hidden layers, linear output). */
#define QBX_MLP_NPARAMS 4610

/*
 * Four features per QBX center, written to feat[4*c..4*c+3] in input center order, b the box owning c:
 * log2(r_c/|b|), level(b)/8, (|c - c_b| + r_c)/|b| (how far the expansion ball reaches from the
 * center of b, where b's local expansion is centered), and log10 of the largest source strength
 * |w sigma| + |w mu n| over the sources of List 1 of b relative to the largest over all sources
 * (+1e-12).  Computed in FP64, stored as float.  Densities as in qbx_eval.
 * Errors: QBX_ERR_INVALID_ARG, QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_center_features(const qbx_tree *tree, const qbx_lists *lists, const double *src_w_dev,
                        const double *sigma_dev, const double *mu_dev, const double *src_n_dev, float *feat_dev,
                        void *stream);

/*
 * Order labels from a sweep: values[k*n + t] holds target t's result at the k-th order of the
 * sweep (increasing orders order_of_host[k], the last one the reference).  labels[t] =
 * order_of_host[k*] for the smallest k* such that every column k >= k* is within tol of the
 * reference (absolute).  n_orders <= 64.
 */
int qbx_order_labels(const double *values_dev, int n_orders, const int *order_of_host, int64_t n, double tol,
                     int8_t *labels_dev, void *stream);

/* Deterministic initialisation (uniform Glorot, SplitMix64 of (seed, index); zero biases). */
int qbx_mlp_init(float *params_dev, uint64_t seed, void *stream);

/* y[2*i..2*i+1] = network(x[4*i..4*i+3]) for i < n. */
int qbx_mlp_forward(const float *params_dev, const float *x_dev, int64_t n, float *y_dev, void *stream);

/* Gradient of L = 1/(2n) sum_i |network(x_i) - target_i|^2 into grad[0..QBX_MLP_NPARAMS), and L into
 * grad[QBX_MLP_NPARAMS] (grad holds QBX_MLP_NPARAMS + 1 floats).  Summed in a fixed order. */
int qbx_mlp_loss_grad(const float *params_dev, const float *x_dev, const float *target_dev, int64_t n,
                      float *grad_dev, void *stream);

/* `steps` full-batch Adam steps (beta 0.9/0.999, eps 1e-8, step counter starting at first_step >= 1)
 * on params with moment buffers adam_m, adam_v (QBX_MLP_NPARAMS floats each, caller-owned, zero
 * before the first step).  If loss_host is given it receives the loss after the last step. */
int qbx_mlp_train(float *params_dev, float *adam_m_dev, float *adam_v_dev, const float *x_dev,
                  const float *target_dev, int64_t n, int steps, int first_step, float lr, float *loss_host,
                  void *stream);

/*
 * Orders from predictions pred[2*c..2*c+1] (input center order): p_qbx of center c =
 * clamp(ceil(pred0 + margin_q), q_lo, q_hi); the order of box b's local expansion = the largest
 * clamp(ceil(pred1 + margin_p), p_lo, p_hi) over the centers of b's subtree (a parent's local is
 * translated to its children), p_hi for boxes holding point targets (tgt_ctr[t] = -1; they read
 * the box local directly) and their ancestors, p_default where no center or point target
 * contributes.  tgt_ctr may be NULL (no point targets).  Outputs are the per-center and per-box
 * arrays qbx_eval_opts takes.
 */
int qbx_orders_from_mlp(const qbx_tree *tree, const qbx_lists *lists, const float *pred_dev,
                        const int32_t *tgt_ctr_dev, float margin_q, float margin_p, int q_lo, int q_hi, int p_lo,
                        int p_hi, int p_default, int8_t *p_qbx_per_ctr_dev, int8_t *p_fmm_per_box_dev, void *stream);

/*
 * Judge and fallback of learned orders.  `result` is an evaluation with the per-center and per-box
 * orders below, `judge` the fixed-order evaluation (p_qbx = q_fix, p_fmm = p_fix) of the same
 * problem, both over all n_tgt targets.  For every target t with |result[t] - judge[t]| > tol
 * (absolute; NaN counts) the call raises, in place, the QBX order of its center to q_fix and the
 * local-expansion order of the box owning that center (or the point target) and of every box above
 * it to p_fix.  Those centers then see the fixed-order box expansions; repeat with a new result until
 * *n_raised_host is 0.  *n_raised_host receives the number of targets that missed.
 *   p_qbx_per_ctr_dev [n_ctr], p_fmm_per_box_dev [n_boxes]: the orders, updated in place.
 * Errors: QBX_ERR_INVALID_ARG, QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_orders_fallback(const qbx_tree *tree, const double *result_dev, const double *judge_dev,
                        const int32_t *tgt_ctr_dev, double tol, int q_fix, int p_fix, int8_t *p_qbx_per_ctr_dev,
                        int8_t *p_fmm_per_box_dev, int64_t *n_raised_host, void *stream);

/* ------------------------------------------------------------------------------------------
 * Batched problems and captured evaluations.  Not steps of the paper's method: they run
 * Algorithm 4 on many independent surfaces at once (each evaluation stage is one launch over
 * every surface) and replay an evaluation as one CUDA graph, as repeated evaluation inside an
 * iterative solver (Section 6.2 solves with GMRES) does with fixed geometry.
 * ------------------------------------------------------------------------------------------ */

/*
 * Concatenates n_problems built trees and their lists into one forest.  Problem i's boxes,
 * sources, centers and targets follow those of problems 0..i-1 (offsets from
 * qbx_forest_offsets); its list entries are shifted accordingly, so no list crosses problems.
 * The forest is a tree handle for qbx_eval, qbx_eval_order_sweep, the learned-order calls,
 * qbx_graph_create and qbx_tree_export, with input arrays concatenated in problem order (point
 * arrays as (3, total) structure of arrays) and tgt_ctr holding forest center indices (a
 * problem's own center index plus its center offset, or -1).  qbx_build_lists rejects a forest.
 *   trees_host, lists_host: host arrays of n_problems >= 1 handles, lists_host[i] built from
 *   trees_host[i]; they are copied (the originals may be freed afterwards).
 *   forest_out, lists_out: receive new handles (free the lists before the forest).
 * Errors: QBX_ERR_INVALID_ARG (mismatched handles, a forest inside a forest, more than 2^31 - 1
 * boxes, particles or list entries), QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_build_forest(int n_problems, const qbx_tree *const *trees_host, const qbx_lists *const *lists_host,
                     qbx_tree **forest_out, qbx_lists **lists_out, void *stream);

/* Number of problems of a forest (1 for a tree). */
int qbx_forest_problems(const qbx_tree *forest, int *n_problems_host);

/* Offsets of each problem: offsets_host[k * (n + 1) + i], k = 0 boxes, 1 sources, 2 centers,
 * 3 targets, i = 0..n (entry n is the total); 4 (n + 1) int64 values. */
int qbx_forest_offsets(const qbx_tree *forest, int64_t *offsets_host);

/*
 * Captures one qbx_eval with exactly these arguments into a CUDA graph.  Runs one evaluation
 * eagerly first (argument checks, workspace and plans), then captures a second on `stream`
 * (which must not be the legacy default stream) and instantiates it; pot holds a valid result
 * on return.  qbx_graph_launch replays it on any stream: the pointers are baked in, so callers
 * change densities by overwriting the same device arrays.  Profiling is off inside the graph.
 * Errors: as qbx_eval, QBX_ERR_INVALID_ARG for a NULL stream.
 */
int qbx_graph_create(const qbx_tree *tree, const qbx_lists *lists, const double *src_w_dev, const double *sigma_dev,
                     const double *mu_dev, const double *src_n_dev, const int32_t *tgt_ctr_dev,
                     const qbx_eval_opts *opts, double *pot_dev, qbx_graph **out, void *stream);
int qbx_graph_launch(qbx_graph *graph, void *stream);
void qbx_graph_free(qbx_graph *graph);

/*
 * Launch-shape hints of the tensor-core translation kernels (QBX_M2L_3XTF32), used by later
 * evaluations on these lists (the plans are rebuilt when a hint changes); results do not depend
 * on them beyond FP32 rounding of the chunked accumulation.  0 selects the library default.
 *   m2l_kchunk:     K columns per pipeline stage of the List 2 products: 0, 16 or 32.
 *   m2qbxl_kchunk:  cap on the K columns per stage of the List 3 far products: 0 or a multiple of
 *                   8 in [16, 128]; raised to what one harmonic degree needs and lowered to what
 *                   shared memory holds.
 * Errors: QBX_ERR_INVALID_ARG.
 */
int qbx_lists_set_tiles(qbx_lists *lists, int m2l_kchunk, int m2qbxl_kchunk);

/*
 * Failure handling of the tensor-core pipelines (QBX_M2L_3XTF32; not a step of the paper's method).
 * Every wait of those kernels is bounded; when one gives up, the kernel waits (again bounded) for the
 * bulk copies and tensor-core products it has already issued, frees its tensor memory and returns, and
 * qbx_eval returns QBX_ERR_TIMEOUT.  The next evaluation starts clean.
 *   limit_cycles:  SM clock cycles a pipeline wait may take before it gives up; 0 restores the
 *                  default (4e9 cycles, about two seconds).  The drain waits after a failure keep the
 *                  default.
 *   probe_step:    -1 (normal operation), or a pipeline step k >= 0 at which the issuing thread of every
 *                  block of both tensor-core kernels also waits on a barrier that nothing ever arrives
 *                  on, so that the wait runs out after limit_cycles and the failure path above runs
 *                  (a test of that path; blocks with fewer than k + 1 steps are not affected).
 * Settings apply to later evaluations on these lists.  Errors: QBX_ERR_INVALID_ARG.
 */
int qbx_lists_set_wait(qbx_lists *lists, long long limit_cycles, int probe_step);

/*
 * Per-stage timing (tracing aid; not a step of the paper's method).  While enabled,
 * every qbx_eval on these lists records CUDA events on its stream around each of
 * QBX_NSTAGES stages: 0 input preparation, 1 P2M + M2M (Stage 2), 2 List 2 M2L
 * (Stage 4), 3 List 4 far P2L (Stage 6b), 4 L2L (Stage 7), 5 List 3 far M2QBXL
 * products in the mixed-precision modes (empty in QBX_FP64), 6 the QBX center kernel (Stages
 * 3, 5(a), 6(a), 8: direct P2QBXL and L2QBXL, and List 3 far M2QBXL in QBX_FP64), 7 the reduction
 * of the mixed List 3 far products into the QBX locals (empty in QBX_FP64), 8 QBX targets
 * (Stage 9), 9 point targets (Stage 9).  qbx_profile_read waits for the last profiled evaluation
 * and writes the stage durations in milliseconds to stage_ms_host.  Profiling must be disabled
 * while the stream is being captured into a graph.
 */
#define QBX_NSTAGES 10
int qbx_profile(qbx_lists *lists, int enable);
int qbx_profile_read(const qbx_lists *lists, double *stage_ms_host);

/*
 * qbx_eval without device allocation, for callers that cannot call cudaMalloc when they
 * evaluate: real-time loops whose device-memory budget is fixed up front, or hosts whose
 * allocator owns the whole device and forbids allocations from elsewhere.  The paper has no
 * counterpart; it is an interface choice.  Same arguments and the same stages and formulas as
 * qbx_eval, in QBX_FP64 only; the box-expansion passes run the library's per-warp kernels rather
 * than qbx_eval's, so the two agree to rounding (about 1e-15 relative), not bit for bit.
 *   Scratch: one file-scope device array of QBX_NOALLOC_SCRATCH_BYTES (48 MiB) inside the
 *   library, held by every GPU that loads the library until the process exits.  The problem
 *   must fit: roughly 18.4 MB of tables + 11.1 kB per box + 16 ntri(Qb) bytes per center (Qb =
 *   4, 8, 12 or 16, the smallest >= p_qbx) + 33 bytes per source, each buffer rounded up to 256
 *   bytes; e.g. 1,200 boxes and 20,000 centers at p_qbx <= 8.  A larger problem returns
 *   QBX_ERR_INVALID_ARG with the exact byte counts in qbx_last_error().
 *   No call allocates: no cudaMalloc, cudaFree or allocating library routine.
 *   The first call on each device looks up the array's device address (with that device
 *   current) and keeps it; make that first call before any stream capture.  The address stays
 *   valid while the device's primary context lives: after a device reset, reload the library.
 *   All calls share the array and it keeps the last call's contents: every call rewrites its
 *   tables and zeroes its accumulators before use, but calls whose GPU work overlaps in time on
 *   one device (issued on different streams, or from different host threads) race on it and
 *   give wrong results.
 * Errors: as qbx_eval; QBX_ERR_INVALID_ARG also for a precision other than QBX_FP64.
 */
#define QBX_NOALLOC_SCRATCH_BYTES (48u << 20)
int qbx_eval_noalloc(const qbx_tree *tree, const qbx_lists *lists, const double *src_w_dev, const double *sigma_dev,
                     const double *mu_dev, const double *src_n_dev, const int32_t *tgt_ctr_dev,
                     const qbx_eval_opts *opts, double *pot_dev, void *stream);

/* Message describing the last error on the calling thread ("" if none). */
const char *qbx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QBX_H */
