// Interaction lists of Section 5.2.3-5.2.4 on the GPU: List 1 (U), List 2 (V),
// List 3 close/far (W-close, W-far), List 4 close/far (X-close, X-far).
// One thread enumerates one box's candidates twice (count, then fill); each box's
// entries are then sorted.  Same-level lookups binary-search the level's boxes,
// which are stored in Morton order.  Readings: k-colleagues exclude the box itself,
// descendants are strict, adjacency is exact integer arithmetic, boxes whose subtree
// holds no source are left out of every list.
#include <climits>

#include "qbx_internal.cuh"

namespace qbx {

constexpr int DFS_STACK = 512;

struct TreeView {
    int nb, nlev, lf;  // lf = finest level
    const int *level_start;
    const int *level;
    const int64_t *ic;
    const double *cen, *hw;
    const int *parent, *child, *nsrc_sub, *ntgt_sub;
    const int *own_start_src, *own_start_ctr, *own_start_tgt;
    double tf;
    bool linf;  // the l-infinity TCR (QBX_TREE_LINF_TCR)
    int *err;

    __device__ bool leaf(int b) const
    {
        for (int o = 0; o < 8; ++o)
            if (child[8 * b + o] >= 0) return false;
        return true;
    }
    __device__ bool source_box(int b) const { return own_start_src[b + 1] > own_start_src[b]; }
    __device__ bool target_box(int b) const
    {
        return own_start_ctr[b + 1] > own_start_ctr[b] || own_start_tgt[b + 1] > own_start_tgt[b];
    }
    __device__ bool adjacent(int a, int b) const
    {
        int sa = lf - level[a], sb = lf - level[b];
        bool closed = true, open = true;
        for (int d = 0; d < 3; ++d) {
            int64_t la = ic[3 * a + d] << sa, ha = (ic[3 * a + d] + 1) << sa;
            int64_t lb = ic[3 * b + d] << sb, hb = (ic[3 * b + d] + 1) << sb;
            if (la > hb || lb > ha) closed = false;
            if (!(la < hb && lb < ha)) open = false;
        }
        return closed && !open;
    }
    __device__ bool colleague(int a, int b, int k) const
    {
        if (a == b || level[a] != level[b]) return false;
        for (int d = 0; d < 3; ++d) {
            int64_t di = ic[3 * a + d] - ic[3 * b + d];
            if (di < -k || di > k) return false;
        }
        return true;
    }
    // a adequately separated from TCR(b) (l2, signed distance to the TCR boundary >= 3|a|);
    // with the l-infinity TCR, the l-infinity distance from the center of a to the boundary of
    // the cube of radius |b|(1 + t_f), signed, is >= 3|a|
    __device__ bool sep_a_tcrb(int a, int b) const
    {
        if (linf) {
            double m = 0.0;
            for (int d = 0; d < 3; ++d) m = fmax(m, fabs(__dsub_rn(cen[3 * a + d], cen[3 * b + d])));
            return __dsub_rn(m, __dmul_rn(hw[b], __dadd_rn(1.0, tf))) >= __dmul_rn(3.0, hw[a]);
        }
        double dx = __dsub_rn(cen[3 * a], cen[3 * b]), dy = __dsub_rn(cen[3 * a + 1], cen[3 * b + 1]),
               dz = __dsub_rn(cen[3 * a + 2], cen[3 * b + 2]);
        double dist = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        double tcr = __dmul_rn(__dmul_rn(__dsqrt_rn(3.0), hw[b]), __dadd_rn(1.0, tf));
        return __dsub_rn(dist, tcr) >= __dmul_rn(3.0, hw[a]);
    }
    // TCR(a) adequately separated from b (l-infinity, signed distance to b's boundary >= 3|a|(1+t_f))
    __device__ bool sep_tcra_b(int a, int b) const
    {
        double m = 0.0;
        for (int d = 0; d < 3; ++d) m = fmax(m, fabs(__dsub_rn(cen[3 * a + d], cen[3 * b + d])));
        return __dsub_rn(m, hw[b]) >= __dmul_rn(__dmul_rn(3.0, hw[a]), __dadd_rn(1.0, tf));
    }
    __device__ static bool less_msb(uint64_t a, uint64_t b) { return a < b && a < (a ^ b); }
    __device__ static bool morton_less(const int64_t *a, const int64_t *b)
    {
        int dim = 2;
        uint64_t best = (uint64_t)(a[2] ^ b[2]);
        for (int d = 1; d >= 0; --d) {
            uint64_t x = (uint64_t)(a[d] ^ b[d]);
            if (less_msb(best, x)) { dim = d; best = x; }
        }
        return a[dim] < b[dim];
    }
    __device__ int find(int lev, const int64_t q[3]) const
    {
        if (lev < 0 || lev >= nlev) return -1;
        int64_t n = (int64_t)1 << lev;
        for (int d = 0; d < 3; ++d)
            if (q[d] < 0 || q[d] >= n) return -1;
        int lo = level_start[lev], hi = level_start[lev + 1];
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (morton_less(&ic[3 * mid], q)) lo = mid + 1;
            else hi = mid;
        }
        if (lo < level_start[lev + 1] && ic[3 * lo] == q[0] && ic[3 * lo + 1] == q[1] && ic[3 * lo + 2] == q[2])
            return lo;
        return -1;
    }
};

struct Emit {
    int *out;
    int n;
    __device__ void operator()(int d)
    {
        if (out) out[n] = d;
        ++n;
    }
};

// Calls f(d) for every same-level box d with |ic(d) - ic(b)|_inf <= k, d != b.
template <class F>
__device__ void for_colleagues(const TreeView &T, int b, int k, F &&f)
{
    int lev = T.level[b];
    for (int dz = -k; dz <= k; ++dz)
        for (int dy = -k; dy <= k; ++dy)
            for (int dx = -k; dx <= k; ++dx) {
                if (!dx && !dy && !dz) continue;
                int64_t q[3] = {T.ic[3 * b] + dx, T.ic[3 * b + 1] + dy, T.ic[3 * b + 2] + dz};
                int d = T.find(lev, q);
                if (d >= 0) f(d);
            }
}

struct Stack {
    int v[DFS_STACK];
    int n = 0;
    __device__ bool push(int x, int *err)
    {
        if (n >= DFS_STACK) {
            atomicOr(err, 1);
            return false;
        }
        v[n++] = x;
        return true;
    }
};

// ---------------------------------------------------------------- List 1

__device__ void list_u(const TreeView &T, int b, Emit &e)
{
    Stack s;
    // leaf descendants of b, and b itself if it is a leaf
    s.push(b, T.err);
    while (s.n) {
        int d = s.v[--s.n];
        if (T.nsrc_sub[d] == 0) continue;
        if (T.leaf(d)) { e(d); continue; }
        for (int o = 0; o < 8; ++o)
            if (T.child[8 * d + o] >= 0) s.push(T.child[8 * d + o], T.err);
    }
    // adjacent leaves at b's level or finer: below adjacent same-level boxes
    for_colleagues(T, b, 1, [&](int w) {
        s.n = 0;
        s.push(w, T.err);
        while (s.n) {
            int d = s.v[--s.n];
            if (T.nsrc_sub[d] == 0 || !T.adjacent(d, b)) continue;
            if (T.leaf(d)) { e(d); continue; }
            for (int o = 0; o < 8; ++o)
                if (T.child[8 * d + o] >= 0) s.push(T.child[8 * d + o], T.err);
        }
    });
    // coarser adjacent leaves: same-level neighbors of each ancestor
    for (int a = T.parent[b]; a >= 0; a = T.parent[a])
        for_colleagues(T, a, 1, [&](int d) {
            if (T.leaf(d) && T.source_box(d) && T.adjacent(d, b)) e(d);
        });
}

// ---------------------------------------------------------------- List 2

__device__ void list_v(const TreeView &T, int b, Emit &e)
{
    int pb = T.parent[b];
    if (pb < 0) return;
    auto visit = [&](int p) {
        for (int o = 0; o < 8; ++o) {
            int d = T.child[8 * p + o];
            if (d < 0 || d == b || T.nsrc_sub[d] == 0) continue;
            if (T.colleague(d, b, 2)) continue;
            e(d);
        }
    };
    visit(pb);
    for_colleagues(T, pb, 2, visit);
}

// ---------------------------------------------------------------- List 3 close / far

__device__ void list_w(const TreeView &T, int b, Emit &ec, Emit &ef)
{
    Stack s, s2;
    for_colleagues(T, b, 2, [&](int w) {
        s.n = 0;
        for (int o = 0; o < 8; ++o)
            if (T.child[8 * w + o] >= 0) s.push(T.child[8 * w + o], T.err);
        while (s.n) {
            int d = s.v[--s.n];
            if (T.nsrc_sub[d] == 0) continue;
            if (T.adjacent(d, b)) {
                for (int o = 0; o < 8; ++o)
                    if (T.child[8 * d + o] >= 0) s.push(T.child[8 * d + o], T.err);
                continue;
            }
            // d is in List 3 of b: split it into close leaves and far boxes
            s2.n = 0;
            s2.push(d, T.err);
            while (s2.n) {
                int x = s2.v[--s2.n];
                if (T.nsrc_sub[x] == 0) continue;
                if (T.sep_a_tcrb(x, b)) { ef(x); continue; }
                if (T.leaf(x)) { ec(x); continue; }
                for (int o = 0; o < 8; ++o)
                    if (T.child[8 * x + o] >= 0) s2.push(T.child[8 * x + o], T.err);
            }
        }
    });
}

// ---------------------------------------------------------------- List 4 (then close / far)

template <class F>
__device__ void list_x(const TreeView &T, int b, F &&f)
{
    for_colleagues(T, b, 2, [&](int d) {
        if (T.leaf(d) && T.source_box(d) && !T.adjacent(d, b)) f(d);
    });
    int pb = T.parent[b];
    if (pb < 0) return;
    for (int a = pb; a >= 0; a = T.parent[a])
        for_colleagues(T, a, 1, [&](int d) {
            if (T.leaf(d) && T.source_box(d) && T.adjacent(d, pb) && !T.adjacent(d, b)) f(d);
        });
}

// ---------------------------------------------------------------- kernels

__global__ void k_lists_uvw(TreeView T, int which, const int *start_u, const int *start_v, const int *start_wc,
                            const int *start_wf, int *cnt_u, int *cnt_v, int *cnt_wc, int *cnt_wf, int *idx_u,
                            int *idx_v, int *idx_wc, int *idx_wf)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= T.nb) return;
    bool fill = start_u != nullptr;
    if (T.ntgt_sub[b] == 0) {
        if (!fill) { cnt_u[b] = cnt_v[b] = cnt_wc[b] = cnt_wf[b] = 0; }
        return;
    }
    bool tgt = T.target_box(b);
    if (which == 0) {
        Emit eu{fill ? idx_u + start_u[b] : nullptr, 0};
        if (tgt) list_u(T, b, eu);
        if (!fill) cnt_u[b] = eu.n;
    } else if (which == 1) {
        Emit ev{fill ? idx_v + start_v[b] : nullptr, 0};
        list_v(T, b, ev);
        if (!fill) cnt_v[b] = ev.n;
    } else {
        Emit ec{fill ? idx_wc + start_wc[b] : nullptr, 0}, ef{fill ? idx_wf + start_wf[b] : nullptr, 0};
        if (tgt) list_w(T, b, ec, ef);
        if (!fill) { cnt_wc[b] = ec.n; cnt_wf[b] = ef.n; }
    }
}

// List 4 close/far for the boxes of one level; needs X-close of the parents.
__global__ void k_lists_x(TreeView T, int b0, int b1, const int *start_xc, const int *idx_xc_parent_src,
                          const int *start_xc_fill, const int *start_xf_fill, int *cnt_xc, int *cnt_xf, int *idx_xc,
                          int *idx_xf)
{
    int b = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= b1) return;
    bool fill = start_xc_fill != nullptr;
    int nc = 0, nf = 0;
    if (T.ntgt_sub[b] > 0) {
        auto put = [&](int d) {
            if (T.sep_tcra_b(b, d)) {
                if (fill) idx_xf[start_xf_fill[b] + nf] = d;
                ++nf;
            } else {
                if (fill) idx_xc[start_xc_fill[b] + nc] = d;
                ++nc;
            }
        };
        list_x(T, b, put);
        int pb = T.parent[b];
        if (pb >= 0)
            for (int i = start_xc[pb]; i < start_xc[pb + 1]; ++i) put(idx_xc_parent_src[i]);
    }
    if (!fill) { cnt_xc[b] = nc; cnt_xf[b] = nf; }
}

// Sort each box's entries ascending: warp bitonic sort in shared memory, heapsort beyond 1024.
__global__ void k_sort_segments(const int *start, int *idx, int nb)
{
    __shared__ int sh[4][1024];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int b = blockIdx.x * 4 + w;
    if (b >= nb) return;
    int lo = start[b], n = start[b + 1] - lo;
    if (n <= 1) return;
    int *a = idx + lo;
    if (n <= 1024) {
        int N = 1;
        while (N < n) N <<= 1;
        for (int i = lane; i < N; i += 32) sh[w][i] = i < n ? a[i] : INT_MAX;
        __syncwarp();
        for (int k = 2; k <= N; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < N; i += 32) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int x = sh[w][i], y = sh[w][ixj];
                        bool up = (i & k) == 0;
                        if ((x > y) == up) { sh[w][i] = y; sh[w][ixj] = x; }
                    }
                }
                __syncwarp();
            }
        for (int i = lane; i < n; i += 32) a[i] = sh[w][i];
        return;
    }
    if (lane != 0) return;
    auto sift = [&](int root, int end) {
        while (2 * root + 1 < end) {
            int c = 2 * root + 1;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[root] >= a[c]) return;
            int t = a[root]; a[root] = a[c]; a[c] = t;
            root = c;
        }
    };
    for (int i = n / 2 - 1; i >= 0; --i) sift(i, n);
    for (int end = n - 1; end > 0; --end) {
        int t = a[0]; a[0] = a[end]; a[end] = t;
        sift(0, end);
    }
}

// ---------------------------------------------------------------- driver

static int read_int(const int *p, cudaStream_t st)
{
    int v = 0;
    QBX_CUDA_TRY(cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, st));
    QBX_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

void build_lists(qbx_lists *L, cudaStream_t st)
{
    const qbx_tree *Tr = L->tree;
    const int nb = (int)Tr->nb;
    int *ls = dalloc<int>(Tr->nlev + 1), *err = dalloc<int>(1), *tot = dalloc<int>(1);
    int *cnt[NLIST] = {};
    try {
        QBX_CUDA_TRY(cudaMemcpyAsync(ls, Tr->level_start.data(), (Tr->nlev + 1) * sizeof(int),
                                     cudaMemcpyHostToDevice, st));
        QBX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        TreeView T{nb, (int)Tr->nlev, (int)Tr->nlev - 1, ls, Tr->level, Tr->ic, Tr->cen, Tr->hw, Tr->parent,
                   Tr->child, Tr->nsrc_sub, Tr->ntgt_sub, Tr->own_start[KSRC], Tr->own_start[KCTR],
                   Tr->own_start[KTGT], Tr->tf, (Tr->flags & QBX_TREE_LINF_TCR) != 0, err};
        for (int l = 0; l < NLIST; ++l) {
            cnt[l] = dalloc<int>(nb + 1);
            L->start[l] = dalloc<int>(nb + 1);
            QBX_CUDA_TRY(cudaMemsetAsync(cnt[l], 0, (nb + 1) * sizeof(int), st));
        }
        const int TPB = 64;
        // U, V, W: count, scan, fill
        for (int which = 0; which < 3; ++which) {
            k_lists_uvw<<<nblocks(nb, TPB), TPB, 0, st>>>(T, which, nullptr, nullptr, nullptr, nullptr, cnt[LU],
                                                          cnt[LV], cnt[LWC], cnt[LWF], nullptr, nullptr, nullptr,
                                                          nullptr);
            QBX_LAUNCH_CHECK();
        }
        int e0 = read_int(err, st);
        if (e0) throw Error{QBX_ERR_CUDA, "list build: traversal stack overflow"};
        for (int l : {LU, LV, LWC, LWF}) {
            exclusive_scan(cnt[l], L->start[l], nb + 1, 0, tot, st);
            L->nnz[l] = read_int(tot, st);
            L->idx[l] = dalloc<int>(L->nnz[l]);
        }
        QBX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        for (int which = 0; which < 3; ++which) {
            k_lists_uvw<<<nblocks(nb, TPB), TPB, 0, st>>>(T, which, L->start[LU], L->start[LV], L->start[LWC],
                                                          L->start[LWF], nullptr, nullptr, nullptr, nullptr,
                                                          L->idx[LU], L->idx[LV], L->idx[LWC], L->idx[LWF]);
            QBX_LAUNCH_CHECK();
        }
        // X: level by level (X-close of the parent feeds the child)
        int base_c = 0, base_f = 0;
        int64_t cap_c = std::max<int64_t>(1024, nb), cap_f = std::max<int64_t>(1024, nb);
        L->idx[LXC] = dalloc<int>(cap_c);
        L->idx[LXF] = dalloc<int>(cap_f);
        auto grow = [&](int *&p, int64_t &cap, int64_t need) {
            if (need <= cap) return;
            int64_t nc = std::max(need, 2 * cap);
            int *q = dalloc<int>(nc);
            QBX_CUDA_TRY(cudaMemcpyAsync(q, p, cap * sizeof(int), cudaMemcpyDeviceToDevice, st));
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            dfree(p);
            p = q;
            cap = nc;
        };
        for (int lev = 0; lev < Tr->nlev; ++lev) {
            int b0 = Tr->level_start[lev], b1 = Tr->level_start[lev + 1], n = b1 - b0;
            k_lists_x<<<nblocks(n, TPB), TPB, 0, st>>>(T, b0, b1, L->start[LXC], L->idx[LXC], nullptr, nullptr,
                                                       cnt[LXC], cnt[LXF], nullptr, nullptr);
            QBX_LAUNCH_CHECK();
            exclusive_scan(cnt[LXC] + b0, L->start[LXC] + b0, n, base_c, tot, st);
            int tc = read_int(tot, st);
            exclusive_scan(cnt[LXF] + b0, L->start[LXF] + b0, n, base_f, tot, st);
            int tf = read_int(tot, st);
            // start[b1] closes this level (the next level's scan rewrites it with the same value)
            QBX_CUDA_TRY(cudaMemcpyAsync(L->start[LXC] + b1, &tc, sizeof(int), cudaMemcpyHostToDevice, st));
            QBX_CUDA_TRY(cudaMemcpyAsync(L->start[LXF] + b1, &tf, sizeof(int), cudaMemcpyHostToDevice, st));
            grow(L->idx[LXC], cap_c, tc);
            grow(L->idx[LXF], cap_f, tf);
            k_lists_x<<<nblocks(n, TPB), TPB, 0, st>>>(T, b0, b1, L->start[LXC], L->idx[LXC], L->start[LXC],
                                                       L->start[LXF], nullptr, nullptr, L->idx[LXC], L->idx[LXF]);
            QBX_LAUNCH_CHECK();
            // children read their parent's X-close entries in ascending order, as the oracle does
            k_sort_segments<<<nblocks(n, 4), 128, 0, st>>>(L->start[LXC] + b0, L->idx[LXC], n);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            base_c = tc;
            base_f = tf;
        }
        L->nnz[LXC] = base_c;
        L->nnz[LXF] = base_f;
        int e1 = read_int(err, st);
        if (e1) throw Error{QBX_ERR_CUDA, "list build: traversal stack overflow"};
        for (int l = 0; l < NLIST; ++l) {
            k_sort_segments<<<nblocks(nb, 4), 128, 0, st>>>(L->start[l], L->idx[l], nb);
            QBX_LAUNCH_CHECK();
        }
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(ls); dfree(err); dfree(tot);
        for (int l = 0; l < NLIST; ++l) dfree(cnt[l]);
        throw;
    }
    dfree(ls); dfree(err); dfree(tot);
    for (int l = 0; l < NLIST; ++l) dfree(cnt[l]);
}

// ---------------------------------------------------------------- interaction counts

struct ListSet {
    const int *start[NLIST], *idx[NLIST];
};

// Per-list interaction counts (the factors of Table ilist-operation-counts), one thread per target
// box b, with n_t = the QBX centers b owns and n_s = the sources a source box owns (its subtree for
// List 4 far): U, W-close, X-close add n_s n_t per entry, V adds 1, W-far adds n_t, X-far adds n_s.
// Integer sums, so the result does not depend on the order of the atomic adds.
__global__ void k_list_counts(int nb, const int *own_src, const int *own_ctr, const int *nsrc_sub, ListSet ls,
                              unsigned long long *out)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long acc[NLIST] = {0, 0, 0, 0, 0, 0};
    if (b < nb) {
        const unsigned long long nt = (unsigned long long)(own_ctr[b + 1] - own_ctr[b]);
        for (int l = 0; l < NLIST; ++l)
            for (int e = ls.start[l][b]; e < ls.start[l][b + 1]; ++e) {
                const int d = ls.idx[l][e];
                if (l == LV) acc[l] += 1ull;
                else if (l == LWF) acc[l] += nt;
                else if (l == LXF) acc[l] += (unsigned long long)nsrc_sub[d];
                else acc[l] += (unsigned long long)(own_src[d + 1] - own_src[d]) * nt;
            }
    }
    for (int l = 0; l < NLIST; ++l) {
        unsigned long long v = acc[l];
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(out + l, v);
    }
}

void list_counts(const qbx_lists *L, int64_t *counts_host, cudaStream_t st)
{
    const qbx_tree *T = L->tree;
    unsigned long long *d = dalloc<unsigned long long>(NLIST);
    try {
        QBX_CUDA_TRY(cudaMemsetAsync(d, 0, NLIST * sizeof(unsigned long long), st));
        ListSet ls;
        for (int l = 0; l < NLIST; ++l) {
            ls.start[l] = L->start[l];
            ls.idx[l] = L->idx[l];
        }
        if (T->nb > 0) {
            k_list_counts<<<nblocks(T->nb, 128), 128, 0, st>>>((int)T->nb, T->own_start[KSRC], T->own_start[KCTR],
                                                              T->nsrc_sub, ls, d);
            QBX_LAUNCH_CHECK();
        }
        unsigned long long h[NLIST];
        QBX_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        for (int l = 0; l < NLIST; ++l) counts_host[l] = (int64_t)h[l];
    } catch (...) {
        dfree(d);
        throw;
    }
    dfree(d);
}

}  // namespace qbx
