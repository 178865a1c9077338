// Octree with target confinement (Algorithm 4 Stage 1; Section 5.2.1-5.2.2), built
// level by level on the GPU.  Every decision is order independent (integer atomics
// only count or OR), every floating-point predicate is written with explicitly
// rounded operations, and boxes are numbered by (level, Morton code), so the tree is
// reproducible bit for bit.  Also holds the device-wide scan and the stable radix
// sort used across the library.
#include <algorithm>
#include <cmath>

#include "qbx_internal.cuh"

namespace qbx {

// ---------------------------------------------------------------- exclusive scan

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;

// Single-block chunked scan: out[i] = base + sum(in[0..i)), *total = base + sum(in).
// in and out may alias.
__global__ void k_scan(const int *in, int *out, int64_t n, int base, int *total)
{
    __shared__ int wsum[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = base;
    __syncthreads();
    for (int64_t off = 0; off < n; off += (int64_t)SCAN_THREADS * SCAN_ITEMS) {
        int v[SCAN_ITEMS];
        int local = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            int64_t idx = off + (int64_t)t * SCAN_ITEMS + i;
            v[i] = idx < n ? in[idx] : 0;
            local += v[i];
        }
        int incl = local;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
            int si = s;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, si, d);
                if (lane >= d) si += y;
            }
            wsum[lane] = si - s;  // exclusive warp offsets
        }
        __syncthreads();
        int run = carry + wsum[w] + incl - local;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            int64_t idx = off + (int64_t)t * SCAN_ITEMS + i;
            if (idx < n) out[idx] = run;
            run += v[i];
        }
        __syncthreads();
        if (t == SCAN_THREADS - 1) carry = run;
        __syncthreads();
    }
    if (t == 0 && total) *total = carry;
}

void exclusive_scan(const int *in, int *out, int64_t n, int base_offset, int *total_dev, cudaStream_t st)
{
    k_scan<<<1, SCAN_THREADS, 0, st>>>(in, out, n, base_offset, total_dev);
    QBX_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- stable LSD radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void k_rs_hist(const int *keys, int64_t n, int shift, int *hist, int nblk)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = t0 + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: within a tile, elements keep their index order (rounds in order,
// warps in order, lanes in order); tiles keep their order through the digit-major scan.
__global__ void k_rs_scatter(const int *kin, const int *vin, int *kout, int *vout, int64_t n, int shift,
                             const int *offs, int nblk)
{
    __shared__ int wcnt[RS_THREADS / 32][256];
    __shared__ int base[256];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    base[t] = offs[(int64_t)t * nblk + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int i = t; i < (RS_THREADS / 32) * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        int64_t i = t0 + r * RS_THREADS + t;
        bool valid = i < n;
        int key = valid ? kin[i] : 0;
        int d = (key >> shift) & 255;
        unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 256 + lane);
        int rk = __popc(peers & lt);
        if (valid && rk == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {
            int run = base[t];
            for (int ww = 0; ww < RS_THREADS / 32; ++ww) {
                int c = wcnt[ww][t];
                wcnt[ww][t] = run;
                run += c;
            }
            base[t] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = wcnt[w][d] + rk;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

void sort_pairs_by_key(int *keys, int *vals, int64_t n, int key_bits, cudaStream_t st)
{
    if (n <= 1) return;
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    int *k2 = dalloc<int>(n), *v2 = dalloc<int>(n), *hist = dalloc<int>((int64_t)256 * nblk);
    int *ka = keys, *va = vals, *kb = k2, *vb = v2;
    int passes = std::max(1, (key_bits + 7) / 8);
    try {
        for (int p = 0; p < passes; ++p) {
            k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(ka, n, 8 * p, hist, nblk);
            QBX_LAUNCH_CHECK();
            exclusive_scan(hist, hist, (int64_t)256 * nblk, 0, nullptr, st);
            k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, 8 * p, hist, nblk);
            QBX_LAUNCH_CHECK();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        if (ka != keys) {
            QBX_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(int), cudaMemcpyDeviceToDevice, st));
            QBX_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(int), cudaMemcpyDeviceToDevice, st));
        }
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(k2); dfree(v2); dfree(hist);
        throw;
    }
    dfree(k2); dfree(v2); dfree(hist);
}

// ---------------------------------------------------------------- geometry predicates

// Center fits inside the TCR B2(sqrt(3) h (1 + t_f), c) of a box with center c and
// l-infinity radius h: |x - c|_2 + r <= (sqrt(3) h)(1 + t_f), evaluated in this order.
__device__ __forceinline__ bool fits_tcr(double x, double y, double z, double r, double cx, double cy, double cz,
                                         double h, double tf)
{
    double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy), dz = __dsub_rn(z, cz);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double lhs = __dadd_rn(__dsqrt_rn(d2), r);
    double rhs = __dmul_rn(__dmul_rn(__dsqrt_rn(3.0), h), __dadd_rn(1.0, tf));
    return lhs <= rhs;
}

// The box-shaped TCR of the two-dimensional method (the l-infinity columns of Table
// l2-comparison): the cube of l-infinity radius h (1 + t_f) about c holds the ball,
// |x - c|_inf + r <= h (1 + t_f).
__device__ __forceinline__ bool fits_tcr_linf(double x, double y, double z, double r, double cx, double cy,
                                              double cz, double h, double tf)
{
    double m = fmax(fmax(fabs(__dsub_rn(x, cx)), fabs(__dsub_rn(y, cy))), fabs(__dsub_rn(z, cz)));
    return __dadd_rn(m, r) <= __dmul_rn(h, __dadd_rn(1.0, tf));
}

struct Particles {
    const double *xyz[3];
    const double *cr;
    int64_t n[3];
    int *owner[3];
    __device__ __forceinline__ void locate(int64_t g, int &k, int64_t &i) const
    {
        if (g < n[0]) { k = 0; i = g; }
        else if (g < n[0] + n[1]) { k = 1; i = g - n[0]; }
        else { k = 2; i = g - n[0] - n[1]; }
    }
};

// ---------------------------------------------------------------- root box

__global__ void k_bbox(Particles P, double *part, int *bad)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int64_t N = P.n[0] + P.n[1] + P.n[2];
    int badl = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        int k;
        int64_t i;
        P.locate(g, k, i);
        double r = (k == KCTR) ? P.cr[i] : 0.0;
        if (k == KCTR && !(r > 0.0 && r < INFINITY)) badl = 1;
        for (int d = 0; d < 3; ++d) {
            double x = P.xyz[k][d * P.n[k] + i];
            if (!isfinite(x)) badl = 1;
            if (k == KCTR) {
                lo[d] = fmin(lo[d], __dsub_rn(x, r));
                hi[d] = fmax(hi[d], __dadd_rn(x, r));
            } else {
                lo[d] = fmin(lo[d], x);
                hi[d] = fmax(hi[d], x);
            }
        }
    }
    if (badl) atomicOr(bad, 1);
    __shared__ double s[6][256];
    for (int d = 0; d < 3; ++d) { s[d][threadIdx.x] = lo[d]; s[3 + d][threadIdx.x] = hi[d]; }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 6; ++d) part[blockIdx.x * 6 + d] = s[d][0];
}

// Root: midpoint of the bounding box rounded to a multiple of R/8, R the smallest power
// of two >= 1.25 x the largest half extent.
__global__ void k_root(const double *part, int nparts, double *rootp, double *cen, double *hw, int *level,
                       int64_t *ic, int *parent, int *child)
{
    if (threadIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nparts; ++b)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[b * 6 + d]);
            hi[d] = fmax(hi[d], part[b * 6 + 3 + d]);
        }
    double mid[3], h = 0.0;
    for (int d = 0; d < 3; ++d) {
        mid[d] = __dmul_rn(0.5, __dadd_rn(lo[d], hi[d]));
        h = fmax(h, __dmul_rn(0.5, __dsub_rn(hi[d], lo[d])));
    }
    double R = 1.0;
    // h is finite here unless the input was (the host rejects that case after this kernel);
    // both loops are bounded by the exponent range of a double either way
    if (h > 0.0 && h < 1e300) {
        for (int it = 0; it < 2200 && R < __dmul_rn(1.25, h); ++it) R = __dmul_rn(R, 2.0);
        for (int it = 0; it < 2200 && __dmul_rn(0.5, R) >= __dmul_rn(1.25, h); ++it) R = __dmul_rn(R, 0.5);
    }
    double q8 = __ddiv_rn(R, 8.0);
    for (int d = 0; d < 3; ++d) {
        double c = __dmul_rn(rint(__ddiv_rn(mid[d], q8)), q8);
        rootp[d] = c;
        cen[d] = c;
        ic[d] = 0;
    }
    rootp[3] = R;
    hw[0] = R;
    level[0] = 0;
    parent[0] = -1;
    for (int o = 0; o < 8; ++o) child[o] = -1;
}

// ---------------------------------------------------------------- level loop kernels

__global__ void k_count(Particles P, int b0, int b1, int *cnt)
{
    int64_t N = P.n[0] + P.n[1] + P.n[2];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        int k;
        int64_t i;
        P.locate(g, k, i);
        int o = P.owner[k][i];
        if (o >= b0 && o < b1) atomicAdd(&cnt[o - b0], 1);
    }
}

// Destination octant of every particle owned by a splitting box at this level, or -1.
// A box splits when it owns more than n_max particles or, in a rebuild for level
// restriction, when its box of the previous tree (oid) had children or was marked (oforce).
__global__ void k_dest(Particles P, int b0, int b1, const int *cnt, int n_max, bool can_split, const double *cen,
                       const double *hw, double tf, bool linf, const int *oid, const unsigned char *oforce,
                       signed char *dest, int *cmask)
{
    int64_t N = P.n[0] + P.n[1] + P.n[2];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        int k;
        int64_t i;
        P.locate(g, k, i);
        signed char dd = -1;
        int o = P.owner[k][i];
        if (can_split && o >= b0 && o < b1 &&
            (cnt[o - b0] > n_max || (oid && oid[o] >= 0 && oforce[oid[o]]))) {
            double x = P.xyz[k][i], y = P.xyz[k][P.n[k] + i], z = P.xyz[k][2 * P.n[k] + i];
            double cx = cen[3 * o], cy = cen[3 * o + 1], cz = cen[3 * o + 2];
            int oc = (x >= cx ? 1 : 0) | (y >= cy ? 2 : 0) | (z >= cz ? 4 : 0);
            bool ok = true;
            if (k == KCTR) {
                double hc = __dmul_rn(0.5, hw[o]);
                double ccx = __dadd_rn(cx, (oc & 1) ? hc : -hc);
                double ccy = __dadd_rn(cy, (oc & 2) ? hc : -hc);
                double ccz = __dadd_rn(cz, (oc & 4) ? hc : -hc);
                ok = linf ? fits_tcr_linf(x, y, z, P.cr[i], ccx, ccy, ccz, hc, tf)
                          : fits_tcr(x, y, z, P.cr[i], ccx, ccy, ccz, hc, tf);
            }
            if (ok) {
                dd = (signed char)oc;
                atomicOr(&cmask[o - b0], 1 << oc);
            }
        }
        dest[g] = dd;
    }
}

__global__ void k_popc(const int *cmask, const int *cnt, int nbl, int n_max, bool at_max_depth, int *nch,
                       int *overfull)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbl) return;
    nch[b] = __popc(cmask[b]);
    if (at_max_depth && cnt[b] > n_max) atomicAdd(overfull, 1);
}

// Children of the splitting boxes of one level, in (parent, octant) = Morton order.  In a
// rebuild, oid maps each new box to the same box of the previous tree (ochild), or -1.
__global__ void k_children(int b0, int nbl, int first_new, int lev, const int *cmask, const int *choff, int *level,
                           int64_t *ic, double *cen, double *hw, int *parent, int *child, const int *ochild,
                           int *oid)
{
    int bb = blockIdx.x * blockDim.x + threadIdx.x;
    if (bb >= nbl) return;
    int b = b0 + bb;
    int m = cmask[bb];
    int nxt = first_new + choff[bb];
    double hc = __dmul_rn(0.5, hw[b]);
    for (int oc = 0; oc < 8; ++oc) {
        if (!((m >> oc) & 1)) continue;
        int c = nxt++;
        level[c] = lev + 1;
        for (int d = 0; d < 3; ++d) {
            int bit = (oc >> d) & 1;
            ic[3 * c + d] = 2 * ic[3 * b + d] + bit;
            cen[3 * c + d] = __dadd_rn(cen[3 * b + d], bit ? hc : -hc);
        }
        hw[c] = hc;
        parent[c] = b;
        for (int o = 0; o < 8; ++o) child[8 * c + o] = -1;
        child[8 * b + oc] = c;
        if (oid) oid[c] = oid[b] >= 0 ? ochild[8 * oid[b] + oc] : -1;
    }
}

// Level restriction (Remark "Effect of level-restriction on List 3 complexity", Section
// 5.3): one round's marks on the current tree.  force[b] = 1 for boxes with children (they
// stay split) and for every leaf that touches a leaf two or more levels finer (closed cubes
// meet; distinct leaves never overlap, so that is adjacency), found by a depth-first walk
// from the root over the boxes whose closed cube meets b's, exact in integer units of the
// finest level lf.  nviol counts the marked leaves; a stack overflow sets *err.
constexpr int RESTRICT_STACK = 8 * 64;

__global__ void k_restrict_marks(int nb, int lf, int max_depth, const int *level, const int64_t *ic,
                                 const int *child, unsigned char *force, int *nviol, int *err)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    bool has_child = false;
    for (int o = 0; o < 8; ++o) has_child |= child[8 * b + o] >= 0;
    force[b] = has_child ? 1 : 0;
    const int lb = level[b];
    if (has_child || lb + 2 > lf || lb >= max_depth) return;
    int64_t lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = ic[3 * b + d] << (lf - lb);
        hi[d] = (ic[3 * b + d] + 1) << (lf - lb);
    }
    int stack[RESTRICT_STACK];
    int n = 0;
    stack[n++] = 0;
    bool viol = false;
    while (n && !viol) {
        int c = stack[--n];
        if (c == b) continue;
        const int sh = lf - level[c];
        bool meets = true;
        for (int d = 0; d < 3; ++d) {
            int64_t l = ic[3 * c + d] << sh, h = (ic[3 * c + d] + 1) << sh;
            if (l > hi[d] || lo[d] > h) meets = false;
        }
        if (!meets) continue;
        bool leaf = true;
        for (int o = 0; o < 8; ++o) {
            int ch = child[8 * c + o];
            if (ch < 0) continue;
            leaf = false;
            if (n >= RESTRICT_STACK) {
                atomicOr(err, 1);
                return;
            }
            stack[n++] = ch;
        }
        if (leaf && level[c] >= lb + 2) viol = true;
    }
    if (viol) {
        force[b] = 1;
        atomicAdd(nviol, 1);
    }
}

__global__ void k_move(Particles P, const signed char *dest, const int *child)
{
    int64_t N = P.n[0] + P.n[1] + P.n[2];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        if (dest[g] < 0) continue;
        int k;
        int64_t i;
        P.locate(g, k, i);
        int o = P.owner[k][i];
        P.owner[k][i] = child[8 * o + dest[g]];
    }
}

// ---------------------------------------------------------------- finishing kernels

__global__ void k_iota(int *v, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int)i;
}

__global__ void k_count_owned(const int *owner, int64_t n, int *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[owner[i]], 1);
}

__global__ void k_accum_parent(int b0, int b1, const int *parent, int *a, int *b)
{
    int x = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= b1) return;
    int p = parent[x];
    if (p >= 0) {
        atomicAdd(&a[p], a[x]);
        atomicAdd(&b[p], b[x]);
    }
}

__global__ void k_gather_xyz(const double *in, const int *perm, int64_t n, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = perm[i];
    out[i] = in[j];
    out[n + i] = in[n + j];
    out[2 * n + i] = in[2 * n + j];
}

__global__ void k_gather_ctr(const double *r, const int *perm, const int *owner, int64_t n, double *rout,
                             int *box_out, int *rank)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = perm[i];
    if (rout) rout[i] = r[j];
    box_out[i] = owner[j];
    if (rank) rank[j] = (int)i;
}

// ---------------------------------------------------------------- driver

static void grow(qbx_tree *T, int64_t &cap, int64_t need, cudaStream_t st)
{
    if (need <= cap) return;
    int64_t nc = std::max(need, 2 * cap);
    auto re = [&](auto *&p, int per) {
        using E = std::remove_reference_t<decltype(*p)>;
        E *q = dalloc<E>(nc * per);
        if (p) QBX_CUDA_TRY(cudaMemcpyAsync(q, p, cap * per * sizeof(E), cudaMemcpyDeviceToDevice, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        dfree(p);
        p = q;
    };
    re(T->level, 1);
    re(T->ic, 3);
    re(T->cen, 3);
    re(T->hw, 1);
    re(T->parent, 1);
    re(T->child, 8);
    cap = nc;
}

void build_tree(qbx_tree *T, const double *sxyz, const double *cxyz, const double *cr, const double *txyz,
                cudaStream_t st)
{
    const int64_t ns = T->np[0], nc = T->np[1], nt = T->np[2], N = ns + nc + nt;
    Particles P;
    P.xyz[0] = sxyz;
    P.xyz[1] = cxyz;
    P.xyz[2] = txyz;
    P.cr = cr;
    for (int k = 0; k < 3; ++k) {
        P.n[k] = T->np[k];
        T->owner[k] = dalloc<int>(T->np[k]);
        QBX_CUDA_TRY(cudaMemsetAsync(T->owner[k], 0, std::max<int64_t>(T->np[k], 1) * sizeof(int), st));
        P.owner[k] = T->owner[k];
    }
    int64_t cap = 0;
    grow(T, cap, std::max<int64_t>(1024, N / 4), st);

    const int nbb = 256;
    double *part = dalloc<double>(6 * nbb), *rootp = dalloc<double>(4);
    int *flags = dalloc<int>(4);  // [0] bad input, [1] overfull, [2] scan total
    double rootp_h[4];
    signed char *dest = dalloc<signed char>(N);
    int *cnt = nullptr, *cmask = nullptr, *nch = nullptr, *oid = nullptr;
    try {
        QBX_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
        k_bbox<<<nbb, 256, 0, st>>>(P, part, flags);
        QBX_LAUNCH_CHECK();
        k_root<<<1, 32, 0, st>>>(part, nbb, rootp, T->cen, T->hw, T->level, T->ic, T->parent, T->child);
        QBX_LAUNCH_CHECK();
        int flags_h[4];
        QBX_CUDA_TRY(cudaMemcpyAsync(flags_h, flags, sizeof(flags_h), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaMemcpyAsync(rootp_h, rootp, sizeof(rootp_h), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        if (flags_h[0]) throw Error{QBX_ERR_INVALID_ARG, "non-finite coordinate or center radius <= 0"};
        for (int d = 0; d < 3; ++d) T->root_c[d] = rootp_h[d];
        T->root_h = rootp_h[3];

        const bool linf = (T->flags & QBX_TREE_LINF_TCR) != 0;
        const unsigned gp = std::min<unsigned>(nblocks(N, 256), 152 * 16);
        int64_t lvcap = 0, oid_cap = 0;
        // Stage 1 level by level from the root.  With ochild/oforce (a rebuild for level
        // restriction), oid tracks each new box's box in the previous tree, whose split is kept
        // (it had children) or made (it was marked).
        auto run_levels = [&](const int *ochild, const unsigned char *oforce) {
            int b0 = 0, b1 = 1, lev = 0;
            T->level_start.assign(1, 0);
            if (ochild) {
                if (oid_cap < cap) {
                    dfree(oid);
                    oid = dalloc<int>(cap);
                    oid_cap = cap;
                }
                QBX_CUDA_TRY(cudaMemsetAsync(oid, 0, sizeof(int), st));  // the root is the root
            }
            QBX_CUDA_TRY(cudaMemsetAsync(flags + 1, 0, sizeof(int), st));
            for (;; ++lev) {
                T->level_start.push_back(b1);
                int nbl = b1 - b0;
                if (nbl > lvcap) {
                    dfree(cnt); dfree(cmask); dfree(nch);
                    cnt = cmask = nch = nullptr;
                    lvcap = std::max<int64_t>(nbl, 2 * lvcap);
                    cnt = dalloc<int>(lvcap);
                    cmask = dalloc<int>(lvcap);
                    nch = dalloc<int>(lvcap);
                }
                QBX_CUDA_TRY(cudaMemsetAsync(cnt, 0, nbl * sizeof(int), st));
                QBX_CUDA_TRY(cudaMemsetAsync(cmask, 0, nbl * sizeof(int), st));
                bool can_split = lev < T->max_depth;
                k_count<<<gp, 256, 0, st>>>(P, b0, b1, cnt);
                QBX_LAUNCH_CHECK();
                k_dest<<<gp, 256, 0, st>>>(P, b0, b1, cnt, T->n_max, can_split, T->cen, T->hw, T->tf, linf,
                                           ochild ? oid : nullptr, oforce, dest, cmask);
                QBX_LAUNCH_CHECK();
                k_popc<<<nblocks(nbl, 256), 256, 0, st>>>(cmask, cnt, nbl, T->n_max, !can_split, nch, flags + 1);
                QBX_LAUNCH_CHECK();
                exclusive_scan(nch, nch, nbl, 0, flags + 2, st);
                int total = 0;
                QBX_CUDA_TRY(cudaMemcpyAsync(&total, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
                QBX_CUDA_TRY(cudaStreamSynchronize(st));
                if (total == 0) break;
                grow(T, cap, (int64_t)b1 + total, st);
                if (ochild && oid_cap < cap) {  // keep the old-box map as long as the box arrays
                    int *o2 = dalloc<int>(cap);
                    QBX_CUDA_TRY(cudaMemcpyAsync(o2, oid, b1 * sizeof(int), cudaMemcpyDeviceToDevice, st));
                    QBX_CUDA_TRY(cudaStreamSynchronize(st));
                    dfree(oid);
                    oid = o2;
                    oid_cap = cap;
                }
                k_children<<<nblocks(nbl, 128), 128, 0, st>>>(b0, nbl, b1, lev, cmask, nch, T->level, T->ic, T->cen,
                                                              T->hw, T->parent, T->child, ochild,
                                                              ochild ? oid : nullptr);
                QBX_LAUNCH_CHECK();
                k_move<<<gp, 256, 0, st>>>(P, dest, T->child);
                QBX_LAUNCH_CHECK();
                b0 = b1;
                b1 += total;
            }
            T->nb = b1;
            T->nlev = lev + 1;
            T->level_start.resize(T->nlev + 1);
            T->level_start[T->nlev] = b1;
        };
        run_levels(nullptr, nullptr);

        // Level restriction (Remark "Effect of level-restriction on List 3 complexity", Section
        // 5.3), in rounds: mark every leaf touching a leaf two or more levels finer, then rebuild
        // with those leaves split as well (a rebuild equals splitting them in place: the boxes
        // above are unchanged, and a split leaf owned at most n_max particles, so its children
        // do not split on count); stop when a round marks nothing or splits nothing.
        if (T->flags & QBX_TREE_LEVEL_RESTRICT) {
            // every round that changes the tree makes new leaves; a few rounds per level are plenty
            const int max_rounds = 4 * (T->max_depth + 1);
            bool settled = false;
            for (int round = 0; round < max_rounds && !settled; ++round) {
                const int nb0 = (int)T->nb;
                unsigned char *force = dalloc<unsigned char>(nb0);
                QBX_CUDA_TRY(cudaMemsetAsync(flags + 2, 0, 2 * sizeof(int), st));
                k_restrict_marks<<<nblocks(nb0, 128), 128, 0, st>>>(nb0, (int)T->nlev - 1, T->max_depth, T->level,
                                                                     T->ic, T->child, force, flags + 2, flags + 3);
                int marks[2] = {0, 0};
                try {
                    QBX_LAUNCH_CHECK();
                    QBX_CUDA_TRY(cudaMemcpyAsync(marks, flags + 2, sizeof(marks), cudaMemcpyDeviceToHost, st));
                    QBX_CUDA_TRY(cudaStreamSynchronize(st));
                    if (marks[1]) throw Error{QBX_ERR_CUDA, "level restriction: search stack overflow"};
                } catch (...) {
                    dfree(force);
                    throw;
                }
                if (marks[0] == 0) {
                    dfree(force);
                    settled = true;
                    break;
                }
                // keep the previous tree's child array and marks; rebuild into fresh box arrays
                int *ochild = T->child;
                T->child = nullptr;
                dfree(T->level); dfree(T->ic); dfree(T->cen); dfree(T->hw); dfree(T->parent);
                T->level = T->parent = nullptr;
                T->ic = nullptr;
                T->cen = T->hw = nullptr;
                cap = 0;
                try {
                    grow(T, cap, std::max<int64_t>(1024, nb0), st);
                    k_root<<<1, 32, 0, st>>>(part, nbb, rootp, T->cen, T->hw, T->level, T->ic, T->parent, T->child);
                    QBX_LAUNCH_CHECK();
                    for (int k = 0; k < 3; ++k)
                        QBX_CUDA_TRY(cudaMemsetAsync(T->owner[k], 0, std::max<int64_t>(T->np[k], 1) * sizeof(int), st));
                    run_levels(ochild, force);
                } catch (...) {
                    dfree(ochild);
                    dfree(force);
                    throw;
                }
                dfree(ochild);
                dfree(force);
                if (T->nb == nb0) settled = true;  // the marked leaves could not move a particle
            }
            if (!settled) throw Error{QBX_ERR_CUDA, "level restriction did not settle"};
        }
        int ov = 0;
        QBX_CUDA_TRY(cudaMemcpyAsync(&ov, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        T->n_overfull = ov;

        // subtree counts
        T->nsrc_sub = dalloc<int>(T->nb);
        T->ntgt_sub = dalloc<int>(T->nb);
        QBX_CUDA_TRY(cudaMemsetAsync(T->nsrc_sub, 0, T->nb * sizeof(int), st));
        QBX_CUDA_TRY(cudaMemsetAsync(T->ntgt_sub, 0, T->nb * sizeof(int), st));
        if (ns) k_count_owned<<<nblocks(ns, 256), 256, 0, st>>>(T->owner[0], ns, T->nsrc_sub);
        if (nc) k_count_owned<<<nblocks(nc, 256), 256, 0, st>>>(T->owner[1], nc, T->ntgt_sub);
        if (nt) k_count_owned<<<nblocks(nt, 256), 256, 0, st>>>(T->owner[2], nt, T->ntgt_sub);
        QBX_LAUNCH_CHECK();
        for (int l = (int)T->nlev - 1; l >= 1; --l) {
            int a = T->level_start[l], b = T->level_start[l + 1];
            k_accum_parent<<<nblocks(b - a, 256), 256, 0, st>>>(a, b, T->parent, T->nsrc_sub, T->ntgt_sub);
            QBX_LAUNCH_CHECK();
        }

        // particles grouped by owning box, input order within a box
        int key_bits = 1;
        while ((int64_t(1) << key_bits) < T->nb) ++key_bits;
        for (int k = 0; k < 3; ++k) {
            int64_t n = T->np[k];
            T->perm[k] = dalloc<int>(n);
            T->own_start[k] = dalloc<int>(T->nb + 1);
            QBX_CUDA_TRY(cudaMemsetAsync(T->own_start[k], 0, (T->nb + 1) * sizeof(int), st));
            if (n == 0) continue;
            int *keys = dalloc<int>(n);
            QBX_CUDA_TRY(cudaMemcpyAsync(keys, T->owner[k], n * sizeof(int), cudaMemcpyDeviceToDevice, st));
            k_iota<<<nblocks(n, 256), 256, 0, st>>>(T->perm[k], n);
            QBX_LAUNCH_CHECK();
            try {
                sort_pairs_by_key(keys, T->perm[k], n, key_bits, st);
            } catch (...) {
                dfree(keys);
                throw;
            }
            dfree(keys);
            k_count_owned<<<nblocks(n, 256), 256, 0, st>>>(T->owner[k], n, T->own_start[k]);
            QBX_LAUNCH_CHECK();
            exclusive_scan(T->own_start[k], T->own_start[k], T->nb + 1, 0, nullptr, st);
        }
        T->sxyz = dalloc<double>(3 * ns);
        T->cxyz = dalloc<double>(3 * nc);
        T->cr = dalloc<double>(nc);
        T->txyz = dalloc<double>(3 * nt);
        T->ctr_box = dalloc<int>(nc);
        T->tgt_box = dalloc<int>(nt);
        T->ctr_rank = dalloc<int>(nc);
        if (ns) k_gather_xyz<<<nblocks(ns, 256), 256, 0, st>>>(sxyz, T->perm[0], ns, T->sxyz);
        if (nc) {
            k_gather_xyz<<<nblocks(nc, 256), 256, 0, st>>>(cxyz, T->perm[1], nc, T->cxyz);
            k_gather_ctr<<<nblocks(nc, 256), 256, 0, st>>>(cr, T->perm[1], T->owner[1], nc, T->cr, T->ctr_box,
                                                           T->ctr_rank);
        }
        if (nt) {
            k_gather_xyz<<<nblocks(nt, 256), 256, 0, st>>>(txyz, T->perm[2], nt, T->txyz);
            k_gather_ctr<<<nblocks(nt, 256), 256, 0, st>>>(nullptr, T->perm[2], T->owner[2], nt, nullptr, T->tgt_box,
                                                           nullptr);
        }
        QBX_LAUNCH_CHECK();
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(part); dfree(rootp); dfree(flags); dfree(dest); dfree(cnt); dfree(cmask); dfree(nch); dfree(oid);
        throw;
    }
    dfree(part); dfree(rootp); dfree(flags); dfree(dest); dfree(cnt); dfree(cmask); dfree(nch); dfree(oid);
}

}  // namespace qbx
