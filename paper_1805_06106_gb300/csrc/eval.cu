// GIGAQBX FMM evaluation (Algorithm 4, Stages 2-9), FP64.
//
// Expansion forms (all coefficients m >= 0, tri layout, conjugate symmetry for m < 0):
//   multipole of box b (center c, half width h):  Mu_n^m = sum_s q R_n^m((s-c)/h) (+ dipole)
//       phi(t) = 1/(4 pi h) sum_{n,m} Mu_n^m conj S_n^m((t-c)/h)
//   local of box b:                               phi(t) = 1/(4 pi) sum_{n,m} B_n^m R_n^m((c-t)/h)
//   QBX local at center c with radius rho:        phi(t) = 1/(4 pi) sum_{k,l} A_k^l R_k^l((c-t)/rho)
// which give the operators
//   P2M   Mu_n^m += q R_n^m(x) + (d/h).grad R_n^m(x),                 x = (s-c)/h
//   P2L   B_n^m  += conj[q S_n^m(x) - (d/h).grad S_n^m(x)] / h,      x = (c-s)/h   (also P2QBXL with h -> rho)
//   M2M   Mu'_n^m = sum_{k,l} 2^-k Mu_k^l R_{n-k}^{m-l}((c_child - c_par)/h_par)
//   M2L   B_k^l  += 1/h sum_{n,m} Mu_n^m conj S_{n+k}^{m+l}((c_b - c_d)/h)
//   M2QBXL A_k^l += 1/h_d (rho/h_d)^k sum_{n,m} Mu_n^m conj S_{n+k}^{m+l}((c - c_d)/h_d)
//   L2L   B'_k^l  = 2^-k sum_{n>=k,m} B_n^m R_{n-k}^{m-l}((c_par - c_child)/h_par)
//   L2QBXL A_k^l += (rho/h)^k sum_{n>=k,m} B_n^m R_{n-k}^{m-l}((c_b - c)/h)
// (Section 4.1 operators, written in these harmonics.)
#include <algorithm>
#include <cmath>

#include <math_constants.h>

#include "harmonics.cuh"
#include "df64.cuh"

namespace qbx {

constexpr double INV4PI = 0.079577471545947667884;  // 1 / (4 pi)

struct M2LPlan;
void free_m2l_plan(M2LPlan *p);
M2LPlan *m2l_plan_build(const qbx_tree *T, const qbx_lists *L, int P, int PMT, const double2 *stab, bool tc,
                        int kc_hint, cudaStream_t st);
void m2l_mixed_run(const qbx_tree *T, const qbx_lists *L, M2LPlan *pl, int PMT, const double2 *Mu, double2 *B,
                   const signed char *pb, int *err, cudaStream_t st);
int m2l_plan_order(const M2LPlan *p);
struct WfarPlan;
void free_wfar_plan(WfarPlan *p);
int wfar_plan_orders(const WfarPlan *p);
const int *wfar_empty_start(const WfarPlan *p);
WfarPlan *wfar_plan_build(const qbx_tree *T, const qbx_lists *L, int P, int Q, bool tc, int w_hint, cudaStream_t st);
void wfar_mixed_run(const qbx_tree *T, WfarPlan *pl, int PMT, const double2 *Mu, const signed char *pb, const float *cf,
                    int *err, long long wait_limit, int probe_step, cudaStream_t st);
void wfar_mixed_reduce(const qbx_tree *T, WfarPlan *pl, int QMS, const signed char *qc, double2 *A, cudaStream_t st);


}  // namespace qbx

struct qbx_workspace {
    int PM = -1, QM = -1;          // orders the buffers were sized for
    int64_t nb = 0, nc = 0, ns = 0;
    double2 *Mu = nullptr, *B = nullptr, *A = nullptr;
    double2 *m2l_tab = nullptr;    // 1331 offsets x ntri(2 PM): S_j^i(2 o)
    double2 *oct_tab = nullptr;    // 8 octants x ntri(PM): R_j^i(delta_o)
    double *sq = nullptr, *sd = nullptr;
    double *pd = nullptr;          // per target: the direct sources' part of its QBX expansion (k_qbx_direct)
    float *sf = nullptr, *cf = nullptr, *tf = nullptr;  // double-float copies of sources (+ densities), centers, targets
    float4 *Bf = nullptr;          // double-float copy of the box locals (k_l2qbxl)
    float4 *Muf = nullptr, *octf = nullptr;  // double-float copies of the multipoles and the octant table
    signed char *qc = nullptr, *pb = nullptr, *ps = nullptr;  // per-center QBX, per-box local and multipole orders
    int *flags = nullptr;
    std::vector<int> lvl_first;    // host copies of level ranges
    qbx::M2LPlan *m2l = nullptr;   // mixed-precision List 2 plan (built on first use)
    qbx::WfarPlan *wfar = nullptr; // mixed-precision List 3 far plan (built on first use)
    int wfar_key = -1;             // (orders, form, tile) the List 3 far plan was built for
    // point targets: (target, List 3 far box) pairs, listed on every evaluation
    int64_t pt_cap = -1;           // pairs if every target were a point target
    int *pt_cnt = nullptr, *pt_off = nullptr, *pt_total = nullptr, *pt_it = nullptr, *pt_box = nullptr;
    double *pt_part = nullptr;
    int m2l_key = -1;              // (order, form, tile) the List 2 plan was built for
};

namespace qbx {

void free_workspace(qbx_workspace *ws)
{
    if (!ws) return;
    dfree(ws->Mu); dfree(ws->B); dfree(ws->A); dfree(ws->m2l_tab); dfree(ws->oct_tab); dfree(ws->pd);
    dfree(ws->sf); dfree(ws->cf); dfree(ws->tf); dfree(ws->Bf); dfree(ws->Muf); dfree(ws->octf);
    dfree(ws->sq); dfree(ws->sd); dfree(ws->qc); dfree(ws->pb); dfree(ws->ps); dfree(ws->flags);
    free_m2l_plan(ws->m2l);
    free_wfar_plan(ws->wfar);
    dfree(ws->pt_cnt); dfree(ws->pt_off); dfree(ws->pt_total); dfree(ws->pt_it); dfree(ws->pt_box);
    dfree(ws->pt_part);
    delete ws;
}

// ---------------------------------------------------------------- setup kernels

__global__ void k_m2l_table(int pmax2, double2 *tab)
{
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= 1331) return;
    int ox = o % 11 - 5, oy = (o / 11) % 11 - 5, oz = o / 121 - 5;
    double2 *t = tab + (int64_t)o * ntri(pmax2);
    if (ox == 0 && oy == 0 && oz == 0) {
        for (int i = 0; i < ntri(pmax2); ++i) t[i] = make_double2(0.0, 0.0);
        return;
    }
    irregular_table(pmax2, 2.0 * ox, 2.0 * oy, 2.0 * oz, 1.0, 1.0, t);
}

// R_j^i(delta_o) with delta_o = (+-1/2, +-1/2, +-1/2), sign + where octant bit d is set
__global__ void k_oct_table(int p, double2 *tab)
{
    int o = threadIdx.x;
    if (o >= 8) return;
    regular_table(p, (o & 1) ? 0.5 : -0.5, (o & 2) ? 0.5 : -0.5, (o & 4) ? 0.5 : -0.5, tab + o * ntri(p));
}

// sorted charges q = w sigma and dipoles d = w mu n; flags[0] |= 1 on invalid input
__global__ void k_prep_src(const int *perm, int64_t ns, const double *w, const double *sigma, const double *mu,
                           const double *nrm, double *sq, double *sd, int *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int j = perm[i];
    double wj = w[j];
    bool bad = !(wj > 0.0 && isfinite(wj));
    double s = sigma ? sigma[j] : 0.0;
    if (!isfinite(s)) bad = true;
    sq[i] = wj * s;
    if (mu) {
        double m = mu[j];
        double nx = nrm[j], ny = nrm[ns + j], nz = nrm[2 * ns + j];
        if (!isfinite(m) || !isfinite(nx) || !isfinite(ny) || !isfinite(nz)) bad = true;
        double a = wj * m;
        sd[i] = a * nx;
        sd[ns + i] = a * ny;
        sd[2 * ns + i] = a * nz;
    }
    if (bad) atomicOr(flags, 1);
}

// Double-float copies (leading parts, then trailing parts) of n points stored as 3 x n FP64 (SoA),
// and of k further FP64 arrays of length n: out = [xh yh zh xl yl zl] then [vh vl] per extra array.
__global__ void k_to_df(int64_t n, const double *xyz, const double *v0, const double *v1, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const df a = df_from(xyz[d * n + i]);
        out[d * n + i] = a.h;
        out[(3 + d) * n + i] = a.l;
    }
    if (v0) {
        const df a = df_from(v0[i]);
        out[6 * n + i] = a.h;
        out[7 * n + i] = a.l;
    }
    if (v1) {  // three components (dipole vectors), after the charge
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const df a = df_from(v1[d * n + i]);
            out[(8 + d) * n + i] = a.h;
            out[(11 + d) * n + i] = a.l;
        }
    }
}

void prep_sources(const int *perm, int64_t ns, const double *w, const double *sigma, const double *mu,
                  const double *nrm, double *sq, double *sd, int *flags, cudaStream_t st)
{
    k_prep_src<<<nblocks(ns, 256), 256, 0, st>>>(perm, ns, w, sigma, mu, nrm, sq, sd, flags);
    QBX_LAUNCH_CHECK();
}

// qfix / pfix are the fixed orders, or the bounds of the per-center / per-box arrays
// qc: per-center QBX order; pb: per-box order of the local expansions a box receives; ps: order of
// the multipole expansions every box sends (the fixed bound p_fmm)
__global__ void k_prep_orders(const int *ctr_perm, int64_t nc, const signed char *qin, int qfix, int64_t nb,
                              const signed char *pin, int pfix, signed char *qc, signed char *pb, signed char *ps,
                              int *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) {
        int q = qin ? qin[ctr_perm[i]] : qfix;
        if (q < 0 || q > qfix) atomicOr(flags, 2);
        qc[i] = (signed char)min(max(q, 0), qfix);  // clamped so that no kernel indexes past its tables
    }
    if (i < nb) {
        int p = pin ? pin[i] : pfix;
        if (p < 0 || p > pfix) atomicOr(flags, 2);
        pb[i] = (signed char)min(max(p, 0), pfix);
        ps[i] = (signed char)pfix;
    }
}

__global__ void k_check_tgt(const int *tc, int64_t nt, int64_t nc, int *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int c = tc[i];
    if (c < -1 || c >= nc) atomicOr(flags, 4);
}

// ---------------------------------------------------------------- upward pass

// P2M (Stage 2): one warp per box, lane m computes column m of R_n^m for each source in turn.
// PM bounds the orders (registers, unrolled rows); ST is the coefficient stride of the workspace.
template <int PM, int ST = PM>
__global__ void k_p2m(int64_t nb, const int *own_start, const double *sxyz, int64_t ns, const double *sq,
                      const double *sd, const double *cen, const double *hw, const signed char *pb, double2 *Mu)
{
    int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int m = threadIdx.x & 31;
    if (b >= nb) return;
    int s0 = own_start[b], s1 = own_start[b + 1];
    if (s0 == s1) return;
    const int P = pb[b];
    double hinv = 1.0 / hw[b];
    double cx = cen[3 * b], cy = cen[3 * b + 1], cz = cen[3 * b + 2];
    double2 acc[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) acc[n] = make_double2(0.0, 0.0);
    const double fm = m ? 0.5 / m : 0.0;
    for (int s = s0; s < s1; ++s) {
        double x = (sxyz[s] - cx) * hinv, y = (sxyz[ns + s] - cy) * hinv, z = (sxyz[2 * ns + s] - cz) * hinv;
        double r2 = x * x + y * y + z * z;
        double q = sq[s];
        double2 dw = make_double2(0.0, 0.0), dwb = make_double2(0.0, 0.0);
        double dz = 0.0;
        if (sd) {
            double dx = sd[s] * hinv, dy = sd[ns + s] * hinv;
            dz = sd[2 * ns + s] * hinv;
            dw = make_double2(0.5 * dx, 0.5 * dy);
            dwb = make_double2(0.5 * dx, -0.5 * dy);
        }
        // diagonal R_m^m = w^m / (2^m m!): inclusive prefix product over the lanes of w / (2m)
        double2 diag = (m == 0) ? make_double2(1.0, 0.0) : make_double2(x * fm, y * fm);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            double2 o;
            o.x = __shfl_up_sync(0xffffffffu, diag.x, off);
            o.y = __shfl_up_sync(0xffffffffu, diag.y, off);
            if (m >= off) diag = cmul(o, diag);
        }
        double2 p2 = make_double2(0.0, 0.0), p1 = make_double2(0.0, 0.0);
#pragma unroll
        for (int n = 0; n <= PM; ++n) {
            double2 cur = make_double2(0.0, 0.0);
            if (n == m) cur = diag;
            else if (n > m) {
                double inv = 1.0 / ((double)(n + m) * (double)(n - m));
                cur = make_double2(((2 * n - 1) * z * p1.x - r2 * p2.x) * inv, ((2 * n - 1) * z * p1.y - r2 * p2.y) * inv);
            }
            // neighbor columns of the previous row: R_{n-1}^{m+1} and R_{n-1}^{m-1}
            double2 up, dn;
            up.x = __shfl_down_sync(0xffffffffu, p1.x, 1);
            up.y = __shfl_down_sync(0xffffffffu, p1.y, 1);
            dn.x = __shfl_up_sync(0xffffffffu, p1.x, 1);
            dn.y = __shfl_up_sync(0xffffffffu, p1.y, 1);
            if (m == 31) up = make_double2(0.0, 0.0);
            if (m == 0) dn = make_double2(-up.x, up.y);  // R^{-1} = -conj R^1
            if (n >= m && n <= P) {
                double2 v = cscale(cur, q);
                if (sd) {
                    double2 t1 = cmul(dwb, up), t2 = cmul(dw, dn);
                    v.x += -t1.x + t2.x + dz * p1.x;
                    v.y += -t1.y + t2.y + dz * p1.y;
                }
                acc[n] = cadd(acc[n], v);
            }
            p2 = p1;
            p1 = cur;
        }
    }
    if (m <= P) {
#pragma unroll
        for (int n = 0; n <= PM; ++n)
            if (n >= m && n <= P) Mu[(int64_t)b * ntri(ST) + tri(n, m)] = acc[n];
    }
}

// M2M (Stage 2, postorder by level): one warp per parent, lanes over output coefficients.
template <int PM>
__global__ void k_m2m(int b0, int b1, const int *lvl_boxes, const int *child, const int *nsrc_sub,
                      const signed char *pb, const double2 *oct, double2 *Mu)
{
    int b = b0 + blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (b >= b1) return;
    if (lvl_boxes) b = lvl_boxes[b];
    if (nsrc_sub[b] == 0) return;
    const int P = pb[b];
    bool any = false;
    for (int o = 0; o < 8; ++o) any |= child[8 * b + o] >= 0;
    if (!any) return;
    for (int out = lane; out < ntri(P); out += 32) {
        int n = 0;
        while (tri(n + 1, 0) <= out) ++n;
        int m = out - tri(n, 0);
        double2 acc = Mu[(int64_t)b * ntri(PM) + out];  // the box's own sources (none for non-leaves)
        for (int o = 0; o < 8; ++o) {
            int c = child[8 * b + o];
            if (c < 0 || nsrc_sub[c] == 0) continue;
            const int Pc = pb[c];
            const double2 *Mc = Mu + (int64_t)c * ntri(PM);
            // child center - parent center = -(parent - child); delta = (c_child - c_par)/h_par
            const double2 *R = oct + o * ntri(PM);
            double sk = 1.0;
            for (int k = 0; k <= n && k <= Pc; ++k, sk *= 0.5) {
                int j = n - k;
                int lmin = max(-k, m - j), lmax = min(k, m + j);
                for (int l = lmin; l <= lmax; ++l) {
                    double2 t = cmul(sym_get(Mc, k, l), sym_get(R, j, m - l));
                    acc.x += sk * t.x;
                    acc.y += sk * t.y;
                }
            }
        }
        Mu[(int64_t)b * ntri(PM) + out] = acc;
    }
}

// M2M with one block of 8 warps per parent: warp o translates child octant o (lanes over the
// outputs), the 8 contributions are added in octant order in shared memory, so the serial work per
// parent is that of one child (the coarse levels hold few parents).
template <int PM>
__global__ void __launch_bounds__(256) k_m2m8(int b0, int b1, const int *lvl_boxes, const int *child,
                                              const int *nsrc_sub, const signed char *pb, const double2 *oct,
                                              double2 *Mu)
{
    __shared__ double2 part[8][ntri(PM)];
    int b = b0 + blockIdx.x;
    if (b >= b1) return;
    if (lvl_boxes) b = lvl_boxes[b];
    if (nsrc_sub[b] == 0) return;
    const int o = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = pb[b];
    const int c = child[8 * b + o];
    const bool live = c >= 0 && nsrc_sub[c] > 0;
    for (int out = lane; out < ntri(P); out += 32) {
        double2 acc = make_double2(0.0, 0.0);
        if (live) {
            int n = 0;
            while (tri(n + 1, 0) <= out) ++n;
            const int m = out - tri(n, 0);
            const int Pc = pb[c];
            const double2 *Mc = Mu + (int64_t)c * ntri(PM);
            const double2 *R = oct + o * ntri(PM);
            double sk = 1.0;
            for (int k = 0; k <= n && k <= Pc; ++k, sk *= 0.5) {
                const int j = n - k;
                const int lmin = max(-k, m - j), lmax = min(k, m + j);
                double2 t = make_double2(0.0, 0.0);
                for (int l = lmin; l <= lmax; ++l) {
                    const double2 a = sym_get(Mc, k, l), r = sym_get(R, j, m - l);
                    t.x = fma(a.x, r.x, fma(-a.y, r.y, t.x));
                    t.y = fma(a.x, r.y, fma(a.y, r.x, t.y));
                }
                acc.x = fma(sk, t.x, acc.x);
                acc.y = fma(sk, t.y, acc.y);
            }
        }
        part[o][out] = acc;
    }
    __syncthreads();
    for (int out = threadIdx.x; out < ntri(P); out += blockDim.x) {
        double2 v = Mu[(int64_t)b * ntri(PM) + out];  // the box's own sources (none for non-leaves)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v.x += part[k][out].x;
            v.y += part[k][out].y;
        }
        Mu[(int64_t)b * ntri(PM) + out] = v;
    }
}

// ---------------------------------------------------------------- upward pass on double-floats

// Reciprocals of the regular recurrence's integer divisors as double-floats (leading, trailing):
// c_l2q_rinv[tri(n, m)] = 1/((n+m)(n-m)) for m < n, c_l2q_half[m] = 1/(2m).  Uniform indices across a
// warp, so constant memory broadcasts them.
__constant__ float2 c_l2q_rinv[ntri(PMAX)];
__constant__ float2 c_l2q_half[PMAX + 1];

static float2 split_f2(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

void set_l2q_tables(cudaStream_t st)
{
    static float2 rinv[ntri(PMAX)], half[PMAX + 1];
    for (int n = 0; n <= PMAX; ++n)
        for (int m = 0; m <= n; ++m)
            rinv[tri(n, m)] = m < n ? split_f2(1.0 / ((double)(n + m) * (double)(n - m))) : make_float2(0.f, 0.f);
    half[0] = make_float2(0.f, 0.f);
    for (int m = 1; m <= PMAX; ++m) half[m] = split_f2(1.0 / (2.0 * m));
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_l2q_rinv, rinv, sizeof(rinv), 0, cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_l2q_half, half, sizeof(half), 0, cudaMemcpyHostToDevice, st));
}

__device__ __forceinline__ df df_shfl_up(df v, int off)
{
    return df{__shfl_up_sync(0xffffffffu, v.h, off), __shfl_up_sync(0xffffffffu, v.l, off)};
}
__device__ __forceinline__ df df_shfl_down(df v, int off)
{
    return df{__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off)};
}


__device__ __forceinline__ float4 df2_pack(df re, df im) { return make_float4(re.h, re.l, im.h, im.l); }

// double2 array -> double-float copy (re.h, re.l, im.h, im.l)
__global__ void k_c2df(int64_t n, const double2 *a, float4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = df2_pack(df_from(a[i].x), df_from(a[i].y));
}

// value at (n, m) for any m from a double-float table holding m >= 0: X_n^{-m} = (-1)^m conj X_n^m
__device__ __forceinline__ void df_sym_get(const float4 *tab, int n, int m, df &re, df &im)
{
    const float4 v = tab[tri(n, m < 0 ? -m : m)];
    re = df{v.x, v.y};
    im = df{v.z, v.w};
    if (m < 0) {
        if (m & 1) re = df_neg(re);
        else im = df_neg(im);
    }
}

// P2M (Stage 2) on double-floats: the structure of k_p2m (one warp per box, lane m carrying column m of
// R_n^m((s - c_b)/h) for each source in turn, the diagonal by a prefix product over the lanes), the
// arithmetic in double-float.  Writes the FP64 multipole and its double-float copy.
template <int PM, int ST>
__global__ void k_p2m_df(int64_t nb, const int *own_start, int64_t ns, const float *sf, int dip, const double *cen,
                         const double *hw, const signed char *pb, double2 *Mu, float4 *Muf)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int m = threadIdx.x & 31;
    if (b >= nb) return;
    const int s0 = own_start[b], s1 = own_start[b + 1];
    if (s0 == s1) return;
    const int P = pb[b];
    const float hinv = (float)(1.0 / hw[b]);  // a power of two: exact
    const df cx = df_from(cen[3 * b]), cy = df_from(cen[3 * b + 1]), cz = df_from(cen[3 * b + 2]);
    dacc ar[PM + 1], ai[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) ar[n] = ai[n] = dacc{0.f, 0.f};
    const df fm = m ? df_from(0.5 / m) : df{0.f, 0.f};
    for (int s = s0; s < s1; ++s) {
        const df x = df_mul_f(df_sub(df{sf[s], sf[3 * ns + s]}, cx), hinv),
                 y = df_mul_f(df_sub(df{sf[ns + s], sf[4 * ns + s]}, cy), hinv),
                 z = df_mul_f(df_sub(df{sf[2 * ns + s], sf[5 * ns + s]}, cz), hinv);
        const df r2 = df_add(df_add(df_sqr(x), df_sqr(y)), df_sqr(z));
        const df q{sf[6 * ns + s], sf[7 * ns + s]};
        df dwx{0.f, 0.f}, dwy{0.f, 0.f}, dz{0.f, 0.f};  // d/2 = (dwx, dwy), dz, scaled by 1/h
        if (dip) {
            dwx = df_mul_f(df{sf[8 * ns + s], sf[11 * ns + s]}, 0.5f * hinv);
            dwy = df_mul_f(df{sf[9 * ns + s], sf[12 * ns + s]}, 0.5f * hinv);
            dz = df_mul_f(df{sf[10 * ns + s], sf[13 * ns + s]}, hinv);
        }
        // diagonal R_m^m = w^m / (2^m m!): inclusive prefix product over the lanes of w / (2m)
        df gr = m == 0 ? df{1.f, 0.f} : df_mul(x, fm), gi = m == 0 ? df{0.f, 0.f} : df_mul(y, fm);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const df orr = df_shfl_up(gr, off), oi = df_shfl_up(gi, off);
            if (m >= off) {
                const df nr = df_sub(df_mul(orr, gr), df_mul(oi, gi));
                gi = df_add(df_mul(orr, gi), df_mul(oi, gr));
                gr = nr;
            }
        }
        df p2r{0.f, 0.f}, p2i{0.f, 0.f}, p1r{0.f, 0.f}, p1i{0.f, 0.f};
#pragma unroll
        for (int n = 0; n <= PM; ++n) {
            df cr{0.f, 0.f}, ci{0.f, 0.f};
            if (n == m) {
                cr = gr;
                ci = gi;
            } else if (n > m) {
                const float2 iv = c_l2q_rinv[tri(n, m)];
                const df inv{iv.x, iv.y}, c1 = df_mul_f(z, (float)(2 * n - 1));
                cr = df_mul(df_sub(df_mul(c1, p1r), df_mul(r2, p2r)), inv);
                ci = df_mul(df_sub(df_mul(c1, p1i), df_mul(r2, p2i)), inv);
            }
            if (dip) {
                // neighbour columns of the previous row: R_{n-1}^{m+1} and R_{n-1}^{m-1}
                df upr = df_shfl_down(p1r, 1), upi = df_shfl_down(p1i, 1);
                df dnr = df_shfl_up(p1r, 1), dni = df_shfl_up(p1i, 1);
                if (m == 31) upr = upi = df{0.f, 0.f};
                if (m == 0) {
                    dnr = df_neg(upr);  // R^{-1} = -conj R^1
                    dni = upi;
                }
                if (n >= m && n <= P) {
                    // q R_n^m - (dbar/2) R_{n-1}^{m+1} + (d/2) R_{n-1}^{m-1} + dz R_{n-1}^m
                    dacc_add_prod(ar[n], q, cr);
                    dacc_add_prod(ar[n], dwx, df_sub(dnr, upr));
                    dacc_add_prod(ar[n], dwy, df_neg(df_add(upi, dni)));
                    dacc_add_prod(ar[n], dz, p1r);
                    dacc_add_prod(ai[n], q, ci);
                    dacc_add_prod(ai[n], dwx, df_sub(dni, upi));
                    dacc_add_prod(ai[n], dwy, df_add(upr, dnr));
                    dacc_add_prod(ai[n], dz, p1i);
                }
            } else if (n >= m && n <= P) {
                dacc_add_prod(ar[n], q, cr);
                dacc_add_prod(ai[n], q, ci);
            }
            p2r = p1r;
            p2i = p1i;
            p1r = cr;
            p1i = ci;
        }
    }
    if (m <= P) {
#pragma unroll
        for (int n = 0; n <= PM; ++n)
            if (n >= m && n <= P) {
                const df vr = dacc_get(ar[n]), vi = dacc_get(ai[n]);
                const int64_t at = (int64_t)b * ST + tri(n, m);
                Mu[at] = make_double2(df_to(vr), df_to(vi));
                Muf[at] = df2_pack(vr, vi);
            }
    }
}

// M2M (Stage 2, one level) on double-floats: the structure of k_m2m8 (a block of 8 warps per parent,
// warp o translating child octant o with lanes over the outputs, the contributions added in octant
// order in shared memory), reading the children's double-float copies and the octant table's.
template <int PM>
__global__ void __launch_bounds__(256) k_m2m8_df(int b0, int b1, const int *lvl_boxes, const int *child,
                                                 const int *nsrc_sub, const signed char *pb, const float4 *octf,
                                                 double2 *Mu, float4 *Muf)
{
    __shared__ float4 part[8][ntri(PM)];
    int b = b0 + blockIdx.x;
    if (b >= b1) return;
    if (lvl_boxes) b = lvl_boxes[b];
    if (nsrc_sub[b] == 0) return;
    const int o = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = pb[b];
    const int c = child[8 * b + o];
    const bool live = c >= 0 && nsrc_sub[c] > 0;
    for (int out = lane; out < ntri(P); out += 32) {
        df vr{0.f, 0.f}, vi{0.f, 0.f};
        if (live) {
            int n = 0;
            while (tri(n + 1, 0) <= out) ++n;
            const int m = out - tri(n, 0);
            const int Pc = pb[c];
            const float4 *Mc = Muf + (int64_t)c * ntri(PM);
            const float4 *R = octf + o * ntri(PM);
            dacc tr{0.f, 0.f}, ti{0.f, 0.f};
            float sk = 1.0f;
            for (int k = 0; k <= n && k <= Pc; ++k, sk *= 0.5f) {
                const int j = n - k;
                const int lmin = max(-k, m - j), lmax = min(k, m + j);
                for (int l = lmin; l <= lmax; ++l) {
                    df ar, ai, rr, ri;
                    df_sym_get(Mc, k, l, ar, ai);
                    df_sym_get(R, j, m - l, rr, ri);
                    ar = df_mul_f(ar, sk);  // a power of two: exact
                    ai = df_mul_f(ai, sk);
                    dacc_add_prod(tr, ar, rr);
                    dacc_add_prod(tr, df_neg(ai), ri);
                    dacc_add_prod(ti, ar, ri);
                    dacc_add_prod(ti, ai, rr);
                }
            }
            vr = dacc_get(tr);
            vi = dacc_get(ti);
        }
        part[o][out] = df2_pack(vr, vi);
    }
    __syncthreads();
    for (int out = threadIdx.x; out < ntri(P); out += blockDim.x) {
        const double2 own = Mu[(int64_t)b * ntri(PM) + out];  // the box's own sources (none for non-leaves)
        df sr = df_from(own.x), si = df_from(own.y);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 f = part[k][out];
            sr = df_add(sr, df{f.x, f.y});
            si = df_add(si, df{f.z, f.w});
        }
        Mu[(int64_t)b * ntri(PM) + out] = make_double2(df_to(sr), df_to(si));
        Muf[(int64_t)b * ntri(PM) + out] = df2_pack(sr, si);
    }
}

// ---------------------------------------------------------------- List 2 M2L (Stage 4), FP64

template <int PM>
__global__ void k_m2l(int64_t nb, const int *vstart, const int *vidx, const int64_t *ic, const double *hw,
                      const signed char *pb, const signed char *ps, const double2 *Mu, const double2 *tab, double2 *B)
{
    extern __shared__ double2 sh[];
    int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int b = blockIdx.x * (blockDim.x / 32) + wl;
    if (b >= nb) return;
    int e0 = vstart[b], e1 = vstart[b + 1];
    if (e0 == e1) return;
    const int P = pb[b];
    double2 *Ms = sh + wl * ntri(PM);
    constexpr int NO = (ntri(PM) + 31) / 32;
    double2 acc[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) acc[i] = make_double2(0.0, 0.0);
    for (int e = e0; e < e1; ++e) {
        int d = vidx[e];
        const int Pd = ps[d];
        __syncwarp();
        for (int i = lane; i < ntri(PM); i += 32) Ms[i] = i < ntri(Pd) ? Mu[(int64_t)d * ntri(PM) + i] : make_double2(0, 0);
        __syncwarp();
        int ox = (int)(ic[3 * b] - ic[3 * d]), oy = (int)(ic[3 * b + 1] - ic[3 * d + 1]),
            oz = (int)(ic[3 * b + 2] - ic[3 * d + 2]);
        if (ox < -5 || ox > 5 || oy < -5 || oy > 5 || oz < -5 || oz > 5) continue;  // not a List 2 offset
        const double2 *S = tab + (int64_t)((ox + 5) + 11 * (oy + 5) + 121 * (oz + 5)) * ntri(2 * PM);
#pragma unroll
        for (int i = 0; i < NO; ++i) {
            int out = lane + 32 * i;
            if (out >= ntri(P)) continue;
            int k = 0;
            while (tri(k + 1, 0) <= out) ++k;
            int l = out - tri(k, 0);
            double2 a = acc[i];
            for (int n = 0; n <= Pd; ++n)
                for (int m = -n; m <= n; ++m) {
                    double2 mv = sym_get(Ms, n, m);
                    double2 sv = cconj(sym_get(S, n + k, m + l));
                    a.x += mv.x * sv.x - mv.y * sv.y;
                    a.y += mv.x * sv.y + mv.y * sv.x;
                }
            acc[i] = a;
        }
    }
    double hinv = 1.0 / hw[b];
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        int out = lane + 32 * i;
        if (out < ntri(P)) {
            double2 v = B[(int64_t)b * ntri(PM) + out];
            B[(int64_t)b * ntri(PM) + out] = make_double2(v.x + acc[i].x * hinv, v.y + acc[i].y * hinv);
        }
    }
}

// ---------------------------------------------------------------- List 4 far P2L (Stage 6b)

// One warp per box, lane m computes column m of S_n^m((c-s)/h), one source at a time.
template <int PM, int ST = PM>
__global__ void k_p2l(int64_t nb, const int *xs, const int *xi, const int *own_start, const double *sxyz, int64_t ns,
                      const double *sq, const double *sd, const double *cen, const double *hw, const signed char *pb,
                      double2 *B)
{
    int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int m = threadIdx.x & 31;
    if (b >= nb) return;
    int e0 = xs[b], e1 = xs[b + 1];
    if (e0 == e1) return;
    const int P = pb[b];
    double h = hw[b], hinv = 1.0 / h;
    double cx = cen[3 * b], cy = cen[3 * b + 1], cz = cen[3 * b + 2];
    double2 acc[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) acc[n] = make_double2(0.0, 0.0);
    for (int e = e0; e < e1; ++e) {
        int d = xi[e];
        for (int s = own_start[d]; s < own_start[d + 1]; ++s) {
            double x = (cx - sxyz[s]) * hinv, y = (cy - sxyz[ns + s]) * hinv, z = (cz - sxyz[2 * ns + s]) * hinv;
            double ir2 = 1.0 / (x * x + y * y + z * z);
            double rinv = sqrt(ir2);
            double q = sq[s];
            double2 dw = make_double2(0.0, 0.0), dwb = make_double2(0.0, 0.0);
            double dz = 0.0;
            if (sd) {
                double dx = sd[s] * hinv, dy = sd[ns + s] * hinv;
                dz = sd[2 * ns + s] * hinv;
                dw = make_double2(0.5 * dx, 0.5 * dy);
                dwb = make_double2(0.5 * dx, -0.5 * dy);
            }
            double2 wr = make_double2(x * ir2, y * ir2);
            double zz = z * ir2;
            double2 diag = make_double2(rinv, 0.0);
            for (int j = 1; j <= m && j <= PM + 1; ++j) diag = cscale(cmul(diag, wr), 2.0 * j - 1.0);
            double2 p2 = make_double2(0.0, 0.0), p1 = make_double2(0.0, 0.0);
#pragma unroll
            for (int n1 = 0; n1 <= PM + 1; ++n1) {  // row n1 = n + 1 closes output row n
                double2 cur = make_double2(0.0, 0.0);
                if (n1 == m) cur = diag;
                else if (n1 > m) {
                    double c1 = (2 * n1 - 1) * zz, c2 = (double)(n1 + m - 1) * (double)(n1 - m - 1) * ir2;
                    cur = make_double2(c1 * p1.x - c2 * p2.x, c1 * p1.y - c2 * p2.y);
                }
                int n = n1 - 1;
                double2 up, dn;  // S_{n+1}^{m+1}, S_{n+1}^{m-1}
                up.x = __shfl_down_sync(0xffffffffu, cur.x, 1);
                up.y = __shfl_down_sync(0xffffffffu, cur.y, 1);
                dn.x = __shfl_up_sync(0xffffffffu, cur.x, 1);
                dn.y = __shfl_up_sync(0xffffffffu, cur.y, 1);
                if (m == 31) up = make_double2(0.0, 0.0);
                if (m == 0) dn = make_double2(-up.x, up.y);
                if (n >= m && n <= P) {
                    // conj[q S_n^m + (dbar/2) S_{n+1}^{m+1} - (d/2) S_{n+1}^{m-1} + dz S_{n+1}^m]
                    double2 v = cscale(p1, q);
                    if (sd) {
                        double2 t1 = cmul(dwb, up), t2 = cmul(dw, dn);
                        v.x += t1.x - t2.x + dz * cur.x;
                        v.y += t1.y - t2.y + dz * cur.y;
                    }
                    acc[n] = cadd(acc[n], cconj(v));
                }
                p2 = p1;
                p1 = cur;
            }
        }
    }
    if (m <= P) {
#pragma unroll
        for (int n = 0; n <= PM; ++n)
            if (n >= m && n <= P) {
                double2 v = B[(int64_t)b * ntri(ST) + tri(n, m)];
                B[(int64_t)b * ntri(ST) + tri(n, m)] = make_double2(v.x + acc[n].x * hinv, v.y + acc[n].y * hinv);
            }
    }
}

// P2L with a block of 4 warps per box: warp w takes the List 4 far entries e = w (mod 4) (lane m
// computes column m of S_n^m((c-s)/h) for one source at a time, the diagonal by a prefix product
// over the lanes), and the 4 partial locals are added in warp order in shared memory.
template <int PM, int ST = PM>
__global__ void __launch_bounds__(128) k_p2l4(int64_t nb, const int *xs, const int *xi, const int *own_start,
                                              const double *sxyz, int64_t ns, const double *sq, const double *sd,
                                              const double *cen, const double *hw, const signed char *pb, double2 *B)
{
    __shared__ double2 part[4][PM + 1][PM + 1];
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int e0 = xs[b], e1 = xs[b + 1];
    if (e0 == e1) return;
    const int w = threadIdx.x >> 5, m = threadIdx.x & 31;
    const int P = pb[b];
    const double h = hw[b], hinv = 1.0 / h;
    const double cx = cen[3 * b], cy = cen[3 * b + 1], cz = cen[3 * b + 2];
    double2 acc[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) acc[n] = make_double2(0.0, 0.0);
    const double fm = 2.0 * m - 1.0;
    for (int e = e0 + w; e < e1; e += 4) {
        const int d = xi[e];
        for (int s = own_start[d]; s < own_start[d + 1]; ++s) {
            double x = (cx - sxyz[s]) * hinv, y = (cy - sxyz[ns + s]) * hinv, z = (cz - sxyz[2 * ns + s]) * hinv;
            double ir2 = 1.0 / (x * x + y * y + z * z);
            double rinv = sqrt(ir2);
            double q = sq[s];
            double2 dw = make_double2(0.0, 0.0), dwb = make_double2(0.0, 0.0);
            double dz = 0.0;
            if (sd) {
                double dx = sd[s] * hinv, dy = sd[ns + s] * hinv;
                dz = sd[2 * ns + s] * hinv;
                dw = make_double2(0.5 * dx, 0.5 * dy);
                dwb = make_double2(0.5 * dx, -0.5 * dy);
            }
            const double2 wr = make_double2(x * ir2, y * ir2);
            const double zz = z * ir2;
            // diagonal S_m^m = rinv prod_{j<=m} (2j-1) wr: inclusive prefix product of the lane factors
            double2 diag = (m == 0) ? make_double2(rinv, 0.0) : cscale(wr, fm);
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                double2 o;
                o.x = __shfl_up_sync(0xffffffffu, diag.x, off);
                o.y = __shfl_up_sync(0xffffffffu, diag.y, off);
                if (m >= off) diag = cmul(o, diag);
            }
            double2 p2 = make_double2(0.0, 0.0), p1 = make_double2(0.0, 0.0);
#pragma unroll
            for (int n1 = 0; n1 <= PM + 1; ++n1) {  // row n1 = n + 1 closes output row n
                double2 cur = make_double2(0.0, 0.0);
                if (n1 == m) cur = diag;
                else if (n1 > m) {
                    double c1 = (2 * n1 - 1) * zz, c2 = (double)(n1 + m - 1) * (double)(n1 - m - 1) * ir2;
                    cur = make_double2(c1 * p1.x - c2 * p2.x, c1 * p1.y - c2 * p2.y);
                }
                int n = n1 - 1;
                double2 up, dn;  // S_{n+1}^{m+1}, S_{n+1}^{m-1}
                up.x = __shfl_down_sync(0xffffffffu, cur.x, 1);
                up.y = __shfl_down_sync(0xffffffffu, cur.y, 1);
                dn.x = __shfl_up_sync(0xffffffffu, cur.x, 1);
                dn.y = __shfl_up_sync(0xffffffffu, cur.y, 1);
                if (m == 31) up = make_double2(0.0, 0.0);
                if (m == 0) dn = make_double2(-up.x, up.y);
                if (n >= m && n <= P) {
                    // conj[q S_n^m + (dbar/2) S_{n+1}^{m+1} - (d/2) S_{n+1}^{m-1} + dz S_{n+1}^m]
                    double2 v = cscale(p1, q);
                    if (sd) {
                        double2 t1 = cmul(dwb, up), t2 = cmul(dw, dn);
                        v.x += t1.x - t2.x + dz * cur.x;
                        v.y += t1.y - t2.y + dz * cur.y;
                    }
                    acc[n] = cadd(acc[n], cconj(v));
                }
                p2 = p1;
                p1 = cur;
            }
        }
    }
    if (m <= PM) {
#pragma unroll
        for (int n = 0; n <= PM; ++n) part[w][n][m] = acc[n];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntri(P); t += blockDim.x) {
        int n = 0;
        while (tri(n + 1, 0) <= t) ++n;
        const int mm = t - tri(n, 0);
        double2 sum = part[0][n][mm];
#pragma unroll
        for (int k = 1; k < 4; ++k) sum = cadd(sum, part[k][n][mm]);
        double2 v = B[(int64_t)b * ntri(ST) + t];
        B[(int64_t)b * ntri(ST) + t] = make_double2(v.x + sum.x * hinv, v.y + sum.y * hinv);
    }
}

// Stage 6(b) on double-floats: the structure of k_p2l4 (a block of four warps per target box, the
// List 4 far sources over the warps, lane m carrying column m of the irregular harmonics S_n^m(c_b - s)
// scaled by the box size, the diagonal by a prefix product over the lanes), with every product and
// sum in double-float arithmetic (df64.cuh) from double-float copies of the sources (k_to_df).
template <int PM, int ST>
__global__ void __launch_bounds__(128) k_p2l4_df(int64_t nb, const int *xs, const int *xi, const int *own_start,
                                                 int64_t ns, const float *sf, int dip, const double *cen,
                                                 const double *hw, const signed char *pb, double2 *B)
{
    __shared__ float4 part[4][PM + 1][PM + 1];
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int e0 = xs[b], e1 = xs[b + 1];
    if (e0 == e1) return;
    const int w = threadIdx.x >> 5, m = threadIdx.x & 31;
    const int P = pb[b];
    const double h = hw[b];
    const float hinv = (float)(1.0 / h);  // h is a power of two: exact
    const df cx = df_from(cen[3 * b]), cy = df_from(cen[3 * b + 1]), cz = df_from(cen[3 * b + 2]);
    dacc ar[PM + 1], ai[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) ar[n] = ai[n] = dacc{0.f, 0.f};
    const float fm = 2.0f * m - 1.0f;
    for (int e = e0 + w; e < e1; e += 4) {
        const int d = xi[e];
        for (int s = own_start[d]; s < own_start[d + 1]; ++s) {
            const df x = df_mul_f(df_sub(cx, df{sf[s], sf[3 * ns + s]}), hinv),
                     y = df_mul_f(df_sub(cy, df{sf[ns + s], sf[4 * ns + s]}), hinv),
                     z = df_mul_f(df_sub(cz, df{sf[2 * ns + s], sf[5 * ns + s]}), hinv);
            const df rinv = df_rsqrt(df_add(df_add(df_sqr(x), df_sqr(y)), df_sqr(z)));
            const df ir2 = df_sqr(rinv);
            const df q{sf[6 * ns + s], sf[7 * ns + s]};
            df dwx{0.f, 0.f}, dwy{0.f, 0.f}, dz{0.f, 0.f};  // d/2 = (dwx, dwy), dz, all scaled by 1/h
            if (dip) {
                dwx = df_mul_f(df{sf[8 * ns + s], sf[11 * ns + s]}, 0.5f * hinv);
                dwy = df_mul_f(df{sf[9 * ns + s], sf[12 * ns + s]}, 0.5f * hinv);
                dz = df_mul_f(df{sf[10 * ns + s], sf[13 * ns + s]}, hinv);
            }
            const df wrx = df_mul(x, ir2), wry = df_mul(y, ir2), zz = df_mul(z, ir2);
            // diagonal S_m^m = rinv prod_{j<=m} (2j-1) wr: inclusive prefix product of the lane factors
            df gr = m == 0 ? rinv : df_mul_f(wrx, fm), gi = m == 0 ? df{0.f, 0.f} : df_mul_f(wry, fm);
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const df orr = df_shfl_up(gr, off), oi = df_shfl_up(gi, off);
                if (m >= off) {
                    const df nr = df_sub(df_mul(orr, gr), df_mul(oi, gi));
                    gi = df_add(df_mul(orr, gi), df_mul(oi, gr));
                    gr = nr;
                }
            }
            df p2r{0.f, 0.f}, p2i{0.f, 0.f}, p1r{0.f, 0.f}, p1i{0.f, 0.f};
#pragma unroll
            for (int n1 = 0; n1 <= PM + 1; ++n1) {  // row n1 = n + 1 closes output row n
                df cr{0.f, 0.f}, ci{0.f, 0.f};
                if (n1 == m) {
                    cr = gr;
                    ci = gi;
                } else if (n1 > m) {
                    const df c1 = df_mul_f(zz, (float)(2 * n1 - 1));
                    const df c2 = df_mul_f(ir2, (float)((n1 + m - 1) * (n1 - m - 1)));
                    cr = df_sub(df_mul(c1, p1r), df_mul(c2, p2r));
                    ci = df_sub(df_mul(c1, p1i), df_mul(c2, p2i));
                }
                const int n = n1 - 1;
                if (dip) {
                    df upr = df_shfl_down(cr, 1), upi = df_shfl_down(ci, 1);  // S_{n+1}^{m+1}
                    df dnr = df_shfl_up(cr, 1), dni = df_shfl_up(ci, 1);      // S_{n+1}^{m-1}
                    if (m == 31) upr = upi = df{0.f, 0.f};
                    if (m == 0) {
                        dnr = df_neg(upr);  // S^{-1} = -conj S^1
                        dni = upi;
                    }
                    if (n >= m && n <= P) {
                        // conj[q S_n^m + (dbar/2) S_{n+1}^{m+1} - (d/2) S_{n+1}^{m-1} + dz S_{n+1}^m]:
                        //   (dbar/2) up = (dwx up.r + dwy up.i) + i (dwx up.i - dwy up.r)
                        //   (d/2) dn    = (dwx dn.r - dwy dn.i) + i (dwx dn.i + dwy dn.r)
                        dacc_add_prod(ar[n], q, p1r);
                        dacc_add_prod(ar[n], dwx, df_sub(upr, dnr));
                        dacc_add_prod(ar[n], dwy, df_add(upi, dni));
                        dacc_add_prod(ar[n], dz, cr);
                        dacc_add_prod(ai[n], df_neg(q), p1i);
                        dacc_add_prod(ai[n], df_neg(dwx), df_sub(upi, dni));
                        dacc_add_prod(ai[n], dwy, df_add(upr, dnr));
                        dacc_add_prod(ai[n], df_neg(dz), ci);
                    }
                } else if (n >= m && n <= P) {
                    dacc_add_prod(ar[n], q, p1r);
                    dacc_add_prod(ai[n], df_neg(q), p1i);
                }
                p2r = p1r;
                p2i = p1i;
                p1r = cr;
                p1i = ci;
            }
        }
    }
    if (m <= PM) {
#pragma unroll
        for (int n = 0; n <= PM; ++n) {
            const df vr = dacc_get(ar[n]), vi = dacc_get(ai[n]);
            part[w][n][m] = make_float4(vr.h, vr.l, vi.h, vi.l);
        }
    }
    __syncthreads();
    const double dh = 1.0 / h;
    for (int t = threadIdx.x; t < ntri(P); t += blockDim.x) {
        int n = 0;
        while (tri(n + 1, 0) <= t) ++n;
        const int mm = t - tri(n, 0);
        float4 f = part[0][n][mm];
        df sr{f.x, f.y}, si{f.z, f.w};
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            f = part[k][n][mm];
            sr = df_add(sr, df{f.x, f.y});
            si = df_add(si, df{f.z, f.w});
        }
        double2 v = B[(int64_t)b * ntri(ST) + t];
        B[(int64_t)b * ntri(ST) + t] = make_double2(v.x + df_to(sr) * dh, v.y + df_to(si) * dh);
    }
}

// ---------------------------------------------------------------- L2L (Stage 7), by level

template <int PM>
__global__ void k_l2l(int b0, int b1, const int *lvl_boxes, const int *parent, const int *ntgt_sub, const int *child,
                      const signed char *pb, const double2 *oct, double2 *B)
{
    int b = b0 + blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (b >= b1) return;
    if (lvl_boxes) b = lvl_boxes[b];
    if (ntgt_sub[b] == 0) return;
    int pa = parent[b];
    if (pa < 0) return;
    int o = 0;
    while (o < 8 && child[8 * pa + o] != b) ++o;
    if (o == 8) return;
    // delta = (c_par - c_child)/h_par: the opposite corner of octant o
    const double2 *R = oct + (7 - o) * ntri(PM);
    const int P = pb[b], Pp = pb[pa];
    const double2 *Lp = B + (int64_t)pa * ntri(PM);
    for (int out = lane; out < ntri(P); out += 32) {
        int k = 0;
        while (tri(k + 1, 0) <= out) ++k;
        int l = out - tri(k, 0);
        double2 acc = make_double2(0.0, 0.0);
        for (int n = k; n <= Pp; ++n) {
            int j = n - k;
            for (int m = max(-n, l - j); m <= min(n, l + j); ++m) {
                double2 t = cmul(sym_get(Lp, n, m), sym_get(R, j, m - l));
                acc.x += t.x;
                acc.y += t.y;
            }
        }
        double sk = ldexp(1.0, -k);
        double2 v = B[(int64_t)b * ntri(PM) + out];
        B[(int64_t)b * ntri(PM) + out] = make_double2(v.x + sk * acc.x, v.y + sk * acc.y);
    }
}

// ---------------------------------------------------------------- QBX centers (Stages 3, 5, 6a, 8)

struct ListRef {
    const int *start, *idx;
};

// Per-lane accumulation of q conj S_k^l((c-s)/rho)/rho (+ dipole) for one source.
template <int QM>
__device__ __forceinline__ void p2qbxl_accum(double bx, double by, double bz, double q, bool dip, double dx, double dy,
                                             double dz, int Q, double *ar, double *ai)
{
    double ir2 = 1.0 / (bx * bx + by * by + bz * bz);
    double rinv = sqrt(ir2);
    double wr = bx * ir2, wi = by * ir2, zz = bz * ir2;
    // rows n-2, n-1, n of S
    double s2r[QM + 2], s2i[QM + 2], s1r[QM + 2], s1i[QM + 2], s0r[QM + 2], s0i[QM + 2];
#pragma unroll
    for (int m = 0; m < QM + 2; ++m) { s2r[m] = s2i[m] = s1r[m] = s1i[m] = s0r[m] = s0i[m] = 0.0; }
    s1r[0] = rinv;  // row 0
    if (!dip) {
        ar[0] += q * rinv;
    }
    const double hdx = 0.5 * dx, hdy = 0.5 * dy;
    const double nq = -q, ndz = -dz, nhdx = -hdx;
#pragma unroll
    for (int n = 1; n <= QM + 1; ++n) {
        if (n > Q + (dip ? 1 : 0)) break;
        const double c1 = (2 * n - 1) * zz;
#pragma unroll
        for (int m = 0; m < n; ++m) {
            if (m <= n - 2) {
                double c2 = (double)(n + m - 1) * (double)(n - m - 1) * ir2;
                s0r[m] = c1 * s1r[m] - c2 * s2r[m];
                s0i[m] = c1 * s1i[m] - c2 * s2i[m];
            } else {
                s0r[m] = c1 * s1r[m];
                s0i[m] = c1 * s1i[m];
            }
        }
        {
            double f = 2 * n - 1;
            double pr = s1r[n - 1], pi = s1i[n - 1];
            s0r[n] = f * (pr * wr - pi * wi);
            s0i[n] = f * (pr * wi + pi * wr);
        }
        if (!dip) {
            if (n <= QM) {
#pragma unroll
                for (int m = 0; m <= n && n <= QM; ++m) {
                    ar[tri(n, m)] += q * s0r[m];
                    ai[tri(n, m)] -= q * s0i[m];
                }
            }
        } else {
            // close row k = n - 1: q S_k^l + (dbar/2) S_n^{l+1} - (d/2) S_n^{l-1} + dz S_n^l, conjugated
            const int k = n - 1;
            if (k <= QM) {
#pragma unroll
                for (int l = 0; l <= k && k <= QM; ++l) {
                    // (dbar/2) S^{l+1} = (hdx - i hdy)(ur + i ui); -(d/2) S^{l-1} with S^{-1} = -conj S^1:
                    //   Re: q S_k^l + dz S_n^l + hdx (ur - tr) + hdy (ui + ti)
                    //   Im: q S_k^l + dz S_n^l + hdx (ui - ti) - hdy (ur + tr), accumulated conjugated
                    const double ur = s0r[l + 1], ui = s0i[l + 1];
                    double tr, ti;
                    if (l >= 1) { tr = s0r[l - 1]; ti = s0i[l - 1]; }
                    else { tr = -s0r[1]; ti = s0i[1]; }
                    double xr = ar[tri(k, l)], xi = ai[tri(k, l)];
                    xr = fma(q, s1r[l], xr);
                    xr = fma(dz, s0r[l], xr);
                    xr = fma(hdx, ur - tr, xr);
                    xr = fma(hdy, ui + ti, xr);
                    xi = fma(nq, s1i[l], xi);
                    xi = fma(ndz, s0i[l], xi);
                    xi = fma(nhdx, ui - ti, xi);
                    xi = fma(hdy, ur + tr, xi);
                    ar[tri(k, l)] = xr;
                    ai[tri(k, l)] = xi;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < QM + 2; ++m) {
            s2r[m] = s1r[m]; s2i[m] = s1i[m];
            s1r[m] = s0r[m]; s1i[m] = s0i[m];
        }
    }
}

// One warp per QBX center: List 3 far M2QBXL in FP64 (Stage 5(b); an empty list in the mixed modes) and,
// with `direct`, the direct P2QBXL of Lists 1, 3 close and 4 close in the coefficient form (Stages 3,
// 5(a), 6(a)); the warp's sums are reduced and stored to A.  L2QBXL (Stage 8) is k_l2qbxl.
template <int QM, int PM>
__global__ void __launch_bounds__(128) k_centers(
    int64_t nc, const int *ctr_box, const double *cxyz, const double *cr, const signed char *qc,
    const signed char *ps, ListRef lu, ListRef lwc, ListRef lxc, ListRef lwf, const int *own_start, const double *sxyz,
    int64_t ns, const double *sq, const double *sd, const double *cen, const double *hw, const double2 *Mu,
    double2 *A, int direct)
{
    extern __shared__ double2 sh[];
    constexpr int NT = ntri(QM);
    constexpr int TAB = ntri(PM + QM) + PM + 1;
    int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + wl;
    if (i >= nc) return;
    double2 *tab = sh + wl * TAB;
    const int b = ctr_box[i];
    const int Q = min((int)qc[i], QM);
    const double cx = cxyz[i], cy = cxyz[nc + i], cz = cxyz[2 * nc + i];
    const double rho = cr[i], rinv_c = 1.0 / rho;
    double ar[NT], ai[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) ar[t] = ai[t] = 0.0;

    double *pw = reinterpret_cast<double *>(tab + TAB - (PM + 1));  // powers, at the end of the warp's table

    // Stage 5(b): List 3 far multipoles to the QBX local
    for (int e = lwf.start[b]; e < lwf.start[b + 1]; ++e) {
        const int d = lwf.idx[e];
        const int Pd = min((int)ps[d], PM);
        const double hd = hw[d], hdinv = 1.0 / hd, ratio = rho * hdinv;
        __syncwarp();
        // S_j^i((c - c_d)/h_d) (rho/h_d)^j / h_d, j <= Pd + Q; pw[n] = (h_d/rho)^n
        irregular_table_warp(Pd + Q, (cx - cen[3 * d]) * hdinv, (cy - cen[3 * d + 1]) * hdinv,
                             (cz - cen[3 * d + 2]) * hdinv, ratio, hdinv, tab, lane);
        if (lane <= Pd) pw[lane] = pow(ratio, -lane);
        __syncwarp();
        const double2 *Md = Mu + (int64_t)d * ntri(PM);
        for (int in = lane; in < (Pd + 1) * (Pd + 1); in += 32) {
            int n = (int)sqrtf((float)in);
            while (n * n > in) --n;
            while ((n + 1) * (n + 1) <= in) ++n;
            int m = in - n * n - n;
            double2 mv = cscale(sym_get(Md, n, m), pw[n]);
            const double nmy = -mv.y;
#pragma unroll
            for (int k = 0; k <= QM; ++k) {
                if (k > Q) break;
#pragma unroll
                for (int l = 0; l <= k; ++l) {
                    double2 sv = cconj(sym_get(tab, n + k, m + l));
                    ar[tri(k, l)] = fma(mv.x, sv.x, fma(nmy, sv.y, ar[tri(k, l)]));
                    ai[tri(k, l)] = fma(mv.x, sv.y, fma(mv.y, sv.x, ai[tri(k, l)]));
                }
            }
        }
    }

    // Stages 3, 5(a), 6(a): direct P2QBXL from List 1, List 3 close and List 4 close sources, the three
    // lists walked as one sequence of boxes so that partial batches of 32 sources are rare (in the
    // coefficient form; qbx_eval sums them at the targets instead, in k_qbx_direct)
    const bool dip = sd != nullptr;
    if (direct) {
        const int u0 = lu.start[b], n0 = lu.start[b + 1] - u0;
        const int w0 = lwc.start[b], n1 = lwc.start[b + 1] - w0;
        const int x0 = lxc.start[b], n2 = lxc.start[b + 1] - x0;
        const int e1 = n0 + n1 + n2;
        for (int base = 0; base < e1; base += 32) {
            int e = base + lane;
            int d = -1;
            if (e < n0) d = lu.idx[u0 + e];
            else if (e < n0 + n1) d = lwc.idx[w0 + e - n0];
            else if (e < e1) d = lxc.idx[x0 + e - n0 - n1];
            int s0 = d >= 0 ? own_start[d] : 0;
            int cnt = d >= 0 ? own_start[d + 1] - s0 : 0;
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int k0 = 0; k0 < total; k0 += 32) {
                int k = k0 + lane;
                int j = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
                    if (v <= k) j += step;
                }
                int sj = __shfl_sync(0xffffffffu, s0, j);
                int ij = __shfl_sync(0xffffffffu, incl, j);
                int cj = __shfl_sync(0xffffffffu, cnt, j);
                if (k < total) {
                    int s = sj + (k - (ij - cj));
                    double bx = (cx - sxyz[s]) * rinv_c, by = (cy - sxyz[ns + s]) * rinv_c,
                           bz = (cz - sxyz[2 * ns + s]) * rinv_c;
                    double q = sq[s] * rinv_c;
                    double dx = 0.0, dy = 0.0, dz = 0.0;
                    if (dip) {
                        double f = rinv_c * rinv_c;
                        dx = sd[s] * f;
                        dy = sd[ns + s] * f;
                        dz = sd[2 * ns + s] * f;
                    }
                    p2qbxl_accum<QM>(bx, by, bz, q, dip, dx, dy, dz, Q, ar, ai);
                }
            }
        }
    }

    // reduce over the warp and store
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        double vr = ar[t], vi = ai[t];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, off);
            vi += __shfl_xor_sync(0xffffffffu, vi, off);
        }
        if ((t & 31) == lane) A[i * NT + t] = make_double2(vr, vi);
    }
}

// ---------------------------------------------------------------- Stage 8: L2QBXL, one thread per center

// Double-float copy of the box locals (re.h, re.l, im.h, im.l per coefficient), the first
// ntri(pb[b]) coefficients of every box, same stride as B.
__global__ void k_locals_to_df(int64_t nb, int stride, const signed char *pb, const double2 *B, float4 *Bf)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb * stride) return;
    const int64_t b = q / stride;
    const int t = (int)(q % stride);
    if (t >= ntri(min((int)pb[b], PMAX))) return;
    const double2 v = B[q];
    const df re = df_from(v.x), im = df_from(v.y);
    Bf[q] = make_float4(re.h, re.l, im.h, im.l);
}

__device__ __forceinline__ df df_negif(df a, bool f) { return f ? df{-a.h, -a.l} : a; }

// Outputs k in [K0, K1] of the QBX local of one center (Algorithm 4 Stage 8).  By the addition theorem
// R_n^m(u + v) = sum_{k,l} R_{n-k}^{m-l}(u) R_k^l(v), the box local sum B_n^m R_n^m((c_b - x)/h) regrouped
// by the power of v = (c - x)/h gives, with u = (c_b - c)/h and the QBX local scaled by rho,
//   A_k^l = (rho/h)^k sum_{j <= P-k} sum_{|mu| <= j} R_j^mu(u) B_{j+k}^{mu+l}.
// The harmonics R_j^mu(u) come from their recurrence column by column (mu >= 0, rows j = mu..P-K0),
// each value serving mu and -mu (R_j^-mu = (-1)^mu conj R_j^mu); the K1-K0+1 output rows stay in
// registers, so nothing is reduced across threads.  Double-float arithmetic, the sums as compensated
// dot products (df64.cuh).  Ac receives the sums (add: accumulates onto it).
template <int K0, int K1>
__device__ __forceinline__ void l2q_pass(int P, int Q, df ux, df uy, df uz, double ratio,
                                         const float4 *__restrict__ Lb, double2 *__restrict__ Ac,
                                         float4 *__restrict__ Acf, bool add, const float4 *__restrict__ Rtab = nullptr)
{
    if (add && Q < K0) return;
    constexpr int T0 = K0 * (K0 + 1) / 2;  // tri(K0, 0)
    constexpr int NA = ntri(K1) - T0;
    dacc ar[NA], ai[NA];
#pragma unroll
    for (int t = 0; t < NA; ++t) ar[t] = ai[t] = dacc{0.f, 0.f};
    const df r2 = df_add(df_add(df_sqr(ux), df_sqr(uy)), df_sqr(uz));
    const int jmax = P - K0;
    df dr{1.f, 0.f}, di{0.f, 0.f};  // R_mu^mu(u)
    for (int mu = 0; mu <= jmax; ++mu) {
        if (mu > 0 && !Rtab) {
            const float2 hs = c_l2q_half[mu];
            const df s{hs.x, hs.y};
            const df nr = df_mul(df_sub(df_mul(dr, ux), df_mul(di, uy)), s);
            const df ni = df_mul(df_add(df_mul(dr, uy), df_mul(di, ux)), s);
            dr = nr;
            di = ni;
        }
        df p1r = dr, p1i = di, p2r{0.f, 0.f}, p2i{0.f, 0.f};  // R_{j-1}^mu, R_{j-2}^mu
        const bool smu = mu & 1;
        for (int j = mu; j <= jmax; ++j) {
            df rr = dr, ri = di;
            if (Rtab) {  // R_j^mu(u) tabulated (a fixed translation)
                const float4 v = Rtab[tri(j, mu)];
                rr = df{v.x, v.y};
                ri = df{v.z, v.w};
            } else if (j > mu) {
                const float2 iv = c_l2q_rinv[tri(j, mu)];
                const df inv{iv.x, iv.y}, c1 = df_mul_f(uz, (float)(2 * j - 1));
                rr = df_mul(df_sub(df_mul(c1, p1r), df_mul(r2, p2r)), inv);
                ri = df_mul(df_sub(df_mul(c1, p1i), df_mul(r2, p2i)), inv);
                p2r = p1r;
                p2i = p1i;
                p1r = rr;
                p1i = ri;
            }
            const df nri = df_neg(ri);
#pragma unroll
            for (int k = K0; k <= K1; ++k) {
                if (k > Q || j + k > P) break;
                const float4 *Bn = Lb + tri(j + k, 0);
#pragma unroll
                for (int l = 0; l <= k; ++l) {
                    const int t = tri(k, l) - T0;
                    const float4 b1 = Bn[mu + l];
                    const df b1x{b1.x, b1.y}, b1y{b1.z, b1.w};
                    dacc_add_prod(ar[t], rr, b1x);
                    dacc_add_prod(ar[t], nri, b1y);
                    dacc_add_prod(ai[t], rr, b1y);
                    dacc_add_prod(ai[t], ri, b1x);
                    if (mu > 0) {
                        // B_n^{m2}, m2 = l - mu: (-1)^m2 conj B_n^{-m2} when m2 < 0; times (-1)^mu, then
                        // conj(R_j^mu) B'': Re = rr b''x + ri b''y, Im = rr b''y - ri b''x
                        const int m2 = l - mu;
                        const float4 b2 = Bn[m2 < 0 ? -m2 : m2];
                        const bool neg = m2 < 0, sm2 = neg && (m2 & 1);
                        const df bx = df_negif(df{b2.x, b2.y}, smu != sm2);
                        const df by = df_negif(df{b2.z, b2.w}, smu != (neg != sm2));
                        dacc_add_prod(ar[t], rr, bx);
                        dacc_add_prod(ar[t], ri, by);
                        dacc_add_prod(ai[t], rr, by);
                        dacc_add_prod(ai[t], nri, bx);
                    }
                }
            }
        }
    }
    double pk = 1.0;
#pragma unroll
    for (int k = 0; k < K0; ++k) pk *= ratio;
#pragma unroll
    for (int k = K0; k <= K1; ++k) {
        if (add && k > Q) break;
#pragma unroll
        for (int l = 0; l <= k; ++l) {
            const int t = tri(k, l) - T0;
            double2 v = make_double2(df_to(dacc_get(ar[t])) * pk, df_to(dacc_get(ai[t])) * pk);
            if (add) {
                const double2 o = Ac[tri(k, l)];
                v = make_double2(o.x + v.x, o.y + v.y);
            }
            Ac[tri(k, l)] = v;
            if (Acf) {
                const df re = df_from(v.x), im = df_from(v.y);
                Acf[tri(k, l)] = make_float4(re.h, re.l, im.h, im.l);
            }
        }
        pk *= ratio;
    }
}

// All output rows k <= KMAX (at most Q of them used) in passes whose accumulators fit in registers.
template <int KMAX>
__device__ __forceinline__ void l2x_passes(int P, int Q, df ux, df uy, df uz, double ratio, const float4 *Lb,
                                           double2 *Ac, float4 *Acf, bool add)
{
    if constexpr (KMAX <= 4) {
        l2q_pass<0, 4>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
    } else {
        l2q_pass<0, 5>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        l2q_pass<6, 8>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 9) l2q_pass<9, 10>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 11) l2q_pass<11, 12>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 13) l2q_pass<13, 14>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 15) l2q_pass<15, 15>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 16) l2q_pass<16, 16>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 17) l2q_pass<17, 17>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 18) l2q_pass<18, 18>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 19) l2q_pass<19, 19>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
        if constexpr (KMAX >= 20) l2q_pass<20, 20>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add);
    }
}

// One thread per QBX center (sorted order): A (+)= L2QBXL of its box's local at the box's order.
template <int QM>
__global__ void __launch_bounds__(128) k_l2qbxl(int64_t nc, const int *ctr_box, const double *cxyz, const double *cr,
                                                const signed char *qc, const signed char *pb, const double *cen,
                                                const double *hw, const float4 *Bf, int pm_stride, double2 *A, int add)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int b = ctr_box[i];
    const int Q = min((int)qc[i], QM), P = min((int)pb[b], PMAX);
    const double h = hw[b], hinv = 1.0 / h;
    const df ux = df_from((cen[3 * b] - cxyz[i]) * hinv), uy = df_from((cen[3 * b + 1] - cxyz[nc + i]) * hinv),
             uz = df_from((cen[3 * b + 2] - cxyz[2 * nc + i]) * hinv);
    const double ratio = cr[i] * hinv;
    const float4 *Lb = Bf + (int64_t)b * pm_stride;
    l2x_passes<QM>(P, Q, ux, uy, uz, ratio, Lb, A + i * ntri(QM), nullptr, add);
}

// Stage 7, one level: one thread per box b of the level with targets below it; its local receives
// its parent's local translated to b's center (the same regrouping with u = (c_parent - c_b)/h_parent,
// a corner of the parent's half-width cube, and the box scaling ratio 1/2), at b's order from the
// parent's order.  B (FP64) is updated and its double-float copy Bf written for b's children and
// for L2QBXL.
// Number of output passes of l2x_passes<KMAX> and one of them by index.
__host__ __device__ constexpr int l2x_npass(int kmax)
{
    return kmax <= 4 ? 1 : kmax <= 8 ? 2 : kmax <= 10 ? 3 : kmax <= 12 ? 4 : kmax <= 14 ? 5 : kmax - 9;
}

template <int KMAX>
__device__ __forceinline__ void l2x_one_pass(int pass, int P, int Q, df ux, df uy, df uz, double ratio,
                                             const float4 *Lb, double2 *Ac, float4 *Acf, bool add, const float4 *Rtab)
{
    static_assert(KMAX >= 10, "passes of the box-to-box translations");
    switch (pass) {
    case 0: l2q_pass<0, 5>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 1: l2q_pass<6, 8>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 2: l2q_pass<9, 10>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 3: if constexpr (KMAX >= 11) l2q_pass<11, 12>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 4: if constexpr (KMAX >= 13) l2q_pass<13, 14>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 5: if constexpr (KMAX >= 15) l2q_pass<15, 15>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 6: if constexpr (KMAX >= 16) l2q_pass<16, 16>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 7: if constexpr (KMAX >= 17) l2q_pass<17, 17>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 8: if constexpr (KMAX >= 18) l2q_pass<18, 18>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 9: if constexpr (KMAX >= 19) l2q_pass<19, 19>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    case 10: if constexpr (KMAX >= 20) l2q_pass<20, 20>(P, Q, ux, uy, uz, ratio, Lb, Ac, Acf, add, Rtab); break;
    default: break;
    }
}

// Stage 7, one level: one thread per (box b of the level with targets below it, output pass); b's
// local receives its parent's local translated to b's center (the same regrouping with
// u = (c_parent - c_b)/h_parent, a corner of the parent's half-width cube, whose harmonics are
// tabulated, and the box scaling ratio 1/2), at b's order from the parent's order.  The passes of
// a box write disjoint rows.  B (FP64) is updated and its double-float copy Bf written for b's
// children and for L2QBXL.  Thread index = pass * (boxes of the level) + box, so a warp runs one pass.
template <int PB>
__global__ void __launch_bounds__(128) k_l2l_df(int b0, int b1, const int *lvl_boxes, const int *parent,
                                                const int *ntgt_sub, const int *child, const signed char *pb,
                                                const float4 *octf, int stride, double2 *B, float4 *Bf)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nbl = b1 - b0;
    if (g >= (int64_t)nbl * l2x_npass(PB)) return;
    const int pass = (int)(g / nbl);
    int b = b0 + (int)(g % nbl);
    if (lvl_boxes) b = lvl_boxes[b];
    if (ntgt_sub[b] == 0) return;
    const int pa = parent[b];
    if (pa < 0) return;
    int o = 0;
    while (o < 8 && child[8 * pa + o] != b) ++o;
    if (o == 8) return;
    const df ux{(o & 1) ? -0.5f : 0.5f, 0.f}, uy{(o & 2) ? -0.5f : 0.5f, 0.f}, uz{(o & 4) ? -0.5f : 0.5f, 0.f};
    l2x_one_pass<PB>(pass, min((int)pb[pa], PMAX), min((int)pb[b], PB), ux, uy, uz, 0.5, Bf + (int64_t)pa * stride,
                     B + (int64_t)b * stride, Bf + (int64_t)b * stride, true, octf + (7 - o) * stride);
}

// Double-float copy of the locals of the boxes [b0, b1) of one level (the roots before Stage 7).
__global__ void k_level_to_df(int b0, int b1, const int *lvl_boxes, int stride, const signed char *pb,
                              const double2 *B, float4 *Bf)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)(b1 - b0) * stride) return;
    int b = b0 + (int)(q / stride);
    if (lvl_boxes) b = lvl_boxes[b];
    const int t = (int)(q % stride);
    if (t >= ntri(min((int)pb[b], PMAX))) return;
    const double2 v = B[(int64_t)b * stride + t];
    const df re = df_from(v.x), im = df_from(v.y);
    Bf[(int64_t)b * stride + t] = make_float4(re.h, re.l, im.h, im.l);
}

// Legendre-recurrence coefficients of T_n = A_n (x u) T_{n-1} - B_n x^2 T_{n-2}, A_n = (2n-1)/n,
// B_n = (n-1)/n, as double-floats (leading, trailing): c_leg[n] = (A_h, A_l, B_h, B_l).
__constant__ float4 c_leg[QMAX + 1];

void set_leg_table(cudaStream_t st)
{
    static float4 t[QMAX + 1];
    for (int n = 1; n <= QMAX; ++n) {
        const double A = (2.0 * n - 1.0) / n, B = (n - 1.0) / n;
        const float ah = (float)A, bh = (float)B;
        t[n] = make_float4(ah, (float)(A - (double)ah), bh, (float)(B - (double)bh));
    }
    t[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_leg, t, sizeof(t), 0, cudaMemcpyHostToDevice, st));
}

__device__ __forceinline__ df df_warp_sum(df v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v = df_add(v, df{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)});
    return v;
}

// Stages 3, 5(a), 6(a) + 9 for one QBX target: the order-Q QBX expansion about its center c of the
// sources of List 1, List 3 close and List 4 close of c's box, evaluated at the target t.  By the
// addition theorem the m-sum of an order-n term of the expansion (eqs. qbxcoeff, qbxlocal) collapses,
// for charge q at s, to q rho^n / r^(n+1) P_n(u) (rho = |t - c|, r = |s - c|, u = the cosine of the
// angle between t - c and s - c), and the dipole term is d . grad_s of it:
//   d . grad_s [r^-(n+1) P_n(u)] = r^-(n+2) [ (d.a - u d.e) P_n'(u) - (n+1) (d.e) P_n(u) ]
// (a, e the unit vectors of t - c and s - c).  With T_n = x^n P_n(u), T'_n = x^n P_n'(u), x = rho / r:
//   T_n = (2n-1)/n (x u) T_{n-1} - (n-1)/n x^2 T_{n-2},   T'_n = (2n-1) x T_{n-1} + x^2 T'_{n-2}.
// The value is sum_s [q sum_n T_n + (1/r) sum_n ((d.a - u d.e) T'_n - (n+1)(d.e) T_n)] / r, the same
// truncated expansion as the coefficient form up to rounding, at O(Q) work per (source, target) pair
// instead of O(Q^2) per (source, center).  Arithmetic in double-float (df64.cuh) from double-float
// copies of the points and densities (k_to_df).  One warp per target; lanes take the sources of the
// three lists walked as one sequence of boxes.  out[t] (input order) receives the sum without
// 1/(4 pi); with SWEEP, out[n * nt + t] receives the order-n part for n = 0..QM.
template <int QM, bool SWEEP>
__global__ void __launch_bounds__(128) k_qbx_direct(int64_t nt, const int *tperm, const float *tf, const int *tgt_ctr,
                                                    const int *ctr_rank, const int *ctr_box, int64_t nc,
                                                    const float *cf, const signed char *qc, ListRef lu, ListRef lwc,
                                                    ListRef lxc, const int *own_start, int64_t ns, const float *sf,
                                                    int dip, double *out)
{
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t it = (int64_t)blockIdx.x * 4 + wl;
    if (it >= nt) return;
    const int t = tperm[it];
    const int c = tgt_ctr[t];
    if (c < 0 || c >= nc) return;  // point targets (out of range indices are flagged by the argument check)
    const int i = ctr_rank[c], b = ctr_box[i];
    const int Q = min((int)qc[i], QM);
    const df cx{cf[i], cf[3 * nc + i]}, cy{cf[nc + i], cf[4 * nc + i]}, cz{cf[2 * nc + i], cf[5 * nc + i]};
    df ax = df_sub(df{tf[it], tf[3 * nt + it]}, cx), ay = df_sub(df{tf[nt + it], tf[4 * nt + it]}, cy),
       az = df_sub(df{tf[2 * nt + it], tf[5 * nt + it]}, cz);
    const df rho2 = df_add(df_add(df_sqr(ax), df_sqr(ay)), df_sqr(az));
    df rho{0.f, 0.f};
    if (rho2.h > 0.f) {  // t = c: a = 0 and rho = 0, only the n = 0 terms remain
        const df ri = df_rsqrt(rho2);
        rho = df_mul(rho2, ri);
        ax = df_mul(ax, ri);
        ay = df_mul(ay, ri);
        az = df_mul(az, ri);
    }
    df acc[SWEEP ? QM + 1 : 1];
#pragma unroll
    for (int n = 0; n < (SWEEP ? QM + 1 : 1); ++n) acc[n] = df{0.f, 0.f};
    const int u0 = lu.start[b], n0 = lu.start[b + 1] - u0;
    const int w0 = lwc.start[b], n1 = lwc.start[b + 1] - w0;
    const int x0 = lxc.start[b], n2 = lxc.start[b + 1] - x0;
    const int e1 = n0 + n1 + n2;
    for (int base = 0; base < e1; base += 32) {
        const int e = base + lane;
        int d = -1;
        if (e < n0) d = lu.idx[u0 + e];
        else if (e < n0 + n1) d = lwc.idx[w0 + e - n0];
        else if (e < e1) d = lxc.idx[x0 + e - n0 - n1];
        const int s0 = d >= 0 ? own_start[d] : 0;
        const int cnt = d >= 0 ? own_start[d + 1] - s0 : 0;
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
                if (v <= k) j += step;
            }
            const int sj = __shfl_sync(0xffffffffu, s0, j);
            const int ij = __shfl_sync(0xffffffffu, incl, j);
            const int cj = __shfl_sync(0xffffffffu, cnt, j);
            if (k >= total) continue;
            const int s = sj + (k - (ij - cj));
            const df ex = df_sub(df{sf[s], sf[3 * ns + s]}, cx), ey = df_sub(df{sf[ns + s], sf[4 * ns + s]}, cy),
                     ez = df_sub(df{sf[2 * ns + s], sf[5 * ns + s]}, cz);
            const df rinv = df_rsqrt(df_add(df_add(df_sqr(ex), df_sqr(ey)), df_sqr(ez)));
            const df u = df_mul(df_add(df_add(df_mul(ax, ex), df_mul(ay, ey)), df_mul(az, ez)), rinv);
            const df x = df_mul(rho, rinv), x2 = df_sqr(x), xu = df_mul(x, u);
            const df q{sf[6 * ns + s], sf[7 * ns + s]};
            df alpha{0.f, 0.f}, dE{0.f, 0.f};
            if (dip) {
                const df dx{sf[8 * ns + s], sf[11 * ns + s]}, dy{sf[9 * ns + s], sf[12 * ns + s]},
                    dz{sf[10 * ns + s], sf[13 * ns + s]};
                dE = df_mul(df_add(df_add(df_mul(dx, ex), df_mul(dy, ey)), df_mul(dz, ez)), rinv);
                alpha = df_sub(df_add(df_add(df_mul(dx, ax), df_mul(dy, ay)), df_mul(dz, az)), df_mul(u, dE));
            }
            // n = 0: T_0 = 1, T'_0 = 0
            df T2{0.f, 0.f}, T1{1.f, 0.f}, D2{0.f, 0.f}, D1{0.f, 0.f};
            df L{1.f, 0.f}, sdp = df_neg(dE);  // sum of T_n; dipole part (times r), order by order
            if (SWEEP) acc[0] = df_add(acc[0], df_mul(rinv, df_sub(q, df_mul(dE, rinv))));
#pragma unroll
            for (int n = 1; n <= QM; ++n) {
                if (n > Q) break;
                const float4 cl = c_leg[n];
                const df Tn = df_sub(df_mul(df_mul(df{cl.x, cl.y}, xu), T1), df_mul(df_mul(df{cl.z, cl.w}, x2), T2));
                T2 = T1;
                T1 = Tn;
                if (!SWEEP) L = df_add(L, Tn);
                if (dip) {
                    const df Dn = df_add(df_mul(df_mul_f(x, 2.0f * n - 1.0f), T2), df_mul(x2, D2));
                    D2 = D1;
                    D1 = Dn;
                    const df term = df_sub(df_mul(alpha, Dn), df_mul(df_mul_f(dE, n + 1.0f), Tn));
                    if (SWEEP) acc[n] = df_add(acc[n], df_mul(rinv, df_add(df_mul(q, Tn), df_mul(term, rinv))));
                    else sdp = df_add(sdp, term);
                } else if (SWEEP) {
                    acc[n] = df_add(acc[n], df_mul(df_mul(rinv, q), Tn));
                }
            }
            if (!SWEEP) acc[0] = df_add(acc[0], df_mul(rinv, df_add(df_mul(q, L), df_mul(sdp, rinv))));
        }
    }
#pragma unroll
    for (int n = 0; n < (SWEEP ? QM + 1 : 1); ++n) {
        const df v = df_warp_sum(acc[n]);
        if (lane == 0) out[SWEEP ? (int64_t)n * nt + t : t] = df_to(v);
    }
}

// ---------------------------------------------------------------- Stage 9

// QBX targets: phi(t) = 1/(4 pi) sum A_k^l R_k^l((c - t)/rho), real part with conjugate symmetry.
template <int QM>
__global__ void k_qbxl2p(int64_t nt, const int *tperm, const double *txyz, const int *tgt_ctr, const int *ctr_rank,
                         int64_t nc, const double *cxyz, const double *cr, const signed char *qc, const double2 *A,
                         const double *pd, double *pot)
{
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nt) return;
    int t = tperm[it];
    int c = tgt_ctr[t];
    if (c < 0 || c >= nc) {
        if (c < -1 || c >= nc) pot[t] = CUDART_NAN;
        return;
    }
    int i = ctr_rank[c];
    int Q = min((int)qc[i], QM);
    double rinv = 1.0 / cr[i];
    double x = (cxyz[i] - txyz[it]) * rinv, y = (cxyz[nc + i] - txyz[nt + it]) * rinv,
           z = (cxyz[2 * nc + i] - txyz[2 * nt + it]) * rinv;
    double r2 = x * x + y * y + z * z;
    const double2 *Ac = A + (int64_t)i * ntri(QM);
    double acc = 0.0;
    double2 diag = make_double2(1.0, 0.0);
    for (int m = 0; m <= Q; ++m) {
        if (m > 0) diag = cscale(cmul(diag, make_double2(x, y)), 1.0 / (2.0 * m));
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        double wgt = m ? 2.0 : 1.0;
        double2 cv = Ac[tri(m, m)];
        acc += wgt * (cv.x * diag.x - cv.y * diag.y);
        for (int n = m + 1; n <= Q; ++n) {
            double inv = 1.0 / ((double)(n + m) * (double)(n - m));
            double2 v = make_double2(((2 * n - 1) * z * a1.x - r2 * a2.x) * inv, ((2 * n - 1) * z * a1.y - r2 * a2.y) * inv);
            double2 cc = Ac[tri(n, m)];
            acc += wgt * (cc.x * v.x - cc.y * v.y);
            a2 = a1;
            a1 = v;
        }
    }
    // the direct sources' part, summed at this target by k_qbx_direct (null: it is in A)
    pot[t] = INV4PI * (pd ? acc + pd[t] : acc);
}

// Point targets: P2P from List 1 / 3 close / 4 close, M2P from List 3 far, L2P of the box local.
template <int PM>
__global__ void k_points(int64_t nt, const int *tperm, const double *txyz, const int *tgt_ctr, const int *tgt_box,
                         const signed char *pb, const signed char *ps, ListRef lu, ListRef lwc, ListRef lxc, ListRef lwf,
                         const int *own_start, const double *sxyz, int64_t ns, const double *sq, const double *sd,
                         const double *cen, const double *hw, const double2 *Mu, const double2 *B, double *pot)
{
    int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + wl;
    if (it >= nt) return;
    int t = tperm[it];
    if (tgt_ctr[t] >= 0) return;
    int b = tgt_box[it];
    double tx = txyz[it], ty = txyz[nt + it], tz = txyz[2 * nt + it];
    double acc = 0.0;
    // P2P
    const ListRef lists[3] = {lu, lwc, lxc};
    for (int li = 0; li < 3; ++li)
        for (int e = lists[li].start[b]; e < lists[li].start[b + 1]; ++e) {
            int d = lists[li].idx[e];
            for (int s = own_start[d] + lane; s < own_start[d + 1]; s += 32) {
                double rx = tx - sxyz[s], ry = ty - sxyz[ns + s], rz = tz - sxyz[2 * ns + s];
                double r2 = rx * rx + ry * ry + rz * rz;
                if (r2 == 0.0) continue;
                double ri = 1.0 / sqrt(r2);
                double v = sq[s] * ri;
                if (sd) v += (sd[s] * rx + sd[ns + s] * ry + sd[2 * ns + s] * rz) * ri * ri * ri;
                acc += v;
            }
        }
    // M2P: one List 3 far box per lane
    for (int e = lwf.start[b] + lane; e < lwf.start[b + 1]; e += 32) {
        int d = lwf.idx[e];
        int P = ps[d];
        double hinv = 1.0 / hw[d];
        double x = (tx - cen[3 * d]) * hinv, y = (ty - cen[3 * d + 1]) * hinv, z = (tz - cen[3 * d + 2]) * hinv;
        double ir2 = 1.0 / (x * x + y * y + z * z);
        double2 wr = make_double2(x * ir2, y * ir2);
        double zz = z * ir2;
        const double2 *Md = Mu + (int64_t)d * ntri(PM);
        double2 diag = make_double2(sqrt(ir2), 0.0);
        double s = 0.0;
        for (int m = 0; m <= P; ++m) {
            if (m > 0) diag = cscale(cmul(diag, wr), 2.0 * m - 1.0);
            double wgt = m ? 2.0 : 1.0;
            double2 a2 = make_double2(0.0, 0.0), a1 = diag;
            double2 mv = Md[tri(m, m)];
            s += wgt * (mv.x * diag.x + mv.y * diag.y);
            for (int n = m + 1; n <= P; ++n) {
                double c1 = (2 * n - 1) * zz, c2 = (double)(n + m - 1) * (double)(n - m - 1) * ir2;
                double2 v = make_double2(c1 * a1.x - c2 * a2.x, c1 * a1.y - c2 * a2.y);
                double2 mm = Md[tri(n, m)];
                s += wgt * (mm.x * v.x + mm.y * v.y);
                a2 = a1;
                a1 = v;
            }
        }
        acc += s * hinv;
    }
    // L2P
    if (lane == 0) {
        int P = pb[b];
        double hinv = 1.0 / hw[b];
        double x = (cen[3 * b] - tx) * hinv, y = (cen[3 * b + 1] - ty) * hinv, z = (cen[3 * b + 2] - tz) * hinv;
        double r2 = x * x + y * y + z * z;
        const double2 *Lb = B + (int64_t)b * ntri(PM);
        double2 diag = make_double2(1.0, 0.0);
        for (int m = 0; m <= P; ++m) {
            if (m > 0) diag = cscale(cmul(diag, make_double2(x, y)), 1.0 / (2.0 * m));
            double wgt = m ? 2.0 : 1.0;
            double2 a2 = make_double2(0.0, 0.0), a1 = diag;
            double2 cv = Lb[tri(m, m)];
            acc += wgt * (cv.x * diag.x - cv.y * diag.y);
            for (int n = m + 1; n <= P; ++n) {
                double inv = 1.0 / ((double)(n + m) * (double)(n - m));
                double2 v = make_double2(((2 * n - 1) * z * a1.x - r2 * a2.x) * inv, ((2 * n - 1) * z * a1.y - r2 * a2.y) * inv);
                double2 cc = Lb[tri(n, m)];
                acc += wgt * (cc.x * v.x - cc.y * v.y);
                a2 = a1;
                a1 = v;
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) pot[t] = INV4PI * acc;
}

// Point targets with the List 3 far M2P spread over (target, box) pairs: the lists of point targets
// differ by orders of magnitude in length, so one thread per pair keeps the FP64 pipes busy.  The
// pairs are listed on the device on every evaluation (targets change role with tgt_ctr), their
// partial potentials are summed per target in list order (deterministic).
// pairs of each sorted target (every target when tgt_ctr is NULL); cnt[nt] = 0 closes the scan
__global__ void k_pt_count(int64_t nt, const int *tperm, const int *tgt_ctr, const int *tgt_box, const int *wfs,
                           int *cnt)
{
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it > nt) return;
    int c = 0;
    if (it < nt && (!tgt_ctr || tgt_ctr[tperm[it]] < 0)) {
        const int b = tgt_box[it];
        c = wfs[b + 1] - wfs[b];
    }
    cnt[it] = c;
}

__global__ void k_pt_fill(int64_t nt, const int *tgt_box, const int *wfs, const int *wfi, const int *off,
                          int *pair_it, int *pair_box)
{
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nt) return;
    const int o0 = off[it], n = off[it + 1] - o0;
    if (n == 0) return;
    const int b = tgt_box[it], e0 = wfs[b];
    for (int j = 0; j < n; ++j) {
        pair_it[o0 + j] = (int)it;
        pair_box[o0 + j] = wfi[e0 + j];
    }
}

// M2P of one (point target, List 3 far box) pair per thread: 1/h sum Mu_n^m conj S_n^m((t - c_d)/h).
template <int PM>
__global__ void k_m2p_pairs(int64_t cap, const int *total, const int *pair_it, const int *pair_box,
                            const double *txyz, int64_t nt, const signed char *pb, const double *cen, const double *hw,
                            const double2 *Mu, double *part)
{
    const int64_t np = *total;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np && e < cap;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int it = pair_it[e], d = pair_box[e];
        const int P = pb[d];
        const double hinv = 1.0 / hw[d];
        const double x = (txyz[it] - cen[3 * d]) * hinv, y = (txyz[nt + it] - cen[3 * d + 1]) * hinv,
                     z = (txyz[2 * nt + it] - cen[3 * d + 2]) * hinv;
        const double ir2 = 1.0 / (x * x + y * y + z * z);
        const double2 wr = make_double2(x * ir2, y * ir2);
        const double zz = z * ir2;
        const double2 *Md = Mu + (int64_t)d * ntri(PM);
        double2 diag = make_double2(sqrt(ir2), 0.0);
        double s = 0.0;
        for (int m = 0; m <= P; ++m) {
            if (m > 0) diag = cscale(cmul(diag, wr), 2.0 * m - 1.0);
            const double wgt = m ? 2.0 : 1.0;
            double2 a2 = make_double2(0.0, 0.0), a1 = diag;
            double2 mv = Md[tri(m, m)];
            double sm = mv.x * diag.x + mv.y * diag.y;
            for (int n = m + 1; n <= P; ++n) {
                const double c1 = (2 * n - 1) * zz, c2 = (double)(n + m - 1) * (double)(n - m - 1) * ir2;
                double2 v = make_double2(c1 * a1.x - c2 * a2.x, c1 * a1.y - c2 * a2.y);
                double2 mm = Md[tri(n, m)];
                sm = fma(mm.x, v.x, fma(mm.y, v.y, sm));
                a2 = a1;
                a1 = v;
            }
            s = fma(wgt, sm, s);
        }
        part[e] = s * hinv;
    }
}

// Point targets: P2P from List 1 / 3 close / 4 close, the M2P partials of List 3 far, L2P.
template <int PM>
__global__ void k_points2(int64_t nt, const int *tperm, const double *txyz, const int *tgt_ctr, const int *tgt_box,
                          const signed char *pb, ListRef lu, ListRef lwc, ListRef lxc, const int *pt_off,
                          const double *part, const int *own_start, const double *sxyz, int64_t ns, const double *sq,
                          const double *sd, const double *cen, const double *hw, const double2 *B, double *pot)
{
    int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + wl;
    if (it >= nt) return;
    int t = tperm[it];
    if (tgt_ctr[t] >= 0) return;
    int b = tgt_box[it];
    double tx = txyz[it], ty = txyz[nt + it], tz = txyz[2 * nt + it];
    double acc = 0.0;
    // P2P: the sources of Lists 1, 3 close and 4 close as one sequence over the lanes (shuffle
    // prefix scan of the box source counts, 32 boxes at a time)
    {
        const int u0 = lu.start[b], n0 = lu.start[b + 1] - u0;
        const int w0 = lwc.start[b], n1 = lwc.start[b + 1] - w0;
        const int x0 = lxc.start[b], n2 = lxc.start[b + 1] - x0;
        const int e1 = n0 + n1 + n2;
        for (int base = 0; base < e1; base += 32) {
            const int e = base + lane;
            int d = -1;
            if (e < n0) d = lu.idx[u0 + e];
            else if (e < n0 + n1) d = lwc.idx[w0 + e - n0];
            else if (e < e1) d = lxc.idx[x0 + e - n0 - n1];
            const int s0 = d >= 0 ? own_start[d] : 0;
            const int cnt = d >= 0 ? own_start[d + 1] - s0 : 0;
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int k0 = 0; k0 < total; k0 += 32) {
                const int k = k0 + lane;
                int j = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
                    if (v <= k) j += step;
                }
                const int sj = __shfl_sync(0xffffffffu, s0, j);
                const int ij = __shfl_sync(0xffffffffu, incl, j);
                const int cj = __shfl_sync(0xffffffffu, cnt, j);
                if (k < total) {
                    const int s = sj + (k - (ij - cj));
                    double rx = tx - sxyz[s], ry = ty - sxyz[ns + s], rz = tz - sxyz[2 * ns + s];
                    double r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 != 0.0) {
                        double ri = 1.0 / sqrt(r2);
                        double v = sq[s] * ri;
                        if (sd) v += (sd[s] * rx + sd[ns + s] * ry + sd[2 * ns + s] * rz) * ri * ri * ri;
                        acc += v;
                    }
                }
            }
        }
    }
    for (int e = pt_off[it] + lane; e < pt_off[it + 1]; e += 32) acc += part[e];
    if (lane == 0) {
        int P = pb[b];
        double hinv = 1.0 / hw[b];
        double x = (cen[3 * b] - tx) * hinv, y = (cen[3 * b + 1] - ty) * hinv, z = (cen[3 * b + 2] - tz) * hinv;
        double r2 = x * x + y * y + z * z;
        const double2 *Lb = B + (int64_t)b * ntri(PM);
        double2 diag = make_double2(1.0, 0.0);
        for (int m = 0; m <= P; ++m) {
            if (m > 0) diag = cscale(cmul(diag, make_double2(x, y)), 1.0 / (2.0 * m));
            double wgt = m ? 2.0 : 1.0;
            double2 a2 = make_double2(0.0, 0.0), a1 = diag;
            double2 cv = Lb[tri(m, m)];
            acc += wgt * (cv.x * diag.x - cv.y * diag.y);
            for (int n = m + 1; n <= P; ++n) {
                double inv = 1.0 / ((double)(n + m) * (double)(n - m));
                double2 v = make_double2(((2 * n - 1) * z * a1.x - r2 * a2.x) * inv, ((2 * n - 1) * z * a1.y - r2 * a2.y) * inv);
                double2 cc = Lb[tri(n, m)];
                acc += wgt * (cc.x * v.x - cc.y * v.y);
                a2 = a1;
                a1 = v;
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) pot[t] = INV4PI * acc;
}

// ---------------------------------------------------------------- driver

static int read_flags(const int *f, cudaStream_t st)
{
    int v = 0;
    QBX_CUDA_TRY(cudaMemcpyAsync(&v, f, sizeof(int), cudaMemcpyDeviceToHost, st));
    QBX_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

constexpr int PM_T = 20;  // compile-time order bound of the box-expansion kernels
constexpr int QB[] = {4, 8, 12, 16};

template <int QM>
static void launch_centers(const qbx_tree *T, qbx_lists *L, qbx_workspace *ws, bool dip, const int *tgt_ctr,
                           double *pot, cudaStream_t st, WfarPlan *wf = nullptr)
{
    stage_mark(L, 6, st);
    // with a mixed List 3 far plan the FP64 kernel sees an empty List 3 far and the plan's
    // products are added to the QBX locals before they are evaluated
    const int *wf_start = wf ? wfar_empty_start(wf) : L->start[LWF];
    const int WPB = 4;
    size_t smem = (size_t)WPB * (ntri(PM_T + QM) + PM_T + 1) * sizeof(double2);
    static bool attr_set = false;
    if (!attr_set) {
        QBX_CUDA_TRY(cudaFuncSetAttribute(k_centers<QM, PM_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    // k_centers runs when it has work (List 3 far in FP64); k_l2qbxl then adds the box local's part
    const bool far64 = wf == nullptr;
    if (T->np[KCTR] > 0 && far64) {
        k_centers<QM, PM_T><<<nblocks(T->np[KCTR], WPB), 32 * WPB, smem, st>>>(
            T->np[KCTR], T->ctr_box, T->cxyz, T->cr, ws->qc, ws->ps, ListRef{L->start[LU], L->idx[LU]},
            ListRef{L->start[LWC], L->idx[LWC]}, ListRef{L->start[LXC], L->idx[LXC]},
            ListRef{wf_start, L->idx[LWF]}, T->own_start[KSRC], T->sxyz, T->np[KSRC], ws->sq,
            dip ? ws->sd : nullptr, T->cen, T->hw, ws->Mu, ws->A, 0);
        QBX_LAUNCH_CHECK();
    }
    if (T->np[KCTR] > 0) {
        k_l2qbxl<QM><<<nblocks(T->np[KCTR], 128), 128, 0, st>>>(T->np[KCTR], T->ctr_box, T->cxyz, T->cr, ws->qc,
                                                                ws->pb, T->cen, T->hw, ws->Bf, ntri(PM_T), ws->A,
                                                                far64 ? 1 : 0);
        QBX_LAUNCH_CHECK();
    }
    if (T->np[KTGT] > 0 && T->np[KCTR] > 0) {
        k_qbx_direct<QM, false><<<nblocks(T->np[KTGT], 4), 128, 0, st>>>(
            T->np[KTGT], T->perm[KTGT], ws->tf, tgt_ctr, T->ctr_rank, T->ctr_box, T->np[KCTR], ws->cf, ws->qc,
            ListRef{L->start[LU], L->idx[LU]}, ListRef{L->start[LWC], L->idx[LWC]}, ListRef{L->start[LXC], L->idx[LXC]},
            T->own_start[KSRC], T->np[KSRC], ws->sf, dip ? 1 : 0, ws->pd);
        QBX_LAUNCH_CHECK();
    }
    stage_mark(L, 7, st);
    if (T->np[KCTR] > 0 && wf) wfar_mixed_reduce(T, wf, QM, ws->qc, ws->A, st);
    stage_mark(L, 8, st);
    if (T->np[KTGT] > 0) {
        k_qbxl2p<QM><<<nblocks(T->np[KTGT], 128), 128, 0, st>>>(T->np[KTGT], T->perm[KTGT], T->txyz, tgt_ctr,
                                                                T->ctr_rank, T->np[KCTR], T->cxyz, T->cr, ws->qc,
                                                                ws->A, T->np[KCTR] > 0 ? ws->pd : nullptr, pot);
        QBX_LAUNCH_CHECK();
    }
}

void eval(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu, const double *nrm,
          const int *tgt_ctr, const qbx_eval_opts *o, double *pot, cudaStream_t st)
{
    const int64_t nb = T->nb, ns = T->np[KSRC], nc = T->np[KCTR], nt = T->np[KTGT];
    // orders: compile-time bucket for the QBX order, runtime orders per center / box
    const int qmax = o->p_qbx, pmax = o->p_fmm;  // fixed orders, or bounds of the per-center / per-box arrays
    int QM = 0;
    for (int qb : QB)
        if (qmax <= qb) { QM = qb; break; }
    qbx_workspace *ws = L->ws;
    if (!ws || ws->QM < QM || ws->PM < 0) {
        if (ws) free_workspace(ws);
        ws = L->ws = new qbx_workspace();
        ws->PM = PM_T;
        ws->QM = QM;
        ws->nb = nb; ws->nc = nc; ws->ns = ns;
        ws->Mu = dalloc<double2>(nb * ntri(PM_T));
        ws->B = dalloc<double2>(nb * ntri(PM_T));
        ws->Bf = dalloc<float4>(nb * ntri(PM_T));
        ws->Muf = dalloc<float4>(nb * ntri(PM_T));
        ws->octf = dalloc<float4>(8 * ntri(PM_T));
        ws->A = dalloc<double2>(std::max<int64_t>(nc, 1) * ntri(QM));
        ws->m2l_tab = dalloc<double2>((int64_t)1331 * ntri(2 * PM_T));
        ws->oct_tab = dalloc<double2>(8 * ntri(PM_T));
        ws->sq = dalloc<double>(ns);
        ws->sd = dalloc<double>(3 * ns);
        ws->pd = dalloc<double>(std::max<int64_t>(nt, 1));
        ws->sf = dalloc<float>(14 * std::max<int64_t>(ns, 1));
        ws->cf = dalloc<float>(6 * std::max<int64_t>(nc, 1));
        ws->tf = dalloc<float>(6 * std::max<int64_t>(nt, 1));
        ws->qc = dalloc<signed char>(nc);
        ws->pb = dalloc<signed char>(nb);
        ws->ps = dalloc<signed char>(nb);
        ws->flags = dalloc<int>(1);
        set_l2q_tables(st);
        set_leg_table(st);
        k_m2l_table<<<nblocks(1331, 64), 64, 0, st>>>(2 * PM_T, ws->m2l_tab);
        k_oct_table<<<1, 32, 0, st>>>(PM_T, ws->oct_tab);
        k_c2df<<<nblocks(8 * ntri(PM_T), 256), 256, 0, st>>>(8 * ntri(PM_T), ws->oct_tab, ws->octf);
        QBX_LAUNCH_CHECK();
    }
    (void)pot;
    stage_mark(L, 0, st);
    QBX_CUDA_TRY(cudaMemsetAsync(ws->flags, 0, sizeof(int), st));
    k_prep_src<<<nblocks(ns, 256), 256, 0, st>>>(T->perm[KSRC], ns, w, sigma, mu, nrm, ws->sq, ws->sd, ws->flags);
    if (ns > 0) k_to_df<<<nblocks(ns, 256), 256, 0, st>>>(ns, T->sxyz, ws->sq, mu ? ws->sd : nullptr, ws->sf);
    if (nc > 0) k_to_df<<<nblocks(nc, 256), 256, 0, st>>>(nc, T->cxyz, nullptr, nullptr, ws->cf);
    if (nt > 0) k_to_df<<<nblocks(nt, 256), 256, 0, st>>>(nt, T->txyz, nullptr, nullptr, ws->tf);
    k_prep_orders<<<nblocks(std::max(nb, nc), 256), 256, 0, st>>>(T->perm[KCTR], nc, o->p_qbx_per_ctr, o->p_qbx, nb,
                                                                  o->p_fmm_per_box, o->p_fmm, ws->qc, ws->pb, ws->ps,
                                                                  ws->flags);
    k_check_tgt<<<nblocks(nt, 256), 256, 0, st>>>(tgt_ctr, nt, nc, ws->flags);
    QBX_LAUNCH_CHECK();
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    QBX_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone) {
        int f = read_flags(ws->flags, st);
        if (f & 1) throw Error{QBX_ERR_INVALID_ARG, "source weight <= 0 or non-finite density/normal"};
        if (f & 2) throw Error{QBX_ERR_INVALID_ARG, "expansion order out of range"};
        if (f & 4) throw Error{QBX_ERR_INVALID_ARG, "tgt_ctr entry out of range"};
    }
    QBX_CUDA_TRY(cudaMemsetAsync(ws->Mu, 0, nb * ntri(PM_T) * sizeof(double2), st));
    QBX_CUDA_TRY(cudaMemsetAsync(ws->B, 0, nb * ntri(PM_T) * sizeof(double2), st));

    const int WPB = 4;
    const bool dip = mu != nullptr;
    // Stage 2
    stage_mark(L, 1, st);
    // the P2M and P2L kernels unroll their rows: instantiate them for the smallest order bound that covers p_fmm
#define QBX_P2M(PB)                                                                                                 \
    k_p2m_df<PB, ntri(PM_T)><<<nblocks(nb, WPB), 32 * WPB, 0, st>>>(nb, T->own_start[KSRC], ns, ws->sf, dip ? 1 : 0,   \
                                                                    T->cen, T->hw, ws->ps, ws->Mu, ws->Muf)
    if (pmax <= 10) QBX_P2M(10);
    else if (pmax <= 16) QBX_P2M(16);
    else QBX_P2M(PM_T);
#undef QBX_P2M
    QBX_LAUNCH_CHECK();
    for (int l = (int)T->nlev - 2; l >= 0; --l) {
        int b0 = T->level_start[l], b1 = T->level_start[l + 1];
        if (b1 > b0)
            k_m2m8_df<PM_T><<<b1 - b0, 256, 0, st>>>(b0, b1, T->lvl_boxes, T->child, T->nsrc_sub, ws->ps, ws->octf,
                                                     ws->Mu, ws->Muf);
        QBX_LAUNCH_CHECK();
    }
    // reduced precision per stage: QBX_MIXED_*_ONLY keeps the other stage in FP64
    const int pbase = o->precision & 0xF;
    const bool tc = pbase == QBX_M2L_3XTF32;
    const bool m2l_mixed = pbase != QBX_FP64 && !(o->precision & QBX_MIXED_M2QBXL_ONLY);
    const bool wfar_mixed = pbase != QBX_FP64 && !(o->precision & QBX_MIXED_M2L_ONLY);
    // Stage 4
    stage_mark(L, 2, st);
    if (!m2l_mixed) {
        size_t smem = (size_t)WPB * ntri(PM_T) * sizeof(double2);
        k_m2l<PM_T><<<nblocks(nb, WPB), 32 * WPB, smem, st>>>(nb, L->start[LV], L->idx[LV], T->ic, T->hw, ws->pb,
                                                              ws->ps, ws->Mu, ws->m2l_tab, ws->B);
        QBX_LAUNCH_CHECK();
    } else {
        const int Pm = o->p_fmm;
        const int mkey = (Pm * 2 + (tc ? 1 : 0)) * 64 + L->tile_m2l_kc;
        if (!ws->m2l || ws->m2l_key != mkey) {
            free_m2l_plan(ws->m2l);
            ws->m2l = nullptr;
            ws->m2l = m2l_plan_build(T, L, Pm, PM_T, ws->m2l_tab, tc, L->tile_m2l_kc, st);
            ws->m2l_key = mkey;
        }
        m2l_mixed_run(T, L, ws->m2l, PM_T, ws->Mu, ws->B, ws->pb, ws->flags, st);
    }
    // Stage 6(b)
    stage_mark(L, 3, st);
#define QBX_P2L(PB)                                                                                                 \
    k_p2l4_df<PB, PM_T><<<(unsigned)nb, 128, 0, st>>>(nb, L->start[LXF], L->idx[LXF], T->own_start[KSRC], ns, ws->sf, \
                                                      dip ? 1 : 0, T->cen, T->hw, ws->pb, ws->B)
    if (pmax <= 10) QBX_P2L(10);
    else if (pmax <= 16) QBX_P2L(16);
    else QBX_P2L(PM_T);
#undef QBX_P2L
    QBX_LAUNCH_CHECK();
    // Stage 7
    stage_mark(L, 4, st);
    {
        const int r0 = T->level_start[0], r1 = T->level_start[1];
        k_level_to_df<<<nblocks((int64_t)(r1 - r0) * ntri(PM_T), 256), 256, 0, st>>>(r0, r1, T->lvl_boxes, ntri(PM_T),
                                                                                      ws->pb, ws->B, ws->Bf);
        QBX_LAUNCH_CHECK();
    }
    for (int l = 1; l < T->nlev; ++l) {
        int b0 = T->level_start[l], b1 = T->level_start[l + 1];
#define QBX_L2L(PB)                                                                                                 \
    k_l2l_df<PB><<<nblocks((int64_t)(b1 - b0) * l2x_npass(PB), 128), 128, 0, st>>>(                                  \
        b0, b1, T->lvl_boxes, T->parent, T->ntgt_sub, T->child, ws->pb, ws->octf, ntri(PM_T), ws->B, ws->Bf)
        if (pmax <= 10) QBX_L2L(10);
        else if (pmax <= 16) QBX_L2L(16);
        else QBX_L2L(PM_T);
#undef QBX_L2L
        QBX_LAUNCH_CHECK();
    }
    // Stage 5(b) in mixed precision: List 3 far products, reduced into the QBX locals below
    stage_mark(L, 5, st);
    WfarPlan *wf = nullptr;
    if (wfar_mixed && T->np[KCTR] > 0) {
        const int Pm = o->p_fmm, Qm = o->p_qbx;
        const int wkey = ((Pm * 100 + Qm) * 2 + (tc ? 1 : 0)) * 256 + L->tile_wfar_w;
        if (!ws->wfar || ws->wfar_key != wkey) {
            free_wfar_plan(ws->wfar);
            ws->wfar = nullptr;
            ws->wfar = wfar_plan_build(T, L, Pm, Qm, tc, L->tile_wfar_w, st);
            ws->wfar_key = wkey;
        }
        wf = ws->wfar;
        wfar_mixed_run(T, wf, PM_T, ws->Mu, ws->ps, ws->cf, ws->flags, L->wait_limit, L->probe_step, st);
    }
    // Stages 3, 5, 6(a), 8, 9 at QBX centers and their targets
    switch (QM) {
    case 4: launch_centers<4>(T, L, ws, dip, tgt_ctr, pot, st, wf); break;
    case 8: launch_centers<8>(T, L, ws, dip, tgt_ctr, pot, st, wf); break;
    case 12: launch_centers<12>(T, L, ws, dip, tgt_ctr, pot, st, wf); break;
    default: launch_centers<16>(T, L, ws, dip, tgt_ctr, pot, st, wf); break;
    }
    // Stage 9 at point targets
    stage_mark(L, 9, st);
    if (nt > 0) {
        if (ws->pt_cap < 0) {  // first evaluation: size the pair buffers for any choice of point targets
            ws->pt_cnt = dalloc<int>(nt + 1);
            ws->pt_off = dalloc<int>(nt + 1);
            ws->pt_total = dalloc<int>(1);
            k_pt_count<<<nblocks(nt + 1, 256), 256, 0, st>>>(nt, T->perm[KTGT], nullptr, T->tgt_box, L->start[LWF],
                                                             ws->pt_cnt);
            QBX_LAUNCH_CHECK();
            exclusive_scan(ws->pt_cnt, ws->pt_off, nt + 1, 0, ws->pt_total, st);
            int cap = 0;
            QBX_CUDA_TRY(cudaMemcpyAsync(&cap, ws->pt_total, sizeof(int), cudaMemcpyDeviceToHost, st));
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            ws->pt_cap = cap;
            ws->pt_it = dalloc<int>(std::max(cap, 1));
            ws->pt_box = dalloc<int>(std::max(cap, 1));
            ws->pt_part = dalloc<double>(std::max(cap, 1));
        }
        k_pt_count<<<nblocks(nt + 1, 256), 256, 0, st>>>(nt, T->perm[KTGT], tgt_ctr, T->tgt_box, L->start[LWF],
                                                         ws->pt_cnt);
        QBX_LAUNCH_CHECK();
        exclusive_scan(ws->pt_cnt, ws->pt_off, nt + 1, 0, ws->pt_total, st);
        k_pt_fill<<<nblocks(nt, 256), 256, 0, st>>>(nt, T->tgt_box, L->start[LWF], L->idx[LWF], ws->pt_off, ws->pt_it,
                                                    ws->pt_box);
        QBX_LAUNCH_CHECK();
        if (ws->pt_cap > 0) {
            const unsigned grid = std::min<unsigned>(nblocks(ws->pt_cap, 128), 152 * 64);
            k_m2p_pairs<PM_T><<<grid, 128, 0, st>>>(ws->pt_cap, ws->pt_total, ws->pt_it, ws->pt_box, T->txyz, nt, ws->ps,
                                                     T->cen, T->hw, ws->Mu, ws->pt_part);
            QBX_LAUNCH_CHECK();
        }
        k_points2<PM_T><<<nblocks(nt, WPB), 32 * WPB, 0, st>>>(
            nt, T->perm[KTGT], T->txyz, tgt_ctr, T->tgt_box, ws->pb, ListRef{L->start[LU], L->idx[LU]},
            ListRef{L->start[LWC], L->idx[LWC]}, ListRef{L->start[LXC], L->idx[LXC]}, ws->pt_off, ws->pt_part,
            T->own_start[KSRC], T->sxyz, ns, ws->sq, dip ? ws->sd : nullptr, T->cen, T->hw, ws->B, pot);
        QBX_LAUNCH_CHECK();
    }
    stage_mark(L, 10, st);
    L->prof_valid = L->prof;
    if (tc && cap == cudaStreamCaptureStatusNone) {
        // the tensor-core kernels report a wait that gave up through the flags word
        if (read_flags(ws->flags, st) & 8) throw Error{QBX_ERR_TIMEOUT, "a tensor-core pipeline wait timed out"};
    }
}

}  // namespace qbx

// ---------------------------------------------------------------- order sweep of the QBX locals

namespace qbx {

template <int QM>
__global__ void k_qbx_partials(int64_t nt, int Q, const int *tperm, const double *txyz, const int *tgt_ctr,
                               const int *ctr_rank, int64_t nc, const double *cxyz, const double *cr,
                               const double2 *A, const double *dir, double *partial)
{
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nt) return;
    int t = tperm[it];
    int c = tgt_ctr[t];
    if (c < 0 || c >= nc) {
        double v = partial[t];  // column 0 holds the point-target potential
        for (int q = 1; q <= Q; ++q) partial[(int64_t)q * nt + t] = v;
        return;
    }
    int i = ctr_rank[c];
    double rinv = 1.0 / cr[i];
    double x = (cxyz[i] - txyz[it]) * rinv, y = (cxyz[nc + i] - txyz[nt + it]) * rinv,
           z = (cxyz[2 * nc + i] - txyz[2 * nt + it]) * rinv;
    double r2 = x * x + y * y + z * z;
    const double2 *Ac = A + (int64_t)i * ntri(QM);
    double row[QMAX + 1];
    for (int k = 0; k <= Q; ++k) row[k] = 0.0;
    double2 diag = make_double2(1.0, 0.0);
    for (int m = 0; m <= Q; ++m) {
        if (m > 0) diag = cscale(cmul(diag, make_double2(x, y)), 1.0 / (2.0 * m));
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        double wgt = m ? 2.0 : 1.0;
        double2 cv = Ac[tri(m, m)];
        row[m] += wgt * (cv.x * diag.x - cv.y * diag.y);
        for (int n = m + 1; n <= Q; ++n) {
            double inv = 1.0 / ((double)(n + m) * (double)(n - m));
            double2 v = make_double2(((2 * n - 1) * z * a1.x - r2 * a2.x) * inv, ((2 * n - 1) * z * a1.y - r2 * a2.y) * inv);
            double2 cc = Ac[tri(n, m)];
            row[n] += wgt * (cc.x * v.x - cc.y * v.y);
            a2 = a1;
            a1 = v;
        }
    }
    double acc = 0.0;
    for (int k = 0; k <= Q; ++k) {
        acc += row[k] + dir[(int64_t)k * nt + t];  // the direct sources' order-k part (k_qbx_direct)
        partial[(int64_t)k * nt + t] = INV4PI * acc;
    }
}

void eval_order_sweep(const qbx_tree *T, qbx_lists *L, const double *w, const double *sigma, const double *mu,
                      const double *nrm, const int *tgt_ctr, const qbx_eval_opts *o, double *partial, cudaStream_t st)
{
    eval(T, L, w, sigma, mu, nrm, tgt_ctr, o, partial, st);
    const int64_t nt = T->np[KTGT];
    if (nt == 0) return;
    qbx_workspace *ws = L->ws;
    const bool dip = mu != nullptr;
    double *dir = dalloc<double>((int64_t)(ws->QM + 1) * nt);
    try {
        QBX_CUDA_TRY(cudaMemsetAsync(dir, 0, (size_t)(ws->QM + 1) * nt * sizeof(double), st));
        switch (ws->QM) {
#define QBX_PARTIALS(QB)                                                                                        \
    case QB:                                                                                                     \
        if (T->np[KCTR] > 0)                                                                                     \
            k_qbx_direct<QB, true><<<nblocks(nt, 4), 128, 0, st>>>(                                              \
                nt, T->perm[KTGT], ws->tf, tgt_ctr, T->ctr_rank, T->ctr_box, T->np[KCTR], ws->cf, ws->qc,         \
                ListRef{L->start[LU], L->idx[LU]}, ListRef{L->start[LWC], L->idx[LWC]},                          \
                ListRef{L->start[LXC], L->idx[LXC]}, T->own_start[KSRC], T->np[KSRC], ws->sf, dip ? 1 : 0, dir);     \
        k_qbx_partials<QB><<<nblocks(nt, 128), 128, 0, st>>>(nt, o->p_qbx, T->perm[KTGT], T->txyz, tgt_ctr,     \
                                                            T->ctr_rank, T->np[KCTR], T->cxyz, T->cr, ws->A,    \
                                                            dir, partial);                                      \
        break;
        QBX_PARTIALS(4)
        QBX_PARTIALS(8)
        QBX_PARTIALS(12)
        QBX_PARTIALS(16)
#undef QBX_PARTIALS
        }
        QBX_LAUNCH_CHECK();
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(dir);
        throw;
    }
    dfree(dir);
}

}  // namespace qbx

// ---------------------------------------------------------------- evaluation on caller-provided storage
//
// Same stages and kernels as eval(), with every scratch buffer carved out of `base` (at least
// fixed_workspace_bytes() bytes, 256-byte aligned).  Nothing is allocated.  Used by the
// no-allocation entry point; the tables are regenerated on every call.

namespace qbx {

static size_t carve(size_t &off, size_t bytes)
{
    size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
}

static int fixed_qbucket(const qbx_eval_opts *o)
{
    int qmax = o->p_qbx;
    for (int qb : QB)
        if (qmax <= qb) return qb;
    return 16;
}

size_t fixed_workspace_bytes(const qbx_tree *T, const qbx_eval_opts *o)
{
    const int64_t nb = T->nb, ns = T->np[KSRC], nc = T->np[KCTR];
    const int QM = fixed_qbucket(o);
    size_t off = 0;
    carve(off, (size_t)nb * ntri(PM_T) * sizeof(double2));                 // Mu
    carve(off, (size_t)nb * ntri(PM_T) * sizeof(double2));                 // B
    carve(off, (size_t)nb * ntri(PM_T) * sizeof(float4));                  // B as double-floats
    carve(off, (size_t)std::max<int64_t>(nc, 1) * ntri(QM) * sizeof(double2));  // A
    carve(off, (size_t)1331 * ntri(2 * PM_T) * sizeof(double2));           // List 2 offset table
    carve(off, (size_t)8 * ntri(PM_T) * sizeof(double2));                  // octant table
    carve(off, (size_t)std::max<int64_t>(ns, 1) * sizeof(double));         // charges
    carve(off, (size_t)3 * std::max<int64_t>(ns, 1) * sizeof(double));     // dipoles
    carve(off, (size_t)std::max<int64_t>(nc, 1));                           // per-center orders
    carve(off, (size_t)std::max<int64_t>(nb, 1));                           // per-box local orders
    carve(off, (size_t)std::max<int64_t>(nb, 1));                           // per-box multipole orders
    carve(off, sizeof(int));                                                // flags
    return off;
}

template <int QM>
static void fixed_centers(const qbx_tree *T, const qbx_lists *L, const qbx_workspace &ws, bool dip,
                          const int *tgt_ctr, double *pot, cudaStream_t st)
{
    const int WPB = 4;
    size_t smem = (size_t)WPB * (ntri(PM_T + QM) + PM_T + 1) * sizeof(double2);
    QBX_CUDA_TRY(cudaFuncSetAttribute(k_centers<QM, PM_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (T->np[KCTR] > 0) {
        k_centers<QM, PM_T><<<nblocks(T->np[KCTR], WPB), 32 * WPB, smem, st>>>(
            T->np[KCTR], T->ctr_box, T->cxyz, T->cr, ws.qc, ws.ps, ListRef{L->start[LU], L->idx[LU]},
            ListRef{L->start[LWC], L->idx[LWC]}, ListRef{L->start[LXC], L->idx[LXC]},
            ListRef{L->start[LWF], L->idx[LWF]}, T->own_start[KSRC], T->sxyz, T->np[KSRC], ws.sq,
            dip ? ws.sd : nullptr, T->cen, T->hw, ws.Mu, ws.A, 1);
        QBX_LAUNCH_CHECK();
        k_locals_to_df<<<nblocks(T->nb * ntri(PM_T), 256), 256, 0, st>>>(T->nb, ntri(PM_T), ws.pb, ws.B, ws.Bf);
        k_l2qbxl<QM><<<nblocks(T->np[KCTR], 128), 128, 0, st>>>(T->np[KCTR], T->ctr_box, T->cxyz, T->cr, ws.qc, ws.pb,
                                                                T->cen, T->hw, ws.Bf, ntri(PM_T), ws.A, 1);
        QBX_LAUNCH_CHECK();
    }
    if (T->np[KTGT] > 0) {
        k_qbxl2p<QM><<<nblocks(T->np[KTGT], 128), 128, 0, st>>>(T->np[KTGT], T->perm[KTGT], T->txyz, tgt_ctr,
                                                                T->ctr_rank, T->np[KCTR], T->cxyz, T->cr, ws.qc,
                                                                ws.A, nullptr, pot);
        QBX_LAUNCH_CHECK();
    }
}

void eval_fixed(const qbx_tree *T, const qbx_lists *L, unsigned char *base, size_t cap, const double *w,
                const double *sigma, const double *mu, const double *nrm, const int *tgt_ctr,
                const qbx_eval_opts *o, double *pot, cudaStream_t st)
{
    const int64_t nb = T->nb, ns = T->np[KSRC], nc = T->np[KCTR], nt = T->np[KTGT];
    if (fixed_workspace_bytes(T, o) > cap) throw Error{QBX_ERR_INVALID_ARG, "problem exceeds the fixed scratch"};
    const int QM = fixed_qbucket(o);
    qbx_workspace ws;  // a view into `base`; owns nothing
    size_t off = 0;
    ws.Mu = reinterpret_cast<double2 *>(base + carve(off, (size_t)nb * ntri(PM_T) * sizeof(double2)));
    ws.B = reinterpret_cast<double2 *>(base + carve(off, (size_t)nb * ntri(PM_T) * sizeof(double2)));
    ws.Bf = reinterpret_cast<float4 *>(base + carve(off, (size_t)nb * ntri(PM_T) * sizeof(float4)));
    ws.A = reinterpret_cast<double2 *>(base + carve(off, (size_t)std::max<int64_t>(nc, 1) * ntri(QM) * sizeof(double2)));
    ws.m2l_tab = reinterpret_cast<double2 *>(base + carve(off, (size_t)1331 * ntri(2 * PM_T) * sizeof(double2)));
    ws.oct_tab = reinterpret_cast<double2 *>(base + carve(off, (size_t)8 * ntri(PM_T) * sizeof(double2)));
    ws.sq = reinterpret_cast<double *>(base + carve(off, (size_t)std::max<int64_t>(ns, 1) * sizeof(double)));
    ws.sd = reinterpret_cast<double *>(base + carve(off, (size_t)3 * std::max<int64_t>(ns, 1) * sizeof(double)));
    ws.qc = reinterpret_cast<signed char *>(base + carve(off, (size_t)std::max<int64_t>(nc, 1)));
    ws.pb = reinterpret_cast<signed char *>(base + carve(off, (size_t)std::max<int64_t>(nb, 1)));
    ws.ps = reinterpret_cast<signed char *>(base + carve(off, (size_t)std::max<int64_t>(nb, 1)));
    ws.flags = reinterpret_cast<int *>(base + carve(off, sizeof(int)));
    ws.PM = PM_T;
    ws.QM = QM;

    set_l2q_tables(st);
    set_leg_table(st);
    k_m2l_table<<<nblocks(1331, 64), 64, 0, st>>>(2 * PM_T, ws.m2l_tab);
    k_oct_table<<<1, 32, 0, st>>>(PM_T, ws.oct_tab);
    QBX_LAUNCH_CHECK();
    QBX_CUDA_TRY(cudaMemsetAsync(ws.flags, 0, sizeof(int), st));
    k_prep_src<<<nblocks(ns, 256), 256, 0, st>>>(T->perm[KSRC], ns, w, sigma, mu, nrm, ws.sq, ws.sd, ws.flags);
    k_prep_orders<<<nblocks(std::max(nb, nc), 256), 256, 0, st>>>(T->perm[KCTR], nc, o->p_qbx_per_ctr, o->p_qbx, nb,
                                                                  o->p_fmm_per_box, o->p_fmm, ws.qc, ws.pb, ws.ps,
                                                                  ws.flags);
    k_check_tgt<<<nblocks(nt, 256), 256, 0, st>>>(tgt_ctr, nt, nc, ws.flags);
    QBX_LAUNCH_CHECK();
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    QBX_CUDA_TRY(cudaStreamIsCapturing(st, &cap_st));
    if (cap_st == cudaStreamCaptureStatusNone) {
        int f = read_flags(ws.flags, st);
        if (f & 1) throw Error{QBX_ERR_INVALID_ARG, "source weight <= 0 or non-finite density/normal"};
        if (f & 2) throw Error{QBX_ERR_INVALID_ARG, "expansion order out of range"};
        if (f & 4) throw Error{QBX_ERR_INVALID_ARG, "tgt_ctr entry out of range"};
    }
    // the expansions accumulate: they must start at zero on every call
    QBX_CUDA_TRY(cudaMemsetAsync(ws.Mu, 0, nb * ntri(PM_T) * sizeof(double2), st));
    QBX_CUDA_TRY(cudaMemsetAsync(ws.B, 0, nb * ntri(PM_T) * sizeof(double2), st));
    const int WPB = 4;
    const bool dip = mu != nullptr;
    k_p2m<PM_T><<<nblocks(nb, WPB), 32 * WPB, 0, st>>>(nb, T->own_start[KSRC], T->sxyz, ns, ws.sq,
                                                       dip ? ws.sd : nullptr, T->cen, T->hw, ws.ps, ws.Mu);
    QBX_LAUNCH_CHECK();
    for (int l = (int)T->nlev - 2; l >= 0; --l) {
        int b0 = T->level_start[l], b1 = T->level_start[l + 1];
        k_m2m<PM_T><<<nblocks(b1 - b0, WPB), 32 * WPB, 0, st>>>(b0, b1, T->lvl_boxes, T->child, T->nsrc_sub, ws.ps, ws.oct_tab, ws.Mu);
        QBX_LAUNCH_CHECK();
    }
    k_m2l<PM_T><<<nblocks(nb, WPB), 32 * WPB, (size_t)WPB * ntri(PM_T) * sizeof(double2), st>>>(
        nb, L->start[LV], L->idx[LV], T->ic, T->hw, ws.pb, ws.ps, ws.Mu, ws.m2l_tab, ws.B);
    QBX_LAUNCH_CHECK();
    k_p2l<PM_T><<<nblocks(nb, WPB), 32 * WPB, 0, st>>>(nb, L->start[LXF], L->idx[LXF], T->own_start[KSRC], T->sxyz,
                                                       ns, ws.sq, dip ? ws.sd : nullptr, T->cen, T->hw, ws.pb, ws.B);
    QBX_LAUNCH_CHECK();
    for (int l = 1; l < T->nlev; ++l) {
        int b0 = T->level_start[l], b1 = T->level_start[l + 1];
        k_l2l<PM_T><<<nblocks(b1 - b0, WPB), 32 * WPB, 0, st>>>(b0, b1, T->lvl_boxes, T->parent, T->ntgt_sub, T->child, ws.pb,
                                                                ws.oct_tab, ws.B);
        QBX_LAUNCH_CHECK();
    }
    switch (QM) {
    case 4: fixed_centers<4>(T, L, ws, dip, tgt_ctr, pot, st); break;
    case 8: fixed_centers<8>(T, L, ws, dip, tgt_ctr, pot, st); break;
    case 12: fixed_centers<12>(T, L, ws, dip, tgt_ctr, pot, st); break;
    default: fixed_centers<16>(T, L, ws, dip, tgt_ctr, pot, st); break;
    }
    if (nt > 0) {
        k_points<PM_T><<<nblocks(nt, WPB), 32 * WPB, 0, st>>>(
            nt, T->perm[KTGT], T->txyz, tgt_ctr, T->tgt_box, ws.pb, ws.ps, ListRef{L->start[LU], L->idx[LU]},
            ListRef{L->start[LWC], L->idx[LWC]}, ListRef{L->start[LXC], L->idx[LXC]},
            ListRef{L->start[LWF], L->idx[LWF]}, T->own_start[KSRC], T->sxyz, ns, ws.sq, dip ? ws.sd : nullptr,
            T->cen, T->hw, ws.Mu, ws.B, pot);
        QBX_LAUNCH_CHECK();
    }
}

}  // namespace qbx
