// List 3 far M2QBXL (Algorithm 4 Stage 5(b)) in mixed precision.
//
// For a List 3 far box d (center c_d, half width h_d) and a QBX center c (radius rho) of a box
// b with d in List 3 far of b, the QBX local receives
//   A_k^l += 1/h (rho/h)^k sum_{j,i} Mu_{j-k}^{i-l} conj S_j^i(X),   X = (c - c_d)/h,  h = h_d.
// In the balanced scaling (Mh = Mu F, Sh = S / F, Ah = A / F, F(n,m) = sqrt((n+|m|)!(n-|m|)!))
//   Ah_k^l (h (h/rho)^k) = sum_{j,i} Mh_{j-k}^{i-l} G(j-k, i-l, k, l) conj Sh_j^i(X),
//   G(n,m,k,l) = F(n+k, m+l) / (F(n,m) F(k,l)) <= 2^(n+k),
// a product of a matrix that depends on d only (a Hankel arrangement of its multipole, built in
// FP64 and rounded to FP32) with a vector that depends on the pair (irregular harmonics of X up
// to order P+Q, computed in FP64 and rounded).  Pairs are grouped by d, each group is one FP32
// GEMM, each pair's result is stored, and a per-center reduction adds the center's pairs in
// List 3 far order in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "harmonics.cuh"
#include "tc_common.cuh"
#include "df64.cuh"

namespace qbx {

constexpr int WF_MAXCH = 48;  // K chunks of the tensor-core form

// K slots of harmonic degree j in the tensor-core layout: [Re S_j^0, 0, 0, 0] then, for each odd i,
// [Re S_j^i, Im S_j^i, Re S_j^{i+1}, Im S_j^{i+1}] (zeros for i + 1 > j): 16-byte groups that one
// thread writes with one store.
__host__ __device__ __forceinline__ int wfar_degree_slots(int j) { return 4 + 4 * ((j + 1) / 2); }

struct WfarPlan {
    int P = -1, Q = -1, K = 0, R = 0;
    int64_t npairs = 0;
    int ndsrc = 0, ntiles = 0;
    int *slot = nullptr;      // n_boxes: H slot of a List 3 far source box, -1 otherwise
    int *slot_box = nullptr;  // ndsrc: box of each slot
    float *H = nullptr;       // ndsrc x R x K
    int *pair_ctr = nullptr;  // sorted center of each pair (pairs grouped by d)
    int *pair_d = nullptr;    // source box of each pair
    int *pos_cm = nullptr;    // center-major entry -> pair position
    int *cm_start = nullptr;  // nc + 1
    int2 *tiles = nullptr;    // (first pair, last pair + 1) per GEMM tile
    float *Y = nullptr;       // npairs x R
    int *zero_start = nullptr;  // n_boxes + 1 zeros: an empty List 3 far for the FP64 center kernel
    // split-TF32 tensor-core form (QBX_M2L_3XTF32): K (the harmonic index) in chunks of whole
    // degrees [cj0, cj1), each padded to a multiple of 8 columns; H in K-major tiles per chunk
    bool tc = false;
    int Rp = 0, Kp = 0, nch = 0, WMAX = 0, ntc = 0, NU = 0;
    int cj0[WF_MAXCH] = {}, cj1[WF_MAXCH] = {}, ckoff[WF_MAXCH + 1] = {};
    float *H_tc = nullptr;     // ndsrc x 2 x Rp x Kp: per K chunk the TF32 hi tile then the lo tile
    float *cenf = nullptr;     // n_boxes x 8: box centers as double-floats and 1/h
    float *rec_fac = nullptr;        // Rp x Kp: |factor| of each H entry
    uint32_t *rec_code = nullptr;    // Rp x Kp: packed terms of each H entry (see k_wfar_H_tc)
    int4 *tc_tiles = nullptr;  // (source box, first pair, last pair + 1) per 128-pair tile
};

int wfar_plan_orders(const WfarPlan *p) { return p ? (p->P * 100 + p->Q) * 2 + (p->tc ? 1 : 0) : -1; }
const int *wfar_empty_start(const WfarPlan *p) { return p->zero_start; }

void free_wfar_plan(WfarPlan *p)
{
    if (!p) return;
    dfree(p->slot); dfree(p->slot_box); dfree(p->H); dfree(p->pair_ctr); dfree(p->pair_d); dfree(p->pos_cm);
    dfree(p->cm_start); dfree(p->tiles); dfree(p->Y); dfree(p->zero_start);
    dfree(p->H_tc); dfree(p->tc_tiles); dfree(p->rec_fac); dfree(p->rec_code); dfree(p->cenf);
    delete p;
}

__constant__ double c_F[ntri(40)];     // F(n,m), m >= 0, n <= 40
__constant__ double c_Finv[ntri(40)];  // 1 / F(n,m)

__device__ __forceinline__ double Fnm(int n, int m) { return c_F[tri(n, m < 0 ? -m : m)]; }
__device__ __forceinline__ double Finv(int n, int m) { return c_Finv[tri(n, m < 0 ? -m : m)]; }

// row index of (k, l, part) and column index of (j, i, part) in the real layouts
__device__ __forceinline__ void decode(int r, int &n, int &m, int &part)
{
    n = (int)sqrtf((float)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    int rr = r - n * n;
    m = (rr + 1) / 2;
    part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
}

__global__ void k_wfar_count(int64_t nc, const int *ctr_box, const int *wstart, const int *widx, int *cm_cnt,
                             int *d_cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int b = ctr_box[i];
    cm_cnt[i] = wstart[b + 1] - wstart[b];
    for (int e = wstart[b]; e < wstart[b + 1]; ++e) atomicAdd(&d_cnt[widx[e]], 1);
}

__global__ void k_wfar_fill(int64_t nc, const int *ctr_box, const int *wstart, const int *widx, const int *cm_start,
                            int *d_fill, int *pair_ctr, int *pair_d, int *pos_cm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int b = ctr_box[i];
    for (int e = wstart[b]; e < wstart[b + 1]; ++e) {
        int d = widx[e];
        int p = atomicAdd(&d_fill[d], 1);
        pair_ctr[p] = (int)i;
        pair_d[p] = d;
        pos_cm[cm_start[i] + (e - wstart[b])] = p;
    }
}

__global__ void k_wfar_slots(int nb, const int *d_cnt, const int *slot_scan, int *slot, int *slot_box)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nb) return;
    if (d_cnt[d] > 0) {
        slot[d] = slot_scan[d];
        slot_box[slot_scan[d]] = d;
    } else {
        slot[d] = -1;
    }
}

__global__ void k_flag_pos(int nb, const int *cnt, int *flag)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < nb) flag[d] = cnt[d] > 0 ? 1 : 0;
}

// Entry (row = (k,l,rp), col = (j,i,cp)) of the Hankel operator of a source box with multipole M
// (tri layout, stride PMT) truncated at order Pd.
__device__ double wfar_H_entry(int row, int col, int Pd, const double2 *M)
{
    int k, l, rp, j, i, cp;
    decode(row, k, l, rp);
    decode(col, j, i, cp);
    int n = j - k;
    double2 a1 = make_double2(0, 0), a2 = make_double2(0, 0);
    if (n >= 0 && n <= Pd) {
        int m1 = i - l, m2 = -i - l;
        // Mh_n^m G(n,m,k,l) = Mu_n^m F(n+k, m+l) / F(k,l)
        if (m1 >= -n && m1 <= n) a1 = cscale(sym_get(M, n, m1), Fnm(n + k, m1 + l) * Finv(k, l));
        if (i > 0 && m2 >= -n && m2 <= n) a2 = cscale(sym_get(M, n, m2), Fnm(n + k, m2 + l) * Finv(k, l));
    }
    double sg = (i & 1) ? -1.0 : 1.0;
    double2 plus = make_double2(a1.x + sg * a2.x, a1.y + sg * a2.y);   // a1 + s a2
    double2 mins = make_double2(sg * a2.x - a1.x, sg * a2.y - a1.y);   // s a2 - a1
    if (rp == 0 && cp == 0) return plus.x;
    if (rp == 0 && cp == 1) return -mins.y;
    if (rp == 1 && cp == 0) return plus.y;
    return mins.x;
}

// H[slot][(k,l,rp)][(j,i,cp)] from the FP64 multipole of the slot's box.
__global__ void k_wfar_H(int ndsrc, int P, int Q, int PMT, const int *slot_box, const signed char *pb,
                         const double2 *Mu, float *H)
{
    const int K = (P + Q + 1) * (P + Q + 1), R = (Q + 1) * (Q + 1);
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ndsrc * R * K) return;
    int s = (int)(idx / ((int64_t)R * K));
    int rem = (int)(idx % ((int64_t)R * K));
    int row = rem / K, col = rem % K;
    int d = slot_box[s];
    int Pd = min((int)pb[d], P);
    H[idx] = (float)wfar_H_entry(row, col, Pd, Mu + (int64_t)d * ntri(PMT));
}

struct WfarChunks {
    int nch, R, Rp, Kp;
    int cj0[WF_MAXCH], cj1[WF_MAXCH], ckoff[WF_MAXCH + 1];
};

// IEEE double -> float from the bit fields, rounding the 24-bit significand half away from zero
// (a carry out of the significand moves into the exponent); magnitudes below the float normal
// range become 0, beyond its range infinite.  Integer operations only (no FP64 instruction).
__device__ __forceinline__ float dbl_to_f32_rn(double v)
{
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int e = (hi >> 20) & 0x7ff;
    if (e < 897) return 0.0f;
    if (e > 1150) return __uint_as_float(((unsigned)hi & 0x80000000u) | 0x7f800000u);
    const unsigned mant = (((unsigned)(hi & 0xfffff) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    return __uint_as_float(((unsigned)hi & 0x80000000u) | (((unsigned)(e - 896) << 23) + mant));
}

// H of the tensor-core form: for each slot and chunk c, Rp rows x W_c columns (W_c = ckoff[c+1] -
// ckoff[c]) as a K-major tile with SBO = 32 W_c, FP32 (split into TF32 parts when loaded).  The
// harmonics it multiplies are scaled per degree (A = S_j^i / D(j), D(j) = sqrt((2j)!)), so entry
// (row, (j,i,cp)) is the balanced operator entry times D(j) / F(j,i).  Each entry is one or two
// multipole coefficients times constants: the recipe table (one record per entry, in output order,
// built once per plan) holds them, and the kernel only gathers and multiplies (in FP32).
struct WfarRecipe {
    float f1, f2;    // factors of the two terms (signs and scales folded in; computed in FP64, rounded)
    int t1, t2;      // tri index of the multipole coefficient, -1 for none
    int bits;        // bit 0: term 1 takes .y, bit 1: term 2 takes .y, bits 8..: degree n of both terms
    int pad;
};

// The recipe as the kernel reads it, one float and one word per entry: |f| (both terms of an entry
// have the same magnitude D(j)/F(k,l)), and code = t1 | t2 << 10 | n << 20 | ty << 26 | s1 << 27 |
// s2 << 28 (tri indices, 1023 for none; the degree n of both terms; ty: the terms read .y; s1, s2: the
// terms' signs).  An entry is s1 |f| M[t1] + s2 |f| M[t2], as fmaf(s2 |f|, M[t2], s1 |f| M[t1]).
constexpr uint32_t WF_NOTERM = 1023u;

__device__ __forceinline__ float wfar_recipe_entry(float f, uint32_t c, int Pd, const float2 *Ms)
{
    const uint32_t t1 = c & 1023u, t2 = (c >> 10) & 1023u;
    const int n = (int)((c >> 20) & 63u);
    const bool ty = (c >> 26) & 1u;
    float e = 0.f;
    if (n <= Pd) {
        if (t1 != WF_NOTERM) {
            const float2 v = Ms[t1];
            e = ((c >> 27) & 1u ? -f : f) * (ty ? v.y : v.x);
        }
        if (t2 != WF_NOTERM) {
            const float2 v = Ms[t2];
            e = fmaf((c >> 28) & 1u ? -f : f, ty ? v.y : v.x, e);
        }
    }
    return e;
}

// One block per slot (source box): its multipole rounded to FP32 once into shared memory (by integer
// operations: FP64 arithmetic on ~10^10 entries per evaluation would bound this kernel by the FP64
// pipe), then the slot's Rp x Kp entries four at a time from the recipe (L2-resident, shared by all
// slots), split into TF32 hi and lo parts once here rather than by every tile that reads them.  Layout
// per slot and K chunk c: the hi tile (Rp x W_c, K-major) then the lo tile, so that the products fetch
// each part of a chunk with one bulk copy.
__global__ void __launch_bounds__(256) k_wfar_H_tc(int P, int PMT, int Rp, WfarChunks ch, const float4 *fac,
                                                   const uint4 *code, const int *slot_box, const signed char *pb,
                                                   const double2 *Mu, float4 *H)
{
    __shared__ float2 Ms[ntri(PMAX)];
    const int s = blockIdx.x, d = slot_box[s];
    const int Pd = min((int)pb[d], P);
    const double2 *M = Mu + (int64_t)d * ntri(PMT);
    for (int t = threadIdx.x; t < ntri(P); t += blockDim.x) {
        const double2 v = M[t];
        Ms[t] = make_float2(dbl_to_f32_rn(v.x), dbl_to_f32_rn(v.y));
    }
    __syncthreads();
    float4 *out = H + (int64_t)s * (2 * (int64_t)Rp * ch.Kp / 4);
    for (int c = 0; c < ch.nch; ++c) {
        const int q0 = ch.ckoff[c] * Rp / 4, n4 = (ch.ckoff[c + 1] - ch.ckoff[c]) * Rp / 4;
        float4 *hi = out + 2 * q0, *lo = hi + n4;
        for (int q = threadIdx.x; q < n4; q += blockDim.x) {
            const float4 f = __ldg(fac + q0 + q);
            const uint4 cd = __ldg(code + q0 + q);
            const float4 v = make_float4(wfar_recipe_entry(f.x, cd.x, Pd, Ms), wfar_recipe_entry(f.y, cd.y, Pd, Ms),
                                         wfar_recipe_entry(f.z, cd.z, Pd, Ms), wfar_recipe_entry(f.w, cd.w, Pd, Ms));
            float4 h, l;
            tc::split_tf32(v.x, h.x, l.x);
            tc::split_tf32(v.y, h.y, l.y);
            tc::split_tf32(v.z, h.z, l.z);
            tc::split_tf32(v.w, h.w, l.w);
            hi[q] = h;
            lo[q] = l;
        }
    }
}

// Unit-vector harmonics scaled per degree: Yh_j^i = |x|^{j+1} S_j^i(x) / D(j) obey
//   Yh_0^0 = 1,  Yh_i^i = a_i (x + i y)/|x| Yh_{i-1}^{i-1},
//   Yh_j^i = a_j (z/|x|) Yh_{j-1}^i - b_j^i Yh_{j-2}^i,
//   a_j = sqrt((2j-1)/(2j)),  b_j^i = (j+i-1)(j-i-1) / sqrt(2j (2j-1) (2j-2) (2j-3)),
// and |Yh_j^i| <= F(j,i)/F(j,j) <= 1.  Bounded by 1 and forward-stable in j, the recurrence runs in
// FP32: its rounding (a few units of 2^-24 at the degrees used) stays below the 2^-22 of the TF32
// split that the products then apply to it.
__constant__ float c_al[41], c_be[ntri(40)], c_cd[41];  // c_cd[i] = a_1 a_2 ... a_i

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

struct WfarTcArgs {
    int ntiles, P, Q, PQ, R, Rp, WMAX, acc_cols, tmem_cols;
    WfarChunks ch;
    const int4 *tiles;
    const int *pair_ctr, *slot;
    const float *H;
    const float *cf;    // centers as double-floats: [xh yh zh xl yl zl] x nc (sorted order)
    const float *cenf;  // per box: xh yh zh xl yl zl, 1/h (exact: h is a power of two), pad
    const double *cr;
    int64_t nc;
    float *Y;
    int *err;
    long long wait_limit;  // clock cycles a pipeline wait may take before it gives up
    int probe_step;        // failure-path probe: pipeline step at which the wait on bar_never runs out (-1: off)
};

// Tensor-core List 3 far products, warp-specialised and persistent (one CTA per SM walking 128-pair
// tiles of one source box d):
//   warps 0-11  producers: three threads per pair of the tile (pair p = tid % 128; r = tid / 128 takes
//               the harmonic column groups g = r (mod 3)); per K chunk (whole degrees) they generate
//               the scaled irregular harmonics of their pairs in FP32 and split them into TF32 parts,
//               and load and split their share of the chunk of H_d, into one of two shared-memory
//               stages; the pair geometry and the radial powers run in double-float.  Once every
//               producer has filled a stage, one thread of warp 0 issues a_hi b_hi + a_lo b_hi +
//               a_hi b_lo per 8-column step into one of two 128 x Rp FP32 accumulators in tensor
//               memory and releases the stage by a commit.
//   warps 12-15 epilogue, one TMEM lane quadrant each: Y[pair][row] = acc F(k,l) (rho/h)^k / h,
//               drained while the next tile accumulates in the other buffer.
// Stages and accumulators hand over on mbarriers; no block-wide barrier inside the tile loop.  Every
// wait is bounded (wait_limit): a role that gives up records the failure and leaves its loop, the
// others then give up too, the issued products are drained and the tensor memory is freed.
constexpr int WF_PROD = 384;                       // producer threads
constexpr int WF_THREADS = WF_PROD + 128;          // + 4 epilogue warps
constexpr int WF_SPLIT = WF_PROD / 128;            // producer threads per pair
constexpr int WF_STAGES = 2;

__device__ __forceinline__ void mbar_arrive1(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <int NU>
__global__ void __launch_bounds__(WF_THREADS, 1) k_wfar_tc(WfarTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ uint64_t bar_full[WF_STAGES], bar_empty[WF_STAGES], bar_b[WF_STAGES], bar_afull[2], bar_aempty[2],
        bar_drain, bar_never;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Q = a.Q, PQ = a.PQ, Rp = a.Rp, WMAX = a.WMAX;
    const uint32_t sboA = (uint32_t)WMAX * 32u + 16u;
    const uint32_t bytesA = 16u * sboA, bytesB = (uint32_t)Rp * WMAX * 4u;
    // stage s, part 0 (hi) / 1 (lo) of the A and B tiles
    auto Abuf = [&](int s, int part) { return smem_tc + (size_t)(2 * s + part) * bytesA; };
    auto Bbuf = [&](int s, int part) {
        return smem_tc + (size_t)2 * WF_STAGES * bytesA + (size_t)(2 * s + part) * bytesB;
    };
    float *colF = reinterpret_cast<float *>(smem_tc + (size_t)2 * WF_STAGES * (bytesA + bytesB));  // Rp
    int *colK = reinterpret_cast<int *>(colF + Rp);                                                 // Rp
    for (int r = tid; r < Rp; r += WF_THREADS) {
        int k = 0, l = 0, part = 0;
        if (r < a.R) decode(r, k, l, part);
        colF[r] = (float)Fnm(k, l);
        colK[r] = r < a.R ? k : Q + 1;
    }
    if (tid == 0) {
        for (int s = 0; s < WF_STAGES; ++s) {
            tc::mbar_init(&bar_full[s], WF_PROD / 32);
            tc::mbar_init(&bar_empty[s], 1);
            tc::mbar_init(&bar_b[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&bar_afull[b], 1);
            tc::mbar_init(&bar_aempty[b], 4);
        }
        tc::mbar_init(&bar_drain, 1);
        tc::mbar_init(&bar_never, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, (uint32_t)a.tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (tid < WF_PROD) {
        // ------------------------------------------------------------ producers (+ the MMA issue)
        const int p = tid & 127, par = tid >> 7;  // warps 4 par .. 4 par + 3 (uniform per warp)
        const bool issuer = tid == 0;             // also fetches the operator chunks and issues the products
        const uint32_t idesc = tc::idesc_tf32(128, Rp);
        uint32_t g = 0, tt = 0;
        uint32_t pend = 0, pend_par = 0;          // stages with an operator copy not yet waited for, its phase
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tt) {
            const int4 tl = a.tiles[t];
            const int d = tl.x, p0 = tl.y, np = tl.z - tl.y;
            const float *Hd = a.H + (int64_t)a.slot[d] * 2 * Rp * a.ch.Kp;  // hi / lo tiles per chunk
            const bool valid = p < np;
            // pair geometry X = (c - c_d)/h in double-float; an idle row takes X = (3, 0, 0)
            const float *bc = a.cenf + 8 * (int64_t)d;
            const float hinv = bc[6];
            df x{3.f, 0.f}, y{0.f, 0.f}, z{0.f, 0.f};
            if (valid) {
                const int64_t c = a.pair_ctr[p0 + p], nc = a.nc;
                x = df_mul_f(df_sub(df{a.cf[c], a.cf[3 * nc + c]}, df{bc[0], bc[3]}), hinv);
                y = df_mul_f(df_sub(df{a.cf[nc + c], a.cf[4 * nc + c]}, df{bc[1], bc[4]}), hinv);
                z = df_mul_f(df_sub(df{a.cf[2 * nc + c], a.cf[5 * nc + c]}, df{bc[2], bc[5]}), hinv);
            }
            const df rinv = df_rsqrt(df_add(df_add(df_sqr(x), df_sqr(y)), df_sqr(z)));
            const float zh = df_mul(z, rinv).h;
            df rpj = rinv;  // |X|^{-(j+1)} at the current degree j (starts at j = 0)
            float a1r[NU][2], a1i[NU][2], a2r[NU][2], a2i[NU][2];
            {
                // diagonals Yh_i^i = cd_i w^i (w = (x + iy)/|x|, cd_i = a_1 ... a_i) of this thread's groups:
                // group g = par + 3u holds column 0 (g = 0) or columns 2g-1, 2g
                const float2 w1 = make_float2(df_mul(x, rinv).h, df_mul(y, rinv).h);
                const float2 w2 = cmulf(w1, w1), w3 = cmulf(w2, w1), w5 = cmulf(w3, w2), w6 = cmulf(w3, w3);
                // w^(first column of group par): 1 (par 0), w (1), w^3 (2)
                float2 cur = par == 0 ? make_float2(1.f, 0.f) : par == 1 ? w1 : w3;
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    const int g0 = par + WF_SPLIT * u;
                    const int i0 = g0 == 0 ? 0 : 2 * g0 - 1;
                    a2r[u][0] = a2i[u][0] = a2r[u][1] = a2i[u][1] = 0.f;
                    const float c0 = c_cd[min(i0, 40)], c1 = c_cd[min(i0 + 1, 40)];
                    a1r[u][0] = c0 * cur.x;
                    a1i[u][0] = c0 * cur.y;
                    const float2 nxt = cmulf(cur, w1);
                    a1r[u][1] = c1 * nxt.x;
                    a1i[u][1] = c1 * nxt.y;
                    // next group of this thread: 6 columns on (from column 0: group 3 starts at column 5)
                    cur = (g0 == 0) ? w5 : cmulf(cur, w6);
                }
            }
            for (int c = 0; c < a.ch.nch; ++c, ++g) {
                const int s = g % WF_STAGES;
                const uint32_t use = g / WF_STAGES;
                // the products that last read stage s must have completed (lane 0 waits for the warp)
                if (use > 0) {
                    bool w = true;
                    if (lane == 0) w = tc::mbar_wait(&bar_empty[s], (use - 1) & 1, a.wait_limit);
                    ok = __shfl_sync(0xffffffffu, w, 0);
                    if (!ok) break;
                }
                const int j0 = a.ch.cj0[c], j1 = a.ch.cj1[c];
                const int W = a.ch.ckoff[c + 1] - a.ch.ckoff[c];
                if (issuer) {
                    // the chunk of H_d, TF32 hi and lo tiles, by two bulk copies into the free stage
                    const uint32_t bytes = (uint32_t)Rp * W * 4u;
                    const float *src = Hd + (int64_t)2 * a.ch.ckoff[c] * Rp;
                    tc::mbar_arrive_expect_tx(&bar_b[s], 2u * bytes);
                    tc::bulk_g2s(Bbuf(s, 0), src, bytes, &bar_b[s]);
                    tc::bulk_g2s(Bbuf(s, 1), src + (int64_t)W * Rp, bytes, &bar_b[s]);
                    pend |= 1u << s;
                    pend_par = (pend_par & ~(1u << s)) | ((use & 1u) << s);
                }
                // A: S_j^i / D(j) = Yh_j^i |x|^{-(j+1)} for degrees j0 .. j1-1 of this thread's column groups;
                // the recurrence in FP32, the radial factor (a double-float power) rounded to FP32, one
                // 16-byte store per group and TF32 part
                {
                    unsigned char *Ah = Abuf(s, 0), *Al = Abuf(s, 1);
                    const uint32_t rowoff = (uint32_t)(p >> 3) * sboA + (uint32_t)(p & 7) * 16u;
                    int kb = 0;
                    for (int j = j0; j < j1; kb += wfar_degree_slots(j), ++j) {
                        const float c1 = c_al[j] * zh;
                        const float rf = rpj.h;
                        rpj = df_mul(rpj, rinv);
#pragma unroll
                        for (int u = 0; u < NU; ++u) {
                            const int gg = par + WF_SPLIT * u;
                            const int i0 = gg == 0 ? 0 : 2 * gg - 1;  // first column of the group
                            if (i0 > j || i0 > PQ) break;  // later groups start at higher columns
                            float v[4];
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                const int i = i0 + h2;
                                v[2 * h2] = v[2 * h2 + 1] = 0.f;
                                if ((gg == 0 && h2 == 1) || i > j) continue;
                                float vr = a1r[u][h2], vi = a1i[u][h2];
                                if (j > i) {
                                    const float bb = c_be[tri(j, i)];
                                    vr = fmaf(c1, a1r[u][h2], -bb * a2r[u][h2]);
                                    vi = fmaf(c1, a1i[u][h2], -bb * a2i[u][h2]);
                                    a2r[u][h2] = a1r[u][h2]; a2i[u][h2] = a1i[u][h2];
                                    a1r[u][h2] = vr; a1i[u][h2] = vi;
                                }
                                v[2 * h2] = vr * rf;
                                v[2 * h2 + 1] = (i == 0) ? 0.f : vi * rf;
                            }
                            float4 hv, lv;
                            tc::split_tf32(v[0], hv.x, lv.x);
                            tc::split_tf32(v[1], hv.y, lv.y);
                            tc::split_tf32(v[2], hv.z, lv.z);
                            tc::split_tf32(v[3], hv.w, lv.w);
                            const uint32_t off = (uint32_t)((kb + 4 * gg) >> 2) * 128u + rowoff;
                            *reinterpret_cast<float4 *>(Ah + off) = hv;
                            *reinterpret_cast<float4 *>(Al + off) = lv;
                        }
                    }
                    if (par == 0 && kb < W) {  // chunk padding to a multiple of 8 columns (one 16-byte group)
                        const uint32_t off = (uint32_t)(kb >> 2) * 128u + rowoff;
                        *reinterpret_cast<float4 *>(Ah + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4 *>(Al + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive1(&bar_full[s]);
                if (warp == 0) {
                    bool w = true;
                    if (issuer) {
                        const int ab = tt & 1;
                        const uint32_t v = tt >> 1;
                        // the accumulator's previous tile must have been drained; every producer must have
                        // filled the stage
                        if (c == 0 && v > 0) w = tc::mbar_wait(&bar_aempty[ab], (v - 1) & 1, a.wait_limit);
                        if (w) w = tc::mbar_wait(&bar_full[s], use & 1, a.wait_limit);
                        if (w) {
                            w = tc::mbar_wait(&bar_b[s], use & 1, a.wait_limit);
                            if (w) pend &= ~(1u << s);
                        }
                        // failure-path probe: a wait on a barrier nothing arrives on runs out
                        if (w && (int)g == a.probe_step) w = tc::mbar_wait(&bar_never, 0, a.wait_limit);
                        if (w) {
                            tc::tc_fence_after();
                            const uint32_t dt = tmem + (uint32_t)(ab * a.acc_cols);
                            const uint32_t a_hi = tc::smem_u32(Abuf(s, 0)), a_lo = tc::smem_u32(Abuf(s, 1));
                            const uint32_t b_hi = tc::smem_u32(Bbuf(s, 0)), b_lo = tc::smem_u32(Bbuf(s, 1));
                            const uint32_t sboB = (uint32_t)W * 32u;
                            for (int ks = 0; ks < W / 8; ++ks) {
                                const uint32_t off = 256u * ks;
                                const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                                tc::mma_tf32(dt, tc::sdesc(a_hi + off, 128, sboA), tc::sdesc(b_hi + off, 128, sboB),
                                             idesc, acc0);
                                tc::mma_tf32(dt, tc::sdesc(a_lo + off, 128, sboA), tc::sdesc(b_hi + off, 128, sboB),
                                             idesc, 1u);
                                tc::mma_tf32(dt, tc::sdesc(a_hi + off, 128, sboA), tc::sdesc(b_lo + off, 128, sboB),
                                             idesc, 1u);
                            }
                            tc::mma_commit(&bar_empty[s]);  // releases the stage when these products complete
                            if (c + 1 == a.ch.nch) tc::mma_commit(&bar_afull[ab]);
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, w, 0);
                    if (!ok) break;
                }
            }
        }
        if (issuer) {
            // every product issued so far completes before the tensor memory is released, and every
            // operator copy still in flight lands before the shared memory is
            tc::mma_commit(&bar_drain);
            tc::mbar_wait(&bar_drain, 0, tc::WAIT_LIMIT);
            for (int s2 = 0; s2 < WF_STAGES; ++s2)
                if (pend & (1u << s2)) tc::mbar_wait(&bar_b[s2], (pend_par >> s2) & 1u, tc::WAIT_LIMIT);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int qd = warp & 3, row = 32 * qd + lane;
        uint32_t tt = 0;
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tt) {
            const int4 tl = a.tiles[t];
            const int d = tl.x, p0 = tl.y, np = tl.z - tl.y;
            const int ab = tt & 1;
            const uint32_t v = tt >> 1;
            // (rho/h)^k / h, k = 0, 1, ... in double-float, advanced as the columns' degree grows
            const float hinv = a.cenf[8 * (int64_t)d + 6];
            const bool valid = row < np;
            const df ratio = valid ? df_mul_f(df_from(a.cr[a.pair_ctr[p0 + row]]), hinv) : df{0.f, 0.f};
            bool w = true;
            if (lane == 0) w = tc::mbar_wait(&bar_afull[ab], v & 1, a.wait_limit);
            ok = __shfl_sync(0xffffffffu, w, 0);
            if (!ok) break;
            tc::tc_fence_after();
            df pw{hinv, 0.f};
            int kc = 0;
            float *yrow = a.Y + (int64_t)(p0 + row) * a.R;
            for (int cg = 0; cg * 16 < Rp; ++cg) {
                float vals[16];
                tc::tmem_ld16(tmem + (uint32_t)(ab * a.acc_cols) + ((uint32_t)(32 * qd) << 16) + (uint32_t)(cg * 16),
                              vals);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = cg * 16 + j;
                    while (kc < colK[col] && kc <= Q) {  // uniform across the warp
                        pw = df_mul(pw, ratio);
                        ++kc;
                    }
                    if (valid && col < a.R) yrow[col] = vals[j] * colF[col] * pw.h;
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(&bar_aempty[ab]);
        }
    }
    if (!ok) atomicOr(a.err, 8);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

static size_t wfar_tc_smem(int Rp, int WMAX, int Q)
{
    (void)Q;
    return (size_t)2 * WF_STAGES * 16 * (WMAX * 32 + 16) + (size_t)2 * WF_STAGES * Rp * WMAX * 4 + (size_t)Rp * 8;
}

constexpr int WKC = 32;  // K chunk of the H tile

// One tile = up to WT pairs of one source box d: balanced irregular harmonics of the pairs (FP64
// -> FP32, shared memory), then Y = H_d x S in FP32, scaled per output row.  256 threads: 256/WT
// per pair for the harmonics; (256/(WT/4)) row groups x (WT/4) column groups of 4 for the product.
template <int WT, int MR>
__global__ void __launch_bounds__(256) k_wfar_gemm(int P, int Q, const int2 *tiles, const int *pair_ctr,
                                                   const int *pair_d, const int *slot, const float *H,
                                                   const double *cxyz, int64_t nc, const double *cr,
                                                   const double *cen, const double *hw, float *Y)
{
    extern __shared__ float smem[];
    constexpr int TPP = 256 / WT, CG = WT / 4, RG = 256 / CG;
    const int K = (P + Q + 1) * (P + Q + 1), R = (Q + 1) * (Q + 1), PQ = P + Q;
    float *Ss = smem;                       // K x WT
    float *Hs = smem + (size_t)K * WT;      // R x WKC
    float *Pw = Hs + (size_t)R * WKC;       // WT x (Q+1): (rho/h)^k / h per pair
    const int2 tl = tiles[blockIdx.x];
    const int p0 = tl.x, np = tl.y - tl.x;
    const int d = pair_d[p0];
    const float *Hd = H + (int64_t)slot[d] * R * K;
    const double h = hw[d], hinv = 1.0 / h;
    {
        const int pc = threadIdx.x / TPP, r = threadIdx.x % TPP;
        bool valid = pc < np;
        double x = 3.0, y = 0.0, z = 0.0;
        if (valid) {
            int c = pair_ctr[p0 + pc];
            x = (cxyz[c] - cen[3 * d]) * hinv;
            y = (cxyz[nc + c] - cen[3 * d + 1]) * hinv;
            z = (cxyz[2 * nc + c] - cen[3 * d + 2]) * hinv;
        }
        double ir2 = 1.0 / (x * x + y * y + z * z);
        double rinv = sqrt(ir2);
        double2 wr = make_double2(x * ir2, y * ir2);
        double zz = z * ir2;
        if (r == 0) {
            double ratio = valid ? cr[pair_ctr[p0 + pc]] * hinv : 0.0, pk = hinv;
            for (int k = 0; k <= Q; ++k, pk *= ratio) Pw[pc * (Q + 1) + k] = (float)pk;
        }
        // lockstep rounds: in round k thread r fills column i = k*TPP + r; every thread advances
        // its own diagonal S_i^i by TPP steps per round, so the warp stays converged
        double2 diag = make_double2(rinv, 0.0);
        for (int t = 1; t <= r; ++t) diag = cscale(cmul(diag, wr), 2.0 * t - 1.0);
        for (int base = 0; base <= PQ; base += TPP) {
            const int i = base + r;
            if (base > 0)
                for (int t = i - TPP + 1; t <= i; ++t) diag = cscale(cmul(diag, wr), 2.0 * t - 1.0);
            if (i > PQ) continue;
            double2 a2 = make_double2(0.0, 0.0), a1 = diag;
            const double fz = valid ? 1.0 : 0.0;
            Ss[(size_t)(i * i + (i == 0 ? 0 : 2 * i - 1)) * WT + pc] = (float)(diag.x * Finv(i, i) * fz);
            if (i > 0) Ss[(size_t)(i * i + 2 * i) * WT + pc] = (float)(diag.y * Finv(i, i) * fz);
            for (int j = i + 1; j <= PQ; ++j) {
                double c1 = (2 * j - 1) * zz, c2 = (double)(j + i - 1) * (double)(j - i - 1) * ir2;
                double2 v = make_double2(c1 * a1.x - c2 * a2.x, c1 * a1.y - c2 * a2.y);
                a2 = a1;
                a1 = v;
                double f = Finv(j, i) * fz;
                // the balanced harmonic itself (Re, Im); H carries the conjugation
                Ss[(size_t)(j * j + (i == 0 ? 0 : 2 * i - 1)) * WT + pc] = (float)(v.x * f);
                if (i > 0) Ss[(size_t)(j * j + 2 * i) * WT + pc] = (float)(v.y * f);
            }
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % CG, ty = threadIdx.x / CG;
    float acc[MR][4] = {};
    for (int k0 = 0; k0 < K; k0 += WKC) {
        for (int t = threadIdx.x; t < R * WKC; t += 256) {
            int rr = t / WKC, kk = t % WKC;
            Hs[t] = (k0 + kk < K) ? Hd[(int64_t)rr * K + k0 + kk] : 0.f;
        }
        __syncthreads();
        int kmax = min(WKC, K - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            float b[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) b[jj] = Ss[(size_t)(k0 + kk) * WT + tx * 4 + jj];
#pragma unroll
            for (int ii = 0; ii < MR; ++ii) {
                int row = ty + RG * ii;
                float a = row < R ? Hs[row * WKC + kk] : 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fmaf(a, b[jj], acc[ii][jj]);
            }
        }
        __syncthreads();
    }
    // epilogue: A_k^l = Ah_k^l F(k,l) (rho/h)^k / h
#pragma unroll
    for (int ii = 0; ii < MR; ++ii) {
        int row = ty + RG * ii;
        if (row >= R) continue;
        int k = (int)sqrtf((float)row);
        while (k * k > row) --k;
        while ((k + 1) * (k + 1) <= row) ++k;
        int rr = row - k * k, l = (rr + 1) / 2;
        float fk = (float)Fnm(k, l);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            int pc = tx * 4 + jj;
            if (pc < np) Y[(int64_t)(p0 + pc) * R + row] = acc[ii][jj] * (fk * Pw[pc * (Q + 1) + k]);
        }
    }
}

static int wfar_tile_width(int, int) { return 32; }
static int wfar_rows_per_thread(int R) { return R <= 64 ? 2 : R <= 96 ? 3 : R <= 160 ? 5 : 10; }

template <int MR>
static void wfar_launch(const qbx_tree *T, WfarPlan *pl, size_t smem, cudaStream_t st)
{
    k_wfar_gemm<32, MR><<<pl->ntiles, 256, smem, st>>>(pl->P, pl->Q, pl->tiles, pl->pair_ctr, pl->pair_d, pl->slot,
                                                       pl->H, T->cxyz, T->np[KCTR], T->cr, T->cen, T->hw, pl->Y);
}

template <int MR>
static void wfar_set_smem(size_t smem)
{
    QBX_CUDA_TRY(cudaFuncSetAttribute(k_wfar_gemm<32, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}
static size_t wfar_smem(int K, int R, int WT)
{
    int Q = (int)std::lround(std::sqrt((double)R)) - 1;
    return ((size_t)K * WT + (size_t)R * WKC + (size_t)WT * (Q + 1)) * sizeof(float);
}

// A[c][tri(k,l)] += sum over the center's List 3 far pairs (list order, compensated FP32).
__global__ void k_wfar_reduce(int64_t nc, int Q, int QMS, const int *cm_start, const int *pos_cm, const float *Y,
                              const signed char *qc, double2 *A)
{
    const int R = (Q + 1) * (Q + 1);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * R) return;
    int64_t i = t / R;
    int row = (int)(t % R);
    int k = (int)sqrtf((float)row);
    while (k * k > row) --k;
    while ((k + 1) * (k + 1) <= row) ++k;
    if (k > qc[i]) return;
    int rr = row - k * k, l = (rr + 1) / 2, part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
    int e0 = cm_start[i], e1 = cm_start[i + 1];
    if (e0 == e1) return;
    // list-order sum in compensated FP32 (FP64 adds of converted terms would occupy the FP64 pipe);
    // eight independent loads in flight per step
    float hi = 0.f, lo = 0.f;
    int e = e0;
    for (; e + 8 <= e1; e += 8) {
        int q[8];
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = pos_cm[e + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(Y + (int64_t)q[u] * R + row);
#pragma unroll
        for (int u = 0; u < 8; ++u) tc::df_add(hi, lo, v[u]);
    }
    for (; e < e1; ++e) tc::df_add(hi, lo, __ldg(Y + (int64_t)pos_cm[e] * R + row));
    const double s = (double)hi + (double)lo;
    double2 *a = A + i * ntri(QMS) + tri(k, l);
    if (part) a->y += s;
    else a->x += s;
}

// Box centers as double-floats (xh yh zh xl yl zl) and 1/h (h a power of two, so exact in FP32).
__global__ void k_cen_to_df(int nb, const double *cen, const double *hw, float *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const df v = df_from(cen[3 * b + d]);
        out[8 * b + d] = v.h;
        out[8 * b + 3 + d] = v.l;
    }
    out[8 * b + 6] = (float)(1.0 / hw[b]);
    out[8 * b + 7] = 0.f;
}

// Degree chunks of the tensor-core form and its shared-memory budget; false when the orders do not fit.

static bool wfar_tc_layout(WfarPlan *pl, int w_hint)
{
    const int P = pl->P, Q = pl->Q, PQ = P + Q;
    pl->Rp = (pl->R + 15) / 16 * 16;
    if (pl->Rp > 256 || PQ > 35) return false;
    pl->NU = PQ <= 28 ? 5 : 7;  // 16-byte groups per thread: ceil((1 + ceil(PQ/2)) / 3)
    const int wmin = (wfar_degree_slots(PQ) + 7) / 8 * 8;
    int W = std::max(w_hint > 0 ? w_hint / 8 * 8 : 64, wmin);
    while (W > wmin && wfar_tc_smem(pl->Rp, W, Q) > 220 * 1024) W -= 8;
    if (wfar_tc_smem(pl->Rp, W, Q) > 220 * 1024) return false;
    if (pl->Rp > 256) return false;                          // two accumulators in 512 TMEM columns
    pl->WMAX = W;
    int nch = 0, j = 0, koff = 0;
    while (j <= PQ) {
        int j1 = j + 1, w = wfar_degree_slots(j);
        while (j1 <= PQ && w + wfar_degree_slots(j1) <= W) w += wfar_degree_slots(j1++);  // add degree j1 while it fits
        if (nch >= WF_MAXCH) return false;
        pl->cj0[nch] = j;
        pl->cj1[nch] = j1;
        pl->ckoff[nch] = koff;
        koff += (w + 7) / 8 * 8;
        ++nch;
        j = j1;
    }
    pl->ckoff[nch] = koff;
    pl->nch = nch;
    pl->Kp = koff;
    return true;
}

static void set_recurrence_tables(cudaStream_t st)
{
    // computed in FP64, stored rounded to FP32
    std::vector<double> al(41, 0.0), cd(41, 1.0);
    std::vector<float> alf(41, 0.f), cdf(41, 1.f), bef(ntri(40), 0.f);
    for (int j = 1; j <= 40; ++j) al[j] = std::sqrt((2.0 * j - 1.0) / (2.0 * j));
    for (int i = 1; i <= 40; ++i) cd[i] = cd[i - 1] * al[i];
    for (int j = 0; j <= 40; ++j) { alf[j] = (float)al[j]; cdf[j] = (float)cd[j]; }
    for (int j = 2; j <= 40; ++j)
        for (int i = 0; i < j; ++i)
            bef[tri(j, i)] = (float)((double)(j + i - 1) * (double)(j - i - 1) /
                                     std::sqrt(2.0 * j * (2.0 * j - 1.0) * (2.0 * j - 2.0) * (2.0 * j - 3.0)));
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_al, alf.data(), alf.size() * sizeof(float), 0, cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_cd, cdf.data(), cdf.size() * sizeof(float), 0, cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_be, bef.data(), bef.size() * sizeof(float), 0, cudaMemcpyHostToDevice, st));
}

// F(n, m) = sqrt((n+|m|)! (n-|m|)!) on the host
static double host_F(int n, int m)
{
    m = m < 0 ? -m : m;
    double f = 1.0;
    for (int i = 2; i <= n + m; ++i) f *= i;
    for (int i = 2; i <= n - m; ++i) f *= i;
    return std::sqrt(f);
}

static void host_decode(int r, int &n, int &m, int &part)
{
    n = (int)std::sqrt((double)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    int rr = r - n * n;
    m = (rr + 1) / 2;
    part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
}

// Recipe of every entry of the tensor-core H block of one slot, in output order (see k_wfar_H_tc):
// the operator entry of row (k,l,rp), column (j,i,cp) is a1.c + s a2.c combinations of
// a1 = M_n^{i-l} F(n+k, i)/F(k,l) and a2 = M_n^{-i-l} F(n+k, -i)/F(k,l) (n = j - k, s = (-1)^i,
// M_n^{-m} = (-1)^m conj M_n^m), scaled by D(j)/F(j,i).
static std::vector<WfarRecipe> wfar_recipe(const WfarPlan *pl)
{
    std::vector<WfarRecipe> out((size_t)pl->Rp * pl->Kp);
    for (auto &r : out) r = WfarRecipe{0.f, 0.f, -1, -1, 0, 0};
    for (int c = 0; c < pl->nch; ++c) {
        const int W = pl->ckoff[c + 1] - pl->ckoff[c];
        int kb = 0;  // first slot of degree j in the chunk
        for (int j = pl->cj0[c]; j < pl->cj1[c]; kb += wfar_degree_slots(j), ++j)
            for (int sl = 0; sl < wfar_degree_slots(j); ++sl) {
                int i, cp;  // harmonic column and part held by this slot, or a padding slot
                if (sl < 4) {
                    if (sl != 0) continue;
                    i = 0;
                    cp = 0;
                } else {
                    i = 2 * ((sl - 4) / 4) + 1 + ((sl & 3) >> 1);
                    cp = sl & 1;
                    if (i > j) continue;
                }
                for (int row = 0; row < pl->R; ++row) {
                    int k, l, rp;
                    host_decode(row, k, l, rp);
                    const int n = j - k;
                    WfarRecipe rc{0.f, 0.f, -1, -1, 0, 0};
                    if (n >= 0) {
                        const double colscale = host_F(j, j) / host_F(j, i), inv_kl = 1.0 / host_F(k, l);
                        const bool take_y = (rp != cp);  // (0,0), (1,1) read .x; (0,1), (1,0) read .y
                        // sign applied to the chosen component of M_n^m for m < 0 (M_n^{-m} = (-1)^m conj M_n^m)
                        auto sgn = [&](int m) {
                            if (m >= 0) return 1.0;
                            return take_y ? ((m & 1) ? 1.0 : -1.0) : ((m & 1) ? -1.0 : 1.0);
                        };
                        const double sg = (i & 1) ? -1.0 : 1.0;
                        double w1, w2;  // coefficients of a1 and a2 in the entry
                        if (rp == 0 && cp == 0) { w1 = 1.0; w2 = sg; }
                        else if (rp == 0 && cp == 1) { w1 = 1.0; w2 = -sg; }
                        else if (rp == 1 && cp == 0) { w1 = 1.0; w2 = sg; }
                        else { w1 = -1.0; w2 = sg; }
                        const int m1 = i - l, m2 = -i - l;
                        if (m1 >= -n && m1 <= n) {
                            rc.t1 = tri(n, m1 < 0 ? -m1 : m1);
                            rc.f1 = (float)(w1 * sgn(m1) * host_F(n + k, m1 + l) * inv_kl * colscale);
                        }
                        if (i > 0 && m2 >= -n && m2 <= n) {
                            rc.t2 = tri(n, m2 < 0 ? -m2 : m2);
                            rc.f2 = (float)(w2 * sgn(m2) * host_F(n + k, m2 + l) * inv_kl * colscale);
                        }
                        rc.bits = (take_y ? 3 : 0) | (n << 8);
                    }
                    const size_t pos = (size_t)pl->ckoff[c] * pl->Rp + tc::kmajor_off(row, kb + sl, (uint32_t)W * 32u) / 4u;
                    out[pos] = rc;
                }
            }
    }
    return out;
}

WfarPlan *wfar_plan_build(const qbx_tree *T, const qbx_lists *L, int P, int Q, bool tc, int w_hint, cudaStream_t st)
{
    WfarPlan *pl = new WfarPlan();
    int *cm_cnt = nullptr, *d_cnt = nullptr, *d_start = nullptr, *flag = nullptr, *tot = nullptr;
    try {
        pl->P = P;
        pl->Q = Q;
        pl->K = (P + Q + 1) * (P + Q + 1);
        pl->R = (Q + 1) * (Q + 1);
        const int nb = (int)T->nb;
        const int64_t nc = T->np[KCTR];
        {  // F(n, m) table in constant memory
            std::vector<double> F(ntri(40));
            std::vector<double> fact(81, 1.0);
            for (int i = 1; i <= 80; ++i) fact[i] = fact[i - 1] * i;
            for (int n = 0; n <= 40; ++n)
                for (int m = 0; m <= n; ++m) F[tri(n, m)] = std::sqrt(fact[n + m] * fact[n - m]);
            std::vector<double> Fi(F.size());
            for (size_t i = 0; i < F.size(); ++i) Fi[i] = 1.0 / F[i];
            QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_F, F.data(), F.size() * sizeof(double), 0, cudaMemcpyHostToDevice, st));
            QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(c_Finv, Fi.data(), Fi.size() * sizeof(double), 0,
                                                 cudaMemcpyHostToDevice, st));
        }
        cm_cnt = dalloc<int>(nc + 1);
        d_cnt = dalloc<int>(nb + 1);
        d_start = dalloc<int>(nb + 1);
        flag = dalloc<int>(nb + 1);
        tot = dalloc<int>(1);
        pl->cm_start = dalloc<int>(nc + 1);
        pl->zero_start = dalloc<int>(nb + 1);
        pl->slot = dalloc<int>(nb);
        QBX_CUDA_TRY(cudaMemsetAsync(pl->zero_start, 0, (nb + 1) * sizeof(int), st));
        QBX_CUDA_TRY(cudaMemsetAsync(cm_cnt, 0, (nc + 1) * sizeof(int), st));
        QBX_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, (nb + 1) * sizeof(int), st));
        QBX_CUDA_TRY(cudaMemsetAsync(flag, 0, (nb + 1) * sizeof(int), st));  // flag[nb] stays 0 for the scan
        if (nc > 0)
            k_wfar_count<<<nblocks(nc, 256), 256, 0, st>>>(nc, T->ctr_box, L->start[LWF], L->idx[LWF], cm_cnt, d_cnt);
        QBX_LAUNCH_CHECK();
        exclusive_scan(cm_cnt, pl->cm_start, nc + 1, 0, tot, st);
        int np = 0;
        QBX_CUDA_TRY(cudaMemcpyAsync(&np, tot, sizeof(int), cudaMemcpyDeviceToHost, st));
        exclusive_scan(d_cnt, d_start, nb + 1, 0, nullptr, st);
        k_flag_pos<<<nblocks(nb, 256), 256, 0, st>>>(nb, d_cnt, flag);
        exclusive_scan(flag, flag, nb + 1, 0, tot, st);
        int nd = 0;
        QBX_CUDA_TRY(cudaMemcpyAsync(&nd, tot, sizeof(int), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        pl->npairs = np;
        pl->ndsrc = nd;
        pl->slot_box = dalloc<int>(std::max(nd, 1));
        k_wfar_slots<<<nblocks(nb, 256), 256, 0, st>>>(nb, d_cnt, flag, pl->slot, pl->slot_box);
        pl->pair_ctr = dalloc<int>(std::max(np, 1));
        pl->pair_d = dalloc<int>(std::max(np, 1));
        pl->pos_cm = dalloc<int>(std::max(np, 1));
        int *d_fill = flag;  // reuse
        QBX_CUDA_TRY(cudaMemcpyAsync(d_fill, d_start, (nb + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
        if (nc > 0)
            k_wfar_fill<<<nblocks(nc, 256), 256, 0, st>>>(nc, T->ctr_box, L->start[LWF], L->idx[LWF], pl->cm_start,
                                                          d_fill, pl->pair_ctr, pl->pair_d, pl->pos_cm);
        QBX_LAUNCH_CHECK();
        std::vector<int> ds(nb + 1);
        QBX_CUDA_TRY(cudaMemcpyAsync(ds.data(), d_start, (nb + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        const int WT = wfar_tile_width(pl->K, pl->R);
        pl->tc = tc && wfar_tc_layout(pl, w_hint);  // orders beyond the tensor-core layout use the FP32 form
        if (pl->tc) {
            set_recurrence_tables(st);
            std::vector<int4> tct;
            for (int d = 0; d < nb; ++d)
                for (int p = ds[d]; p < ds[d + 1]; p += 128) tct.push_back(make_int4(d, p, std::min(p + 128, ds[d + 1]), 0));
            pl->ntc = (int)tct.size();
            pl->tc_tiles = dalloc<int4>(std::max<size_t>(tct.size(), 1));
            if (!tct.empty())
                QBX_CUDA_TRY(cudaMemcpyAsync(pl->tc_tiles, tct.data(), tct.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                             st));
            pl->H_tc = dalloc<float>((int64_t)std::max(nd, 1) * 2 * pl->Rp * pl->Kp);  // TF32 hi and lo tiles
            {
                const std::vector<WfarRecipe> rec = wfar_recipe(pl);
                std::vector<float> fac(rec.size());
                std::vector<uint32_t> code(rec.size());
                for (size_t e = 0; e < rec.size(); ++e) {
                    const WfarRecipe &r = rec[e];
                    if (r.t1 >= 0 && r.t2 >= 0 && std::fabs(r.f1) != std::fabs(r.f2))
                        throw Error{QBX_ERR_CUDA, "List 3 far recipe: terms of unequal magnitude"};
                    fac[e] = r.t1 >= 0 ? std::fabs(r.f1) : (r.t2 >= 0 ? std::fabs(r.f2) : 0.f);
                    code[e] = (uint32_t)(r.t1 >= 0 ? r.t1 : WF_NOTERM) | (uint32_t)(r.t2 >= 0 ? r.t2 : WF_NOTERM) << 10 |
                              (uint32_t)(r.bits >> 8) << 20 | (uint32_t)(r.bits & 1) << 26 |
                              (uint32_t)(r.t1 >= 0 && r.f1 < 0.f) << 27 | (uint32_t)(r.t2 >= 0 && r.f2 < 0.f) << 28;
                }
                pl->rec_fac = dalloc<float>(fac.size());
                pl->rec_code = dalloc<uint32_t>(code.size());
                QBX_CUDA_TRY(cudaMemcpyAsync(pl->rec_fac, fac.data(), fac.size() * sizeof(float), cudaMemcpyHostToDevice, st));
                QBX_CUDA_TRY(cudaMemcpyAsync(pl->rec_code, code.data(), code.size() * sizeof(uint32_t),
                                             cudaMemcpyHostToDevice, st));
                QBX_CUDA_TRY(cudaStreamSynchronize(st));
            }
            pl->Y = dalloc<float>((int64_t)std::max(np, 1) * pl->R);
            const size_t sm = wfar_tc_smem(pl->Rp, pl->WMAX, Q);
            if (pl->NU == 5)
                QBX_CUDA_TRY(cudaFuncSetAttribute(k_wfar_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            else
                QBX_CUDA_TRY(cudaFuncSetAttribute(k_wfar_tc<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            pl->cenf = dalloc<float>((int64_t)std::max(nb, 1) * 8);
            if (nb > 0) k_cen_to_df<<<nblocks(nb, 256), 256, 0, st>>>(nb, T->cen, T->hw, pl->cenf);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            dfree(cm_cnt); dfree(d_cnt); dfree(d_start); dfree(flag); dfree(tot);
            return pl;
        }
        if (pl->R > 320 || wfar_smem(pl->K, pl->R, WT) > 227 * 1024)
            throw Error{QBX_ERR_INVALID_ARG, "orders too high for the mixed List 3 far product"};
        std::vector<int2> tiles;
        for (int d = 0; d < nb; ++d)
            for (int p = ds[d]; p < ds[d + 1]; p += WT) tiles.push_back(make_int2(p, std::min(p + WT, ds[d + 1])));
        pl->ntiles = (int)tiles.size();
        pl->tiles = dalloc<int2>(std::max<size_t>(tiles.size(), 1));
        if (!tiles.empty())
            QBX_CUDA_TRY(cudaMemcpyAsync(pl->tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                         st));
        pl->H = dalloc<float>((int64_t)std::max(nd, 1) * pl->R * pl->K);
        pl->Y = dalloc<float>((int64_t)std::max(np, 1) * pl->R);
        size_t smem = wfar_smem(pl->K, pl->R, WT);
        switch (wfar_rows_per_thread(pl->R)) {
        case 2: wfar_set_smem<2>(smem); break;
        case 3: wfar_set_smem<3>(smem); break;
        case 5: wfar_set_smem<5>(smem); break;
        default: wfar_set_smem<10>(smem); break;
        }
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(cm_cnt); dfree(d_cnt); dfree(d_start); dfree(flag); dfree(tot);
        free_wfar_plan(pl);
        throw;
    }
    dfree(cm_cnt); dfree(d_cnt); dfree(d_start); dfree(flag); dfree(tot);
    return pl;
}

void wfar_mixed_run(const qbx_tree *T, WfarPlan *pl, int PMT, const double2 *Mu, const signed char *pb, const float *cf,
                    int *err, long long wait_limit, int probe_step, cudaStream_t st)
{
    if (pl->npairs == 0) return;
    if (pl->tc) {
        WfarChunks ch;
        ch.nch = pl->nch;
        ch.R = pl->R;
        ch.Rp = pl->Rp;
        ch.Kp = pl->Kp;
        for (int c = 0; c < WF_MAXCH; ++c) {
            ch.cj0[c] = pl->cj0[c];
            ch.cj1[c] = pl->cj1[c];
        }
        for (int c = 0; c <= WF_MAXCH; ++c) ch.ckoff[c] = pl->ckoff[c];
        if (pl->ndsrc > 0)
            k_wfar_H_tc<<<pl->ndsrc, 256, 0, st>>>(pl->P, PMT, pl->Rp, ch, reinterpret_cast<const float4 *>(pl->rec_fac),
                                                    reinterpret_cast<const uint4 *>(pl->rec_code), pl->slot_box, pb,
                                                    Mu, reinterpret_cast<float4 *>(pl->H_tc));
        QBX_LAUNCH_CHECK();
        int dev = 0, nsm = 0;
        QBX_CUDA_TRY(cudaGetDevice(&dev));
        QBX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        int cols = 32;
        while (cols < pl->Rp) cols <<= 1;  // one accumulator; two are allocated
        WfarTcArgs a{pl->ntc, pl->P, pl->Q, pl->P + pl->Q, pl->R, pl->Rp, pl->WMAX, cols, 2 * cols, ch, pl->tc_tiles,
                     pl->pair_ctr, pl->slot, pl->H_tc, cf, pl->cenf, T->cr, T->np[KCTR], pl->Y, err,
                     wait_limit > 0 ? wait_limit : tc::WAIT_LIMIT, probe_step};
        const size_t sm = wfar_tc_smem(pl->Rp, pl->WMAX, pl->Q);
        const int grid = std::min(pl->ntc, nsm);
        if (pl->NU == 5) k_wfar_tc<5><<<grid, WF_THREADS, sm, st>>>(a);
        else k_wfar_tc<7><<<grid, WF_THREADS, sm, st>>>(a);
        QBX_LAUNCH_CHECK();
        return;
    }
    int64_t nH = (int64_t)pl->ndsrc * pl->R * pl->K;
    k_wfar_H<<<nblocks(nH, 256), 256, 0, st>>>(pl->ndsrc, pl->P, pl->Q, PMT, pl->slot_box, pb, Mu, pl->H);
    QBX_LAUNCH_CHECK();
    const int WT = wfar_tile_width(pl->K, pl->R);
    size_t smem = wfar_smem(pl->K, pl->R, WT);
    switch (wfar_rows_per_thread(pl->R)) {
    case 2: wfar_launch<2>(T, pl, smem, st); break;
    case 3: wfar_launch<3>(T, pl, smem, st); break;
    case 5: wfar_launch<5>(T, pl, smem, st); break;
    default: wfar_launch<10>(T, pl, smem, st); break;
    }
    QBX_LAUNCH_CHECK();
}

void wfar_mixed_reduce(const qbx_tree *T, WfarPlan *pl, int QMS, const signed char *qc, double2 *A, cudaStream_t st)
{
    if (pl->npairs == 0) return;
    const int64_t nc = T->np[KCTR];
    k_wfar_reduce<<<nblocks(nc * pl->R, 256), 256, 0, st>>>(nc, pl->Q, QMS, pl->cm_start, pl->pos_cm, pl->Y, qc, A);
    QBX_LAUNCH_CHECK();
}

}  // namespace qbx
