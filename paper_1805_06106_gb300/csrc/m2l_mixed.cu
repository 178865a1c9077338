// List 2 M2L (Algorithm 4 Stage 4) in mixed precision, as batched dense per-offset products.
//
// With box-scaled expansions the M2L operator between two same-level boxes depends only on
// their integer offset o = ic_b - ic_d (|o|_inf in [3, 5]).  In the balanced scaling
//   Mh_n^m = Mu_n^m F(n,m),  Bh_k^l = B_k^l / F(k,l),  F(n,m) = sqrt((n+|m|)!(n-|m|)!),
// the operator is
//   Bh_k^l = 1/h sum_{n,m} Mh_n^m conj S_{n+k}^{m+l}(2o) / (F(n,m) F(k,l)),
// whose entries are bounded by 2^(n+k) / 6^(n+k+1) <= 1, so it is well represented in FP32.
// Written on real vectors of length D = (P+1)^2 (per degree n: Re X_n^0, then Re X_n^m, Im X_n^m
// for m = 1..n) it becomes one real D x D matrix per offset.  The operator is generated in FP64
// from the irregular-harmonic table and rounded to FP32.
//
// Per evaluation: multipoles are converted to the balanced real layout (FP32), one GEMM per
// offset multiplies the offset's matrix by the gathered source multipoles of all pairs with that
// offset (FP32 accumulation), each pair's result is stored, and a per-box reduction adds the
// pairs of the box's List 2 in list order in compensated FP32 (deterministic), undoes the scaling
// and adds into the FP64 local expansion.
#include <algorithm>
#include <cmath>
#include <vector>

#include "harmonics.cuh"
#include "tc_common.cuh"

namespace qbx {

struct M2LPlan {
    int P = -1, D = 0;
    int64_t npairs = 0;
    int ntiles = 0;
    float *mats = nullptr;        // 1331 x D x D, row-major (output row, input column)
    int *pair_src = nullptr;      // source box of each pair, pairs sorted by offset
    int *pair_pos = nullptr;      // for List 2 entry e (CSR order): its position in the sorted pairs
    int2 *tiles = nullptr;        // (offset, first pair) of each GEMM column tile
    int *off_start = nullptr;     // 1332: pair range of each offset
    float *mh = nullptr;          // n_boxes x D balanced multipoles
    float *y = nullptr;           // npairs x D per-pair results
    // split-TF32 tensor-core form (QBX_M2L_3XTF32)
    bool tc = false;
    int Np = 0, Dp = 0, KC = 0, nch = 0, ntc = 0;
    float *mats_tc = nullptr;     // 1331 x nch x {hi, lo} x (Np x KC K-major tiles)
    float *mh_hi = nullptr, *mh_lo = nullptr;  // n_boxes x Dp
    int4 *tc_tiles = nullptr;     // (offset, first pair, last pair + 1) per 128-pair tile
};

int m2l_plan_order(const M2LPlan *p) { return p ? (p->P * 2 + (p->tc ? 1 : 0)) * 64 + (p->tc ? p->KC : 0) : -1; }

void free_m2l_plan(M2LPlan *p)
{
    if (!p) return;
    dfree(p->mats); dfree(p->pair_src); dfree(p->pair_pos); dfree(p->tiles); dfree(p->off_start);
    dfree(p->mh); dfree(p->y);
    dfree(p->mats_tc); dfree(p->mh_hi); dfree(p->mh_lo); dfree(p->tc_tiles);
    delete p;
}

__device__ __forceinline__ double ffac_sqrt(int n, int m)  // F(n, m) = sqrt((n+|m|)!(n-|m|)!)
{
    int am = m < 0 ? -m : m;
    double f = 1.0;
    for (int i = 2; i <= n + am; ++i) f *= i;
    for (int i = 2; i <= n - am; ++i) f *= i;
    return sqrt(f);
}

// F(n, m) for n <= PMAX, m >= 0 (tri layout), the same products and correctly rounded square root as
// ffac_sqrt, computed on the host when a plan is built: the per-element kernels look it up (an FP64
// product chain and square root per element would occupy the FP64 pipe)
__device__ double g_fsq[ntri(PMAX)];

static void set_fsq_table(cudaStream_t st)
{
    double h[ntri(PMAX)];
    for (int n = 0; n <= PMAX; ++n)
        for (int m = 0; m <= n; ++m) {
            double f = 1.0;
            for (int i = 2; i <= n + m; ++i) f *= i;
            for (int i = 2; i <= n - m; ++i) f *= i;
            h[tri(n, m)] = std::sqrt(f);
        }
    QBX_CUDA_TRY(cudaMemcpyToSymbolAsync(g_fsq, h, sizeof h, 0, cudaMemcpyHostToDevice, st));
    QBX_CUDA_TRY(cudaStreamSynchronize(st));
}

// real-layout index of (n, m >= 0, part)
__host__ __device__ __forceinline__ int ridx(int n, int m, int part) { return n * n + (m == 0 ? 0 : 2 * m - 1 + part); }

// Entry (row, col) of the balanced real operator of List 2 offset with irregular table S (FP64).
__device__ double m2l_entry(int D, const double2 *S, int row, int col)
{
    int k = (int)sqrtf((float)row);
    while (k * k > row) --k;
    while ((k + 1) * (k + 1) <= row) ++k;
    int rr = row - k * k;  // 0 -> (l=0,re), 2l-1 -> (l,re), 2l -> (l,im)
    int l = (rr + 1) / 2, rpart = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
    int n = (int)sqrtf((float)col);
    while (n * n > col) --n;
    while ((n + 1) * (n + 1) <= col) ++n;
    int cc = col - n * n;
    int m = (cc + 1) / 2, cpart = (cc == 0) ? 0 : ((cc & 1) ? 0 : 1);
    double scale = 1.0 / (ffac_sqrt(n, m) * ffac_sqrt(k, l));
    double2 c1 = cconj(sym_get(S, n + k, m + l));
    double2 c2 = make_double2(0.0, 0.0);
    if (m > 0) c2 = cconj(sym_get(S, n + k, -m + l));
    double s = (m & 1) ? -1.0 : 1.0;
    double2 plus = make_double2(c1.x + s * c2.x, c1.y + s * c2.y);
    double2 minus = make_double2(c1.x - s * c2.x, c1.y - s * c2.y);
    double e;
    if (rpart == 0 && cpart == 0) e = plus.x;
    else if (rpart == 0 && cpart == 1) e = -minus.y;
    else if (rpart == 1 && cpart == 0) e = plus.y;
    else e = minus.x;
    return e * scale;
}

__device__ __forceinline__ bool m2l_offset_valid(int o)
{
    int ox = o % 11 - 5, oy = (o / 11) % 11 - 5, oz = o / 121 - 5;
    return max(abs(ox), max(abs(oy), abs(oz))) >= 3;
}

// One block per offset; entries from the FP64 irregular table (stride ntri(2 PMT)).
__global__ void k_m2l_mats(int P, int PMT, const double2 *stab, float *mats)
{
    const int o = blockIdx.x;
    const int D = (P + 1) * (P + 1);
    float *Mo = mats + (int64_t)o * D * D;
    const double2 *S = stab + (int64_t)o * ntri(2 * PMT);
    const bool valid = m2l_offset_valid(o);
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x)
        Mo[idx] = valid ? (float)m2l_entry(D, S, idx / D, idx % D) : 0.f;
}

// Split-TF32 operators in K-major tiles: for offset o and K chunk c (columns c KC .. c KC + KC - 1)
// the hi tile (Np rows x KC) then the lo tile, each laid out as tc::kmajor_off with SBO = KC * 32.
// Rows >= D and columns >= D are zero.
__global__ void k_m2l_mats_tc(int P, int PMT, int Np, int Dp, int KC, const double2 *stab, float *mats)
{
    const int o = blockIdx.x;
    const int D = (P + 1) * (P + 1), nch = Dp / KC;
    const double2 *S = stab + (int64_t)o * ntri(2 * PMT);
    const bool valid = m2l_offset_valid(o);
    float *Mo = mats + (int64_t)o * Np * Dp * 2;
    for (int idx = threadIdx.x; idx < Np * Dp; idx += blockDim.x) {
        int row = idx / Dp, col = idx % Dp;
        double e = (valid && row < D && col < D) ? m2l_entry(D, S, row, col) : 0.0;
        float hi, lo;
        tc::split_tf32(e, hi, lo);
        int c = col / KC, kk = col % KC;
        float *tile = Mo + (int64_t)c * 2 * Np * KC;
        uint32_t off = tc::kmajor_off(row, kk, (uint32_t)KC * 32u) / 4u;
        tile[off] = hi;
        tile[(int64_t)Np * KC + off] = lo;
    }
    (void)nch;
}

__global__ void k_pair_offsets(int nb, const int *vstart, const int *vidx, const int64_t *ic, int *code, int *cnt)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int e = vstart[b]; e < vstart[b + 1]; ++e) {
        int d = vidx[e];
        int ox = (int)(ic[3 * b] - ic[3 * d]), oy = (int)(ic[3 * b + 1] - ic[3 * d + 1]),
            oz = (int)(ic[3 * b + 2] - ic[3 * d + 2]);
        int c = (ox + 5) + 11 * (oy + 5) + 121 * (oz + 5);
        bool ok = ox >= -5 && ox <= 5 && oy >= -5 && oy <= 5 && oz >= -5 && oz <= 5;
        code[e] = ok ? c : 0;  // offset 0 holds a zero operator
        atomicAdd(&cnt[ok ? c : 0], 1);
    }
}

// Balanced real multipoles: Mh[b][ridx(n,m,part)] = (Mu_n^m F(n,m)).{re,im}
__global__ void k_mhat(int64_t nb, int P, int PMT, const double2 *Mu, float *mh)
{
    const int D = (P + 1) * (P + 1);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * D) return;
    int64_t b = i / D;
    int r = (int)(i % D);
    int n = (int)sqrtf((float)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    int rr = r - n * n;
    int m = (rr + 1) / 2, part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
    double2 v = Mu[b * ntri(PMT) + tri(n, m)];
    mh[i] = (float)((part ? v.y : v.x) * __ldg(&g_fsq[tri(n, m)]));
}

// FP32 SIMT GEMM per offset tile: Y[pair] = Mats[o] * Mh[src(pair)], block = 64 rows x 64 pairs.
constexpr int GM = 64, GN = 64, GK = 16;
__global__ void __launch_bounds__(256) k_m2l_gemm_fp32(int D, const int2 *tiles, const int *off_start,
                                                       const int *pair_src, const float *mats, const float *mh,
                                                       float *y)
{
    __shared__ float As[GK][GM + 4];
    __shared__ float Bs[GK][GN + 4];
    const int2 tl = tiles[blockIdx.x];
    const int o = tl.x, p0 = tl.y, p1 = min(off_start[o + 1], p0 + GN);
    const int row0 = blockIdx.y * GM;
    const float *A = mats + (int64_t)o * D * D;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 outputs each
    float acc[4][4] = {};
    for (int k0 = 0; k0 < D; k0 += GK) {
        for (int i = threadIdx.x; i < GM * GK; i += 256) {
            int r = i / GK, k = i % GK;
            int gr = row0 + r, gk = k0 + k;
            As[k][r] = (gr < D && gk < D) ? A[(int64_t)gr * D + gk] : 0.f;
        }
        for (int i = threadIdx.x; i < GN * GK; i += 256) {
            int c = i / GK, k = i % GK;
            int p = p0 + c, gk = k0 + k;
            Bs[k][c] = (p < p1 && gk < D) ? mh[(int64_t)pair_src[p] * D + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int r = row0 + ty * 4 + i, p = p0 + tx * 4 + j;
            if (r < D && p < p1) y[(int64_t)p * D + r] = acc[i][j];
        }
}

// Balanced real multipoles split into TF32 hi / lo parts, rows padded to Dp with zeros.
__global__ void k_mhat_tc(int64_t nb, int P, int PMT, int Dp, const double2 *Mu, float *mh_hi, float *mh_lo)
{
    const int D = (P + 1) * (P + 1);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * Dp) return;
    int64_t b = i / Dp;
    int r = (int)(i % Dp);
    double v = 0.0;
    if (r < D) {
        int n = (int)sqrtf((float)r);
        while (n * n > r) --n;
        while ((n + 1) * (n + 1) <= r) ++n;
        int rr = r - n * n;
        int m = (rr + 1) / 2, part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
        double2 c = Mu[b * ntri(PMT) + tri(n, m)];
        v = (part ? c.y : c.x) * __ldg(&g_fsq[tri(n, m)]);
    }
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    mh_hi[i] = hi;
    mh_lo[i] = lo;
}

// Tensor-core List 2 products.  Persistent CTAs of 256 threads walk the 128-pair tiles; a tile
// computes Y[pair][row] = sum_col Mats_o[row][col] Mh[src(pair)][col] as D = A B^T with
// A = gathered multipoles (128 pairs x Dp, K-major) and B = the offset's operator (Np x Dp,
// K-major), in K chunks of KC columns through a two-stage pipeline: the operator chunk arrives by
// a bulk copy, the multipole chunk is gathered by the threads, one thread issues the split-TF32
// MMAs (a_hi b_hi + a_lo b_hi + a_hi b_lo) into a 128 x Np FP32 accumulator in tensor memory.
struct M2LTcArgs {
    int ntiles, D, Dp, Np, KC, tmem_cols;
    const int4 *tiles;
    const int *pair_src;
    const float *mh_hi, *mh_lo, *mats;
    float *y;
    int *err;
    long long wait_limit;  // clock cycles a pipeline wait may take before it gives up
    int probe_step;        // failure-path probe: pipeline step at which the wait on bar_never runs out (-1: off)
};

__global__ void __launch_bounds__(256, 1) k_m2l_tc(M2LTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ uint64_t bar_b[2], bar_mma[2], bar_never;  // bar_never: nothing ever arrives on it
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = a.KC, Np = a.Np, nch = a.Dp / KC;
    const uint32_t sboA = (uint32_t)KC * 32u + 16u, sboB = (uint32_t)KC * 32u;
    const uint32_t bytesA = 16u * sboA, bytesB = (uint32_t)Np * KC * 4u;
    // stage s, part 0 (hi) / 1 (lo) of the A and B tiles
    auto Abuf = [&](int s, int part) { return smem_tc + (size_t)(2 * s + part) * bytesA; };
    auto Bbuf = [&](int s, int part) { return smem_tc + (size_t)4 * bytesA + (size_t)(2 * s + part) * bytesB; };
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&bar_b[s], 1);
            tc::mbar_init(&bar_mma[s], 1);
        }
        tc::mbar_init(&bar_never, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, (uint32_t)a.tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t nsplit = Np > 256 ? 2u : 1u;
    const int N0 = Np > 256 ? 256 : Np, N1 = Np - N0;
    const uint32_t id0 = tc::idesc_tf32(128, N0), id1 = tc::idesc_tf32(128, N1 > 0 ? N1 : 16);
    bool ok = true;
    uint32_t g = 0;  // chunks issued by this CTA (pipeline position)
    const int pieces = KC / 4, nq = (128 * pieces) / 256;  // float4 pieces per thread: 4 (KC 32) or 2 (KC 16)
    float4 hv[4], lv[4];
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const int o = tl.x, p0 = tl.y, np = tl.z - tl.y;
        auto load_a = [&](int cc) {
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                hv[it] = lv[it] = make_float4(0.f, 0.f, 0.f, 0.f);
                const int q = tid + 256 * it;
                const int row = (q & 7) + 8 * (q / (8 * pieces)), pc = (q >> 3) % pieces;
                if (it < nq && row < np) {
                    int64_t src = (int64_t)a.pair_src[p0 + row] * a.Dp + cc * KC + 4 * pc;
                    hv[it] = __ldg(reinterpret_cast<const float4 *>(a.mh_hi + src));
                    lv[it] = __ldg(reinterpret_cast<const float4 *>(a.mh_lo + src));
                }
            }
        };
        load_a(0);
        for (int c = 0; c < nch; ++c, ++g) {
            const int s = g & 1;
            const uint32_t use = g >> 1;
            if (g >= 2 && ok) ok = tc::mbar_wait(&bar_mma[s], (use - 1) & 1, a.wait_limit);
            if (__syncthreads_or(!ok)) { ok = false; break; }
            if (tid == 0) {
                tc::mbar_arrive_expect_tx(&bar_b[s], 2u * bytesB);
                tc::bulk_g2s(Bbuf(s, 0), a.mats + ((int64_t)o * nch + c) * 2 * Np * KC, 2u * bytesB, &bar_b[s]);
            }
            // eight consecutive threads fill one 128-byte core matrix (rows 8g..8g+7 of one 16-byte
            // column piece): conflict-free stores, 64-byte row segments per warp in global memory.
            // The multipoles of the next chunk are loaded before this chunk's MMAs are issued.
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int q = tid + 256 * it;
                const int row = (q & 7) + 8 * (q / (8 * pieces)), pc = (q >> 3) % pieces;
                if (it < nq) {
                    uint32_t off = tc::kmajor_off(row, 4 * pc, sboA);
                    *reinterpret_cast<float4 *>(Abuf(s, 0) + off) = hv[it];
                    *reinterpret_cast<float4 *>(Abuf(s, 1) + off) = lv[it];
                }
            }
            if (c + 1 < nch) load_a(c + 1);
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                bool got;
                if ((int)g == a.probe_step) {
                    got = tc::mbar_wait(&bar_never, 0, a.wait_limit);  // runs out: nothing arrives
                    tc::mbar_wait(&bar_b[s], use & 1, tc::WAIT_LIMIT);  // drain this step's copy
                } else {
                    got = tc::mbar_wait(&bar_b[s], use & 1, a.wait_limit);
                    if (!got) tc::mbar_wait(&bar_b[s], use & 1, tc::WAIT_LIMIT);  // drain a late copy
                }
                if (got) {
                    tc::tc_fence_after();
                    const uint32_t a_hi = tc::smem_u32(Abuf(s, 0)), a_lo = tc::smem_u32(Abuf(s, 1));
                    const uint32_t b_hi = tc::smem_u32(Bbuf(s, 0)), b_lo = tc::smem_u32(Bbuf(s, 1));
                    for (int ks = 0; ks < KC / 8; ++ks) {
                        for (uint32_t h = 0; h < nsplit; ++h) {
                            const uint32_t boff = h * 32u * sboB + 256u * ks, aoff = 256u * ks;
                            const uint32_t dcol = tmem + h * 256u, id = h ? id1 : id0;
                            const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                            tc::mma_tf32(dcol, tc::sdesc(a_hi + aoff, 128, sboA), tc::sdesc(b_hi + boff, 128, sboB), id, acc0);
                            tc::mma_tf32(dcol, tc::sdesc(a_lo + aoff, 128, sboA), tc::sdesc(b_hi + boff, 128, sboB), id, 1u);
                            tc::mma_tf32(dcol, tc::sdesc(a_hi + aoff, 128, sboA), tc::sdesc(b_lo + boff, 128, sboB), id, 1u);
                        }
                    }
                } else {
                    atomicOr(a.err, 8);
                    ok = false;  // the other threads learn it at the next barrier
                }
                tc::mma_commit(&bar_mma[s]);  // also releases the stage when the MMAs were skipped
            }
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        // epilogue: lane quarter (warp & 3) holds pairs 32 q .. 32 q + 31; column groups of 16 split
        // between warps w and w + 4
        const int sl = (g - 1) & 1;
        ok = tc::mbar_wait(&bar_mma[sl], ((g - 1) >> 1) & 1, a.wait_limit);
        if (__syncthreads_or(!ok)) { ok = false; break; }
        tc::tc_fence_after();
        // Output rows of consecutive pairs are contiguous in Y: stage column blocks of 128 through
        // shared memory (row stride 132 floats) and copy them out with coalesced 16-byte stores.
        const int qd = warp & 3, row = 32 * qd + lane;
        float *stage = reinterpret_cast<float *>(smem_tc);  // 128 x 132 floats; the operand tiles are idle
        for (int c0 = 0; c0 < a.D; c0 += 128) {
            const int cw = min(128, a.D - c0);
            for (int cg = warp >> 2; cg * 16 < cw; cg += 2) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(c0 + cg * 16), v);
                float4 *dst = reinterpret_cast<float4 *>(stage + row * 132 + cg * 16);
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
            __syncthreads();
            const int c4 = cw / 4;  // D is a multiple of 4 only for odd P; copy scalars otherwise
            if ((a.D & 3) == 0) {
                for (int q = tid; q < np * c4; q += 256) {
                    const int r = q / c4, cc = q % c4;
                    *reinterpret_cast<float4 *>(a.y + (int64_t)(p0 + r) * a.D + c0 + 4 * cc) =
                        *reinterpret_cast<const float4 *>(stage + r * 132 + 4 * cc);
                }
            } else {
                for (int q = tid; q < np * cw; q += 256) {
                    const int r = q / cw, cc = q % cw;
                    a.y[(int64_t)(p0 + r) * a.D + c0 + cc] = stage[r * 132 + cc];
                }
            }
            __syncthreads();
        }
        tc::tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(a.err, 8);
    // wait for this CTA's last MMAs before releasing tensor memory
    if (g > 0 && tid == 0) tc::mbar_wait(&bar_mma[(g - 1) & 1], ((g - 1) >> 1) & 1, tc::WAIT_LIMIT);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// operand stages, or the 128 x 132 float epilogue stage that reuses them, whichever is larger
static size_t m2l_tc_smem(int Np, int KC)
{
    return std::max((size_t)4 * 16 * (KC * 32 + 16) + (size_t)4 * Np * KC * 4, (size_t)128 * 132 * 4);
}

// B[b] += F(k,l)/h_b * sum_{e in V(b)} Y[pos(e)], summed in list order in compensated FP32.
__global__ void k_m2l_reduce(int64_t nb, int P, int PMT, const int *vstart, const int *pair_pos, const float *y,
                             const double *hw, const signed char *pb, double2 *B)
{
    const int D = (P + 1) * (P + 1);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * D) return;
    int b = (int)(i / D), r = (int)(i % D);
    int e0 = vstart[b], e1 = vstart[b + 1];
    if (e0 == e1) return;
    int k = (int)sqrtf((float)r);
    while (k * k > r) --k;
    while ((k + 1) * (k + 1) <= r) ++k;
    if (k > pb[b]) return;
    int rr = r - k * k;
    int l = (rr + 1) / 2, part = (rr == 0) ? 0 : ((rr & 1) ? 0 : 1);
    // list-order sum in compensated FP32 (FP64 adds of converted terms would occupy the FP64 pipe);
    // eight independent loads in flight per step
    float hi = 0.f, lo = 0.f;
    int e = e0;
    for (; e + 8 <= e1; e += 8) {
        int q[8];
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = pair_pos[e + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(y + (int64_t)q[u] * D + r);
#pragma unroll
        for (int u = 0; u < 8; ++u) tc::df_add(hi, lo, v[u]);
    }
    for (; e < e1; ++e) tc::df_add(hi, lo, __ldg(y + (int64_t)pair_pos[e] * D + r));
    double s = ((double)hi + (double)lo) * (__ldg(&g_fsq[tri(k, l)]) / hw[b]);
    double2 *t = B + (int64_t)b * ntri(PMT) + tri(k, l);
    if (part) t->y += s;
    else t->x += s;
}

__global__ void k_scatter_pairs(int nb, const int *vstart, const int *vidx, const int *code, int *fill,
                                int *pair_src, int *pair_pos)
{
    // one thread per box: entries are placed in CSR order within an offset, so the
    // assignment is deterministic only up to the order boxes reach the atomic; the
    // reduction reads pairs through pair_pos in list order, which keeps sums deterministic.
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int e = vstart[b]; e < vstart[b + 1]; ++e) {
        int p = atomicAdd(&fill[code[e]], 1);
        pair_src[p] = vidx[e];
        pair_pos[e] = p;
    }
}

M2LPlan *m2l_plan_build(const qbx_tree *T, const qbx_lists *L, int P, int PMT, const double2 *stab, bool tc,
                        int kc_hint, cudaStream_t st)
{
    M2LPlan *pl = new M2LPlan();
    try {
        set_fsq_table(st);
        pl->P = P;
        pl->D = (P + 1) * (P + 1);
        pl->tc = tc;
        const int nb = (int)T->nb;
        const int64_t np = L->nnz[LV];
        pl->npairs = np;
        if (tc) {
            pl->Np = (pl->D + 15) / 16 * 16;
            pl->KC = pl->Np > 256 ? 16 : 32;
            if (kc_hint == 16 || (kc_hint == 32 && m2l_tc_smem(pl->Np, 32) <= 220 * 1024)) pl->KC = kc_hint;
            pl->Dp = (pl->D + pl->KC - 1) / pl->KC * pl->KC;
            pl->nch = pl->Dp / pl->KC;
            pl->mats_tc = dalloc<float>((int64_t)1331 * pl->Np * pl->Dp * 2);
            k_m2l_mats_tc<<<1331, 256, 0, st>>>(P, PMT, pl->Np, pl->Dp, pl->KC, stab, pl->mats_tc);
            QBX_LAUNCH_CHECK();
            pl->mh_hi = dalloc<float>((int64_t)nb * pl->Dp);
            pl->mh_lo = dalloc<float>((int64_t)nb * pl->Dp);
            QBX_CUDA_TRY(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)m2l_tc_smem(pl->Np, pl->KC)));
        } else {
            pl->mats = dalloc<float>((int64_t)1331 * pl->D * pl->D);
            k_m2l_mats<<<1331, 256, 0, st>>>(P, PMT, stab, pl->mats);
            QBX_LAUNCH_CHECK();
        }
        int *code = dalloc<int>(np), *cnt = dalloc<int>(1332), *fill = dalloc<int>(1332);
        pl->off_start = dalloc<int>(1332);
        pl->pair_src = dalloc<int>(np);
        pl->pair_pos = dalloc<int>(np);
        QBX_CUDA_TRY(cudaMemsetAsync(cnt, 0, 1332 * sizeof(int), st));
        k_pair_offsets<<<nblocks(nb, 128), 128, 0, st>>>(nb, L->start[LV], L->idx[LV], T->ic, code, cnt);
        QBX_LAUNCH_CHECK();
        exclusive_scan(cnt, pl->off_start, 1332, 0, nullptr, st);
        QBX_CUDA_TRY(cudaMemcpyAsync(fill, pl->off_start, 1332 * sizeof(int), cudaMemcpyDeviceToDevice, st));
        k_scatter_pairs<<<nblocks(nb, 128), 128, 0, st>>>(nb, L->start[LV], L->idx[LV], code, fill, pl->pair_src,
                                                          pl->pair_pos);
        QBX_LAUNCH_CHECK();
        std::vector<int> os(1332);
        QBX_CUDA_TRY(cudaMemcpyAsync(os.data(), pl->off_start, 1332 * sizeof(int), cudaMemcpyDeviceToHost, st));
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
        dfree(code); dfree(cnt); dfree(fill);
        std::vector<int2> tiles;
        std::vector<int4> tct;
        for (int o = 0; o < 1331; ++o) {
            for (int p = os[o]; p < os[o + 1]; p += GN) tiles.push_back(make_int2(o, p));
            for (int p = os[o]; p < os[o + 1]; p += 128) tct.push_back(make_int4(o, p, std::min(p + 128, os[o + 1]), 0));
        }
        if (tc) {
            pl->ntc = (int)tct.size();
            pl->tc_tiles = dalloc<int4>(std::max<size_t>(tct.size(), 1));
            if (!tct.empty())
                QBX_CUDA_TRY(cudaMemcpyAsync(pl->tc_tiles, tct.data(), tct.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                             st));
        } else {
            pl->ntiles = (int)tiles.size();
            pl->tiles = dalloc<int2>(std::max<size_t>(tiles.size(), 1));
            if (!tiles.empty())
                QBX_CUDA_TRY(cudaMemcpyAsync(pl->tiles, tiles.data(), tiles.size() * sizeof(int2),
                                             cudaMemcpyHostToDevice, st));
            pl->mh = dalloc<float>((int64_t)nb * pl->D);
        }
        pl->y = dalloc<float>(std::max<int64_t>(np, 1) * pl->D);
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        free_m2l_plan(pl);
        throw;
    }
    return pl;
}

void m2l_mixed_run(const qbx_tree *T, const qbx_lists *L, M2LPlan *pl, int PMT, const double2 *Mu, double2 *B,
                   const signed char *pb, int *err, cudaStream_t st)
{
    const int64_t nb = T->nb;
    const int D = pl->D;
    if (pl->tc) {
        k_mhat_tc<<<nblocks(nb * pl->Dp, 256), 256, 0, st>>>(nb, pl->P, PMT, pl->Dp, Mu, pl->mh_hi, pl->mh_lo);
        QBX_LAUNCH_CHECK();
        if (pl->ntc > 0) {
            int dev = 0, nsm = 0;
            QBX_CUDA_TRY(cudaGetDevice(&dev));
            QBX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            int cols = 32;
            while (cols < pl->Np) cols <<= 1;
            M2LTcArgs a{pl->ntc,      D,         pl->Dp,   pl->Np,   pl->KC, cols,
                        pl->tc_tiles, pl->pair_src, pl->mh_hi, pl->mh_lo, pl->mats_tc, pl->y,
                        err,          L->wait_limit > 0 ? L->wait_limit : tc::WAIT_LIMIT, L->probe_step};
            k_m2l_tc<<<std::min(pl->ntc, nsm), 256, m2l_tc_smem(pl->Np, pl->KC), st>>>(a);
            QBX_LAUNCH_CHECK();
        }
        k_m2l_reduce<<<nblocks(nb * D, 256), 256, 0, st>>>(nb, pl->P, PMT, L->start[LV], pl->pair_pos, pl->y, T->hw, pb,
                                                          B);
        QBX_LAUNCH_CHECK();
        return;
    }
    k_mhat<<<nblocks(nb * D, 256), 256, 0, st>>>(nb, pl->P, PMT, Mu, pl->mh);
    QBX_LAUNCH_CHECK();
    if (pl->ntiles > 0) {
        dim3 grid(pl->ntiles, (D + GM - 1) / GM);
        k_m2l_gemm_fp32<<<grid, 256, 0, st>>>(D, pl->tiles, pl->off_start, pl->pair_src, pl->mats, pl->mh, pl->y);
        QBX_LAUNCH_CHECK();
    }
    k_m2l_reduce<<<nblocks(nb * D, 256), 256, 0, st>>>(nb, pl->P, PMT, L->start[LV], pl->pair_pos, pl->y, T->hw, pb, B);
    QBX_LAUNCH_CHECK();
}

}  // namespace qbx
