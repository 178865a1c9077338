// Learned expansion orders: per-center features, order labels from sweeps of the method,
// a small MLP (4 -> 64 -> 64 -> 2, tanh, FP32) with forward, backward and Adam kernels, and
// the map from its predictions to per-center QBX orders and per-box FMM orders.
//
// Parameter vector (float, QBX_MLP_NPARAMS entries): W1[64][4], b1[64], W2[64][64], b2[64],
// W3[2][64], b3[2].  Loss: (1/(2n)) sum_i |y_i - t_i|^2.  Gradients are summed in a fixed order
// (warp butterflies, then warps, then blocks), so training is deterministic.
#include <cmath>

#include "qbx_internal.cuh"

namespace qbx {

constexpr int H1 = 64, H2 = 64, NIN = 4, NOUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + H1 * NIN, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1, OW3 = OB2 + H2,
              OB3 = OW3 + NOUT * H2, NPAR = OB3 + NOUT;
static_assert(NPAR == QBX_MLP_NPARAMS, "parameter layout");

// ---------------------------------------------------------------- features

// f0 = log2(rho / |b|), f1 = level(b) / 8, f2 = (|c - c_b| + rho) / |b| (how far the expansion ball
// reaches from the center of the box local), f3 = log10(max near-field source strength / max strength
// + 1e-12), near field = the sources of List 1 of b: b = owner box of c.
__global__ void k_features(int64_t nc, const int *ctr_perm, const int *ctr_box, const double *cxyz, const double *cr,
                           const int *level, const double *cen, const double *hw, const int *ustart,
                           const int *uidx, const int *own_start, const double *sq, const double *sd, int64_t ns,
                           const double *gmax, float *feat)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int b = ctr_box[i];
    const double x = cxyz[i], y = cxyz[nc + i], z = cxyz[2 * nc + i];
    const int out = ctr_perm[i];
    feat[4 * out + 0] = (float)log2(cr[i] / hw[b]);
    feat[4 * out + 1] = (float)(level[b] / 8.0);
    const double dx = x - cen[3 * b], dy = y - cen[3 * b + 1], dz = z - cen[3 * b + 2];
    feat[4 * out + 2] = (float)((sqrt(dx * dx + dy * dy + dz * dz) + cr[i]) / hw[b]);
    double m = 0.0;
    for (int e = ustart[b]; e < ustart[b + 1]; ++e) {
        int d = uidx[e];
        for (int s = own_start[d]; s < own_start[d + 1]; ++s) {
            double v = fabs(sq[s]);
            if (sd) v += sqrt(sd[s] * sd[s] + sd[ns + s] * sd[ns + s] + sd[2 * ns + s] * sd[2 * ns + s]);
            m = fmax(m, v);
        }
    }
    feat[4 * out + 3] = (float)log10(m / fmax(gmax[0], 1e-300) + 1e-12);
}

__global__ void k_strength_max(int64_t ns, const double *sq, const double *sd, double *gmax)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        double v = fabs(sq[s]);
        if (sd) v += sqrt(sd[s] * sd[s] + sd[ns + s] * sd[ns + s] + sd[2 * ns + s] * sd[2 * ns + s]);
        m = fmax(m, v);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // max of non-negative doubles: compare as integers (order independent)
        atomicMax(reinterpret_cast<unsigned long long *>(gmax), (unsigned long long)__double_as_longlong(red[0]));
    }
}

// ---------------------------------------------------------------- labels

// label[t] = order_of[k*] where k* = smallest k with |v_k' - v_ref| <= tol for all k' in [k, K-1]
// (v_ref = column K-1); values[k * nt + t].
__global__ void k_labels(int64_t nt, int K, const double *values, const int *order_of, double tol, int8_t *label)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double ref = values[(int64_t)(K - 1) * nt + t];
    int k = K - 1;
    while (k > 0 && fabs(values[(int64_t)(k - 1) * nt + t] - ref) <= tol) --k;
    label[t] = (int8_t)order_of[k];
}

// ---------------------------------------------------------------- MLP

__device__ __forceinline__ void mlp_forward(const float *P, const float *x, float *h1, float *h2, float *y)
{
    for (int j = 0; j < H1; ++j) {
        float a = P[OB1 + j];
        for (int k = 0; k < NIN; ++k) a = fmaf(P[OW1 + j * NIN + k], x[k], a);
        h1[j] = tanhf(a);
    }
    for (int j = 0; j < H2; ++j) {
        float a = P[OB2 + j];
        for (int k = 0; k < H1; ++k) a = fmaf(P[OW2 + j * H1 + k], h1[k], a);
        h2[j] = tanhf(a);
    }
    for (int o = 0; o < NOUT; ++o) {
        float a = P[OB3 + o];
        for (int k = 0; k < H2; ++k) a = fmaf(P[OW3 + o * H2 + k], h2[k], a);
        y[o] = a;
    }
}

__global__ void k_mlp_forward(const float *P, const float *x, int64_t n, float *y)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h1[H1], h2[H2], yy[NOUT], xx[NIN];
    for (int k = 0; k < NIN; ++k) xx[k] = x[NIN * i + k];
    mlp_forward(P, xx, h1, h2, yy);
    for (int o = 0; o < NOUT; ++o) y[NOUT * i + o] = yy[o];
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Per-block partial gradients of the loss and of the loss value (last slot).  One sample per
// thread; each parameter's contributions are summed over a warp by a butterfly and over the
// block's warps in warp order.
constexpr int GTHREADS = 64;  // 2 warps: the per-warp sums fit in static shared memory
__global__ void __launch_bounds__(GTHREADS) k_mlp_grad(const float *P, const float *x, const float *tgt, int64_t n,
                                                       float inv_n, float *part)
{
    __shared__ float wsum[GTHREADS / 32][NPAR + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t i = (int64_t)blockIdx.x * GTHREADS + threadIdx.x;
    bool valid = i < n;
    float xx[NIN] = {0, 0, 0, 0}, h1[H1], h2[H2], y[NOUT], dy[NOUT], d2[H2], d1[H1];
    if (valid)
        for (int k = 0; k < NIN; ++k) xx[k] = x[NIN * i + k];
    mlp_forward(P, xx, h1, h2, y);
    float loss = 0.f;
    for (int o = 0; o < NOUT; ++o) {
        float r = valid ? (y[o] - tgt[NOUT * i + o]) : 0.f;
        dy[o] = r * inv_n;
        loss += 0.5f * r * r * inv_n;
    }
    for (int j = 0; j < H2; ++j) {
        float g = 0.f;
        for (int o = 0; o < NOUT; ++o) g = fmaf(P[OW3 + o * H2 + j], dy[o], g);
        d2[j] = g * (1.f - h2[j] * h2[j]);
    }
    for (int k = 0; k < H1; ++k) {
        float g = 0.f;
        for (int j = 0; j < H2; ++j) g = fmaf(P[OW2 + j * H1 + k], d2[j], g);
        d1[k] = g * (1.f - h1[k] * h1[k]);
    }
    auto put = [&](int idx, float v) {
        v = warp_sum(v);
        if (lane == 0) wsum[w][idx] = v;
    };
    for (int j = 0; j < H1; ++j) {
        for (int k = 0; k < NIN; ++k) put(OW1 + j * NIN + k, d1[j] * xx[k]);
        put(OB1 + j, d1[j]);
    }
    for (int j = 0; j < H2; ++j) {
        for (int k = 0; k < H1; ++k) put(OW2 + j * H1 + k, d2[j] * h1[k]);
        put(OB2 + j, d2[j]);
    }
    for (int o = 0; o < NOUT; ++o) {
        for (int k = 0; k < H2; ++k) put(OW3 + o * H2 + k, dy[o] * h2[k]);
        put(OB3 + o, dy[o]);
    }
    put(NPAR, loss);
    __syncthreads();
    for (int idx = threadIdx.x; idx <= NPAR; idx += GTHREADS) {
        float v = 0.f;
        for (int ww = 0; ww < GTHREADS / 32; ++ww) v += wsum[ww][idx];
        part[(int64_t)blockIdx.x * (NPAR + 1) + idx] = v;
    }
}

__global__ void k_mlp_reduce(const float *part, int nblk, float *grad)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx > NPAR) return;
    float v = 0.f;
    for (int b = 0; b < nblk; ++b) v += part[(int64_t)b * (NPAR + 1) + idx];
    grad[idx] = v;
}

__global__ void k_adam(float *P, float *m, float *v, const float *grad, int step, float lr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float g = grad[i];
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v[i] = b2 * v[i] + (1.f - b2) * g * g;
    float mh = m[i] / (1.f - powf(b1, (float)step)), vh = v[i] / (1.f - powf(b2, (float)step));
    P[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Deterministic initialisation: uniform(-a, a) per layer (a = sqrt(6/(fan_in+fan_out))), from
// SplitMix64 (Steele, Lea & Flood) of (seed, index); biases zero.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void k_mlp_init(float *P, uint64_t seed)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    float a = 0.f;
    if (i < OB1) a = sqrtf(6.f / (NIN + H1));
    else if (i >= OW2 && i < OB2) a = sqrtf(6.f / (H1 + H2));
    else if (i >= OW3 && i < OB3) a = sqrtf(6.f / (H2 + NOUT));
    uint64_t r = splitmix64(seed * 0x100000001b3ULL + (uint64_t)i);
    float u = (float)((r >> 11) * (1.0 / 9007199254740992.0));  // [0, 1)
    P[i] = a * (2.f * u - 1.f);
}

// ---------------------------------------------------------------- orders

// clamp(ceil(y + margin), lo, hi) in single precision; a NaN prediction gives hi
__device__ __forceinline__ int order_from_pred(float y, float margin, int lo, int hi)
{
    if (y != y) return hi;
    const float v = ceilf(y + margin);
    if (v < (float)lo) return lo;
    if (v > (float)hi) return hi;
    return (int)v;
}

// q_out[c] (input order) = clamp(ceil(y0 + mq), qlo, qhi); per box (the order of its local
// expansion): max over the centers of its subtree of clamp(ceil(y1 + mp), plo, phi) (atomicMax up
// the parent chain from -1), p_default where nothing contributes.
__global__ void k_orders_centers(int64_t nc, const int *ctr_perm, const int *ctr_box, const int *parent, const float *y,
                                 float mq, float mp, int qlo, int qhi, int plo, int phi, int8_t *q_out, int *pbox)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int c = ctr_perm[i];
    const int q = order_from_pred(y[NOUT * c], mq, qlo, qhi), p = order_from_pred(y[NOUT * c + 1], mp, plo, phi);
    q_out[c] = (int8_t)q;
    for (int b = ctr_box[i]; b >= 0; b = parent[b]) atomicMax(&pbox[b], p);
}

// Point targets read their box's local expansion directly: their boxes and all ancestors keep the
// highest order.
__global__ void k_orders_points(int64_t nt, const int *tgt_ctr, const int *tgt_owner, const int *parent, int phi,
                                int *pbox)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt || tgt_ctr[t] >= 0) return;
    for (int b = tgt_owner[t]; b >= 0; b = parent[b]) atomicMax(&pbox[b], phi);
}

__global__ void k_orders_boxes(int64_t nb, const int *pbox, int p_default, int8_t *p_out)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int p = pbox[b];
    p_out[b] = (int8_t)(p >= 0 ? p : p_default);
}

// Judge and fallback: a target whose learned-order result misses the fixed-order judge by more than
// tol raises its center's QBX order to qfix and the local order of the box owning that center (or the
// point target) and of every box above it to pfix.  NaN differences count as misses.
__global__ void k_orders_fallback(int64_t nt, const double *res, const double *judge, const int *tgt_ctr,
                                  const int *ctr_owner, const int *tgt_owner, const int *parent, double tol, int qfix,
                                  int pfix, int8_t *q, int8_t *pb, unsigned long long *count)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    if (fabs(res[t] - judge[t]) <= tol) return;
    atomicAdd(count, 1ull);
    const int c = tgt_ctr[t];
    int b;
    if (c >= 0) {
        q[c] = (int8_t)qfix;
        b = ctr_owner[c];
    } else {
        b = tgt_owner[t];
    }
    for (; b >= 0; b = parent[b]) pb[b] = (int8_t)pfix;  // same value from every thread
}

}  // namespace qbx

using namespace qbx;

template <class F>
static int learned_guard(F &&f)
{
    try {
        set_error("");
        return f();
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected exception");
        return QBX_ERR_CUDA;
    }
}

extern "C" {

int qbx_center_features(const qbx_tree *T, const qbx_lists *L, const double *w, const double *sigma, const double *mu,
                        const double *nrm, float *feat, void *stream)
{
    return learned_guard([&]() -> int {
        if (!T || !L || L->tree != T || !feat || (T->np[KSRC] && !w) || (mu && !nrm))
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t ns = T->np[KSRC], nc = T->np[KCTR];
        double *sq = dalloc<double>(ns), *sd = dalloc<double>(3 * ns), *gmax = dalloc<double>(1);
        int *flags = dalloc<int>(1);
        try {
            QBX_CUDA_TRY(cudaMemsetAsync(gmax, 0, sizeof(double), st));
            QBX_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), st));
            if (ns) {
                prep_sources(T->perm[KSRC], ns, w, sigma, mu, nrm, sq, sd, flags, st);
                k_strength_max<<<152, 256, 0, st>>>(ns, sq, mu ? sd : nullptr, gmax);
                QBX_LAUNCH_CHECK();
            }
            if (nc)
                k_features<<<nblocks(nc, 128), 128, 0, st>>>(nc, T->perm[KCTR], T->ctr_box, T->cxyz, T->cr, T->level,
                                                             T->cen, T->hw, L->start[LU], L->idx[LU],
                                                             T->own_start[KSRC], sq, mu ? sd : nullptr, ns, gmax, feat);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
        } catch (...) {
            dfree(sq); dfree(sd); dfree(gmax); dfree(flags);
            throw;
        }
        dfree(sq); dfree(sd); dfree(gmax); dfree(flags);
        return QBX_OK;
    });
}

int qbx_order_labels(const double *values, int n_orders, const int *order_of_host, int64_t n, double tol,
                     int8_t *labels, void *stream)
{
    return learned_guard([&]() -> int {
        if (!values || !labels || !order_of_host || n_orders < 1 || n_orders > 64 || !(tol >= 0.0) || n < 0)
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        int *ord = dalloc<int>(n_orders);
        try {
            QBX_CUDA_TRY(cudaMemcpyAsync(ord, order_of_host, n_orders * sizeof(int), cudaMemcpyHostToDevice, st));
            if (n) k_labels<<<nblocks(n, 256), 256, 0, st>>>(n, n_orders, values, ord, tol, labels);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
        } catch (...) {
            dfree(ord);
            throw;
        }
        dfree(ord);
        return QBX_OK;
    });
}

int qbx_mlp_init(float *params, uint64_t seed, void *stream)
{
    return learned_guard([&]() -> int {
        if (!params) throw Error{QBX_ERR_INVALID_ARG, "params is NULL"};
        k_mlp_init<<<nblocks(NPAR, 256), 256, 0, (cudaStream_t)stream>>>(params, seed);
        QBX_LAUNCH_CHECK();
        return QBX_OK;
    });
}

int qbx_mlp_forward(const float *params, const float *x, int64_t n, float *y, void *stream)
{
    return learned_guard([&]() -> int {
        if (!params || n < 0 || (n && (!x || !y))) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        if (n) k_mlp_forward<<<nblocks(n, 128), 128, 0, (cudaStream_t)stream>>>(params, x, n, y);
        QBX_LAUNCH_CHECK();
        return QBX_OK;
    });
}

static void mlp_grad(const float *params, const float *x, const float *t, int64_t n, float *grad, cudaStream_t st)
{
    int nblk = (int)std::max<int64_t>(1, (n + GTHREADS - 1) / GTHREADS);
    float *part = dalloc<float>((int64_t)nblk * (NPAR + 1));
    try {
        k_mlp_grad<<<nblk, GTHREADS, 0, st>>>(params, x, t, n, 1.f / (float)std::max<int64_t>(n, 1), part);
        k_mlp_reduce<<<nblocks(NPAR + 1, 256), 256, 0, st>>>(part, nblk, grad);
        QBX_LAUNCH_CHECK();
        QBX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        dfree(part);
        throw;
    }
    dfree(part);
}

int qbx_mlp_loss_grad(const float *params, const float *x, const float *target, int64_t n, float *grad,
                      void *stream)
{
    return learned_guard([&]() -> int {
        if (!params || !grad || n < 1 || !x || !target) throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        mlp_grad(params, x, target, n, grad, (cudaStream_t)stream);
        return QBX_OK;
    });
}

int qbx_mlp_train(float *params, float *adam_m, float *adam_v, const float *x, const float *target, int64_t n,
                  int steps, int first_step, float lr, float *loss_host, void *stream)
{
    return learned_guard([&]() -> int {
        if (!params || !adam_m || !adam_v || !x || !target || n < 1 || steps < 0 || first_step < 1 || !(lr > 0.f))
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        float *grad = dalloc<float>(NPAR + 1);
        try {
            for (int s = 0; s < steps; ++s) {
                mlp_grad(params, x, target, n, grad, st);
                k_adam<<<nblocks(NPAR, 256), 256, 0, st>>>(params, adam_m, adam_v, grad, first_step + s, lr);
                QBX_LAUNCH_CHECK();
            }
            if (loss_host) {
                mlp_grad(params, x, target, n, grad, st);
                QBX_CUDA_TRY(cudaMemcpyAsync(loss_host, grad + NPAR, sizeof(float), cudaMemcpyDeviceToHost, st));
            }
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
        } catch (...) {
            dfree(grad);
            throw;
        }
        dfree(grad);
        return QBX_OK;
    });
}

int qbx_orders_from_mlp(const qbx_tree *T, const qbx_lists *L, const float *pred, const int32_t *tgt_ctr,
                        float margin_q, float margin_p, int q_lo, int q_hi, int p_lo, int p_hi, int p_default,
                        int8_t *p_qbx_per_ctr, int8_t *p_fmm_per_box, void *stream)
{
    return learned_guard([&]() -> int {
        if (!T || !L || L->tree != T || !pred || !p_qbx_per_ctr || !p_fmm_per_box || q_lo < 0 || q_hi > QMAX ||
            q_lo > q_hi || p_lo < 0 || p_hi > PMAX || p_lo > p_hi || p_default < 0 || p_default > PMAX)
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t nb = T->nb, nc = T->np[KCTR];
        int *pbox = dalloc<int>(nb);
        try {
            QBX_CUDA_TRY(cudaMemsetAsync(pbox, 0xff, nb * sizeof(int), st));  // -1: no contribution yet
            if (nc)
                k_orders_centers<<<nblocks(nc, 256), 256, 0, st>>>(nc, T->perm[KCTR], T->ctr_box, T->parent, pred,
                                                                   margin_q, margin_p, q_lo, q_hi, p_lo, p_hi,
                                                                   p_qbx_per_ctr, pbox);
            if (tgt_ctr && T->np[KTGT])
                k_orders_points<<<nblocks(T->np[KTGT], 256), 256, 0, st>>>(T->np[KTGT], tgt_ctr, T->owner[KTGT],
                                                                           T->parent, p_hi, pbox);
            k_orders_boxes<<<nblocks(nb, 256), 256, 0, st>>>(nb, pbox, p_default, p_fmm_per_box);
            QBX_LAUNCH_CHECK();
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
        } catch (...) {
            dfree(pbox);
            throw;
        }
        dfree(pbox);
        return QBX_OK;
    });
}

int qbx_orders_fallback(const qbx_tree *T, const double *result, const double *judge, const int32_t *tgt_ctr,
                        double tol, int q_fix, int p_fix, int8_t *p_qbx_per_ctr, int8_t *p_fmm_per_box,
                        int64_t *n_raised, void *stream)
{
    return learned_guard([&]() -> int {
        if (!T || !result || !judge || !tgt_ctr || !p_qbx_per_ctr || !p_fmm_per_box || !n_raised || !(tol >= 0.0) ||
            q_fix < 0 || q_fix > QMAX || p_fix < 0 || p_fix > PMAX)
            throw Error{QBX_ERR_INVALID_ARG, "bad argument"};
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t nt = T->np[KTGT];
        unsigned long long *cnt = dalloc<unsigned long long>(1);
        try {
            QBX_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
            if (nt)
                k_orders_fallback<<<nblocks(nt, 256), 256, 0, st>>>(nt, result, judge, tgt_ctr, T->owner[KCTR],
                                                                    T->owner[KTGT], T->parent, tol, q_fix, p_fix,
                                                                    p_qbx_per_ctr, p_fmm_per_box, cnt);
            QBX_LAUNCH_CHECK();
            unsigned long long h = 0;
            QBX_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
            QBX_CUDA_TRY(cudaStreamSynchronize(st));
            *n_raised = (int64_t)h;
        } catch (...) {
            dfree(cnt);
            throw;
        }
        dfree(cnt);
        return QBX_OK;
    });
}

}  // extern "C"
