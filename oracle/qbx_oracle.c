/*
 * Oracle for the GIGAQBX 3D Laplace evaluation (Wala & Kloeckner, "A Fast
 * Algorithm for Quadrature by Expansion in Three Dimensions").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, serial, FP64 C written for readability.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code with the CUDA library.
 *
 * Notation follows the paper:
 *   - Green's function G(x,y) = 1 / (4 pi |x - y|)                 (eq. laplace-fs-green)
 *   - Y_n^m(theta, phi) = sqrt((2n+1)/(4pi) (n-|m|)!/(n+|m|)!)
 *                         P_n^|m|(cos theta) e^{i m phi}             (eq. spherical-harmonics)
 *     with P_n^m the associated Legendre function WITHOUT the
 *     Condon-Shortley phase (the paper does not state one; G does not
 *     depend on it).
 *   - local coefficients  L_n^m = q/(2n+1) |s-c|^{-n-1} Y_n^{-m}(s-c)  (eq. local-expansion-coeff)
 *     evaluated as        sum L_n^m |t-c|^n Y_n^m(t-c)
 *   - multipole coeffs.   M_n^m = q/(2n+1) |s-c|^n Y_n^m(s-c)          (eq. mpole-expansion-coeff)
 *     evaluated as        sum M_n^m |t-c|^{-n-1} Y_n^{-m}(t-c)
 *   - coefficients of an order-p expansion are stored as (p+1)^2 complex
 *     numbers B_0^0, B_1^-1, B_1^0, B_1^1, ... (Section 4.1).
 *   - the double layer D u(x) = int d/dn(y) G(x,y) u(y) dS(y) (the kernel of
 *     Green's formula in Section 6.1): every source-side operation has a
 *     dipole form, the directional derivative n(y) . grad_y of the charge form.
 *
 * The translation operators (M2M, L2L, M2L, Section 4.1) are not printed in
 * the paper; they are written here as plain double sums obtained by
 * re-expanding solid harmonics with the addition theorems of the regular
 * solid harmonics |x|^n Y_n^m and the irregular ones |x|^{-n-1} Y_n^m, in the
 * paper's normalisation.
 *
 * Tree, interaction lists and the nine stages follow Section 5.2 and
 * Algorithm 4; readings of passages the paper leaves open are noted where
 * they are used.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_NMAX 96 /* highest harmonic degree supported by the factor tables */
#define ORC_PI 3.14159265358979323846

static double g_fact[2 * ORC_NMAX + 4];
static int g_init = 0;

static double g_afac[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
static double g_bfac[(ORC_NMAX + 1) * (ORC_NMAX + 1)];

static inline int IDX(int n, int m) { return n * n + n + m; }

static double Afac_eval(int n, int m);
static double Bfac_eval(int n, int m);

static void init_tables(void)
{
    if (g_init) return;
    g_fact[0] = 1.0;
    for (int i = 1; i < 2 * ORC_NMAX + 4; ++i) g_fact[i] = g_fact[i - 1] * (double)i;
    for (int n = 0; n <= ORC_NMAX; ++n)
        for (int m = -n; m <= n; ++m) {
            g_afac[IDX(n, m)] = Afac_eval(n, m);
            g_bfac[IDX(n, m)] = Bfac_eval(n, m);
        }
    g_init = 1;
}

/* ------------------------------------------------------------------------ */
/* spherical harmonics (eq. spherical-harmonics)                              */
/* ------------------------------------------------------------------------ */

/* Normalised Legendre functions Pbar_n^m(x) = sqrt((2n+1)/(4pi)(n-m)!/(n+m)!) P_n^m(x),
 * 0 <= m <= n <= p, stored at IDX(n, m), by the standard three-term
 * recurrences for normalised functions (no Condon-Shortley phase). */
static void legendre_norm(int p, double ct, double st, double *Pb)
{
    Pb[IDX(0, 0)] = 1.0 / sqrt(4.0 * ORC_PI);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) Pb[IDX(m, m)] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * Pb[IDX(m - 1, m - 1)];
        if (m + 1 <= p) Pb[IDX(m + 1, m)] = sqrt(2.0 * m + 3.0) * ct * Pb[IDX(m, m)];
        for (int n = m + 2; n <= p; ++n) {
            double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = sqrt((((double)(n - 1) * (n - 1)) - (double)m * m) / (4.0 * (n - 1) * (n - 1) - 1.0));
            Pb[IDX(n, m)] = a * (ct * Pb[IDX(n - 1, m)] - b * Pb[IDX(n - 2, m)]);
        }
    }
}

/* Y_n^m at the direction of v for all n <= p, |m| <= n.  theta = acos(z/r) and
 * phi = atan2(y, x) (Section 2.1); cos(theta) = z/r and sin(theta) = rho/r are
 * used directly.  Returns r = |v|; Y is left untouched when r == 0. */
static double ylm_dir(int p, const double v[3], cplx *Y)
{
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (r == 0.0) return 0.0;
    double rho = sqrt(v[0] * v[0] + v[1] * v[1]);
    double ct = v[2] / r, st = rho / r;
    double phi = atan2(v[1], v[0]);
    double Pb[(p + 1) * (p + 1)];
    legendre_norm(p, ct, st, Pb);
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx e = cexp(I * (double)m * phi);
            Y[IDX(n, m)] = Pb[IDX(n, m)] * e;
            if (m > 0) Y[IDX(n, -m)] = Pb[IDX(n, m)] * conj(e);
        }
    return r;
}

/* regular solid harmonics |v|^n Y_n^m(v), n <= p */
static void solid_reg(int p, const double v[3], cplx *out)
{
    double r = ylm_dir(p, v, out);
    if (r == 0.0) {
        for (int i = 0; i < (p + 1) * (p + 1); ++i) out[i] = 0.0;
        out[0] = 1.0 / sqrt(4.0 * ORC_PI);
        return;
    }
    double rn = 1.0;
    for (int n = 0; n <= p; ++n) {
        for (int m = -n; m <= n; ++m) out[IDX(n, m)] *= rn;
        rn *= r;
    }
}

/* irregular solid harmonics |v|^{-n-1} Y_n^m(v), n <= p, v != 0 */
static void solid_irr(int p, const double v[3], cplx *out)
{
    double r = ylm_dir(p, v, out);
    double rn = 1.0 / r;
    for (int n = 0; n <= p; ++n) {
        for (int m = -n; m <= n; ++m) out[IDX(n, m)] *= rn;
        rn /= r;
    }
}

/* Conversion factors between |x|^n Y_n^m and the polynomial harmonics used to
 * write the addition theorems:
 *   |x|^n Y_n^m          = Afac(n,m) * R_n^m(x),
 *   |x|^{-n-1} Y_n^m     = Bfac(n,m) * S_n^m(x),
 * where R_n^m(a+b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b) and
 *       conj S_n^m(X+y) = sum_{k,l} (-1)^k R_k^l(y) conj S_{n+k}^{m+l}(X), |y| < |X|. */
static double Afac_eval(int n, int m)
{
    int am = m < 0 ? -m : m;
    double s = (m < 0 && (am & 1)) ? -1.0 : 1.0;
    return s * sqrt((2.0 * n + 1.0) / (4.0 * ORC_PI)) * sqrt(g_fact[n + am] * g_fact[n - am]);
}

static double Bfac_eval(int n, int m)
{
    int am = m < 0 ? -m : m;
    double s = (m < 0 && (am & 1)) ? -1.0 : 1.0;
    return s * sqrt((2.0 * n + 1.0) / (4.0 * ORC_PI)) / sqrt(g_fact[n + am] * g_fact[n - am]);
}

static inline double Afac(int n, int m) { return g_afac[IDX(n, m)]; }
static inline double Bfac(int n, int m) { return g_bfac[IDX(n, m)]; }

/* ------------------------------------------------------------------------ */
/* source <-> expansion operators                                             */
/* ------------------------------------------------------------------------ */

/* Directional derivative d . grad of the regular solid harmonic |x|^n Y_n^m at x,
 * given the table Rg of |x|^k Y_k^l for k <= n - 1, via the ladder relations
 *   (dx - i dy) R_n^m = R_{n-1}^{m-1},  (dx + i dy) R_n^m = -R_{n-1}^{m+1},  dz R_n^m = R_{n-1}^m. */
static cplx dreg(int n, int m, const cplx *Rg, const double d[3])
{
    if (n == 0) return 0.0;
    cplx dw = d[0] + I * d[1], dwb = d[0] - I * d[1];
    cplx acc = 0.0;
    double A = Afac(n, m);
    if (m + 1 <= n - 1) acc += -(dwb / 2.0) * (A / Afac(n - 1, m + 1)) * Rg[IDX(n - 1, m + 1)];
    if (m - 1 >= -(n - 1)) acc += (dw / 2.0) * (A / Afac(n - 1, m - 1)) * Rg[IDX(n - 1, m - 1)];
    if (m <= n - 1 && m >= -(n - 1)) acc += d[2] * (A / Afac(n - 1, m)) * Rg[IDX(n - 1, m)];
    return acc;
}

/* Directional derivative d . grad of |x|^{-n-1} Y_n^m at x, given the table Ir of
 * |x|^{-k-1} Y_k^l for k <= n + 1, via
 *   dz S_n^m = -S_{n+1}^m,  (dx + i dy) S_n^m = -S_{n+1}^{m+1},  (dx - i dy) S_n^m = S_{n+1}^{m-1}. */
static cplx dirr(int n, int m, const cplx *Ir, const double d[3])
{
    cplx dw = d[0] + I * d[1], dwb = d[0] - I * d[1];
    double B = Bfac(n, m);
    cplx acc = 0.0;
    acc += -(dwb / 2.0) * (B / Bfac(n + 1, m + 1)) * Ir[IDX(n + 1, m + 1)];
    acc += (dw / 2.0) * (B / Bfac(n + 1, m - 1)) * Ir[IDX(n + 1, m - 1)];
    acc += -d[2] * (B / Bfac(n + 1, m)) * Ir[IDX(n + 1, m)];
    return acc;
}

/* P2M: M_n^m += q/(2n+1) |s-c|^n Y_n^m(s-c) + dipole d . grad_s of the same. */
static void p2m(int p, const double c[3], const double s[3], double q, const double *d, cplx *M)
{
    cplx Rg[(p + 1) * (p + 1)];
    double v[3] = {s[0] - c[0], s[1] - c[1], s[2] - c[2]};
    solid_reg(p, v, Rg);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx val = q * Rg[IDX(n, m)];
            if (d) val += dreg(n, m, Rg, d);
            M[IDX(n, m)] += val / (2.0 * n + 1.0);
        }
}

/* P2L (also P2QBXL): L_n^m += q/(2n+1) |s-c|^{-n-1} Y_n^{-m}(s-c) + dipole form. */
static void p2l(int p, const double c[3], const double s[3], double q, const double *d, cplx *L)
{
    cplx Ir[(p + 2) * (p + 2)];
    double v[3] = {s[0] - c[0], s[1] - c[1], s[2] - c[2]};
    solid_irr(p + 1, v, Ir);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx val = q * Ir[IDX(n, -m)];
            if (d) val += dirr(n, -m, Ir, d);
            L[IDX(n, m)] += val / (2.0 * n + 1.0);
        }
}

/* M2P: sum M_n^m |t-c|^{-n-1} Y_n^{-m}(t-c) (real part). */
static double m2p(int p, const double c[3], const cplx *M, const double t[3])
{
    cplx Ir[(p + 1) * (p + 1)];
    double v[3] = {t[0] - c[0], t[1] - c[1], t[2] - c[2]};
    solid_irr(p, v, Ir);
    cplx acc = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) acc += M[IDX(n, m)] * Ir[IDX(n, -m)];
    return creal(acc);
}

/* L2P (also QBXL2P, eq. qbxlocal): sum L_n^m |t-c|^n Y_n^m(t-c) (real part). */
static double l2p(int p, const double c[3], const cplx *L, const double t[3])
{
    cplx Rg[(p + 1) * (p + 1)];
    double v[3] = {t[0] - c[0], t[1] - c[1], t[2] - c[2]};
    solid_reg(p, v, Rg);
    cplx acc = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) acc += L[IDX(n, m)] * Rg[IDX(n, m)];
    return creal(acc);
}

/* P2P: point potential at t of a charge q and dipole d at s; coincident pairs skipped. */
static double p2p(const double s[3], double q, const double *d, const double t[3])
{
    double v[3] = {t[0] - s[0], t[1] - s[1], t[2] - s[2]};
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (r == 0.0) return 0.0;
    double val = q / (4.0 * ORC_PI * r);
    if (d) val += (d[0] * v[0] + d[1] * v[1] + d[2] * v[2]) / (4.0 * ORC_PI * r * r * r);
    return val;
}

/* ------------------------------------------------------------------------ */
/* translation operators (Section 4.1), orders p_src -> p_dst                 */
/* ------------------------------------------------------------------------ */

/* M2M c -> c2: M2_n^m += 1/(2n+1) sum_{k,l} (2k+1) M_k^l |c-c2|^{n-k} Y_{n-k}^{m-l}(c-c2)
 *                                   * A(n,m) / (A(k,l) A(n-k,m-l)). */
static void m2m(int ps, const double c[3], const cplx *M, int pd, const double c2[3], cplx *M2)
{
    cplx Rg[(pd + 1) * (pd + 1)];
    double v[3] = {c[0] - c2[0], c[1] - c2[1], c[2] - c2[2]};
    solid_reg(pd, v, Rg);
    for (int n = 0; n <= pd; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0.0;
            for (int k = 0; k <= n && k <= ps; ++k)
                for (int l = -k; l <= k; ++l) {
                    int j = n - k, i = m - l;
                    if (i < -j || i > j) continue;
                    acc += (2.0 * k + 1.0) * M[IDX(k, l)] * Rg[IDX(j, i)] * (Afac(n, m) / (Afac(k, l) * Afac(j, i)));
                }
            M2[IDX(n, m)] += acc / (2.0 * n + 1.0);
        }
}

/* L2L c -> c2: L2_k^l += sum_{n>=k,m} L_n^m |c2-c|^{n-k} Y_{n-k}^{m-l}(c2-c) A(n,m)/(A(k,l)A(n-k,m-l)). */
static void l2l(int ps, const double c[3], const cplx *L, int pd, const double c2[3], cplx *L2)
{
    cplx Rg[(ps + 1) * (ps + 1)];
    double v[3] = {c2[0] - c[0], c2[1] - c[1], c2[2] - c[2]};
    solid_reg(ps, v, Rg);
    for (int k = 0; k <= pd; ++k)
        for (int l = -k; l <= k; ++l) {
            cplx acc = 0.0;
            for (int n = k; n <= ps; ++n)
                for (int m = -n; m <= n; ++m) {
                    int j = n - k, i = m - l;
                    if (i < -j || i > j) continue;
                    acc += L[IDX(n, m)] * Rg[IDX(j, i)] * (Afac(n, m) / (Afac(k, l) * Afac(j, i)));
                }
            L2[IDX(k, l)] += acc;
        }
}

/* M2L cM -> cL: L_k^l += sum_{n,m} M_n^m (-1)^{k+l} B(n,-m) |X|^{-(n+k)-1} Y_{n+k}^{-(m+l)}(X)
 *                                   / (A(k,l) B(n+k, -(m+l))),   X = cL - cM. */
static void m2l(int ps, const double cM[3], const cplx *M, int pd, const double cL[3], cplx *L)
{
    int pt = ps + pd;
    cplx Ir[(pt + 1) * (pt + 1)];
    double X[3] = {cL[0] - cM[0], cL[1] - cM[1], cL[2] - cM[2]};
    solid_irr(pt, X, Ir);
    for (int k = 0; k <= pd; ++k)
        for (int l = -k; l <= k; ++l) {
            cplx acc = 0.0;
            double sgn = ((k + l) & 1) ? -1.0 : 1.0;
            for (int n = 0; n <= ps; ++n)
                for (int m = -n; m <= n; ++m) {
                    int j = n + k, i = -(m + l);
                    acc += M[IDX(n, m)] * Ir[IDX(j, i)] * (Bfac(n, -m) / (Afac(k, l) * Bfac(j, i)));
                }
            L[IDX(k, l)] += sgn * acc;
        }
}

/* ------------------------------------------------------------------------ */
/* exported single-operator entry points (used by the pin tests)              */
/* ------------------------------------------------------------------------ */

/* Y_n^m for direction v, n <= p; out is (p+1)^2 complex as interleaved re/im. */
int orc_ylm(int p, const double *v, double *out)
{
    init_tables();
    if (p < 0 || p > ORC_NMAX) return -1;
    if (ylm_dir(p, v, (cplx *)out) == 0.0) return -1;
    return 0;
}

int orc_p2m(int p, const double *c, const double *s, double q, const double *d, double *M)
{
    init_tables();
    p2m(p, c, s, q, d, (cplx *)M);
    return 0;
}

int orc_p2l(int p, const double *c, const double *s, double q, const double *d, double *L)
{
    init_tables();
    p2l(p, c, s, q, d, (cplx *)L);
    return 0;
}

double orc_m2p(int p, const double *c, const double *M, const double *t)
{
    init_tables();
    return m2p(p, c, (const cplx *)M, t);
}

double orc_l2p(int p, const double *c, const double *L, const double *t)
{
    init_tables();
    return l2p(p, c, (const cplx *)L, t);
}

double orc_p2p(const double *s, double q, const double *d, const double *t) { return p2p(s, q, d, t); }

int orc_m2m(int ps, const double *c, const double *M, int pd, const double *c2, double *M2)
{
    init_tables();
    m2m(ps, c, (const cplx *)M, pd, c2, (cplx *)M2);
    return 0;
}

int orc_l2l(int ps, const double *c, const double *L, int pd, const double *c2, double *L2)
{
    init_tables();
    l2l(ps, c, (const cplx *)L, pd, c2, (cplx *)L2);
    return 0;
}

int orc_m2l(int ps, const double *cM, const double *M, int pd, const double *cL, double *L)
{
    init_tables();
    m2l(ps, cM, (const cplx *)M, pd, cL, (cplx *)L);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* octree with target confinement (Section 5.2, Algorithm 4 Stage 1)          */
/* ------------------------------------------------------------------------ */

enum { KSRC = 0, KCTR = 1, KTGT = 2 };

typedef struct {
    int nb, cap, nlev;
    int *level;
    int64_t *ic;  /* 3 per box: integer coordinates at the box's level */
    double *cen;  /* 3 per box */
    double *hw;   /* |b|, the l-infinity radius */
    int *parent;
    int *child;   /* 8 per box, -1 = none */
    int *level_start; /* nlev + 1 */
    int np[3];
    int *owner[3];
    int *own_start[3]; /* nb + 1 (CSR over boxes) */
    int *own_idx[3];   /* particle indices grouped by box, ascending within a box */
    int *nsrc_sub;     /* sources in the subtree */
    int *ntgt_sub;     /* centers + targets in the subtree */
    int n_overfull;    /* leaves left above n_max because max_depth was reached */
    double root_c[3], root_h;
    double tf;
    int linf;          /* 1: the l-infinity TCR of the two-dimensional method (Table l2-comparison) */
} otree;

/* tree variants (orc_build_tree's flags) */
#define ORC_TREE_LINF_TCR 1
#define ORC_TREE_LEVEL_RESTRICT 2

static void tree_grow(otree *T)
{
    if (T->nb < T->cap) return;
    T->cap = T->cap ? 2 * T->cap : 1024;
    T->level = realloc(T->level, sizeof(int) * T->cap);
    T->ic = realloc(T->ic, sizeof(int64_t) * 3 * T->cap);
    T->cen = realloc(T->cen, sizeof(double) * 3 * T->cap);
    T->hw = realloc(T->hw, sizeof(double) * T->cap);
    T->parent = realloc(T->parent, sizeof(int) * T->cap);
    T->child = realloc(T->child, sizeof(int) * 8 * T->cap);
}

static int tree_add(otree *T, int lev, const int64_t ic[3], const double c[3], double h, int parent)
{
    tree_grow(T);
    int b = T->nb++;
    T->level[b] = lev;
    for (int d = 0; d < 3; ++d) {
        T->ic[3 * b + d] = ic[d];
        T->cen[3 * b + d] = c[d];
    }
    T->hw[b] = h;
    T->parent[b] = parent;
    for (int o = 0; o < 8; ++o) T->child[8 * b + o] = -1;
    return b;
}

/* Center fits inside the target confinement region B2(sqrt(3)|b|(1+t_f), c_b) of a box
 * with center cc and l-infinity radius h (Section 5.2.2): |x - cc|_2 + r <= sqrt(3) h (1 + t_f).
 * With linf set, the TCR is the cube of l-infinity radius h (1 + t_f) about cc (the box-shaped
 * region of the two-dimensional method that Section 5 compares against):
 * |x - cc|_inf + r <= h (1 + t_f). */
static int fits_tcr(const double x[3], double r, const double cc[3], double h, double tf, int linf)
{
    double dx = x[0] - cc[0], dy = x[1] - cc[1], dz = x[2] - cc[2];
    if (linf) {
        double m = fmax(fmax(fabs(dx), fabs(dy)), fabs(dz));
        return m + r <= h * (1.0 + tf);
    }
    double dist = sqrt(dx * dx + dy * dy + dz * dz);
    return dist + r <= (sqrt(3.0) * h) * (1.0 + tf);
}

/* Octant of a point relative to a box center: bit d set iff x_d >= c_d (x = bit 0, y = 1, z = 2). */
static int octant(const double x[3], const double c[3])
{
    return (x[0] >= c[0] ? 1 : 0) | (x[1] >= c[1] ? 2 : 0) | (x[2] >= c[2] ? 4 : 0);
}

static void get_pt(const double *xyz, int n, int i, double out[3])
{
    out[0] = xyz[i];
    out[1] = xyz[n + i];
    out[2] = xyz[2 * n + i];
}

static int is_leaf(const otree *T, int b);
static int adjacent(const otree *T, int a, int b, int Lf);
static int morton_less(const int64_t *a, const int64_t *b);

/* Subdivides leaf b by the Stage 1 rule for which particles move (points to the octant
 * "coordinate >= center", a center only into a child whose TCR holds its ball); only
 * children that receive a particle are made, appended after the existing boxes.
 * Returns the number of children made (0: no particle can move, b stays a leaf). */
static int split_leaf(otree *T, int b, const double *xyz_k[3], const double *cr)
{
    int cmask = 0;
    double hc = 0.5 * T->hw[b], x[3], cc[3];
    int *dest[3];
    for (int k = 0; k < 3; ++k) {
        dest[k] = malloc(sizeof(int) * (T->np[k] > 0 ? T->np[k] : 1));
        for (int i = 0; i < T->np[k]; ++i) {
            dest[k][i] = -1;
            if (T->owner[k][i] != b) continue;
            get_pt(xyz_k[k], T->np[k], i, x);
            int oc = octant(x, &T->cen[3 * b]);
            if (k == KCTR) {
                for (int d = 0; d < 3; ++d) cc[d] = T->cen[3 * b + d] + (((oc >> d) & 1) ? hc : -hc);
                if (!fits_tcr(x, cr[i], cc, hc, T->tf, T->linf)) continue;
            }
            dest[k][i] = oc;
            cmask |= 1 << oc;
        }
    }
    int made = 0;
    for (int oc = 0; oc < 8; ++oc) {
        if (!((cmask >> oc) & 1)) continue;
        int64_t ic[3];
        for (int d = 0; d < 3; ++d) {
            int bit = (oc >> d) & 1;
            ic[d] = 2 * T->ic[3 * b + d] + bit;
            cc[d] = T->cen[3 * b + d] + (bit ? hc : -hc);
        }
        int c = tree_add(T, T->level[b] + 1, ic, cc, hc, b);
        T->child[8 * b + oc] = c;
        ++made;
    }
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < T->np[k]; ++i)
            if (dest[k][i] >= 0) T->owner[k][i] = T->child[8 * b + dest[k][i]];
        free(dest[k]);
    }
    return made;
}

static const otree *g_order_tree;

static int box_order_cmp(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    const otree *T = g_order_tree;
    if (T->level[a] != T->level[b]) return T->level[a] < T->level[b] ? -1 : 1;
    if (morton_less(&T->ic[3 * a], &T->ic[3 * b])) return -1;
    if (morton_less(&T->ic[3 * b], &T->ic[3 * a])) return 1;
    return 0;
}

/* Renumbers the boxes into (level, Morton code) order and rebuilds level_start. */
static void tree_renumber(otree *T)
{
    int nb = T->nb;
    int *ord = malloc(sizeof(int) * nb), *nid = malloc(sizeof(int) * nb);
    for (int i = 0; i < nb; ++i) ord[i] = i;
    g_order_tree = T;
    qsort(ord, nb, sizeof(int), box_order_cmp);
    for (int i = 0; i < nb; ++i) nid[ord[i]] = i;
    int *level = malloc(sizeof(int) * T->cap), *parent = malloc(sizeof(int) * T->cap);
    int *child = malloc(sizeof(int) * 8 * T->cap);
    int64_t *ic = malloc(sizeof(int64_t) * 3 * T->cap);
    double *cen = malloc(sizeof(double) * 3 * T->cap), *hw = malloc(sizeof(double) * T->cap);
    for (int j = 0; j < nb; ++j) {
        int i = ord[j];
        level[j] = T->level[i];
        hw[j] = T->hw[i];
        parent[j] = T->parent[i] >= 0 ? nid[T->parent[i]] : -1;
        for (int d = 0; d < 3; ++d) {
            ic[3 * j + d] = T->ic[3 * i + d];
            cen[3 * j + d] = T->cen[3 * i + d];
        }
        for (int o = 0; o < 8; ++o) child[8 * j + o] = T->child[8 * i + o] >= 0 ? nid[T->child[8 * i + o]] : -1;
    }
    free(T->level); free(T->parent); free(T->child); free(T->ic); free(T->cen); free(T->hw);
    T->level = level; T->parent = parent; T->child = child; T->ic = ic; T->cen = cen; T->hw = hw;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < T->np[k]; ++i) T->owner[k][i] = nid[T->owner[k][i]];
    T->nlev = level[nb - 1] + 1;
    free(T->level_start);
    T->level_start = malloc(sizeof(int) * (T->nlev + 1));
    for (int l = 0, j = 0; l <= T->nlev; ++l) {
        while (j < nb && level[j] < l) ++j;
        T->level_start[l] = j;
    }
    free(ord);
    free(nid);
}

/*
 * Level restriction (Remark "Effect of level-restriction on List 3 complexity", Section 5.3):
 * adjacent leaves may differ by at most one level; a tree is made so by repeatedly
 * subdividing the larger leaf of a pair that violates this.  Taken here in rounds: a round
 * finds, on the current tree, every leaf that has an adjacent leaf two or more levels finer
 * (literally, over all pairs of leaves) and subdivides all of them (split_leaf); rounds repeat
 * until one subdivides nothing.  A violating leaf none of whose particles can move stays a leaf.
 */
static void level_restrict(otree *T, const double *xyz_k[3], const double *cr, int max_depth)
{
    for (;;) {
        int nb = T->nb, Lf = 0;
        for (int b = 0; b < nb; ++b)
            if (T->level[b] > Lf) Lf = T->level[b];
        char *leaf = malloc(nb), *viol = calloc(nb, 1);
        for (int b = 0; b < nb; ++b) leaf[b] = (char)is_leaf(T, b);
        for (int b = 0; b < nb; ++b) {
            if (!leaf[b]) continue;
            for (int a = 0; a < nb && !viol[b]; ++a)
                if (leaf[a] && T->level[a] >= T->level[b] + 2 && adjacent(T, a, b, Lf)) viol[b] = 1;
        }
        int made = 0;
        for (int b = 0; b < nb; ++b)
            if (viol[b] && T->level[b] < max_depth) made += split_leaf(T, b, xyz_k, cr);
        free(leaf);
        free(viol);
        if (!made) break;
        tree_renumber(T);
    }
}

/*
 * Builds the tree.  Readings of Stage 1:
 *  - root: centered at the midpoint of the bounding box of all points and balls,
 *    rounded to a multiple of R/8, with R the smallest power of two >= 1.25 x the
 *    largest half extent, so every box center is an exact dyadic number;
 *  - a box splits when it owns more than n_max particles (sources + centers +
 *    targets) and at least one particle would move to a child; points go to the
 *    octant with "coordinate >= center" meaning the upper half; a center moves only
 *    if its ball fits the child's TCR; only children receiving a particle are made;
 *  - no box below level max_depth is made;
 *  - boxes are numbered level by level, children in octant order, which is the
 *    (level, Morton code) order.
 * flags: ORC_TREE_LINF_TCR selects the l-infinity TCR (fits_tcr, sep_a_tcrb);
 * ORC_TREE_LEVEL_RESTRICT makes the finished tree level-restricted (level_restrict).
 */
otree *orc_build_tree(const double *sxyz, int ns, const double *cxyz, const double *cr, int nc,
                      const double *txyz, int nt, int nmax, double tf, int max_depth, int flags)
{
    init_tables();
    otree *T = calloc(1, sizeof(otree));
    T->linf = (flags & ORC_TREE_LINF_TCR) ? 1 : 0;
    T->np[KSRC] = ns;
    T->np[KCTR] = nc;
    T->np[KTGT] = nt;
    T->tf = tf;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double x[3];
    for (int i = 0; i < ns; ++i) {
        get_pt(sxyz, ns, i, x);
        for (int d = 0; d < 3; ++d) { lo[d] = fmin(lo[d], x[d]); hi[d] = fmax(hi[d], x[d]); }
    }
    for (int i = 0; i < nt; ++i) {
        get_pt(txyz, nt, i, x);
        for (int d = 0; d < 3; ++d) { lo[d] = fmin(lo[d], x[d]); hi[d] = fmax(hi[d], x[d]); }
    }
    for (int i = 0; i < nc; ++i) {
        get_pt(cxyz, nc, i, x);
        for (int d = 0; d < 3; ++d) { lo[d] = fmin(lo[d], x[d] - cr[i]); hi[d] = fmax(hi[d], x[d] + cr[i]); }
    }
    double mid[3], h = 0.0;
    for (int d = 0; d < 3; ++d) {
        mid[d] = 0.5 * (lo[d] + hi[d]);
        h = fmax(h, 0.5 * (hi[d] - lo[d]));
    }
    double R = 1.0;
    if (h > 0.0 && h < 1e300) {
        while (R < 1.25 * h) R *= 2.0;
        while (0.5 * R >= 1.25 * h) R *= 0.5;
    }
    double q8 = R / 8.0, c0[3];
    for (int d = 0; d < 3; ++d) c0[d] = nearbyint(mid[d] / q8) * q8;
    T->root_h = R;
    for (int d = 0; d < 3; ++d) T->root_c[d] = c0[d];
    int64_t ic0[3] = {0, 0, 0};
    tree_add(T, 0, ic0, c0, R, -1);

    int ntot = ns + nc + nt;
    for (int k = 0; k < 3; ++k) T->owner[k] = calloc(T->np[k] > 0 ? T->np[k] : 1, sizeof(int));
    const double *xyz_k[3] = {sxyz, cxyz, txyz};
    int *lev_start = malloc(sizeof(int) * (max_depth + 3));
    lev_start[0] = 0;
    int nlev = 0;
    int *dest = malloc(sizeof(int) * (ntot > 0 ? ntot : 1));
    for (int lev = 0;; ++lev) {
        int b0 = (lev == 0) ? 0 : lev_start[lev], b1 = T->nb;
        if (b0 == b1) break;
        nlev = lev + 1;
        lev_start[lev + 1] = b1;
        int nbl = b1 - b0;
        int *cnt = calloc(nbl, sizeof(int));
        int *movers = calloc(nbl, sizeof(int));
        int *cmask = calloc(nbl, sizeof(int));
        for (int k = 0, g = 0; k < 3; ++k)
            for (int i = 0; i < T->np[k]; ++i, ++g) {
                int o = T->owner[k][i];
                if (o >= b0 && o < b1) cnt[o - b0]++;
            }
        for (int k = 0, g = 0; k < 3; ++k)
            for (int i = 0; i < T->np[k]; ++i, ++g) {
                dest[g] = -1;
                int o = T->owner[k][i];
                if (o < b0 || o >= b1) continue;
                if (cnt[o - b0] <= nmax || lev >= max_depth) continue;
                get_pt(xyz_k[k], T->np[k], i, x);
                int oc = octant(x, &T->cen[3 * o]);
                if (k == KCTR) {
                    double hc = 0.5 * T->hw[o], cc[3];
                    for (int d = 0; d < 3; ++d) cc[d] = T->cen[3 * o + d] + (((oc >> d) & 1) ? hc : -hc);
                    if (!fits_tcr(x, cr[i], cc, hc, tf, T->linf)) continue;
                }
                dest[g] = oc;
                movers[o - b0]++;
                cmask[o - b0] |= 1 << oc;
            }
        for (int bb = 0; bb < nbl; ++bb) {
            int b = b0 + bb;
            if (cnt[bb] > nmax && lev >= max_depth) T->n_overfull++;
            if (movers[bb] == 0) continue;
            double hc = 0.5 * T->hw[b];
            for (int oc = 0; oc < 8; ++oc) {
                if (!((cmask[bb] >> oc) & 1)) continue;
                int64_t ic[3];
                double cc[3];
                for (int d = 0; d < 3; ++d) {
                    int bit = (oc >> d) & 1;
                    ic[d] = 2 * T->ic[3 * b + d] + bit;
                    cc[d] = T->cen[3 * b + d] + (bit ? hc : -hc);
                }
                int nbx = tree_add(T, lev + 1, ic, cc, hc, b);
                T->child[8 * b + oc] = nbx;
            }
        }
        for (int k = 0, g = 0; k < 3; ++k)
            for (int i = 0; i < T->np[k]; ++i, ++g)
                if (dest[g] >= 0) T->owner[k][i] = T->child[8 * T->owner[k][i] + dest[g]];
        free(cnt);
        free(movers);
        free(cmask);
        if (lev + 1 > max_depth + 1) break;
    }
    free(dest);
    T->nlev = nlev;
    T->level_start = malloc(sizeof(int) * (nlev + 1));
    for (int l = 0; l < nlev; ++l) T->level_start[l] = lev_start[l];
    T->level_start[nlev] = T->nb;
    free(lev_start);
    if (flags & ORC_TREE_LEVEL_RESTRICT) level_restrict(T, xyz_k, cr, max_depth);

    /* owned particles grouped by box (counting sort, stable in the particle index) */
    for (int k = 0; k < 3; ++k) {
        T->own_start[k] = calloc(T->nb + 1, sizeof(int));
        T->own_idx[k] = malloc(sizeof(int) * (T->np[k] > 0 ? T->np[k] : 1));
        for (int i = 0; i < T->np[k]; ++i) T->own_start[k][T->owner[k][i] + 1]++;
        for (int b = 0; b < T->nb; ++b) T->own_start[k][b + 1] += T->own_start[k][b];
        int *fill = malloc(sizeof(int) * (T->nb + 1));
        memcpy(fill, T->own_start[k], sizeof(int) * (T->nb + 1));
        for (int i = 0; i < T->np[k]; ++i) T->own_idx[k][fill[T->owner[k][i]]++] = i;
        free(fill);
    }
    T->nsrc_sub = calloc(T->nb, sizeof(int));
    T->ntgt_sub = calloc(T->nb, sizeof(int));
    for (int b = T->nb - 1; b >= 0; --b) {
        T->nsrc_sub[b] += T->own_start[KSRC][b + 1] - T->own_start[KSRC][b];
        T->ntgt_sub[b] += (T->own_start[KCTR][b + 1] - T->own_start[KCTR][b]) +
                          (T->own_start[KTGT][b + 1] - T->own_start[KTGT][b]);
        if (T->parent[b] >= 0) {
            T->nsrc_sub[T->parent[b]] += T->nsrc_sub[b];
            T->ntgt_sub[T->parent[b]] += T->ntgt_sub[b];
        }
    }
    return T;
}

void orc_tree_free(otree *T)
{
    if (!T) return;
    free(T->level); free(T->ic); free(T->cen); free(T->hw); free(T->parent); free(T->child);
    free(T->level_start); free(T->nsrc_sub); free(T->ntgt_sub);
    for (int k = 0; k < 3; ++k) { free(T->owner[k]); free(T->own_start[k]); free(T->own_idx[k]); }
    free(T);
}

/* info: [n_boxes, n_levels, n_overfull, n_src, n_ctr, n_tgt] and root center/radius */
void orc_tree_info(const otree *T, int64_t *info, double *root)
{
    info[0] = T->nb; info[1] = T->nlev; info[2] = T->n_overfull;
    info[3] = T->np[0]; info[4] = T->np[1]; info[5] = T->np[2];
    root[0] = T->root_c[0]; root[1] = T->root_c[1]; root[2] = T->root_c[2]; root[3] = T->root_h;
}

void orc_tree_arrays(const otree *T, int *level, int64_t *ic, double *cen, double *hw, int *parent, int *child,
                     int *src_owner, int *ctr_owner, int *tgt_owner)
{
    memcpy(level, T->level, sizeof(int) * T->nb);
    memcpy(ic, T->ic, sizeof(int64_t) * 3 * T->nb);
    memcpy(cen, T->cen, sizeof(double) * 3 * T->nb);
    memcpy(hw, T->hw, sizeof(double) * T->nb);
    memcpy(parent, T->parent, sizeof(int) * T->nb);
    memcpy(child, T->child, sizeof(int) * 8 * T->nb);
    memcpy(src_owner, T->owner[0], sizeof(int) * T->np[0]);
    memcpy(ctr_owner, T->owner[1], sizeof(int) * T->np[1]);
    memcpy(tgt_owner, T->owner[2], sizeof(int) * T->np[2]);
}

/* ------------------------------------------------------------------------ */
/* interaction lists (Section 5.2.3-5.2.4)                                    */
/* ------------------------------------------------------------------------ */

enum { L_U = 0, L_V, L_WCLOSE, L_WFAR, L_XCLOSE, L_XFAR, L_N };

typedef struct {
    int nb;
    int *start[L_N]; /* nb + 1 */
    int *idx[L_N];
} olists;

static int is_leaf(const otree *T, int b)
{
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * b + o] >= 0) return 0;
    return 1;
}

/* integer extent of a box in units of the finest level Lf: [lo, hi] per dimension */
static void box_extent(const otree *T, int b, int Lf, int64_t lo[3], int64_t hi[3])
{
    int sh = Lf - T->level[b];
    for (int d = 0; d < 3; ++d) {
        lo[d] = T->ic[3 * b + d] << sh;
        hi[d] = (T->ic[3 * b + d] + 1) << sh;
    }
}

/* Adjacent: the closed cubes intersect and their interiors do not (exact integer test). */
static int adjacent(const otree *T, int a, int b, int Lf)
{
    int64_t la[3], ha[3], lb[3], hb[3];
    box_extent(T, a, Lf, la, ha);
    box_extent(T, b, Lf, lb, hb);
    int closed = 1, open = 1;
    for (int d = 0; d < 3; ++d) {
        if (la[d] > hb[d] || lb[d] > ha[d]) closed = 0;
        if (!(la[d] < hb[d] && lb[d] < ha[d])) open = 0;
    }
    return closed && !open;
}

/* k-colleague: same level, inside the k-near neighborhood (|di| <= k per axis), not the box itself. */
static int colleague(const otree *T, int a, int b, int k)
{
    if (T->level[a] != T->level[b] || a == b) return 0;
    for (int d = 0; d < 3; ++d) {
        int64_t di = T->ic[3 * a + d] - T->ic[3 * b + d];
        if (di < -k || di > k) return 0;
    }
    return 1;
}

/* a adequately separated from TCR(b): l2 distance from the center of a to the boundary of
 * TCR(b), taken as signed (negative inside), is at least 3|a|. */
static int sep_a_tcrb(const otree *T, int a, int b)
{
    if (T->linf) {
        /* l-infinity TCR: l-infinity distance from the center of a to the boundary of the cube
         * of radius |b|(1 + t_f), signed, is at least 3|a| */
        double m = 0.0;
        for (int d = 0; d < 3; ++d) m = fmax(m, fabs(T->cen[3 * a + d] - T->cen[3 * b + d]));
        return m - T->hw[b] * (1.0 + T->tf) >= 3.0 * T->hw[a];
    }
    double dx = T->cen[3 * a] - T->cen[3 * b], dy = T->cen[3 * a + 1] - T->cen[3 * b + 1],
           dz = T->cen[3 * a + 2] - T->cen[3 * b + 2];
    double dist = sqrt(dx * dx + dy * dy + dz * dz);
    return dist - (sqrt(3.0) * T->hw[b]) * (1.0 + T->tf) >= 3.0 * T->hw[a];
}

/* TCR(a) adequately separated from b: l-infinity distance from the center of a to the boundary
 * of b, signed, is at least 3|a|(1 + t_f). */
static int sep_tcra_b(const otree *T, int a, int b)
{
    double m = 0.0;
    for (int d = 0; d < 3; ++d) m = fmax(m, fabs(T->cen[3 * a + d] - T->cen[3 * b + d]));
    return m - T->hw[b] >= (3.0 * T->hw[a]) * (1.0 + T->tf);
}

static int is_desc(const otree *T, int d, int b) /* strict descendant */
{
    for (int w = T->parent[d]; w >= 0; w = T->parent[w])
        if (w == b) return 1;
    return 0;
}

static int finest_level(const otree *T) { return T->nlev - 1; }

static int is_target_box(const otree *T, int b)
{
    return (T->own_start[KCTR][b + 1] - T->own_start[KCTR][b]) + (T->own_start[KTGT][b + 1] - T->own_start[KTGT][b]) > 0;
}

static int is_source_box(const otree *T, int b) { return T->own_start[KSRC][b + 1] - T->own_start[KSRC][b] > 0; }

typedef struct {
    int n, cap;
    int *v;
} ivec;

static void iv_push(ivec *a, int x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 16;
        a->v = realloc(a->v, sizeof(int) * a->cap);
    }
    a->v[a->n++] = x;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static void iv_sort_unique(ivec *a)
{
    if (a->n == 0) return;
    qsort(a->v, a->n, sizeof(int), cmp_int);
    int k = 1;
    for (int i = 1; i < a->n; ++i)
        if (a->v[i] != a->v[k - 1]) a->v[k++] = a->v[i];
    a->n = k;
}

static int iv_has(const ivec *a, int x)
{
    for (int i = 0; i < a->n; ++i)
        if (a->v[i] == x) return 1;
    return 0;
}

static olists *lists_from_vecs(int nb, ivec *vec /* nb * L_N */)
{
    olists *Ls = calloc(1, sizeof(olists));
    Ls->nb = nb;
    for (int l = 0; l < L_N; ++l) {
        Ls->start[l] = calloc(nb + 1, sizeof(int));
        for (int b = 0; b < nb; ++b) Ls->start[l][b + 1] = Ls->start[l][b] + vec[b * L_N + l].n;
        Ls->idx[l] = malloc(sizeof(int) * (Ls->start[l][nb] > 0 ? Ls->start[l][nb] : 1));
        for (int b = 0; b < nb; ++b) {
            memcpy(Ls->idx[l] + Ls->start[l][b], vec[b * L_N + l].v, sizeof(int) * vec[b * L_N + l].n);
            free(vec[b * L_N + l].v);
        }
    }
    free(vec);
    return Ls;
}

/*
 * Literal construction of the six lists: every definition of Section 5.2.3-5.2.4
 * checked by brute force over all boxes (O(N_B^2) and worse).  Readings:
 *  - k-colleagues exclude the box itself (otherwise a box would be its own
 *    non-adjacent 2-colleague and List 3/4 would count its own sources twice);
 *  - descendants are strict; "adjacent" is the exact integer test above;
 *  - target box = owns a QBX center or a target; lists U, W are made for target
 *    boxes, lists V, X for target and target-ancestor boxes;
 *  - boxes whose subtree holds no source are left out of every list.
 */
olists *orc_build_lists_slow(const otree *T)
{
    int nb = T->nb, Lf = finest_level(T);
    ivec *vec = calloc((size_t)nb * L_N, sizeof(ivec));
    ivec *X = calloc(nb, sizeof(ivec));
    for (int b = 0; b < nb; ++b) {
        int tgt = is_target_box(T, b), tanc = T->ntgt_sub[b] > 0;
        if (!tanc) continue;
        /* List 4 of b */
        for (int d = 0; d < nb; ++d) {
            if (!is_leaf(T, d) || !is_source_box(T, d)) continue;
            int in4 = 0;
            if (T->parent[b] >= 0 && adjacent(T, d, T->parent[b], Lf) && !adjacent(T, d, b, Lf))
                for (int a = T->parent[b]; a >= 0; a = T->parent[a])
                    if (colleague(T, d, a, 2)) in4 = 1;
            if (colleague(T, d, b, 2) && !adjacent(T, d, b, Lf)) in4 = 1;
            if (in4) iv_push(&X[b], d);
        }
        if (tgt) {
            /* List 1 */
            for (int d = 0; d < nb; ++d)
                if (is_leaf(T, d) && is_source_box(T, d) && (d == b || is_desc(T, d, b) || adjacent(T, d, b, Lf)))
                    iv_push(&vec[b * L_N + L_U], d);
            /* List 3, then its close/far split */
            ivec W = {0};
            for (int d = 0; d < nb; ++d) {
                if (T->nsrc_sub[d] == 0) continue;
                int inDT = 0;
                for (int w = 0; w < nb && !inDT; ++w)
                    if (colleague(T, w, b, 2) && is_desc(T, d, w)) inDT = 1;
                if (!inDT || adjacent(T, d, b, Lf)) continue;
                int ok = 1;
                for (int w = T->parent[d]; w >= 0; w = T->parent[w]) {
                    int wDT = 0;
                    for (int u = 0; u < nb && !wDT; ++u)
                        if (colleague(T, u, b, 2) && is_desc(T, w, u)) wDT = 1;
                    if (wDT && !adjacent(T, w, b, Lf)) ok = 0;
                }
                if (ok) iv_push(&W, d);
            }
            for (int d = 0; d < nb; ++d) {
                if (T->nsrc_sub[d] == 0) continue;
                int inDW = iv_has(&W, d);
                for (int i = 0; i < W.n && !inDW; ++i)
                    if (is_desc(T, d, W.v[i])) inDW = 1;
                if (!inDW) continue;
                if (!sep_a_tcrb(T, d, b)) {
                    if (is_leaf(T, d)) iv_push(&vec[b * L_N + L_WCLOSE], d);
                } else {
                    int ok = 1;
                    for (int w = T->parent[d]; w >= 0; w = T->parent[w]) {
                        int wDW = iv_has(&W, w);
                        for (int i = 0; i < W.n && !wDW; ++i)
                            if (is_desc(T, w, W.v[i])) wDW = 1;
                        if (wDW && sep_a_tcrb(T, w, b)) ok = 0;
                    }
                    if (ok) iv_push(&vec[b * L_N + L_WFAR], d);
                }
            }
            free(W.v);
        }
        /* List 2 */
        if (T->parent[b] >= 0) {
            int pb = T->parent[b];
            for (int d = 0; d < nb; ++d) {
                if (T->level[d] != T->level[b] || d == b || T->nsrc_sub[d] == 0) continue;
                int pd = T->parent[d];
                if (!(pd == pb || colleague(T, pd, pb, 2))) continue;
                if (colleague(T, d, b, 2)) continue;
                iv_push(&vec[b * L_N + L_V], d);
            }
        }
    }
    /* List 4 close/far: needs X of all ancestors */
    for (int b = 0; b < nb; ++b) {
        if (T->ntgt_sub[b] == 0) continue;
        for (int d = 0; d < nb; ++d) {
            int inX_anc = 0;
            for (int w = b; w >= 0; w = T->parent[w])
                if (iv_has(&X[w], d)) inX_anc = 1;
            if (inX_anc && !sep_tcra_b(T, b, d)) iv_push(&vec[b * L_N + L_XCLOSE], d);
        }
    }
    for (int b = 0; b < nb; ++b) {
        if (T->ntgt_sub[b] == 0) continue;
        for (int i = 0; i < X[b].n; ++i)
            if (sep_tcra_b(T, b, X[b].v[i])) iv_push(&vec[b * L_N + L_XFAR], X[b].v[i]);
        int pb = T->parent[b];
        if (pb >= 0)
            for (int i = 0; i < vec[pb * L_N + L_XCLOSE].n; ++i) {
                int d = vec[pb * L_N + L_XCLOSE].v[i];
                if (sep_tcra_b(T, b, d)) iv_push(&vec[b * L_N + L_XFAR], d);
            }
    }
    for (int b = 0; b < nb; ++b) {
        free(X[b].v);
        for (int l = 0; l < L_N; ++l) iv_sort_unique(&vec[b * L_N + l]);
    }
    free(X);
    return lists_from_vecs(nb, vec);
}

/* Morton order of two same-level integer coordinate triples (z most significant in
 * each octal digit): the axis with the highest differing bit decides. */
static int less_msb(uint64_t a, uint64_t b) { return a < b && a < (a ^ b); }

static int morton_less(const int64_t *a, const int64_t *b)
{
    int dim = 2;
    uint64_t best = (uint64_t)(a[2] ^ b[2]);
    for (int d = 1; d >= 0; --d) {
        uint64_t x = (uint64_t)(a[d] ^ b[d]);
        if (less_msb(best, x)) { dim = d; best = x; }
    }
    return a[dim] < b[dim];
}

/* box at (level, ic) or -1; binary search over the level's boxes (Morton-sorted) */
static int find_box(const otree *T, int lev, const int64_t ic[3])
{
    if (lev < 0 || lev >= T->nlev) return -1;
    int64_t n = (int64_t)1 << lev;
    for (int d = 0; d < 3; ++d)
        if (ic[d] < 0 || ic[d] >= n) return -1;
    int lo = T->level_start[lev], hi = T->level_start[lev + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (morton_less(&T->ic[3 * mid], ic)) lo = mid + 1;
        else hi = mid;
    }
    if (lo < T->level_start[lev + 1] && T->ic[3 * lo] == ic[0] && T->ic[3 * lo + 1] == ic[1] && T->ic[3 * lo + 2] == ic[2])
        return lo;
    return -1;
}

static void colleagues(const otree *T, int b, int k, ivec *out)
{
    out->n = 0;
    for (int dz = -k; dz <= k; ++dz)
        for (int dy = -k; dy <= k; ++dy)
            for (int dx = -k; dx <= k; ++dx) {
                if (!dx && !dy && !dz) continue;
                int64_t ic[3] = {T->ic[3 * b] + dx, T->ic[3 * b + 1] + dy, T->ic[3 * b + 2] + dz};
                int d = find_box(T, T->level[b], ic);
                if (d >= 0) iv_push(out, d);
            }
}

static void leaf_desc_sources(const otree *T, int b, ivec *out)
{
    if (T->nsrc_sub[b] == 0) return;
    if (is_leaf(T, b)) { iv_push(out, b); return; }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * b + o] >= 0) leaf_desc_sources(T, T->child[8 * b + o], out);
}

static void adj_leaves_below(const otree *T, int d, int b, int Lf, ivec *out)
{
    if (T->nsrc_sub[d] == 0 || !adjacent(T, d, b, Lf)) return;
    if (is_leaf(T, d)) { iv_push(out, d); return; }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * d + o] >= 0) adj_leaves_below(T, T->child[8 * d + o], b, Lf, out);
}

/* List 3 search below a box d that is a descendant of a 2-colleague of b */
static void list3_walk(const otree *T, int d, int b, int Lf, ivec *W)
{
    if (T->nsrc_sub[d] == 0) return;
    if (!adjacent(T, d, b, Lf)) { iv_push(W, d); return; }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * d + o] >= 0) list3_walk(T, T->child[8 * d + o], b, Lf, W);
}

static void list3_split(const otree *T, int d, int b, ivec *cl, ivec *fa)
{
    if (T->nsrc_sub[d] == 0) return;
    if (sep_a_tcrb(T, d, b)) { iv_push(fa, d); return; }
    if (is_leaf(T, d)) { iv_push(cl, d); return; }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * d + o] >= 0) list3_split(T, T->child[8 * d + o], b, cl, fa);
}

/* Same lists as orc_build_lists_slow, built by walking neighborhoods. */
olists *orc_build_lists(const otree *T)
{
    int nb = T->nb, Lf = finest_level(T);
    ivec *vec = calloc((size_t)nb * L_N, sizeof(ivec));
    ivec *X = calloc(nb, sizeof(ivec));
    ivec C = {0}, CA = {0};
    for (int b = 0; b < nb; ++b) {
        if (T->ntgt_sub[b] == 0) continue;
        int pb = T->parent[b];
        colleagues(T, b, 2, &C);
        /* List 4 */
        for (int i = 0; i < C.n; ++i) {
            int d = C.v[i];
            if (is_leaf(T, d) && is_source_box(T, d) && !adjacent(T, d, b, Lf)) iv_push(&X[b], d);
        }
        for (int a = pb; a >= 0; a = T->parent[a]) {
            colleagues(T, a, 2, &CA);
            for (int i = 0; i < CA.n; ++i) {
                int d = CA.v[i];
                if (is_leaf(T, d) && is_source_box(T, d) && adjacent(T, d, pb, Lf) && !adjacent(T, d, b, Lf))
                    iv_push(&X[b], d);
            }
        }
        iv_sort_unique(&X[b]);
        /* List 2 */
        if (pb >= 0) {
            colleagues(T, pb, 2, &CA);
            iv_push(&CA, pb);
            for (int i = 0; i < CA.n; ++i)
                for (int o = 0; o < 8; ++o) {
                    int d = T->child[8 * CA.v[i] + o];
                    if (d < 0 || d == b || T->nsrc_sub[d] == 0) continue;
                    if (colleague(T, d, b, 2)) continue;
                    iv_push(&vec[b * L_N + L_V], d);
                }
        }
        if (!is_target_box(T, b)) continue;
        /* List 1: b if leaf, leaf descendants, adjacent leaves at this level or below, and coarser adjacent leaves */
        ivec *U = &vec[b * L_N + L_U];
        leaf_desc_sources(T, b, U);
        for (int i = 0; i < C.n; ++i) adj_leaves_below(T, C.v[i], b, Lf, U);
        for (int a = pb; a >= 0; a = T->parent[a]) {
            colleagues(T, a, 1, &CA);
            for (int i = 0; i < CA.n; ++i) {
                int d = CA.v[i];
                if (is_leaf(T, d) && is_source_box(T, d) && adjacent(T, d, b, Lf)) iv_push(U, d);
            }
        }
        /* List 3 and its split */
        ivec W = {0};
        for (int i = 0; i < C.n; ++i)
            for (int o = 0; o < 8; ++o) {
                int d = T->child[8 * C.v[i] + o];
                if (d >= 0) list3_walk(T, d, b, Lf, &W);
            }
        for (int i = 0; i < W.n; ++i) list3_split(T, W.v[i], b, &vec[b * L_N + L_WCLOSE], &vec[b * L_N + L_WFAR]);
        free(W.v);
    }
    /* List 4 close/far, top-down (parents precede children in box order) */
    for (int b = 0; b < nb; ++b) {
        if (T->ntgt_sub[b] == 0) continue;
        int pb = T->parent[b];
        ivec cand = {0};
        for (int i = 0; i < X[b].n; ++i) iv_push(&cand, X[b].v[i]);
        if (pb >= 0)
            for (int i = 0; i < vec[pb * L_N + L_XCLOSE].n; ++i) iv_push(&cand, vec[pb * L_N + L_XCLOSE].v[i]);
        iv_sort_unique(&cand);
        for (int i = 0; i < cand.n; ++i) {
            int d = cand.v[i];
            if (sep_tcra_b(T, b, d)) iv_push(&vec[b * L_N + L_XFAR], d);
            else iv_push(&vec[b * L_N + L_XCLOSE], d);
        }
        free(cand.v);
    }
    for (int b = 0; b < nb; ++b) {
        free(X[b].v);
        for (int l = 0; l < L_N; ++l) iv_sort_unique(&vec[b * L_N + l]);
    }
    free(X);
    free(C.v);
    free(CA.v);
    return lists_from_vecs(nb, vec);
}

void orc_lists_free(olists *Ls)
{
    if (!Ls) return;
    for (int l = 0; l < L_N; ++l) { free(Ls->start[l]); free(Ls->idx[l]); }
    free(Ls);
}

int64_t orc_lists_nnz(const olists *Ls, int which) { return Ls->start[which][Ls->nb]; }

void orc_lists_get(const olists *Ls, int which, int *start, int *idx)
{
    memcpy(start, Ls->start[which], sizeof(int) * (Ls->nb + 1));
    memcpy(idx, Ls->idx[which], sizeof(int) * Ls->start[which][Ls->nb]);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4, Stages 2-9                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *sxyz, *tgxyz, *cxyz;
    int ns, nc, nt;
    double *q;   /* ns charges, w sigma */
    double *dip; /* 3 * ns dipoles w mu n, or NULL */
} srcset;

static void src_q_d(const srcset *S, int j, double s[3], double *q, double d[3], int *has_d)
{
    get_pt(S->sxyz, S->ns, j, s);
    *q = S->q[j];
    *has_d = S->dip != NULL;
    if (S->dip) { d[0] = S->dip[3 * j]; d[1] = S->dip[3 * j + 1]; d[2] = S->dip[3 * j + 2]; }
}

/* QBX local at center c (order q) += P2QBXL over all sources owned by the boxes of a list */
static void direct_to_center(const otree *T, const srcset *S, const int *lst, int n, const double c[3], int q, cplx *Lq)
{
    double s[3], d[3], qq;
    int hd;
    for (int i = 0; i < n; ++i) {
        int box = lst[i];
        for (int k = T->own_start[KSRC][box]; k < T->own_start[KSRC][box + 1]; ++k) {
            int j = T->own_idx[KSRC][k];
            src_q_d(S, j, s, &qq, d, &hd);
            p2l(q, c, s, qq, hd ? d : NULL, Lq);
        }
    }
}

static double direct_to_point(const otree *T, const srcset *S, const int *lst, int n, const double t[3])
{
    double s[3], d[3], qq, acc = 0.0;
    int hd;
    for (int i = 0; i < n; ++i) {
        int box = lst[i];
        for (int k = T->own_start[KSRC][box]; k < T->own_start[KSRC][box + 1]; ++k) {
            int j = T->own_idx[KSRC][k];
            src_q_d(S, j, s, &qq, d, &hd);
            acc += p2p(s, qq, hd ? d : NULL, t);
        }
    }
    return acc;
}

static int sq(int p) { return (p + 1) * (p + 1); }

static void setup_sources(srcset *S, const double *sxyz, int ns, const double *w, const double *sigma,
                          const double *mu, const double *nrm)
{
    S->sxyz = sxyz;
    S->ns = ns;
    S->q = calloc(ns > 0 ? ns : 1, sizeof(double));
    S->dip = NULL;
    for (int j = 0; j < ns; ++j) S->q[j] = sigma ? w[j] * sigma[j] : 0.0;
    if (mu) {
        S->dip = malloc(sizeof(double) * 3 * (ns > 0 ? ns : 1));
        for (int j = 0; j < ns; ++j)
            for (int d = 0; d < 3; ++d) S->dip[3 * j + d] = w[j] * mu[j] * nrm[d * ns + j];
    }
}

/*
 * GIGAQBX FMM (Algorithm 4, Stages 2-9).  pot[t] = S[sigma](t) + D[mu](t) at every target.
 * Charges are w sigma, dipoles w mu n.  tgt_ctr[t] >= 0: t is evaluated through the QBX
 * local of that center (Stage 9, second loop); tgt_ctr[t] < 0: t is a conventional
 * (point) target.  Orders: every multipole expansion has the order p_fmm; the local
 * expansion of box b has the order pbox[b] (or p_fmm); the QBX local of center c has
 * p_qbx[c] (or p_qbx); a translation between different orders truncates or pads.
 * If qbx_out is given it receives each center's QBX local, (qmax+1)^2 complex per center.
 */
int orc_fmm_eval(const otree *T, const olists *Ls, const double *sxyz, int ns, const double *w, const double *sigma,
                 const double *mu, const double *nrm, const double *cxyz, int nc, const double *txyz,
                 const int *tgt_ctr, int nt, int p_qbx, int p_fmm, const signed char *qctr, const signed char *pbox,
                 double *pot, double *qbx_out, int qmax)
{
    init_tables();
    if (ns != T->np[KSRC] || nc != T->np[KCTR] || nt != T->np[KTGT]) return -1;
    srcset S;
    setup_sources(&S, sxyz, ns, w, sigma, mu, nrm);
    int nb = T->nb;
    int pmax = p_fmm;
    if (pbox) for (int b = 0; b < nb; ++b) if (pbox[b] > pmax) pmax = pbox[b];
    int qm = p_qbx;
    if (qctr) { qm = 0; for (int c = 0; c < nc; ++c) if (qctr[c] > qm) qm = qctr[c]; }
    int nP = sq(pmax), nQ = sq(qm);
    cplx *M = calloc((size_t)nb * nP, sizeof(cplx));
    cplx *L = calloc((size_t)nb * nP, sizeof(cplx));
    cplx *Lq = calloc((size_t)(nc > 0 ? nc : 1) * nQ, sizeof(cplx));
    double *pnear = calloc(nt > 0 ? nt : 1, sizeof(double));
#define PB(b) (pbox ? (int)pbox[b] : p_fmm) /* order of the local expansion of box b */
#define PM p_fmm                            /* order of every multipole expansion */
#define QC(cc) (qctr ? (int)qctr[cc] : p_qbx)

    /* Every loop below that is marked "omp parallel for" writes, per iteration, only the expansions
     * and potentials of its own box, center or target; compiled with -fopenmp it runs on all cores,
     * otherwise serially.  Each result is accumulated in the same order either way. */

    /* Stage 2: multipoles of leaves, then the upward pass: level by level from the deepest, each
     * parent adding its children from the highest box number down (postorder) */
#pragma omp parallel for schedule(dynamic, 64)
    for (int b = 0; b < nb; ++b) {
        double s[3], d[3], qq;
        int hd;
        for (int k = T->own_start[KSRC][b]; k < T->own_start[KSRC][b + 1]; ++k) {
            src_q_d(&S, T->own_idx[KSRC][k], s, &qq, d, &hd);
            p2m(PM, &T->cen[3 * b], s, qq, hd ? d : NULL, &M[(size_t)b * nP]);
        }
    }
    for (int lev = T->nlev - 2; lev >= 0; --lev) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int pa = T->level_start[lev]; pa < T->level_start[lev + 1]; ++pa)
            for (int o = 7; o >= 0; --o) {
                int b = T->child[8 * pa + o];
                if (b >= 0 && T->nsrc_sub[b] > 0)
                    m2m(PM, &T->cen[3 * b], &M[(size_t)b * nP], PM, &T->cen[3 * pa], &M[(size_t)pa * nP]);
            }
    }

    /* Stages 3, 5(a), 6(a): direct interactions from U, W-close, X-close */
    const int direct_lists[3] = {L_U, L_WCLOSE, L_XCLOSE};
    for (int li = 0; li < 3; ++li) {
        int l = direct_lists[li];
#pragma omp parallel for schedule(dynamic, 16)
        for (int b = 0; b < nb; ++b) {
            double c[3], t[3];
            const int *lst = Ls->idx[l] + Ls->start[l][b];
            int n = Ls->start[l][b + 1] - Ls->start[l][b];
            if (n == 0) continue;
            for (int k = T->own_start[KTGT][b]; k < T->own_start[KTGT][b + 1]; ++k) {
                int ti = T->own_idx[KTGT][k];
                if (tgt_ctr[ti] >= 0) continue;
                get_pt(txyz, nt, ti, t);
                pnear[ti] += direct_to_point(T, &S, lst, n, t);
            }
            for (int k = T->own_start[KCTR][b]; k < T->own_start[KCTR][b + 1]; ++k) {
                int ci = T->own_idx[KCTR][k];
                get_pt(cxyz, nc, ci, c);
                direct_to_center(T, &S, lst, n, c, QC(ci), &Lq[(size_t)ci * nQ]);
            }
        }
    }

    /* Stage 4: List 2 multipole-to-local */
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b)
        for (int i = Ls->start[L_V][b]; i < Ls->start[L_V][b + 1]; ++i) {
            int dd = Ls->idx[L_V][i];
            m2l(PM, &T->cen[3 * dd], &M[(size_t)dd * nP], PB(b), &T->cen[3 * b], &L[(size_t)b * nP]);
        }

    /* Stage 5(b): List 3 far multipoles at point targets and QBX centers */
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b)
        for (int i = Ls->start[L_WFAR][b]; i < Ls->start[L_WFAR][b + 1]; ++i) {
            double c[3], t[3];
            int dd = Ls->idx[L_WFAR][i];
            for (int k = T->own_start[KTGT][b]; k < T->own_start[KTGT][b + 1]; ++k) {
                int ti = T->own_idx[KTGT][k];
                if (tgt_ctr[ti] >= 0) continue;
                get_pt(txyz, nt, ti, t);
                pnear[ti] += m2p(PM, &T->cen[3 * dd], &M[(size_t)dd * nP], t);
            }
            for (int k = T->own_start[KCTR][b]; k < T->own_start[KCTR][b + 1]; ++k) {
                int ci = T->own_idx[KCTR][k];
                get_pt(cxyz, nc, ci, c);
                m2l(PM, &T->cen[3 * dd], &M[(size_t)dd * nP], QC(ci), c, &Lq[(size_t)ci * nQ]);
            }
        }

    /* Stage 6(b): List 4 far sources to local expansions of the box */
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b)
        for (int i = Ls->start[L_XFAR][b]; i < Ls->start[L_XFAR][b + 1]; ++i) {
            double s[3], d[3], qq;
            int hd;
            int dd = Ls->idx[L_XFAR][i];
            for (int k = T->own_start[KSRC][dd]; k < T->own_start[KSRC][dd + 1]; ++k) {
                src_q_d(&S, T->own_idx[KSRC][k], s, &qq, d, &hd);
                p2l(PB(b), &T->cen[3 * b], s, qq, hd ? d : NULL, &L[(size_t)b * nP]);
            }
        }

    /* Stage 7: downward pass in preorder (level by level) */
    for (int lev = 1; lev < T->nlev; ++lev) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int b = T->level_start[lev]; b < T->level_start[lev + 1]; ++b) {
            int pa = T->parent[b];
            if (T->ntgt_sub[b] > 0)
                l2l(PB(pa), &T->cen[3 * pa], &L[(size_t)pa * nP], PB(b), &T->cen[3 * b], &L[(size_t)b * nP]);
        }
    }

    /* Stage 8: box locals to QBX centers */
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b)
        for (int k = T->own_start[KCTR][b]; k < T->own_start[KCTR][b + 1]; ++k) {
            double c[3];
            int ci = T->own_idx[KCTR][k];
            get_pt(cxyz, nc, ci, c);
            l2l(PB(b), &T->cen[3 * b], &L[(size_t)b * nP], QC(ci), c, &Lq[(size_t)ci * nQ]);
        }

    /* Stage 9: final potentials */
#pragma omp parallel for schedule(dynamic, 64)
    for (int b = 0; b < nb; ++b)
        for (int k = T->own_start[KTGT][b]; k < T->own_start[KTGT][b + 1]; ++k) {
            double c[3], t[3];
            int ti = T->own_idx[KTGT][k];
            get_pt(txyz, nt, ti, t);
            int ci = tgt_ctr[ti];
            if (ci < 0) {
                pot[ti] = pnear[ti] + l2p(PB(b), &T->cen[3 * b], &L[(size_t)b * nP], t);
            } else {
                get_pt(cxyz, nc, ci, c);
                pot[ti] = l2p(QC(ci), c, &Lq[(size_t)ci * nQ], t);
            }
        }
    if (qbx_out)
        for (int ci = 0; ci < nc; ++ci)
            for (int i = 0; i < sq(qmax); ++i) {
                cplx v = (i < nQ) ? Lq[(size_t)ci * nQ + i] : 0.0;
                qbx_out[2 * ((size_t)ci * sq(qmax) + i)] = creal(v);
                qbx_out[2 * ((size_t)ci * sq(qmax) + i) + 1] = cimag(v);
            }
#undef PB
#undef PM
#undef QC
    free(M); free(L); free(Lq); free(pnear); free(S.q); free(S.dip);
    return 0;
}

/*
 * Direct (unaccelerated) QBX: every source into every center's order-q local
 * (eq. qbxcoeff discretised by the source quadrature), evaluated at the associated
 * targets (eq. qbxlocal); point targets get the plain quadrature sum of G.
 */
int orc_direct_eval(const double *sxyz, int ns, const double *w, const double *sigma, const double *mu,
                    const double *nrm, const double *cxyz, int nc, const double *txyz, const int *tgt_ctr, int nt,
                    int p_qbx, const signed char *qctr, double *pot)
{
    init_tables();
    srcset S;
    setup_sources(&S, sxyz, ns, w, sigma, mu, nrm);
    int qm = p_qbx;
    if (qctr) { qm = 0; for (int c = 0; c < nc; ++c) if (qctr[c] > qm) qm = qctr[c]; }
    cplx *Lq = malloc(sizeof(cplx) * sq(qm));
    double s[3], d[3], c[3], t[3], qq;
    int hd;
    for (int ti = 0; ti < nt; ++ti) {
        get_pt(txyz, nt, ti, t);
        int ci = tgt_ctr[ti];
        if (ci < 0) {
            double acc = 0.0;
            for (int j = 0; j < ns; ++j) {
                src_q_d(&S, j, s, &qq, d, &hd);
                acc += p2p(s, qq, hd ? d : NULL, t);
            }
            pot[ti] = acc;
        } else {
            int q = qctr ? qctr[ci] : p_qbx;
            for (int i = 0; i < sq(q); ++i) Lq[i] = 0.0;
            get_pt(cxyz, nc, ci, c);
            for (int j = 0; j < ns; ++j) {
                src_q_d(&S, j, s, &qq, d, &hd);
                p2l(q, c, s, qq, hd ? d : NULL, Lq);
            }
            pot[ti] = l2p(q, c, Lq, t);
        }
    }
    free(Lq); free(S.q); free(S.dip);
    return 0;
}

/*
 * Interaction counts per list, from the built lists (the quantities Table ilist-operation-counts
 * multiplies by the per-entry cost), n_t = QBX centers owned by the target box, n_s = sources of the
 * source box (owned sources; U, W-close and X-close entries are leaves) or of its subtree (X-far):
 *   counts[U], counts[W-close], counts[X-close] = sum over entries of n_s n_t
 *   counts[V] = number of entries,  counts[W-far] = sum over entries of n_t,
 *   counts[X-far] = sum over entries of n_s.
 */
void orc_lists_counts(const otree *T, const olists *Ls, int64_t *counts)
{
    for (int l = 0; l < L_N; ++l) counts[l] = 0;
    for (int b = 0; b < T->nb; ++b) {
        int64_t nt = T->own_start[KCTR][b + 1] - T->own_start[KCTR][b];
        for (int l = 0; l < L_N; ++l)
            for (int i = Ls->start[l][b]; i < Ls->start[l][b + 1]; ++i) {
                int d = Ls->idx[l][i];
                int64_t nsd = T->own_start[KSRC][d + 1] - T->own_start[KSRC][d];
                if (l == L_U || l == L_WCLOSE || l == L_XCLOSE) counts[l] += nsd * nt;
                else if (l == L_V) counts[l] += 1;
                else if (l == L_WFAR) counts[l] += nt;
                else counts[l] += T->nsrc_sub[d];
            }
    }
}

/*
 * Modeled operation counts (Section 6.3): out[0..5] = the per-list costs of Table
 * ilist-operation-counts (U, W-close, X-close: p_qbx^2 n_s n_t; V: p_fmm^3; W-far: p_fmm^3 n_t;
 * X-far: p_fmm^2 n_s) summed over the entries; out[6] = the stage terms of Table
 * complexity-analysis that no list carries: N_S p_fmm^2 + N_B p_fmm^3 (Stage 2),
 * 8 N_B p_fmm^3 (Stage 7), N_C p_fmm^3 (Stage 8), N_T p_qbx^2 (Stage 9); out[7] = the sum.
 */
void orc_lists_cost(const otree *T, const olists *Ls, int p_qbx, int p_fmm, double *out)
{
    double q2 = (double)p_qbx * p_qbx, p3 = (double)p_fmm * p_fmm * p_fmm, p2 = (double)p_fmm * p_fmm;
    int64_t c[L_N];
    orc_lists_counts(T, Ls, c);
    out[L_U] = q2 * (double)c[L_U];
    out[L_V] = p3 * (double)c[L_V];
    out[L_WCLOSE] = q2 * (double)c[L_WCLOSE];
    out[L_WFAR] = p3 * (double)c[L_WFAR];
    out[L_XCLOSE] = q2 * (double)c[L_XCLOSE];
    out[L_XFAR] = p2 * (double)c[L_XFAR];
    out[6] = (double)T->np[KSRC] * p2 + (double)T->nb * p3 + 8.0 * (double)T->nb * p3 + (double)T->np[KCTR] * p3 +
             (double)T->np[KTGT] * q2;
    out[7] = 0.0;
    for (int l = 0; l < 7; ++l) out[7] += out[l];
}

/* ------------------------------------------------------------------------ */
/* reference for the learned-order network (not part of the paper's method)   */
/* ------------------------------------------------------------------------ */

/*
 * Network 4 -> 64 -> 64 -> 2 with tanh hidden layers and a linear output; parameters
 * W1[64][4], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].  Loss L = 1/(2n) sum_i |y_i - t_i|^2.
 * Forward pass and gradient by the chain rule, in double precision, sample by sample.
 * grad receives dL/dparams (4610 doubles) followed by L.  This core takes double parameters,
 * inputs and labels; orc_mlp_loss_grad below is the same computation on float arrays.
 */
void orc_mlp_loss_grad_f64(const double *P, const double *x, const double *t, int n, double *grad)
{
    enum { NI = 4, A = 64, B = 64, NO = 2 };
    const int oW1 = 0, ob1 = oW1 + A * NI, oW2 = ob1 + A, ob2 = oW2 + B * A, oW3 = ob2 + B, ob3 = oW3 + NO * B,
              np = ob3 + NO;
    for (int i = 0; i <= np; ++i) grad[i] = 0.0;
    for (int s = 0; s < n; ++s) {
        double h1[A], h2[B], y[NO], dy[NO], d2[B], d1[A];
        for (int j = 0; j < A; ++j) {
            double a = P[ob1 + j];
            for (int k = 0; k < NI; ++k) a += P[oW1 + j * NI + k] * x[NI * s + k];
            h1[j] = tanh(a);
        }
        for (int j = 0; j < B; ++j) {
            double a = P[ob2 + j];
            for (int k = 0; k < A; ++k) a += P[oW2 + j * A + k] * h1[k];
            h2[j] = tanh(a);
        }
        for (int o = 0; o < NO; ++o) {
            double a = P[ob3 + o];
            for (int k = 0; k < B; ++k) a += P[oW3 + o * B + k] * h2[k];
            y[o] = a;
            double r = y[o] - t[NO * s + o];
            dy[o] = r / n;
            grad[np] += 0.5 * r * r / n;
        }
        for (int j = 0; j < B; ++j) {
            double g = 0.0;
            for (int o = 0; o < NO; ++o) g += P[oW3 + o * B + j] * dy[o];
            d2[j] = g * (1.0 - h2[j] * h2[j]);
        }
        for (int k = 0; k < A; ++k) {
            double g = 0.0;
            for (int j = 0; j < B; ++j) g += P[oW2 + j * A + k] * d2[j];
            d1[k] = g * (1.0 - h1[k] * h1[k]);
        }
        for (int j = 0; j < A; ++j) {
            for (int k = 0; k < NI; ++k) grad[oW1 + j * NI + k] += d1[j] * x[NI * s + k];
            grad[ob1 + j] += d1[j];
        }
        for (int j = 0; j < B; ++j) {
            for (int k = 0; k < A; ++k) grad[oW2 + j * A + k] += d2[j] * h1[k];
            grad[ob2 + j] += d2[j];
        }
        for (int o = 0; o < NO; ++o) {
            for (int k = 0; k < B; ++k) grad[oW3 + o * B + k] += dy[o] * h2[k];
            grad[ob3 + o] += dy[o];
        }
    }
}

int orc_mlp_loss_grad(const float *P, const float *x, const float *t, int n, double *grad)
{
    enum { NP = 4610 };
    double *Pd = malloc(sizeof(double) * NP), *xd = malloc(sizeof(double) * 4 * (n > 0 ? n : 1)),
           *td = malloc(sizeof(double) * 2 * (n > 0 ? n : 1));
    for (int i = 0; i < NP; ++i) Pd[i] = P[i];
    for (int i = 0; i < 4 * n; ++i) xd[i] = x[i];
    for (int i = 0; i < 2 * n; ++i) td[i] = t[i];
    orc_mlp_loss_grad_f64(Pd, xd, td, n, grad);
    free(Pd); free(xd); free(td);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* learned orders: sweep labels and the map from predictions to orders       */
/* (not part of the paper's method; the order network's inputs and outputs)  */
/* ------------------------------------------------------------------------ */

/*
 * Labels from an order sweep.  values[k * n + t] is target t's result at the k-th order of the
 * sweep (orders order_of[0] < ... < order_of[K-1], the last column the reference).  The label of
 * t is order_of[k*] for the smallest k* such that every column k >= k* lies within tol of the
 * reference: |values[k][t] - values[K-1][t]| <= tol.
 */
void orc_order_labels(const double *values, int K, const int *order_of, int n, double tol, int *labels)
{
    for (int t = 0; t < n; ++t) {
        double ref = values[(size_t)(K - 1) * n + t];
        int best = K - 1;
        for (int ks = 0; ks < K; ++ks) {
            int all_within = 1;
            for (int k = ks; k < K; ++k)
                if (!(fabs(values[(size_t)k * n + t] - ref) <= tol)) all_within = 0;
            if (all_within) { best = ks; break; }
        }
        labels[t] = order_of[best];
    }
}

/* clamp(ceil(y + margin), lo, hi) in single precision; a NaN prediction gives hi */
static int order_from_pred(float y, float margin, int lo, int hi)
{
    if (y != y) return hi;
    float v = ceilf(y + margin);
    if (v < (float)lo) return lo;
    if (v > (float)hi) return hi;
    return (int)v;
}

/*
 * Orders from network predictions pred[2c], pred[2c+1] (input center order).  The QBX order of
 * center c is clamp(ceil(pred[2c] + margin_q), q_lo, q_hi).  The order of box b's local expansion is
 * the largest clamp(ceil(pred[2c+1] + margin_p), p_lo, p_hi) over the centers c owned by b or by a
 * box below b; a box owning a point target (tgt_ctr[t] < 0), and every box above it, gets p_hi; a box
 * that neither holds a center nor a point target in its subtree gets p_default.  tgt_ctr may be
 * NULL (no point targets).
 */
void orc_orders_from_pred(const otree *T, const float *pred, const int *tgt_ctr, float margin_q, float margin_p,
                          int q_lo, int q_hi, int p_lo, int p_hi, int p_default, int *q_out, int *p_out)
{
    int nb = T->nb;
    int *best = malloc(sizeof(int) * (nb > 0 ? nb : 1));
    for (int b = 0; b < nb; ++b) best[b] = -1;
    for (int c = 0; c < T->np[KCTR]; ++c) {
        q_out[c] = order_from_pred(pred[2 * c], margin_q, q_lo, q_hi);
        int p = order_from_pred(pred[2 * c + 1], margin_p, p_lo, p_hi);
        for (int b = T->owner[KCTR][c]; b >= 0; b = T->parent[b])
            if (p > best[b]) best[b] = p;
    }
    if (tgt_ctr)
        for (int t = 0; t < T->np[KTGT]; ++t)
            if (tgt_ctr[t] < 0)
                for (int b = T->owner[KTGT][t]; b >= 0; b = T->parent[b])
                    if (p_hi > best[b]) best[b] = p_hi;
    for (int b = 0; b < nb; ++b) p_out[b] = best[b] >= 0 ? best[b] : p_default;
    free(best);
}

/*
 * Four inputs of the order network per QBX center c (input order), b the box owning c:
 *   feat[4c]   = log2(r_c / |b|)                        (expansion radius relative to the box)
 *   feat[4c+1] = level(b) / 8                           (box size: |b| = |root| 2^-level)
 *   feat[4c+2] = (|c - c_b|_2 + r_c) / |b|              (how far the expansion ball reaches from the
 *                                                        box center, where the box local is expanded)
 *   feat[4c+3] = log10(s_near / s_max + 1e-12)          (near-field source strength)
 * with the source strength |w sigma| + |w mu n|_2, s_near its largest value over the sources of the
 * List 1 boxes of b and s_max its largest value over all sources (0 for a zero density).  Computed in
 * double precision and rounded to float.  sigma or mu may be NULL.
 */
void orc_center_features(const otree *T, const olists *Ls, const double *w, const double *sigma, const double *mu,
                         const double *nrm, const double *cxyz, const double *cr, float *feat)
{
    int ns = T->np[KSRC], nc = T->np[KCTR];
    double *str = malloc(sizeof(double) * (ns > 0 ? ns : 1));
    double smax = 0.0;
    for (int j = 0; j < ns; ++j) {
        double q = sigma ? w[j] * sigma[j] : 0.0, v = fabs(q);
        if (mu) {
            double a = w[j] * mu[j], dx = a * nrm[j], dy = a * nrm[ns + j], dz = a * nrm[2 * ns + j];
            v += sqrt(dx * dx + dy * dy + dz * dz);
        }
        str[j] = v;
        if (v > smax) smax = v;
    }
    for (int ci = 0; ci < nc; ++ci) {
        int b = T->owner[KCTR][ci];
        double x[3], r = cr[ci];
        get_pt(cxyz, nc, ci, x);
        double dx = x[0] - T->cen[3 * b], dy = x[1] - T->cen[3 * b + 1], dz = x[2] - T->cen[3 * b + 2];
        double snear = 0.0;
        for (int e = Ls->start[L_U][b]; e < Ls->start[L_U][b + 1]; ++e) {
            int d = Ls->idx[L_U][e];
            for (int k = T->own_start[KSRC][d]; k < T->own_start[KSRC][d + 1]; ++k) {
                double v = str[T->own_idx[KSRC][k]];
                if (v > snear) snear = v;
            }
        }
        feat[4 * ci] = (float)log2(r / T->hw[b]);
        feat[4 * ci + 1] = (float)(T->level[b] / 8.0);
        feat[4 * ci + 2] = (float)((sqrt(dx * dx + dy * dy + dz * dz) + r) / T->hw[b]);
        feat[4 * ci + 3] = (float)log10(snear / (smax > 0.0 ? smax : 1e-300) + 1e-12);
    }
    free(str);
}

/*
 * Judge and fallback of learned orders: every target t with |res[t] - judge[t]| > tol (NaN counts)
 * raises the QBX order of its center (tgt_ctr[t] >= 0) to q_fix, and the local-expansion order of
 * the box owning that center (or the point target) and of every box above it to p_fix.  q and pb are
 * updated in place; returns the number of targets that missed.
 */
int orc_orders_fallback(const otree *T, const double *res, const double *judge, const int *tgt_ctr, double tol,
                        int q_fix, int p_fix, int *q, int *pb)
{
    int raised = 0;
    for (int t = 0; t < T->np[KTGT]; ++t) {
        if (fabs(res[t] - judge[t]) <= tol) continue;
        ++raised;
        int b;
        if (tgt_ctr[t] >= 0) {
            q[tgt_ctr[t]] = q_fix;
            b = T->owner[KCTR][tgt_ctr[t]];
        } else {
            b = T->owner[KTGT][t];
        }
        for (; b >= 0; b = T->parent[b]) pb[b] = p_fix;
    }
    return raised;
}

/* ------------------------------------------------------------------------ */
/* target association (Section 3.4, Algorithm 3) with area queries           */
/* (Appendix A, Algorithm 5)                                                  */
/* ------------------------------------------------------------------------ */

/* |x - y|_2 as sqrt(dx^2 + dy^2 + dz^2), summed in that order */
static double dist3(const double x[3], const double y[3])
{
    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* a peer box p of b (Algorithm 5): p is b or adjacent to b, and |p| >= |b| */
static int peer_like(const otree *T, int p, int b, int Lf)
{
    return T->level[p] <= T->level[b] && (p == b || adjacent(T, p, b, Lf));
}

static void leaves_meeting_cube(const otree *T, int p, const double c[3], double r, ivec *out, char *seen)
{
    for (int d = 0; d < 3; ++d)
        if (fabs(c[d] - T->cen[3 * p + d]) > r + T->hw[p]) return;  /* closed cubes do not meet */
    if (is_leaf(T, p)) {
        if (!seen[p]) { seen[p] = 1; iv_push(out, p); }
        return;
    }
    for (int o = 0; o < 8; ++o)
        if (T->child[8 * p + o] >= 0) leaves_meeting_cube(T, T->child[8 * p + o], c, r, out, seen);
}

/*
 * Area query (Algorithm 5): the leaf boxes that meet the closed cube of half side r around c.
 * Guiding box: from the root, descend to the child containing c while |b| >= r (the first box with
 * |b| < r <= 2|b|), or stop where no child contains c.  Then every leaf descendant of every peer of
 * the guiding box is tested against the cube.  `seen` (n_boxes bytes, zero) is restored on return.
 */
static void area_query(const otree *T, const double c[3], double r, ivec *out, char *seen)
{
    int Lf = finest_level(T), b = 0;
    out->n = 0;
    for (;;) {
        double h = T->hw[b];
        if ((h < r && r <= 2.0 * h) || r > 2.0 * h) break;
        int ch = T->child[8 * b + octant(c, &T->cen[3 * b])];
        if (ch < 0) break;
        b = ch;
    }
    for (int p = 0; p < T->nb; ++p) {
        if (!peer_like(T, p, b, Lf)) continue;
        int child_peer = 0;
        for (int o = 0; o < 8 && !child_peer; ++o) {
            int ch = T->child[8 * p + o];
            if (ch >= 0 && peer_like(T, ch, b, Lf)) child_peer = 1;
        }
        if (!child_peer) leaves_meeting_cube(T, p, c, r, out, seen);
    }
    for (int i = 0; i < out->n; ++i) seen[out->v[i]] = 0;
}

/*
 * Algorithm 3.  Stage 1: an area query of radius rdanger[s] around every source s marks the targets t
 * with |t - s| <= rdanger[s] as endangered.  Stage 2: an area query of radius r_c (1 + eps) around every
 * center c (in index order) associates an endangered target t to c when |t - c| <= r_c (1 + eps), c lies
 * on t's preferred side, and c is strictly closer than any center before it (ties keep the lower index).
 * The preferred side of t is +1 if (t - s*) . n(s*) > 0 and -1 otherwise, s* the source nearest to t
 * (lowest index among equals); with snrm == NULL (no side preference) every center qualifies.  Stage 3:
 * endangered targets left without a center are flagged.  Outputs in input order: tgt_ctr[t] (center or
 * -1) and flagged[t] (0/1).  Targets must be the tree's targets, in input order.
 */
void orc_assoc_targets(const otree *T, const double *sxyz, const double *rdanger, const double *snrm,
                       const double *cxyz, const double *cr, const signed char *cside, const double *txyz,
                       double eps, int *tgt_ctr, int *flagged)
{
    int ns = T->np[KSRC], nc = T->np[KCTR], nt = T->np[KTGT];
    char *seen = calloc(T->nb > 0 ? T->nb : 1, 1);
    char *endangered = calloc(nt > 0 ? nt : 1, 1);
    double *best = malloc(sizeof(double) * (nt > 0 ? nt : 1));
    ivec leaves = {0};
    double x[3], y[3];
    for (int t = 0; t < nt; ++t) { tgt_ctr[t] = -1; flagged[t] = 0; best[t] = INFINITY; }
    /* Stage 1 */
    for (int s = 0; s < ns; ++s) {
        get_pt(sxyz, ns, s, x);
        area_query(T, x, rdanger[s], &leaves, seen);
        for (int i = 0; i < leaves.n; ++i) {
            int l = leaves.v[i];
            for (int k = T->own_start[KTGT][l]; k < T->own_start[KTGT][l + 1]; ++k) {
                int t = T->own_idx[KTGT][k];
                get_pt(txyz, nt, t, y);
                if (dist3(y, x) <= rdanger[s]) endangered[t] = 1;
            }
        }
    }
    /* preferred sides: nearest source by brute force */
    signed char *side = calloc(nt > 0 ? nt : 1, 1);
    if (snrm)
        for (int t = 0; t < nt; ++t) {
            if (!endangered[t]) continue;
            get_pt(txyz, nt, t, y);
            int sb = -1;
            double db = INFINITY;
            for (int s = 0; s < ns; ++s) {
                get_pt(sxyz, ns, s, x);
                double dd = dist3(y, x);
                if (dd < db) { db = dd; sb = s; }
            }
            get_pt(sxyz, ns, sb, x);
            double dot = (y[0] - x[0]) * snrm[sb] + (y[1] - x[1]) * snrm[ns + sb];
            dot = dot + (y[2] - x[2]) * snrm[2 * ns + sb];
            side[t] = dot > 0.0 ? 1 : -1;
        }
    /* Stage 2 */
    for (int c = 0; c < nc; ++c) {
        get_pt(cxyz, nc, c, x);
        double rr = cr[c] * (1.0 + eps);
        area_query(T, x, rr, &leaves, seen);
        for (int i = 0; i < leaves.n; ++i) {
            int l = leaves.v[i];
            for (int k = T->own_start[KTGT][l]; k < T->own_start[KTGT][l + 1]; ++k) {
                int t = T->own_idx[KTGT][k];
                if (!endangered[t]) continue;
                if (snrm && cside[c] != side[t]) continue;
                get_pt(txyz, nt, t, y);
                double dd = dist3(y, x);
                if (dd <= rr && dd < best[t]) { best[t] = dd; tgt_ctr[t] = c; }
            }
        }
    }
    /* Stage 3 */
    for (int t = 0; t < nt; ++t) flagged[t] = endangered[t] && tgt_ctr[t] < 0;
    free(seen); free(endangered); free(best); free(side); free(leaves.v);
}

/* ------------------------------------------------------------------------ */
/* refinement marks of the geometry processing (Section 3.2 and 3.3)        */
/* ------------------------------------------------------------------------ */

/*
 * The tests that decide which elements Algorithms 1 and 2 bisect, as their definitions read,
 * over all (center, source) pairs (no tree):
 *  which = 0, Algorithm 1 (interfering source geometry, Section 3.2): the element elem[i] that
 *    spawned center i is marked if some source s has |c_i - s| < (1 - eps) r_i, eps the
 *    disturbance tolerance (0.025 in the paper);
 *  which = 1, Algorithm 2 (quadrature resolution, Section 3.3): the element elem[j] of source j is
 *    marked if some center c has |c - s_j| <= 0.5 (3/4) eta_k = 0.375 eta_k, k = elem[j].
 * marks[n_elem] receives 0 or 1.
 */
void orc_refine_marks(int which, const double *sxyz, int ns, const double *cxyz, const double *cr, int nc,
                      const int *elem, const double *eta, int n_elem, double eps, unsigned char *marks)
{
    double x[3], y[3];
    memset(marks, 0, (size_t)n_elem);
    if (which == 0) {
        for (int i = 0; i < nc; ++i) {
            get_pt(cxyz, nc, i, x);
            double rad = (1.0 - eps) * cr[i];
            for (int j = 0; j < ns && !marks[elem[i]]; ++j) {
                get_pt(sxyz, ns, j, y);
                if (dist3(x, y) < rad) marks[elem[i]] = 1;
            }
        }
    } else {
        for (int j = 0; j < ns; ++j) {
            get_pt(sxyz, ns, j, y);
            double rad = 0.375 * eta[elem[j]];
            for (int i = 0; i < nc && !marks[elem[j]]; ++i) {
                get_pt(cxyz, nc, i, x);
                if (dist3(x, y) <= rad) marks[elem[j]] = 1;
            }
        }
    }
}
