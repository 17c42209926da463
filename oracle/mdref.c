/*
 * mdref.c -- CPU oracle for multiple-double least squares.
 * TEST INFRASTRUCTURE ONLY (see mdref.h): never part of the product path.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math).
 *
 * Multiple-double arithmetic is defined here from first principles rather
 * than by an error-free-transform algorithm: every operand limb is split into
 * an integer significand and a power of two, sums and products are formed
 * EXACTLY in a wide fixed-point accumulator (two nonnegative big integers, a
 * positive part and a negative part), and the exact value is then rounded to
 * p doubles greedily -- each limb is the double nearest to what is left.
 * That is the plain meaning of "a multiple double number is an unevaluated
 * sum of doubles" (arXiv 2110.08375, Section 1.1); the result has the
 * property |x_{i+1}| <= ulp(x_i)/2.
 */
#include "mdref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXP 8

/* ------------------------------------------------------------------------
 * Exact fixed-point accumulator.
 * Bit k of word w has weight 2^(64*w + k + ACC_EMIN).  Two magnitudes are
 * kept (pos, neg); the value is pos - neg.  Range: 2^ACC_EMIN .. 2^2023.
 * ---------------------------------------------------------------------- */
#define ACC_W 66
#define ACC_EMIN (-2200)

typedef struct {
    uint64_t pos[ACC_W + 3];
    uint64_t neg[ACC_W + 3];
    int lo, hi; /* dirty word range (inclusive) */
} acc_t;

typedef struct {
    uint64_t c[7];
} cnt_t;

static int g_threads = 1;
static cnt_t g_cnt;

static void acc_init(acc_t *a) {
    memset(a, 0, sizeof(*a));
    a->lo = ACC_W;
    a->hi = -1;
}

static void acc_clear(acc_t *a) {
    if (a->hi >= a->lo) {
        size_t nb = (size_t)(a->hi - a->lo + 1) * sizeof(uint64_t);
        memset(a->pos + a->lo, 0, nb);
        memset(a->neg + a->lo, 0, nb);
    }
    a->lo = ACC_W;
    a->hi = -1;
}

/* adds mant * 2^(bitpos + ACC_EMIN) to magnitude x, mant < 2^107 */
static void mag_add(acc_t *a, uint64_t *x, int64_t bitpos, unsigned __int128 mant) {
    if (mant == 0) return;
    if (bitpos < 0 || bitpos / 64 + 3 >= ACC_W) abort(); /* outside the oracle's domain */
    int wi = (int)(bitpos >> 6), sh = (int)(bitpos & 63);
    uint64_t mlo = (uint64_t)mant, mhi = (uint64_t)(mant >> 64);
    uint64_t w0, w1, w2;
    if (sh == 0) {
        w0 = mlo; w1 = mhi; w2 = 0;
    } else {
        w0 = mlo << sh;
        w1 = (mlo >> (64 - sh)) | (mhi << sh);
        w2 = mhi >> (64 - sh);
    }
    uint64_t add[3] = {w0, w1, w2};
    unsigned carry = 0;
    int k = wi;
    for (int t = 0; t < 3; t++, k++) {
        uint64_t old = x[k];
        uint64_t s = old + add[t];
        unsigned c1 = s < old;
        uint64_t s2 = s + carry;
        unsigned c2 = s2 < s;
        x[k] = s2;
        carry = c1 | c2;
    }
    while (carry) {
        if (k >= ACC_W + 3) abort();
        x[k] += 1;
        carry = (x[k] == 0);
        k++;
    }
    if (wi < a->lo) a->lo = wi;
    if (k - 1 > a->hi) a->hi = k - 1;
    if (wi + 2 > a->hi) a->hi = wi + 2;
}

/* splits a finite nonzero double into (significand, exponent): x = +-m * 2^e */
static void split_double(double x, uint64_t *m, int *e, int *neg) {
    int ex;
    double f = frexp(fabs(x), &ex); /* f in [0.5, 1) */
    *m = (uint64_t)ldexp(f, 53);
    *e = ex - 53;
    *neg = x < 0;
}

static void acc_add_double(acc_t *a, double x) {
    if (x == 0.0) return;
    uint64_t m; int e, ng;
    split_double(x, &m, &e, &ng);
    mag_add(a, ng ? a->neg : a->pos, (int64_t)e - ACC_EMIN, (unsigned __int128)m);
}

/* adds the exact product x*y (106-bit significand) */
static void acc_add_prod(acc_t *a, double x, double y) {
    if (x == 0.0 || y == 0.0) return;
    uint64_t mx, my; int ex, ey, nx, ny;
    split_double(x, &mx, &ex, &nx);
    split_double(y, &my, &ey, &ny);
    unsigned __int128 m = (unsigned __int128)mx * my;
    mag_add(a, (nx ^ ny) ? a->neg : a->pos, (int64_t)ex + ey - ACC_EMIN, m);
}

/* bits [s, s+63] of the magnitude D (bits below 0 read as zero) */
static uint64_t get_bits64(const uint64_t *D, int nw, int64_t s) {
    if (s < 0) {
        if (s <= -64) return 0;
        return get_bits64(D, nw, 0) << (-s);
    }
    int64_t wi = s >> 6;
    int sh = (int)(s & 63);
    if (wi >= nw) return 0;
    uint64_t v = D[wi] >> sh;
    if (sh && wi + 1 < nw) v |= D[wi + 1] << (64 - sh);
    return v;
}

/* any bit set in [0, s] ? */
static int any_bits_upto(const uint64_t *D, int64_t s) {
    if (s < 0) return 0;
    int64_t wi = s >> 6;
    for (int64_t k = 0; k < wi; k++)
        if (D[k]) return 1;
    int sh = (int)(s & 63);
    uint64_t mask = (sh == 63) ? ~(uint64_t)0 : (((uint64_t)1 << (sh + 1)) - 1);
    return (D[wi] & mask) != 0;
}

/* Rounds the exact value pos - neg to the nearest double (ties to even),
 * removes that double from the accumulator, and returns it. */
static double acc_take_nearest(acc_t *a) {
    if (a->hi < a->lo) return 0.0;
    int top = a->hi;
    int bot = a->lo;
    /* compare magnitudes from the top */
    int sign = 0;
    for (int k = top; k >= bot; k--) {
        if (a->pos[k] != a->neg[k]) {
            sign = a->pos[k] > a->neg[k] ? 1 : -1;
            break;
        }
    }
    if (sign == 0) return 0.0;
    const uint64_t *big = sign > 0 ? a->pos : a->neg;
    const uint64_t *sml = sign > 0 ? a->neg : a->pos;
    uint64_t D[ACC_W + 3];
    memset(D, 0, sizeof(D));
    unsigned borrow = 0;
    for (int k = bot; k <= top; k++) {
        uint64_t x = big[k], y = sml[k];
        uint64_t d = x - y;
        unsigned b1 = x < y;
        uint64_t d2 = d - borrow;
        unsigned b2 = d < (uint64_t)borrow;
        D[k] = d2;
        borrow = b1 | b2;
    }
    int64_t t = -1;
    for (int k = top; k >= bot; k--) {
        if (D[k]) {
            t = (int64_t)k * 64 + 63 - __builtin_clzll(D[k]);
            break;
        }
    }
    if (t < 0) return 0.0;
    uint64_t m = get_bits64(D, top + 1, t - 52) & (((uint64_t)1 << 53) - 1);
    int rbit = (t - 53 >= 0) ? (int)((get_bits64(D, top + 1, t - 53)) & 1) : 0;
    int sticky = any_bits_upto(D, t - 54);
    if (rbit && (sticky || (m & 1))) m++;
    double v = ldexp((double)m, (int)(t - 52 + ACC_EMIN));
    if (sign < 0) v = -v;
    /* subtract v exactly: add its magnitude to the opposite side */
    acc_add_double(a, -v);
    return v;
}

static void acc_round_to(acc_t *a, int p, double *out) {
    for (int k = 0; k < p; k++) out[k] = acc_take_nearest(a);
}

/* ------------------------------------------------------------------------
 * Scalar md operations (p contiguous limbs).
 * ---------------------------------------------------------------------- */

static void md_zero(int p, double *c) {
    for (int k = 0; k < p; k++) c[k] = 0.0;
}

static int md_is_zero(int p, const double *a) {
    for (int k = 0; k < p; k++)
        if (a[k] != 0.0) return 0;
    return 1;
}

static void md_copy(int p, const double *a, double *c) {
    for (int k = 0; k < p; k++) c[k] = a[k];
}

static void md_neg(int p, const double *a, double *c) {
    for (int k = 0; k < p; k++) c[k] = -a[k];
}

static void md_norm(acc_t *A, int p, const double *a, double *c) {
    acc_clear(A);
    for (int k = 0; k < p; k++) acc_add_double(A, a[k]);
    acc_round_to(A, p, c);
}

static void md_add(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    acc_clear(A);
    for (int k = 0; k < p; k++) acc_add_double(A, a[k]);
    for (int k = 0; k < p; k++) acc_add_double(A, b[k]);
    acc_round_to(A, p, c);
    K->c[0]++;
}

static void md_sub(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    acc_clear(A);
    for (int k = 0; k < p; k++) acc_add_double(A, a[k]);
    for (int k = 0; k < p; k++) acc_add_double(A, -b[k]);
    acc_round_to(A, p, c);
    K->c[0]++;
}

static void md_mul(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) acc_add_prod(A, a[i], b[j]);
    acc_round_to(A, p, c);
    K->c[1]++;
}

/* Long division: quotient digits q_k = RN(r_k) / b0 with the exact remainder
 * r_{k+1} = r_k - q_k * b kept in the accumulator; p+2 digits, then the
 * digits are summed exactly and rounded to p limbs. */
static void md_div_nocount(acc_t *A, int p, const double *a, const double *b, double *c) {
    double q[MAXP + 2];
    int nq = 0;
    acc_clear(A);
    for (int k = 0; k < p; k++) acc_add_double(A, a[k]);
    for (int d = 0; d < p + 2; d++) {
        /* leading double of the remainder, without consuming it */
        acc_t T = *A;
        double r = acc_take_nearest(&T);
        if (r == 0.0) break;
        double qd = r / b[0];
        q[nq++] = qd;
        for (int k = 0; k < p; k++) acc_add_prod(A, -qd, b[k]);
    }
    acc_clear(A);
    for (int d = 0; d < nq; d++) acc_add_double(A, q[d]);
    acc_round_to(A, p, c);
}

static void md_div(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    md_div_nocount(A, p, a, b, c);
    K->c[2]++;
}

/* Newton's iteration x <- (x + a/x)/2 from the double square root of the
 * leading limb; each step is md arithmetic rounded to p limbs. */
static void md_sqrt(acc_t *A, cnt_t *K, int p, const double *a, double *c) {
    K->c[3]++;
    if (md_is_zero(p, a)) {
        md_zero(p, c);
        return;
    }
    if (a[0] < 0) {
        for (int k = 0; k < p; k++) c[k] = NAN;
        return;
    }
    double x[MAXP], q[MAXP], s[MAXP];
    md_zero(p, x);
    x[0] = sqrt(a[0]);
    int iters = (p == 2) ? 3 : (p == 4) ? 4 : 5;
    for (int it = 0; it < iters; it++) {
        md_div_nocount(A, p, a, x, q);
        acc_clear(A);
        for (int k = 0; k < p; k++) acc_add_double(A, x[k]);
        for (int k = 0; k < p; k++) acc_add_double(A, q[k]);
        acc_round_to(A, p, s);
        for (int k = 0; k < p; k++) x[k] = 0.5 * s[k];
    }
    md_copy(p, x, c);
}

/* ------------------------------------------------------------------------
 * Exported scalar interface
 * ---------------------------------------------------------------------- */
int mdref_version(void) { return 1; }

void mdref_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int mdref_get_threads(void) { return g_threads; }

void mdref_two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bb = x - a;
    double err = (a - (x - bb)) + (b - bb);
    *s = x;
    *e = err;
}

void mdref_two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

void mdref_normalize(int p, const double *a, double *c) {
    acc_t A; acc_init(&A);
    md_norm(&A, p, a, c);
}
void mdref_add(int p, const double *a, const double *b, double *c) {
    acc_t A; acc_init(&A);
    md_add(&A, &g_cnt, p, a, b, c);
}
void mdref_sub(int p, const double *a, const double *b, double *c) {
    acc_t A; acc_init(&A);
    md_sub(&A, &g_cnt, p, a, b, c);
}
void mdref_mul(int p, const double *a, const double *b, double *c) {
    acc_t A; acc_init(&A);
    md_mul(&A, &g_cnt, p, a, b, c);
}
void mdref_div(int p, const double *a, const double *b, double *c) {
    acc_t A; acc_init(&A);
    md_div(&A, &g_cnt, p, a, b, c);
}
void mdref_sqrt(int p, const double *a, double *c) {
    acc_t A; acc_init(&A);
    md_sqrt(&A, &g_cnt, p, a, c);
}
double mdref_diff(int p, const double *a, const double *b) {
    acc_t A; acc_init(&A);
    for (int k = 0; k < p; k++) acc_add_double(&A, a[k]);
    for (int k = 0; k < p; k++) acc_add_double(&A, -b[k]);
    return acc_take_nearest(&A);
}

void mdref_diff_array(int p, int64_t count, const double *a, int64_t psa, const double *b,
                      int64_t psb, double *out) {
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        acc_t A; acc_init(&A);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < count; i++) {
            acc_clear(&A);
            for (int k = 0; k < p; k++) acc_add_double(&A, a[(size_t)k * psa + i]);
            for (int k = 0; k < p; k++) acc_add_double(&A, -b[(size_t)k * psb + i]);
            out[i] = acc_take_nearest(&A);
        }
    }
}

void mdref_reset_counts(void) { memset(&g_cnt, 0, sizeof(g_cnt)); }
void mdref_get_counts(uint64_t out[7]) {
    for (int k = 0; k < 7; k++) out[k] = g_cnt.c[k];
}

static void cnt_merge(const cnt_t *local) {
#ifdef _OPENMP
#pragma omp critical(mdref_cnt)
#endif
    {
        for (int k = 0; k < 7; k++) g_cnt.c[k] += local->c[k];
    }
}

/* ------------------------------------------------------------------------
 * Element-major work matrices: entry (i, j) of an r x c matrix occupies
 * p contiguous doubles at ((j * r) + i) * p.
 * ---------------------------------------------------------------------- */
#define EL(M, r, i, j, p) ((M) + (((size_t)(j) * (size_t)(r)) + (size_t)(i)) * (size_t)(p))

static double *load_planar(int p, int64_t rows, int64_t cols, const double *X, int64_t ld,
                           int64_t ps) {
    double *M = (double *)malloc(sizeof(double) * (size_t)p * rows * cols + 8);
    acc_t A; acc_init(&A);
    double tmp[MAXP];
    for (int64_t j = 0; j < cols; j++)
        for (int64_t i = 0; i < rows; i++) {
            for (int k = 0; k < p; k++) tmp[k] = X[(size_t)k * ps + (size_t)j * ld + i];
            md_norm(&A, p, tmp, EL(M, rows, i, j, p));
        }
    return M;
}

static void store_planar(int p, int64_t rows, int64_t cols, const double *M, double *X,
                         int64_t ld, int64_t ps) {
    for (int64_t j = 0; j < cols; j++)
        for (int64_t i = 0; i < rows; i++)
            for (int k = 0; k < p; k++)
                X[(size_t)k * ps + (size_t)j * ld + i] = EL(M, rows, i, j, p)[k];
}

/* Householder vector of x (length L) following Golub & Van Loan Alg. 5.1.1:
 * v(0) = 1, beta = 2/(v^T v), (I - beta v v^T) x = ||x|| e1.  v[1..L-1] and
 * beta are written; *rjj receives the new diagonal entry (>= 0). */
static void house(acc_t *A, cnt_t *K, int p, int64_t L, const double *x, double *v,
                  double *beta, double *rjj) {
    double sigma[MAXP], t[MAXP], mu[MAXP], v0[MAXP], v0sq[MAXP], den[MAXP], q[MAXP];
    md_zero(p, sigma);
    for (int64_t i = 1; i < L; i++) {
        md_mul(A, K, p, x + i * p, x + i * p, t);
        md_add(A, K, p, sigma, t, sigma);
    }
    md_zero(p, v);
    v[0] = 1.0;
    if (md_is_zero(p, sigma)) {
        for (int64_t i = 1; i < L; i++) md_zero(p, v + i * p);
        md_zero(p, beta);
        if (x[0] >= 0.0) { /* x is already +||x|| e1 */
            md_copy(p, x, rjj);
            K->c[5]++;
        } else { /* reflect e1: x -> -x */
            beta[0] = 2.0;
            md_neg(p, x, rjj);
            K->c[6]++;
        }
        return;
    }
    md_mul(A, K, p, x, x, t);
    md_add(A, K, p, t, sigma, t);
    md_sqrt(A, K, p, t, mu);
    if (x[0] <= 0.0) {
        md_sub(A, K, p, x, mu, v0);
    } else { /* v0 = -sigma / (x0 + mu), free of cancellation */
        md_add(A, K, p, x, mu, t);
        md_div(A, K, p, sigma, t, q);
        md_neg(p, q, v0);
        K->c[4]++;
    }
    md_mul(A, K, p, v0, v0, v0sq);
    md_add(A, K, p, sigma, v0sq, den);
    md_div(A, K, p, v0sq, den, q);
    for (int k = 0; k < p; k++) beta[k] = 2.0 * q[k];
    for (int64_t i = 1; i < L; i++) md_div(A, K, p, x + i * p, v0, v + i * p);
    md_copy(p, mu, rjj);
}

/* a <- (I - beta v v^T) a for one column of length L */
static void apply_reflector(acc_t *A, cnt_t *K, int p, int64_t L, const double *v,
                            const double *beta, double *a) {
    double s[MAXP], t[MAXP], w[MAXP];
    md_zero(p, s);
    for (int64_t i = 0; i < L; i++) {
        md_mul(A, K, p, v + i * p, a + i * p, t);
        md_add(A, K, p, s, t, s);
    }
    md_mul(A, K, p, beta, s, w);
    for (int64_t i = 0; i < L; i++) {
        md_mul(A, K, p, v + i * p, w, t);
        md_sub(A, K, p, a + i * p, t, a + i * p);
    }
}

/* applies H_j to columns [c0, c1) of the element-major matrix M (rows r),
 * rows j..r-1, in parallel over columns */
static void apply_to_columns(int p, int64_t r, int64_t j, const double *v, const double *beta,
                             double *M, int64_t c0, int64_t c1) {
    if (c1 <= c0 || md_is_zero(p, beta)) return;
    int64_t L = r - j;
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        acc_t A; acc_init(&A);
        cnt_t K; memset(&K, 0, sizeof(K));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t c = c0; c < c1; c++) apply_reflector(&A, &K, p, L, v, beta, EL(M, r, j, c, p));
        cnt_merge(&K);
    }
}

/* Unblocked QR of the element-major m x n matrix M (in place).  V (m x n)
 * receives the Householder vectors (rows j.. of column j), B the betas.
 * extra columns [n, n + nextra) of M (e.g. a right-hand side) are
 * transformed along with the trailing columns. */
static void qr_unblocked(int p, int64_t m, int64_t n, int64_t nextra, double *M, double *V,
                         double *B) {
    acc_t A; acc_init(&A);
    for (int64_t j = 0; j < n; j++) {
        int64_t L = m - j;
        double *x = EL(M, m, j, j, p);
        double *v = EL(V, m, j, j, p);
        double rjj[MAXP];
        house(&A, &g_cnt, p, L, x, v, B + j * p, rjj);
        apply_to_columns(p, m, j, v, B + j * p, M, j + 1, n + nextra);
        md_copy(p, rjj, x);
        for (int64_t i = 1; i < L; i++) md_zero(p, x + i * p);
    }
}

int mdref_qr(int p, int64_t m, int64_t n, double *Ap, int64_t lda, int64_t psa, double *Qp,
             int64_t ldq, int64_t psq, double *beta) {
    if (!(p == 2 || p == 4 || p == 8) || m < n || n < 0 || !Ap || lda < m) return -1;
    if (Qp && ldq < m) return -1;
    double *M = load_planar(p, m, n, Ap, lda, psa);
    double *V = (double *)calloc((size_t)p * m * (n ? n : 1), sizeof(double));
    double *B = (double *)calloc((size_t)p * (n ? n : 1), sizeof(double));
    qr_unblocked(p, m, n, 0, M, V, B);
    store_planar(p, m, n, M, Ap, lda, psa);
    if (beta)
        for (int64_t j = 0; j < n; j++)
            for (int k = 0; k < p; k++) beta[(size_t)k * n + j] = B[j * p + k];
    if (Qp) {
        /* backward accumulation: Q = H_0 (H_1 (... (H_{n-1} I))) */
        double *Qm = (double *)calloc((size_t)p * m * (m ? m : 1), sizeof(double));
        for (int64_t i = 0; i < m; i++) EL(Qm, m, i, i, p)[0] = 1.0;
        for (int64_t j = n - 1; j >= 0; j--)
            apply_to_columns(p, m, j, EL(V, m, j, j, p), B + j * p, Qm, j, m);
        store_planar(p, m, m, Qm, Qp, ldq, psq);
        free(Qm);
    }
    free(M);
    free(V);
    free(B);
    return 0;
}

static int backsub_em(acc_t *A, int p, int64_t n, const double *R, int64_t rrows,
                      const double *y, double *x) {
    double s[MAXP], t[MAXP];
    for (int64_t i = n - 1; i >= 0; i--) {
        md_copy(p, y + i * p, s);
        for (int64_t j = i + 1; j < n; j++) {
            md_mul(A, &g_cnt, p, EL(R, rrows, i, j, p), x + j * p, t);
            md_sub(A, &g_cnt, p, s, t, s);
        }
        const double *rii = EL(R, rrows, i, i, p);
        if (md_is_zero(p, rii)) return -2;
        md_div(A, &g_cnt, p, s, rii, x + i * p);
    }
    return 0;
}

int mdref_backsub(int p, int64_t n, const double *Rp, int64_t ldr, int64_t psr,
                  const double *yp, double *xp) {
    if (!(p == 2 || p == 4 || p == 8) || n < 0 || ldr < n) return -1;
    double *R = load_planar(p, n, n, Rp, ldr, psr);
    double *y = load_planar(p, n, 1, yp, n, n);
    double *x = (double *)calloc((size_t)p * (n ? n : 1), sizeof(double));
    acc_t A; acc_init(&A);
    int rc = backsub_em(&A, p, n, R, n, y, x);
    store_planar(p, n, 1, x, xp, n, n);
    free(R); free(y); free(x);
    return rc;
}

int mdref_lstsq(int p, int64_t m, int64_t n, const double *Ap, int64_t lda, int64_t psa,
                const double *bp, double *xp) {
    if (!(p == 2 || p == 4 || p == 8) || m < n || n < 1 || lda < m) return -1;
    /* [A | b] as one element-major m x (n+1) matrix */
    double *M = (double *)malloc(sizeof(double) * (size_t)p * m * (n + 1));
    double *MA = load_planar(p, m, n, Ap, lda, psa);
    double *Mb = load_planar(p, m, 1, bp, m, m);
    memcpy(M, MA, sizeof(double) * (size_t)p * m * n);
    memcpy(M + (size_t)p * m * n, Mb, sizeof(double) * (size_t)p * m);
    free(MA); free(Mb);
    double *V = (double *)calloc((size_t)p * m * n, sizeof(double));
    double *B = (double *)calloc((size_t)p * n, sizeof(double));
    qr_unblocked(p, m, n, 1, M, V, B);
    double *x = (double *)calloc((size_t)p * n, sizeof(double));
    acc_t A; acc_init(&A);
    int rc = backsub_em(&A, p, n, M, m, EL(M, m, 0, n, p), x);
    store_planar(p, n, 1, x, xp, n, n);
    free(M); free(V); free(B); free(x);
    return rc;
}

void mdref_gemv(int p, int trans, int64_t m, int64_t n, const double *Ap, int64_t lda,
                int64_t psa, const double *xp, double *yp) {
    int64_t nx = trans ? m : n, ny = trans ? n : m;
    double *M = load_planar(p, m, n, Ap, lda, psa);
    double *x = load_planar(p, nx, 1, xp, nx, nx);
    double *y = (double *)calloc((size_t)p * (ny ? ny : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        acc_t A; acc_init(&A);
        cnt_t K; memset(&K, 0, sizeof(K));
        double t[MAXP];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t o = 0; o < ny; o++) {
            double *s = y + o * p;
            md_zero(p, s);
            for (int64_t k = 0; k < nx; k++) {
                const double *a = trans ? EL(M, m, k, o, p) : EL(M, m, o, k, p);
                md_mul(&A, &K, p, a, x + k * p, t);
                md_add(&A, &K, p, s, t, s);
            }
        }
        cnt_merge(&K);
    }
    store_planar(p, ny, 1, y, yp, ny, ny);
    free(M); free(x); free(y);
}

void mdref_gemm(int p, int64_t m, int64_t n, int64_t k, const double *Ap, int64_t lda,
                int64_t psa, const double *Bp, int64_t ldb, int64_t psb, double *Cp,
                int64_t ldc, int64_t psc) {
    double *MA = load_planar(p, m, k, Ap, lda, psa);
    double *MB = load_planar(p, k, n, Bp, ldb, psb);
    double *MC = (double *)calloc((size_t)p * ((m * n) > 0 ? (m * n) : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        acc_t A; acc_init(&A);
        cnt_t K; memset(&K, 0, sizeof(K));
        double t[MAXP];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < m; i++) {
                double *s = EL(MC, m, i, j, p);
                md_zero(p, s);
                for (int64_t l = 0; l < k; l++) {
                    md_mul(&A, &K, p, EL(MA, m, i, l, p), EL(MB, k, l, j, p), t);
                    md_add(&A, &K, p, s, t, s);
                }
            }
        cnt_merge(&K);
    }
    store_planar(p, m, n, MC, Cp, ldc, psc);
    free(MA); free(MB); free(MC);
}

/* ------------------------------------------------------------------------
 * Complex multiple doubles (the paper's remark in Section 3: on complex data
 * the transpose becomes the Hermitian transpose; real and imaginary parts
 * are kept separately, Section 2).  A complex md value is 2p contiguous
 * doubles in element-major work arrays: the p limbs of the real part, then
 * the p limbs of the imaginary part.  Each part of a sum or product is
 * formed exactly and rounded once.
 * ---------------------------------------------------------------------- */
#define ZEL(M, r, i, j, p) ((M) + (((size_t)(j) * (size_t)(r)) + (size_t)(i)) * (size_t)(2 * (p)))

static void z_zero(int p, double *c) { md_zero(2 * p, c); }

static void z_add(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    md_add(A, K, p, a, b, c);
    md_add(A, K, p, a + p, b + p, c + p);
}

static void z_sub(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    md_sub(A, K, p, a, b, c);
    md_sub(A, K, p, a + p, b + p, c + p);
}

/* c = (conj(a) if ca) * b, each part exact then rounded; c may alias a or b */
static void z_mul_opt(acc_t *A, cnt_t *K, int p, const double *a, int ca, const double *b, double *c) {
    double re[MAXP], im[MAXP];
    const double sa = ca ? -1.0 : 1.0;
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            acc_add_prod(A, a[i], b[j]);
            acc_add_prod(A, -sa * a[p + i], b[p + j]);
        }
    acc_round_to(A, p, re);
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            acc_add_prod(A, a[i], b[p + j]);
            acc_add_prod(A, sa * a[p + i], b[j]);
        }
    acc_round_to(A, p, im);
    md_copy(p, re, c);
    md_copy(p, im, c + p);
    K->c[1] += 4;
    K->c[0] += 2;
}

static void z_mul(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    z_mul_opt(A, K, p, a, 0, b, c);
}

/* |a|^2 = re^2 + im^2, exact then rounded (real, p limbs) */
static void z_abs2(acc_t *A, cnt_t *K, int p, const double *a, double *c) {
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            acc_add_prod(A, a[i], a[j]);
            acc_add_prod(A, a[p + i], a[p + j]);
        }
    acc_round_to(A, p, c);
    K->c[1] += 2;
    K->c[0] += 1;
}

/* a / b = (a conj(b)) / |b|^2: numerator and denominator each exact then
 * rounded, then two md divisions */
static void z_div(acc_t *A, cnt_t *K, int p, const double *a, const double *b, double *c) {
    double num[2 * MAXP], den[MAXP];
    double re[MAXP], im[MAXP];
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            acc_add_prod(A, a[i], b[j]);
            acc_add_prod(A, a[p + i], b[p + j]);
        }
    acc_round_to(A, p, num);
    acc_clear(A);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            acc_add_prod(A, a[p + i], b[j]);
            acc_add_prod(A, -a[i], b[p + j]);
        }
    acc_round_to(A, p, num + p);
    z_abs2(A, K, p, b, den);
    md_div(A, K, p, num, den, re);
    md_div(A, K, p, num + p, den, im);
    md_copy(p, re, c);
    md_copy(p, im, c + p);
}

static int z_is_zero(int p, const double *a) { return md_is_zero(2 * p, a); }

/* Complex Householder vector of x (length L): H = I - beta v v^H with v(0) = 1
 * and beta real, H x = rho e1 with rho = e^{i theta} ||x||, theta = arg x(0)
 * (theta = 0 when x(0) = 0).  With sigma = sum_{i>0} |x_i|^2,
 * mu = sqrt(|x0|^2 + sigma): v0 = x0 - rho = -e^{i theta} sigma / (|x0| + mu)
 * (no cancellation), v = x / v0, beta = 2 |v0|^2 / (sigma + |v0|^2).
 * sigma = 0: H = I (beta = 0, v = e1) and rho = x0.  This is Golub and Van
 * Loan's Alg. 5.1.1 with the sign of the real case replaced by the phase of
 * x0, so that H is Hermitian and the diagonal of R carries the phases of the
 * leading entries. */
static void zhouse(acc_t *A, cnt_t *K, int p, int64_t L, const double *x, double *v,
                   double *beta, double *rho) {
    double sigma[MAXP], t[MAXP], a2[MAXP], mu[MAXP], ax[MAXP], den[MAXP], q[MAXP];
    double v0[2 * MAXP], ph[2 * MAXP], v0a2[MAXP];
    md_zero(p, sigma);
    for (int64_t i = 1; i < L; i++) {
        z_abs2(A, K, p, x + i * 2 * p, t);
        md_add(A, K, p, sigma, t, sigma);
    }
    z_zero(p, v);
    v[0] = 1.0;
    if (md_is_zero(p, sigma)) {
        for (int64_t i = 1; i < L; i++) z_zero(p, v + i * 2 * p);
        md_zero(p, beta);
        md_copy(2 * p, x, rho);
        K->c[5]++;
        return;
    }
    z_abs2(A, K, p, x, a2);
    md_add(A, K, p, a2, sigma, t);
    md_sqrt(A, K, p, t, mu);
    /* phase e^{i theta} = x0 / |x0| (1 when x0 = 0) */
    z_zero(p, ph);
    if (md_is_zero(p, a2)) {
        ph[0] = 1.0;
        md_zero(p, ax);
    } else {
        md_sqrt(A, K, p, a2, ax);
        md_div(A, K, p, x, ax, ph);
        md_div(A, K, p, x + p, ax, ph + p);
    }
    /* v0 = -ph * sigma / (|x0| + mu) */
    md_add(A, K, p, ax, mu, den);
    md_div(A, K, p, sigma, den, q);
    md_mul(A, K, p, ph, q, v0);
    md_mul(A, K, p, ph + p, q, v0 + p);
    md_neg(2 * p, v0, v0);
    /* beta = 2 |v0|^2 / (sigma + |v0|^2) */
    z_abs2(A, K, p, v0, v0a2);
    md_add(A, K, p, sigma, v0a2, den);
    md_div(A, K, p, v0a2, den, q);
    for (int k = 0; k < p; k++) beta[k] = 2.0 * q[k];
    for (int64_t i = 1; i < L; i++) z_div(A, K, p, x + i * 2 * p, v0, v + i * 2 * p);
    /* rho = ph * mu */
    md_mul(A, K, p, ph, mu, rho);
    md_mul(A, K, p, ph + p, mu, rho + p);
}

/* a <- (I - beta v v^H) a for one column of length L */
static void zapply_reflector(acc_t *A, cnt_t *K, int p, int64_t L, const double *v,
                             const double *beta, double *a) {
    double s[2 * MAXP], t[2 * MAXP], w[2 * MAXP];
    z_zero(p, s);
    for (int64_t i = 0; i < L; i++) {
        z_mul_opt(A, K, p, v + i * 2 * p, 1, a + i * 2 * p, t); /* conj(v_i) a_i */
        z_add(A, K, p, s, t, s);
    }
    md_mul(A, K, p, beta, s, w);
    md_mul(A, K, p, beta, s + p, w + p);
    for (int64_t i = 0; i < L; i++) {
        z_mul(A, K, p, v + i * 2 * p, w, t);
        z_sub(A, K, p, a + i * 2 * p, t, a + i * 2 * p);
    }
}

static void zapply_to_columns(int p, int64_t r, int64_t j, const double *v, const double *beta,
                              double *M, int64_t c0, int64_t c1) {
    if (c1 <= c0 || md_is_zero(p, beta)) return;
    int64_t L = r - j;
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        acc_t A; acc_init(&A);
        cnt_t K; memset(&K, 0, sizeof(K));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t c = c0; c < c1; c++)
            zapply_reflector(&A, &K, p, L, v, beta, ZEL(M, r, j, c, p));
        cnt_merge(&K);
    }
}

static void zqr_unblocked(int p, int64_t m, int64_t n, int64_t nextra, double *M, double *V,
                          double *B) {
    acc_t A; acc_init(&A);
    for (int64_t j = 0; j < n; j++) {
        int64_t L = m - j;
        double *x = ZEL(M, m, j, j, p);
        double *v = ZEL(V, m, j, j, p);
        double rho[2 * MAXP];
        zhouse(&A, &g_cnt, p, L, x, v, B + j * p, rho);
        zapply_to_columns(p, m, j, v, B + j * p, M, j + 1, n + nextra);
        md_copy(2 * p, rho, x);
        for (int64_t i = 1; i < L; i++) z_zero(p, x + i * 2 * p);
    }
}

/* planar complex (re and im planes) <-> element-major complex */
static double *zload(int p, int64_t rows, int64_t cols, const double *Xr, const double *Xi,
                     int64_t ld, int64_t ps) {
    double *M = (double *)malloc(sizeof(double) * (size_t)2 * p * rows * (cols ? cols : 1) + 8);
    acc_t A; acc_init(&A);
    double tmp[MAXP];
    for (int64_t j = 0; j < cols; j++)
        for (int64_t i = 0; i < rows; i++) {
            for (int k = 0; k < p; k++) tmp[k] = Xr[(size_t)k * ps + (size_t)j * ld + i];
            md_norm(&A, p, tmp, ZEL(M, rows, i, j, p));
            for (int k = 0; k < p; k++) tmp[k] = Xi[(size_t)k * ps + (size_t)j * ld + i];
            md_norm(&A, p, tmp, ZEL(M, rows, i, j, p) + p);
        }
    return M;
}

static void zstore(int p, int64_t rows, int64_t cols, const double *M, double *Xr, double *Xi,
                   int64_t ld, int64_t ps) {
    for (int64_t j = 0; j < cols; j++)
        for (int64_t i = 0; i < rows; i++)
            for (int k = 0; k < p; k++) {
                Xr[(size_t)k * ps + (size_t)j * ld + i] = ZEL(M, rows, i, j, p)[k];
                Xi[(size_t)k * ps + (size_t)j * ld + i] = ZEL(M, rows, i, j, p)[p + k];
            }
}

int mdref_zqr(int p, int64_t m, int64_t n, double *Ar, double *Ai, int64_t lda, int64_t psa,
              double *Qr, double *Qi, int64_t ldq, int64_t psq, double *beta) {
    if (!(p == 2 || p == 4 || p == 8) || m < n || n < 0 || !Ar || !Ai || lda < m) return -1;
    if ((Qr || Qi) && (!Qr || !Qi || ldq < m)) return -1;
    double *M = zload(p, m, n, Ar, Ai, lda, psa);
    double *V = (double *)calloc((size_t)2 * p * m * (n ? n : 1), sizeof(double));
    double *B = (double *)calloc((size_t)p * (n ? n : 1), sizeof(double));
    zqr_unblocked(p, m, n, 0, M, V, B);
    zstore(p, m, n, M, Ar, Ai, lda, psa);
    if (beta)
        for (int64_t j = 0; j < n; j++)
            for (int k = 0; k < p; k++) beta[(size_t)k * n + j] = B[j * p + k];
    if (Qr) {
        /* backward accumulation: Q = H_0 (H_1 (... (H_{n-1} I))), each H_j Hermitian */
        double *Qm = (double *)calloc((size_t)2 * p * m * (m ? m : 1), sizeof(double));
        for (int64_t i = 0; i < m; i++) ZEL(Qm, m, i, i, p)[0] = 1.0;
        for (int64_t j = n - 1; j >= 0; j--)
            zapply_to_columns(p, m, j, ZEL(V, m, j, j, p), B + j * p, Qm, j, m);
        zstore(p, m, m, Qm, Qr, Qi, ldq, psq);
        free(Qm);
    }
    free(M); free(V); free(B);
    return 0;
}

static int zbacksub_em(acc_t *A, int p, int64_t n, const double *R, int64_t rrows,
                       const double *y, double *x) {
    double s[2 * MAXP], t[2 * MAXP];
    for (int64_t i = n - 1; i >= 0; i--) {
        md_copy(2 * p, y + i * 2 * p, s);
        for (int64_t j = i + 1; j < n; j++) {
            z_mul(A, &g_cnt, p, ZEL(R, rrows, i, j, p), x + j * 2 * p, t);
            z_sub(A, &g_cnt, p, s, t, s);
        }
        const double *rii = ZEL(R, rrows, i, i, p);
        if (z_is_zero(p, rii)) return -2;
        z_div(A, &g_cnt, p, s, rii, x + i * 2 * p);
    }
    return 0;
}

int mdref_zbacksub(int p, int64_t n, const double *Rr, const double *Ri, int64_t ldr, int64_t psr,
                   const double *yr, const double *yi, double *xr, double *xi) {
    if (!(p == 2 || p == 4 || p == 8) || n < 0 || ldr < n) return -1;
    double *R = zload(p, n, n, Rr, Ri, ldr, psr);
    double *y = zload(p, n, 1, yr, yi, n, n);
    double *x = (double *)calloc((size_t)2 * p * (n ? n : 1), sizeof(double));
    acc_t A; acc_init(&A);
    int rc = zbacksub_em(&A, p, n, R, n, y, x);
    zstore(p, n, 1, x, xr, xi, n, n);
    free(R); free(y); free(x);
    return rc;
}

int mdref_zlstsq(int p, int64_t m, int64_t n, const double *Ar, const double *Ai, int64_t lda,
                 int64_t psa, const double *br, const double *bi, double *xr, double *xi) {
    if (!(p == 2 || p == 4 || p == 8) || m < n || n < 1 || lda < m) return -1;
    double *M = (double *)malloc(sizeof(double) * (size_t)2 * p * m * (n + 1));
    double *MA = zload(p, m, n, Ar, Ai, lda, psa);
    double *Mb = zload(p, m, 1, br, bi, m, m);
    memcpy(M, MA, sizeof(double) * (size_t)2 * p * m * n);
    memcpy(M + (size_t)2 * p * m * n, Mb, sizeof(double) * (size_t)2 * p * m);
    free(MA); free(Mb);
    double *V = (double *)calloc((size_t)2 * p * m * n, sizeof(double));
    double *B = (double *)calloc((size_t)p * n, sizeof(double));
    zqr_unblocked(p, m, n, 1, M, V, B);
    double *x = (double *)calloc((size_t)2 * p * n, sizeof(double));
    acc_t A; acc_init(&A);
    int rc = zbacksub_em(&A, p, n, M, m, ZEL(M, m, 0, n, p), x);
    zstore(p, n, 1, x, xr, xi, n, n);
    free(M); free(V); free(B); free(x);
    return rc;
}
