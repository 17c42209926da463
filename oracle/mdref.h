/*
 * mdref -- the CPU oracle for multiple-double least squares.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library
 * (libmdls) never links, loads or calls it, and shares no code with it.
 *
 * What it computes (arXiv 2110.08375, "Least Squares on GPUs in Multiple
 * Double Precision"):
 *   - multiple-double numbers (Section 1.1): an unevaluated sum of p doubles,
 *     p = 2 (double double), 4 (quad double), 8 (octo double);
 *   - every md operation here is the EXACT result of the operation rounded to
 *     p limbs greedily: x0 = RN(v), x1 = RN(v - x0), ...  (add, sub, mul are
 *     exact before rounding; div uses a long division carried to p+2 quotient
 *     digits; sqrt uses Newton's iteration in md arithmetic);
 *   - unblocked Householder QR (Section 3, with the reflector sign convention
 *     of Golub & Van Loan Algorithm 5.1.1 that the paper cites), Q by backward
 *     accumulation, Q^T b, and plain back substitution (Section 2's problem
 *     U x = b solved row by row, without tile inversion);
 *   - least squares x = R^{-1} (Q^T b)  (Section 1: A = QR reduces Ax = b to
 *     Rx = Q^T b).
 *
 * Storage: limb-planar ("staggered", Section 2): plane l of a matrix holds
 * limb l of every entry, column-major with leading dimension ld; planes are
 * ps doubles apart.  Vectors: plane stride given by the caller.
 *
 * Domain: all limbs finite, with |limb| in [2^-1000, 2^1000] or zero.
 * Inputs are taken as the exact sum of their limbs and rounded to p limbs on
 * entry.
 */
#ifndef MDREF_H
#define MDREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int mdref_version(void);
void mdref_set_threads(int nthreads);
int mdref_get_threads(void);

/* error-free transforms (Knuth two-sum; product via fma) */
void mdref_two_sum(double a, double b, double *s, double *e);
void mdref_two_prod(double a, double b, double *p, double *e);

/* scalar md operations on p contiguous limbs */
void mdref_normalize(int p, const double *a, double *c);
void mdref_add(int p, const double *a, const double *b, double *c);
void mdref_sub(int p, const double *a, const double *b, double *c);
void mdref_mul(int p, const double *a, const double *b, double *c);
void mdref_div(int p, const double *a, const double *b, double *c);
void mdref_sqrt(int p, const double *a, double *c);
/* RN(a - b) as one double, exact before rounding (used for error norms) */
double mdref_diff(int p, const double *a, const double *b);

/* out[i] = RN(a_i - b_i) for count md values stored limb-planar with plane
 * strides psa, psb (exact before rounding). */
void mdref_diff_array(int p, int64_t count, const double *a, int64_t psa, const double *b,
                      int64_t psb, double *out);

/* operation counters: [0] md add (incl. sub), [1] md mul, [2] md div,
 * [3] md sqrt, [4] columns with x0 > 0 in the general reflector branch,
 * [5] columns with sigma == 0 and x0 >= 0 (identity reflector),
 * [6] columns with sigma == 0 and x0 < 0 (reflector v = e1, beta = 2). */
void mdref_reset_counts(void);
void mdref_get_counts(uint64_t out[7]);

/* Householder QR of the m x n matrix A (m >= n), in place: R overwrites A
 * (zeros below the diagonal).  If Q != NULL, the m x m orthogonal Q with
 * A = QR is written.  beta (n md values, plane stride n) receives the
 * reflector coefficients when non-NULL.  Returns 0, or -1 on bad arguments. */
int mdref_qr(int p, int64_t m, int64_t n, double *A, int64_t lda, int64_t psa,
             double *Q, int64_t ldq, int64_t psq, double *beta);

/* Solves R x = y for the n x n upper triangular R (diagonal nonzero).
 * y, x: plane stride n.  Returns 0, or -2 when a diagonal entry is zero. */
int mdref_backsub(int p, int64_t n, const double *R, int64_t ldr, int64_t psr,
                  const double *y, double *x);

/* Least squares min ||b - Ax||: QR of A applied to b (Q not formed), then
 * back substitution.  A is not modified.  b: plane stride m; x: plane
 * stride n.  Returns 0, -1 (arguments) or -2 (zero diagonal in R). */
int mdref_lstsq(int p, int64_t m, int64_t n, const double *A, int64_t lda, int64_t psa,
                const double *b, double *x);

/* y = op(A) x with op = A (trans = 0, A m x n, x length n, y length m) or
 * A^T (trans = 1, x length m, y length n).  Sums run in increasing index.
 * x, y: plane stride = their length. */
void mdref_gemv(int p, int trans, int64_t m, int64_t n, const double *A, int64_t lda,
                int64_t psa, const double *x, double *y);

/* C = A B for A (m x k), B (k x n), C (m x n); sums in increasing index. */
void mdref_gemm(int p, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                int64_t psa, const double *B, int64_t ldb, int64_t psb, double *C,
                int64_t ldc, int64_t psc);

/* Complex multiple doubles: real and imaginary parts in separate limb-planar
 * arrays (re and im pointers, same ld and plane stride).  Householder
 * reflectors H = I - beta v v^H with beta real and H x = e^{i arg x0} ||x|| e1
 * (the diagonal of R carries the phases of the leading entries). */
int mdref_zqr(int p, int64_t m, int64_t n, double *Ar, double *Ai, int64_t lda, int64_t psa,
              double *Qr, double *Qi, int64_t ldq, int64_t psq, double *beta);
int mdref_zbacksub(int p, int64_t n, const double *Rr, const double *Ri, int64_t ldr, int64_t psr,
                   const double *yr, const double *yi, double *xr, double *xi);
int mdref_zlstsq(int p, int64_t m, int64_t n, const double *Ar, const double *Ai, int64_t lda,
                 int64_t psa, const double *br, const double *bi, double *xr, double *xi);

#ifdef __cplusplus
}
#endif
#endif
