// Multiple-double arithmetic on the FP64 CUDA cores (device code).
//
// A multiple double (arXiv 2110.08375, Section 1.1) is an unevaluated sum of
// P doubles, most significant first: P = 2 double double, 4 quad double,
// 8 octo double.  As in the paper's implementation notes (Section 4.1) a value
// lives in P separate registers, never in an array in memory.
//
// Building blocks are the error-free transforms
//   two_sum   (an FP64 addition, its error on the integer pipe): s + e == a + b exactly,
//   two_prod  (FMA):    p + e == a * b exactly (no underflow),
// written with explicit round-to-nearest intrinsics so that the compiler can
// neither contract nor reassociate them.
//
// add / mul / fused multiply-add use one scheme for every P ("bins by order"):
// each term of the exact result has a nominal order d (a_i*b_j has order i+j,
// the low half of a two_prod one order more, limb c_d of an addend order d).
// Bin d (d < P-1) is summed with two_sum, every rounding error going on to bin
// d+1 as a new term; bin P-1 is summed with plain additions and FMAs, whose
// errors are of order P and are dropped.  The P bin sums are then renormalised
// (a bottom-up then a top-down two_sum sweep).  The absolute error is a small
// multiple of 2^(-53P) (|a||b| + |c|), the bound used by the normwise error
// analysis of Householder QR; the result limbs decrease by about 2^-53 each.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace mdls {

// Host compilation (unit tests of the arithmetic on the CPU) uses plain IEEE
// operations; the host compiler must not contract them (-ffp-contract=off).
#define MD_INLINE __host__ __device__ __forceinline__

template <int P>
struct md {
    double v[P];
};

#ifdef __CUDA_ARCH__
MD_INLINE double dadd(double a, double b) { return __dadd_rn(a, b); }
MD_INLINE double dsub(double a, double b) { return __dsub_rn(a, b); }
MD_INLINE double dmul(double a, double b) { return __dmul_rn(a, b); }
MD_INLINE double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }
MD_INLINE double dnan() { return __longlong_as_double(0x7ff8000000000000LL); }
#else
inline double dadd(double a, double b) { return a + b; }
inline double dsub(double a, double b) { return a - b; }
inline double dmul(double a, double b) { return a * b; }
inline double dfma(double a, double b, double c) { return ::fma(a, b, c); }
inline double dnan() { return __builtin_nan(""); }
#endif

MD_INLINE uint64_t dbits64(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

MD_INLINE double dfrom64(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

// Signed significand m (two's complement) and exponent e of the last bit of
// a finite double: x = m 2^e.
MD_INLINE void sig_exp(uint64_t u, uint64_t& m, int& e) {
    const int be = (int)((u >> 52) & 0x7ff);
    const uint64_t mag = (u & 0xfffffffffffffULL) | ((uint64_t)(be != 0) << 52);
    e = (be > 1 ? be : 1) - 1075;
    m = (u >> 63) ? (uint64_t)0 - mag : mag;
}

MD_INLINE uint64_t shl_or_zero(uint64_t x, int k) { return k >= 64 ? 0 : x << k; }

// The exact error (a + b) - s of s = fl(a + b), by integer arithmetic.  With
// L the lowest last-bit exponent of a, b and s, the error is an integer
// multiple of 2^L and below min(|a|, |b|) (or zero when s has the finest
// last bit), so (a + b - s) / 2^L fits in 54 bits and is exact modulo 2^64
// whatever the wrap-around of the shifted terms; it is then written out as
// a double (exact: at most 53 significant bits).  The sign of a zero error
// follows Fast2Sum's.  A non-finite s gives NaN.
MD_INLINE double sum_error(double a, double b, double s) {
    const uint64_t ua = dbits64(a), ub = dbits64(b), us = dbits64(s);
    if (((us >> 52) & 0x7ff) == 0x7ff) return dfrom64(0x7ff8000000000000ULL);
    uint64_t ma, mb, ms;
    int ea, eb, es;
    sig_exp(ua, ma, ea);
    sig_exp(ub, mb, eb);
    sig_exp(us, ms, es);
    int L = ea < eb ? ea : eb;
    L = L < es ? L : es;
    const int64_t v = (int64_t)(shl_or_zero(ma, ea - L) + shl_or_zero(mb, eb - L) - shl_or_zero(ms, es - L));
    constexpr uint64_t kNegZero = 0x8000000000000000ULL;
    if (v == 0) return dfrom64((ub == kNegZero || (ua == kNegZero && ub != 0)) ? kNegZero : 0);
    const uint64_t mag = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
#ifdef __CUDA_ARCH__
    const int n = 63 - __clzll((long long)mag);
#else
    const int n = 63 - __builtin_clzll(mag);
#endif
    const int E = n + L;  // exponent of the leading bit
    uint64_t r = E >= -1022 ? (((uint64_t)(E + 1023) << 52) | ((mag << (52 - n)) & 0xfffffffffffffULL))
                            : (mag << (L + 1074));
    return dfrom64(r | ((uint64_t)(v < 0) << 63));
}

// TwoSum: s = fl(a+b), e = (a+b) - s exactly, in two forms with the same
// bits (s and e are unique).  two_sum_int: s is one FP64 addition and e comes
// from sum_error on the integer pipe, which has some 30 times the FP64 pipe's
// throughput on GB300.  two_sum_fast: Dekker's Fast2Sum (3 FP64
// operations) after ordering the operands by exponent with an integer compare
// of the sign-cleared high words; fewer registers.  Knuth's branch-free
// TwoSum would take 6 FP64 operations.
MD_INLINE void two_sum_int(double a, double b, double& s, double& e) {
    const double x = dadd(a, b);
    e = sum_error(a, b, x);
    s = x;
}

MD_INLINE void two_sum_fast(double a, double b, double& s, double& e) {
    const bool ab = (dbits64(a) << 1) >> 33 >= (dbits64(b) << 1) >> 33;
    const double big = ab ? a : b, small = ab ? b : a;
    const double x = dadd(big, small);
    e = dsub(small, dsub(x, big));
    s = x;
}

// The form bin D of a P-limb operation uses: the integer error for double
// and quad double and the first five bins of octo double.  The later od bins
// carry up to 49 live error terms: the integer form there takes the od
// product kernel from three blocks per SM to two (od slower by a quarter),
// and with it in bin 5 as well the product is already bound by the integer
// pipe (first 4 / 5 / 6 bins: 907 / 904 / 920 ms per od solve at n = 1024).
template <int P, int D>
MD_INLINE void two_sum_pd(double a, double b, double& s, double& e) {
    if constexpr (P <= 4 || D < 5) two_sum_int(a, b, s, e);
    else two_sum_fast(a, b, s, e);
}

// TwoProd with FMA (2 flops): p = fl(ab), e = ab - p exactly.
MD_INLINE void two_prod(double a, double b, double& p, double& e) {
    double x = dmul(a, b);
    e = dfma(a, b, -x);
    p = x;
}

template <int P>
MD_INLINE md<P> md_zero() {
    md<P> r;
#pragma unroll
    for (int i = 0; i < P; ++i) r.v[i] = 0.0;
    return r;
}

template <int P>
MD_INLINE md<P> md_from_double(double x) {
    md<P> r = md_zero<P>();
    r.v[0] = x;
    return r;
}

template <int P>
MD_INLINE md<P> md_neg(const md<P>& a) {
    md<P> r;
#pragma unroll
    for (int i = 0; i < P; ++i) r.v[i] = -a.v[i];
    return r;
}

MD_INLINE bool nonzero(double x) {
#ifdef __CUDA_ARCH__
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0;  // integer test, not the FP64 pipe
#else
    return x != 0.0;
#endif
}

// Renormalisation of K terms of (roughly) decreasing order into P limbs.
// 1. A bottom-up two_sum sweep moves the total towards s[0] (exact).
// 2. A top-down two_sum sweep emits a limb each time the running sum leaves
//    a nonzero error, and otherwise carries the sum on.  Zero terms are thus
//    skipped: after heavy cancellation the bins can sum to zero in front of
//    nonzero lower terms, and the result must still start with a nonzero
//    leading limb and have no zero limb in front of a nonzero one.  Limb
//    slots are written with selects, so everything stays in registers.
// Terms beyond the P-th emitted limb are of order P and are dropped.
template <int K, int P>
MD_INLINE md<P> renorm_n(double (&s)[K]) {
#pragma unroll
    for (int i = K - 2; i >= 0; --i) two_sum_pd<P, P>(s[i], s[i + 1], s[i], s[i + 1]);
    md<P> y;
#pragma unroll
    for (int k = 0; k < P; ++k) y.v[k] = 0.0;
    int j = 0;
    double e = s[0];
#pragma unroll
    for (int i = 1; i < K; ++i) {
        double r, e2;
        two_sum_pd<P, P>(e, s[i], r, e2);
        const bool emit = nonzero(e2);
#pragma unroll
        for (int k = 0; k < P; ++k) y.v[k] = (emit && j == k) ? r : y.v[k];
        j += emit ? 1 : 0;
        e = emit ? e2 : r;
    }
#pragma unroll
    for (int k = 0; k < P; ++k) y.v[k] = (j == k) ? e : y.v[k];
    return y;
}

template <int P>
MD_INLINE md<P> renorm(double (&s)[P]) {
    return renorm_n<P, P>(s);
}

// Bin D of a fused multiply-add c + a*b (WC: with addend c) or a product:
// receives c_D (WC), the high halves of the D+1 products a_i b_{D-i}, the D
// low halves of the order D-1 products (lo_prev) and the NE two_sum errors
// of bin D-1 (err_prev).  Bins below P-1 are summed with two_sum and pass
// their errors on; bin P-1 is summed with plain FMAs and additions.
// Template recursion keeps every array size and index a compile-time
// constant, so all terms stay in registers.
template <int P, bool WC, int D, int NE>
struct FmaBin {
    static constexpr int NLO = D;
    static constexpr int NTERMS = (WC ? 1 : 0) + (D + 1) + NLO + NE;
    static constexpr int NOUT = NTERMS - 1;
    MD_INLINE static void run(const md<P>& c, const md<P>& a, const md<P>& b,
                              const double (&lo_prev)[NLO > 0 ? NLO : 1],
                              const double (&err_prev)[NE > 0 ? NE : 1], double (&s)[P]) {
        if constexpr (D < P - 1) {
            double lo_cur[D + 1];
            double err_cur[NOUT > 0 ? NOUT : 1];
            int ne = 0;
            double acc;
            bool have = WC;
            if constexpr (WC) acc = c.v[D];
            else acc = 0.0;
#pragma unroll
            for (int i = 0; i <= D; ++i) {
                double hi, lo;
                two_prod(a.v[i], b.v[D - i], hi, lo);
                lo_cur[i] = lo;
                if (have) {
                    two_sum_pd<P, D>(acc, hi, acc, err_cur[ne]);
                    ++ne;
                } else {
                    acc = hi;
                    have = true;
                }
            }
#pragma unroll
            for (int i = 0; i < NLO; ++i) {
                two_sum_pd<P, D>(acc, lo_prev[i], acc, err_cur[ne]);
                ++ne;
            }
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                two_sum_pd<P, D>(acc, err_prev[k], acc, err_cur[ne]);
                ++ne;
            }
            s[D] = acc;
            FmaBin<P, WC, D + 1, NOUT>::run(c, a, b, lo_cur, err_cur, s);
        } else {
            double acc;
            if constexpr (WC) acc = c.v[D];
            else acc = 0.0;
#pragma unroll
            for (int i = 0; i <= D; ++i) acc = dfma(a.v[i], b.v[D - i], acc);
#pragma unroll
            for (int i = 0; i < NLO; ++i) acc = dadd(acc, lo_prev[i]);
#pragma unroll
            for (int k = 0; k < NE; ++k) acc = dadd(acc, err_prev[k]);
            s[D] = acc;
        }
    }
};

template <int P, bool WC>
MD_INLINE md<P> md_fma_impl(const md<P>& c, const md<P>& a, const md<P>& b) {
    double s[P];
    const double none[1] = {0.0};
    FmaBin<P, WC, 0, 0>::run(c, a, b, none, none, s);
    return renorm<P>(s);
}

template <int P>
MD_INLINE md<P> md_fma(const md<P>& c, const md<P>& a, const md<P>& b) {
    return md_fma_impl<P, true>(c, a, b);
}

// Accumulation of products into P bins without renormalising: bins[d] +=
// (order-d terms of a*b), every two_sum error passed on to bin d+1 exactly as
// in md_fma; only the last bin's plain additions round.  A product loop calls
// md_bins_renorm every few steps (the loops here: every 16) so that the last
// bin stays small and its rounding stays at the md_fma level; the saving is
// the renormalisation of every other step (about a third of a dd md FMA, a
// fifth of qd, 8 % of od).
template <int P>
MD_INLINE void md_fma_bins(double (&bins)[P], const md<P>& a, const md<P>& b) {
    md<P> c;
#pragma unroll
    for (int d = 0; d < P; ++d) c.v[d] = bins[d];
    const double none[1] = {0.0};
    FmaBin<P, true, 0, 0>::run(c, a, b, none, none, bins);
}

template <int P>
MD_INLINE void md_bins_renorm(double (&bins)[P]) {
    const md<P> r = renorm<P>(bins);
#pragma unroll
    for (int d = 0; d < P; ++d) bins[d] = r.v[d];
}

template <int P>
MD_INLINE md<P> md_from_bins(double (&bins)[P]) {
    return renorm<P>(bins);
}

template <int P>
MD_INLINE md<P> md_mul(const md<P>& a, const md<P>& b) {
    return md_fma_impl<P, false>(a, a, b);
}

// c - a*b
template <int P>
MD_INLINE md<P> md_fms(const md<P>& c, const md<P>& a, const md<P>& b) {
    return md_fma_impl<P, true>(c, md_neg(a), b);
}

// Bin D of a + b: a_D, b_D and the NE errors of bin D-1.
template <int P, int D, int NE>
struct AddBin {
    static constexpr int NOUT = NE + 1;
    MD_INLINE static void run(const md<P>& a, const md<P>& b, const double (&err_prev)[NE > 0 ? NE : 1],
                              double (&s)[P]) {
        if constexpr (D < P - 1) {
            double err_cur[NOUT];
            double acc;
            two_sum_pd<P, D>(a.v[D], b.v[D], acc, err_cur[0]);
#pragma unroll
            for (int k = 0; k < NE; ++k) two_sum_pd<P, D>(acc, err_prev[k], acc, err_cur[k + 1]);
            s[D] = acc;
            AddBin<P, D + 1, NOUT>::run(a, b, err_cur, s);
        } else {
            double acc = dadd(a.v[D], b.v[D]);
#pragma unroll
            for (int k = 0; k < NE; ++k) acc = dadd(acc, err_prev[k]);
            s[D] = acc;
        }
    }
};

template <int P>
MD_INLINE md<P> md_add(const md<P>& a, const md<P>& b) {
    double s[P];
    const double none[1] = {0.0};
    AddBin<P, 0, 0>::run(a, b, none, s);
    return renorm<P>(s);
}

template <int P>
MD_INLINE md<P> md_sub(const md<P>& a, const md<P>& b) {
    return md_add<P>(a, md_neg(b));
}

// Bin D of c + q*b for a double q: c_D, high half of q*b_D, low half of
// q*b_{D-1}, and the NE errors of bin D-1.
template <int P, int D, int NE>
struct FmaDBin {
    static constexpr int NOUT = NE + 1 + (D > 0 ? 1 : 0);
    MD_INLINE static void run(const md<P>& c, double q, const md<P>& b, double lo_prev,
                              const double (&err_prev)[NE > 0 ? NE : 1], double (&s)[P]) {
        if constexpr (D < P - 1) {
            double err_cur[NOUT];
            double hi, lo, acc;
            two_prod(q, b.v[D], hi, lo);
            two_sum_pd<P, D>(c.v[D], hi, acc, err_cur[0]);
            int ne = 1;
            if constexpr (D > 0) {
                two_sum_pd<P, D>(acc, lo_prev, acc, err_cur[ne]);
                ++ne;
            }
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                two_sum_pd<P, D>(acc, err_prev[k], acc, err_cur[ne]);
                ++ne;
            }
            s[D] = acc;
            FmaDBin<P, D + 1, NOUT>::run(c, q, b, lo, err_cur, s);
        } else {
            double acc = dfma(q, b.v[D], c.v[D]);
            if constexpr (D > 0) acc = dadd(acc, lo_prev);
#pragma unroll
            for (int k = 0; k < NE; ++k) acc = dadd(acc, err_prev[k]);
            s[D] = acc;
        }
    }
};

// c + q*b for a double q: products q*b_d have order d.
template <int P>
MD_INLINE md<P> md_fma_d(const md<P>& c, double q, const md<P>& b) {
    double s[P];
    const double none[1] = {0.0};
    FmaDBin<P, 0, 0>::run(c, q, b, 0.0, none, s);
    return renorm<P>(s);
}

// Truncation / extension between precisions (no arithmetic).
template <int Q, int P>
MD_INLINE md<Q> md_take(const md<P>& x) {
    md<Q> r;
#pragma unroll
    for (int l = 0; l < Q; ++l) r.v[l] = l < P ? x.v[l] : 0.0;
    return r;
}

// a / b by long division: quotient digit q_k = r_k / b_0 (one double
// division) and remainder r_{k+1} = r_k - q_k b.  The remainder after k
// digits is ~2^(-52k) |a| and only its leading min(P, P+1-k) limbs matter
// for a P-limb quotient, so later digits run in fewer limbs.  The P+1
// digits (each ~2^-52 below the previous) are renormalised to P limbs.
template <int P, int K, int Q>
MD_INLINE void long_div(const md<Q>& r, const md<P>& b, double (&q)[P + 1]) {
    q[K] = r.v[0] / b.v[0];
    if constexpr (K < P) {
        constexpr int Q2 = (P + 1 - (K + 1)) < P ? (P + 1 - (K + 1)) : P;
        constexpr int QN = Q2 < 1 ? 1 : Q2;
        const md<QN> rn = md_fma_d<QN>(md_take<QN>(r), -q[K], md_take<QN>(b));
        long_div<P, K + 1, QN>(rn, b, q);
    }
}

template <int P>
MD_INLINE md<P> md_div(const md<P>& a, const md<P>& b) {
    double q[P + 1];
    long_div<P, 0, P>(a, b, q);
    return renorm_n<P + 1, P>(q);
}

// sqrt(a) for a >= 0: x <- x + (a - x^2) / (2 x_0) from the double square
// root of the leading limb; each step gains ~53 bits, so step k works in
// min(P, k+2) limbs (x has at most k+1 nonzero limbs before it).  Zero for
// a == 0, NaN limbs for a < 0.
template <int P, int IT>
MD_INLINE void sqrt_steps(const md<P>& a, md<P>& x) {
    if constexpr (IT < P) {
        constexpr int Q = (IT + 2) < P ? (IT + 2) : P;
        const md<Q> xq = md_take<Q>(x);
        const md<Q> r = md_fms<Q>(md_take<Q>(a), xq, xq);
        const double d = r.v[0] / dmul(2.0, x.v[0]);
        const md<Q> xn = md_add<Q>(xq, md_from_double<Q>(d));
#pragma unroll
        for (int l = 0; l < P; ++l) x.v[l] = l < Q ? xn.v[l] : 0.0;
        sqrt_steps<P, IT + 1>(a, x);
    }
}

template <int P>
MD_INLINE md<P> md_sqrt(const md<P>& a) {
    if (a.v[0] == 0.0) return md_zero<P>();
    if (!(a.v[0] > 0.0)) {
        md<P> r;
#pragma unroll
        for (int i = 0; i < P; ++i) r.v[i] = dnan();
        return r;
    }
    md<P> x = md_from_double<P>(sqrt(a.v[0]));
    sqrt_steps<P, 0>(a, x);
    return x;
}


}  // namespace mdls
