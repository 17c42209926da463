// Multiprecision arithmetic on the integer pipe: 24-bit digits with exact
// int64 accumulation.
//
// On GB300 an FP64 warp instruction occupies its SM sub-partition for 64
// cycles whatever the number of active lanes, while a 32-bit integer
// multiply-add issues every 2 cycles with a 4.5-cycle dependent latency.  The
// Householder panel (Section 3.1, step 1 of Algorithm 2) is a long chain of
// dependent dot products, norms and scalar operations, so it is computed here
// in integer arithmetic and only its results are rounded to multiple doubles.
//
// Representations (all digits "sign-consistent": every digit has the sign of
// the value and magnitude below 2^24, so truncating low digits truncates the
// value toward zero):
//  * fixed<D>: a panel entry, value = (sum_k d_k 2^(24k)) * 2^(24 e), with e a
//    per-column scale shared by all entries (the column's norm bounds them);
//  * xf<N>: a scalar with its own digit exponent, normalised so that d[N-1]
//    is nonzero (zero: all digits and e zero).
// Products of two digits are exact in int64; sums of up to 2^14 of them
// cannot overflow, so dot products accumulate exactly by diagonals and are
// carried only once.  Every function is host/device so that the host tests
// can compare it with exact rational arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#include "md.cuh"

namespace mdls {
namespace fx {

// The scalar routines are large when unrolled; they are real calls so that
// the single thread running them keeps one copy of each.
#define FX_CALL __host__ __device__ __noinline__

constexpr int kB = 24;
constexpr int64_t kMask = (int64_t(1) << kB) - 1;

// Digits of a panel entry for P limbs (53P bits, 64 bits of guard and
// headroom) and of a scalar.
template <int P>
struct Cfg {
    static constexpr int D = (53 * P + 64 + kB - 1) / kB;
    static constexpr int N = D + 1;
};

MD_INLINE uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

MD_INLINE double dfrom(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

MD_INLINE int bitlen64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return 64 - __clzll((long long)x);
#else
    return x ? 64 - __builtin_clzll(x) : 0;
#endif
}

MD_INLINE int floordiv24(int x) { return x >= 0 ? x / kB : -((-x + kB - 1) / kB); }

// sum_k c_k 2^(24k) -> sign-consistent digits.  The top entry keeps whatever
// does not fit below it; callers size n so that it is a digit.
template <int n>
MD_INLINE void carry_norm(int64_t (&c)[n]) {
#pragma unroll
    for (int k = 0; k < n - 1; ++k) {
        c[k + 1] += c[k] >> kB;
        c[k] &= kMask;
    }
    if (c[n - 1] < 0) {
#pragma unroll
        for (int k = 0; k < n; ++k) c[k] = -c[k];
#pragma unroll
        for (int k = 0; k < n - 1; ++k) {
            c[k + 1] += c[k] >> kB;
            c[k] &= kMask;
        }
#pragma unroll
        for (int k = 0; k < n; ++k) c[k] = -c[k];
    }
}

// Adds the double v to sum_k c_k 2^(24(k+e)); bits below 2^(24e) are
// truncated (toward zero), digits at or above index n are dropped (callers
// make sure there are none).
template <int n>
MD_INLINE void add_double(int64_t (&c)[n], double v, int e) {
    uint64_t u = dbits(v);
    const bool neg = (u >> 63) != 0;
    u &= 0x7fffffffffffffffULL;
    if (u == 0 || (u >> 52) == 0x7ff) return;
    const int be = (int)(u >> 52);
    uint64_t m = u & ((uint64_t(1) << 52) - 1);
    int L;  // exponent of the mantissa's last bit
    if (be == 0) {
        L = -1074;
    } else {
        m |= uint64_t(1) << 52;
        L = be - 1075;
    }
    int p = L - kB * e;
    if (p < 0) {
        if (p <= -64) return;
        m >>= -p;
        p = 0;
    }
    const int q = p / kB, b = p % kB;
    const int64_t lo = (int64_t)((m & (uint64_t)kMask) << b);  // < 2^47
    const int64_t hi = (int64_t)((m >> kB) << b);              // < 2^52
    int64_t t0 = lo & kMask, t1 = (lo >> kB) + (hi & kMask), t2 = hi >> kB;
    if (neg) {
        t0 = -t0;
        t1 = -t1;
        t2 = -t2;
    }
    if (q < n) c[q] += t0;
    if (q + 1 < n) c[q + 1] += t1;
    if (q + 2 < n) c[q + 2] += t2;
}

// ---------------------------------------------------------------------------
// Scalars
// ---------------------------------------------------------------------------
template <int N>
struct xf {
    int32_t d[N];
    int e;
};

template <int N>
MD_INLINE xf<N> xf_zero() {
    xf<N> r;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = 0;
    r.e = 0;
    return r;
}

template <int N>
MD_INLINE bool xf_is_zero(const xf<N>& x) {
    return x.d[N - 1] == 0;
}

template <int N>
MD_INLINE int xf_sign(const xf<N>& x) {
    return x.d[N - 1] > 0 ? 1 : (x.d[N - 1] < 0 ? -1 : 0);
}

template <int N>
MD_INLINE xf<N> xf_neg(const xf<N>& x) {
    xf<N> r = x;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -x.d[k];
    return r;
}

// Normalises sum_k c_k 2^(24(k+e0)) to N digits (the low ones truncated).
// Scalar code: the digit shift is data dependent and goes through a local
// array.
template <int N, int M>
MD_INLINE xf<N> xf_from_acc(int64_t (&c)[M], int e0) {
    carry_norm<M>(c);
    int t = -1;
#pragma unroll
    for (int k = 0; k < M; ++k)
        if (c[k] != 0) t = k;
    if (t < 0) return xf_zero<N>();
    int32_t buf[M];
#pragma unroll
    for (int k = 0; k < M; ++k) buf[k] = (int32_t)c[k];
    xf<N> r;
    const int lo = t - (N - 1);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int s = lo + k;
        r.d[k] = (s >= 0) ? buf[s] : 0;
    }
    r.e = e0 + lo;
    return r;
}

template <int N>
MD_INLINE xf<N> xf_from_int(int64_t v) {
    int64_t c[N + 2];
#pragma unroll
    for (int k = 0; k < N + 2; ++k) c[k] = 0;
    c[0] = v;
    return xf_from_acc<N>(c, 0);
}

// exact value of a double (N >= 4 digits hold any 53-bit mantissa)
template <int N>
MD_INLINE xf<N> xf_from_double(double v) {
    const uint64_t u = dbits(v) & 0x7fffffffffffffffULL;
    if (u == 0) return xf_zero<N>();
    int msb;  // exponent of the leading bit
    const int be = (int)(u >> 52);
    if (be == 0) msb = bitlen64(u) - 1 - 1074;
    else msb = be - 1023;
    const int e = floordiv24(msb) - 3;
    int64_t c[6] = {0, 0, 0, 0, 0, 0};
    add_double<6>(c, v, e);
    int64_t w[N + 2];
#pragma unroll
    for (int k = 0; k < N + 2; ++k) w[k] = k < 6 ? c[k] : 0;
    return xf_from_acc<N>(w, e);
}

template <int N>
FX_CALL xf<N> xf_mul(const xf<N>& a, const xf<N>& b) {
    // product diagonals s = N-2 .. 2N-2, one carry entry above
    int64_t c[N + 2];
#pragma unroll
    for (int k = 0; k < N + 2; ++k) c[k] = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int l = 0; l < N; ++l)
            if (j + l >= N - 2) c[j + l - (N - 2)] += (int64_t)a.d[j] * b.d[l];
    return xf_from_acc<N>(c, a.e + b.e + N - 2);
}

template <int N>
FX_CALL xf<N> xf_add(const xf<N>& a, const xf<N>& b) {
    if (xf_is_zero(a)) return b;
    if (xf_is_zero(b)) return a;
    const int top = (a.e > b.e ? a.e : b.e) + N - 1;
    const int base = top - N - 1;  // window [base, top + 1]
    int64_t c[N + 3];
#pragma unroll
    for (int k = 0; k < N + 3; ++k) c[k] = 0;
    const int oa = a.e - base, ob = b.e - base;  // both <= 2
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (oa + k >= 0) c[oa + k] += a.d[k];
        if (ob + k >= 0) c[ob + k] += b.d[k];
    }
    return xf_from_acc<N>(c, base);
}

template <int N>
MD_INLINE xf<N> xf_sub(const xf<N>& a, const xf<N>& b) {
    return xf_add<N>(a, xf_neg<N>(b));
}

// x * 2^k for |k| < 24
template <int N>
MD_INLINE xf<N> xf_shift_bits(const xf<N>& x, int k) {
    const int64_t f = int64_t(1) << (k >= 0 ? k : k + kB);
    int64_t c[N + 2];
#pragma unroll
    for (int j = 0; j < N; ++j) c[j] = (int64_t)x.d[j] * f;
    c[N] = 0;
    c[N + 1] = 0;
    return xf_from_acc<N>(c, k >= 0 ? x.e : x.e - 1);
}

// The value as (mantissa, digit exponent): x ~= m * 2^(24 k) from the three
// leading digits, |m| >= 2^48, relative error below 2^-47.
template <int N>
MD_INLINE double xf_lead(const xf<N>& x, int& k) {
    k = x.e + N - 3;
    return (double)x.d[N - 1] * 281474976710656.0 + (double)x.d[N - 2] * 16777216.0 + (double)x.d[N - 3];
}

// y * 2^(24 k) for a double y (exact)
template <int N>
MD_INLINE xf<N> xf_from_double_scaled(double y, int k) {
    xf<N> r = xf_from_double<N>(y);
    if (!xf_is_zero(r)) r.e += k;
    return r;
}

// Newton iteration count: a double start is good to 46 bits, each step
// doubles that, and 24(N-1) bits are wanted.
template <int N>
struct NewtonSteps {
    static constexpr int bits = kB * (N - 1);
    static constexpr int value = bits <= 46 ? 0 : bits <= 92 ? 1 : bits <= 184 ? 2 : bits <= 368 ? 3 : 4;
};

// Digits for Newton step I (0-based): enough for the 46 * 2^(I+1) bits it
// delivers plus a guard digit, at most N (the last step runs at full width).
template <int N, int I>
struct StepDigits {
    static constexpr int want = 46 << (I + 1);
    static constexpr int k0 = (want + 2 * kB - 1) / kB + 1;
    static constexpr int value = k0 < N ? k0 : N;
};

// x with K digits: the leading ones kept, or zeros appended below.
template <int K, int N>
MD_INLINE xf<K> xf_resize(const xf<N>& x) {
    xf<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int s = k + N - K;
        r.d[k] = (s >= 0 && s < N) ? x.d[s] : 0;
    }
    r.e = xf_is_zero(x) ? 0 : x.e + N - K;
    return r;
}

// y <- y + y (1 - x y), each step at the precision it can deliver.
template <int N, int I>
MD_INLINE void recip_steps(const xf<N>& x, xf<N>& y) {
    if constexpr (I < NewtonSteps<N>::value) {
        constexpr int K = StepDigits<N, I>::value;
        const xf<K> xk = xf_resize<K, N>(x), yk = xf_resize<K, N>(y);
        const xf<K> t = xf_sub<K>(xf_from_int<K>(1), xf_mul<K>(xk, yk));
        y = xf_resize<N, K>(xf_add<K>(yk, xf_mul<K>(yk, t)));
        recip_steps<N, I + 1>(x, y);
    }
}

// 1/x (x nonzero) by Newton's iteration from a double start.
template <int N>
FX_CALL xf<N> xf_recip(const xf<N>& x) {
    int k;
    const double m = xf_lead<N>(x, k);
    xf<N> y = xf_from_double_scaled<N>(1.0 / m, -k);
    recip_steps<N, 0>(x, y);
    return y;
}

// y <- y + y (1 - a y^2) / 2, each step at the precision it can deliver.
template <int N, int I>
MD_INLINE void rsqrt_steps(const xf<N>& a, xf<N>& y) {
    if constexpr (I < NewtonSteps<N>::value) {
        constexpr int K = StepDigits<N, I>::value;
        const xf<K> ak = xf_resize<K, N>(a), yk = xf_resize<K, N>(y);
        xf<K> t = xf_sub<K>(xf_from_int<K>(1), xf_mul<K>(ak, xf_mul<K>(yk, yk)));
        t = xf_shift_bits<K>(t, -1);
        y = xf_resize<N, K>(xf_add<K>(yk, xf_mul<K>(yk, t)));
        rsqrt_steps<N, I + 1>(a, y);
    }
}

// 1/sqrt(a) (a > 0) by Newton's iteration from a double start.
template <int N>
FX_CALL xf<N> xf_rsqrt(const xf<N>& a) {
    int k;
    double m = xf_lead<N>(a, k);
    if (k & 1) {  // make the digit exponent even: 2^(24k) = 2^(24(k-1)) 2^24
        m *= 16777216.0;
        k -= 1;
    }
    xf<N> y = xf_from_double_scaled<N>(1.0 / sqrt(m), -(k / 2));
    rsqrt_steps<N, 0>(a, y);
    return y;
}

// Householder scalars of x = (x0, x_1, ...) from sigma = sum_{i>0} x_i^2
// (Golub and Van Loan, Algorithm 5.1.1, with the vector left unscaled:
// u = (v0, x_1, ...), H = I - bp u u^T, bp = 2/||u||^2 = -1/(mu v0)).
// Returns the kind: 0 a reflector (R = mu = ||x||, v0 = x0 - mu, written
// -sigma/(x0 + mu) for x0 > 0 to avoid cancellation); 1 sigma = 0 and
// x0 >= 0 (H = I: bp = 0, R = x0); 2 sigma = 0 and x0 < 0 (H = I - 2 e1 e1^T:
// bp = 2, R = -x0).  Also returns 1/v0 and beta = bp v0^2, the factor of the
// normalised vector v = u / v0 (v0 = 1 for kinds 1 and 2).
template <int N>
FX_CALL int xf_house(const xf<N>& sig, const xf<N>& x0, xf<N>& v0, xf<N>& bp, xf<N>& rcc, xf<N>& inv_v0,
                     xf<N>& beta) {
    if (xf_is_zero(sig)) {
        v0 = xf_from_int<N>(1);
        inv_v0 = v0;
        if (xf_sign(x0) >= 0) {
            bp = xf_zero<N>();
            rcc = x0;
            beta = bp;
            return 1;
        }
        bp = xf_from_int<N>(2);
        rcc = xf_neg<N>(x0);
        beta = bp;
        return 2;
    }
    // one Newton reciprocal in either branch: R = 1/(mu v0) for x0 <= 0;
    // for x0 > 0, R = 1/(sigma s) with s = x0 + mu gives 1/s = sigma R and
    // 1/sigma = s R, so v0 = -sigma^2 R, 1/v0 = -s^2 R, bp = s^2 R / mu
    const xf<N> a2 = xf_add<N>(xf_mul<N>(x0, x0), sig);
    const xf<N> rs = xf_rsqrt<N>(a2);
    const xf<N> mu = xf_mul<N>(a2, rs);
    if (xf_sign(x0) <= 0) {
        v0 = xf_sub<N>(x0, mu);
        const xf<N> R = xf_recip<N>(xf_mul<N>(mu, v0));
        bp = xf_neg<N>(R);
        inv_v0 = xf_mul<N>(mu, R);
    } else {
        const xf<N> sx = xf_add<N>(x0, mu);
        const xf<N> R = xf_recip<N>(xf_mul<N>(sig, sx));
        v0 = xf_neg<N>(xf_mul<N>(sig, xf_mul<N>(sig, R)));
        const xf<N> s2R = xf_mul<N>(sx, xf_mul<N>(sx, R));
        inv_v0 = xf_neg<N>(s2R);
        bp = xf_mul<N>(s2R, rs);
    }
    beta = xf_mul<N>(xf_mul<N>(bp, v0), v0);
    rcc = mu;
    return 0;
}

// ---------------------------------------------------------------------------
// Conversions to and from multiple doubles
// ---------------------------------------------------------------------------

// Exponent of the leading bit of a nonzero finite double.
MD_INLINE int dmsb(double v) {
    const uint64_t u = dbits(v) & 0x7fffffffffffffffULL;
    const int be = (int)(u >> 52);
    return be == 0 ? bitlen64(u) - 1 - 1074 : be - 1023;
}

template <int P, int N>
FX_CALL xf<N> xf_from_md(const md<P>& x) {
    int msb = -100000;
#pragma unroll
    for (int l = 0; l < P; ++l)
        if ((dbits(x.v[l]) & 0x7fffffffffffffffULL) != 0) {
            const int m = dmsb(x.v[l]);
            msb = m > msb ? m : msb;
        }
    if (msb == -100000) return xf_zero<N>();
    const int e = floordiv24(msb) - (N - 1);
    int64_t c[N + 2];
#pragma unroll
    for (int k = 0; k < N + 2; ++k) c[k] = 0;
#pragma unroll
    for (int l = 0; l < P; ++l) add_double<N + 2>(c, x.v[l], e);
    return xf_from_acc<N>(c, e);
}

// 53 bits of the magnitude digits m starting at bit lo (bits below 0 are 0).
template <int N>
MD_INLINE uint64_t extract53(const uint32_t (&m)[N], int lo) {
    const int q = floordiv24(lo);
    const int off = lo - kB * q;  // 0..23
    uint64_t r = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int s = q + i;
        uint64_t dig = 0;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k == s) dig = m[k];
        const int sh = kB * i - off;  // position of this digit in the result
        if (sh >= 64) continue;
        r |= sh >= 0 ? (dig << sh) : (dig >> -sh);
    }
    return r & ((uint64_t(1) << 53) - 1);
}

// Highest set bit of the magnitude with index below pos, or -1.
template <int N>
MD_INLINE int top_bit_below(const uint32_t (&m)[N], int pos) {
    int r = -1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        uint32_t dig = m[k];
        const int base = kB * k;
        if (base >= pos) dig = 0;
        else if (pos - base < kB) dig &= (uint32_t(1) << (pos - base)) - 1;
        if (dig) r = base + bitlen64(dig) - 1;
    }
    return r;
}

// Rounds toward zero to P limbs; each limb is a 53-bit slice starting at a
// set bit, so the limbs do not overlap and carry no zero gaps.
template <int P, int N>
FX_CALL md<P> xf_to_md(const xf<N>& x) {
    md<P> r = md_zero<P>();
    if (xf_is_zero(x)) return r;
    const bool neg = x.d[N - 1] < 0;
    uint32_t m[N];
#pragma unroll
    for (int k = 0; k < N; ++k) m[k] = (uint32_t)(neg ? -x.d[k] : x.d[k]);
    int cur = kB * (N - 1) + bitlen64(m[N - 1]) - 1;
#pragma unroll
    for (int l = 0; l < P; ++l) {
        if (cur < 0) break;
        const uint64_t chunk = extract53<N>(m, cur - 52);  // bit 52 set
        const int L = cur - 52 + kB * x.e;                // exponent of its last bit
        const int be = L + 1075;
        if (be <= 0) {  // subnormal (truncated), nothing representable below it
            const int sh = 1 - be;
            if (sh < 53) r.v[l] = dfrom(((uint64_t)neg << 63) | (chunk >> sh));
            break;
        }
        if (be >= 2047) {
            r.v[l] = neg ? -INFINITY : INFINITY;
            break;
        }
        const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)be << 52) | (chunk & ((uint64_t(1) << 52) - 1));
        r.v[l] = dfrom(bits);
        cur = top_bit_below<N>(m, cur - 52);
    }
    return r;
}

// The same Householder scalars computed in P-limb arithmetic on the FP64
// pipe (csrc/md.cuh) from the digit inputs rounded to P limbs, and returned
// exactly as digits.  The results carry P-limb accuracy (about 2^(2-53P)
// relative) instead of 24(N-1) bits, and the reflector they define is
// orthogonal to the accuracy of the P-limb output.  For double double they
// take a few hundred FP64 instructions on one thread, far fewer cycles than
// the digit Newton iterations (the panels use them for P = 2 only).  Same
// kinds and formulas as xf_house (one reciprocal in either branch).
template <int P, int N>
FX_CALL int xf_house_md(const xf<N>& sig_x, const xf<N>& x0_x, xf<N>& v0, xf<N>& bp, xf<N>& rcc,
                        xf<N>& inv_v0, xf<N>& beta) {
    if (xf_is_zero(sig_x)) {
        v0 = xf_from_int<N>(1);
        inv_v0 = v0;
        if (xf_sign(x0_x) >= 0) {
            bp = xf_zero<N>();
            rcc = x0_x;
            beta = bp;
            return 1;
        }
        bp = xf_from_int<N>(2);
        rcc = xf_neg<N>(x0_x);
        beta = bp;
        return 2;
    }
    const md<P> sig = xf_to_md<P, N>(sig_x), x0 = xf_to_md<P, N>(x0_x);
    const md<P> one = md_from_double<P>(1.0);
    const md<P> a2 = md_fma<P>(sig, x0, x0);
    const md<P> mu = md_sqrt<P>(a2);
    md<P> v0m, bpm, invm;
    if (xf_sign(x0_x) <= 0) {
        v0m = md_sub<P>(x0, mu);
        const md<P> R = md_div<P>(one, md_mul<P>(mu, v0m));
        bpm = md_neg<P>(R);
        invm = md_mul<P>(mu, R);
    } else {
        const md<P> sx = md_add<P>(x0, mu);
        const md<P> R = md_div<P>(one, md_mul<P>(sig, sx));
        v0m = md_neg<P>(md_mul<P>(sig, md_mul<P>(sig, R)));
        const md<P> s2R = md_mul<P>(sx, md_mul<P>(sx, R));
        invm = md_neg<P>(s2R);
        bpm = md_div<P>(s2R, mu);
    }
    const md<P> betam = md_mul<P>(md_mul<P>(bpm, v0m), v0m);
    v0 = xf_from_md<P, N>(v0m);
    bp = xf_from_md<P, N>(bpm);
    inv_v0 = xf_from_md<P, N>(invm);
    beta = xf_from_md<P, N>(betam);
    rcc = xf_from_md<P, N>(mu);
    return 0;
}

// ---------------------------------------------------------------------------
// Double-double Householder scalars with short dependency chains
// ---------------------------------------------------------------------------
// One thread (or one warp in lockstep) computes the scalars, so their cost is
// the length of the chain of dependent FP64 operations, each waiting out the
// pipe's latency (about 63 cycles measured here; an IEEE division or square
// root about 630).  Hence: one Newton correction of the double reciprocal or
// square root instead of long division, and v0, bp, 1/v0, beta from mu, 1/mu
// and products instead of further divisions.

// Dekker's fast two-sum: s + e == a + b exactly when |a| >= |b| (or a == 0).
MD_INLINE md<2> dd_fast_sum(double a, double b) {
    const double s = dadd(a, b);
    return md<2>{{s, dsub(b, dsub(s, a))}};
}

// a * b: the exact product of the leading limbs plus the two cross terms
// (a1 b1, below 2^-106 |ab|, is dropped); relative error below 2^-103.
MD_INLINE md<2> dd_mul(const md<2>& a, const md<2>& b) {
    double p, e;
    two_prod(a.v[0], b.v[0], p, e);
    e = dfma(a.v[0], b.v[1], dfma(a.v[1], b.v[0], e));
    return dd_fast_sum(p, e);
}

// 1 / b (b nonzero, no overflow): q = RN(1/b0), whose residual 1 - q b0 is a
// double (exact by FMA), then 1/b = q / (1 - r) with r = 1 - q b, |r| <=
// 2^-52, taken as q (1 + r + r^2); relative error below 2^-103.
MD_INLINE md<2> dd_recip(const md<2>& b) {
    const double q = 1.0 / b.v[0];
    const double r = dfma(-q, b.v[1], dfma(-q, b.v[0], 1.0));
    return dd_fast_sum(q, dmul(q, dfma(r, r, r)));
}

// sqrt(a) for a0 > 0: s = RN(sqrt(a0)), whose residual a0 - s^2 is a double
// (exact by FMA); sqrt(a) = s sqrt(1 + t) with t = (a - s^2) / s^2, |t| <=
// 2^-51, taken as s + (a - s^2) / (2 s); relative error below 2^-103.
MD_INLINE md<2> dd_sqrt(const md<2>& a) {
    const double s = sqrt(a.v[0]);
    const double y = 1.0 / s;
    const double r = dadd(dfma(-s, s, a.v[0]), a.v[1]);
    return dd_fast_sum(s, dmul(dmul(r, y), 0.5));
}

// The Householder scalars of xf_house from sig > 0 (the squared norm below
// the diagonal) and x0 in double double: mu = sqrt(x0^2 + sig),
// v0 = x0 - mu (x0 <= 0) or -sig / (x0 + mu) (x0 > 0, no cancellation),
// inv = 1/v0, bp = -1/(mu v0) = -inv/mu, beta = bp v0^2 = -v0/mu.  The
// chain: mu, then one addition, one reciprocal and one product each way;
// 1/mu and 1/sig are formed beside it.
MD_INLINE void house_dd(const md<2>& sig, const md<2>& x0, md<2>& mu, md<2>& v0, md<2>& bp, md<2>& inv,
                        md<2>& beta) {
    const md<2> rsig = dd_recip(sig);
    mu = dd_sqrt(md_add<2>(sig, dd_mul(x0, x0)));
    const md<2> rmu = dd_recip(mu);
    if (x0.v[0] <= 0.0) {
        v0 = md_sub<2>(x0, mu);
        inv = dd_recip(v0);
    } else {
        const md<2> sx = md_add<2>(x0, mu);
        v0 = md_neg<2>(dd_mul(sig, dd_recip(sx)));
        inv = md_neg<2>(dd_mul(sx, rsig));
    }
    bp = md_neg<2>(dd_mul(rmu, inv));
    beta = md_neg<2>(dd_mul(v0, rmu));
}

// house_dd between digit scalars, one thread: the form the host replay and
// the tests use (the panels run house_dd with the conversions spread over a
// warp and get the same digits).  Kinds and degenerate cases as xf_house.
template <int N>
FX_CALL int xf_house_dd(const xf<N>& sig_x, const xf<N>& x0_x, xf<N>& v0, xf<N>& bp, xf<N>& rcc, xf<N>& inv_v0,
                        xf<N>& beta) {
    if (xf_is_zero(sig_x)) return xf_house_md<2, N>(sig_x, x0_x, v0, bp, rcc, inv_v0, beta);
    md<2> mu, v0m, bpm, invm, betam;
    house_dd(xf_to_md<2, N>(sig_x), xf_to_md<2, N>(x0_x), mu, v0m, bpm, invm, betam);
    v0 = xf_from_md<2, N>(v0m);
    bp = xf_from_md<2, N>(bpm);
    inv_v0 = xf_from_md<2, N>(invm);
    beta = xf_from_md<2, N>(betam);
    rcc = xf_from_md<2, N>(mu);
    return 0;
}

// ---------------------------------------------------------------------------
// Panel entries (fixed point with a per-column digit scale e)
// ---------------------------------------------------------------------------

// md -> D digits at scale e (bits below 2^(24e) truncated).
template <int P, int D>
MD_INLINE void fixed_from_md(const md<P>& x, int e, int32_t (&d)[D]) {
    int64_t c[D + 2];
#pragma unroll
    for (int k = 0; k < D + 2; ++k) c[k] = 0;
#pragma unroll
    for (int l = 0; l < P; ++l) add_double<D + 2>(c, x.v[l], e);
    carry_norm<D + 2>(c);
#pragma unroll
    for (int k = 0; k < D; ++k) d[k] = (int32_t)c[k];
}

template <int N, int D>
FX_CALL xf<N> xf_from_fixed(const int32_t (&d)[D], int e) {
    int64_t c[(D > N ? D : N) + 1];
    constexpr int M = (D > N ? D : N) + 1;
#pragma unroll
    for (int k = 0; k < M; ++k) c[k] = k < D ? d[k] : 0;
    return xf_from_acc<N>(c, e);
}

// xf -> D digits at scale e, truncated; returns false if the value does not
// fit (|value| >= 2^(24(e+D)) ).
template <int N, int D>
FX_CALL bool fixed_from_xf(const xf<N>& x, int e, int32_t (&d)[D]) {
    const int off = x.e - e;  // digit k of x lands at index k + off
    bool ok = true;
    int32_t buf[D];
#pragma unroll
    for (int i = 0; i < D; ++i) buf[i] = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int s = k + off;
        if (s >= D) {
            if (x.d[k] != 0) ok = false;
        } else if (s >= 0) {
            buf[s] = x.d[k];
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) d[i] = buf[i];
    return ok;
}

// Index of the leading nonzero digit (-1 for zero).
template <int D>
MD_INLINE int fixed_top(const int32_t (&d)[D]) {
    int t = -1;
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (d[k] != 0) t = k;
    return t;
}

// acc[s - (D-3)] += sum_{j+l=s} u_j a_l for the diagonals s >= D-3 (the rest
// is below 2^(24(D-3)) * D * 2^48 and is dropped).  acc has D+3 entries.
template <int D>
MD_INLINE void dot_acc(const int32_t (&u)[D], const int32_t (&a)[D], int64_t (&acc)[D + 3]) {
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int l = 0; l < D; ++l)
            if (j + l >= D - 3) acc[j + l - (D - 3)] += (int64_t)u[j] * a[l];
}

// a -= (w * u) / 2^(24(D-2)), truncated: w carries two integer digits and
// D-2 fractional ones.  Two guard digits below a's last are kept until the
// final carry.
template <int D>
MD_INLINE void axpy_row(int32_t (&a)[D], const int32_t (&w)[D], const int32_t (&u)[D]) {
    int64_t c[D + 3];  // positions -2 .. D
    c[0] = 0;
    c[1] = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) c[k + 2] = a[k];
    c[D + 2] = 0;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const int k = j + l - (D - 2);
            if (k >= -2) c[k + 2] -= (int64_t)w[j] * u[l];
        }
    carry_norm<D + 3>(c);
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = (int32_t)c[k + 2];
}

}  // namespace fx
}  // namespace mdls
