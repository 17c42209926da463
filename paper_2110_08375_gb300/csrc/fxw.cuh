// Warp-parallel digit scalars: the Householder scalars of the integer-digit
// panel (Section 3, step 1 of Algorithm 2) spread over the 32 lanes of one
// warp.
//
// A scalar of fx.cuh (xf<N>: N sign-consistent 24-bit digits and a digit
// exponent) is held with digit k in lane k (lanes >= N hold 0) and the
// exponent in every lane.  Every routine here computes the same value, digit
// for digit, as its scalar namesake in fx.cuh: products and sums are exact in
// int64 whatever their order, and the sign-consistent normal form of an
// integer is unique.  One thread runs a 22-digit product in about 2700 cycles;
// the warp forms each lane's diagonal in N steps and propagates carries in a
// few parallel rounds.  Every lane of the warp must call every routine
// (full-mask shuffles); the results are uniform where the scalar ones are.
#pragma once
#include "fx.cuh"

namespace mdls {
namespace fxw {

using fx::kB;
using fx::kMask;
constexpr unsigned kFull = 0xffffffffu;

struct wxf {
    int32_t d;  // this lane's digit
    int e;      // digit exponent (uniform)
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int32_t digit(const wxf& x, int k) { return __shfl_sync(kFull, x.d, k); }

template <int N>
__device__ __forceinline__ bool is_zero(const wxf& x) {
    return digit(x, N - 1) == 0;
}

template <int N>
__device__ __forceinline__ int sign(const wxf& x) {
    const int32_t t = digit(x, N - 1);
    return t > 0 ? 1 : (t < 0 ? -1 : 0);
}

__device__ __forceinline__ wxf zero() { return wxf{0, 0}; }

__device__ __forceinline__ wxf neg(const wxf& x) { return wxf{-x.d, x.e}; }

// Floor carries over lanes 0 .. n-1 until every lane below n-1 holds a digit
// in [0, 2^24); lane n-1 keeps the rest.  First every entry below the top
// (|c| < 2^62) is cut into 24-bit pieces c = lo + mid 2^24 + hi 2^48 that move
// up zero, one and two lanes at once (a hi piece that would pass the top
// lands in it with weight 2^24); the entries are then below 2^25 + 2^15, a
// 32-bit round brings every carry into {-1, 0, 1}, and a remaining ripple
// moves one lane per round, so n + 2 voting rounds always suffice (the loop
// stops as soon as no lane is out of range, usually at once).
template <int n>
__device__ __forceinline__ int64_t carry_pass(int64_t c) {
    const int k = lane_id();
    const bool below = k < n - 1, top = k == n - 1;
    {
        const int32_t mid = below ? (int32_t)((c >> kB) & kMask) : 0;
        const int32_t hi = below ? (int32_t)(c >> (2 * kB)) : 0;
        int32_t m1 = __shfl_up_sync(kFull, mid, 1);
        int32_t h1 = __shfl_up_sync(kFull, hi, 1);
        int32_t h2 = __shfl_up_sync(kFull, hi, 2);
        m1 = k >= 1 ? m1 : 0;
        h1 = k >= 1 ? h1 : 0;
        h2 = k >= 2 ? h2 : 0;
        const int64_t lo = below ? (c & kMask) : c;
        c = (below || top) ? lo + m1 + h2 + (top ? ((int64_t)h1 << kB) : 0) : c;
    }
    for (int it = 0; it < n + 3; ++it) {
        const bool out = below && (c < 0 || c > kMask);
        if (it > 0 && !__any_sync(kFull, out)) break;
        const int32_t carry = below ? (int32_t)(c >> kB) : 0;
        int32_t cin = __shfl_up_sync(kFull, carry, 1);
        cin = k >= 1 ? cin : 0;
        c = below ? (c & kMask) + cin : (top ? c + cin : c);
    }
    return c;
}

// fx::carry_norm: sign-consistent digits of sum_k c_k 2^(24k).  For a
// negative total (top T < 0 over floor digits d_k) the digits follow from
// one ballot: with j the lowest nonzero digit, digit j becomes
// -(2^24 - d_j), digits above it -(2^24 - 1 - d_k) and the top T + 1 (the
// base-2^24 complement), which is the unique sign-consistent form the scalar
// routine reaches by negating, carrying and negating back.
template <int n>
__device__ __forceinline__ int64_t carry_norm(int64_t c) {
    c = carry_pass<n>(c);
    if (__shfl_sync(kFull, c, n - 1) < 0) {
        const int k = lane_id();
        const unsigned nz = __ballot_sync(kFull, k < n - 1 && c != 0);
        if (nz != 0) {
            const int j = __ffs((int)nz) - 1;
            if (k < n - 1) c = k < j ? 0 : (k == j ? c - (kMask + 1) : c - kMask);
            else if (k == n - 1) c += 1;
        }
    }
    return c;
}

// fx::xf_from_acc<N, M>: c_k in lane k (lanes >= M hold 0).
template <int N, int M>
__device__ __forceinline__ wxf from_acc(int64_t c, int e0) {
    static_assert(M <= 32 && N <= 32, "one digit per lane");
    c = carry_norm<M>(c);
    const unsigned nz = __ballot_sync(kFull, c != 0);
    if (nz == 0) return zero();
    const int t = 31 - __clz((int)nz);
    const int lo = t - (N - 1);
    const int k = lane_id(), src = lo + k;
    const int32_t v = __shfl_sync(kFull, (int32_t)c, src & 31);
    return wxf{(k < N && src >= 0) ? v : 0, e0 + lo};
}

template <int N>
__device__ __forceinline__ wxf from_int(int64_t v) {
    return from_acc<N, N + 2>(lane_id() == 0 ? v : 0, 0);
}

// fx::xf_mul: lane t forms the product diagonal N-2+t (t = 0..N).
template <int N>
__device__ __forceinline__ wxf mul(const wxf& a, const wxf& b) {
    const int k = lane_id();
    int64_t c = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int32_t aj = __shfl_sync(kFull, a.d, j);
        const int l = k + N - 2 - j;
        const int32_t bl = __shfl_sync(kFull, b.d, l & 31);
        if (k <= N && l >= 0 && l < N) c += (int64_t)aj * bl;
    }
    return from_acc<N, N + 2>(c, a.e + b.e + N - 2);
}

// fx::xf_add
template <int N>
__device__ __forceinline__ wxf add(const wxf& a, const wxf& b) {
    if (is_zero<N>(a)) return b;
    if (is_zero<N>(b)) return a;
    const int top = (a.e > b.e ? a.e : b.e) + N - 1;
    const int base = top - N - 1;
    const int k = lane_id();
    const int sa = k - (a.e - base), sb = k - (b.e - base);
    const int32_t av = __shfl_sync(kFull, a.d, sa & 31), bv = __shfl_sync(kFull, b.d, sb & 31);
    int64_t c = 0;
    if (k < N + 3) {
        if (sa >= 0 && sa < N) c += av;
        if (sb >= 0 && sb < N) c += bv;
    }
    return from_acc<N, N + 3>(c, base);
}

template <int N>
__device__ __forceinline__ wxf sub(const wxf& a, const wxf& b) {
    return add<N>(a, neg(b));
}

// fx::xf_shift_bits: x * 2^s for |s| < 24
template <int N>
__device__ __forceinline__ wxf shift_bits(const wxf& x, int s) {
    const int64_t f = int64_t(1) << (s >= 0 ? s : s + kB);
    return from_acc<N, N + 2>((int64_t)x.d * f, s >= 0 ? x.e : x.e - 1);
}

// fx::xf_lead: x ~= m 2^(24 k) from the three leading digits.
template <int N>
__device__ __forceinline__ double lead(const wxf& x, int& k) {
    k = x.e + N - 3;
    return (double)digit(x, N - 1) * 281474976710656.0 + (double)digit(x, N - 2) * 16777216.0 +
           (double)digit(x, N - 3);
}

// The lane's entry of fx::add_double<n>(c, v, e) into zeros: digit k of v at
// digit scale e (bits below 2^(24e) truncated), 0 in lanes >= n.
template <int n>
__device__ __forceinline__ int64_t double_part(double v, int e) {
    uint64_t u = fx::dbits(v);
    const bool negv = (u >> 63) != 0;
    u &= 0x7fffffffffffffffULL;
    if (u == 0 || (u >> 52) == 0x7ff) return 0;
    const int be = (int)(u >> 52);
    uint64_t m = u & ((uint64_t(1) << 52) - 1);
    int L;
    if (be == 0) {
        L = -1074;
    } else {
        m |= uint64_t(1) << 52;
        L = be - 1075;
    }
    int p = L - kB * e;
    if (p < 0) {
        if (p <= -64) return 0;
        m >>= -p;
        p = 0;
    }
    const int q = p / kB, b = p % kB;
    const int64_t lo = (int64_t)((m & (uint64_t)kMask) << b);
    const int64_t hi = (int64_t)((m >> kB) << b);
    int64_t t = 0;
    const int k = lane_id();
    if (k < n) {
        if (k == q) t = lo & kMask;
        if (k == q + 1) t = (lo >> kB) + (hi & kMask);
        if (k == q + 2) t = hi >> kB;
    }
    return negv ? -t : t;
}

// fx::xf_from_double
template <int N>
__device__ __forceinline__ wxf from_double(double v) {
    if ((fx::dbits(v) & 0x7fffffffffffffffULL) == 0) return zero();
    const int e = fx::floordiv24(fx::dmsb(v)) - 3;
    return from_acc<N, N + 2>(double_part<6>(v, e), e);
}

// fx::xf_from_md: every limb at the digit scale that puts the leading bit in
// digit N-1, summed by lanes, carried once.
template <int P, int N>
__device__ __forceinline__ wxf from_md(const md<P>& x) {
    int msb = -100000;
#pragma unroll
    for (int l = 0; l < P; ++l)
        if ((fx::dbits(x.v[l]) & 0x7fffffffffffffffULL) != 0) {
            const int m = fx::dmsb(x.v[l]);
            msb = m > msb ? m : msb;
        }
    if (msb == -100000) return zero();
    const int e = fx::floordiv24(msb) - (N - 1);
    int64_t mine = 0;
#pragma unroll
    for (int l = 0; l < P; ++l) mine += double_part<N + 2>(x.v[l], e);
    return from_acc<N, N + 2>(mine, e);
}

template <int N>
__device__ __forceinline__ wxf from_double_scaled(double y, int k) {
    wxf r = from_double<N>(y);
    if (!is_zero<N>(r)) r.e += k;
    return r;
}

// fx::xf_resize<K, N>: the leading digits kept, or zeros appended below.
template <int K, int N>
__device__ __forceinline__ wxf resize(const wxf& x) {
    const int k = lane_id(), s = k + N - K;
    const int32_t v = __shfl_sync(kFull, x.d, s & 31);
    const bool z = is_zero<N>(x);
    return wxf{(k < K && s >= 0 && s < N) ? v : 0, z ? 0 : x.e + N - K};
}

template <int N, int I>
__device__ __forceinline__ void recip_steps(const wxf& x, wxf& y) {
    if constexpr (I < fx::NewtonSteps<N>::value) {
        constexpr int K = fx::StepDigits<N, I>::value;
        const wxf xk = resize<K, N>(x), yk = resize<K, N>(y);
        const wxf t = sub<K>(from_int<K>(1), mul<K>(xk, yk));
        y = resize<N, K>(add<K>(yk, mul<K>(yk, t)));
        recip_steps<N, I + 1>(x, y);
    }
}

// fx::xf_recip: 1/x (x nonzero)
template <int N>
__device__ __noinline__ wxf recip(const wxf& x) {
    int k;
    const double m = lead<N>(x, k);
    wxf y = from_double_scaled<N>(1.0 / m, -k);
    recip_steps<N, 0>(x, y);
    return y;
}

template <int N, int I>
__device__ __forceinline__ void rsqrt_steps(const wxf& a, wxf& y) {
    if constexpr (I < fx::NewtonSteps<N>::value) {
        constexpr int K = fx::StepDigits<N, I>::value;
        const wxf ak = resize<K, N>(a), yk = resize<K, N>(y);
        wxf t = sub<K>(from_int<K>(1), mul<K>(ak, mul<K>(yk, yk)));
        t = shift_bits<K>(t, -1);
        y = resize<N, K>(add<K>(yk, mul<K>(yk, t)));
        rsqrt_steps<N, I + 1>(a, y);
    }
}

// fx::xf_rsqrt: 1/sqrt(a) (a > 0)
template <int N>
__device__ __noinline__ wxf rsqrt(const wxf& a) {
    int k;
    double m = lead<N>(a, k);
    if (k & 1) {
        m *= 16777216.0;
        k -= 1;
    }
    wxf y = from_double_scaled<N>(1.0 / sqrt(m), -(k / 2));
    rsqrt_steps<N, 0>(a, y);
    return y;
}

// fx::xf_house: the Householder scalars (Golub and Van Loan, Algorithm 5.1.1)
// of x = (x0, x_1, ...) from sigma = sum_{i>0} x_i^2; same outputs and kinds.
template <int N>
__device__ __noinline__ int house(const wxf& sig, const wxf& x0, wxf& v0, wxf& bp, wxf& rcc, wxf& inv_v0,
                                  wxf& beta) {
    if (is_zero<N>(sig)) {
        v0 = from_int<N>(1);
        inv_v0 = v0;
        if (sign<N>(x0) >= 0) {
            bp = zero();
            rcc = x0;
            beta = bp;
            return 1;
        }
        bp = from_int<N>(2);
        rcc = neg(x0);
        beta = bp;
        return 2;
    }
    const wxf a2 = add<N>(mul<N>(x0, x0), sig);
    const wxf rs = rsqrt<N>(a2);
    const wxf mu = mul<N>(a2, rs);
    if (sign<N>(x0) <= 0) {
        v0 = sub<N>(x0, mu);
        const wxf R = recip<N>(mul<N>(mu, v0));
        bp = neg(R);
        inv_v0 = mul<N>(mu, R);
    } else {
        const wxf sx = add<N>(x0, mu);
        const wxf R = recip<N>(mul<N>(sig, sx));
        v0 = neg(mul<N>(sig, mul<N>(sig, R)));
        const wxf s2R = mul<N>(sx, mul<N>(sx, R));
        inv_v0 = neg(s2R);
        bp = mul<N>(s2R, rs);
    }
    beta = mul<N>(mul<N>(bp, v0), v0);
    rcc = mu;
    return 0;
}

// fx::xf_from_fixed<N, D>: lane k < D holds digit k of the fixed-point value.
template <int N, int D>
__device__ __forceinline__ wxf from_fixed(int32_t dk, int e) {
    constexpr int M = (D > N ? D : N) + 1;
    return from_acc<N, M>(lane_id() < D ? (int64_t)dk : 0, e);
}

// fx::fixed_from_xf<N, D>: lane s < D receives digit s of x at scale e;
// returns false (in every lane) if a nonzero digit lands at D or above.
template <int N, int D>
__device__ __forceinline__ bool fixed_from_xf(const wxf& x, int e, int32_t& dk) {
    const int off = x.e - e;
    const int k = lane_id();
    const bool lost = k < N && k + off >= D && x.d != 0;
    const int src = k - off;
    const int32_t v = __shfl_sync(kFull, x.d, src & 31);
    dk = (k < D && src >= 0 && src < N) ? v : 0;
    return __ballot_sync(kFull, lost) == 0;
}

// The scalar form (every lane gets all digits).
template <int N>
__device__ __forceinline__ fx::xf<N> to_scalar(const wxf& x) {
    fx::xf<N> r;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = digit(x, k);
    r.e = x.e;
    return r;
}

template <int N>
__device__ __forceinline__ wxf from_scalar(const fx::xf<N>& x) {
    const int k = lane_id();
    int32_t v = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j == k) v = x.d[j];
    return wxf{v, x.e};
}

}  // namespace fxw
}  // namespace mdls
