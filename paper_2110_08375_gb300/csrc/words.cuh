// Exact sums of the split products' digit diagonals as multiword integers,
// and their rounding to P limbs, on the integer pipe only.
//
// A split product's value for one output is 2^e0 sum_g W[g] 2^(32 g) with
// int64 words W (unnormalised: each word may exceed 32 bits and be
// negative).  words::add_md adds an md value into the same words exactly (its
// bits below 2^e0 dropped toward zero: they lie below the product's own
// truncation), and words::to_md rounds the total toward zero to P limbs
// greedily: limb 0 is the leading 53 bits of |value|, limb l + 1 the leading
// 53 bits of what is left, so that the limbs are non-overlapping and every
// limb carries a full significand.  Every array index is a compile-time
// constant (positions found at run time select words by comparison), so the
// words stay in registers; a GB300 FP64 instruction holds its SM
// sub-partition for 64 cycles, an integer one for 2.
#pragma once
#include <stdint.h>

#include "fx.cuh"
#include "md.cuh"

namespace mdls {
namespace words {

// Adds the double v into sum_g W[g] 2^(32 g + e0) exactly, bits below 2^e0
// truncated toward zero.  The caller keeps v below 2^(e0 + 32 (GW - 1)).
template <int GW>
MD_INLINE void add_double(int64_t (&W)[GW], double v, int e0) {
    uint64_t u = fx::dbits(v);
    const bool neg = (u >> 63) != 0;
    u &= 0x7fffffffffffffffULL;
    if (u == 0) return;
    const int be = (int)(u >> 52);
    uint64_t m = u & ((uint64_t(1) << 52) - 1);
    int L;  // exponent of the significand's last bit
    if (be == 0) {
        L = -1074;
    } else {
        m |= uint64_t(1) << 52;
        L = be - 1075;
    }
    int pos = L - e0;
    if (pos < 0) {
        if (pos <= -53) return;
        m >>= -pos;
        pos = 0;
    }
    const int w = pos >> 5, sh = pos & 31;
    // m 2^sh < 2^85 in three 32-bit pieces (the shift's low 64 bits are exact)
    const uint64_t lo64 = m << sh;
    const int64_t p0 = (int64_t)(lo64 & 0xffffffffULL);
    const int64_t p1 = (int64_t)(lo64 >> 32);
    const int64_t p2 = sh ? (int64_t)(m >> (64 - sh)) : 0;
#pragma unroll
    for (int g = 0; g < GW; ++g) {
        int64_t add = 0;
        if (g == w) add = p0;
        if (g == w + 1) add = p1;
        if (g == w + 2) add = p2;
        W[g] += neg ? -add : add;
    }
}

template <int GW, int P>
MD_INLINE void add_md(int64_t (&W)[GW], const md<P>& x, int e0) {
#pragma unroll 1
    for (int l = 0; l < P; ++l) add_double<GW>(W, x.v[l], e0);  // rolled: one copy of the code
}

// Bits [lo, lo + 63] of the magnitude u (32-bit words, bits below 0 zero).
template <int GW>
MD_INLINE uint64_t window64(const uint32_t (&u)[GW], int lo) {
    uint64_t r = 0;
#pragma unroll
    for (int g = 0; g < GW; ++g) {
        const int s = 32 * g - lo;  // where word g's bit 0 lands in the window
        const uint64_t x = u[g];
        if (s >= 0 && s < 64) r |= x << s;
        else if (s < 0 && s > -32) r |= x >> (-s);
    }
    return r;
}

// Index of the highest set bit of u below bit `below` (-1 if none).
template <int GW>
MD_INLINE int top_below(const uint32_t (&u)[GW], int below) {
    int t = -1;
#pragma unroll
    for (int g = 0; g < GW; ++g) {
        uint32_t x = u[g];
        const int lo = 32 * g;
        if (below <= lo) x = 0;
        else if (below < lo + 32) x &= (uint32_t)((1ULL << (below - lo)) - 1);
        if (x != 0) t = lo + fx::bitlen64(x) - 1;
    }
    return t;
}

// The value 2^e0 sum_g W[g] 2^(32 g), negated when `negate`, rounded toward
// zero to P limbs as described above.  |value| < 2^(e0 + 32 GW - 1).
template <int P, int GW>
MD_INLINE md<P> to_md(const int64_t (&W)[GW], int e0, bool negate) {
    uint32_t u[GW];
    int64_t carry = 0;
#pragma unroll
    for (int g = 0; g < GW; ++g) {
        const int64_t t = W[g] + carry;
        u[g] = (uint32_t)(uint64_t)t;
        carry = t >> 32;
    }
    bool neg = carry < 0;  // two's complement over GW words
    if (neg) {
        uint64_t c = 1;
#pragma unroll
        for (int g = 0; g < GW; ++g) {
            const uint64_t t = (uint64_t)(uint32_t)~u[g] + c;
            u[g] = (uint32_t)t;
            c = t >> 32;
        }
    }
    if (negate) neg = !neg;
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = 0.0;
    int cur = top_below<GW>(u, 32 * GW);
#pragma unroll 1
    for (int l = 0; l < P; ++l) {  // rolled: one copy of the code
        if (cur >= 0) {
            const int lo = cur - 52;
            const uint64_t chunk = window64<GW>(u, lo) & ((uint64_t(1) << 53) - 1);  // bit 52 set
            const int be = lo + e0 + 1075;                                           // biased exponent
            if (be <= 0) {  // subnormal: truncated, nothing representable below it
                const int sh = 1 - be;
                if (sh < 53) r.v[l] = fx::dfrom(((uint64_t)neg << 63) | (chunk >> sh));
                cur = -1;
            } else if (be >= 2047) {
                r.v[l] = fx::dfrom(((uint64_t)neg << 63) | (uint64_t(0x7ff) << 52));
                cur = -1;
            } else {
                r.v[l] = fx::dfrom(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (chunk & ((uint64_t(1) << 52) - 1)));
                cur = top_below<GW>(u, lo);
            }
        }
    }
    return r;
}

}  // namespace words
}  // namespace mdls
