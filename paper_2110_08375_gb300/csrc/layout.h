// Workspace layouts (host only).  Offsets are bytes from the start of the
// caller's workspace; every region starts on a 256-byte boundary.  Offset 0
// holds the 256-byte header (status word, barrier state).
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace mdls {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Bump {
    size_t off = 256;  // after the header
    size_t take(size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    }
};

struct QrLayout {
    size_t flags, flag_bytes, beta, G, T, X, W, split;
    int64_t xcols, wcols, split_cap;
};
struct BsLayout {
    size_t D, b;
};
struct LsLayout {
    QrLayout qr;
    size_t Aw;
    BsLayout bs;
    size_t total;
};

inline QrLayout qr_layout_at(Bump& B, int P, int64_t m, int64_t n, int t, bool want_q, int nextra) {
    QrLayout L;
    L.flag_bytes = align256((size_t)t * sizeof(unsigned int));
    L.flags = B.take(L.flag_bytes);
    const size_t d = sizeof(double) * (size_t)P;
    L.beta = B.take(d * t);
    L.G = B.take(d * t * t);
    L.T = B.take(d * t * t);
    L.xcols = n + nextra;
    if (want_q && m > L.xcols) L.xcols = m;
    L.X = B.take(d * t * (size_t)L.xcols);
    L.wcols = want_q ? n : t;
    L.W = B.take(d * (size_t)m * (size_t)L.wcols);
    L.split_cap = 16 * (int64_t)t * t;   // split-K partial sums, md values per plane
    L.split = B.take(d * (size_t)L.split_cap);
    return L;
}

inline BsLayout bs_layout_at(Bump& B, int P, int64_t n, int t) {
    BsLayout L;
    const size_t d = sizeof(double) * (size_t)P;
    const int64_t N = (n + t - 1) / t;
    L.D = B.take(d * (size_t)N * t * t);
    L.b = B.take(d * (size_t)n);
    return L;
}

inline QrLayout qr_layout(int P, int64_t m, int64_t n, int t, bool want_q, int nextra,
                          size_t* total = nullptr) {
    Bump B;
    QrLayout L = qr_layout_at(B, P, m, n, t, want_q, nextra);
    if (total) *total = B.off;
    return L;
}

inline BsLayout bs_layout(int P, int64_t n, int t, size_t* total = nullptr) {
    Bump B;
    BsLayout L = bs_layout_at(B, P, n, t);
    if (total) *total = B.off;
    return L;
}

inline LsLayout ls_layout(int P, int64_t m, int64_t n, int t) {
    Bump B;
    LsLayout L;
    L.qr = qr_layout_at(B, P, m, n, t, false, 1);
    L.Aw = B.take(sizeof(double) * (size_t)P * (size_t)m * (size_t)(n + 1));
    L.bs = bs_layout_at(B, P, n, t);
    L.total = B.off;
    return L;
}

// tile 0 = default; a tile wider than the problem is clipped to it
inline int norm_tile(int tile, int64_t n) {
    if (tile < 0 || tile > 256) return -1;
    int t = tile == 0 ? 128 : tile;
    if (n > 0 && t > n) t = (int)n;
    return t;
}

}  // namespace mdls
