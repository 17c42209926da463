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


// Integer-digit panel: 24-bit digits per entry for P limbs (53P bits plus 64
// of guard and headroom) and the ints of a column's published record; the
// device side (fx::Cfg, FxMeta) uses the same formulas.
constexpr int fx_digits(int P) { return (53 * P + 64 + 23) / 24; }
constexpr int fx_meta_ints(int P) { return 4 + 2 * (fx_digits(P) + 1); }

struct QrLayout {
    size_t flags, flag_bytes, beta, fxF, fxmeta, G, T, X, W, split, split_side;
    int64_t xcols, wcols, split_cap, split_side_cap;
    // tensor-core digit slices (split mode; caps 0 otherwise)
    size_t tc_as, tc_bs, tc_ea, tc_fb, tc_as_cap, tc_bs_cap;
    int64_t tc_sc_cap;
};

inline int split_slices(int P) { return (53 * P + 12 + 7) / 8; }
inline int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }
// Split matrix-vector partial sums of the back substitution (md values).
constexpr int64_t kBsPartCap = 4096;
struct BsLayout {
    size_t D, b, part;
    // persistent schedule of step 2 (tiles that are multiples of 32 wide):
    // the per-(chunk, slice) running sums, the two trees of partial sums of
    // the chain x_i -> x_{i-1} and the counters
    size_t acc, tree_cu, tree_xt, ctr;
    int64_t part_ps;  // doubles per plane of acc; the trees hold twice as many
};

// Persistent back substitution: columns per slice of its products, and the
// unsigned-int counters it needs (see csrc/bs_persist.cuh).
constexpr int kBsSliceCols = 8;
inline int64_t bs_ctr_ints(int64_t nchunks, int64_t S, int64_t N) {
    return 96 + 2 * 1024 + 3 * nchunks * S + 2 * N;
}

// Process-wide schedule of the back substitution's step 2 (MDLS_BS_*; set by
// mdls_set_backsub_schedule, defined in api.cu).
int& bs_schedule_ref();
int& split_engine_ref();
struct LsLayout {
    QrLayout qr;
    size_t Aw;
    BsLayout bs;
    size_t total;
};

inline QrLayout qr_layout_at(Bump& B, int P, int64_t m, int64_t n, int t, bool want_q, int nextra,
                             bool keep_w = false, bool split = false) {
    QrLayout L;
    L.flag_bytes = align256(2 * (size_t)t * sizeof(unsigned int));
    L.flags = B.take(L.flag_bytes);
    const size_t d = sizeof(double) * (size_t)P;
    L.beta = B.take(d * t);
    // integer-digit panel: the panel's digits and each column's record
    L.fxF = B.take(4 * (size_t)fx_digits(P) * (size_t)t * (size_t)m);
    L.fxmeta = B.take(4 * (size_t)fx_meta_ints(P) * (size_t)t);
    L.G = B.take(d * t * t);
    L.T = B.take(d * t * t);
    L.xcols = n + nextra;
    if (want_q && m > L.xcols) L.xcols = m;
    L.X = B.take(d * t * (size_t)L.xcols);
    // every tile's W, or two tiles' W: the next tile's W is formed beside
    // the current tile's trailing update, which still reads its own
    L.wcols = (want_q || keep_w) ? n : 2 * (int64_t)t;
    L.W = B.take(d * (size_t)m * (size_t)L.wcols);
    // split-K partial sums, md values per plane: room for 8 partial products
    // of a tile's W^T C (t x xcols), so that a product of one to two waves
    // can be split into whole waves
    L.split_cap = 16 * (int64_t)t * t;
    if (8 * (int64_t)t * L.xcols > L.split_cap) L.split_cap = 8 * (int64_t)t * L.xcols;
    L.split = B.take(d * (size_t)L.split_cap);
    // split-K partial sums of the next tile's G = Y^T Y on the side stream
    L.split_side_cap = 16 * (int64_t)t * t;
    L.split_side = B.take(d * (size_t)L.split_side_cap);
    L.tc_as = L.tc_bs = L.tc_ea = L.tc_fb = 0;
    L.tc_as_cap = L.tc_bs_cap = 0;
    L.tc_sc_cap = 0;
    if (split) {
        // A operands: W^T, Y^T (t x m) and Y, W (m x t); B operands: the trailing
        // columns and right-hand sides, Q (m x m), X, T, Y (K <= m)
        const int64_t S = split_slices(P), mp = round16(m), tp = round16(t);
        int64_t bcols = n + nextra;
        if (want_q && m > bcols) bcols = m;
        if (t > bcols) bcols = t;
        L.tc_as_cap = (size_t)S * (size_t)((t * mp > m * tp) ? t * mp : m * tp);
        L.tc_bs_cap = (size_t)S * (size_t)(bcols * mp);
        // the tcgen05 products' tiled slices: A rows padded to 128, B rows to
        // 16, one more B slice (octo double's padding slice)
        const int64_t m128 = (m + 127) / 128 * 128, t128 = (t + 127) / 128 * 128;
        const size_t tiled_a = (size_t)S * (size_t)((t128 * mp > m128 * tp) ? t128 * mp : m128 * tp);
        const size_t tiled_b = (size_t)(S + 1) * (size_t)(round16(bcols) * mp);
        if (tiled_a > L.tc_as_cap) L.tc_as_cap = tiled_a;
        if (tiled_b > L.tc_bs_cap) L.tc_bs_cap = tiled_b;
        L.tc_sc_cap = (m > bcols ? m : bcols);
        L.tc_as = B.take(2 * L.tc_as_cap);
        L.tc_bs = B.take(2 * L.tc_bs_cap);
        L.tc_ea = B.take(4 * (size_t)L.tc_sc_cap);
        L.tc_fb = B.take(4 * (size_t)L.tc_sc_cap);
    }
    return L;
}

inline BsLayout bs_layout_at(Bump& B, int P, int64_t n, int t) {
    BsLayout L;
    const size_t d = sizeof(double) * (size_t)P;
    const int64_t N = (n + t - 1) / t;
    L.D = B.take(d * (size_t)N * t * t);
    L.b = B.take(d * (size_t)n);
    L.part = B.take(d * (size_t)kBsPartCap);
    L.acc = L.tree_cu = L.tree_xt = L.ctr = 0;
    L.part_ps = 0;
    if (t % 32 == 0) {
        const int64_t nchunks = (n + 31) / 32, S = t / kBsSliceCols;
        L.part_ps = nchunks * S * 32;
        L.acc = B.take(d * (size_t)L.part_ps);
        L.tree_cu = B.take(2 * d * (size_t)L.part_ps);
        L.tree_xt = B.take(2 * d * (size_t)L.part_ps);
        L.ctr = B.take(4 * (size_t)bs_ctr_ints(nchunks, S, N));
    }
    return L;
}

inline QrLayout qr_layout(int P, int64_t m, int64_t n, int t, bool want_q, int nextra,
                          size_t* total = nullptr, bool split = false) {
    Bump B;
    QrLayout L = qr_layout_at(B, P, m, n, t, want_q, nextra, false, split);
    if (total) *total = B.off;
    return L;
}

inline BsLayout bs_layout(int P, int64_t n, int t, size_t* total = nullptr) {
    Bump B;
    BsLayout L = bs_layout_at(B, P, n, t);
    if (total) *total = B.off;
    return L;
}

// Least squares by double-double factorisation and refinement in P limbs:
// the dd QR of A (every tile's W kept; its WY products on the tensor cores,
// the digit slices included), dd back substitution, and the vectors of the
// refinement loop.
struct RefLayout {
    QrLayout qr;
    size_t A2, res, f, g, c, h, d, up;
    BsLayout bs;
    // digit slices of A and A^T in P limbs (the residual products b - A x
    // and A^T r on the tensor cores), of the vector operand, and the scales
    size_t dA, dAT, dv, eA, eAT, ev;
    size_t total;
};

inline RefLayout ref_layout(int P, int64_t m, int64_t n, int t) {
    Bump B;
    RefLayout L;
    L.qr = qr_layout_at(B, 2, m, n, t, false, 0, true, true);  // dd factorisation with split products
    const size_t d2 = 2 * sizeof(double), dP = (size_t)P * sizeof(double);
    L.A2 = B.take(d2 * (size_t)m * (size_t)n);
    L.res = B.take(dP * (size_t)m);
    L.f = B.take(dP * (size_t)m);
    L.g = B.take(dP * (size_t)n);
    L.c = B.take(d2 * (size_t)m);
    L.h = B.take(d2 * (size_t)n);
    L.d = B.take(d2 * (size_t)n);
    L.up = B.take(dP * (size_t)m);
    L.bs = bs_layout_at(B, 2, n, t);
    const int64_t S = split_slices(P), mp = round16(m), np = round16(n);
    L.dA = B.take(2 * (size_t)S * (size_t)m * (size_t)np);
    L.dAT = B.take(2 * (size_t)S * (size_t)n * (size_t)mp);
    L.dv = B.take(2 * (size_t)S * (size_t)(mp > np ? mp : np));
    L.eA = B.take(4 * (size_t)m);
    L.eAT = B.take(4 * (size_t)n);
    L.ev = B.take(4);
    L.total = B.off;
    return L;
}

inline LsLayout ls_layout(int P, int64_t m, int64_t n, int t, bool split = false) {
    Bump B;
    LsLayout L;
    L.qr = qr_layout_at(B, P, m, n, t, false, 1, false, split);
    L.Aw = B.take(sizeof(double) * (size_t)P * (size_t)m * (size_t)(n + 1));
    L.bs = bs_layout_at(B, P, n, t);
    L.total = B.off;
    return L;
}

// Back substitution alone: tile 0 = 128 in double and quad double, 64 in
// octo double.  Measured on GB300 (qd, n = 2560 .. 20480, tiles 32 .. 256):
// tile 128 is fastest at every n (n = 17920: 58.6 / 38.4 / 35.1 / 53.7 ms at
// tiles 32 / 64 / 128 / 256); in od the tile inversions (n t^2 / 6 md FMAs)
// dominate and tile 64 is faster (n = 2048: 14.1 against 18.9 ms).
inline int norm_tile_bs(int tile, int64_t n, int prec) {
    if (tile < 0 || tile > 256) return -1;
    int t = tile == 0 ? (prec == 8 ? 64 : 128) : tile;
    if (n > 0 && t > n) t = (int)n;
    return t;
}

// tile 0 = default; a tile wider than the problem is clipped to it
inline int norm_tile(int tile, int64_t n) {
    if (tile < 0 || tile > 256) return -1;
    int t = tile == 0 ? 128 : tile;
    if (n > 0 && t > n) t = (int)n;
    return t;
}

// Lower triangular block-Toeplitz solve: the QR of the diagonal block with
// every tile's W kept, its inverted diagonal tiles, and the work vector.
struct ToeLayout {
    QrLayout qr;
    size_t A2, r;
    BsLayout bs;
    size_t total;
};

inline ToeLayout toe_layout(int P, int64_t m, int64_t n, int t) {
    Bump B;
    ToeLayout L;
    L.qr = qr_layout_at(B, P, m, n, t, false, 0, true, false);
    L.A2 = B.take(sizeof(double) * (size_t)P * (size_t)m * (size_t)n);
    L.r = B.take(sizeof(double) * (size_t)P * (size_t)m);
    L.bs = bs_layout_at(B, P, n, t);
    L.total = B.off;
    return L;
}

// ---------------------------------------------------------------------------
// Complex md (real and imaginary planes) workspaces.
// ---------------------------------------------------------------------------
// Workspace of the complex QR.
struct ZqrLayout {
    size_t beta, v0r, v0i, wr, wi, Gr, Gi, Tr, Ti, Xr, Xi, Wr, Wi, Zr, Zi, split;
    int64_t xcols, wcols, split_cap;
};

inline ZqrLayout zqr_layout_at(Bump& B, int P, int64_t m, int64_t n, int t, bool want_q, int nextra) {
    ZqrLayout L;
    const size_t d = sizeof(double) * (size_t)P;
    L.beta = B.take(d * t);
    L.v0r = B.take(d * t);
    L.v0i = B.take(d * t);
    L.wr = B.take(d * t);
    L.wi = B.take(d * t);
    L.Gr = B.take(d * t * t);
    L.Gi = B.take(d * t * t);
    L.Tr = B.take(d * t * t);
    L.Ti = B.take(d * t * t);
    L.xcols = n + nextra;
    if (want_q && m > L.xcols) L.xcols = m;
    L.Xr = B.take(d * t * (size_t)L.xcols);
    L.Xi = B.take(d * t * (size_t)L.xcols);
    L.wcols = want_q ? n : t;
    L.Wr = B.take(d * (size_t)m * (size_t)L.wcols);
    L.Wi = B.take(d * (size_t)m * (size_t)L.wcols);
    L.Zr = B.take(d * t * t);
    L.Zi = B.take(d * t * t);
    L.split_cap = 16 * (int64_t)t * t;
    L.split = B.take(d * (size_t)L.split_cap);
    return L;
}

// Workspace of the complex back substitution: the inverted diagonal tiles,
// the working right-hand side, scratch for the level products and split-K.
struct ZbsLayout {
    size_t Dr, Di, br, bi, Zr, Zi, split;
    int64_t split_cap;
};

inline ZbsLayout zbs_layout_at(Bump& B, int P, int64_t n, int t) {
    ZbsLayout L;
    const size_t d = sizeof(double) * (size_t)P;
    const int64_t N = (n + t - 1) / t;
    L.Dr = B.take(d * (size_t)N * t * t);
    L.Di = B.take(d * (size_t)N * t * t);
    L.br = B.take(d * (size_t)n);
    L.bi = B.take(d * (size_t)n);
    L.Zr = B.take(d * (size_t)t * t);
    L.Zi = B.take(d * (size_t)t * t);
    L.split_cap = 16 * (int64_t)t * t > kBsPartCap ? 16 * (int64_t)t * t : kBsPartCap;
    L.split = B.take(d * (size_t)L.split_cap);
    return L;
}

inline ZqrLayout zqr_layout(int P, int64_t m, int64_t n, int t, bool want_q, size_t* total) {
    Bump B;
    ZqrLayout L = zqr_layout_at(B, P, m, n, t, want_q, 0);
    if (total) *total = B.off;
    return L;
}
inline ZbsLayout zbs_layout(int P, int64_t n, int t, size_t* total) {
    Bump B;
    ZbsLayout L = zbs_layout_at(B, P, n, t);
    if (total) *total = B.off;
    return L;
}
struct ZlsLayout {
    ZqrLayout qr;
    size_t Ar, Ai;
    ZbsLayout bs;
    size_t total;
};
inline ZlsLayout zls_layout(int P, int64_t m, int64_t n, int t) {
    Bump B;
    ZlsLayout L;
    L.qr = zqr_layout_at(B, P, m, n, t, false, 1);
    L.Ar = B.take(sizeof(double) * (size_t)P * (size_t)m * (size_t)(n + 1));
    L.Ai = B.take(sizeof(double) * (size_t)P * (size_t)m * (size_t)(n + 1));
    L.bs = zbs_layout_at(B, P, n, t);
    L.total = B.off;
    return L;
}

}  // namespace mdls
