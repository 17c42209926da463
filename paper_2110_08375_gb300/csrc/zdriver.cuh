// Complex multiple-double QR, back substitution and least squares: the
// paper's algorithms on complex data (Section 3: the transpose becomes the
// Hermitian transpose; Section 2: real and imaginary parts are kept
// separately).  A complex md matrix is two real md matrices of the same
// layout, its real part and its imaginary part.
//
// Householder reflectors are Hermitian, H = I - beta v v^H with beta real and
// v(0) = 1; H x = rho e1 with rho = e^{i arg x0} ||x|| (Golub and Van Loan's
// Alg. 5.1.1 with the sign of the real case replaced by the phase of x0, so
// that the diagonal of R carries the phases of the reflected columns'
// leading entries).  The compact WY form of a tile is H_1 ... H_w =
// I - Y T Y^H = I + W Y^H with W = -Y T; the trailing update is
// C := C + Y (W^H C) and Q is accumulated backward, Q := Q + W (Y^H Q).
//
// The WY products -- Y^H Y, W = -Y T, W^H C, C + Y X, Y^H Q, Q + W X, the
// block combinations of T and of the inverted diagonal tiles, and the
// matrix-vector products of the back substitution -- each run as four real md
// products (launch_gemm: the tuned real kernels) on the separate planes.
// The panel (one column at a time: norm and reflector, scaling, dot
// products, update) and the 16-wide leaves of T and of the tile inverses are
// complex kernels of their own.
#pragma once
#include "driver.cuh"

namespace mdls {

// Imaginary part of the unit lower trapezoid Y: Y(i, k) stored for i > k,
// zero on and above the diagonal.
struct ViewTrapIm {
    static constexpr bool kRowContig = true;
    static constexpr bool kZeroKBelowI = false, kZeroKAboveI = true;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const { return i > k ? ptr[l * ps + k * ld + i] : 0.0; }
};
struct ViewTrapImT {  // its transpose
    static constexpr bool kRowContig = false;
    static constexpr bool kZeroKBelowI = true, kZeroKAboveI = false;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const { return k > i ? ptr[l * ps + i * ld + k] : 0.0; }
};

// Complex md matrix in two planes sets with one layout.
struct ZDense {
    double* re;
    double* im;
    int64_t ld, ps;
    __host__ __device__ Dense r() const { return Dense{re, ld, ps}; }
    __host__ __device__ Dense i() const { return Dense{im, ld, ps}; }
    __host__ __device__ ZDense at(int64_t row, int64_t col) const {
        return ZDense{re + col * ld + row, im + col * ld + row, ld, ps};
    }
};

template <int P>
struct zmd {
    md<P> re, im;
};

template <int P>
DEV_INLINE zmd<P> zld(const ZDense& a, int64_t off) {
    return zmd<P>{ld_md<P>(a.re, a.ps, off), ld_md<P>(a.im, a.ps, off)};
}
template <int P>
DEV_INLINE void zst(const ZDense& a, int64_t off, const zmd<P>& v) {
    st_md<P>(a.re, a.ps, off, v.re);
    st_md<P>(a.im, a.ps, off, v.im);
}
template <int P>
DEV_INLINE zmd<P> zmul(const zmd<P>& a, const zmd<P>& b) {
    return zmd<P>{md_fms<P>(md_mul<P>(a.re, b.re), a.im, b.im), md_fma<P>(md_mul<P>(a.re, b.im), a.im, b.re)};
}
template <int P>
DEV_INLINE zmd<P> zsub(const zmd<P>& a, const zmd<P>& b) {
    return zmd<P>{md_sub<P>(a.re, b.re), md_sub<P>(a.im, b.im)};
}
template <int P>
DEV_INLINE zmd<P> zadd(const zmd<P>& a, const zmd<P>& b) {
    return zmd<P>{md_add<P>(a.re, b.re), md_add<P>(a.im, b.im)};
}
template <int P>
DEV_INLINE zmd<P> zzero() {
    return zmd<P>{md_zero<P>(), md_zero<P>()};
}
// 1 / a = conj(a) / |a|^2
template <int P>
DEV_INLINE zmd<P> zinv(const zmd<P>& a) {
    const md<P> d = md_fma<P>(md_mul<P>(a.re, a.re), a.im, a.im);
    return zmd<P>{md_div<P>(a.re, d), md_neg<P>(md_div<P>(a.im, d))};
}

// Fixed-order block sum of one md value per thread (blockDim.x a power of
// two, at most 256); the total is returned to thread 0.
template <int P>
DEV_INLINE md<P> block_sum(md<P> v, md<P>* red) {
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] = md_add<P>(red[tid], red[tid + h]);
        __syncthreads();
    }
    const md<P> r = red[0];
    __syncthreads();
    return r;
}

// Scalars of one reflector, written by zhouse_kernel: 1 / v0 (complex) and
// beta (real), in P planes of stride sps.
struct ZScal {
    double* v0inv_re;
    double* v0inv_im;
    double* beta;
    int64_t sps;
};

// Panel step 1 (one block): sigma = sum_{i > 0} |x_i|^2 over the column
// below row0, then the reflector of x = A[row0:m, col]: rho into A(row0, col),
// 1 / v0 and beta into the scalars (slot c).  sigma = 0: H = I (beta = 0,
// 1 / v0 = 0 so that v's entries below row0 become 0) and rho = x0.
template <int P>
__global__ void __launch_bounds__(256) zhouse_kernel(ZDense A, int64_t m, int64_t row0, int64_t col, ZScal s, int c) {
    __shared__ md<P> red[256];
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    int cnt = 0;
    for (int64_t i = row0 + 1 + threadIdx.x; i < m; i += blockDim.x) {
        const zmd<P> x = zld<P>(A, col * A.ld + i);
        md_fma_bins<P>(bins, x.re, x.re);
        md_fma_bins<P>(bins, x.im, x.im);
        if ((++cnt & 7) == 0) md_bins_renorm<P>(bins);
    }
    const md<P> sigma = block_sum<P>(md_from_bins<P>(bins), red);
    if (threadIdx.x != 0) return;
    const int64_t o0 = col * A.ld + row0;
    const zmd<P> x0 = zld<P>(A, o0);
    if (sigma.v[0] == 0.0) {
        st_md<P>(s.beta, s.sps, c, md_zero<P>());
        st_md<P>(s.v0inv_re, s.sps, c, md_zero<P>());
        st_md<P>(s.v0inv_im, s.sps, c, md_zero<P>());
        return;  // rho = x0 stays in place
    }
    const md<P> a2 = md_fma<P>(md_mul<P>(x0.re, x0.re), x0.im, x0.im);
    const md<P> mu = md_sqrt<P>(md_add<P>(a2, sigma));
    zmd<P> ph;
    md<P> ax = md_zero<P>();
    if (a2.v[0] == 0.0) {
        ph = zmd<P>{md_from_double<P>(1.0), md_zero<P>()};
    } else {
        ax = md_sqrt<P>(a2);
        ph = zmd<P>{md_div<P>(x0.re, ax), md_div<P>(x0.im, ax)};
    }
    const md<P> q = md_div<P>(sigma, md_add<P>(ax, mu));  // |v0|
    const zmd<P> v0 = zmd<P>{md_neg<P>(md_mul<P>(ph.re, q)), md_neg<P>(md_mul<P>(ph.im, q))};
    const md<P> v0a2 = md_fma<P>(md_mul<P>(v0.re, v0.re), v0.im, v0.im);
    md<P> beta = md_div<P>(v0a2, md_add<P>(sigma, v0a2));
#pragma unroll
    for (int l = 0; l < P; ++l) beta.v[l] *= 2.0;
    const zmd<P> vi = zinv<P>(v0);
    st_md<P>(s.beta, s.sps, c, beta);
    st_md<P>(s.v0inv_re, s.sps, c, vi.re);
    st_md<P>(s.v0inv_im, s.sps, c, vi.im);
    zst<P>(A, o0, zmd<P>{md_mul<P>(ph.re, mu), md_mul<P>(ph.im, mu)});
}

// Panel step 2: v_i = x_i / v0 for rows below row0 (stored in place).
template <int P>
__global__ void zscale_kernel(ZDense A, int64_t m, int64_t row0, int64_t col, ZScal s, int c) {
    const int64_t i = row0 + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const zmd<P> vi{ld_md<P>(s.v0inv_re, s.sps, c), ld_md<P>(s.v0inv_im, s.sps, c)};
    const int64_t off = col * A.ld + i;
    zst<P>(A, off, zmul<P>(zld<P>(A, off), vi));
}

// Panel step 3 (block j of the grid for column col + 1 + j): w_j =
// beta sum_{i >= row0} conj(v_i) A(i, col + 1 + j) with v(row0) = 1.
template <int P>
__global__ void __launch_bounds__(256) zpanel_dot_kernel(ZDense A, int64_t m, int64_t row0, int64_t col, ZScal s,
                                                          int c, ZDense w) {
    __shared__ md<P> red[256];
    const int64_t cj = col + 1 + blockIdx.x;
    double br[P], bi[P];
#pragma unroll
    for (int l = 0; l < P; ++l) br[l] = bi[l] = 0.0;
    int cnt = 0;
    for (int64_t i = row0 + threadIdx.x; i < m; i += blockDim.x) {
        const zmd<P> a = zld<P>(A, cj * A.ld + i);
        if (i == row0) {
#pragma unroll
            for (int l = 0; l < P; ++l) {
                br[l] = a.re.v[l];
                bi[l] = a.im.v[l];
            }
            continue;
        }
        const zmd<P> v = zld<P>(A, col * A.ld + i);
        md_fma_bins<P>(br, v.re, a.re);  // re: vr ar + vi ai
        md_fma_bins<P>(br, v.im, a.im);
        md_fma_bins<P>(bi, v.re, a.im);  // im: vr ai - vi ar
        md_fma_bins<P>(bi, md_neg<P>(v.im), a.re);
        if ((++cnt & 7) == 0) {
            md_bins_renorm<P>(br);
            md_bins_renorm<P>(bi);
        }
    }
    const md<P> sr = block_sum<P>(md_from_bins<P>(br), red);
    const md<P> si = block_sum<P>(md_from_bins<P>(bi), red);
    if (threadIdx.x != 0) return;
    const md<P> beta = ld_md<P>(s.beta, s.sps, c);
    st_md<P>(w.re, w.ps, blockIdx.x, md_mul<P>(beta, sr));
    st_md<P>(w.im, w.ps, blockIdx.x, md_mul<P>(beta, si));
}

// Panel step 4: A(i, col + 1 + j) -= v_i w_j for rows i >= row0 (v(row0) = 1).
template <int P>
__global__ void zpanel_update_kernel(ZDense A, int64_t m, int64_t row0, int64_t col, int ncols, ZDense w) {
    const int64_t i = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= m || j >= ncols) return;
    const zmd<P> wj{ld_md<P>(w.re, w.ps, j), ld_md<P>(w.im, w.ps, j)};
    const int64_t off = (col + 1 + j) * A.ld + i;
    const zmd<P> a = zld<P>(A, off);
    if (i == row0) {
        zst<P>(A, off, zsub<P>(a, wj));
        return;
    }
    const zmd<P> v = zld<P>(A, col * A.ld + i);
    zst<P>(A, off, zsub<P>(a, zmul<P>(v, wj)));
}

// Leaves of T (one block of L threads per L x L diagonal block, thread l
// owns row l of the leaf): T[l,l] = beta_l, T[l,j] = -beta_j sum_{q=l}^{j-1}
// T[l,q] G[q,j] for l < j < leaf end (G = Y^H Y, upper part read).
template <int P>
__global__ void zwy_t_leaf_kernel(ZDense G, const double* beta, int64_t bps, int w, int L, ZDense T) {
    const int leaf0 = blockIdx.x * L;
    const int l = leaf0 + threadIdx.x;
    const int le = (leaf0 + L) < w ? (leaf0 + L) : w;
    if (l >= le) return;
    zmd<P> row[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) row[q] = zzero<P>();
    row[l - leaf0] = zmd<P>{ld_md<P>(beta, bps, l), md_zero<P>()};
    for (int j = l + 1; j < le; ++j) {
        zmd<P> acc = zzero<P>();
        for (int q = l; q < j; ++q) {
            zmd<P> tq;
#pragma unroll
            for (int qq = 0; qq < 16; ++qq)
                if (qq == q - leaf0) tq = row[qq];
            acc = zadd<P>(acc, zmul<P>(tq, zld<P>(G, (int64_t)j * G.ld + q)));
        }
        const md<P> bj = ld_md<P>(beta, bps, j);
        const zmd<P> tj{md_neg<P>(md_mul<P>(bj, acc.re)), md_neg<P>(md_mul<P>(bj, acc.im))};
#pragma unroll
        for (int qq = 0; qq < 16; ++qq)
            if (qq == j - leaf0) row[qq] = tj;
    }
    for (int q = l; q < le; ++q) {
        zmd<P> tq;
#pragma unroll
        for (int qq = 0; qq < 16; ++qq)
            if (qq == q - leaf0) tq = row[qq];
        zst<P>(T, (int64_t)q * T.ld + l, tq);
    }
}

// Leaves of the inverses of the diagonal tiles of a complex upper triangular
// R: thread c of block (tile, leaf) solves U v = e_c within the leaf
// (v_c = 1 / U_cc, v_l = -(sum_{q=l+1}^{c} U_lq v_q) / U_ll), writing column
// c of the leaf's inverse into D (tile at D + tile * dtile, ld dld).  A zero
// pivot records MDLS_ERR_SINGULAR.
template <int P>
__global__ void ztri_leaf_inv_kernel(ZDense U, int64_t n, int t, int L, ZDense D, int64_t dtile, WsHeader* hdr) {
    const int64_t tile = blockIdx.y;
    const int64_t o = tile * t;
    const int tt = (int)((n - o) < t ? (n - o) : t);
    const int leaf0 = blockIdx.x * L;
    const int c = leaf0 + threadIdx.x;
    const int le = (leaf0 + L) < tt ? (leaf0 + L) : tt;
    if (leaf0 >= tt || c >= le) return;
    const ZDense Ut = U.at(o, o);
    const ZDense Dt{D.re + tile * dtile, D.im + tile * dtile, D.ld, D.ps};
    zmd<P> v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = zzero<P>();
    const zmd<P> ucc = zld<P>(Ut, (int64_t)c * Ut.ld + c);
    if (ucc.re.v[0] == 0.0 && ucc.im.v[0] == 0.0) {
        set_status(&hdr->status, MDLS_ERR_SINGULAR);
        return;
    }
#pragma unroll
    for (int qq = 0; qq < 16; ++qq)
        if (qq == c - leaf0) v[qq] = zinv<P>(ucc);
    for (int l = c - 1; l >= leaf0; --l) {
        zmd<P> acc = zzero<P>();
        for (int q = l + 1; q <= c; ++q) {
            zmd<P> vq;
#pragma unroll
            for (int qq = 0; qq < 16; ++qq)
                if (qq == q - leaf0) vq = v[qq];
            acc = zadd<P>(acc, zmul<P>(zld<P>(Ut, (int64_t)q * Ut.ld + l), vq));
        }
        const zmd<P> ull = zld<P>(Ut, (int64_t)l * Ut.ld + l);
        if (ull.re.v[0] == 0.0 && ull.im.v[0] == 0.0) {
            set_status(&hdr->status, MDLS_ERR_SINGULAR);
            return;
        }
        const zmd<P> r = zmul<P>(acc, zinv<P>(ull));
#pragma unroll
        for (int qq = 0; qq < 16; ++qq)
            if (qq == l - leaf0) v[qq] = zmd<P>{md_neg<P>(r.re), md_neg<P>(r.im)};
    }
    for (int q = leaf0; q <= c; ++q) {
        zmd<P> vq;
#pragma unroll
        for (int qq = 0; qq < 16; ++qq)
            if (qq == q - leaf0) vq = v[qq];
        zst<P>(Dt, (int64_t)c * Dt.ld + q, vq);
    }
}

// Zeroes a complex matrix's strictly lower part, or sets it to the identity.
template <int P>
int zzero_lower(cudaStream_t st, ZDense A, int64_t m, int64_t n) {
    dim3 g((unsigned)((m + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    StageScope sc(ST_OTHER, st);
    zero_lower_kernel<P><<<g, 256, 0, st>>>(A.re, A.ld, A.ps, m, n);
    MDLS_LAUNCH_CHECK();
    zero_lower_kernel<P><<<g, 256, 0, st>>>(A.im, A.ld, A.ps, m, n);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// C = [C] +/- op(A) B as four real md products on the planes; op(A) = A or,
// with conj_a, the entrywise conjugate of A (its imaginary view negated):
//   Cr = [Cr] +/- (Ar Br -/+ Ai Bi),  Ci = [Ci] +/- (Ar Bi +/- Ai Br).
template <int P, class AR, class AI, class BR, class BI>
int zgemm(int stage, cudaStream_t st, SplitBuf sb, int64_t M, int64_t N, int64_t K, AR ar, AI ai, bool conj_a,
          BR br, BI bi, ZDense c, bool neg, bool acc) {
    int rc = launch_gemm<P>(stage, st, sb, M, N, K, ar, br, c.r(), neg, acc);
    if (rc) return rc;
    rc = launch_gemm<P>(stage, st, sb, M, N, K, ai, bi, c.r(), neg != !conj_a, true);
    if (rc) return rc;
    rc = launch_gemm<P>(stage, st, sb, M, N, K, ar, bi, c.i(), neg, acc);
    if (rc) return rc;
    return launch_gemm<P>(stage, st, sb, M, N, K, ai, br, c.i(), neg != conj_a, true);
}

// X12 = -X1 M12 X2 level by level (leaves of size L in place), for the
// upper triangular diagonal blocks of `ntiles` tiles of width t: T of the WY
// form (M = G) or the inverted tiles (M = U).  Z (t x t) is scratch.
template <int P>
int ztri_levels(int stage, cudaStream_t st, SplitBuf sb, ZDense X, int64_t xtile, ZDense M, int64_t mtile, int64_t n,
                int t, int64_t ntiles, int L, ZDense Z) {
    for (int64_t b = 0; b < ntiles; ++b) {
        const int64_t tt = (n - b * t) < t ? (n - b * t) : t;
        const ZDense Xb{X.re + b * xtile, X.im + b * xtile, X.ld, X.ps};
        const ZDense Mb{M.re + b * mtile, M.im + b * mtile, M.ld, M.ps};
        for (int s = L; s < tt; s *= 2) {
            for (int64_t a = 0; a + s < tt; a += 2 * s) {
                const int64_t s2 = (tt - a - s) < s ? (tt - a - s) : s;
                const ZDense X1 = Xb.at(a, a), X2 = Xb.at(a + s, a + s), M12 = Mb.at(a, a + s), X12 = Xb.at(a, a + s);
                // Z = M12 X2 (X2 upper triangular)
                int rc = zgemm<P>(stage, st, sb, s, s2, s2, ViewDense{M12.re, M12.ld, M12.ps},
                                  ViewDense{M12.im, M12.ld, M12.ps}, false, ViewUpper{X2.re, X2.ld, X2.ps},
                                  ViewUpper{X2.im, X2.ld, X2.ps}, Z, false, false);
                if (rc) return rc;
                // X12 = -X1 Z (X1 upper triangular)
                rc = zgemm<P>(stage, st, sb, s, s2, s, ViewUpper{X1.re, X1.ld, X1.ps}, ViewUpper{X1.im, X1.ld, X1.ps},
                              false, ViewDense{Z.re, Z.ld, Z.ps}, ViewDense{Z.im, Z.ld, Z.ps}, X12, true, false);
                if (rc) return rc;
            }
        }
    }
    return MDLS_OK;
}

// Blocked complex Householder QR of the m x n leading part of A; columns
// n .. n+nextra-1 receive the same transformations (Q^H b).  Q (m x m) is
// formed when Q.re != nullptr.  R stays in the upper triangle, Y below it.
template <int P>
int zqr_run(int64_t m, int64_t n, int nextra, ZDense A, ZDense Q, int t, char* ws, const ZqrLayout& L,
            WsHeader* hdr, bool zero_lower, cudaStream_t st) {
    (void)hdr;
    const int64_t tt2 = (int64_t)t * t;
    const ZScal sc{reinterpret_cast<double*>(ws + L.v0r), reinterpret_cast<double*>(ws + L.v0i),
                   reinterpret_cast<double*>(ws + L.beta), (int64_t)t};
    const ZDense wv{reinterpret_cast<double*>(ws + L.wr), reinterpret_cast<double*>(ws + L.wi), 1, t};
    const ZDense G{reinterpret_cast<double*>(ws + L.Gr), reinterpret_cast<double*>(ws + L.Gi), t, tt2};
    const ZDense T{reinterpret_cast<double*>(ws + L.Tr), reinterpret_cast<double*>(ws + L.Ti), t, tt2};
    const ZDense Z{reinterpret_cast<double*>(ws + L.Zr), reinterpret_cast<double*>(ws + L.Zi), t, tt2};
    const int64_t psx = (int64_t)t * L.xcols;
    const ZDense X{reinterpret_cast<double*>(ws + L.Xr), reinterpret_cast<double*>(ws + L.Xi), t, psx};
    const int64_t psw = L.wcols * m;
    const ZDense Wb{reinterpret_cast<double*>(ws + L.Wr), reinterpret_cast<double*>(ws + L.Wi), m, psw};
    const SplitBuf sb{reinterpret_cast<double*>(ws + L.split), L.split_cap, nullptr, true};
    const int64_t ntiles = (n + t - 1) / t;
    const bool want_q = Q.re != nullptr;
    for (int64_t k = 0; k < ntiles; ++k) {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        // 1. panel: the tile's columns one at a time
        for (int c = 0; c < w; ++c) {
            const int64_t col = j0 + c, row0 = j0 + c;
            StageScope s(ST_PANEL, st);
            zhouse_kernel<P><<<1, 256, 0, st>>>(A, m, row0, col, sc, c);
            MDLS_LAUNCH_CHECK();
            if (m - row0 - 1 > 0) {
                zscale_kernel<P><<<(unsigned)((m - row0 - 1 + 127) / 128), 128, 0, st>>>(A, m, row0, col, sc, c);
                MDLS_LAUNCH_CHECK();
            }
            const int rest = w - c - 1;
            if (rest > 0) {
                zpanel_dot_kernel<P><<<rest, 256, 0, st>>>(A, m, row0, col, sc, c, wv);
                MDLS_LAUNCH_CHECK();
                dim3 g((unsigned)((m - row0 + 127) / 128), (unsigned)rest);
                zpanel_update_kernel<P><<<g, 128, 0, st>>>(A, m, row0, col, rest, wv);
                MDLS_LAUNCH_CHECK();
            }
        }
        const int64_t nc = n + nextra - (j0 + w);
        if (nc <= 0 && !want_q) continue;
        // 2. WY form: G = Y^H Y (upper part), T by leaves and levels, W = -Y T
        const ZDense Yp = A.at(j0, j0);
        const ViewTrap Yr{Yp.re, Yp.ld, Yp.ps};
        const ViewTrapIm Yi{Yp.im, Yp.ld, Yp.ps};
        const ViewTrapT Yrt{Yp.re, Yp.ld, Yp.ps};
        const ViewTrapImT Yit{Yp.im, Yp.ld, Yp.ps};
        int rc;
        {
            // G = (Yr^T - i Yi^T)(Yr + i Yi)
            rc = launch_gemm<P>(ST_W, st, sb, w, w, r, Yrt, Yr, G.r(), false, false, true);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_W, st, sb, w, w, r, Yit, Yi, G.r(), false, true, true);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_W, st, sb, w, w, r, Yrt, Yi, G.i(), false, false, true);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_W, st, sb, w, w, r, Yit, Yr, G.i(), true, true, true);
            if (rc) return rc;
        }
        {
            const int Lf = w < kTriLeaf ? w : kTriLeaf;
            StageScope s(ST_W, st);
            if (cudaMemsetAsync(T.re, 0, sizeof(double) * (size_t)P * tt2, st) != cudaSuccess ||
                cudaMemsetAsync(T.im, 0, sizeof(double) * (size_t)P * tt2, st) != cudaSuccess)
                return MDLS_ERR_CUDA;
            zwy_t_leaf_kernel<P><<<(unsigned)((w + Lf - 1) / Lf), Lf, 0, st>>>(G, sc.beta, sc.sps, w, Lf, T);
            MDLS_LAUNCH_CHECK();
            rc = ztri_levels<P>(ST_W, st, sb, T, 0, G, 0, w, t, 1, Lf, Z);
            if (rc) return rc;
        }
        const ZDense Wk = want_q ? Wb.at(j0, j0) : Wb;
        rc = zgemm<P>(ST_W, st, sb, r, w, w, Yr, Yi, false, ViewUpper{T.re, T.ld, T.ps}, ViewUpper{T.im, T.ld, T.ps},
                      Wk, true, false);
        if (rc) return rc;
        // 3. trailing update C := C + Y (W^H C)
        if (nc > 0) {
            const ZDense Cp = A.at(j0, j0 + w);
            rc = zgemm<P>(ST_TRAIL, st, sb, w, nc, r, ViewDenseT{Wk.re, Wk.ld, Wk.ps}, ViewDenseT{Wk.im, Wk.ld, Wk.ps},
                          true, ViewDense{Cp.re, Cp.ld, Cp.ps}, ViewDense{Cp.im, Cp.ld, Cp.ps}, X, false, false);
            if (rc) return rc;
            rc = zgemm<P>(ST_TRAIL, st, sb, r, nc, w, Yr, Yi, false, ViewDense{X.re, X.ld, X.ps},
                          ViewDense{X.im, X.ld, X.ps}, Cp, false, true);
            if (rc) return rc;
        }
    }
    if (want_q) {
        // 4. Q = P_1 ... P_N backward: Q_sub := Q_sub + W (Y^H Q_sub)
        {
            dim3 g((unsigned)((m + 255) / 256), (unsigned)(m < 65535 ? m : 65535));
            StageScope s(ST_OTHER, st);
            identity_kernel<P><<<g, 256, 0, st>>>(Q.re, Q.ld, Q.ps, m);
            MDLS_LAUNCH_CHECK();
            if (cudaMemsetAsync(Q.im, 0, sizeof(double) * (size_t)((P - 1) * Q.ps + Q.ld * m), st) != cudaSuccess)
                return MDLS_ERR_CUDA;
        }
        for (int64_t k = ntiles - 1; k >= 0; --k) {
            const int64_t j0 = k * t;
            const int w = (int)((n - j0) < t ? (n - j0) : t);
            const int64_t r = m - j0;
            const ZDense Yp = A.at(j0, j0);
            const ZDense Qs = Q.at(j0, j0);
            const ZDense Wk = Wb.at(j0, j0);
            int rc = zgemm<P>(ST_QACC, st, sb, w, r, r, ViewTrapT{Yp.re, Yp.ld, Yp.ps}, ViewTrapImT{Yp.im, Yp.ld, Yp.ps},
                              true, ViewDense{Qs.re, Qs.ld, Qs.ps}, ViewDense{Qs.im, Qs.ld, Qs.ps}, X, false, false);
            if (rc) return rc;
            rc = zgemm<P>(ST_QACC, st, sb, r, r, w, ViewDense{Wk.re, Wk.ld, Wk.ps}, ViewDense{Wk.im, Wk.ld, Wk.ps},
                          false, ViewDense{X.re, X.ld, X.ps}, ViewDense{X.im, X.ld, X.ps}, Qs, false, true);
            if (rc) return rc;
        }
    }
    if (zero_lower) return zzero_lower<P>(st, A, m, n);
    return MDLS_OK;
}

// Algorithm 1 on complex data: invert the diagonal tiles (leaves, then the
// levels X12 = -X1 U12 X2), then for i = N..1: x_i = U_i^{-1} y_i and
// y_j -= R_{j,i} x_i for all j < i at once.
template <int P>
int zbs_run(int64_t n, ZDense R, ZDense y, ZDense x, int t, char* ws, const ZbsLayout& L, WsHeader* hdr,
            cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t tt2 = (int64_t)t * t;
    const ZDense D{reinterpret_cast<double*>(ws + L.Dr), reinterpret_cast<double*>(ws + L.Di), t, N * tt2};
    const ZDense bw{reinterpret_cast<double*>(ws + L.br), reinterpret_cast<double*>(ws + L.bi), n, n};
    const ZDense Z{reinterpret_cast<double*>(ws + L.Zr), reinterpret_cast<double*>(ws + L.Zi), t, tt2};
    const SplitBuf sb{reinterpret_cast<double*>(ws + L.split), L.split_cap, nullptr, true};
    const int leaf = t < kTriLeaf ? t : kTriLeaf;
    {
        StageScope s(ST_INV, st);
        if (cudaMemsetAsync(D.re, 0, sizeof(double) * (size_t)P * N * tt2, st) != cudaSuccess ||
            cudaMemsetAsync(D.im, 0, sizeof(double) * (size_t)P * N * tt2, st) != cudaSuccess)
            return MDLS_ERR_CUDA;
        dim3 g((unsigned)((t + leaf - 1) / leaf), (unsigned)N);
        ztri_leaf_inv_kernel<P><<<g, leaf, 0, st>>>(R, n, t, leaf, D, tt2, hdr);
        MDLS_LAUNCH_CHECK();
    }
    int rc = ztri_levels<P>(ST_INV, st, sb, D, tt2, R, (int64_t)t * (R.ld + 1), n, t, N, leaf, Z);
    if (rc) return rc;
    for (int l = 0; l < P; ++l) {
        if (cudaMemcpyAsync(bw.re + l * n, y.re + l * y.ps, n * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(bw.im + l * n, y.im + l * y.ps, n * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            return MDLS_ERR_CUDA;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        const int64_t o = i * t;
        const int tt = (int)((n - o) < t ? (n - o) : t);
        const ZDense Di{D.re + i * tt2, D.im + i * tt2, t, D.ps};
        const ZDense xo = x.at(o, 0);
        rc = zgemm<P>(ST_MULINV, st, sb, tt, 1, tt, ViewUpper{Di.re, Di.ld, Di.ps}, ViewUpper{Di.im, Di.ld, Di.ps},
                      false, ViewDense{bw.re + o, n, n}, ViewDense{bw.im + o, n, n},
                      ZDense{xo.re, xo.im, n, x.ps}, false, false);
        if (rc) return rc;
        if (o > 0) {
            const ZDense Rc = R.at(0, o);
            rc = zgemm<P>(ST_BSUPD, st, sb, o, 1, tt, ViewDense{Rc.re, Rc.ld, Rc.ps}, ViewDense{Rc.im, Rc.ld, Rc.ps},
                          false, ViewDense{xo.re, n, x.ps}, ViewDense{xo.im, n, x.ps}, bw, true, true);
            if (rc) return rc;
        }
    }
    return MDLS_OK;
}

template <int P>
int zqr_entry(int64_t m, int64_t n, ZDense A, ZDense Q, int t, void* ws, cudaStream_t st) {
    const ZqrLayout L = zqr_layout(P, m, n, t, Q.re != nullptr, nullptr);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, sizeof(WsHeader), st) != cudaSuccess) return MDLS_ERR_CUDA;
    return zqr_run<P>(m, n, 0, A, Q, t, w, L, hdr, true, st);
}

template <int P>
int zbs_entry(int64_t n, ZDense R, ZDense y, ZDense x, int t, void* ws, cudaStream_t st) {
    const ZbsLayout L = zbs_layout(P, n, t, nullptr);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, sizeof(WsHeader), st) != cudaSuccess) return MDLS_ERR_CUDA;
    return zbs_run<P>(n, R, y, x, t, w, L, hdr, st);
}

template <int P>
int zls_entry(int64_t m, int64_t n, ZDense A, ZDense b, ZDense x, int t, void* ws, cudaStream_t st) {
    const ZlsLayout L = zls_layout(P, m, n, t);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, sizeof(WsHeader), st) != cudaSuccess) return MDLS_ERR_CUDA;
    const int64_t psw = m * (n + 1);
    const ZDense Aw{reinterpret_cast<double*>(w + L.Ar), reinterpret_cast<double*>(w + L.Ai), m, psw};
    for (int l = 0; l < P; ++l) {
        const size_t rb = m * sizeof(double);
        if (cudaMemcpy2DAsync(Aw.re + l * psw, rb, A.re + l * A.ps, A.ld * sizeof(double), rb, n,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpy2DAsync(Aw.im + l * psw, rb, A.im + l * A.ps, A.ld * sizeof(double), rb, n,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(Aw.re + l * psw + n * m, b.re + l * b.ps, rb, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(Aw.im + l * psw + n * m, b.im + l * b.ps, rb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    }
    int rc = zqr_run<P>(m, n, 1, Aw, ZDense{nullptr, nullptr, 0, 0}, t, w, L.qr, hdr, false, st);
    if (rc) return rc;
    const ZDense yv{Aw.re + n * m, Aw.im + n * m, m, psw};
    return zbs_run<P>(n, Aw, yv, x, t, w, L.bs, hdr, st);
}

}  // namespace mdls

#define MDLS_INSTANTIATE_Z(P)                                                                                   \
    namespace mdls {                                                                                            \
    int zqr_entry_p##P(int64_t m, int64_t n, double* Ar, double* Ai, int64_t lda, int64_t psa, double* Qr,      \
                       double* Qi, int64_t ldq, int64_t psq, int t, void* ws, cudaStream_t st) {                \
        return zqr_entry<P>(m, n, ZDense{Ar, Ai, lda, psa}, ZDense{Qr, Qi, ldq, psq}, t, ws, st);              \
    }                                                                                                           \
    int zbs_entry_p##P(int64_t n, const double* Rr, const double* Ri, int64_t ldr, int64_t psr,                \
                       const double* yr, const double* yi, int64_t psy, double* xr, double* xi, int64_t psx,   \
                       int t, void* ws, cudaStream_t st) {                                                     \
        return zbs_entry<P>(n, ZDense{const_cast<double*>(Rr), const_cast<double*>(Ri), ldr, psr},            \
                            ZDense{const_cast<double*>(yr), const_cast<double*>(yi), 1, psy},                  \
                            ZDense{xr, xi, 1, psx}, t, ws, st);                                                \
    }                                                                                                           \
    int zls_entry_p##P(int64_t m, int64_t n, const double* Ar, const double* Ai, int64_t lda, int64_t psa,     \
                       const double* br, const double* bi, int64_t psb, double* xr, double* xi, int64_t psx,   \
                       int t, void* ws, cudaStream_t st) {                                                     \
        return zls_entry<P>(m, n, ZDense{const_cast<double*>(Ar), const_cast<double*>(Ai), lda, psa},         \
                            ZDense{const_cast<double*>(br), const_cast<double*>(bi), 1, psb},                  \
                            ZDense{xr, xi, 1, psx}, t, ws, st);                                                \
    }                                                                                                           \
    }
