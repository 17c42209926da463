// Kernels of the plain multiple-double path (FP64 CUDA cores), templated on
// the limb count P.  Section and algorithm numbers refer to arXiv 2110.08375.
#pragma once
#include "common.cuh"

namespace mdls {

template <int P>
DEV_INLINE md<P> md_one() {
    return md_from_double<P>(1.0);
}

// loads that bypass L1 (data written by other blocks of the same launch)
template <int P>
DEV_INLINE md<P> ld_md_cg(const double* ptr, int64_t ps, int64_t off) {
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = __ldcg(ptr + l * ps + off);
    return r;
}

// Deterministic block reduction (fixed binary tree), result in every thread.
template <int P, int NT>
DEV_INLINE md<P> block_sum(md<P> x, md<P>* red) {
    const int tid = threadIdx.x;
    red[tid] = x;
    __syncthreads();
#pragma unroll 1
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = md_add<P>(red[tid], red[tid + s]);
        __syncthreads();
    }
    md<P> r = red[0];
    __syncthreads();
    return r;
}

// Deterministic warp reduction: a fixed shfl_down tree ending in lane 0,
// whose sum is then broadcast, so every lane gets the same bits.
template <int P>
DEV_INLINE md<P> warp_sum(md<P> x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        md<P> y;
#pragma unroll
        for (int l = 0; l < P; ++l) y.v[l] = __shfl_down_sync(0xffffffffu, x.v[l], off);
        x = md_add<P>(x, y);
    }
#pragma unroll
    for (int l = 0; l < P; ++l) x.v[l] = __shfl_sync(0xffffffffu, x.v[l], 0);
    return x;
}

constexpr long long kFlagTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz

// Householder scalars of x = (x0, x_1..): sigma = sum_{i>0} x_i^2 given.
// kind 0: general (beta, 1/v0, R = mu), 1: identity (beta = 0, R = x0),
// 2: reflect e1 (beta = 2, R = -x0); Golub & Van Loan Alg. 5.1.1.
template <int P>
DEV_INLINE void house_scalars(const md<P>& sig, const md<P>& x0, md<P>& beta, md<P>& inv, md<P>& rcc,
                              int& kind) {
    if (sig.v[0] == 0.0) {
        inv = md_zero<P>();
        if (x0.v[0] >= 0.0) {
            kind = 1; beta = md_zero<P>(); rcc = x0;
        } else {
            kind = 2; beta = md_from_double<P>(2.0); rcc = md_neg<P>(x0);
        }
        return;
    }
    kind = 0;
    const md<P> mu = md_sqrt<P>(md_fma<P>(sig, x0, x0));
    md<P> v0;
    if (x0.v[0] <= 0.0) v0 = md_sub<P>(x0, mu);
    else v0 = md_neg<P>(md_div<P>(sig, md_add<P>(x0, mu)));  // -sigma/(x0+mu)
    // beta = 2 v0^2 / (sigma + v0^2) = -v0 / mu, since sigma + v0^2 = -2 mu v0
    beta = md_neg<P>(md_div<P>(v0, mu));
    inv = md_div<P>(md_one<P>(), v0);
    rcc = mu;
}

// Waits (thread 0 only) until *flag == want.  Bounded: on timeout it records
// MDLS_ERR_TIMEOUT and returns false.  Also returns false when another block
// has already failed.
DEV_INLINE bool wait_flag(const unsigned int* flag, unsigned int want, WsHeader* h) {
    const volatile unsigned int* vf = flag;
    const volatile int* verr = &h->bar_error;
    long long t0 = clock64();
    while (*vf != want) {
        if (*verr) return false;
        if (clock64() - t0 > kFlagTimeoutCycles) {
            atomicExch(&h->bar_error, 1);
            set_status(&h->status, MDLS_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// ----------------------------------------------------------------------------
// Row-split panel: step 1 of Algorithm 2 with every block sharing every
// column (used with a single block for the small problems of batched solves,
// where a panel must not wait on blocks of its own that other work keeps off
// the SMs).  Block b owns rows [b*rows_per, ...) of the panel (all w columns).
// Per column l: (1) partial sigma over my rows -> grid barrier -> every block
// sums the partials (fixed tree) and computes the reflector's scalars
// ("beta, v"); (2) my rows of v, partial v^T a_c for every column c > l ->
// barrier -> block b sums the partials of column l+1+b (fixed tree), forms
// w_c = beta v^T a_c and publishes it ("beta R^T v") -> barrier; (3) my rows
// of every column c > l get a_c -= v w_c ("update R").  The owner of row l
// writes R_ll.  With one block (small problems) there is no barrier at all.
// Scratch: part (gridDim.x x (w+1) md), wvec (w md).
// ----------------------------------------------------------------------------
struct RowPanelArgs {
    double* A;
    int64_t ld, ps;
    int64_t j0, r;
    int w;
    double* beta;
    int64_t beta_ps;
    double* part;     // [b][c] partials: part + (b*(w+1) + c); plane stride part_ps
    int64_t part_ps;
    double* wvec;     // w_c; plane stride w
    WsHeader* hdr;
};

template <int P, int NT>
__global__ void __launch_bounds__(NT) panel_rows_kernel(RowPanelArgs a) {
    const int tid = threadIdx.x, nb = gridDim.x, b = blockIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = NT / 32;
    const int64_t ld = a.ld, ps = a.ps;
    double* base = a.A + a.j0 * ld + a.j0;
    const int64_t rows_per = (a.r + nb - 1) / nb;
    const int64_t rb0 = (int64_t)b * rows_per;
    const int64_t rb1 = (rb0 + rows_per) < a.r ? (rb0 + rows_per) : a.r;
    const int W1 = a.w + 1;
    __shared__ md<P> red[NT];
    __shared__ md<P> sh_scal[3];
    __shared__ int sh_kind;
    for (int ell = 0; ell < a.w; ++ell) {
        double* col = base + (int64_t)ell * ld;
        // (1) sigma
        md<P> sig = md_zero<P>();
        for (int64_t i = (rb0 > ell + 1 ? rb0 : ell + 1) + tid; i < rb1; i += NT) {
            const md<P> xi = ld_md<P>(col, ps, i);
            sig = md_fma<P>(sig, xi, xi);
        }
        sig = block_sum<P, NT>(sig, red);
        if (nb > 1) {
            if (tid == 0) st_md<P>(a.part, a.part_ps, (int64_t)b * W1 + a.w, sig);
            if (!grid_barrier(a.hdr)) return;
            md<P> s = md_zero<P>();
            for (int q = tid; q < nb; q += NT) s = md_add<P>(s, ld_md_cg<P>(a.part, a.part_ps, (int64_t)q * W1 + a.w));
            sig = block_sum<P, NT>(s, red);
        }
        if (tid == 0) {
            md<P> beta, inv, rcc;
            int kind;
            house_scalars<P>(sig, ld_md_cg<P>(col, ps, ell), beta, inv, rcc, kind);
            sh_scal[0] = beta;
            sh_scal[1] = inv;
            sh_scal[2] = rcc;
            sh_kind = kind;
        }
        __syncthreads();
        const int kind = sh_kind;
        const md<P> beta = sh_scal[0];
        if (kind == 0) {
            const md<P> inv = sh_scal[1];
            for (int64_t i = (rb0 > ell + 1 ? rb0 : ell + 1) + tid; i < rb1; i += NT)
                st_md<P>(col, ps, i, md_mul<P>(ld_md<P>(col, ps, i), inv));
        }
        __syncthreads();
        // (2) partial dots v^T a_c over my rows (one warp per column, lanes over rows)
        const int64_t lo = rb0 > ell ? rb0 : ell;
        if (kind != 1) {
            for (int c = ell + 1 + warp; c < a.w; c += NW) {
                const double* cc = base + (int64_t)c * ld;
                md<P> s = md_zero<P>();
                for (int64_t i = lo + lane; i < rb1; i += 32) {
                    const md<P> vi = (i == ell) ? md_one<P>() : ld_md<P>(col, ps, i);
                    s = md_fma<P>(s, vi, ld_md<P>(cc, ps, i));
                }
                s = warp_sum<P>(s);
                if (lane == 0) {
                    if (nb > 1) st_md<P>(a.part, a.part_ps, (int64_t)b * W1 + c, s);
                    else st_md<P>(a.wvec, a.w, c, md_mul<P>(beta, s));
                }
            }
        }
        if (nb > 1) {
            if (!grid_barrier(a.hdr)) return;
            // block b reduces the partials of columns c = ell+1+b, ell+1+b+nb, ...
            for (int c = ell + 1 + b; c < a.w && kind != 1; c += nb) {
                md<P> s = md_zero<P>();
                for (int q = tid; q < nb; q += NT) s = md_add<P>(s, ld_md_cg<P>(a.part, a.part_ps, (int64_t)q * W1 + c));
                s = block_sum<P, NT>(s, red);
                if (tid == 0) st_md<P>(a.wvec, a.w, c, md_mul<P>(beta, s));
            }
            if (!grid_barrier(a.hdr)) return;
        } else {
            __syncthreads();
        }
        // (3) update my rows of the trailing panel columns
        if (kind != 1) {
            for (int c = ell + 1 + warp; c < a.w; c += NW) {
                double* cc = base + (int64_t)c * ld;
                const md<P> wc = nb > 1 ? ld_md_cg<P>(a.wvec, a.w, c) : ld_md<P>(a.wvec, a.w, c);
                for (int64_t i = lo + lane; i < rb1; i += 32) {
                    const md<P> vi = (i == ell) ? md_one<P>() : ld_md<P>(col, ps, i);
                    st_md<P>(cc, ps, i, md_fms<P>(ld_md<P>(cc, ps, i), vi, wc));
                }
            }
        }
        if (tid == 0 && ell >= rb0 && ell < rb1) st_md<P>(col, ps, ell, sh_scal[2]);
        if (tid == 0 && b == 0) st_md<P>(a.beta, a.beta_ps, ell, beta);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// md GEMM: C(i,j) = [C(i,j)] +/- sum_k A(i,k) B(k,j), one output per thread,
// 16x16 output tile per block, operands staged limb-planar in shared memory.
// Used for every product of the WY representation (Section 3):
// G = Y^T Y, W = -Y T, W^T C, C + Y (W^T C), Y^T Q, Q + W (Y^T Q).
// ----------------------------------------------------------------------------
constexpr int kGemmTile = 16;

// With split-K (gridDim.z > 1) block z sums k in [z kchunk, (z+1) kchunk) and
// writes its raw partial sum to C.ptr + z * zstride (negate/accumulate are
// then applied by split_reduce_kernel).  upper_only skips output tiles that
// lie entirely below the diagonal (symmetric products).
template <int P, class AV, class BV>
__global__ void __launch_bounds__(kGemmTile* kGemmTile)
    gemm_kernel(int64_t M, int64_t N, int64_t K, AV A, BV B, Dense C, int negate, int accumulate,
                int64_t kchunk, int64_t zstride, int upper_only) {
    __shared__ double As[P][kGemmTile][kGemmTile + 1];
    __shared__ double Bs[P][kGemmTile][kGemmTile + 1];
    const int tx = threadIdx.x % kGemmTile, ty = threadIdx.x / kGemmTile;
    const int64_t i0 = (int64_t)blockIdx.x * kGemmTile, j0 = (int64_t)blockIdx.y * kGemmTile;
    const int64_t i = i0 + tx, j = j0 + ty;
    if (upper_only && i0 > j0 + kGemmTile - 1) return;  // whole block below the diagonal
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = (kbeg + kchunk) < K ? (kbeg + kchunk) : K;
    md<P> acc = md_zero<P>();
    for (int64_t k0 = kbeg; k0 < kend; k0 += kGemmTile) {
        const bool a_in = (i0 + tx < M) && (k0 + ty < kend);
        const bool b_in = (k0 + tx < kend) && (j0 + ty < N);
#pragma unroll
        for (int l = 0; l < P; ++l) {
            As[l][ty][tx] = a_in ? A.get(i0 + tx, k0 + ty, l) : 0.0;   // A(i0+tx, k0+ty)
            Bs[l][ty][tx] = b_in ? B.get(k0 + tx, j0 + ty, l) : 0.0;   // B(k0+tx, j0+ty)
        }
        __syncthreads();
        const int kmax = (int)((kend - k0) < kGemmTile ? (kend - k0) : kGemmTile);
        for (int kk = 0; kk < kmax; ++kk) {
            md<P> av, bv;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                av.v[l] = As[l][kk][tx];
                bv.v[l] = Bs[l][ty][kk];
            }
            acc = md_fma<P>(acc, av, bv);
        }
        __syncthreads();
    }
    if (i < M && j < N) {
        const int64_t off = j * C.ld + i;
        if (gridDim.z > 1) {
            st_md<P>(C.ptr + blockIdx.z * zstride, C.ps, off, acc);
            return;
        }
        if (negate) acc = md_neg<P>(acc);
        if (accumulate) acc = md_add<P>(ld_md<P>(C.ptr, C.ps, off), acc);
        st_md<P>(C.ptr, C.ps, off, acc);
    }
}

// Matrix-vector products (N = 1): y(i) = [y] +/- sum_k A(i,k) x(k), with the
// K range split over grid.y as in gemm_kernel.  gemv_rows_kernel: one thread
// per row (A contiguous along i); gemv_warps_kernel: one warp per row, lanes
// along k (A contiguous along k), fixed-order warp reduction.
template <int P, class AV, class BV>
__global__ void gemv_rows_kernel(int64_t M, int64_t K, AV A, BV B, Dense C, int negate, int accumulate,
                                 int64_t kchunk, int64_t zstride) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = (kbeg + kchunk) < K ? (kbeg + kchunk) : K;
    md<P> acc = md_zero<P>();
    for (int64_t k = kbeg; k < kend; ++k) {
        md<P> a, x;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            a.v[l] = A.get(i, k, l);
            x.v[l] = B.get(k, 0, l);
        }
        acc = md_fma<P>(acc, a, x);
    }
    if (gridDim.y > 1) {
        st_md<P>(C.ptr + blockIdx.y * zstride, C.ps, i, acc);
        return;
    }
    if (negate) acc = md_neg<P>(acc);
    if (accumulate) acc = md_add<P>(ld_md<P>(C.ptr, C.ps, i), acc);
    st_md<P>(C.ptr, C.ps, i, acc);
}

template <int P, class AV, class BV>
__global__ void gemv_warps_kernel(int64_t M, int64_t K, AV A, BV B, Dense C, int negate, int accumulate,
                                  int64_t kchunk, int64_t zstride) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;  // whole warp
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = (kbeg + kchunk) < K ? (kbeg + kchunk) : K;
    md<P> acc = md_zero<P>();
    for (int64_t k = kbeg + lane; k < kend; k += 32) {
        md<P> a, x;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            a.v[l] = A.get(i, k, l);
            x.v[l] = B.get(k, 0, l);
        }
        acc = md_fma<P>(acc, a, x);
    }
    acc = warp_sum<P>(acc);
    if (lane != 0) return;
    if (gridDim.y > 1) {
        st_md<P>(C.ptr + blockIdx.y * zstride, C.ps, i, acc);
        return;
    }
    if (negate) acc = md_neg<P>(acc);
    if (accumulate) acc = md_add<P>(ld_md<P>(C.ptr, C.ps, i), acc);
    st_md<P>(C.ptr, C.ps, i, acc);
}

// C(i,j) = [C(i,j)] +/- sum_z partial_z(i,j), z in increasing order.
template <int P>
__global__ void split_reduce_kernel(int64_t M, int64_t N, int S, const double* part, int64_t pld,
                                    int64_t pps, int64_t zstride, Dense C, int negate,
                                    int accumulate) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t i = idx % M, j = idx / M;
    md<P> acc = ld_md<P>(part, pps, j * pld + i);
    for (int z = 1; z < S; ++z) acc = md_add<P>(acc, ld_md<P>(part + z * zstride, pps, j * pld + i));
    if (negate) acc = md_neg<P>(acc);
    const int64_t off = j * C.ld + i;
    if (accumulate) acc = md_add<P>(ld_md<P>(C.ptr, C.ps, off), acc);
    st_md<P>(C.ptr, C.ps, off, acc);
}

// ----------------------------------------------------------------------------
// Inversion of upper triangular tiles: step 1 of Algorithm 1.  Diagonal tile
// i covers rows/cols o..o+tt-1 of U (o = i t).  Column k of its inverse
// solves U v = e_k: v_k = 1/U_kk and, for l = k-1 down to 0,
// v_l = -(sum_{s=l+1}^{k} U_ls v_s) / U_ll.  The paper gives each column to
// one thread; here one warp solves one column, its lanes splitting each sum
// (fixed-order reduction), and grid.x * blockDim/32 warps cover the N*t
// columns.  A zero pivot records MDLS_ERR_SINGULAR.  The inverse is written
// upper triangular with zeros below the diagonal, tile i at D + i * dtile,
// column-major with leading dimension dld.
// ----------------------------------------------------------------------------
template <int P>
__global__ void tri_inv_kernel(const double* U, int64_t ld, int64_t ps, int64_t n, int t,
                               int64_t ntiles, double* D, int64_t dld, int64_t dps, int64_t dtile,
                               WsHeader* hdr) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= ntiles * t) return;  // whole warp
    const int64_t tile = gw / t;
    const int k = (int)(gw % t);
    const int64_t o = tile * t;
    const int tt = (int)((n - o) < t ? (n - o) : t);
    const double* Ut = U + o * ld + o;
    double* col = D + tile * dtile + (int64_t)k * dld;
    if (k >= tt) {
        for (int l = lane; l < t; l += 32) st_md<P>(col, dps, l, md_zero<P>());
        return;
    }
    for (int l = k + 1 + lane; l < t; l += 32) st_md<P>(col, dps, l, md_zero<P>());
    if (lane == 0) {
        md<P> d = ld_md<P>(Ut, ps, (int64_t)k * ld + k);
        if (d.v[0] == 0.0) set_status(&hdr->status, MDLS_ERR_SINGULAR);
        st_md<P>(col, dps, k, d.v[0] == 0.0 ? md_zero<P>() : md_div<P>(md_one<P>(), d));
    }
    __syncwarp();
    for (int l = k - 1; l >= 0; --l) {
        md<P> s = md_zero<P>();
        for (int q = l + 1 + lane; q <= k; q += 32)
            s = md_fma<P>(s, ld_md<P>(Ut, ps, (int64_t)q * ld + l), ld_md<P>(col, dps, q));
        s = warp_sum<P>(s);
        if (lane == 0) {
            md<P> d = ld_md<P>(Ut, ps, (int64_t)l * ld + l);
            if (d.v[0] == 0.0) {
                set_status(&hdr->status, MDLS_ERR_SINGULAR);
                st_md<P>(col, dps, l, md_zero<P>());
            } else {
                st_md<P>(col, dps, l, md_neg<P>(md_div<P>(s, d)));
            }
        }
        __syncwarp();
    }
}

// T of the WY representation of one tile.  With G = Y^T Y and the betas of
// the panel, T_jj = beta_j and T[l, j] = -beta_j sum_{q=l}^{j-1} T[l, q] G[q, j]
// for l < j, so that H_1 ... H_w = I - Y T Y^T = I + W Y^T with W = -Y T.
// Column j of W is then z_j = -beta_j (v_j + W_{:,<j} (Y_{:,<j}^T v_j)): the
// paper's formula for z (Section 3), with the products Y^T v read from G.
// Row l of T depends only on its own earlier entries: one warp builds row l,
// its lanes splitting the sum over q (fixed-order reduction).  An identity
// reflector (beta_j = 0) gives a zero column j, as it must.
template <int P>
__global__ void wy_t_kernel(const double* G, int64_t ldg, int64_t psg, const double* beta,
                            int64_t bps, int w, double* T, int64_t ldt, int64_t pst) {
    const int l = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (l >= w) return;  // whole warp
    if (lane == 0) st_md<P>(T, pst, (int64_t)l * ldt + l, ld_md<P>(beta, bps, l));
    __syncwarp();
    for (int j = l + 1; j < w; ++j) {
        md<P> s = md_zero<P>();
        for (int q = l + lane; q < j; q += 32)
            s = md_fma<P>(s, ld_md<P>(T, pst, (int64_t)q * ldt + l), ld_md<P>(G, psg, (int64_t)j * ldg + q));
        s = warp_sum<P>(s);
        if (lane == 0)
            st_md<P>(T, pst, (int64_t)j * ldt + l, md_neg<P>(md_mul<P>(ld_md<P>(beta, bps, j), s)));
        __syncwarp();
    }
}

// Step 2(a) of Algorithm 1: x_i := U_i^{-1} b_i (one block, thread k computes
// entry k; the inverse tile is upper triangular).
template <int P>
__global__ void bs_mulinv_kernel(const double* Dt, int64_t dld, int64_t dps, int tt,
                                 const double* bw, int64_t bps, double* x, int64_t xps,
                                 int64_t o) {
    const int k = threadIdx.x;
    if (k >= tt) return;
    md<P> s = md_zero<P>();
    for (int q = k; q < tt; ++q)
        s = md_fma<P>(s, ld_md<P>(Dt, dps, (int64_t)q * dld + k), ld_md<P>(bw, bps, o + q));
    st_md<P>(x, xps, o + k, s);
}

// Forward substitution with R^T (lower triangular), using the same inverted
// diagonal tiles: h_i := (U_i^{-1})^T g_i (thread k: sum over q <= k of
// D(q, k) g(q)), then g_j := g_j - (R_ij)^T h_i for the rows after tile i.
template <int P>
__global__ void fs_mulinv_t_kernel(const double* Dt, int64_t dld, int64_t dps, int tt,
                                   const double* gw, int64_t gps, double* h, int64_t hps, int64_t o) {
    const int k = threadIdx.x;
    if (k >= tt) return;
    md<P> s = md_zero<P>();
    for (int q = 0; q <= k; ++q)
        s = md_fma<P>(s, ld_md<P>(Dt, dps, (int64_t)k * dld + q), ld_md<P>(gw, gps, o + q));
    st_md<P>(h, hps, o + k, s);
}

template <int P>
__global__ void fs_update_kernel(const double* U, int64_t ld, int64_t ps, int64_t o, int tt,
                                 int64_t n, const double* h, int64_t hps, double* gw, int64_t gps) {
    const int64_t row = o + tt + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    md<P> s = ld_md<P>(gw, gps, row);
    const double* Ucol = U + row * ld + o;   // column `row` of R, rows o..o+tt-1
    for (int q = 0; q < tt; ++q) s = md_fms<P>(s, ld_md<P>(Ucol, ps, q), ld_md<P>(h, hps, o + q));
    st_md<P>(gw, gps, row, s);
}

// Step 2(b) of Algorithm 1: b_j := b_j - A_{j,i} x_i for all rows above tile
// i at once (thread per row).
template <int P>
__global__ void bs_update_kernel(const double* U, int64_t ld, int64_t ps, int64_t o, int tt,
                                 const double* x, int64_t xps, double* bw, int64_t bps) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= o) return;
    md<P> s = ld_md<P>(bw, bps, row);
    const double* Ur = U + o * ld + row;
    for (int q = 0; q < tt; ++q) s = md_fms<P>(s, ld_md<P>(Ur, ps, (int64_t)q * ld), ld_md<P>(x, xps, o + q));
    st_md<P>(bw, bps, row, s);
}

// Elementwise md arithmetic (mdls_vec_op).
template <int P>
__global__ void vec_op_kernel(int op, int64_t count, const double* a, int64_t psa, const double* b,
                              int64_t psb, double* c, int64_t psc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const md<P> x = ld_md<P>(a, psa, i);
    md<P> r;
    switch (op) {
        case MDLS_OP_ADD: r = md_add<P>(x, ld_md<P>(b, psb, i)); break;
        case MDLS_OP_SUB: r = md_sub<P>(x, ld_md<P>(b, psb, i)); break;
        case MDLS_OP_MUL: r = md_mul<P>(x, ld_md<P>(b, psb, i)); break;
        case MDLS_OP_DIV: r = md_div<P>(x, ld_md<P>(b, psb, i)); break;
        case MDLS_OP_FMA: r = md_fma<P>(ld_md<P>(c, psc, i), x, ld_md<P>(b, psb, i)); break;
        default: r = md_sqrt<P>(x); break;
    }
    st_md<P>(c, psc, i, r);
}

// End of the refinement loop: MDLS_ERR_NOT_CONVERGED unless
// max |d| <= 2^e2 max |x| (leading limbs; one block).
static __global__ void refine_check_kernel(const double* d, int64_t n, const double* x, int64_t pad,
                                    int e2, WsHeader* hdr) {
    __shared__ double sd[256], sx[256];
    double md = 0.0, mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        md = fmax(md, fabs(d[i]));
        mx = fmax(mx, fabs(x[i]));
    }
    sd[threadIdx.x] = md;
    sx[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
            sx[threadIdx.x] = fmax(sx[threadIdx.x], sx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && !(sd[0] <= ldexp(sx[0], e2))) set_status(&hdr->status, MDLS_ERR_NOT_CONVERGED);
}

// R output: zero the strictly lower part (rows > col) of an m x n matrix.
template <int P>
__global__ void zero_lower_kernel(double* A, int64_t ld, int64_t ps, int64_t m, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        if (i < m && i > j) {
#pragma unroll
            for (int l = 0; l < P; ++l) A[l * ps + j * ld + i] = 0.0;
        }
    }
}

// Q := I (m x m)
template <int P>
__global__ void identity_kernel(double* Q, int64_t ld, int64_t ps, int64_t m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y) {
        if (i < m) {
#pragma unroll
            for (int l = 0; l < P; ++l) Q[l * ps + j * ld + i] = (l == 0 && i == j) ? 1.0 : 0.0;
        }
    }
}

}  // namespace mdls
