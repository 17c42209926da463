// Kernels of the plain multiple-double path (FP64 CUDA cores), templated on
// the limb count P.  Section and algorithm numbers refer to arXiv 2110.08375.
#pragma once
#include "common.cuh"

namespace mdls {

template <int P>
DEV_INLINE md<P> md_one() {
    return md_from_double<P>(1.0);
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

// Deterministic sum over the 16 lanes of each half warp (fixed shfl_down tree
// ending in the half's first lane, then broadcast within the half).
template <int P>
DEV_INLINE md<P> half_sum(md<P> x) {
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        md<P> y;
#pragma unroll
        for (int l = 0; l < P; ++l) y.v[l] = __shfl_down_sync(0xffffffffu, x.v[l], off, 16);
        x = md_add<P>(x, y);
    }
#pragma unroll
    for (int l = 0; l < P; ++l) x.v[l] = __shfl_sync(0xffffffffu, x.v[l], 0, 16);
    return x;
}

template <int P>
DEV_INLINE md<P> half_shfl(const md<P>& x, int src) {
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = __shfl_sync(0xffffffffu, x.v[l], src, 16);
    return r;
}

template <int P>
DEV_INLINE md<P> md_select(bool c, const md<P>& a, const md<P>& b) {
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = c ? a.v[l] : b.v[l];
    return r;
}

// Bounded waits measure wall time on the GPU's global timer (ns), so that
// the limit does not move with the SM clock.  The limit is the workspace
// header's wait_ns, or 2 s when that is 0 (every entry point clears the
// header, so the default applies unless a caller sets it afterwards).
constexpr unsigned long long kWaitDefaultNs = 2000000000ull;

DEV_INLINE unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits (thread 0 only) until *flag == want.  Bounded: when the limit runs
// out it records MDLS_ERR_TIMEOUT, raises the header's failure flag and
// returns false.  Also returns false as soon as another block has failed.
DEV_INLINE bool wait_flag(const unsigned int* flag, unsigned int want, WsHeader* h) {
    const volatile unsigned int* vf = flag;
    const volatile int* verr = &h->bar_error;
    const unsigned long long lim0 = *reinterpret_cast<const volatile unsigned long long*>(&h->wait_ns);
    const unsigned long long lim = lim0 ? lim0 : kWaitDefaultNs;
    const unsigned long long t0 = globaltimer_ns();
    while (*vf != want) {
        if (*verr) return false;
        if (globaltimer_ns() - t0 > lim) {
            atomicExch(&h->bar_error, 1);
            set_status(&h->status, MDLS_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Diagnostic of the bounded wait (mdls_wait_check): block 1 waits, with the
// limit in the header, for a flag that block 0 publishes only when
// `publish` is set.  Launched cooperatively, so both blocks are resident.
static __global__ void wait_check_kernel(unsigned int* flag, WsHeader* h, int publish) {
    if (threadIdx.x != 0) return;
    if (blockIdx.x == 0) {
        if (publish) {
            __threadfence();
            atomicExch(flag, 1u);
        }
        return;
    }
    wait_flag(flag, 1u, h);
}

// ----------------------------------------------------------------------------
// md GEMM: C(i,j) = [C(i,j)] +/- sum_k A(i,k) B(k,j), one output per thread,
// a 16 x TN output tile per block, operands staged limb-planar in shared
// memory.  Used for every product of the WY representation (Section 3):
// G = Y^T Y, W = -Y T, W^T C, C + Y (W^T C), Y^T Q, Q + W (Y^T Q).  The
// octo-double instance runs 16 x 8 tiles (128 threads, about 150 registers
// each) so that three blocks share an SM: the FP64 pipe needs more than two
// warps per sub-partition to hide the latency of dependent instructions.
// ----------------------------------------------------------------------------
constexpr int kGemmTile = 16;

template <int P>
__host__ __device__ constexpr int gemm_tn() {
    return P == 8 ? 8 : 16;
}

// With split-K (gridDim.z > 1) block z sums k in [z kchunk, (z+1) kchunk) and
// writes its raw partial sum to C.ptr + z * zstride (negate/accumulate are
// then applied by split_reduce_kernel).  upper_only skips output tiles that
// lie entirely below the diagonal (symmetric products).
template <int P, class AV, class BV>
__global__ void __launch_bounds__(kGemmTile* gemm_tn<P>(), P == 8 ? 3 : 1)
    gemm_kernel(int64_t M, int64_t N, int64_t K, AV A, BV B, Dense C, int negate, int accumulate,
                int64_t kchunk, int64_t zstride, int upper_only) {
    constexpr int TN = gemm_tn<P>();
    constexpr int NT = kGemmTile * TN;
    __shared__ double As[P][kGemmTile][kGemmTile + 1];  // [limb][k][i]
    __shared__ double Bs[P][TN][kGemmTile + 1];         // [limb][j][k]
    const int tx = threadIdx.x % kGemmTile, ty = threadIdx.x / kGemmTile;
    const int64_t i0 = (int64_t)blockIdx.x * kGemmTile, j0 = (int64_t)blockIdx.y * TN;
    const int64_t i = i0 + tx, j = j0 + ty;
    if (upper_only && i0 > j0 + TN - 1) return;  // whole block below the diagonal
    int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    int64_t kend = (kbeg + kchunk) < K ? (kbeg + kchunk) : K;
    // k ranges that only meet known zeros of A (rows i0..) or B (columns j0..)
    if constexpr (AV::kZeroKBelowI) kbeg = kbeg > i0 ? kbeg : i0;
    if constexpr (AV::kZeroKAboveI) kend = kend < i0 + kGemmTile ? kend : i0 + kGemmTile;
    if constexpr (BV::kZeroKBelowI) kend = kend < j0 + TN ? kend : j0 + TN;
    if constexpr (BV::kZeroKAboveI) kbeg = kbeg > j0 ? kbeg : j0;
    double bins[P];  // unnormalised accumulator, renormalised once per staged tile
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += kGemmTile) {
#pragma unroll
        for (int idx = threadIdx.x; idx < kGemmTile * kGemmTile; idx += NT) {
            const int ii = idx % kGemmTile, kk = idx / kGemmTile;
            const bool in = (i0 + ii < M) && (k0 + kk < kend);
#pragma unroll
            for (int l = 0; l < P; ++l) As[l][kk][ii] = in ? A.get(i0 + ii, k0 + kk, l) : 0.0;
        }
#pragma unroll
        for (int idx = threadIdx.x; idx < kGemmTile * TN; idx += NT) {
            const int kk = idx % kGemmTile, jj = idx / kGemmTile;
            const bool in = (k0 + kk < kend) && (j0 + jj < N);
#pragma unroll
            for (int l = 0; l < P; ++l) Bs[l][jj][kk] = in ? B.get(k0 + kk, j0 + jj, l) : 0.0;
        }
        __syncthreads();
        const int kmax = (int)((kend - k0) < kGemmTile ? (kend - k0) : kGemmTile);
        // the operands of step kk + 1 are read from shared memory while step
        // kk runs (the staged tiles are zero beyond kend, so the read ahead
        // stays inside them)
        md<P> an, bn;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            an.v[l] = As[l][0][tx];
            bn.v[l] = Bs[l][ty][0];
        }
        for (int kk = 0; kk < kmax; ++kk) {
            const md<P> av = an, bv = bn;
            const int kn = kk + 1 < kGemmTile ? kk + 1 : kk;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                an.v[l] = As[l][kn][tx];
                bn.v[l] = Bs[l][ty][kn];
            }
            md_fma_bins<P>(bins, av, bv);
        }
        md_bins_renorm<P>(bins);
        __syncthreads();
    }
    md<P> acc;
#pragma unroll
    for (int l = 0; l < P; ++l) acc.v[l] = bins[l];
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

// Matrix-vector products (N = 1): y(i) = [y] +/- sum_k A(i,k) x(k).
// gemv_kpar_kernel (A contiguous along i): lanes own 32 consecutive rows
// (coalesced loads), the NW warps of a block take interleaved k and their
// partial sums meet in a fixed tree in shared memory; grid.y splits the K
// range further as in gemm_kernel.  On GB300 an FP64 warp instruction
// holds its SM sub-partition for 64 cycles whatever the number of active
// lanes, so short products must be spread over many warps rather than run as
// long per-thread chains.  gemv_warps_kernel (A contiguous along k): one warp
// per row, lanes along k, fixed-order warp reduction.
template <int P, int NW, class AV, class BV>
__global__ void __launch_bounds__(32 * NW)
    gemv_kpar_kernel(int64_t M, int64_t K, AV A, BV B, Dense C, int negate, int accumulate,
                     int64_t kchunk, int64_t zstride) {
    __shared__ md<P> red[NW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * 32, i = i0 + lane;
    int64_t kb = (int64_t)blockIdx.y * kchunk;
    int64_t ke = (kb + kchunk) < K ? (kb + kchunk) : K;
    if constexpr (AV::kZeroKBelowI) kb = kb > i0 ? kb : i0;
    if constexpr (AV::kZeroKAboveI) ke = ke < i0 + 32 ? ke : i0 + 32;
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    if (i < M) {
        int cnt = 0;
        for (int64_t k = kb + warp; k < ke; k += NW) {
            md<P> a, x;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                a.v[l] = A.get(i, k, l);
                x.v[l] = B.get(k, 0, l);
            }
            md_fma_bins<P>(bins, a, x);
            if ((++cnt & 15) == 0) md_bins_renorm<P>(bins);
        }
    }
    md<P> acc = md_from_bins<P>(bins);
    red[warp][lane] = acc;
    __syncthreads();
#pragma unroll
    for (int h = NW / 2; h > 0; h >>= 1) {
        if (warp < h) red[warp][lane] = md_add<P>(red[warp][lane], red[warp + h][lane]);
        __syncthreads();
    }
    if (warp != 0 || i >= M) return;
    acc = red[0][lane];
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
    int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    int64_t kend = (kbeg + kchunk) < K ? (kbeg + kchunk) : K;
    if constexpr (AV::kZeroKBelowI) kbeg = kbeg > i ? kbeg : i;
    if constexpr (AV::kZeroKAboveI) kend = kend < i + 1 ? kend : i + 1;
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    int cnt = 0;
    for (int64_t k = kbeg + lane; k < kend; k += 32) {
        md<P> a, x;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            a.v[l] = A.get(i, k, l);
            x.v[l] = B.get(k, 0, l);
        }
        md_fma_bins<P>(bins, a, x);
        if ((++cnt & 15) == 0) md_bins_renorm<P>(bins);
    }
    md<P> acc = warp_sum<P>(md_from_bins<P>(bins));
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
// Inversion of upper triangular tiles (step 1 of Algorithm 1) and T of the WY
// form (Section 3), both as a recursion on 2 x 2 block upper triangular
// matrices.  For X = [X1 X12; 0 X2]:
//   inverse of U:    X12 = -inv(U1) U12 inv(U2),
//   T of the WY form (Elmroth and Gustavson): T12 = -T1 (Y1^T Y2) T2,
// i.e. the same combination X12 = -X1 M12 X2 with M12 the off-diagonal block
// of U, or of G = Y^T Y.  Leaves of size L <= 16 are solved directly; every
// level doubles the block size with two small products.  The paper inverts
// each diagonal tile with one thread per column and builds W column by column;
// here every serial chain is at most L - 1 steps long and the rest runs as
// parallel products, which matters on a GPU whose FP64 pipe retires one warp
// instruction per 64 cycles per SM sub-partition.
// ----------------------------------------------------------------------------
constexpr int kTriLeaf = 16;

// Leaves of the tile inversion: column c of the inverse of an L x L diagonal
// block (leaf) of tile `tile` solves U v = e_c by back substitution, column
// by column: with s = e_c, for l = c down to 0, v_l = s_l / U_ll, then
// s_h -= U_hl v_l for every h < l.  Two columns per warp, one per half; lane
// h of a half holds s_h, v_h and the reciprocal of U_hh (computed once, in
// parallel), so a step is one product, one broadcast and one fused
// multiply-subtract per lane: no reductions on the serial chain.  A zero
// pivot records MDLS_ERR_SINGULAR (its reciprocal reads as zero).  Column c
// of tile `tile` goes to D + tile * dtile + c * dld (rows of its leaf only).
template <int P>
__global__ void tri_leaf_inv_kernel(const double* U, int64_t ld, int64_t ps, int64_t n, int t, int L,
                                    int64_t ntiles, double* D, int64_t dld, int64_t dps, int64_t dtile,
                                    WsHeader* hdr) {
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, half = lane >> 4, h = lane & 15;
    const int64_t ppt = (t + 1) / 2;  // column pairs per tile
    if (gw >= ntiles * ppt) return;   // whole warp
    const int64_t tile = gw / ppt;
    const int c0 = 2 * (int)(gw % ppt);
    const int64_t o = tile * t;
    const int tt = (int)((n - o) < t ? (n - o) : t);
    if (c0 >= tt) return;  // whole warp
    const int c = c0 + half;
    const bool valid = c < tt;
    const int leaf0 = (c0 / L) * L;
    const int le = (leaf0 + L) < tt ? (leaf0 + L) : tt;
    const int k = c - leaf0;
    const double* Ul = U + (o + leaf0) * ld + (o + leaf0);
    md<P> r = md_zero<P>();
    if (leaf0 + h < le) {
        const md<P> d = ld_md<P>(Ul, ps, (int64_t)h * ld + h);
        if (d.v[0] == 0.0) set_status(&hdr->status, MDLS_ERR_SINGULAR);
        else r = md_div<P>(md_one<P>(), d);
    }
    md<P> acc = (valid && h == k) ? md_one<P>() : md_zero<P>();  // s_h
    md<P> v = md_zero<P>();
    const int kw = ((c0 + 1) < tt ? (c0 + 1) : c0) - leaf0;  // largest column of the warp
    for (int l = kw; l >= 0; --l) {
        const md<P> vl = half_shfl<P>(md_mul<P>(acc, r), l);  // v_l, from lane l of the half
        v = md_select<P>(valid && h == l && l <= k, vl, v);
        if (valid && h < l && l <= k) acc = md_fms<P>(acc, ld_md<P>(Ul, ps, (int64_t)l * ld + h), vl);
    }
    if (valid && h <= k) st_md<P>(D + tile * dtile + (int64_t)c * dld, dps, leaf0 + h, v);
}

// Leaves of T: inside each L x L diagonal block, row l of T has T[l,l] =
// beta_l and T[l,j] = -beta_j sum_{q=l}^{j-1} T[l,q] G[q,j] for l < j < the
// leaf's end (G = Y^T Y), so that H_1 ... H_w = I - Y T Y^T = I + W Y^T with
// W = -Y T: the paper's z_j = -beta_j (v_j + W Y^T v_j), with Y^T v read
// from G.  Two rows per warp, one per half; lane h holds T[l, leaf0 + h].  An
// identity reflector (beta_j = 0) gives a zero column j.
template <int P>
__global__ void wy_t_leaf_kernel(const double* G, int64_t ldg, int64_t psg, const double* beta,
                                 int64_t bps, int w, int L, double* T, int64_t ldt, int64_t pst) {
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31, half = lane >> 4, h = lane & 15;
    const int l0 = 2 * gw;
    if (l0 >= w) return;  // whole warp
    const int l = l0 + half;
    const bool valid = l < w;
    const int leaf0 = (l0 / L) * L;
    const int le = (leaf0 + L) < w ? (leaf0 + L) : w;
    const int q = leaf0 + h;
    md<P> tv = (valid && q == l) ? ld_md<P>(beta, bps, l) : md_zero<P>();
    for (int j = l0 + 1; j < le; ++j) {
        const bool act = valid && j > l;
        const bool in = act && q >= l && q < j;
        const md<P> g = in ? ld_md<P>(G, psg, (int64_t)j * ldg + q) : md_zero<P>();
        const md<P> sum = half_sum<P>(md_mul<P>(in ? tv : md_zero<P>(), g));
        const md<P> tj = md_neg<P>(md_mul<P>(ld_md<P>(beta, bps, j), sum));
        tv = md_select<P>(act && q == j, tj, tv);
    }
    if (valid && q >= l && q < le) st_md<P>(T, pst, (int64_t)q * ldt + l, tv);
}

// One level of the recursion for all pairs of all tiles: tile b (width
// min(t, n - b t), at X + b xtile and M + b mtile) pairs its blocks
// X1 = X[a:a+s, a:a+s] and X2 = X[a+s:a+s+s2, a+s:a+s+s2] (a = 2 s y).
//   STEP 0: Z = M12 X2 (X2 upper triangular: k <= j), kept in the unused
//           lower block of X as X[a+s+j, a+i] = Z(i, j);
//   STEP 1: X12 = -X1 Z (X1 upper triangular: k >= i) into X[a+i, a+s+j].
// An 8 x 4 output block per warp (lanes along i: coalesced reads of M12 and
// X1); the k range is split over blockDim.x / 32 (at most 8) warps whose
// partial sums meet in a fixed tree.  Small blocks spread a level of one tile
// over most SMs: each SM's shared FP64 unit, not the number of outputs, sets
// the pace; with many tiles the k ranges are longer and the tree shorter.
template <int P, int STEP>
__global__ void __launch_bounds__(256) tri_level_kernel(double* X, int64_t ldx, int64_t psx, int64_t xtile, const double* M,
                                 int64_t ldm, int64_t psm, int64_t mtile, int64_t n, int t, int s) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    md<P>* red = reinterpret_cast<md<P>*>(tl_smem);
    const int KS = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, kz = threadIdx.x >> 5;
    const int nbi = (s + 7) >> 3;
    const int i = (blockIdx.x % nbi) * 8 + (lane & 7), j = (blockIdx.x / nbi) * 4 + (lane >> 3);
    const int64_t b = blockIdx.z;
    const int64_t a = (int64_t)blockIdx.y * 2 * s;
    const int64_t tt = (n - b * t) < t ? (n - b * t) : t;
    if (a + s >= tt) return;  // whole block: this pair has no second block
    const int s2 = (int)((tt - a - s) < s ? (tt - a - s) : s);
    double* Xb = X + b * xtile;
    const double* Mb = M + b * mtile;
    const bool out = i < s && j < s2;
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    if (out) {
        const int kc = (s + KS - 1) / KS;
        int kb = kz * kc, ke = kb + kc;
        if (STEP == 0) {
            ke = ke < j + 1 ? ke : j + 1;
            for (int k = kb; k < ke; ++k) {
                md_fma_bins<P>(bins, ld_md<P>(Mb, psm, (a + s + k) * ldm + a + i),
                               ld_md<P>(Xb, psx, (a + s + j) * ldx + a + s + k));
                if (((k - kb) & 15) == 15) md_bins_renorm<P>(bins);
            }
        } else {
            kb = kb > i ? kb : i;
            ke = ke < s ? ke : s;
            for (int k = kb; k < ke; ++k) {
                md_fma_bins<P>(bins, ld_md<P>(Xb, psx, (a + k) * ldx + a + i),
                               ld_md<P>(Xb, psx, (a + k) * ldx + a + s + j));
                if (((k - kb) & 15) == 15) md_bins_renorm<P>(bins);
            }
        }
    }
    red[kz * 32 + lane] = md_from_bins<P>(bins);
    __syncthreads();
    for (int hh = KS / 2; hh > 0; hh >>= 1) {
        if (kz < hh) red[kz * 32 + lane] = md_add<P>(red[kz * 32 + lane], red[(kz + hh) * 32 + lane]);
        __syncthreads();
    }
    if (kz != 0 || !out) return;
    if (STEP == 0) st_md<P>(Xb, psx, (a + i) * ldx + a + s + j, red[lane]);
    else st_md<P>(Xb, psx, (a + s + j) * ldx + a + i, md_neg<P>(red[lane]));
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
