// The Householder panel on the integer pipe: step 1 of Algorithm 2 ("beta,
// v := house(...)", "beta R^T v", "update R") for the w columns of one tile,
// Section 3.1 of arXiv 2110.08375.
//
// One block per column c (cooperative launch, all blocks resident).  The
// column is converted once to fixed point (24-bit digits at a per-column
// scale set by its norm, which reflections preserve) and kept in an
// L2-resident digit array; every dot product, norm and update is then exact
// integer arithmetic accumulated by digit diagonals, and only the results are
// rounded back to multiple doubles.  For each earlier reflector ell block c
//   (a) waits for "rows ready" of ell and forms the dot product of u_ell's
//       rows below ell with its column (the bulk of u_ell . a_c),
//   (b) waits for "scalars ready" of ell, completes the dot product with
//       v0_ell a_c[ell], forms w = bp_ell (u_ell . a_c), updates row ell and
//       then rows > ell: a_c -= w u_ell.
// After its last update block c publishes its rows below the diagonal
// (rescaled by whole digits so that the largest has a leading digit near
// the top) and only then computes its reflector's scalars: the next block's
// dot product (a) overlaps them.  Every wait is bounded.
#pragma once
#include "common.cuh"
#include "fx.cuh"
#include "fxw.cuh"
#include "kernels.cuh"

namespace mdls {

struct FxPanelArgs {
    double* A;  // working matrix (limb planar)
    int64_t ld, ps;
    int64_t j0;  // panel origin (global row = global column = j0)
    int64_t r;   // rows of the panel
    int w;       // columns of the panel
    double* beta;  // w md values, plane stride beta_ps
    int64_t beta_ps;
    int32_t* F;     // digit k of row i of column c: F[(k * w + c) * r + i]
    int32_t* meta;  // per column: FxMeta<P>::ints ints
    unsigned int* flags;  // 2w: [c] rows of u_c ready, [w + c] scalars of c ready
    unsigned int epoch;   // flag value meaning "ready" for this panel
    WsHeader* hdr;
};

// Per-column record published to the other blocks: scale of the published
// rows (digits), kind, v0 and bp (digits and exponent each).
template <int P>
struct FxMeta {
    static constexpr int N = fx::Cfg<P>::N;
    static constexpr int kScaleU = 0, kKind = 1, kV0 = 2, kBp = 3 + N;
    static constexpr int ints = 4 + 2 * N;
};

// The same record written and read by one warp (digit k by lane k).
template <int N>
DEV_INLINE void wst_xf(int32_t* p, const fxw::wxf& x) {
    const int lane = threadIdx.x & 31;
    if (lane < N) p[lane] = x.d;
    if (lane == 0) p[N] = x.e;
}

template <int N>
DEV_INLINE fxw::wxf wld_xf_cg(const int32_t* p) {
    const int lane = threadIdx.x & 31;
    return fxw::wxf{lane < N ? __ldcg(p + lane) : 0, __ldcg(p + N)};
}

// Block-wide exact sum of per-thread digit accumulators; the total's digit
// sums end up in red[0][0..M) for every thread to read.
template <int M, int NW>
DEV_INLINE void block_digit_sum(int64_t (&acc)[M], int64_t (*red)[M]) {
    fx::carry_norm<M>(acc);  // digits below 2^24: 32 of them sum in an int
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int s = __reduce_add_sync(0xffffffffu, (int)acc[k]);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        int64_t t = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) t += red[q][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
}

// The reflector's scalars on one warp, in two steps: panel_house_lead forms
// what the other columns wait for (the kind, v0 and bp in digits),
// panel_house_tail the rest (1/v0 in digits for the vector; R_cc and beta in
// P limbs).  Double double runs fx::house_dd on the FP64 pipe, every lane
// computing the same values, with the digit conversions spread over lanes;
// quad and octo double run the digit Newton steps spread over the warp,
// which cost less than their P-limb divisions and square roots.
template <int P, int N>
struct PanelHouse {
    int kind;
    fxw::wxf v0, bp, inv;   // digits: published v0 and bp; 1/v0 for the vector
    md<P> rcc, beta;        // R_cc and beta (every lane) after the tail
    fxw::wxf rcc_w, bet_w;  // their digit forms until the tail (P > 2)
    md<P> invm;             // 1/v0 in P limbs until the tail (P = 2, kind 0)
};

template <int P, int N>
DEV_INLINE void panel_house_lead(const fxw::wxf& sig, const fxw::wxf& x0, PanelHouse<P, N>& h) {
    if constexpr (P == 2) {
        const fx::xf<N> s = fxw::to_scalar<N>(sig), x = fxw::to_scalar<N>(x0);
        if (fx::xf_is_zero<N>(s)) {  // kinds 1 and 2: no reflection or a sign flip
            fx::xf<N> a, b, c, d, e;
            h.kind = fx::xf_house_md<P, N>(s, x, a, b, c, d, e);
            h.v0 = fxw::from_scalar<N>(a);
            h.bp = fxw::from_scalar<N>(b);
            h.inv = fxw::from_scalar<N>(d);
            h.rcc = fx::xf_to_md<P, N>(c);
            h.beta = fx::xf_to_md<P, N>(e);
            return;
        }
        // lane 1 rounds x0 to double double, the other lanes sig
        const int lane = threadIdx.x & 31;
        fx::xf<N> in;
#pragma unroll
        for (int k = 0; k < N; ++k) in.d[k] = lane == 1 ? x.d[k] : s.d[k];
        in.e = lane == 1 ? x.e : s.e;
        const md<P> m = fx::xf_to_md<P, N>(in);
        md<P> sm, xm, v0m, bpm;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            sm.v[l] = __shfl_sync(0xffffffffu, m.v[l], 0);
            xm.v[l] = __shfl_sync(0xffffffffu, m.v[l], 1);
        }
        fx::house_dd(sm, xm, h.rcc, v0m, bpm, h.invm, h.beta);
        h.kind = 0;
        h.v0 = fxw::from_md<P, N>(v0m);
        h.bp = fxw::from_md<P, N>(bpm);
    } else {
        h.kind = fxw::house<N>(sig, x0, h.v0, h.bp, h.rcc_w, h.inv, h.bet_w);
    }
}

template <int P, int N>
DEV_INLINE void panel_house_tail(PanelHouse<P, N>& h) {
    if constexpr (P == 2) {
        if (h.kind == 0) h.inv = fxw::from_md<P, N>(h.invm);
    } else {
        const fx::xf<N> bet_s = fxw::to_scalar<N>(h.bet_w), rcc_s = fxw::to_scalar<N>(h.rcc_w);
        h.beta = fx::xf_to_md<P, N>(bet_s);
        h.rcc = fx::xf_to_md<P, N>(rcc_s);
    }
}

template <int P, int NT>
__global__ void __launch_bounds__(NT, 2) fx_panel_kernel(FxPanelArgs a) {
    using namespace fx;
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N, NW = NT / 32, MI = FxMeta<P>::ints;
    constexpr int M = D + 3;  // digit diagonals of a dot product
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r = a.r, ps = a.ps, fs = (int64_t)a.w * r;
    double* colc = a.A + (a.j0 + c) * a.ld + a.j0;
    int32_t* Fc = a.F + (int64_t)c * r;
    int32_t* Mc = a.meta + c * MI;

    __shared__ int64_t red[NW][M];
    __shared__ int32_t sh_w[D];
    __shared__ double sh_d[NW];
    __shared__ unsigned sh_u[NW];
    __shared__ int sh_i[4];
    __shared__ int32_t sh_x[N + 1];

    // 0. column scale: e (digits) with every entry, now and after any
    //    reflection, below 2^(24(e + D) - 3).  Bound from the leading limbs.
    unsigned hmax = 0;
    for (int64_t i = tid; i < r; i += NT) {
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const unsigned h = (unsigned)(dbits(colc[l * ps + i]) >> 32) & 0x7fffffffu;
            hmax = h > hmax ? h : hmax;
        }
    }
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    if (lane == 0) sh_u[warp] = hmax;
    __syncthreads();
    hmax = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) hmax = sh_u[q] > hmax ? sh_u[q] : hmax;
    const bool finite = hmax < 0x7ff00000u;
    int emax = (int)(hmax >> 20) - 1023;  // leading exponent of the largest entry
    if (emax < -1022) emax = -1022;
    if (emax > 1000) emax = 1000;
    const double down = dfrom((uint64_t)(1023 - emax) << 52);  // 2^-emax
    double ss = 0.0;
    if (finite)
        for (int64_t i = tid; i < r; i += NT) {
            const double v = colc[i] * down;
            ss = __fma_rn(v, v, ss);
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if (lane == 0) sh_d[warp] = ss;
    __syncthreads();
    ss = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) ss += sh_d[q];
    int ec = -D;
    if (finite && ss > 0.0) {
        int k;
        frexp(sqrt(ss), &k);         // sqrt(ss) < 2^k
        const int bound = emax + k + 1;  // ||a_c|| < 2^bound, with a factor 2 to spare
        ec = floordiv24(bound + 3 + kB - 1) - D;
    }

    // 1. the column in digits
    for (int64_t i = tid; i < r; i += NT) {
        int32_t d[D];
        if (finite) {
            fixed_from_md<P, D>(ld_md<P>(colc, ps, i), ec, d);
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) d[k] = 0;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) Fc[k * fs + i] = d[k];
    }
    __syncthreads();

    // sum of squares of the rows below the diagonal and their leading digit
    int64_t sacc[M];
#pragma unroll
    for (int k = 0; k < M; ++k) sacc[k] = 0;
    int top = -1;
    int cnt = 0;
    bool fused = false;

    // 2. reflectors 0 .. c-1
    for (int ell = 0; ell < c; ++ell) {
        if (tid == 0) sh_i[0] = wait_flag(a.flags + ell, a.epoch, a.hdr) ? 1 : 0;
        __syncthreads();
        if (!sh_i[0]) return;
        const int eu = __ldcg(a.meta + ell * MI + FxMeta<P>::kScaleU);
        const int32_t* Fu = a.F + (int64_t)ell * r;
        // (a) bulk of the dot product, rows > ell
        int64_t acc[M];
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = 0;
        int cnt = 0;
        for (int64_t i = ell + 1 + tid; i < r; i += NT) {
            int32_t u[D], x[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                u[k] = __ldcg(Fu + k * fs + i);
                x[k] = Fc[k * fs + i];
            }
            dot_acc<D>(u, x, acc);
            if ((++cnt & 255) == 0) carry_norm<M>(acc);
        }
        block_digit_sum<M, NW>(acc, red);
        if (tid == 0) sh_i[1] = wait_flag(a.flags + a.w + ell, a.epoch, a.hdr) ? 1 : 0;
        __syncthreads();
        if (!sh_i[1]) return;
        const int kind = __ldcg(a.meta + ell * MI + FxMeta<P>::kKind);
        // (b) scalars: s = v0 a[ell] + bulk, w = bp s; row ell (one warp,
        //     digit k in lane k: these scalars are on the column chain)
        if (warp == 0) {
            const fxw::wxf v0 = wld_xf_cg<N>(a.meta + ell * MI + FxMeta<P>::kV0);
            const fxw::wxf bp = wld_xf_cg<N>(a.meta + ell * MI + FxMeta<P>::kBp);
            const int64_t tot = lane < M ? red[0][lane] : 0;
            const int32_t xe = lane < D ? Fc[lane * fs + ell] : 0;
            const fxw::wxf x_ell = fxw::from_fixed<N, D>(xe, ec);
            const fxw::wxf s = fxw::add<N>(fxw::from_acc<N, M>(tot, eu + ec + D - 3), fxw::mul<N>(v0, x_ell));
            const fxw::wxf W = fxw::mul<N>(bp, s);
            int32_t xn;
            bool ok = fxw::fixed_from_xf<N, D>(fxw::sub<N>(x_ell, fxw::mul<N>(W, v0)), ec, xn);
            if (lane < D) Fc[lane * fs + ell] = xn;
            int32_t wd = 0;
            if (kind == 0) ok = fxw::fixed_from_xf<N, D>(W, ec - eu - (D - 2), wd) && ok;
            if (!ok && lane == 0) set_status(&a.hdr->status, MDLS_ERR_UNSUPPORTED);
            if (lane < D) sh_w[lane] = kind == 0 ? wd : 0;
        }
        __syncthreads();
        // rows > ell (a kind-1/2 reflector has no rows below ell); after the
        // last reflector (ell = c - 1) the same pass also sums the squares of
        // the rows below the diagonal and finds their leading digit
        if (kind == 0) {
            int32_t wd[D];
#pragma unroll
            for (int k = 0; k < D; ++k) wd[k] = sh_w[k];
            for (int64_t i = ell + 1 + tid; i < r; i += NT) {
                int32_t u[D], x[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    u[k] = __ldcg(Fu + k * fs + i);
                    x[k] = Fc[k * fs + i];
                }
                axpy_row<D>(x, wd, u);
#pragma unroll
                for (int k = 0; k < D; ++k) Fc[k * fs + i] = x[k];
                if (ell == c - 1 && i > c) {
                    dot_acc<D>(x, x, sacc);  // general product: a symmetric variant miscomputed low digits
                    const int tp = fixed_top<D>(x);
                    top = tp > top ? tp : top;
                    if ((++cnt & 255) == 0) carry_norm<M>(sacc);  // keeps the int64 sums far from overflow
                }
            }
        }
        if (ell == c - 1) fused = kind == 0;
        __syncthreads();
    }

    // sum of squares and leading digit of the rows below the diagonal (unless
    // the last update pass has formed them)
    if (!fused) {
        for (int64_t i = c + 1 + tid; i < r; i += NT) {
            int32_t x[D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = Fc[k * fs + i];
            dot_acc<D>(x, x, sacc);
            const int tp = fixed_top<D>(x);
            top = tp > top ? tp : top;
            if ((++cnt & 255) == 0) carry_norm<M>(sacc);
        }
    }

    // 3. the reflector's scalars on warp 0 while the other warps publish the
    //    rows below the diagonal, rescaled by q whole digits so that their
    //    largest entry leads in digit D-2 or D-1
    top = __reduce_max_sync(0xffffffffu, top);
    if (lane == 0) sh_u[warp] = (unsigned)(top + 1);
    block_digit_sum<M, NW>(sacc, red);  // (synchronises)
    int tmax = -1;
#pragma unroll
    for (int q = 0; q < NW; ++q) tmax = (int)sh_u[q] - 1 > tmax ? (int)sh_u[q] - 1 : tmax;
    const int qsh = (tmax >= 0 && tmax < D - 2) ? D - 2 - tmax : 0;
    const int eu_c = ec - qsh;
    if (warp == 0) {
        // the reflector's scalars (Golub and Van Loan, Algorithm 5.1.1), one
        // warp with digit k in lane k; row c is not touched by the shift
        const int64_t tot = lane < M ? red[0][lane] : 0;
        const fxw::wxf sig = fxw::from_acc<N, M>(tot, 2 * ec + D - 3);
        const int32_t xe = lane < D ? Fc[lane * fs + c] : 0;
        PanelHouse<P, N> h;
        panel_house_lead<P, N>(sig, fxw::from_fixed<N, D>(xe, ec), h);
        if (lane == 0) Mc[FxMeta<P>::kKind] = h.kind;
        wst_xf<N>(Mc + FxMeta<P>::kV0, h.v0);
        wst_xf<N>(Mc + FxMeta<P>::kBp, h.bp);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicExch(a.flags + a.w + c, a.epoch);
        }
        // outputs: beta, R_cc; 1/v0 for the vector
        panel_house_tail<P, N>(h);
        if (lane == 0) {
            st_md<P>(a.beta, a.beta_ps, c, finite ? h.beta : md_from_double<P>(dnan()));
            st_md<P>(colc, ps, c, finite ? h.rcc : md_from_double<P>(dnan()));
        }
        if (lane < N) sh_x[lane] = h.inv.d;
        if (lane == 0) sh_x[N] = h.inv.e;
    } else {
        if (qsh > 0) {
            for (int64_t i = c + 1 + (tid - 32); i < r; i += NT - 32) {
#pragma unroll
                for (int k = D - 1; k >= 0; --k) Fc[k * fs + i] = k >= qsh ? Fc[(k - qsh) * fs + i] : 0;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NT - 32) : "memory");  // warps 1.. only
        if (tid == 32) {
            Mc[FxMeta<P>::kScaleU] = eu_c;
            __threadfence();
            atomicExch(a.flags + c, a.epoch);
        }
    }
    __syncthreads();

    // 4. write back: R above the diagonal, v = u / v0 below it
    xf<N> inv;
#pragma unroll
    for (int k = 0; k < N; ++k) inv.d[k] = sh_x[k];
    inv.e = sh_x[N];
    for (int64_t i = tid; i < r; i += NT) {
        if (i == c) continue;
        int32_t x[D];
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = Fc[k * fs + i];
        md<P> y;
        if (!finite) y = md_from_double<P>(dnan());
        else if (i < c) y = xf_to_md<P, N>(xf_from_fixed<N, D>(x, ec));
        else y = xf_to_md<P, N>(xf_mul<N>(xf_from_fixed<N, D>(x, eu_c), inv));
        st_md<P>(colc, ps, i, y);
    }
}

// ----------------------------------------------------------------------------
// The same panel in ONE block, for the small problems of batched solves: a
// panel must not wait on blocks of its own that concurrent work keeps off the
// SMs, so the column chain runs inside the block (right-looking, unblocked
// Householder over the w columns) with the arithmetic of fx_panel_kernel:
// each column in 24-bit digits at the scale set by its norm, dot products and
// updates exact by digit diagonals, the reflector's scalars on warp 0, and
// for each later column j one warp forms u . a_j, that column's
// w = bp (v0 a_j[c] + u . a_j) and the update a_j -= w u.  The vectors and
// R are written back to multiple doubles once, after the last column.
// Scratch: F (digits, as in fx_panel_kernel); the per-column scales and
// 1/v0 live in shared memory (w <= 256).
// ----------------------------------------------------------------------------
struct FxBlockPanelArgs {
    double* A;
    int64_t ld, ps;
    int64_t j0;
    int64_t r;
    int w;
    double* beta;
    int64_t beta_ps;
    int32_t* F;
    WsHeader* hdr;
};

constexpr int kFxBlockMaxW = 256;

template <int P, int NT>
__global__ void __launch_bounds__(NT) fx_panel_block_kernel(FxBlockPanelArgs a) {
    using namespace fx;
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N, NW = NT / 32;
    constexpr int M = D + 3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r = a.r, ps = a.ps, fs = (int64_t)a.w * r;
    const int w = a.w;
    double* base = a.A + a.j0 * a.ld + a.j0;

    __shared__ int64_t red[NW][M];
    __shared__ int sh_ec[kFxBlockMaxW], sh_eu[kFxBlockMaxW], sh_kind[kFxBlockMaxW];
    __shared__ unsigned char sh_fin[kFxBlockMaxW];
    __shared__ int32_t sh_inv[kFxBlockMaxW][N + 1];
    __shared__ int32_t sh_v0[N + 1], sh_bp[N + 1];
    __shared__ double sh_d[NW];
    __shared__ unsigned sh_u[NW];

    // 0. every column in digits at the scale of its norm (see fx_panel_kernel)
    for (int c = 0; c < w; ++c) {
        const double* colc = base + (int64_t)c * a.ld;
        unsigned hmax = 0;
        for (int64_t i = tid; i < r; i += NT) {
#pragma unroll
            for (int l = 0; l < P; ++l) {
                const unsigned h = (unsigned)(dbits(colc[l * ps + i]) >> 32) & 0x7fffffffu;
                hmax = h > hmax ? h : hmax;
            }
        }
        hmax = __reduce_max_sync(0xffffffffu, hmax);
        if (lane == 0) sh_u[warp] = hmax;
        __syncthreads();
        hmax = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) hmax = sh_u[q] > hmax ? sh_u[q] : hmax;
        const bool finite = hmax < 0x7ff00000u;
        int emax = (int)(hmax >> 20) - 1023;
        if (emax < -1022) emax = -1022;
        if (emax > 1000) emax = 1000;
        const double down = dfrom((uint64_t)(1023 - emax) << 52);
        double ss = 0.0;
        if (finite)
            for (int64_t i = tid; i < r; i += NT) {
                const double v = colc[i] * down;
                ss = __fma_rn(v, v, ss);
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
        if (lane == 0) sh_d[warp] = ss;
        __syncthreads();
        ss = 0.0;
#pragma unroll
        for (int q = 0; q < NW; ++q) ss += sh_d[q];
        int ec = -D;
        if (finite && ss > 0.0) {
            int k;
            frexp(sqrt(ss), &k);
            const int bound = emax + k + 1;
            ec = floordiv24(bound + 3 + kB - 1) - D;
        }
        int32_t* Fc = a.F + (int64_t)c * r;
        for (int64_t i = tid; i < r; i += NT) {
            int32_t d[D];
            if (finite) {
                fixed_from_md<P, D>(ld_md<P>(colc, ps, i), ec, d);
            } else {
#pragma unroll
                for (int k = 0; k < D; ++k) d[k] = 0;
            }
#pragma unroll
            for (int k = 0; k < D; ++k) Fc[k * fs + i] = d[k];
        }
        if (tid == 0) {
            sh_ec[c] = ec;
            sh_fin[c] = finite ? 1 : 0;
        }
        __syncthreads();
    }

    for (int c = 0; c < w; ++c) {
        const int ec = sh_ec[c];
        int32_t* Fc = a.F + (int64_t)c * r;
        // 1. sum of squares and leading digit of the rows below the diagonal
        int64_t sacc[M];
#pragma unroll
        for (int k = 0; k < M; ++k) sacc[k] = 0;
        int top = -1, cnt = 0;
        for (int64_t i = c + 1 + tid; i < r; i += NT) {
            int32_t x[D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = Fc[k * fs + i];
            dot_acc<D>(x, x, sacc);
            const int tp = fixed_top<D>(x);
            top = tp > top ? tp : top;
            if ((++cnt & 255) == 0) carry_norm<M>(sacc);
        }
        top = __reduce_max_sync(0xffffffffu, top);
        if (lane == 0) sh_u[warp] = (unsigned)(top + 1);
        block_digit_sum<M, NW>(sacc, red);  // (synchronises)
        int tmax = -1;
#pragma unroll
        for (int q = 0; q < NW; ++q) tmax = (int)sh_u[q] - 1 > tmax ? (int)sh_u[q] - 1 : tmax;
        const int qsh = (tmax >= 0 && tmax < D - 2) ? D - 2 - tmax : 0;
        const int eu = ec - qsh;
        // 2. the reflector's scalars on warp 0; the other warps rescale the
        //    rows below the diagonal by qsh whole digits (row c is untouched)
        if (warp == 0) {
            const int64_t tot = lane < M ? red[0][lane] : 0;
            const fxw::wxf sig = fxw::from_acc<N, M>(tot, 2 * ec + D - 3);
            const int32_t xe = lane < D ? Fc[lane * fs + c] : 0;
            PanelHouse<P, N> h;
            panel_house_lead<P, N>(sig, fxw::from_fixed<N, D>(xe, ec), h);
            panel_house_tail<P, N>(h);
            if (lane < N) {
                sh_v0[lane] = h.v0.d;
                sh_bp[lane] = h.bp.d;
                sh_inv[c][lane] = h.inv.d;
            }
            if (lane == 0) {
                sh_v0[N] = h.v0.e;
                sh_bp[N] = h.bp.e;
                sh_inv[c][N] = h.inv.e;
                sh_kind[c] = h.kind;
                sh_eu[c] = eu;
                const bool fin = sh_fin[c] != 0;
                st_md<P>(a.beta, a.beta_ps, c, fin ? h.beta : md_from_double<P>(dnan()));
                st_md<P>(base + (int64_t)c * a.ld, ps, c, fin ? h.rcc : md_from_double<P>(dnan()));
            }
        } else if (qsh > 0) {
            for (int64_t i = c + 1 + (tid - 32); i < r; i += NT - 32) {
#pragma unroll
                for (int k = D - 1; k >= 0; --k) Fc[k * fs + i] = k >= qsh ? Fc[(k - qsh) * fs + i] : 0;
            }
        }
        __syncthreads();
        // 3. columns j > c, one warp each: u . a_j over the rows below c, the
        //    scalars w = bp (v0 a_j[c] + u . a_j), a_j[c] -= w v0, a_j -= w u
        const int kind = sh_kind[c];
        for (int j = c + 1 + warp; j < w; j += NW) {
            const int ecj = sh_ec[j];
            int32_t* Fj = a.F + (int64_t)j * r;
            int64_t acc[M];
#pragma unroll
            for (int k = 0; k < M; ++k) acc[k] = 0;
            int cj = 0;
            for (int64_t i = c + 1 + lane; i < r; i += 32) {
                int32_t u[D], x[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    u[k] = Fc[k * fs + i];
                    x[k] = Fj[k * fs + i];
                }
                dot_acc<D>(u, x, acc);
                if ((++cj & 255) == 0) carry_norm<M>(acc);
            }
            carry_norm<M>(acc);  // digits below 2^24: 32 of them sum in an int
            int64_t mine = 0;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int sk = __reduce_add_sync(0xffffffffu, (int)acc[k]);
                if (lane == k) mine = sk;
            }
            const fxw::wxf v0{lane < N ? sh_v0[lane] : 0, sh_v0[N]};
            const fxw::wxf bp{lane < N ? sh_bp[lane] : 0, sh_bp[N]};
            const int32_t xe = lane < D ? Fj[lane * fs + c] : 0;
            const fxw::wxf x_c = fxw::from_fixed<N, D>(xe, ecj);
            const fxw::wxf sv = fxw::add<N>(fxw::from_acc<N, M>(mine, eu + ecj + D - 3), fxw::mul<N>(v0, x_c));
            const fxw::wxf W = fxw::mul<N>(bp, sv);
            int32_t xn;
            bool ok = fxw::fixed_from_xf<N, D>(fxw::sub<N>(x_c, fxw::mul<N>(W, v0)), ecj, xn);
            if (lane < D) Fj[lane * fs + c] = xn;
            int32_t wdk = 0;
            if (kind == 0) ok = fxw::fixed_from_xf<N, D>(W, ecj - eu - (D - 2), wdk) && ok;
            if (!ok && lane == 0) set_status(&a.hdr->status, MDLS_ERR_UNSUPPORTED);
            if (kind == 0) {
                int32_t wd[D];
#pragma unroll
                for (int k = 0; k < D; ++k) wd[k] = __shfl_sync(0xffffffffu, wdk, k);
                for (int64_t i = c + 1 + lane; i < r; i += 32) {
                    int32_t u[D], x[D];
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        u[k] = Fc[k * fs + i];
                        x[k] = Fj[k * fs + i];
                    }
                    axpy_row<D>(x, wd, u);
#pragma unroll
                    for (int k = 0; k < D; ++k) Fj[k * fs + i] = x[k];
                }
            }
        }
        __syncthreads();
    }

    // 4. write back every column: R above the diagonal, v = u / v0 below it
    for (int c = 0; c < w; ++c) {
        double* colc = base + (int64_t)c * a.ld;
        const int32_t* Fc = a.F + (int64_t)c * r;
        const bool fin = sh_fin[c] != 0;
        const int ec = sh_ec[c], eu = sh_eu[c];
        xf<N> inv;
#pragma unroll
        for (int k = 0; k < N; ++k) inv.d[k] = sh_inv[c][k];
        inv.e = sh_inv[c][N];
        for (int64_t i = tid; i < r; i += NT) {
            if (i == c) continue;
            int32_t x[D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = Fc[k * fs + i];
            md<P> y;
            if (!fin) y = md_from_double<P>(dnan());
            else if (i < c) y = xf_to_md<P, N>(xf_from_fixed<N, D>(x, ec));
            else y = xf_to_md<P, N>(xf_mul<N>(xf_from_fixed<N, D>(x, eu), inv));
            st_md<P>(colc, ps, i, y);
        }
    }
}

}  // namespace mdls
