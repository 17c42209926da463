// Host-side launch sequences of Algorithms 1 and 2, templated on the limb
// count P.  Each precision is instantiated in its own translation unit.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "split.cuh"
#include "split_tc.cuh"
#include "layout.h"
#include "panel_fx.cuh"
#include "bs_persist.cuh"
#include "profile.h"

namespace mdls {

// Integer-digit panel: threads per column.  The kernel is built for two
// blocks per SM (all w column blocks of a tile up to 256 wide must be
// resident at once); octo double needs more than 128 registers per thread
// and keeps 128 threads.
template <int P>
constexpr int fx_panel_threads() {
    return P == 8 ? 128 : 256;
}

// Single-block digit panel (batched problems): threads of its one block.
template <int P>
constexpr int fx_block_threads() {
    return P == 8 ? 128 : 256;
}

#define MDLS_LAUNCH_CHECK()                                  \
    do {                                                     \
        if (cudaGetLastError() != cudaSuccess) return MDLS_ERR_CUDA; \
    } while (0)

// Width of the diagonal leaves of T (the WY form): each leaf is a serial
// chain of L - 1 md steps on one warp, the levels above it parallel
// products; the longer md operations of qd and od favour shorter chains.
template <int P>
constexpr int wy_leaf() {
    return P == 2 ? 16 : 8;
}

// Per-device values looked up once (the current device's index selects the
// slot; devices beyond kMaxDev share the last slot's lookup each time).
constexpr int kMaxDev = 64;
inline int cur_dev() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}

inline int sm_count() {
    static int sms[kMaxDev] = {};
    const int dev = cur_dev();
    int v = (dev >= 0 && dev < kMaxDev) ? sms[dev] : 0;
    if (v == 0) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
        if (dev >= 0 && dev < kMaxDev) sms[dev] = v;
    }
    return v;
}

// Digit slices of the tensor-core split products (precision mode "split").
struct TcBuf {
    __nv_bfloat16* As;
    __nv_bfloat16* Bs;
    int* ea;
    int* fb;
    size_t as_cap, bs_cap;  // bf16 elements
    int64_t sc_cap;         // ints in ea and in fb
    WsHeader* hdr;          // status word and wait limit of the tcgen05 products
};

// Scratch for split-K partial sums (cap md values per plane), and the
// tensor-core slices when the split mode is on (tc != nullptr).
struct SplitBuf {
    double* ptr;
    int64_t cap;
    const TcBuf* tc = nullptr;
    bool whole_gpu = false;  // the launch has the GPU to itself: split K for whole waves
};

template <int P>
void split_gemm_setup() {
    static bool done[kMaxDev] = {};
    const int dev = cur_dev();
    const int d = (dev >= 0 && dev < kMaxDev) ? dev : kMaxDev - 1;
    if (!done[d]) {
        cudaFuncSetAttribute(split_gemm_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)split_gemm_smem<P>());
        done[d] = true;
    }
}

// C = [C] +/- A B through the digit slices on the tensor cores.
template <int P, class AV, class BV>
int launch_split_gemm(int stage, cudaStream_t st, const TcBuf& tc, int64_t M, int64_t N, int64_t K,
                      AV a, BV b, Dense c, bool neg, bool acc) {
    constexpr int S = SplitCfg<P>::S;
    const int64_t Kp = (K + kSplitTk - 1) / kSplitTk * kSplitTk;
    split_gemm_setup<P>();
    StageScope sc(stage, st);
    split_rows_kernel<P, AV><<<(unsigned)((M * 32 + 255) / 256), 256, 0, st>>>(M, K, Kp, a, tc.As, tc.ea);
    MDLS_LAUNCH_CHECK();
    split_rows_kernel<P, ViewTranspose<BV>><<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(
        N, K, Kp, ViewTranspose<BV>{b}, tc.Bs, tc.fb);
    MDLS_LAUNCH_CHECK();
    dim3 grid((unsigned)((M + kSplitTm - 1) / kSplitTm), (unsigned)((N + kSplitTn - 1) / kSplitTn));
    split_gemm_kernel<P><<<grid, 256, split_gemm_smem<P>(), st>>>(M, N, Kp, tc.As, tc.Bs, tc.ea, tc.fb, c,
                                                                 neg ? 1 : 0, acc ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    (void)S;
    return MDLS_OK;
}

// Which split-product kernel a product uses (mdls_set_split_engine):
// automatic (tcgen05 for products of at least 64 rows and 16 columns on a
// whole GPU, mma.sync otherwise), mma.sync only, or tcgen05 wherever the
// slices fit.
template <int P>
bool split_tc_setup() {
    static bool done[kMaxDev] = {};
    static bool ok[kMaxDev] = {};
    const int dev = cur_dev();
    const int d = (dev >= 0 && dev < kMaxDev) ? dev : kMaxDev - 1;
    if (!done[d]) {
        ok[d] = cudaFuncSetAttribute(split_gemm_tc_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)split_tc_smem<P>()) == cudaSuccess;
        done[d] = true;
    }
    return ok[d];
}

template <int P>
bool split_tc_eligible(const TcBuf& tc, const SplitBuf& sb, int64_t M, int64_t N, int64_t K) {
    const int eng = split_engine_ref();
    if (eng == MDLS_SPLIT_ENGINE_MMA_SYNC || tc.hdr == nullptr) return false;
    if (eng == MDLS_SPLIT_ENGINE_AUTO && (!sb.whole_gpu || M < 64 || N < 16)) return false;
    using Cfg = TcCfg<P>;
    const int64_t Kp = (K + 15) / 16 * 16;
    const int64_t Mp = (M + kTcRows - 1) / kTcRows * kTcRows, Np = (N + Cfg::NT - 1) / Cfg::NT * Cfg::NT;
    return (size_t)Cfg::S * Mp * Kp <= tc.as_cap && (size_t)Cfg::SP * Np * Kp <= tc.bs_cap && M <= tc.sc_cap &&
           N <= tc.sc_cap;
}

// C = [C] +/- A B through the digit slices on tcgen05 (split_tc.cuh).  When
// the output tiles alone would leave SMs idle, K is split over grid.y (each
// block's exact partial product rounded to P limbs into `sb`, added in a
// fixed order by split_reduce_kernel).
template <int P, class AV, class BV>
int launch_split_gemm_tc(int stage, cudaStream_t st, const TcBuf& tc, const SplitBuf& sb, int64_t M, int64_t N,
                         int64_t K, AV a, BV b, Dense c, bool neg, bool acc) {
    using Cfg = TcCfg<P>;
    if (!split_tc_setup<P>()) return MDLS_ERR_CUDA;
    const int64_t KB16 = (K + 15) / 16;
    const int64_t Mp = (M + kTcRows - 1) / kTcRows * kTcRows, Np = (N + Cfg::NT - 1) / Cfg::NT * Cfg::NT;
    StageScope sc(stage, st);
    const unsigned kch = (unsigned)((KB16 * 16 + kTcConvK - 1) / kTcConvK);
    split_scale_kernel<AV><<<(unsigned)((M * 32 + 255) / 256), 256, 0, st>>>(M, K, a, tc.ea);
    MDLS_LAUNCH_CHECK();
    split_rows_tc_kernel<P, kTcRows, Cfg::S, AV><<<dim3((unsigned)((Mp * 32 + 255) / 256), kch), 256, 0, st>>>(
        M, Mp, K, KB16, a, tc.As, tc.ea);
    MDLS_LAUNCH_CHECK();
    split_scale_kernel<ViewTranspose<BV>><<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(N, K, ViewTranspose<BV>{b},
                                                                                            tc.fb);
    MDLS_LAUNCH_CHECK();
    split_rows_tc_kernel<P, Cfg::NT, Cfg::SP, ViewTranspose<BV>>
        <<<dim3((unsigned)((Np * 32 + 255) / 256), kch), 256, 0, st>>>(N, Np, K, KB16, ViewTranspose<BV>{b}, tc.Bs,
                                                                       tc.fb);
    MDLS_LAUNCH_CHECK();
    const int64_t tiles = (Mp / kTcRows) * (Np / Cfg::NT);
    const int64_t groups = (KB16 + Cfg::DK - 1) / Cfg::DK;
    // K split when the tiles alone leave SMs idle: the split minimising
    // waves x groups per block (one block per SM), to at most 16 parts
    int64_t ks = 1;
    const int64_t sms = sm_count();
    if (tiles < sms && sb.ptr != nullptr && groups >= 2) {
        int64_t best = groups;  // one wave of whole K ranges
        for (int64_t s = 2; s <= 16 && s <= groups; ++s) {
            if (s * M * N > sb.cap) break;
            const int64_t c = ((tiles * s + sms - 1) / sms) * ((groups + s - 1) / s);
            if (c < best) {
                best = c;
                ks = s;
            }
        }
    }
    int64_t kb_per = (groups + ks - 1) / ks * Cfg::DK;
    ks = (KB16 + kb_per - 1) / kb_per;
    dim3 grid((unsigned)tiles, (unsigned)ks);
    if (ks == 1) {
        split_gemm_tc_kernel<P><<<grid, kTcThreads, split_tc_smem<P>(), st>>>(
            M, N, KB16, kb_per, tc.As, tc.Bs, tc.ea, tc.fb, c, neg ? 1 : 0, acc ? 1 : 0, 0, tc.hdr);
        MDLS_LAUNCH_CHECK();
        return MDLS_OK;
    }
    split_gemm_tc_kernel<P><<<grid, kTcThreads, split_tc_smem<P>(), st>>>(
        M, N, KB16, kb_per, tc.As, tc.Bs, tc.ea, tc.fb, Dense{sb.ptr, M, sb.cap}, 0, 0, M * N, tc.hdr);
    MDLS_LAUNCH_CHECK();
    const int64_t total = M * N;
    split_reduce_kernel<P><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(M, N, (int)ks, sb.ptr, M, sb.cap, M * N,
                                                                          c, neg ? 1 : 0, acc ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// Digit slices of an operand used in several split products (converted once).
struct TcOperand {
    __nv_bfloat16* s;  // [S][rows][Kp]
    int* e;            // per-row scales
    int64_t rows, K, Kp;
};

template <int P, class AV>
int split_convert(int stage, cudaStream_t st, const TcOperand& op, AV a) {
    StageScope sc(stage, st);
    split_rows_kernel<P, AV><<<(unsigned)((op.rows * 32 + 255) / 256), 256, 0, st>>>(op.rows, op.K, op.Kp, a,
                                                                                     op.s, op.e);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// C = [C] +/- A B with A's slices already in `A` and B (K x N) converted here
// into `bs` / `fb` (room for N columns).
template <int P, class BV>
int split_gemm_pre(int stage, cudaStream_t st, const TcOperand& A, __nv_bfloat16* bs, int* fb, int64_t N, BV b,
                   Dense c, bool neg, bool acc) {
    split_gemm_setup<P>();
    StageScope sc(stage, st);
    split_rows_kernel<P, ViewTranspose<BV>><<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(
        N, A.K, A.Kp, ViewTranspose<BV>{b}, bs, fb);
    MDLS_LAUNCH_CHECK();
    dim3 grid((unsigned)((A.rows + kSplitTm - 1) / kSplitTm), (unsigned)((N + kSplitTn - 1) / kSplitTn));
    split_gemm_kernel<P><<<grid, 256, split_gemm_smem<P>(), st>>>(A.rows, N, A.Kp, A.s, bs, A.e, fb, c,
                                                                 neg ? 1 : 0, acc ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// One md matrix-vector product (N = 1).  Rows contiguous in memory: 32 rows
// per block on the lanes, k split over the block's warps and, when the rows
// alone would leave SM sub-partitions idle, over grid.y (partials in `sb`,
// added in a fixed order).  Otherwise one warp per row, lanes along k.
template <int P, class AV, class BV>
int launch_gemv(int stage, cudaStream_t st, SplitBuf sb, int64_t M, int64_t K, AV a, BV b, Dense c,
                bool neg, bool acc) {
    if (M <= 0) return MDLS_OK;
    StageScope sc(stage, st);
    const int64_t target = 4 * (int64_t)sm_count();  // warps: one per SM sub-partition
    int64_t S = 1;
    int64_t blocks, warps_per_block;
    if constexpr (AV::kRowContig) {
        blocks = (M + 31) / 32;
        warps_per_block = 4;
    } else {
        blocks = (M + 3) / 4;
        warps_per_block = 4;
    }
    const int64_t minK = AV::kRowContig ? 2 * warps_per_block : 64;
    if (blocks * warps_per_block < target && K >= 2 * minK && sb.ptr != nullptr) {
        S = (target + blocks * warps_per_block - 1) / (blocks * warps_per_block);
        if (S > 16) S = 16;
        if (S > K / minK) S = K / minK;
        while (S > 1 && S * M > sb.cap) --S;
    }
    int64_t kchunk = K > 0 ? K : 1;
    if (S > 1) {
        kchunk = (K + S - 1) / S;
        S = (K + kchunk - 1) / kchunk;
    }
    dim3 grid((unsigned)blocks, (unsigned)S);
    Dense out = S > 1 ? Dense{sb.ptr, M, sb.cap} : c;
    const int n_ = S > 1 ? 0 : (neg ? 1 : 0), a_ = S > 1 ? 0 : (acc ? 1 : 0);
    if constexpr (AV::kRowContig)
        gemv_kpar_kernel<P, 4, AV, BV><<<grid, 128, 0, st>>>(M, K, a, b, out, n_, a_, kchunk, M);
    else
        gemv_warps_kernel<P, AV, BV><<<grid, 128, 0, st>>>(M, K, a, b, out, n_, a_, kchunk, M);
    MDLS_LAUNCH_CHECK();
    if (S > 1) {
        split_reduce_kernel<P><<<(unsigned)((M + 127) / 128), 128, 0, st>>>(M, 1, (int)S, sb.ptr, M, sb.cap, M,
                                                                          c, neg ? 1 : 0, acc ? 1 : 0);
        MDLS_LAUNCH_CHECK();
    }
    return MDLS_OK;
}

// The levels of the recursive combination X12 = -X1 M12 X2 (kernels.cuh) for
// `ntiles` tiles of width t (the last one min(t, n - (ntiles-1) t)), whose
// leaves of size L are already in place: block sizes s = L, 2L, ... < t, two
// launches per level for all pairs of all tiles.
template <int P>
int tri_levels(int stage, cudaStream_t st, double* X, int64_t ldx, int64_t psx, int64_t xtile,
               const double* M, int64_t ldm, int64_t psm, int64_t mtile, int64_t n, int t,
               int64_t ntiles, int L, int s_end = 1 << 30) {
    StageScope sc(stage, st);
    for (int s = L; s < t && s < s_end; s *= 2) {
        const int nbi = (s + 7) / 8, nbj = (s + 3) / 4;
        // k groups of at least 8 values of k (16 for s = 128) when the level
        // has few blocks; of at least 32 when the blocks of all tiles already
        // hold eight warps per SM
        const int64_t blocks = (int64_t)nbi * nbj * ((t + 2 * s - 1) / (2 * s)) * ntiles;
        const int kmin = blocks >= 8 * (int64_t)sm_count() ? 32 : 8;
        int KS = 1;
        while (KS * kmin < s && KS < 8) KS *= 2;
        dim3 grid((unsigned)(nbi * nbj), (unsigned)((t + 2 * s - 1) / (2 * s)), (unsigned)ntiles);
        const size_t smem = (size_t)KS * 32 * sizeof(md<P>);
        tri_level_kernel<P, 0><<<grid, 32 * KS, smem, st>>>(X, ldx, psx, xtile, M, ldm, psm, mtile, n, t, s);
        MDLS_LAUNCH_CHECK();
        tri_level_kernel<P, 1><<<grid, 32 * KS, smem, st>>>(X, ldx, psx, xtile, M, ldm, psm, mtile, n, t, s);
        MDLS_LAUNCH_CHECK();
    }
    return MDLS_OK;
}

// Resident blocks per SM of one md GEMM instance (occupancy query, once per
// device).
template <int P, class AV, class BV>
int gemm_blocks_per_sm() {
    static int nb[kMaxDev] = {};
    const int dev = cur_dev();
    const int d = (dev >= 0 && dev < kMaxDev) ? dev : kMaxDev - 1;
    if (nb[d] == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_kernel<P, AV, BV>, kGemmTile * gemm_tn<P>(), 0) !=
                cudaSuccess ||
            v < 1)
            v = 1;
        nb[d] = v;
    }
    return nb[d];
}

// Launches one md GEMM.  The K range may be split over grid.z (at most 16
// ways, partials in `sb`, a reduction kernel adding them in a fixed order).
// When the launch has the GPU to itself the split is the one that minimises
// waves x K-chunk length, the launch's time when every block takes the same
// time, so that small output grids fill the GPU and large ones do not end on
// a mostly idle partial wave (an od product of 648 blocks on 456 block slots
// is 1.4 waves, busy 71 % of the time; split in two over K, 2.8 of 3).  A
// split must save 3 %.  Beside other launches small grids are split to about
// twice the SM count.
template <int P, class AV, class BV>
int launch_gemm(int stage, cudaStream_t st, SplitBuf sb, int64_t M, int64_t N, int64_t K, AV a, BV b,
                Dense c, bool neg, bool acc, bool upper_only = false) {
    if (M <= 0 || N <= 0) return MDLS_OK;
    if (sb.tc != nullptr && K > 0) {
        if (split_tc_eligible<P>(*sb.tc, sb, M, N, K))
            return launch_split_gemm_tc<P>(stage, st, *sb.tc, sb, M, N, K, a, b, c, neg, acc);
        const int64_t Kp = (K + kSplitTk - 1) / kSplitTk * kSplitTk;
        constexpr int S = SplitCfg<P>::S;
        if ((size_t)S * M * Kp <= sb.tc->as_cap && (size_t)S * N * Kp <= sb.tc->bs_cap &&
            M <= sb.tc->sc_cap && N <= sb.tc->sc_cap)
            return launch_split_gemm<P>(stage, st, *sb.tc, M, N, K, a, b, c, neg, acc);
    }
    if (N == 1 && !upper_only) return launch_gemv<P>(stage, st, sb, M, K, a, b, c, neg, acc);
    StageScope sc(stage, st);
    constexpr int TN = gemm_tn<P>();
    const int64_t gx = (M + kGemmTile - 1) / kGemmTile, gy = (N + TN - 1) / TN;
    const int64_t tiles = upper_only ? (gx * gy + gx) / 2 : gx * gy;
    const int64_t target = 2 * (int64_t)sm_count();
    int64_t S = 1;
    if (!sb.whole_gpu) {
        // beside other launches (batched problems): fill twice the SM count
        if (tiles < target && K >= 4 * kGemmTile && sb.ptr != nullptr) {
            S = (target + tiles - 1) / tiles;
            if (S > 16) S = 16;
            if (S > K / (2 * kGemmTile)) S = K / (2 * kGemmTile);
            while (S > 1 && S * M * N > sb.cap) --S;
        }
    } else if (K >= 4 * kGemmTile && sb.ptr != nullptr) {
        const int64_t slots = (int64_t)sm_count() * gemm_blocks_per_sm<P, AV, BV>();
        auto cost = [&](int64_t s, int64_t& parts) {
            int64_t kc = (K + s - 1) / s;
            kc = (kc + kGemmTile - 1) / kGemmTile * kGemmTile;
            parts = (K + kc - 1) / kc;
            return (tiles * parts + slots - 1) / slots * kc;
        };
        int64_t parts = 1;
        int64_t best = cost(1, parts);
        for (int64_t s = 2; s <= 16 && K / s >= 2 * kGemmTile; ++s) {
            const int64_t c = cost(s, parts);
            if (parts * M * N > sb.cap) break;
            if (c * 100 < best * 97) {
                best = c;
                S = parts;
            }
        }
    }
    int64_t kchunk = K;
    if (S > 1) {
        kchunk = (K + S - 1) / S;
        kchunk = (kchunk + kGemmTile - 1) / kGemmTile * kGemmTile;
        S = (K + kchunk - 1) / kchunk;
    }
    if (K <= 0) kchunk = 1;
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)S);
    if (S == 1) {
        gemm_kernel<P, AV, BV><<<grid, kGemmTile * TN, 0, st>>>(
            M, N, K, a, b, c, neg ? 1 : 0, acc ? 1 : 0, kchunk, 0, upper_only ? 1 : 0);
        MDLS_LAUNCH_CHECK();
        return MDLS_OK;
    }
    Dense part{sb.ptr, M, sb.cap};
    gemm_kernel<P, AV, BV><<<grid, kGemmTile * TN, 0, st>>>(M, N, K, a, b, part, 0, 0, kchunk,
                                                             M * N, upper_only ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    const int64_t total = M * N;
    split_reduce_kernel<P><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(
        M, N, (int)S, sb.ptr, M, sb.cap, M * N, c, neg ? 1 : 0, acc ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// Largest panel width the column-per-block cooperative panel can hold.
template <int P>
int panel_capacity() {
    static int cap[kMaxDev] = {};
    const int dev = cur_dev();
    const int d = (dev >= 0 && dev < kMaxDev) ? dev : kMaxDev - 1;
    if (cap[d] <= 0) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fx_panel_kernel<P, fx_panel_threads<P>()>, fx_panel_threads<P>(), 0);
        cap[d] = sm_count() * per;
    }
    return cap[d];
}

// Look-ahead: the next tile's panel runs on a high-priority side stream
// beside the rest of this tile's trailing update (the panel is bound by the
// latency of its column chain and leaves most of each SM's FP64 pipe to the
// product).  One side stream and two events per host thread.
struct LookAhead {
    cudaStream_t hi = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
    bool ok = false;
};

inline LookAhead& look_ahead() {
    // per host thread and per device: the side stream and its events belong
    // to the device that was current when they were created
    thread_local LookAhead la[kMaxDev];
    thread_local bool tried[kMaxDev] = {};
    const int dev = cur_dev();
    const int d = (dev >= 0 && dev < kMaxDev) ? dev : kMaxDev - 1;
    if (!tried[d]) {
        tried[d] = true;
        int least = 0, greatest = 0;
        la[d].ok = dev == d && cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
                   cudaStreamCreateWithPriority(&la[d].hi, cudaStreamNonBlocking, greatest) == cudaSuccess &&
                   cudaEventCreateWithFlags(&la[d].ready, cudaEventDisableTiming) == cudaSuccess &&
                   cudaEventCreateWithFlags(&la[d].done, cudaEventDisableTiming) == cudaSuccess;
    }
    return la[d];
}

// Blocked Householder QR (Algorithm 2) of the m x n leading part of the
// working matrix A (ld, ps); columns n .. n+nextra-1 of A are right-hand
// sides that receive the same transformations (Q^T b).  Q (m x m) is formed
// when Q != nullptr.  R is left in the upper triangle, the Householder
// vectors below it; zero_lower clears them at the end.
template <int P>
int qr_run(int64_t m, int64_t n, int nextra, double* A, int64_t lda, int64_t psa, double* Q,
           int64_t ldq, int64_t psq, int t, char* ws, const QrLayout& L, WsHeader* hdr,
           bool zero_lower, cudaStream_t st, bool keep_w = false, bool single_block = false) {
    static_assert(fx_digits(P) == fx::Cfg<P>::D && fx_meta_ints(P) == FxMeta<P>::ints,
                  "host and device digit layouts differ");
    double* beta = reinterpret_cast<double*>(ws + L.beta);
    double* G = reinterpret_cast<double*>(ws + L.G);
    double* T = reinterpret_cast<double*>(ws + L.T);
    double* X = reinterpret_cast<double*>(ws + L.X);
    double* Wb = reinterpret_cast<double*>(ws + L.W);
    unsigned int* flags = reinterpret_cast<unsigned int*>(ws + L.flags);
    int32_t* fxF = reinterpret_cast<int32_t*>(ws + L.fxF);
    int32_t* fxmeta = reinterpret_cast<int32_t*>(ws + L.fxmeta);
    TcBuf tcb{};
    if (L.tc_as_cap > 0) {
        tcb = TcBuf{reinterpret_cast<__nv_bfloat16*>(ws + L.tc_as), reinterpret_cast<__nv_bfloat16*>(ws + L.tc_bs),
                    reinterpret_cast<int*>(ws + L.tc_ea), reinterpret_cast<int*>(ws + L.tc_fb),
                    L.tc_as_cap, L.tc_bs_cap, L.tc_sc_cap, hdr};
    }
    const SplitBuf sb{reinterpret_cast<double*>(ws + L.split), L.split_cap,
                      L.tc_as_cap > 0 ? &tcb : nullptr, !single_block};
    const int64_t tt2 = (int64_t)t * t;
    const int64_t psx = (int64_t)t * L.xcols;
    const int64_t ldw = m;
    const int64_t psw = L.wcols * m;
    const int64_t ntiles = (n + t - 1) / t;
    const bool want_q = (Q != nullptr);

    // 1. panel of tile k: Householder vectors, beta, R_kk.  One block per
    //    column in integer digits with flags between them (cooperative
    //    launch); the small problems of batched solves use the single-block
    //    panel.
    auto panel = [&](int64_t k, cudaStream_t s) -> int {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        StageScope sc(ST_PANEL, s);
        if (single_block) {
            FxBlockPanelArgs pa{A, lda, psa, j0, r, w, beta, (int64_t)t, fxF, hdr};
            fx_panel_block_kernel<P, fx_block_threads<P>()><<<1, fx_block_threads<P>(), 0, s>>>(pa);
            return cudaGetLastError() == cudaSuccess ? MDLS_OK : MDLS_ERR_CUDA;
        }
        if (w > panel_capacity<P>()) return MDLS_ERR_UNSUPPORTED;
        FxPanelArgs pa{A, lda, psa, j0, r, w, beta, (int64_t)t, fxF, fxmeta, flags, (unsigned int)(k + 1), hdr};
        void* args[] = {&pa};
        if (cudaLaunchCooperativeKernel((const void*)fx_panel_kernel<P, fx_panel_threads<P>()>, dim3(w),
                                        dim3(fx_panel_threads<P>()), args, 0, s) != cudaSuccess)
            return MDLS_ERR_CUDA;
        return MDLS_OK;
    };
    // 2. WY form of tile k: G = Y^T Y, T from G and the betas, W = -Y T.
    //    With look-ahead it runs on the side stream right after tile k's
    //    panel (its own split-K buffer; W alternates between two slots when
    //    only the current tile's W is kept).
    auto wy_w = [&](int64_t k) -> double* {
        const int64_t j0 = k * t;
        return (want_q || keep_w) ? (Wb + j0 * ldw + j0) : (Wb + (k & 1) * (int64_t)t * ldw);
    };
    auto wy = [&](int64_t k, cudaStream_t s, const SplitBuf& sbk) -> int {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        const double* Yp = A + j0 * lda + j0;
        ViewTrap Y{Yp, lda, psa};
        ViewTrapT Yt{Yp, lda, psa};
        int rc = launch_gemm<P>(ST_W, s, sbk, w, w, r, Yt, Y, Dense{G, t, tt2}, false, false, true);
        if (rc) return rc;
        {
            constexpr int kLeaf = wy_leaf<P>();
            const int L = w < kLeaf ? w : kLeaf;
            StageScope sc(ST_W, s);
            // one warp (two rows) per block: the leaves spread over w/2 SMs
            wy_t_leaf_kernel<P><<<(unsigned)((w + 1) / 2), 32, 0, s>>>(G, t, tt2, beta, t, w, L, T, t, tt2);
            MDLS_LAUNCH_CHECK();
            // in octo double split mode the levels of 32 columns and more are
            // split products (tensor cores); the narrower ones, and every level
            // in dd and qd (measured: their shorter md operations make the FP64
            // levels cheaper than the products' launches), stay on the FP64 pipe
            constexpr int kSplitLevel = 32;
            const bool split_levels = P == 8 && sbk.tc != nullptr;
            rc = tri_levels<P>(ST_W, s, T, t, tt2, 0, G, t, tt2, 0, w, w, 1, L, split_levels ? kSplitLevel : 1 << 30);
            if (rc) return rc;
            if (split_levels) {
                for (int lv = kSplitLevel > L ? kSplitLevel : L; lv < w; lv *= 2)
                    for (int a = 0; a + lv < w; a += 2 * lv) {
                        const int s2 = (w - a - lv) < lv ? (w - a - lv) : lv;
                        // T12 = -T1 (G12 T2): Z^T = T2^T G12^T into the unused
                        // lower block (rows a+lv.., columns a..), then T12 = -T1 Z
                        double* Tl = T + (int64_t)a * t + a + lv;
                        rc = launch_gemm<P>(ST_W, s, sbk, s2, lv, s2,
                                            ViewUpperT{T + (int64_t)(a + lv) * t + a + lv, t, tt2},
                                            ViewDenseT{G + (int64_t)(a + lv) * t + a, t, tt2}, Dense{Tl, t, tt2},
                                            false, false);
                        if (rc) return rc;
                        rc = launch_gemm<P>(ST_W, s, sbk, lv, s2, lv, ViewUpper{T + (int64_t)a * t + a, t, tt2},
                                            ViewDenseT{Tl, t, tt2}, Dense{T + (int64_t)(a + lv) * t + a, t, tt2},
                                            true, false);
                        if (rc) return rc;
                    }
            }
        }
        return launch_gemm<P>(ST_W, s, sbk, r, w, w, Y, ViewUpper{T, t, tt2}, Dense{wy_w(k), ldw, psw}, true,
                              false);
    };
    // WY products on the side stream only in plain arithmetic (the split
    // mode's digit buffers are shared by all products)
    const SplitBuf sb_side{reinterpret_cast<double*>(ws + L.split_side), L.split_side_cap, nullptr, false};
    const bool wy_side = (L.tc_as_cap == 0);
    // look-ahead only for the one-problem path outside graph capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LookAhead* la = nullptr;
    if (!single_block && cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone &&
        look_ahead().ok)
        la = &look_ahead();
    bool panel_ahead = false;  // tile k's panel was launched on the side stream
    bool wy_ahead = false;     // and its WY form after it
    // every return joins the side stream back into st
    struct Join {
        LookAhead* la;
        cudaStream_t st;
        const bool& pending;
        ~Join() {
            if (pending) cudaStreamWaitEvent(st, la->done, 0);
        }
    } join{la, st, panel_ahead};

    for (int64_t k = 0; k < ntiles; ++k) {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        const bool have_wy = wy_ahead;
        if (panel_ahead) {
            if (cudaStreamWaitEvent(st, la->done, 0) != cudaSuccess) return MDLS_ERR_CUDA;
            panel_ahead = false;
            wy_ahead = false;
        } else {
            const int prc = panel(k, st);
            if (prc) return prc;
        }
        const int64_t nc = n + nextra - (j0 + w);  // trailing columns incl. right-hand sides
        if (nc <= 0 && !want_q && !keep_w) continue;
        int rc = MDLS_OK;
        if (!have_wy) {
            rc = wy(k, st, sb);
            if (rc) return rc;
        }
        const double* Yp = A + j0 * lda + j0;
        ViewTrap Y{Yp, lda, psa};
        double* Wk = wy_w(k);
        // 3. trailing update C := C + Y (W^T C); with look-ahead first the
        //    next tile's wn columns, then that tile's panel on the side
        //    stream, then the other columns here
        if (nc > 0) {
            const int64_t wn = (k + 1 < ntiles) ? ((n - j0 - w) < t ? (n - j0 - w) : t) : 0;
            const int64_t nfirst = (la != nullptr && wn > 0 && nc > wn) ? wn : nc;
            double* Cp = A + (j0 + w) * lda + j0;
            rc = launch_gemm<P>(ST_TRAIL, st, sb, w, nfirst, r, ViewDenseT{Wk, ldw, psw}, ViewDense{Cp, lda, psa},
                                Dense{X, t, psx}, false, false);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_TRAIL, st, sb, r, nfirst, w, Y, ViewDense{X, t, psx}, Dense{Cp, lda, psa}, false,
                                true);
            if (rc) return rc;
            if (nfirst < nc) {
                if (cudaEventRecord(la->ready, st) != cudaSuccess ||
                    cudaStreamWaitEvent(la->hi, la->ready, 0) != cudaSuccess)
                    return MDLS_ERR_CUDA;
                const int prc = panel(k + 1, la->hi);
                if (prc) return prc;
                panel_ahead = true;
                const int64_t nc1 = n + nextra - (j0 + w + wn);
                if (wy_side && (nc1 > 0 || want_q || keep_w)) {
                    const int wrc = wy(k + 1, la->hi, sb_side);
                    if (wrc) return wrc;
                    wy_ahead = true;
                }
                if (cudaEventRecord(la->done, la->hi) != cudaSuccess) return MDLS_ERR_CUDA;
                double* Cq = Cp + nfirst * lda;
                double* Xq = X + nfirst * t;
                rc = launch_gemm<P>(ST_TRAIL, st, sb, w, nc - nfirst, r, ViewDenseT{Wk, ldw, psw},
                                    ViewDense{Cq, lda, psa}, Dense{Xq, t, psx}, false, false);
                if (rc) return rc;
                rc = launch_gemm<P>(ST_TRAIL, st, sb, r, nc - nfirst, w, Y, ViewDense{Xq, t, psx},
                                    Dense{Cq, lda, psa}, false, true);
                if (rc) return rc;
            }
        }
    }
    if (want_q) {
        // 4. Q = P_1 P_2 ... P_N accumulated backward: Q_sub := Q_sub + W (Y^T Q_sub)
        dim3 g((unsigned)((m + 255) / 256), (unsigned)(m < 65535 ? m : 65535));
        {
            StageScope sc(ST_OTHER, st);
            identity_kernel<P><<<g, 256, 0, st>>>(Q, ldq, psq, m);
            MDLS_LAUNCH_CHECK();
        }
        for (int64_t k = ntiles - 1; k >= 0; --k) {
            const int64_t j0 = k * t;
            const int w = (int)((n - j0) < t ? (n - j0) : t);
            const int64_t r = m - j0;
            const double* Yp = A + j0 * lda + j0;
            double* Qs = Q + j0 * ldq + j0;
            double* Wk = Wb + j0 * ldw + j0;
            int rc = launch_gemm<P>(ST_QACC, st, sb, w, r, r, ViewTrapT{Yp, lda, psa}, ViewDense{Qs, ldq, psq},
                                    Dense{X, t, psx}, false, false);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_QACC, st, sb, r, r, w, ViewDense{Wk, ldw, psw}, ViewDense{X, t, psx},
                                Dense{Qs, ldq, psq}, false, true);
            if (rc) return rc;
        }
    }
    if (zero_lower) {
        dim3 g((unsigned)((m + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
        StageScope sc(ST_OTHER, st);
        zero_lower_kernel<P><<<g, 256, 0, st>>>(A, lda, psa, m, n);
        MDLS_LAUNCH_CHECK();
    }
    return MDLS_OK;
}

// Tiled back substitution (Algorithm 1) of R x = y, R upper triangular n x n.
// Step 1: invert the N diagonal tiles into D (tile i at D + i t^2, ld t):
// leaves of kTriLeaf columns, then the recursive levels, all tiles at once.
template <int P>
int bs_invert(int64_t n, const double* R, int64_t ldr, int64_t psr, int t, char* ws,
              const BsLayout& L, WsHeader* hdr, cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t tt2 = (int64_t)t * t;
    double* D = reinterpret_cast<double*>(ws + L.D);
    const int leaf = t < kTriLeaf ? t : kTriLeaf;
    {
        StageScope sc(ST_INV, st);
        const int64_t warps = N * ((t + 1) / 2);
        tri_leaf_inv_kernel<P><<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(R, ldr, psr, n, t, leaf, N, D, t,
                                                                            N * tt2, tt2, hdr);
        MDLS_LAUNCH_CHECK();
    }
    return tri_levels<P>(ST_INV, st, D, t, N * tt2, tt2, R, ldr, psr, (int64_t)t * (ldr + 1), n, t, N, leaf);
}

// Step 2: i = N..1, x_i := U_i^{-1} y_i, then y_j -= A_{j,i} x_i for all j < i
// (both as split matrix-vector products).
template <int P>
int bs_solve(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy,
             double* x, int64_t psx, int t, char* ws, const BsLayout& L, cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t tt2 = (int64_t)t * t;
    double* D = reinterpret_cast<double*>(ws + L.D);
    double* bw = reinterpret_cast<double*>(ws + L.b);
    const SplitBuf sbp{reinterpret_cast<double*>(ws + L.part), kBsPartCap};
    const int64_t dps = N * tt2;
    for (int l = 0; l < P; ++l)
        if (cudaMemcpyAsync(bw + l * n, y + l * psy, n * sizeof(double), cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    for (int64_t i = N - 1; i >= 0; --i) {
        const int64_t o = i * t;
        const int tt = (int)((n - o) < t ? (n - o) : t);
        int rc = launch_gemv<P>(ST_MULINV, st, sbp, tt, tt, ViewUpper{D + i * tt2, t, dps},
                                ViewDense{bw + o, n, n}, Dense{x + o, n, psx}, false, false);
        if (rc) return rc;
        if (o > 0) {
            rc = launch_gemv<P>(ST_BSUPD, st, sbp, o, tt, ViewDense{R + o * ldr, ldr, psr},
                                ViewDense{x + o, n, psx}, Dense{bw, n, n}, true, true);
            if (rc) return rc;
        }
    }
    return MDLS_OK;
}

// Step 2 in one persistent cooperative launch (csrc/bs_persist.cuh): bulk
// updates from a task queue on most SMs, the critical step x_i -> x_{i-1} on
// kBsCritSms reserved SMs.  Needs t a multiple of 32.
template <int P>
int bs_solve_persist(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy,
                     double* x, int64_t psx, int t, char* ws, const BsLayout& L, WsHeader* hdr,
                     cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t nchunks = (n + 31) / 32;
    double* bw = reinterpret_cast<double*>(ws + L.b);
    for (int l = 0; l < P; ++l)
        if (cudaMemcpyAsync(bw + l * n, y + l * psy, n * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return MDLS_ERR_CUDA;
    const int S = t / kBsSlice;
    unsigned int* ctr = reinterpret_cast<unsigned int*>(ws + L.ctr);
    if (cudaMemsetAsync(ctr, 0, 4 * (size_t)bs_ctr_ints(nchunks, S, N), st) != cudaSuccess) return MDLS_ERR_CUDA;
    // blocks per SM: kBsBlocksPerSm, or fewer if that many do not fit (the
    // cooperative launch needs every block resident)
    static int per_sm_dev[kMaxDev] = {};
    const int dev = cur_dev();
    int per_sm = (dev >= 0 && dev < kMaxDev) ? per_sm_dev[dev] : 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, bs_persist_kernel<P>, 128, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v < kBsBlocksPerSm ? v : kBsBlocksPerSm;
        if (dev >= 0 && dev < kMaxDev) per_sm_dev[dev] = per_sm;
    }
    BsPersistArgs a;
    a.R = R;
    a.ldr = ldr;
    a.psr = psr;
    a.D = reinterpret_cast<const double*>(ws + L.D);
    a.dps = N * (int64_t)t * t;
    a.yb = bw;
    a.x = x;
    a.psx = psx;
    a.acc = reinterpret_cast<double*>(ws + L.acc);
    a.tree_cu = reinterpret_cast<double*>(ws + L.tree_cu);
    a.tree_xt = reinterpret_cast<double*>(ws + L.tree_xt);
    a.part_ps = L.part_ps;
    a.ctr = ctr;
    a.n = n;
    a.t = t;
    a.N = (int)N;
    a.nchunks = (int)nchunks;
    a.S = S;
    a.KS = (t / 32) * S;
    a.ncrit = kBsCritSms < sm_count() / 2 ? kBsCritSms : sm_count() / 2;
    if (a.ncrit < 1) a.ncrit = 1;
    a.hdr = hdr;
    StageScope sc(ST_BSUPD, st);
    void* args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void*)bs_persist_kernel<P>, dim3((unsigned)(per_sm * sm_count())),
                                    dim3(128), args, 0, st) != cudaSuccess)
        return MDLS_ERR_CUDA;
    return MDLS_OK;
}

// Schedule of step 2: one launch pair per tile step (the paper's), or the
// persistent launch (chosen process-wide by mdls_set_backsub_schedule).  The
// automatic choice follows measurements on GB300: the persistent launch wins
// in double double from 8 tiles on (n = 1024 to 4096: 5-35 %) and in quad
// double for n >= 8192 (n = 17920: 41.4 -> 35.2 ms at tile 128), where the
// overlapped steps outweigh its latency-bound chain x_i -> x_{i-1} (about
// 150 us per tile step in quad double); octo double stays per step.
inline bool use_persist(int64_t n, int t, int P) {
    if (t % 32 != 0) return false;
    const int s = bs_schedule_ref();
    if (s == MDLS_BS_PER_STEP) return false;
    if (s == MDLS_BS_PERSISTENT) return true;
    if (P == 2) return (n + t - 1) / t >= 8;
    if (P == 4) return n >= 8192;
    return false;
}

template <int P>
int bs_run(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy,
           double* x, int64_t psx, int t, char* ws, const BsLayout& L, WsHeader* hdr,
           cudaStream_t st) {
    int rc = bs_invert<P>(n, R, ldr, psr, t, ws, L, hdr, st);
    if (rc) return rc;
    if (use_persist(n, t, P) && L.ctr != 0) return bs_solve_persist<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, L, hdr, st);
    return bs_solve<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, L, st);
}

// v := Q^T v for the Q = P_1 ... P_N of a factorisation whose Y sit below the
// diagonal of A (ld m) and whose W_k were kept (ld m, plane stride psw):
// v[j0:] := v[j0:] + Y_k (W_k^T v[j0:]) for k = 1..N (each P_k^T = I + Y W^T).
template <int P>
int apply_qt(int64_t m, int64_t n, int t, const double* A, int64_t psa, const double* Wb,
             int64_t psw, double* v, int64_t psv, double* X, int64_t psx, SplitBuf sb, int stage,
             cudaStream_t st) {
    const int64_t ntiles = (n + t - 1) / t;
    for (int64_t k = 0; k < ntiles; ++k) {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        const double* Wk = Wb + j0 * m + j0;
        int rc = launch_gemm<P>(stage, st, sb, w, 1, r, ViewDenseT{Wk, m, psw}, ViewDense{v + j0, m, psv},
                                Dense{X, t, psx}, false, false);
        if (rc) return rc;
        rc = launch_gemm<P>(stage, st, sb, r, 1, w, ViewTrap{A + j0 * m + j0, m, psa},
                            ViewDense{X, t, psx}, Dense{v + j0, m, psv}, false, true);
        if (rc) return rc;
    }
    return MDLS_OK;
}

// Solves R^T h = g (R upper triangular n x n, its diagonal tiles inverted in
// L.D by bs_invert): the block forward substitution of the transposed system,
// h_i := (U_i^{-1})^T g_i, then g_j := g_j - (R_ij)^T h_i for the rows after
// tile i.
template <int P>
int fs_solve(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* g, int64_t psg,
             double* h, int64_t psh, int t, char* ws, const BsLayout& L, int stage, cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t tt2 = (int64_t)t * t;
    const double* D = reinterpret_cast<const double*>(ws + L.D);
    double* gw = reinterpret_cast<double*>(ws + L.b);
    const SplitBuf sbp{reinterpret_cast<double*>(ws + L.part), kBsPartCap};
    for (int l = 0; l < P; ++l)
        if (cudaMemcpyAsync(gw + l * n, g + l * psg, n * sizeof(double), cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t o = i * t;
        const int tt = (int)((n - o) < t ? (n - o) : t);
        int rc = launch_gemv<P>(stage, st, sbp, tt, tt, ViewUpperT{D + i * tt2, t, N * tt2},
                                ViewDense{gw + o, n, n}, Dense{h + o, n, psh}, false, false);
        if (rc) return rc;
        const int64_t rest = n - o - tt;
        if (rest > 0) {
            rc = launch_gemv<P>(stage, st, sbp, rest, tt, ViewDenseT{R + (o + tt) * ldr + o, ldr, psr},
                                ViewDense{h + o, n, psh}, Dense{gw + o + tt, n, n}, true, true);
            if (rc) return rc;
        }
    }
    return MDLS_OK;
}

// v := Q v = P_1 (P_2 (... (P_N v))): v[j0:] := v[j0:] + W_k (Y_k^T v[j0:]), k = N..1.
template <int P>
int apply_q(int64_t m, int64_t n, int t, const double* A, int64_t psa, const double* Wb,
            int64_t psw, double* v, int64_t psv, double* X, int64_t psx, SplitBuf sb, int stage,
            cudaStream_t st) {
    const int64_t ntiles = (n + t - 1) / t;
    for (int64_t k = ntiles - 1; k >= 0; --k) {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        const double* Wk = Wb + j0 * m + j0;
        int rc = launch_gemm<P>(stage, st, sb, w, 1, r, ViewTrapT{A + j0 * m + j0, m, psa},
                                ViewDense{v + j0, m, psv}, Dense{X, t, psx}, false, false);
        if (rc) return rc;
        rc = launch_gemm<P>(stage, st, sb, r, 1, w, ViewDense{Wk, m, psw}, ViewDense{X, t, psx},
                            Dense{v + j0, m, psv}, false, true);
        if (rc) return rc;
    }
    return MDLS_OK;
}

template <int P>
int qr_entry(int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q, int64_t ldq,
             int64_t psq, int t, int mode, void* ws, cudaStream_t st) {
    QrLayout L = qr_layout(P, m, n, t, Q != nullptr, 0, nullptr, mode == MDLS_MODE_SPLIT);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, L.flags + L.flag_bytes, st) != cudaSuccess) return MDLS_ERR_CUDA;
    return qr_run<P>(m, n, 0, A, lda, psa, Q, ldq, psq, t, w, L, hdr, true, st);
}

template <int P>
int bs_entry(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy,
             double* x, int64_t psx, int t, void* ws, cudaStream_t st) {
    BsLayout L = bs_layout(P, n, t);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, sizeof(WsHeader), st) != cudaSuccess) return MDLS_ERR_CUDA;
    return bs_run<P>(n, R, ldr, psr, y, psy, x, psx, t, w, L, hdr, st);
}

template <int P>
int ls_entry(int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa, const double* b,
             int64_t psb, double* x, int64_t psx, int t, int mode, void* ws, cudaStream_t st,
             bool single_block = false) {
    LsLayout L = ls_layout(P, m, n, t, mode == MDLS_MODE_SPLIT);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, L.qr.flags + L.qr.flag_bytes, st) != cudaSuccess) return MDLS_ERR_CUDA;
    double* Aw = reinterpret_cast<double*>(w + L.Aw);
    const int64_t psw = m * (n + 1);
    for (int l = 0; l < P; ++l) {
        if (cudaMemcpy2DAsync(Aw + l * psw, m * sizeof(double), A + l * psa, lda * sizeof(double),
                              m * sizeof(double), n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return MDLS_ERR_CUDA;
        if (cudaMemcpyAsync(Aw + l * psw + n * m, b + l * psb, m * sizeof(double),
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    }
    int rc = qr_run<P>(m, n, 1, Aw, m, psw, nullptr, 0, 0, t, w, L.qr, hdr, false, st, false,
                       single_block);
    if (rc) return rc;
    return bs_run<P>(n, Aw, m, psw, Aw + n * m, psw, x, psx, t, w, L.bs, hdr, st);
}

// Step 2 with the process-wide schedule (per tile step or one persistent
// launch), the diagonal tiles already inverted.
template <int P>
int bs_solve_sched(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy, double* x,
                   int64_t psx, int t, char* ws, const BsLayout& L, WsHeader* hdr, cudaStream_t st) {
    if (use_persist(n, t, P) && L.ctr != 0) return bs_solve_persist<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, L, hdr, st);
    return bs_solve<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, L, st);
}

// Lower triangular block-Toeplitz system (the linear systems of Newton's
// method on power series, the motivation of the paper's Section 1): with
// J(t) = sum_i J_i t^i and b(t) = sum_k b_k t^k, the coefficients x_k of
// J(t) x(t) = b(t) mod t^{d+1} follow by block forward substitution,
//   J_0 x_k = b_k - sum_{i=1}^{k} J_i x_{k-i},   k = 0, ..., d,
// each in the least-squares sense with the one QR of the diagonal block J_0
// (Algorithm 2, every tile's W kept) and Algorithm 1 on its R (diagonal tiles
// inverted once): x_k = R^{-1} (Q^T r_k)[0:n].
template <int P>
int toe_entry(int64_t m, int64_t n, int64_t d, const double* J, int64_t ldj, int64_t psj, int64_t bsj,
              const double* b, int64_t psb, int64_t bsb, double* x, int64_t psx, int64_t bsx, int t, void* ws,
              cudaStream_t st) {
    const ToeLayout L = toe_layout(P, m, n, t);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, L.qr.flags + L.qr.flag_bytes, st) != cudaSuccess) return MDLS_ERR_CUDA;
    double* A2 = reinterpret_cast<double*>(w + L.A2);
    double* r = reinterpret_cast<double*>(w + L.r);
    const int64_t ps2 = m * n;
    const size_t vb = sizeof(double);
    for (int l = 0; l < P; ++l)
        if (cudaMemcpy2DAsync(A2 + l * ps2, m * vb, J + l * psj, ldj * vb, m * vb, n, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return MDLS_ERR_CUDA;
    int rc = qr_run<P>(m, n, 0, A2, m, ps2, nullptr, 0, 0, t, w, L.qr, hdr, false, st, true);
    if (rc) return rc;
    rc = bs_invert<P>(n, A2, m, ps2, t, w, L.bs, hdr, st);
    if (rc) return rc;
    const double* Wb = reinterpret_cast<const double*>(w + L.qr.W);
    double* X = reinterpret_cast<double*>(w + L.qr.X);
    const int64_t psw = L.qr.wcols * m, psX = (int64_t)t * L.qr.xcols;
    const SplitBuf sb{reinterpret_cast<double*>(w + L.qr.split), L.qr.split_cap};
    for (int64_t k = 0; k <= d; ++k) {
        for (int l = 0; l < P; ++l)
            if (cudaMemcpyAsync(r + l * m, b + l * psb + k * bsb, m * vb, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
                return MDLS_ERR_CUDA;
        for (int64_t i = 1; i <= k; ++i) {  // r -= J_i x_{k-i}
            rc = launch_gemv<P>(ST_OTHER, st, sb, m, n, ViewDense{J + i * bsj, ldj, psj},
                                ViewDense{x + (k - i) * bsx, n, psx}, Dense{r, m, m}, true, true);
            if (rc) return rc;
        }
        rc = apply_qt<P>(m, n, t, A2, ps2, Wb, psw, r, m, X, psX, sb, ST_OTHER, st);
        if (rc) return rc;
        rc = bs_solve_sched<P>(n, A2, m, ps2, r, m, x + k * bsx, psx, t, w, L.bs, hdr, st);
        if (rc) return rc;
    }
    return MDLS_OK;
}

template <int P>
int vec_entry(int op, int64_t count, const double* a, int64_t psa, const double* b, int64_t psb,
              double* c, int64_t psc, cudaStream_t st) {
    if (count <= 0) return MDLS_OK;
    StageScope sc(ST_OTHER, st);
    vec_op_kernel<P><<<(unsigned)((count + 127) / 128), 128, 0, st>>>(op, count, a, psa, b, psb, c, psc);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// Least squares in P limbs by double-double factorisation and iterative
// refinement of the augmented system [I A; A^T 0][r; x] = [b; 0] (Bjorck's
// refinement, which converges for inconsistent systems too).  The QR of A
// rounded to dd (its two leading limbs; WY products as split products on the
// tensor cores) gives x0 and r0 = b - A x0; then,
// `iters` times, with the residuals formed in P limbs
//   f = b - r - A x,  g = -A^T r,
// and the corrections solved in dd with the factors A = Q [R; 0]:
//   [f1; f2] = Q^T f,  h = R^{-T} g,  dr = Q [h; f2],  dx = R^{-1} (f1 - h),
// r := r + dr and x := x + dx in P limbs.  A last check records
// MDLS_ERR_NOT_CONVERGED when the final |dx| exceeds 2^(53-53P) |x|.
template <int P>
int ls_refine_entry(int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa, const double* b,
                    int64_t psb, double* x, int64_t psx, int t, int iters, void* ws, cudaStream_t st) {
    RefLayout L = ref_layout(P, m, n, t);
    char* w = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(w, 0, L.qr.flags + L.qr.flag_bytes, st) != cudaSuccess) return MDLS_ERR_CUDA;
    double* A2 = reinterpret_cast<double*>(w + L.A2);
    const int64_t ps2 = m * n;
    double* res = reinterpret_cast<double*>(w + L.res);     // r, P limbs, length m
    double* f = reinterpret_cast<double*>(w + L.f);         // f, P limbs, length m
    double* g = reinterpret_cast<double*>(w + L.g);         // g, P limbs, length n
    double* c = reinterpret_cast<double*>(w + L.c);         // dd, length m
    double* hv = reinterpret_cast<double*>(w + L.h);        // dd, length n
    double* dx = reinterpret_cast<double*>(w + L.d);        // dd, length n
    double* up = reinterpret_cast<double*>(w + L.up);       // P limbs, length m (promoted corrections)
    double* X = reinterpret_cast<double*>(w + L.qr.X);
    const double* Wb = reinterpret_cast<const double*>(w + L.qr.W);
    const int64_t psw = L.qr.wcols * m, psX = (int64_t)t * L.qr.xcols;
    const SplitBuf sb2{reinterpret_cast<double*>(w + L.qr.split), L.qr.split_cap};
    const size_t vb = sizeof(double);
#define MDLS_CPY(dst, src, cnt) \
    if (cudaMemcpyAsync((dst), (src), (cnt) * vb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return MDLS_ERR_CUDA
    for (int l = 0; l < 2; ++l)
        if (cudaMemcpy2DAsync(A2 + l * ps2, m * vb, A + l * psa, lda * vb, m * vb, n,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    int rc = qr_run<2>(m, n, 0, A2, m, ps2, nullptr, 0, 0, t, w, L.qr, hdr, false, st, true);
    if (rc) return rc;
    rc = bs_invert<2>(n, A2, m, ps2, t, w, L.bs, hdr, st);
    if (rc) return rc;
    if (cudaMemsetAsync(up, 0, (size_t)P * m * vb, st) != cudaSuccess) return MDLS_ERR_CUDA;
    auto vec = [&](int op, int64_t cnt, const double* a, int64_t pa, const double* bb, int64_t pb, double* cc,
                   int64_t pc) -> int {
        StageScope sc(ST_REFINE, st);
        vec_op_kernel<P><<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(op, cnt, a, pa, bb, pb, cc, pc);
        MDLS_LAUNCH_CHECK();
        return MDLS_OK;
    };
    auto vec2 = [&](int op, int64_t cnt, const double* a, int64_t pa, const double* bb, int64_t pb, double* cc,
                    int64_t pc) -> int {
        StageScope sc(ST_REFINE, st);
        vec_op_kernel<2><<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(op, cnt, a, pa, bb, pb, cc, pc);
        MDLS_LAUNCH_CHECK();
        return MDLS_OK;
    };
    // x0 = R^{-1} (Q^T b)[0:n] in dd
    for (int l = 0; l < 2; ++l) { MDLS_CPY(c + l * m, b + l * psb, m); }
    if ((rc = apply_qt<2>(m, n, t, A2, ps2, Wb, psw, c, m, X, psX, sb2, ST_REFINE, st))) return rc;
    if ((rc = bs_solve<2>(n, A2, m, ps2, c, m, dx, n, t, w, L.bs, st))) return rc;
    for (int l = 0; l < P; ++l) {
        if (l < 2) { MDLS_CPY(x + l * psx, dx + l * n, n); }
        else if (cudaMemsetAsync(x + l * psx, 0, n * vb, st) != cudaSuccess) return MDLS_ERR_CUDA;
    }
    // A and A^T as digit slices, once: the residual products below run on the
    // tensor cores (exact digit products, as in the split mode)
    const TcOperand tA{reinterpret_cast<__nv_bfloat16*>(w + L.dA), reinterpret_cast<int*>(w + L.eA), m, n,
                       round16(n)};
    const TcOperand tAT{reinterpret_cast<__nv_bfloat16*>(w + L.dAT), reinterpret_cast<int*>(w + L.eAT), n, m,
                        round16(m)};
    __nv_bfloat16* dv = reinterpret_cast<__nv_bfloat16*>(w + L.dv);
    int* ev = reinterpret_cast<int*>(w + L.ev);
    if ((rc = split_convert<P>(ST_REFINE, st, tA, ViewDense{A, lda, psa}))) return rc;
    if ((rc = split_convert<P>(ST_REFINE, st, tAT, ViewDenseT{A, lda, psa}))) return rc;
    // r0 = b - A x0 in P limbs
    for (int l = 0; l < P; ++l) { MDLS_CPY(res + l * m, b + l * psb, m); }
    if ((rc = split_gemm_pre<P>(ST_REFINE, st, tA, dv, ev, 1, ViewDense{x, n, psx}, Dense{res, m, m}, true, true)))
        return rc;
    for (int it = 0; it < iters; ++it) {
        // f = b - r - A x,  g = -A^T r  (P limbs)
        if ((rc = vec(MDLS_OP_SUB, m, b, psb, res, m, f, m))) return rc;
        if ((rc = split_gemm_pre<P>(ST_REFINE, st, tA, dv, ev, 1, ViewDense{x, n, psx}, Dense{f, m, m}, true,
                                    true)))
            return rc;
        if ((rc = split_gemm_pre<P>(ST_REFINE, st, tAT, dv, ev, 1, ViewDense{res, m, m}, Dense{g, n, n}, true,
                                    false)))
            return rc;
        // [f1; f2] = Q^T f (dd)
        for (int l = 0; l < 2; ++l) { MDLS_CPY(c + l * m, f + l * m, m); }
        if ((rc = apply_qt<2>(m, n, t, A2, ps2, Wb, psw, c, m, X, psX, sb2, ST_REFINE, st))) return rc;
        // h = R^{-T} g (dd); dx = R^{-1} (f1 - h)
        if ((rc = fs_solve<2>(n, A2, m, ps2, g, n, hv, n, t, w, L.bs, ST_REFINE, st))) return rc;
        if ((rc = vec2(MDLS_OP_SUB, n, c, m, hv, n, dx, n))) return rc;   // dx <- f1 - h (temporarily)
        // dr = Q [h; f2]: reuse c with its first n entries replaced by h
        for (int l = 0; l < 2; ++l) { MDLS_CPY(c + l * m, hv + l * n, n); }
        if ((rc = apply_q<2>(m, n, t, A2, ps2, Wb, psw, c, m, X, psX, sb2, ST_REFINE, st))) return rc;
        for (int l = 0; l < 2; ++l) { MDLS_CPY(up + l * m, c + l * m, m); }
        if ((rc = vec(MDLS_OP_ADD, m, res, m, up, m, res, m))) return rc;          // r += dr
        if ((rc = bs_solve<2>(n, A2, m, ps2, dx, n, hv, n, t, w, L.bs, st))) return rc;  // hv <- R^{-1}(f1 - h)
        for (int l = 0; l < 2; ++l) { MDLS_CPY(up + l * m, hv + l * n, n); }
        if ((rc = vec(MDLS_OP_ADD, n, x, psx, up, m, x, psx))) return rc;         // x += dx
        // keep dx for the convergence check
        for (int l = 0; l < 2; ++l) { MDLS_CPY(dx + l * n, hv + l * n, n); }
    }
#undef MDLS_CPY
    {
        StageScope sc(ST_REFINE, st);
        refine_check_kernel<<<1, 256, 0, st>>>(dx, n, x, n, 53 - 53 * P, hdr);
        MDLS_LAUNCH_CHECK();
    }
    return MDLS_OK;
}

}  // namespace mdls

#define MDLS_INSTANTIATE(P)                                                                       \
    namespace mdls {                                                                              \
    int qr_entry_p##P(int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q,       \
                      int64_t ldq, int64_t psq, int t, int mode, void* ws, cudaStream_t st) {     \
        return qr_entry<P>(m, n, A, lda, psa, Q, ldq, psq, t, mode, ws, st);                     \
    }                                                                                             \
    int bs_entry_p##P(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y,      \
                      int64_t psy, double* x, int64_t psx, int t, void* ws, cudaStream_t st) {     \
        return bs_entry<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, st);                           \
    }                                                                                             \
    int ls_entry_p##P(int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa,            \
                      const double* b, int64_t psb, double* x, int64_t psx, int t, int mode,      \
                      void* ws, cudaStream_t st, bool single_block) {                             \
        return ls_entry<P>(m, n, A, lda, psa, b, psb, x, psx, t, mode, ws, st, single_block);    \
    }                                                                                             \
    int ls_refine_entry_p##P(int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa,     \
                             const double* b, int64_t psb, double* x, int64_t psx, int t,         \
                             int iters, void* ws, cudaStream_t st) {                              \
        return ls_refine_entry<P>(m, n, A, lda, psa, b, psb, x, psx, t, iters, ws, st);          \
    }                                                                                             \
    int toe_entry_p##P(int64_t m, int64_t n, int64_t d, const double* J, int64_t ldj, int64_t psj, \
                       int64_t bsj, const double* b, int64_t psb, int64_t bsb, double* x, int64_t psx,   \
                       int64_t bsx, int t, void* ws, cudaStream_t st) {                                 \
        return toe_entry<P>(m, n, d, J, ldj, psj, bsj, b, psb, bsb, x, psx, bsx, t, ws, st);           \
    }                                                                                             \
    int vec_entry_p##P(int op, int64_t count, const double* a, int64_t psa, const double* b,      \
                       int64_t psb, double* c, int64_t psc, cudaStream_t st) {                    \
        return vec_entry<P>(op, count, a, psa, b, psb, c, psc, st);                              \
    }                                                                                             \
    }
