// Split-product md GEMM on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators, operands staged by the bulk-copy engine).
//
// Same arithmetic as split.cuh: the rows of A and the columns of B are
// scaled by powers of two and written as S balanced base-256 digits (exact
// small integers in bf16), D_q = sum_{s+t=q} A_s B_t for q < S, and
//   (A B)_ij = 2^(e_i + f_j) sum_q D_q(i,j) 256^-(q+2)
// (Ozaki, Ogita, Oishi and Rump's error-free splitting).  What changes is how
// the digit products are laid on the hardware.
//
// Diagonals as columns.  For a 128 x NT output tile, TMEM holds one fp32
// accumulator column per (diagonal q, output column j), at column q NT + j.
// Slice s of A (128 rows x 16 k, one k16 block) multiplies a run of the
// stack [B_0; B_1; ...] of B's slices (row t NT + j of the stack is
// B_t(:, j), whose product with A_s belongs to diagonal s + t) into the TMEM
// columns of the diagonals it reaches.  Each k16 block runs two passes: the
// low pass gives slice s < Q the diagonals s .. Q-1, the high pass gives
// every slice the diagonals max(s, Q) .. S-1, one MMA per slice and pass, so
// the pairs (s, t) with s + t < S are each formed once: S(S+1)/2 slice
// products per k, as many as the pairwise form.  The low diagonals are then
// complete before the high pass starts: their drain runs beside it, and the
// high diagonals drain beside the next block's low pass.  For octo double
// NT = 8; an odd run is padded to a multiple of 16 columns downward with a
// zero slice kept in front of the stack (exact zeros added) or upward into
// column group S, which is never read.
//
// Exactness.  |d_a d_b| <= 2^14 and a column of diagonal q gains (q + 1) 16
// products per k16 block, so after DK = floor(1024 / (16 S)) blocks every
// accumulator is an integer of magnitude <= 2^24: exact in fp32, whatever
// the order in which the tensor core adds.  The accumulators are then read
// (tcgen05.ld), converted to integers and added into int64 words (four
// diagonals per word, 2^8 apart), and the next k16 block overwrites them.
//
// Roles (576 threads, one block per SM): warp 16 lane 0 streams operands with
// cp.async.bulk into a ring of stages of SB A slice tiles (4 KB each; the low
// pass's stages stay in until the high pass has read them again) and a ring
// of B stacks, completing on mbarriers; warp 17 lane 0 issues tcgen05.mma and
// tcgen05.commit; warps 0-15 read TMEM (warp w reads lanes 32 (w mod 4) ...,
// quarter w / 4 of the NT columns), keep the exact words, and write the result
// (to C, or as one md partial product when K is split over blocks).  Every
// mbarrier wait is bounded by the workspace header's limit; a block that
// gives up records MDLS_ERR_TIMEOUT, lets its copies and MMAs in flight
// finish (again bounded) and frees its TMEM before it returns.
//
// Operand layout (split_rows_tc_kernel): the tensor core's K-major form with
// the 32-byte swizzle, stored [row tile][k16 block][slice][row][32 bytes]
// (the two 16-byte halves of a row exchanged in rows 4-7 of every 8), so
// that the A slice tiles of a k16 block (128 x 16 each, taken SB at a time)
// and one B stack (SP slices x NT x 16) are each one contiguous bulk copy.
// tcgen05.mma's own rate on this part (probe: M = 128, operands in shared
// memory, back to back) is 4092 multiply-adds per clock per SM from N = 128
// on, with a floor of about 46 cycles per instruction below it; the issuing
// thread therefore waits on one barrier and commits once per SB slices.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "fx.cuh"
#include "split.cuh"

namespace mdls {

template <int P>
struct TcCfg {
    static constexpr int S = SplitCfg<P>::S;           // 15, 28, 55 digit slices
    static constexpr int NT = P == 8 ? 8 : 16;         // output columns per tile
    static constexpr int SP = P == 8 ? S + 1 : S;      // B slices per stack (od: one zero slice)
    static constexpr int DK = 1024 / (16 * S);         // k16 blocks per drain: 4, 2, 1
    static constexpr int G = (S + 3) / 4;              // int64 words per output
    static constexpr int CPT = NT / 4;                 // columns per drain thread (4 warps per TMEM lane quarter)
    static constexpr int TCOLS = SP * NT;              // TMEM columns used: 240, 448, 448
    static constexpr int TALLOC = TCOLS <= 256 ? 256 : 512;
    static constexpr int SB = 8;                       // A slices per stage (one bulk copy)
    static constexpr int NBAT = (S + SB - 1) / SB;     // stages per k16 block
    static constexpr int Q = P == 8 ? 32 : (P == 4 ? 16 : 8);  // low diagonals: q < Q
    static constexpr int QS = Q / SB;                  // stages of the low pass
    static constexpr int NA = 6;                       // A stages in flight
    static constexpr int NB = 2;                       // B stacks in flight
    static constexpr int ZP = NT == 8 ? 1 : 0;         // zero slices in front of a B stack
    static constexpr int ABYTES = 128 * 16 * 2;        // one A slice tile
    static constexpr int ASTAGE = SB * ABYTES;
    static constexpr int BCOPY = SP * NT * 16 * 2;     // one B stack as copied
    static constexpr int BBYTES = (ZP + SP) * NT * 16 * 2;
    static constexpr int NBARS = 2 * NA + 2 * NB + 5;  // full/empty rings, tmem full/empty x 2, final
    static_assert(Q % SB == 0 && Q < S && QS < NA, "the low pass's stages stay resident beside one more");
    static_assert(Q * NT <= 256 && (S - Q + 1) * NT <= 256, "one MMA per slice and pass");
    static_assert(DK >= 1 && TCOLS <= 512, "digit diagonals must fit TMEM");
    static_assert((size_t)CPT * G * 512 * 8 <= (size_t)NA * SB * 128 * 16 * 2, "the epilogue's words fit the A ring");
};

constexpr int kTcRows = 128;     // MMA M: one TMEM lane per output row
constexpr int kTcDrainWarps = 16;                    // 4 per TMEM lane quarter
constexpr int kTcThreads = 32 * (kTcDrainWarps + 2);  // the drain warps, a copy warp, an MMA warp

template <int P>
constexpr size_t split_tc_smem() {
    using C = TcCfg<P>;
    return (size_t)C::NA * C::ASTAGE + (size_t)C::NB * C::BBYTES + (size_t)C::NBARS * 8 + 16;
}

// ---------------------------------------------------------------------------
// PTX wrappers (shared-memory addresses are 32-bit shared-window addresses)
// ---------------------------------------------------------------------------
DEV_INLINE uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

DEV_INLINE void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
DEV_INLINE void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
DEV_INLINE void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
DEV_INLINE bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits until the phase of `bar` with the given parity has completed.  False
// when the limit ran out (the block's abort flag is then raised) or another
// role of the block has already given up.
DEV_INLINE bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long lim, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > lim) {
            *abort_flag = 1;
            return false;
        }
    }
}

DEV_INLINE void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

DEV_INLINE void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
DEV_INLINE void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
DEV_INLINE void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
DEV_INLINE void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
DEV_INLINE void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A B, A from shared memory (128 x 16, K-major), B from shared
// memory (N x 16, K-major), bf16 inputs, fp32 accumulators.
DEV_INLINE void tc_mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The mbarrier receives one arrival once every tcgen05 operation this thread
// issued before has completed.
DEV_INLINE void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
DEV_INLINE void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int X>
DEV_INLINE void tc_ld(uint32_t taddr, float (&v)[X]);
template <>
DEV_INLINE void tc_ld<2>(uint32_t taddr, float (&v)[2]) {
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr) : "memory");
    v[0] = __uint_as_float(r[0]);
    v[1] = __uint_as_float(r[1]);
}
template <>
DEV_INLINE void tc_ld<4>(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __uint_as_float(r[k]);
}
template <>
DEV_INLINE void tc_ld<8>(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// Shared-memory matrix descriptor: K-major with the 32-byte swizzle (mode 6
// in bits 61-63): rows of 32 bytes (one k16 block), 8-row groups 256 bytes
// apart (stride byte offset), leading byte offset unused (16); bits 46-48
// hold the fixed value 0b001.  Every tile starts on a 256-byte boundary.
DEV_INLINE uint64_t tc_smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}
// Instruction descriptor of kind::f16: fp32 D (bits 4-5 = 1), bf16 A and B
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Digit slices in the tiled layout
// ---------------------------------------------------------------------------
// One warp per row i < R of the operand view: the row's power-of-two scale
// e_i (its largest leading-limb exponent + 3, so every scaled entry lies
// below 1/4 in magnitude).
template <class AV>
__global__ void split_scale_kernel(int64_t R, int64_t K, AV A, int* scale) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= R) return;
    int emax = -100000;
    for (int64_t k = lane; k < K; k += 32) {
        const double x0 = A.get(i, k, 0);
        if (x0 != 0.0) emax = max(emax, exponent_of(x0));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    if (lane == 0) scale[i] = (emax == -100000) ? 0 : emax + 3;
}

constexpr int kTcConvK = 128;  // k values per warp of the digit conversion

// One warp per (row i < Rp, k chunk blockIdx.y of kTcConvK values): the S
// digits of every entry (rows R .. Rp-1 and k >= K are zero), written to
// [i / RT][k / 16][s][i mod RT][32 bytes] with the 32-byte swizzle (the two
// 16-byte halves of a row exchanged in rows 4-7 of every 8); slices S .. SP-1
// are zero.
template <int P, int RT, int SP, class AV>
__global__ void split_rows_tc_kernel(int64_t R, int64_t Rp, int64_t K, int64_t KB16, AV A, __nv_bfloat16* out,
                                     const int* scale) {
    constexpr int S = SplitCfg<P>::S;
    constexpr int64_t kSliceStride = (int64_t)RT * 16;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= Rp) return;
    const bool live = i < R;
    const int e = live ? scale[i] : 0;
    const int64_t rt = i / RT;
    const int r = (int)(i % RT);
    const int64_t Kp = KB16 * 16;
    const int64_t kend = ((int64_t)blockIdx.y + 1) * kTcConvK < Kp ? ((int64_t)blockIdx.y + 1) * kTcConvK : Kp;
    for (int64_t k = (int64_t)blockIdx.y * kTcConvK + lane; k < kend; k += 32) {
        double x[P];
#pragma unroll
        for (int l = 0; l < P; ++l) x[l] = (live && k < K) ? A.get(i, k, l) : 0.0;
        int dig[S];
        md_to_digits<P, S>(x, e, dig);
        const int64_t kb = k >> 4;
        __nv_bfloat16* o = out + ((rt * KB16 + kb) * SP) * kSliceStride + r * 16 +
                           ((((int)(k >> 3) & 1) ^ ((r >> 2) & 1)) * 8) + (k & 7);
#pragma unroll
        for (int s = 0; s < S; ++s) o[s * kSliceStride] = __int2bfloat16_rn(dig[s]);
#pragma unroll
        for (int s = S; s < SP; ++s) o[s * kSliceStride] = __int2bfloat16_rn(0);
    }
}

// ---------------------------------------------------------------------------
// The MMAs of one k16 block, unrolled at compile time, in two passes
// ---------------------------------------------------------------------------
// Every offset and instruction descriptor is a constant, so the one issuing
// thread spends a few instructions per MMA (the tensor core's own pace is
// 61-128 cycles per MMA here; a loop computing them took about 200).
//
// Low pass: slice s < Q against the stack slices 0 .. Q-1-s, into the low
// diagonals s .. Q-1 (octo double pads an odd count downward with the zero
// slice in front of the stack: diagonal s-1 gains exact zeros).  High pass:
// every slice s against the stack slices from max(s, Q) - s on, into the
// high diagonals max(s, Q) .. S-1 (an odd count padded upward into the
// unread column group S).  Each pass is one MMA per slice.  The low
// diagonals are complete after the low pass, so their drain runs beside the
// high pass, and the high diagonals drain beside the next block's low pass.
template <int P, int S0>
DEV_INLINE void tc_issue_low_slice(uint32_t tbase, uint64_t ad, uint64_t bd0, uint32_t acc_s0) {
    using Cfg = TcCfg<P>;
    constexpr int NT = Cfg::NT;
    constexpr int ns0 = Cfg::Q - S0;
    constexpr int pad = (NT == 8 && (ns0 & 1)) ? 1 : 0;  // S0 odd, so S0 - 1 >= 0
    constexpr int t0 = -pad, ns = ns0 + pad;
    tc_mma_bf16(tbase + (uint32_t)((S0 + t0) * NT), ad, bd0 + (uint64_t)((Cfg::ZP + t0) * (NT * 32 >> 4)),
                tc_idesc_bf16(kTcRows, ns * NT), S0 == 0 ? acc_s0 : 1u);
}

template <int P, int S0>
DEV_INLINE void tc_issue_high_slice(uint32_t tbase, uint64_t ad, uint64_t bd0, uint32_t acc_s0) {
    using Cfg = TcCfg<P>;
    constexpr int NT = Cfg::NT, S = Cfg::S;
    constexpr int q0 = S0 > Cfg::Q ? S0 : Cfg::Q;
    constexpr int t0 = q0 - S0, ns0 = S - q0;
    constexpr int ns = (NT == 8 && (ns0 & 1)) ? ns0 + 1 : ns0;
    tc_mma_bf16(tbase + (uint32_t)(q0 * NT), ad, bd0 + (uint64_t)((Cfg::ZP + t0) * (NT * 32 >> 4)),
                tc_idesc_bf16(kTcRows, ns * NT), S0 == 0 ? acc_s0 : 1u);
}

template <int P, bool HIGH, int B, int J>
DEV_INLINE void tc_issue_stage(uint32_t tbase, uint64_t ad0, uint64_t bd0, uint32_t acc_s0) {
    using Cfg = TcCfg<P>;
    constexpr int S0 = B * Cfg::SB + J;
    if constexpr (J < Cfg::SB && S0 < (HIGH ? Cfg::S : Cfg::Q)) {
        const uint64_t ad = ad0 + (uint64_t)(J * (Cfg::ABYTES >> 4));
        if constexpr (HIGH)
            tc_issue_high_slice<P, S0>(tbase, ad, bd0, acc_s0);
        else
            tc_issue_low_slice<P, S0>(tbase, ad, bd0, acc_s0);
        tc_issue_stage<P, HIGH, B, J + 1>(tbase, ad0, bd0, acc_s0);
    }
}

// The low pass over stages B .. QS-1 of the block whose first stage is ia:
// wait for each (first use), issue, keep it (the high pass reads it again).
template <int P, int B>
DEV_INLINE bool tc_issue_low(uint32_t tbase, uint32_t sA0, uint64_t bd0, uint32_t acc_s0, uint32_t ia,
                             uint32_t bar0, unsigned long long lim, volatile int* abort_flag) {
    using Cfg = TcCfg<P>;
    if constexpr (B < Cfg::QS) {
        const uint32_t st = ia + B, sa = st % Cfg::NA;
        if (!mbar_wait(bar0 + 8u * sa, (st / Cfg::NA) & 1, lim, abort_flag)) return false;
        tc_issue_stage<P, false, B, 0>(tbase, tc_smem_desc(sA0 + sa * Cfg::ASTAGE), bd0, acc_s0);
        return tc_issue_low<P, B + 1>(tbase, sA0, bd0, acc_s0, ia, bar0, lim, abort_flag);
    }
    return true;
}

// The high pass over stages B .. NBAT-1: the low pass's stages are already
// in, the others are waited for; every stage goes back to the copy warp
// after its high MMAs.
template <int P, int B>
DEV_INLINE bool tc_issue_high(uint32_t tbase, uint32_t sA0, uint64_t bd0, uint32_t acc_s0, uint32_t ia,
                              uint32_t bar0, unsigned long long lim, volatile int* abort_flag) {
    using Cfg = TcCfg<P>;
    if constexpr (B < Cfg::NBAT) {
        const uint32_t st = ia + B, sa = st % Cfg::NA;
        if (B >= Cfg::QS && !mbar_wait(bar0 + 8u * sa, (st / Cfg::NA) & 1, lim, abort_flag)) return false;
        tc_issue_stage<P, true, B, 0>(tbase, tc_smem_desc(sA0 + sa * Cfg::ASTAGE), bd0, acc_s0);
        tc_commit(bar0 + 8u * (Cfg::NA + sa));
        return tc_issue_high<P, B + 1>(tbase, sA0, bd0, acc_s0, ia, bar0, lim, abort_flag);
    }
    return true;
}

// Drain of the diagonals Q0 .. Q1-1 of this thread's TMEM row: four
// tcgen05.ld per wait, each value (an integer below 2^24 in magnitude, exact
// in fp32) added into its int64 word (D_q at bit 8 (S-1-q)).
template <int P, int Q0, int Q1>
DEV_INLINE void tc_drain_range(uint32_t trow, int64_t (&W)[TcCfg<P>::G][TcCfg<P>::CPT]) {
    using Cfg = TcCfg<P>;
    constexpr int S = Cfg::S, NT = Cfg::NT, CPT = Cfg::CPT;
    if constexpr (Q0 < Q1) {
        constexpr int Q2 = (Q0 + 4 < Q1) ? Q0 + 4 : Q1;
        float v[4][CPT];
#pragma unroll
        for (int r = 0; r < Q2 - Q0; ++r) tc_ld<CPT>(trow + (uint32_t)((Q0 + r) * NT), v[r]);
        tc_wait_ld();
#pragma unroll
        for (int r = 0; r < Q2 - Q0; ++r) {
            const int d = S - 1 - (Q0 + r);
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                W[d >> 2][j] += (int64_t)__float2int_rz(v[r][j]) * ((int64_t)1 << (8 * (d & 3)));
        }
        tc_drain_range<P, Q2, Q1>(trow, W);
    }
}

// ---------------------------------------------------------------------------
// The product
// ---------------------------------------------------------------------------
// Block (tile, z): output rows 128 mt .. 128 mt + 127 and columns NT nt ..,
// k16 blocks [z kb_per, min(KB16, (z+1) kb_per)), kb_per a multiple of DK.
// Result: C = [C] +/- (A B) for this block's K range (negate/accumulate), or
// with part_stride > 0 the block's partial product stored at
// C.ptr + z part_stride (negate = accumulate = 0).
template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    split_gemm_tc_kernel(int64_t M, int64_t N, int64_t KB16, int64_t kb_per, const __nv_bfloat16* __restrict__ As,
                         const __nv_bfloat16* __restrict__ Bs, const int* __restrict__ ea,
                         const int* __restrict__ fb, Dense C, int negate, int accumulate, int64_t part_stride,
                         WsHeader* hdr) {
    using Cfg = TcCfg<P>;
    constexpr int S = Cfg::S, NT = Cfg::NT, SP = Cfg::SP, DK = Cfg::DK, G = Cfg::G, CPT = Cfg::CPT;
    constexpr int NA = Cfg::NA, NB = Cfg::NB;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;
    unsigned char* sB = sA + NA * Cfg::ASTAGE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + NB * Cfg::BBYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + Cfg::NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const uint32_t sA0 = smem_addr(sA), sB0 = smem_addr(sB), bar0 = smem_addr(bars);
    auto fullA = [&](uint32_t s) { return bar0 + 8u * s; };
    auto emptyA = [&](uint32_t s) { return bar0 + 8u * (NA + s); };
    auto fullB = [&](uint32_t s) { return bar0 + 8u * (2 * NA + s); };
    auto emptyB = [&](uint32_t s) { return bar0 + 8u * (2 * NA + NB + s); };
    // TMEM hand-over per region (low diagonals q < Q, high q >= Q): full =
    // the MMAs of a drain group are done, empty = the drain warps have read it
    const uint32_t tfull_lo = bar0 + 8u * (2 * NA + 2 * NB), tfull_hi = tfull_lo + 8u, tempty_lo = tfull_lo + 16u,
                   tempty_hi = tfull_lo + 24u, tfinal = tfull_lo + 32u;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t mtiles = (M + kTcRows - 1) / kTcRows;
    const int64_t mt = (int64_t)blockIdx.x % mtiles, nt = (int64_t)blockIdx.x / mtiles;
    const int64_t kb0 = (int64_t)blockIdx.y * kb_per;
    const int64_t kb1 = (kb0 + kb_per < KB16) ? kb0 + kb_per : KB16;
    const int64_t ngroups = (kb1 - kb0 + DK - 1) / DK;
    const unsigned long long lim0 = *reinterpret_cast<const volatile unsigned long long*>(&hdr->wait_ns);
    const unsigned long long lim = lim0 ? lim0 : kWaitDefaultNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(fullA(s), 1);
            mbar_init(emptyA(s), 1);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(fullB(s), 1);
            mbar_init(emptyB(s), 1);
        }
        mbar_init(tfull_lo, 1);
        mbar_init(tfull_hi, 1);
        mbar_init(tempty_lo, kTcDrainWarps);
        mbar_init(tempty_hi, kTcDrainWarps);
        mbar_init(tfinal, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (Cfg::ZP > 0) {  // the zero slices in front of every B stack (never overwritten)
        for (int st = 0; st < NB; ++st)
            for (int o = threadIdx.x; o < Cfg::ZP * NT * 8; o += blockDim.x)
                reinterpret_cast<uint32_t*>(sB + st * Cfg::BBYTES)[o] = 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(tslot), Cfg::TALLOC);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(tslot);

    if (warp == kTcDrainWarps) {
        // ---- copies: per k16 block the B stack, then the A slice tiles in
        //      stages of SB (contiguous in the tiled layout: one copy each)
        if (lane == 0 && kb1 > kb0) {
            uint32_t ia = 0, ib = 0;
            bool ok = true;
            for (int64_t kb = kb0; kb < kb1 && ok; ++kb) {
                const uint32_t sb = ib % NB;
                if (!(ok = mbar_wait(emptyB(sb), ((ib / NB) & 1) ^ 1, lim, abort_flag))) break;
                mbar_expect_tx(fullB(sb), Cfg::BCOPY);
                bulk_copy_g2s(sB0 + sb * Cfg::BBYTES + Cfg::ZP * NT * 32, Bs + ((nt * KB16 + kb) * SP) * (NT * 16),
                              Cfg::BCOPY, fullB(sb));
                ++ib;
                for (int s0 = 0; s0 < S; s0 += Cfg::SB) {
                    const int ns = (S - s0 < Cfg::SB) ? S - s0 : Cfg::SB;
                    const uint32_t sa = ia % NA;
                    if (!(ok = mbar_wait(emptyA(sa), ((ia / NA) & 1) ^ 1, lim, abort_flag))) break;
                    mbar_expect_tx(fullA(sa), (uint32_t)ns * Cfg::ABYTES);
                    bulk_copy_g2s(sA0 + sa * Cfg::ASTAGE, As + (((mt * KB16 + kb) * S) + s0) * (kTcRows * 16),
                                  (uint32_t)ns * Cfg::ABYTES, fullA(sa));
                    ++ia;
                }
            }
            // every copy issued has landed before the block can leave
            for (uint32_t s = 0; s < NA && s < ia; ++s) {
                const uint32_t last = ia - 1 - ((ia - 1 - s) % NA);
                mbar_wait(fullA(s), (last / NA) & 1, lim, abort_flag);
            }
            for (uint32_t s = 0; s < NB && s < ib; ++s) {
                const uint32_t last = ib - 1 - ((ib - 1 - s) % NB);
                mbar_wait(fullB(s), (last / NB) & 1, lim, abort_flag);
            }
        }
    } else if (warp == kTcDrainWarps + 1) {
        // ---- MMAs: per k16 block a low pass and a high pass, one MMA per
        //      slice and pass; one wait per stage, one commit per stage
        if (lane == 0) {
            uint32_t ia = 0, ib = 0, grp = 0;
            bool ok = kb1 > kb0;
            for (int64_t kb = kb0; kb < kb1 && ok; ++kb) {
                const int64_t rel = kb - kb0;
                const bool gfirst = (rel % DK) == 0;
                const bool glast = (rel % DK) == DK - 1 || kb == kb1 - 1;
                const uint32_t acc0 = gfirst ? 0u : 1u;
                if (gfirst && grp > 0) {
                    if (!(ok = mbar_wait(tempty_lo, (grp - 1) & 1, lim, abort_flag))) break;
                }
                const uint32_t sb = ib % NB;
                if (!(ok = mbar_wait(fullB(sb), (ib / NB) & 1, lim, abort_flag))) break;
                tc_fence_after();
                // the start-address field is the descriptor's low bits: a
                // byte offset o moves it by o >> 4
                const uint64_t bd0 = tc_smem_desc(sB0 + sb * Cfg::BBYTES);
                if (!(ok = tc_issue_low<P, 0>(tbase, sA0, bd0, acc0, ia, bar0, lim, abort_flag))) break;
                if (glast) tc_commit(tfull_lo);
                if (gfirst && grp > 0) {
                    if (!(ok = mbar_wait(tempty_hi, (grp - 1) & 1, lim, abort_flag))) break;
                    tc_fence_after();
                }
                if (!(ok = tc_issue_high<P, 0>(tbase, sA0, bd0, acc0, ia, bar0, lim, abort_flag))) break;
                ia += Cfg::NBAT;
                tc_commit(emptyB(sb));
                ++ib;
                if (glast) {
                    tc_commit(tfull_hi);
                    ++grp;
                }
            }
            // every MMA issued has completed before the block can leave
            tc_commit(tfinal);
            mbar_wait(tfinal, 0, lim, abort_flag);
        }
    } else {
        // ---- drain: exact words of this thread's row and columns
        const int quarter = warp & 3, part = warp >> 2;
        const uint32_t trow = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(part * CPT);
        int64_t W[G][CPT];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int j = 0; j < CPT; ++j) W[g][j] = 0;
        bool ok = true;
        for (int64_t gi = 0; gi < ngroups; ++gi) {
            ok = mbar_wait(tfull_lo, (uint32_t)(gi & 1), lim, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            tc_drain_range<P, 0, Cfg::Q>(trow, W);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_lo);
            ok = mbar_wait(tfull_hi, (uint32_t)(gi & 1), lim, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            tc_drain_range<P, Cfg::Q, S>(trow, W);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_hi);
        }
        if (ok) {
            // every MMA has completed and every copy has landed, so the A
            // ring is free: the words go there (thread-private slots), and
            // one rolled copy of the conversion serves the thread's columns
            // (unrolled per column, the conversion code outgrew the
            // instruction cache)
            int64_t* sW = reinterpret_cast<int64_t*>(sA) + threadIdx.x;
#pragma unroll
            for (int j = 0; j < CPT; ++j)
#pragma unroll
                for (int g = 0; g < G; ++g) sW[(j * G + g) * 512] = negate ? -W[g][j] : W[g][j];
            const int64_t i = mt * kTcRows + 32 * quarter + lane;
            if (i < M) {
                const int sci = ea[i];
                double* base = C.ptr + (int64_t)blockIdx.y * part_stride;
#pragma unroll 1
                for (int j = 0; j < CPT; ++j) {
                    const int64_t jc = nt * NT + part * CPT + j;
                    if (jc >= N) break;
                    // value = 2^e0 sum_g W_g 2^(32 g) exactly (D_q at bit
                    // 8 (S-1-q)); C's old value joins it on the integer pipe
                    const int e0 = sci + fb[jc] - 8 * (S + 1);
                    int64_t w[G + 3];
#pragma unroll
                    for (int g = 0; g < G; ++g) w[g] = sW[(j * G + g) * 512];
#pragma unroll
                    for (int g = G; g < G + 3; ++g) w[g] = 0;
                    st_md<P>(base, C.ps, jc * C.ld + i,
                             split_epilogue<P, G + 3>(w, e0, accumulate, base, C.ps, jc * C.ld + i));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        atomicExch(&hdr->bar_error, 1);
        set_status(&hdr->status, MDLS_ERR_TIMEOUT);
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, Cfg::TALLOC);
    }
}

}  // namespace mdls
