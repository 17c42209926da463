// Split-product md GEMM on the tensor cores (precision mode "split").
//
// C = [C] +/- A B for md matrices A (M x K) and B (K x N) with P limbs.  Each
// row i of A is scaled by a power of two 2^-e_i and each column j of B by
// 2^-f_j so that every entry lies below 1/4 in magnitude; each scaled entry
// is then written exactly (up to its last digit) as S balanced base-256
// digits, y = sum_s d_s 256^-(s+1), d_s in [-128, 127].  The digits are exact
// small integers in bf16, so every digit product is exact in fp32, and a sum
// of at most 2^10 such products (|d_a d_b| <= 2^14) stays below 2^24 and is
// exact too.  With D_q = sum_{s+t=q} A_s B_t (exact integers, q < S),
//   (A B)_ij = 2^(e_i + f_j) sum_q D_q(i,j) 256^-(q+2)
// up to the dropped digit pairs s + t >= S, which lie below 2^(-8S) of the
// row-times-column scale.  S = ceil((53P + 12) / 8) keeps that under the md
// unit roundoff.  This is the error-free matrix-product splitting of Ozaki,
// Ogita, Oishi and Rump (2012), with integer slices of a fixed-point form.
//
// Kernels: split_rows_kernel writes the digits of A (and, through a
// transposing view, of B) as bf16 slices [S][rows][Kp], k contiguous;
// split_gemm_kernel computes one 16 x 8 output tile per block with
// mma.sync m16n8k16 (bf16 in, fp32 accumulate), the 8 warps sharing the
// diagonals q round-robin; each warp moves its fp32 sums into int64 after
// every k16 step (at most 16 S products, exact), and the epilogue places the
// S exact diagonal sums into 24-bit digits on the integer pipe and truncates
// the exact total to P limbs.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "fx.cuh"
#include "words.cuh"

namespace mdls {

template <int P>
struct SplitCfg {
    static constexpr int S = (53 * P + 12 + 7) / 8;  // 15 (dd), 28 (qd), 55 (od)
};

constexpr int kSplitTm = 16, kSplitTn = 8, kSplitTk = 16, kSplitPad = 24;

template <class BV>
struct ViewTranspose {  // B^T, so that the columns of B are split like rows
    static constexpr bool kRowContig = false;
    static constexpr bool kZeroKBelowI = BV::kZeroKAboveI, kZeroKAboveI = BV::kZeroKBelowI;
    BV b;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const { return b.get(k, i, l); }
};

DEV_INLINE int exponent_of(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

// Digits of y = x 2^-e (|y| < 1/4): dig[0] most significant, balanced.
// Each limb's 53-bit significand is added bytewise into the fixed-point
// form Y = y 256^S; bits below the last digit are dropped (toward zero).
template <int P, int S>
DEV_INLINE void md_to_digits(const double (&x)[P], int e, int (&dig)[S]) {
    int acc[S];
#pragma unroll
    for (int b = 0; b < S; ++b) acc[b] = 0;
#pragma unroll
    for (int l = 0; l < P; ++l) {
        const long long bits = __double_as_longlong(x[l]);
        if ((bits & 0x7fffffffffffffffLL) == 0) continue;
        const bool neg = bits < 0;
        int E = (int)((bits >> 52) & 0x7ff);
        unsigned long long m = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
        if (E == 0) E = 1;
        else m |= (1ull << 52);
        const int sh = E - 1075 - e + 8 * S;  // x_l 2^-e 256^S = m 2^sh
        if (sh <= -53) continue;
        unsigned long long v;
        int base;
        if (sh < 0) {
            v = m >> (-sh);
            base = 0;
        } else {
            v = m << (sh & 7);  // < 2^60
            base = sh >> 3;
        }
        for (int q = 0; q < 8; ++q) {
            const int b = base + q;
            if (b >= S) break;
            const int byte = (int)((v >> (8 * q)) & 0xff);
            acc[b] += neg ? -byte : byte;
        }
    }
    int carry = 0;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const int v = acc[b] + carry;
        const int d = ((v + 128) & 255) - 128;
        carry = (v - d) >> 8;
        dig[S - 1 - b] = d;
    }
}

// The output of a split product: 2^e0 sum_g w[g] 2^(32 g) (exact, the
// product already negated if asked), plus C's old value when `accumulate`,
// rounded toward zero to P limbs (words.cuh).  C's value joins the words on
// the integer pipe when its leading exponent lies inside their range, which
// it does unless C outweighs the row-times-column scale of the product by
// 2^32 or more; then the sum is one md addition.
template <int P, int GW>
DEV_INLINE md<P> split_epilogue(int64_t (&w)[GW], int e0, int accumulate, const double* base, int64_t ps,
                                int64_t off) {
    if (!accumulate) return words::to_md<P, GW>(w, e0, false);
    const md<P> old = ld_md<P>(base, ps, off);
    if (old.v[0] == 0.0 || exponent_of(old.v[0]) - e0 < 32 * (GW - 2)) {
        words::add_md<GW, P>(w, old, e0);
        return words::to_md<P, GW>(w, e0, false);
    }
    return md_add<P>(old, words::to_md<P, GW>(w, e0, false));
}

// One warp per row i of the operand view: e_i, then the S digit slices.
template <int P, class AV>
__global__ void split_rows_kernel(int64_t M, int64_t K, int64_t Kp, AV A, __nv_bfloat16* slices,
                                  int* scale) {
    constexpr int S = SplitCfg<P>::S;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;
    int emax = -100000;
    for (int64_t k = lane; k < K; k += 32) {
        const double x0 = A.get(i, k, 0);
        if (x0 != 0.0) emax = max(emax, exponent_of(x0));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    const int e = (emax == -100000) ? 0 : emax + 3;
    if (lane == 0) scale[i] = e;
    for (int64_t k = lane; k < Kp; k += 32) {
        double x[P];
#pragma unroll
        for (int l = 0; l < P; ++l) x[l] = (k < K) ? A.get(i, k, l) : 0.0;
        int dig[S];
        md_to_digits<P, S>(x, e, dig);
#pragma unroll
        for (int s = 0; s < S; ++s) slices[((int64_t)s * M + i) * Kp + k] = __int2bfloat16_rn(dig[s]);
    }
}

DEV_INLINE void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared memory: the digit slices staged per k16 step, reused after the k
// loop for the S diagonal sums of the epilogue (two blocks per SM fit).
template <int P>
constexpr size_t split_gemm_smem() {
    constexpr int S = SplitCfg<P>::S;
    constexpr size_t stage = (size_t)S * kSplitTm * kSplitPad * 2 + (size_t)S * kSplitTn * kSplitPad * 2;
    constexpr size_t diag = (size_t)S * kSplitTm * kSplitTn * 8;
    return stage > diag ? stage : diag;
}

// C(i,j) = [C] +/- 2^(ea_i + fb_j) sum_q D_q(i,j) 256^-(q+2), one 16x8 tile
// per block, 8 warps; warp w owns the diagonals q = w, w+8, w+16, ...
template <int P>
__global__ void __launch_bounds__(256)
    split_gemm_kernel(int64_t M, int64_t N, int64_t Kp, const __nv_bfloat16* As,
                      const __nv_bfloat16* Bs, const int* ea, const int* fb, Dense C, int negate,
                      int accumulate) {
    constexpr int S = SplitCfg<P>::S;
    constexpr int NJ = (S + 7) / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* Asm = reinterpret_cast<__nv_bfloat16*>(smem_raw);             // [S][16][24]
    __nv_bfloat16* Bsm = Asm + (size_t)S * kSplitTm * kSplitPad;                  // [S][8][24]
    long long* Dsm = reinterpret_cast<long long*>(smem_raw);  // [S][128], after the k loop
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.x * kSplitTm, j0 = (int64_t)blockIdx.y * kSplitTn;

    float accf[NJ][4];
    long long acci[NJ][4];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            accf[jj][q] = 0.f;
            acci[jj][q] = 0;
        }

    for (int64_t k0 = 0; k0 < Kp; k0 += kSplitTk) {
        // stage all S digit slices of the A rows (16 x 16) and B columns (8 x 16)
        for (int idx = tid; idx < S * kSplitTm * 2; idx += blockDim.x) {
            const int s = idx / (kSplitTm * 2), r = (idx >> 1) % kSplitTm, h = idx & 1;
            const int64_t row = i0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row < M) v = *reinterpret_cast<const uint4*>(As + ((int64_t)s * M + row) * Kp + k0 + h * 8);
            *reinterpret_cast<uint4*>(Asm + ((size_t)s * kSplitTm + r) * kSplitPad + h * 8) = v;
        }
        for (int idx = tid; idx < S * kSplitTn * 2; idx += blockDim.x) {
            const int s = idx / (kSplitTn * 2), r = (idx >> 1) % kSplitTn, h = idx & 1;
            const int64_t col = j0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (col < N) v = *reinterpret_cast<const uint4*>(Bs + ((int64_t)s * N + col) * Kp + k0 + h * 8);
            *reinterpret_cast<uint4*>(Bsm + ((size_t)s * kSplitTn + r) * kSplitPad + h * 8) = v;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            const int q = warp + 8 * jj;
            if (q < S) {
                for (int s = 0; s <= q; ++s) {
                    const __nv_bfloat16* a = Asm + (size_t)s * kSplitTm * kSplitPad;
                    const __nv_bfloat16* b = Bsm + (size_t)(q - s) * kSplitTn * kSplitPad;
                    uint32_t af[4], bf[2];
                    af[0] = *reinterpret_cast<const uint32_t*>(a + g * kSplitPad + t4 * 2);
                    af[1] = *reinterpret_cast<const uint32_t*>(a + (g + 8) * kSplitPad + t4 * 2);
                    af[2] = *reinterpret_cast<const uint32_t*>(a + g * kSplitPad + t4 * 2 + 8);
                    af[3] = *reinterpret_cast<const uint32_t*>(a + (g + 8) * kSplitPad + t4 * 2 + 8);
                    bf[0] = *reinterpret_cast<const uint32_t*>(b + g * kSplitPad + t4 * 2);
                    bf[1] = *reinterpret_cast<const uint32_t*>(b + g * kSplitPad + t4 * 2 + 8);
                    mma_bf16_16816(accf[jj], af, bf);
                }
                // at most 16 S <= 880 products of |.| <= 2^14 since the last move: exact
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acci[jj][c] += (long long)__float2int_rz(accf[jj][c]);  // an integer below 2^24: exact in int32
                    accf[jj][c] = 0.f;
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
        const int q = warp + 8 * jj;
        if (q < S) {
            long long* Dq = Dsm + (size_t)q * (kSplitTm * kSplitTn);
            Dq[g * kSplitTn + t4 * 2] = acci[jj][0];
            Dq[g * kSplitTn + t4 * 2 + 1] = acci[jj][1];
            Dq[(g + 8) * kSplitTn + t4 * 2] = acci[jj][2];
            Dq[(g + 8) * kSplitTn + t4 * 2 + 1] = acci[jj][3];
        }
    }
    __syncthreads();
    if (tid < kSplitTm * kSplitTn) {
        const int r = tid / kSplitTn, cc = tid % kSplitTn;
        const int64_t i = i0 + r, j = j0 + cc;
        if (i < M && j < N) {
            // the value 2^sc sum_q D_q 2^(-8(q+2)) = 2^e0 sum_q D_q 2^(8(S-1-q))
            // exactly in 32-bit-spaced int64 words (D_q is an integer below
            // 2^40 in magnitude: its low and high 32 bits go to adjacent
            // words), C's old value joined on the integer pipe (words.cuh)
            constexpr int G = (S + 3) / 4, GW = G + 3;
            const int e0 = ea[i] + fb[j] - 8 * (S + 1);
            int64_t w[GW];
#pragma unroll
            for (int k = 0; k < GW; ++k) w[k] = 0;
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const int sh = 8 * (S - 1 - q), k = sh / 32, rem = sh % 32;
                int64_t dq = Dsm[(size_t)q * (kSplitTm * kSplitTn) + tid];
                if (negate) dq = -dq;
                w[k] += (int64_t)((uint64_t)dq & 0xffffffffULL) << rem;
                w[k + 1] += (dq >> 32) * ((int64_t)1 << rem);
            }
            const int64_t off = j * C.ld + i;
            const md<P> v = split_epilogue<P, GW>(w, e0, accumulate, C.ptr, C.ps, off);
            st_md<P>(C.ptr, C.ps, off, v);
        }
    }
}

}  // namespace mdls
