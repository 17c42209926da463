// Step 2 of Algorithm 1 (Section 2) in one persistent launch: the tile loop
// i = N..1 of x_i := U_i^{-1} y_i and y_j := y_j - A_{j,i} x_i, with the
// inverted diagonal tiles U_i^{-1} already in place (step 1).
//
// The paper launches kernels per tile step.  On GB300 the FP64 pipe retires
// one warp instruction per 64 cycles per SM sub-partition, so a warp that
// updates 32 rows with a whole tile of 128 columns (128 md FMAs per lane)
// needs 167 us in quad double however the launch is arranged; a launch per
// step waits for its slowest warp, and a chain of such tasks between x_i and
// x_{i-2} would set the pace of the whole solve.  Here the steps overlap and
// every task is short:
//
//  * the rows are cut into 32-row chunks (one row per lane, coalesced reads
//    of R's columns) and every tile's columns into S slices of kBsSlice
//    columns; every (chunk c, slice s) keeps a running sum acc[c][s] of its
//    terms sum_k R(c, k) x_k over the tiles met so far;
//  * bulk tasks (c, i, s) -- chunks at least two tiles above tile i -- come
//    from one queue in order of i, then c downwards, then s: once x_i is
//    published and the tiles N..i+1 are in acc[c][s] (the turn counter of
//    (c, s)), a task continues that running sum with its kBsSlice-column
//    product, so every sum is formed in the same order in every run
//    (deterministic);
//  * the critical chain x_i -> x_{i-1} runs on a few reserved SMs (the other
//    blocks on them stay idle, so each critical warp has an FP64 pipe of its
//    own): the slices of tile i-1's rows times x_i join their running sums,
//    the chunk's S running sums are added in a binary tree whose root forms
//    y_c - sum_s acc[c][s], then x_{i-1} = U_{i-1}^{-1} y_{i-1} in slices
//    whose partial sums meet in a second tree (tree_up: a fixed order, log2 S
//    dependent additions).  Each chain is bound by the latency of one warp's
//    md operations (about three times their issue time on GB300: 8 qd md
//    FMAs take 33 us, a 16-term sequential sum 45 us); two interleaved chains
//    per warp or operands loaded ahead measured slower.
//
// Every wait is bounded (warp_wait_ge): a wait that runs out records
// MDLS_ERR_TIMEOUT and every warp leaves at its next wait or task.  Data
// written by other SMs is read with ld.global.cg (L2), never from L1.
#pragma once
#include "kernels.cuh"
#include "layout.h"

namespace mdls {

constexpr int kBsSlice = kBsSliceCols;  // columns per slice
constexpr int kBsCritSms = 16;          // SMs reserved for the critical chain
constexpr int kBsBlocksPerSm = 4;       // 128-thread blocks per SM: four warps per sub-partition
constexpr int kBsMaxSm = 1024;          // slots of the per-SM role claim

// Counters (unsigned ints, zeroed by the host before the launch).
struct BsCtr {
    int64_t bulk_head, crit_head, crit_claims, sm_role, sm_slot, turn, cu_node, xt_node, yfin, xready, total;
    __host__ __device__ static BsCtr make(int64_t nchunks, int64_t S, int64_t N) {
        BsCtr c;
        c.bulk_head = 0;
        c.crit_head = 32;   // separate 128-byte lines for the queue heads
        c.crit_claims = 64;
        c.sm_role = 96;
        c.sm_slot = c.sm_role + kBsMaxSm;
        c.turn = c.sm_slot + kBsMaxSm;   // (chunk, slice): bulk tiles added to acc
        c.cu_node = c.turn + nchunks * S;     // (chunk, tree node): children arrived, y's sum
        c.xt_node = c.cu_node + nchunks * S;  // (chunk, tree node): children arrived, x's sum
        c.yfin = c.xt_node + nchunks * S;     // tile: chunks whose y is final
        c.xready = c.yfin + N;            // tile: chunks of x published
        c.total = c.xready + N;           // == bs_ctr_ints(nchunks, S, N)
        return c;
    }
};

struct BsPersistArgs {
    const double* R;
    int64_t ldr, psr;
    const double* D;     // inverted diagonal tiles: tile i at D + i t^2, column-major, ld t
    int64_t dps;         // plane stride of D
    double* yb;          // working right-hand side, P planes of n
    double* x;
    int64_t psx;
    double* acc;         // [limb][chunk][slice][lane] running sums of the updates
    double* tree_cu;     // [limb][chunk][node][lane] tree of the sum of a chunk's running sums
    double* tree_xt;     // [limb][chunk][node][lane] tree of the slices' parts of x = U^{-1} y
    int64_t part_ps;     // plane stride of acc (the trees: twice that)
    unsigned int* ctr;
    int64_t n;
    int t, N, nchunks, S, KS, ncrit;
    WsHeader* hdr;
};

// Lane 0 waits until *c >= want (bounded); the result is broadcast to the warp.
DEV_INLINE bool warp_wait_ge(const unsigned int* c, unsigned int want, WsHeader* h) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        const volatile unsigned int* vc = c;
        const volatile int* verr = &h->bar_error;
        if (*vc < want) {
            const unsigned long long lim0 = *reinterpret_cast<const volatile unsigned long long*>(&h->wait_ns);
            const unsigned long long lim = lim0 ? lim0 : kWaitDefaultNs;
            const unsigned long long t0 = globaltimer_ns();
            while (*vc < want) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > lim) {
                    atomicExch(&h->bar_error, 1);
                    set_status(&h->status, MDLS_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

template <int P>
DEV_INLINE md<P> ld_md_cg(const double* ptr, int64_t ps, int64_t off) {
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = __ldcg(ptr + l * ps + off);
    return r;
}

// Publishes the warp's stores, then adds 1 to *c (lane 0); returns the old
// value to every lane.
DEV_INLINE unsigned int warp_publish(unsigned int* c) {
    __threadfence();
    __syncwarp();
    unsigned int old = 0;
    if ((threadIdx.x & 31) == 0) old = atomicAdd(c, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    __threadfence();
    return old;
}

DEV_INLINE int tile_width(int64_t n, int t, int64_t j) {
    const int64_t w = n - j * t;
    return (int)(w < t ? w : t);
}

// sum_{k in [k0, k1)} A(r, k) x_k with lanes on rows (A column-major, coalesced)
template <int P>
DEV_INLINE md<P> rows_times_x(const double* A, int64_t lda, int64_t psa, int64_t r, int64_t k0, int64_t k1,
                              const double* x, int64_t psx) {
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = 0.0;
    int cnt = 0;
    for (int64_t k = k0; k < k1; ++k) {
        md<P> a, xv;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            a.v[l] = A[l * psa + k * lda + r];
            xv.v[l] = __ldcg(x + l * psx + k);
        }
        md_fma_bins<P>(bins, a, xv);
        if ((++cnt & 15) == 0) md_bins_renorm<P>(bins);
    }
    return md_from_bins<P>(bins);
}

// acc[c][s] := (first ? 0 : acc[c][s]) + sum_{k in [k0, k1)} A(r, k) x_k: the
// running sum is the addend of the product's bins, so a bulk task costs one
// renormalisation and no md addition of its own.
template <int P>
DEV_INLINE void acc_rows_times_x(double* acc, int64_t ps, int64_t off, bool first, const double* A, int64_t lda,
                                 int64_t psa, int64_t r, int64_t k0, int64_t k1, const double* x, int64_t psx) {
    double bins[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bins[l] = first ? 0.0 : __ldcg(acc + l * ps + off);
    int cnt = 0;
    for (int64_t k = k0; k < k1; ++k) {
        md<P> a, xv;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            a.v[l] = A[l * psa + k * lda + r];
            xv.v[l] = __ldcg(x + l * psx + k);
        }
        md_fma_bins<P>(bins, a, xv);
        if ((++cnt & 15) == 0) md_bins_renorm<P>(bins);
    }
    st_md<P>(acc, ps, off, md_from_bins<P>(bins));
}

// Columns [k0, k1) of slice s of tile i (empty beyond a ragged last tile).
DEV_INLINE void slice_cols(int64_t n, int t, int i, int s, int64_t& k0, int64_t& k1) {
    const int64_t kend = (int64_t)i * t + tile_width(n, t, i);
    k0 = (int64_t)i * t + (int64_t)s * kBsSlice;
    k1 = k0 + kBsSlice;
    if (k1 > kend) k1 = kend;
    if (k0 > k1) k0 = k1;
}

// Slices of tile j's columns that meet rows [32 cl, 32 cl + 32) of the upper
// triangular U_j^{-1} (slices wholly left of the chunk's diagonal are zero)
// and lie inside the tile of width tt.
DEV_INLINE bool xt_slice_needed(int cl, int s, int tt) {
    return s * kBsSlice < tt && s * kBsSlice + kBsSlice - 1 >= 32 * cl;
}

// acc[c][s] := (first ? 0 : acc[c][s]) + v; returns the new value
template <int P>
DEV_INLINE md<P> acc_add(double* acc, int64_t ps, int64_t off, bool first, const md<P>& v) {
    const md<P> r = first ? v : md_add<P>(ld_md_cg<P>(acc, ps, off), v);
    st_md<P>(acc, ps, off, r);
    return r;
}

// Sum of the S slice values of one chunk as a binary tree (S a power of two;
// heap numbering, leaves S .. 2S-1, root 1): a task stores its leaf and
// climbs; at each node the first of the two children to arrive stops and
// the second adds left + right (a fixed order whatever the arrival order)
// and climbs on.  Returns true, with the total in v, to the task that
// completes the root.  log2(S) dependent additions instead of S - 1.
template <int P>
DEV_INLINE bool tree_up(double* tree, int64_t tps, unsigned int* node_cnt, int64_t c, int S, int s, md<P>& v) {
    const int lane = threadIdx.x & 31;
    int node = S + s;
    const int64_t base = c * 2 * S;
    st_md<P>(tree, tps, (base + node) * 32 + lane, v);
    while (node > 1) {
        const int parent = node >> 1;
        const unsigned old = warp_publish(node_cnt + c * S + parent);
        if (old == 0) return false;
        const md<P> other = ld_md_cg<P>(tree, tps, (base + (node ^ 1)) * 32 + lane);
        v = (node & 1) ? md_add<P>(other, v) : md_add<P>(v, other);
        node = parent;
        if (node > 1) st_md<P>(tree, tps, (base + node) * 32 + lane, v);
    }
    return true;
}

template <int P>
__global__ void __launch_bounds__(128) bs_persist_kernel(BsPersistArgs a) {
    __shared__ int role;  // 0 bulk, 1 critical, 2 idle
    const int lane = threadIdx.x & 31;
    unsigned int* ctr = a.ctr;
    const BsCtr C = BsCtr::make(a.nchunks, a.S, a.N);
    if (threadIdx.x == 0) {
        // the first block on each SM asks for a critical slot; the first
        // ncrit to ask get one, and the other blocks on their SMs stay idle
        unsigned int smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        unsigned int* sm_role = ctr + C.sm_role + (smid % kBsMaxSm);   // 0 unset, 1 bulk SM, 2 critical SM
        unsigned int* sm_slot = ctr + C.sm_slot + (smid % kBsMaxSm);
        const unsigned int slot = atomicAdd(sm_slot, 1u);
        if (slot == 0) {
            const unsigned int g = atomicAdd(ctr + C.crit_claims, 1u);
            role = g < (unsigned)a.ncrit ? 1 : 0;
            __threadfence();
            atomicExch(sm_role, role == 1 ? 2u : 1u);
        } else {
            const volatile unsigned int* vr = sm_role;
            const unsigned long long t0 = globaltimer_ns();
            int r = -1;
            while (r < 0) {
                const unsigned int v = *vr;
                if (v != 0) {
                    r = v == 2 ? 2 : 0;
                } else if (globaltimer_ns() - t0 > kWaitDefaultNs) {
                    atomicExch(&a.hdr->bar_error, 1);
                    set_status(&a.hdr->status, MDLS_ERR_TIMEOUT);
                    r = 2;
                }
            }
            role = r;
        }
    }
    __syncthreads();
    if (role == 2) return;
    const int64_t n = a.n;
    const int t = a.t, N = a.N, S = a.S, tc = t / 32;
    const int64_t pps = a.part_ps;

    if (role == 1) {
        // critical queue: phase 0 = x_{N-1}; then for i = N-1 .. 1, phase
        // 2(N-1-i)+1 = tile i-1's rows times x_i, phase 2(N-1-i)+2 = x_{i-1};
        // KS task slots per phase (unused slots are skipped)
        const int64_t total = (int64_t)(2 * N - 1) * a.KS;
        for (;;) {
            if (*reinterpret_cast<volatile int*>(&a.hdr->bar_error)) return;
            unsigned int q = 0;
            if (lane == 0) q = atomicAdd(ctr + C.crit_head, 1u);
            q = __shfl_sync(0xffffffffu, q, 0);
            if ((int64_t)q >= total) return;
            const int phase = (int)(q / a.KS), k = (int)(q % a.KS);
            if (phase % 2 == 1) {
                // slice s of tile j = i - 1's chunk cl times x_i
                const int i = N - 1 - (phase - 1) / 2, j = i - 1;
                const int cl = k / S, s = k % S;
                if (cl >= tc) continue;
                const int64_t c = (int64_t)j * tc + cl;
                const int64_t r = c * 32 + lane;
                if (!warp_wait_ge(ctr + C.xready + i, (unsigned)((tile_width(n, t, i) + 31) / 32), a.hdr)) return;
                int64_t k0, k1;
                slice_cols(n, t, i, s, k0, k1);
                const md<P> part = rows_times_x<P>(a.R, a.ldr, a.psr, r, k0, k1, a.x, a.psx);
                // after the bulk tiles N-1 .. i+1 of this slice
                const int nb = N - 1 - i;
                if (!warp_wait_ge(ctr + C.turn + c * S + s, (unsigned)nb, a.hdr)) return;
                md<P> v = acc_add<P>(a.acc, pps, (c * S + s) * 32 + lane, nb == 0, part);
                // the chunk's S running sums meet in a tree; the task that
                // completes it forms y_c - (acc[c][0] + ... + acc[c][S-1])
                if (!tree_up<P>(a.tree_cu, 2 * pps, ctr + C.cu_node, c, S, s, v)) continue;
                st_md<P>(a.yb, n, r, md_sub<P>(ld_md_cg<P>(a.yb, n, r), v));
                warp_publish(ctr + C.yfin + j);
            } else {
                // x_j = U_j^{-1} y_j: output chunk cl of tile j, slice s of its columns
                const int j = N - 1 - phase / 2;
                const int tt = tile_width(n, t, j);
                const int cl = k / S, s = k % S;
                if (cl * 32 >= tt) continue;
                // slices wholly left of the chunk's diagonal, or beyond a
                // ragged tile, contribute zero but still enter the tree
                const bool needed = xt_slice_needed(cl, s, tt);
                if (needed && j < N - 1 && !warp_wait_ge(ctr + C.yfin + j, (unsigned)tc, a.hdr)) return;
                const int rl = cl * 32 + lane;  // row within the tile
                const bool rv = rl < tt;
                const double* Dj = a.D + (int64_t)j * t * t;
                const double* yj = a.yb + (int64_t)j * t;
                double bins[P];
#pragma unroll
                for (int l = 0; l < P; ++l) bins[l] = 0.0;
                const int k0 = s * kBsSlice, k1 = needed ? ((k0 + kBsSlice) < tt ? (k0 + kBsSlice) : tt) : k0;
                for (int kk = k0; kk < k1; ++kk) {
                    md<P> dv, yv;
                    const bool in = rv && kk >= rl;  // U^{-1} is upper triangular
#pragma unroll
                    for (int l = 0; l < P; ++l) {
                        dv.v[l] = in ? Dj[l * a.dps + (int64_t)kk * t + rl] : 0.0;
                        yv.v[l] = __ldcg(yj + l * n + kk);
                    }
                    md_fma_bins<P>(bins, dv, yv);
                }
                const int64_t c = (int64_t)j * tc + cl;
                md<P> xs = md_from_bins<P>(bins);
                if (!tree_up<P>(a.tree_xt, 2 * pps, ctr + C.xt_node, c, S, s, xs)) continue;
                if (rv) st_md<P>(a.x, a.psx, (int64_t)j * t + rl, xs);
                warp_publish(ctr + C.xready + j);
            }
        }
    }

    // bulk queue: tasks (c, i, s) for i = N-1 .. 2, chunks c < (i-1) tc in
    // decreasing order, slices s; step sa = N-1-i holds (i-1) tc S tasks
    int sa = 0;
    int64_t base = 0;  // first task of step sa
    for (;;) {
        if (*reinterpret_cast<volatile int*>(&a.hdr->bar_error)) return;
        unsigned int q = 0;
        if (lane == 0) q = atomicAdd(ctr + C.bulk_head, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        while (sa < N - 2 && (int64_t)q >= base + (int64_t)(N - 2 - sa) * tc * S) {
            base += (int64_t)(N - 2 - sa) * tc * S;
            ++sa;
        }
        if (sa >= N - 2) return;
        const int i = N - 1 - sa;
        const int64_t idx = (int64_t)q - base;
        const int64_t c = (int64_t)(i - 1) * tc - 1 - idx / S;
        const int s = (int)(idx % S);
        if (!warp_wait_ge(ctr + C.xready + i, (unsigned)((tile_width(n, t, i) + 31) / 32), a.hdr)) return;
        const int64_t r = c * 32 + lane;
        int64_t k0, k1;
        slice_cols(n, t, i, s, k0, k1);
        // in the slice's fixed order: tiles N-1, N-2, ..., i+1 before i (the
        // queue hands out a slice's tiles a whole step apart, so the turn is
        // almost always there)
        const int nb = N - 1 - i;
        if (!warp_wait_ge(ctr + C.turn + c * S + s, (unsigned)nb, a.hdr)) return;
        acc_rows_times_x<P>(a.acc, pps, (c * S + s) * 32 + lane, nb == 0, a.R, a.ldr, a.psr, r, k0, k1, a.x,
                            a.psx);
        warp_publish(ctr + C.turn + c * S + s);
    }
}

}  // namespace mdls
