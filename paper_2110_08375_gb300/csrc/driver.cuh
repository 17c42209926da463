// Host-side launch sequences of Algorithms 1 and 2, templated on the limb
// count P.  Each precision is instantiated in its own translation unit.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "layout.h"
#include "profile.h"

namespace mdls {

template <int P>
constexpr int panel_threads() {
    return P == 8 ? 128 : 256;
}

#define MDLS_LAUNCH_CHECK()                                  \
    do {                                                     \
        if (cudaGetLastError() != cudaSuccess) return MDLS_ERR_CUDA; \
    } while (0)

inline int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Scratch for split-K partial sums (cap md values per plane).
struct SplitBuf {
    double* ptr;
    int64_t cap;
};

// Launches one md GEMM.  When the output grid alone would leave SMs idle,
// the K range is split over grid.z (at most 16 ways, partials in `sb`) and a
// reduction kernel adds the partials in a fixed order.
template <int P, class AV, class BV>
int launch_gemm(int stage, cudaStream_t st, SplitBuf sb, int64_t M, int64_t N, int64_t K, AV a, BV b,
                Dense c, bool neg, bool acc, bool upper_only = false) {
    if (M <= 0 || N <= 0) return MDLS_OK;
    StageScope sc(stage, st);
    const int64_t gx = (M + kGemmTile - 1) / kGemmTile, gy = (N + kGemmTile - 1) / kGemmTile;
    const int64_t tiles = upper_only ? (gx * (gx + 1)) / 2 : gx * gy;
    const int64_t target = 2 * (int64_t)sm_count();
    int64_t S = 1;
    if (tiles < target && K >= 4 * kGemmTile && sb.ptr != nullptr) {
        S = (target + tiles - 1) / tiles;
        if (S > 16) S = 16;
        if (S > K / (2 * kGemmTile)) S = K / (2 * kGemmTile);
        while (S > 1 && S * M * N > sb.cap) --S;
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
        gemm_kernel<P, AV, BV><<<grid, kGemmTile * kGemmTile, 0, st>>>(
            M, N, K, a, b, c, neg ? 1 : 0, acc ? 1 : 0, kchunk, 0, upper_only ? 1 : 0);
        MDLS_LAUNCH_CHECK();
        return MDLS_OK;
    }
    Dense part{sb.ptr, M, sb.cap};
    gemm_kernel<P, AV, BV><<<grid, kGemmTile * kGemmTile, 0, st>>>(M, N, K, a, b, part, 0, 0, kchunk,
                                                                    M * N, upper_only ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    const int64_t total = M * N;
    split_reduce_kernel<P><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(
        M, N, (int)S, sb.ptr, M, sb.cap, M * N, c, neg ? 1 : 0, acc ? 1 : 0);
    MDLS_LAUNCH_CHECK();
    return MDLS_OK;
}

// largest panel width the cooperative launch can hold on this device
template <int P>
int panel_capacity() {
    static int cap = -1;
    if (cap < 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_kernel<P, panel_threads<P>()>,
                                                      panel_threads<P>(), 0);
        cap = sms * per;
    }
    return cap;
}

// Blocked Householder QR (Algorithm 2) of the m x n leading part of the
// working matrix A (ld, ps); columns n .. n+nextra-1 of A are right-hand
// sides that receive the same transformations (Q^T b).  Q (m x m) is formed
// when Q != nullptr.  R is left in the upper triangle, the Householder
// vectors below it; zero_lower clears them at the end.
template <int P>
int qr_run(int64_t m, int64_t n, int nextra, double* A, int64_t lda, int64_t psa, double* Q,
           int64_t ldq, int64_t psq, int t, char* ws, const QrLayout& L, WsHeader* hdr,
           bool zero_lower, cudaStream_t st) {
    constexpr int NT = panel_threads<P>();
    if (t > panel_capacity<P>()) return MDLS_ERR_UNSUPPORTED;
    double* beta = reinterpret_cast<double*>(ws + L.beta);
    double* G = reinterpret_cast<double*>(ws + L.G);
    double* T = reinterpret_cast<double*>(ws + L.T);
    double* X = reinterpret_cast<double*>(ws + L.X);
    double* Wb = reinterpret_cast<double*>(ws + L.W);
    unsigned int* flags = reinterpret_cast<unsigned int*>(ws + L.flags);
    const SplitBuf sb{reinterpret_cast<double*>(ws + L.split), L.split_cap};
    const int64_t tt2 = (int64_t)t * t;
    const int64_t psx = (int64_t)t * L.xcols;
    const int64_t ldw = m;
    const int64_t psw = L.wcols * m;
    const int64_t ntiles = (n + t - 1) / t;
    const bool want_q = (Q != nullptr);

    for (int64_t k = 0; k < ntiles; ++k) {
        const int64_t j0 = k * t;
        const int w = (int)((n - j0) < t ? (n - j0) : t);
        const int64_t r = m - j0;
        // 1. panel: Householder vectors, beta, R_kk
        PanelArgs pa{A, lda, psa, j0, r, w, beta, (int64_t)t, flags, (unsigned int)(k + 1), hdr};
        void* args[] = {&pa};
        {
            StageScope sc(ST_PANEL, st);
            if (cudaLaunchCooperativeKernel((const void*)panel_kernel<P, NT>, dim3(w), dim3(NT), args,
                                            0, st) != cudaSuccess)
                return MDLS_ERR_CUDA;
        }
        const int64_t nc = n + nextra - (j0 + w);  // trailing columns incl. right-hand sides
        if (nc <= 0 && !want_q) continue;
        // 2. WY form: G = Y^T Y, T from G and the betas, W = -Y T
        const double* Yp = A + j0 * lda + j0;
        ViewTrap Y{Yp, lda, psa};
        ViewTrapT Yt{Yp, lda, psa};
        int rc = launch_gemm<P>(ST_W, st, sb, w, w, r, Yt, Y, Dense{G, t, tt2}, false, false, true);
        if (rc) return rc;
        {
            StageScope sc(ST_W, st);
            wy_t_kernel<P><<<(unsigned)((w + 3) / 4), 128, 0, st>>>(G, t, tt2, beta, t, w, T, t, tt2);
            MDLS_LAUNCH_CHECK();
        }
        double* Wk = want_q ? (Wb + j0 * ldw + j0) : Wb;
        rc = launch_gemm<P>(ST_W, st, sb, r, w, w, Y, ViewUpper{T, t, tt2}, Dense{Wk, ldw, psw}, true, false);
        if (rc) return rc;
        // 3. trailing update C := C + Y (W^T C)
        if (nc > 0) {
            double* Cp = A + (j0 + w) * lda + j0;
            rc = launch_gemm<P>(ST_TRAIL, st, sb, w, nc, r, ViewDenseT{Wk, ldw, psw}, ViewDense{Cp, lda, psa},
                                Dense{X, t, psx}, false, false);
            if (rc) return rc;
            rc = launch_gemm<P>(ST_TRAIL, st, sb, r, nc, w, Y, ViewDense{X, t, psx}, Dense{Cp, lda, psa}, false, true);
            if (rc) return rc;
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
template <int P>
int bs_run(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y, int64_t psy,
           double* x, int64_t psx, int t, char* ws, const BsLayout& L, WsHeader* hdr,
           cudaStream_t st) {
    const int64_t N = (n + t - 1) / t;
    const int64_t tt2 = (int64_t)t * t;
    double* D = reinterpret_cast<double*>(ws + L.D);
    double* bw = reinterpret_cast<double*>(ws + L.b);
    const int64_t dps = N * tt2;
    for (int l = 0; l < P; ++l)
        if (cudaMemcpyAsync(bw + l * n, y + l * psy, n * sizeof(double), cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
            return MDLS_ERR_CUDA;
    // step 1: invert the N diagonal tiles (N blocks of t threads)
    {
        StageScope sc(ST_INV, st);
        tri_inv_kernel<P><<<(unsigned)((N * t + 3) / 4), 128, 0, st>>>(R, ldr, psr, n, t, N, D, t,
                                                                         dps, tt2, hdr);
        MDLS_LAUNCH_CHECK();
    }
    // step 2: i = N..1
    for (int64_t i = N - 1; i >= 0; --i) {
        const int64_t o = i * t;
        const int tt = (int)((n - o) < t ? (n - o) : t);
        {
            StageScope sc(ST_MULINV, st);
            bs_mulinv_kernel<P><<<1, t, 0, st>>>(D + i * tt2, t, dps, tt, bw, n, x, psx, o);
            MDLS_LAUNCH_CHECK();
        }
        if (o > 0) {
            StageScope sc(ST_BSUPD, st);
            bs_update_kernel<P><<<(unsigned)((o + 127) / 128), 128, 0, st>>>(R, ldr, psr, o, tt, x,
                                                                           psx, bw, n);
            MDLS_LAUNCH_CHECK();
        }
    }
    return MDLS_OK;
}

template <int P>
int qr_entry(int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q, int64_t ldq,
             int64_t psq, int t, void* ws, cudaStream_t st) {
    QrLayout L = qr_layout(P, m, n, t, Q != nullptr, 0);
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
             int64_t psb, double* x, int64_t psx, int t, void* ws, cudaStream_t st) {
    LsLayout L = ls_layout(P, m, n, t);
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
    int rc = qr_run<P>(m, n, 1, Aw, m, psw, nullptr, 0, 0, t, w, L.qr, hdr, false, st);
    if (rc) return rc;
    return bs_run<P>(n, Aw, m, psw, Aw + n * m, psw, x, psx, t, w, L.bs, hdr, st);
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

}  // namespace mdls

#define MDLS_INSTANTIATE(P)                                                                       \
    namespace mdls {                                                                              \
    int qr_entry_p##P(int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q,       \
                      int64_t ldq, int64_t psq, int t, void* ws, cudaStream_t st) {               \
        return qr_entry<P>(m, n, A, lda, psa, Q, ldq, psq, t, ws, st);                           \
    }                                                                                             \
    int bs_entry_p##P(int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y,      \
                      int64_t psy, double* x, int64_t psx, int t, void* ws, cudaStream_t st) {     \
        return bs_entry<P>(n, R, ldr, psr, y, psy, x, psx, t, ws, st);                           \
    }                                                                                             \
    int ls_entry_p##P(int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa,            \
                      const double* b, int64_t psb, double* x, int64_t psx, int t, void* ws,      \
                      cudaStream_t st) {                                                          \
        return ls_entry<P>(m, n, A, lda, psa, b, psb, x, psx, t, ws, st);                        \
    }                                                                                             \
    int vec_entry_p##P(int op, int64_t count, const double* a, int64_t psa, const double* b,      \
                       int64_t psb, double* c, int64_t psc, cudaStream_t st) {                    \
        return vec_entry<P>(op, count, a, psa, b, psb, c, psc, st);                              \
    }                                                                                             \
    }
