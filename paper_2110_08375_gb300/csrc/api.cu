// C ABI of libmdls (declared in include/mdls.h): argument checks, workspace
// sizes and dispatch to the per-precision instantiations.
#include <cuda_runtime.h>

#include "../../include/mdls.h"
#include "layout.h"

namespace mdls {
#define MDLS_DECLARE(P)                                                                           \
    int qr_entry_p##P(int64_t, int64_t, double*, int64_t, int64_t, double*, int64_t, int64_t, int, \
                      int, void*, cudaStream_t);                                                   \
    int bs_entry_p##P(int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*,  \
                      int64_t, int, void*, cudaStream_t);                                          \
    int ls_entry_p##P(int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t,  \
                      double*, int64_t, int, int, void*, cudaStream_t, bool);                      \
    int vec_entry_p##P(int, int64_t, const double*, int64_t, const double*, int64_t, double*,     \
                       int64_t, cudaStream_t);                                                     \
    int ls_refine_entry_p##P(int64_t, int64_t, const double*, int64_t, int64_t, const double*,    \
                             int64_t, double*, int64_t, int, int, void*, cudaStream_t);                  \
    int toe_entry_p##P(int64_t, int64_t, int64_t, const double*, int64_t, int64_t, int64_t,          \
                       const double*, int64_t, int64_t, double*, int64_t, int64_t, int, void*,         \
                       cudaStream_t);
MDLS_DECLARE(2)
MDLS_DECLARE(4)
MDLS_DECLARE(8)
#define MDLS_DECLARE_Z(P)                                                                                    \
    int zqr_entry_p##P(int64_t, int64_t, double*, double*, int64_t, int64_t, double*, double*, int64_t,       \
                       int64_t, int, void*, cudaStream_t);                                                     \
    int zbs_entry_p##P(int64_t, const double*, const double*, int64_t, int64_t, const double*, const double*, \
                       int64_t, double*, double*, int64_t, int, void*, cudaStream_t);                         \
    int zls_entry_p##P(int64_t, int64_t, const double*, const double*, int64_t, int64_t, const double*,       \
                       const double*, int64_t, double*, double*, int64_t, int, void*, cudaStream_t);
MDLS_DECLARE_Z(2)
MDLS_DECLARE_Z(4)
MDLS_DECLARE_Z(8)
}  // namespace mdls

using namespace mdls;

int& mdls::bs_schedule_ref() {
    static int s = MDLS_BS_AUTO;
    return s;
}

int& mdls::split_engine_ref() {
    static int e = MDLS_SPLIT_ENGINE_AUTO;
    return e;
}

static bool prec_ok(int p) { return p == 2 || p == 4 || p == 8; }

static bool ws_ok(const void* ws, size_t have, size_t need) {
    return ws != nullptr && have >= need && (reinterpret_cast<uintptr_t>(ws) & 255) == 0;
}

extern "C" {

int mdls_version(void) { return 100; }

const char* mdls_status_string(int code) {
    switch (code) {
        case MDLS_OK: return "ok";
        case MDLS_ERR_ARG: return "invalid argument (size, stride, pointer or tile)";
        case MDLS_ERR_PREC: return "precision must be 2, 4 or 8 limbs";
        case MDLS_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case MDLS_ERR_SINGULAR: return "zero pivot on the diagonal of R";
        case MDLS_ERR_CUDA: return "CUDA launch or copy failed";
        case MDLS_ERR_TIMEOUT: return "a bounded device wait gave up";
        case MDLS_ERR_UNSUPPORTED: return "request not supported by this build or device";
        case MDLS_ERR_NOT_CONVERGED: return "iterative refinement did not reach the target precision";
        default: return "unknown status";
    }
}

size_t mdls_qr_workspace(int prec, int64_t m, int64_t n, int tile, int want_q, int mode) {
    int t = norm_tile(tile, n);
    if (!prec_ok(prec) || t < 1 || m < n || n < 1) return 0;
    if (mode != MDLS_MODE_PLAIN && mode != MDLS_MODE_SPLIT) return 0;
    size_t total = 0;
    qr_layout(prec, m, n, t, want_q != 0, 0, &total, mode == MDLS_MODE_SPLIT);
    return total;
}

size_t mdls_backsub_workspace(int prec, int64_t n, int tile) {
    int t = norm_tile_bs(tile, n, prec);
    if (!prec_ok(prec) || t < 1 || n < 1) return 0;
    size_t total = 0;
    bs_layout(prec, n, t, &total);
    return total;
}

static bool refine_mode(int prec, int mode) { return mode == MDLS_MODE_REFINE && prec > 2; }

size_t mdls_lstsq_workspace(int prec, int64_t m, int64_t n, int tile, int mode) {
    int t = norm_tile(tile, n);
    if (!prec_ok(prec) || t < 1 || m < n || n < 1) return 0;
    if (mode != MDLS_MODE_PLAIN && mode != MDLS_MODE_REFINE && mode != MDLS_MODE_SPLIT) return 0;
    if (refine_mode(prec, mode)) return ref_layout(prec, m, n, t).total;
    return ls_layout(prec, m, n, t, mode == MDLS_MODE_SPLIT).total;
}

int mdls_qr(int prec, int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q,
            int64_t ldq, int64_t psq, int tile, int mode, void* ws, size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (mode != MDLS_MODE_PLAIN && mode != MDLS_MODE_SPLIT) return MDLS_ERR_ARG;
    if (!A || n < 1 || m < n || lda < m || psa < lda * n) return MDLS_ERR_ARG;
    if (Q && (ldq < m || psq < ldq * m)) return MDLS_ERR_ARG;
    const int t = norm_tile(tile, n);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_qr_workspace(prec, m, n, tile, Q != nullptr, mode)))
        return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return qr_entry_p2(m, n, A, lda, psa, Q, ldq, psq, t, mode, ws, st);
        case 4: return qr_entry_p4(m, n, A, lda, psa, Q, ldq, psq, t, mode, ws, st);
        default: return qr_entry_p8(m, n, A, lda, psa, Q, ldq, psq, t, mode, ws, st);
    }
}

int mdls_backsub(int prec, int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y,
                 int64_t psy, double* x, int64_t psx, int tile, void* ws, size_t ws_bytes,
                 void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (!R || !y || !x || n < 1 || ldr < n || psr < ldr * n || psy < n || psx < n)
        return MDLS_ERR_ARG;
    const int t = norm_tile_bs(tile, n, prec);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_backsub_workspace(prec, n, tile))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return bs_entry_p2(n, R, ldr, psr, y, psy, x, psx, t, ws, st);
        case 4: return bs_entry_p4(n, R, ldr, psr, y, psy, x, psx, t, ws, st);
        default: return bs_entry_p8(n, R, ldr, psr, y, psy, x, psx, t, ws, st);
    }
}

int mdls_lstsq(int prec, int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa,
               const double* b, int64_t psb, double* x, int64_t psx, int tile, int mode, void* ws,
               size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (mode != MDLS_MODE_PLAIN && mode != MDLS_MODE_REFINE && mode != MDLS_MODE_SPLIT)
        return MDLS_ERR_ARG;
    if (!A || !b || !x || n < 1 || m < n || lda < m || psa < lda * n || psb < m || psx < n)
        return MDLS_ERR_ARG;
    const int t = norm_tile(tile, n);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_lstsq_workspace(prec, m, n, tile, mode))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (refine_mode(prec, mode)) {
        if (prec == 4) return ls_refine_entry_p4(m, n, A, lda, psa, b, psb, x, psx, t, 3, ws, st);
        return ls_refine_entry_p8(m, n, A, lda, psa, b, psb, x, psx, t, 6, ws, st);
    }
    switch (prec) {
        case 2: return ls_entry_p2(m, n, A, lda, psa, b, psb, x, psx, t, mode, ws, st, false);
        case 4: return ls_entry_p4(m, n, A, lda, psa, b, psb, x, psx, t, mode, ws, st, false);
        default: return ls_entry_p8(m, n, A, lda, psa, b, psb, x, psx, t, mode, ws, st, false);
    }
}

int mdls_vec_op(int prec, int op, int64_t count, const double* a, int64_t psa, const double* b,
                int64_t psb, double* c, int64_t psc, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (op < MDLS_OP_ADD || op > MDLS_OP_SQRT || count < 0 || !a || !c || psa < count || psc < count)
        return MDLS_ERR_ARG;
    if (op != MDLS_OP_SQRT && (!b || psb < count)) return MDLS_ERR_ARG;
    if (op == MDLS_OP_SQRT) { b = a; psb = psa; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return vec_entry_p2(op, count, a, psa, b, psb, c, psc, st);
        case 4: return vec_entry_p4(op, count, a, psa, b, psb, c, psc, st);
        default: return vec_entry_p8(op, count, a, psa, b, psb, c, psc, st);
    }
}

size_t mdls_zqr_workspace(int prec, int64_t m, int64_t n, int tile, int want_q) {
    const int t = norm_tile(tile, n);
    if (!prec_ok(prec) || t < 1 || m < n || n < 1) return 0;
    size_t total = 0;
    zqr_layout(prec, m, n, t, want_q != 0, &total);
    return total;
}

size_t mdls_zbacksub_workspace(int prec, int64_t n, int tile) {
    const int t = norm_tile_bs(tile, n, prec);
    if (!prec_ok(prec) || t < 1 || n < 1) return 0;
    size_t total = 0;
    zbs_layout(prec, n, t, &total);
    return total;
}

size_t mdls_zlstsq_workspace(int prec, int64_t m, int64_t n, int tile) {
    const int t = norm_tile(tile, n);
    if (!prec_ok(prec) || t < 1 || m < n || n < 1) return 0;
    return zls_layout(prec, m, n, t).total;
}

int mdls_zqr(int prec, int64_t m, int64_t n, double* Ar, double* Ai, int64_t lda, int64_t psa, double* Qr,
             double* Qi, int64_t ldq, int64_t psq, int tile, void* ws, size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (!Ar || !Ai || n < 1 || m < n || lda < m || psa < lda * n) return MDLS_ERR_ARG;
    if ((Qr != nullptr) != (Qi != nullptr)) return MDLS_ERR_ARG;
    if (Qr && (ldq < m || psq < ldq * m)) return MDLS_ERR_ARG;
    const int t = norm_tile(tile, n);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_zqr_workspace(prec, m, n, tile, Qr != nullptr))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return zqr_entry_p2(m, n, Ar, Ai, lda, psa, Qr, Qi, ldq, psq, t, ws, st);
        case 4: return zqr_entry_p4(m, n, Ar, Ai, lda, psa, Qr, Qi, ldq, psq, t, ws, st);
        default: return zqr_entry_p8(m, n, Ar, Ai, lda, psa, Qr, Qi, ldq, psq, t, ws, st);
    }
}

int mdls_zbacksub(int prec, int64_t n, const double* Rr, const double* Ri, int64_t ldr, int64_t psr,
                  const double* yr, const double* yi, int64_t psy, double* xr, double* xi, int64_t psx, int tile,
                  void* ws, size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (!Rr || !Ri || !yr || !yi || !xr || !xi || n < 1 || ldr < n || psr < ldr * n || psy < n || psx < n)
        return MDLS_ERR_ARG;
    const int t = norm_tile_bs(tile, n, prec);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_zbacksub_workspace(prec, n, tile))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return zbs_entry_p2(n, Rr, Ri, ldr, psr, yr, yi, psy, xr, xi, psx, t, ws, st);
        case 4: return zbs_entry_p4(n, Rr, Ri, ldr, psr, yr, yi, psy, xr, xi, psx, t, ws, st);
        default: return zbs_entry_p8(n, Rr, Ri, ldr, psr, yr, yi, psy, xr, xi, psx, t, ws, st);
    }
}

int mdls_zlstsq(int prec, int64_t m, int64_t n, const double* Ar, const double* Ai, int64_t lda, int64_t psa,
                const double* br, const double* bi, int64_t psb, double* xr, double* xi, int64_t psx, int tile,
                void* ws, size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (!Ar || !Ai || !br || !bi || !xr || !xi || n < 1 || m < n || lda < m || psa < lda * n || psb < m ||
        psx < n)
        return MDLS_ERR_ARG;
    const int t = norm_tile(tile, n);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_zlstsq_workspace(prec, m, n, tile))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return zls_entry_p2(m, n, Ar, Ai, lda, psa, br, bi, psb, xr, xi, psx, t, ws, st);
        case 4: return zls_entry_p4(m, n, Ar, Ai, lda, psa, br, bi, psb, xr, xi, psx, t, ws, st);
        default: return zls_entry_p8(m, n, Ar, Ai, lda, psa, br, bi, psb, xr, xi, psx, t, ws, st);
    }
}

size_t mdls_toeplitz_lstsq_workspace(int prec, int64_t m, int64_t n, int tile) {
    const int t = norm_tile(tile, n);
    if (!prec_ok(prec) || t < 1 || m < n || n < 1) return 0;
    return toe_layout(prec, m, n, t).total;
}

int mdls_toeplitz_lstsq(int prec, int64_t m, int64_t n, int64_t d, const double* J, int64_t ldj, int64_t psj,
                        int64_t bsj, const double* b, int64_t psb, int64_t bsb, double* x, int64_t psx,
                        int64_t bsx, int tile, void* ws, size_t ws_bytes, void* stream) {
    if (!prec_ok(prec)) return MDLS_ERR_PREC;
    if (!J || !b || !x || n < 1 || m < n || d < 0 || ldj < m || bsj < ldj * n || psj < bsj * (d + 1) ||
        bsb < m || psb < bsb * (d + 1) || bsx < n || psx < bsx * (d + 1))
        return MDLS_ERR_ARG;
    const int t = norm_tile(tile, n);
    if (t < 1) return MDLS_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, mdls_toeplitz_lstsq_workspace(prec, m, n, tile))) return MDLS_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case 2: return toe_entry_p2(m, n, d, J, ldj, psj, bsj, b, psb, bsb, x, psx, bsx, t, ws, st);
        case 4: return toe_entry_p4(m, n, d, J, ldj, psj, bsj, b, psb, bsb, x, psx, bsx, t, ws, st);
        default: return toe_entry_p8(m, n, d, J, ldj, psj, bsj, b, psb, bsb, x, psx, bsx, t, ws, st);
    }
}

int mdls_set_backsub_schedule(int schedule) {
    if (schedule != MDLS_BS_AUTO && schedule != MDLS_BS_PER_STEP && schedule != MDLS_BS_PERSISTENT)
        return MDLS_ERR_ARG;
    bs_schedule_ref() = schedule;
    return MDLS_OK;
}

int mdls_set_split_engine(int engine) {
    if (engine != MDLS_SPLIT_ENGINE_AUTO && engine != MDLS_SPLIT_ENGINE_MMA_SYNC &&
        engine != MDLS_SPLIT_ENGINE_TCGEN05)
        return MDLS_ERR_ARG;
    split_engine_ref() = engine;
    return MDLS_OK;
}

int mdls_read_status(const void* ws, int* status, void* stream) {
    if (!ws || !status) return MDLS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MDLS_ERR_CUDA;
    if (cudaMemcpy(status, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MDLS_ERR_CUDA;
    return MDLS_OK;
}

}  // extern "C"
