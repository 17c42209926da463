/*
 * mdls.h -- multiple-double least squares on one GB300 GPU (sm_103a).
 *
 * C ABI of libmdls.so.  The operations follow arXiv 2110.08375 ("Least Squares
 * on GPUs in Multiple Double Precision", J. Verschelde):
 *   - the problem (Section 1): the least squares solution x of A x = b
 *     minimises ||b - A x||_2^2; A = QR reduces it to R x = Q^T b, solved by
 *     back substitution;
 *   - multiple-double numbers (Section 1.1): an unevaluated sum of p doubles,
 *     p = 2 (double double), 4 (quad double), 8 (octo double);
 *   - blocked Householder QR (Section 3, Algorithm 2) with the WY
 *     representation P = I + W Y^T of each tile (Section 3, equations for
 *     P_WY and z = -beta (v + W Y^T v));
 *   - tiled back substitution with inverted diagonal tiles (Section 2,
 *     Algorithm 1).
 *
 * STORAGE (all matrices and vectors): limb-planar, as in the paper's Section 2
 * ("an array of m matrices, U_1 holds the most significant doubles").  Limb l
 * (0 = most significant) of entry (i, j) of a matrix is at
 *     ptr[l * ps + j * ld + i]            (column-major planes),
 * with ld >= rows and ps >= ld * cols (plane stride, in doubles).  Limb l of
 * entry i of a vector is at ptr[l * ps + i].  Inputs are read as the sum of
 * their limbs and must be normalised (|limb_{k+1}| <= ulp(limb_k)); outputs
 * are normalised the same way (to within a factor 2).
 *
 * POINTERS: every matrix, vector and workspace pointer is a DEVICE pointer
 * (cudaMalloc'd or equivalent) owned by the caller.  The library allocates
 * nothing: scratch space is the caller's workspace `ws`, at least as large as
 * the matching *_workspace() query, 256-byte aligned.  A workspace may be
 * reused by consecutive calls on the same stream, never by two calls that run
 * concurrently.
 *
 * STREAM: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 * asynchronous: they enqueue kernels and return.  Host-detectable errors are
 * returned at once (negative codes below) and nothing is enqueued.  Errors
 * only the device can detect (a zero pivot, a bounded wait that gave up) are
 * recorded in the workspace status word, readable with mdls_read_status()
 * after the call.
 *
 * PRECISION `prec`: 2, 4 or 8 limbs.  TILE `tile`: tile size t in 1..256 (the
 * paper's n), 0 = default (128 for QR and least squares; for mdls_backsub
 * 128 in dd and qd, 64 in od; the problem size when smaller).  The last
 * tile may be narrower than t ("ragged"), so n need not be a multiple of t.
 */
#ifndef MDLS_H
#define MDLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MDLS_OK 0
#define MDLS_ERR_ARG (-1)         /* bad size, stride, pointer or tile   */
#define MDLS_ERR_PREC (-2)        /* prec not in {2, 4, 8}                */
#define MDLS_ERR_WORKSPACE (-3)   /* ws too small, NULL or misaligned     */
#define MDLS_ERR_SINGULAR (-4)    /* device: zero pivot on R's diagonal   */
#define MDLS_ERR_CUDA (-5)        /* a kernel launch failed               */
#define MDLS_ERR_TIMEOUT (-6)     /* device: a bounded wait gave up       */
#define MDLS_ERR_UNSUPPORTED (-7) /* valid request this build cannot run  */
#define MDLS_ERR_NOT_CONVERGED (-8) /* device: refinement short of target */

/* arithmetic modes of the QR and least-squares calls */
#define MDLS_MODE_PLAIN 0  /* all arithmetic in md on the FP64 CUDA cores */
#define MDLS_MODE_SPLIT 1  /* WY products as exact bf16 digit products on the tensor cores */
#define MDLS_MODE_REFINE 2 /* least squares only: factor in double double, refine in prec */

/* Library version (major * 10000 + minor * 100 + patch). */
int mdls_version(void);

/* Human-readable text of a status code (static storage). */
const char* mdls_status_string(int code);

/*
 * mdls_qr -- blocked Householder QR, Algorithm 2 of the paper (Section 3).
 *   A (m x n, m >= n >= 1), in place: on return its upper triangle holds R
 *     (diagonal >= 0; reflectors follow Golub & Van Loan Alg. 5.1.1 so that
 *     each P x = ||x|| e1) and its strictly lower part is exactly zero.
 *   Q (m x m) receives the orthogonal factor with A = Q R when Q != NULL
 *     (Algorithm 2's output); ldq >= m, psq >= ldq * m.  Q must not overlap A.
 *   mode: MDLS_MODE_PLAIN, or MDLS_MODE_SPLIT: every product of the WY form
 *     (Y^T Y, W = -Y T, W^T C, C + Y X, and those of Q) is evaluated by
 *     splitting each md entry, scaled by a power of two per row of the left
 *     and per column of the right factor, into S = ceil((53 prec + 12) / 8)
 *     base-256 digits (15 dd, 28 qd, 55 od) held exactly in bf16; the digit
 *     products accumulate exactly in fp32 on the tensor cores and are
 *     renormalised into prec limbs (error-free splitting of Ozaki, Ogita,
 *     Oishi and Rump).  The panel, T, norms and beta stay in md on the FP64
 *     cores.  Accuracy is normwise: about 2^(-53 prec) times the row and
 *     column scales of each product, as for the plain md products.
 * Per tile of t columns: the Householder vectors of the tile, its WY form
 * (P = I + W Y^T), then the trailing update C := C + Y (W^T C).  Q is
 * accumulated backward from the identity, Q := P_k Q for k = N..1.
 * Workspace: mdls_qr_workspace(prec, m, n, tile, Q != NULL, mode) bytes.
 * Returns MDLS_OK or a negative status; device-side failures (timeout of a
 * bounded wait) are recorded in the workspace status.
 */
int mdls_qr(int prec, int64_t m, int64_t n, double* A, int64_t lda, int64_t psa, double* Q,
            int64_t ldq, int64_t psq, int tile, int mode, void* ws, size_t ws_bytes,
            void* stream);
size_t mdls_qr_workspace(int prec, int64_t m, int64_t n, int tile, int want_q, int mode);

/*
 * mdls_backsub -- tiled accelerated back substitution, Algorithm 1 of the
 * paper (Section 2): solves R x = y for the upper triangular n x n R (only
 * the upper triangle is read; diagonal nonzero).
 *   Step 1 inverts the N = ceil(n / t) diagonal tiles (one thread per column
 *   of each inverse, solving U v = e_k).  Step 2 runs i = N..1:
 *   x_i := U_i^{-1} y_i, then y_j := y_j - A_{j,i} x_i for all j < i at once.
 *   R, y are not modified; x (length n, plane stride psx >= n) is written.
 *   A zero diagonal entry records MDLS_ERR_SINGULAR in the workspace status.
 * Workspace: mdls_backsub_workspace(prec, n, tile) bytes.
 */
int mdls_backsub(int prec, int64_t n, const double* R, int64_t ldr, int64_t psr, const double* y,
                 int64_t psy, double* x, int64_t psx, int tile, void* ws, size_t ws_bytes,
                 void* stream);
size_t mdls_backsub_workspace(int prec, int64_t n, int tile);

/*
 * mdls_set_backsub_schedule -- how step 2 of Algorithm 1 (x_i := U_i^{-1} y_i,
 * y_j := y_j - A_{j,i} x_i for i = N..1) is launched, for every later call
 * of this process (mdls_backsub, mdls_backsub_noalloc and the back
 * substitution inside mdls_lstsq):
 *   MDLS_BS_PER_STEP: as in the paper, kernels per tile step, each step
 *     spread over the whole GPU;
 *   MDLS_BS_PERSISTENT: one cooperative launch in which the steps overlap:
 *     the updates of rows two or more tiles above the current tile run from
 *     a task queue on most SMs while a few reserved SMs carry the chain
 *     x_i -> x_{i-1}; same arithmetic, each y_j receives its terms in the
 *     same fixed order (results are deterministic, though not bitwise equal
 *     to the per-step schedule's);
 *   MDLS_BS_AUTO (default): persistent in double double from 8 tiles on and
 *     in quad double from n = 8192 on, per step otherwise (measured choice).
 * Tiles that are not a multiple of 32 wide always run per step.  Not meant
 * to change while calls are in flight.  Returns MDLS_OK or MDLS_ERR_ARG.
 */
#define MDLS_BS_AUTO 0
#define MDLS_BS_PER_STEP 1
#define MDLS_BS_PERSISTENT 2
int mdls_set_backsub_schedule(int schedule);

/*
 * mdls_set_split_engine -- which tensor-core kernel evaluates the digit
 * products of MDLS_MODE_SPLIT (and of the double double factorisation of
 * MDLS_MODE_REFINE), for every later call of this process.  Both compute the
 * same exact sums of digit products (the error-free splitting of the WY
 * products, Section 3's trailing update and Q accumulation):
 *   MDLS_SPLIT_ENGINE_TCGEN05: fifth-generation tensor cores (tcgen05.mma,
 *     accumulators in tensor memory, operands staged by bulk copies), one
 *     128-row tile per block, K split over blocks when the tiles alone leave
 *     SMs idle (the blocks' exact partial products are then rounded to prec
 *     limbs and added in a fixed order);
 *   MDLS_SPLIT_ENGINE_MMA_SYNC: warp-level mma.sync m16n8k16, 16 x 8 tiles,
 *     K never split;
 *   MDLS_SPLIT_ENGINE_AUTO (default): tcgen05 for products of at least 64
 *     rows and 16 columns of single problems, mma.sync for the rest and for
 *     every product of mdls_lstsq_batched / mdls_batched_*.
 * Without a K split the two give bit-identical products.  Not meant to change
 * while calls are in flight.  Returns MDLS_OK or MDLS_ERR_ARG.
 */
#define MDLS_SPLIT_ENGINE_AUTO 0
#define MDLS_SPLIT_ENGINE_MMA_SYNC 1
#define MDLS_SPLIT_ENGINE_TCGEN05 2
int mdls_set_split_engine(int engine);

/*
 * mdls_backsub_noalloc -- the same back substitution as mdls_backsub, for
 * callers that cannot allocate device memory when they call: a plugin inside
 * a host framework that owns all device memory through its own allocator, a
 * real-time or embedded loop whose memory budget is fixed at start-up, or
 * code that must not risk the implicit device synchronisation of cudaMalloc.
 * The paper has no counterpart to this entry point.
 *   It allocates nothing.  Its scratch (the inverted diagonal tiles, the
 *   working right-hand side and a status word) is a fixed device array of
 *   MDLS_BACKSUB_NOALLOC_MAX_BYTES inside the library, held by every GPU that
 *   loads the library until the process exits.  Problems needing more
 *   scratch than that (mdls_backsub_workspace(prec, n, tile) bytes; at tile
 *   128: n <= 4960 in dd, 2432 in qd, 1152 in od) are rejected with
 *   MDLS_ERR_WORKSPACE before anything is enqueued.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture.  Every call clears the status word itself.
 *   All calls share the one array: calls that overlap on the GPU (other
 *   streams, other host threads) race and corrupt each other's results.
 *   Keep per-stage timing (mdls_profile_enable) off: it creates CUDA events.
 *   status: NULL, or a DEVICE int that receives MDLS_OK or MDLS_ERR_SINGULAR
 *   when the solve has run.
 * Other arguments, layout and errors as for mdls_backsub.
 */
#define MDLS_BACKSUB_NOALLOC_MAX_BYTES (16u << 20)
int mdls_backsub_noalloc(int prec, int64_t n, const double* R, int64_t ldr, int64_t psr,
                         const double* y, int64_t psy, double* x, int64_t psx, int tile,
                         int* status, void* stream);

/*
 * mdls_lstsq -- least squares solution of A x = b (Section 1): the blocked QR
 * of Algorithm 2 applied to [A | b] (so Q^T b is formed by the same WY
 * updates and Q itself is never built), followed by Algorithm 1 on
 * R x = (Q^T b)[0:n].  A (m x n, m >= n >= 1) and b (length m) are read
 * only; x (length n) is written.  The working copy of [A | b] lives in ws.
 * mode MDLS_MODE_SPLIT: the QR of [A | b] with split products (see mdls_qr).
 * mode MDLS_MODE_REFINE (prec 4 or 8; with prec 2 it is the plain solve):
 *   factor A rounded to double double (its two leading limbs), solve in
 *   dd, then refine: r = b - A x in prec limbs, d = R^{-1}(Q^T r)[0:n] in dd,
 *   x = x + d in prec limbs -- 3 refinement steps for qd, 6 for od.  If the
 *   last correction is not below 2^(53-53 prec) |x| (ill-conditioned A),
 *   MDLS_ERR_NOT_CONVERGED is recorded in the workspace status.
 * Workspace: mdls_lstsq_workspace(prec, m, n, tile, mode) bytes.
 */
int mdls_lstsq(int prec, int64_t m, int64_t n, const double* A, int64_t lda, int64_t psa,
               const double* b, int64_t psb, double* x, int64_t psx, int tile, int mode, void* ws,
               size_t ws_bytes, void* stream);
size_t mdls_lstsq_workspace(int prec, int64_t m, int64_t n, int tile, int mode);

/*
 * mdls_toeplitz_lstsq -- lower triangular block-Toeplitz system, the linear
 * systems of Newton's method on power series that motivate the paper
 * (Section 1: the diagonal block is the Jacobian at the current point of a
 * path):  with J(t) = J_0 + J_1 t + ... + J_d t^d (m x n blocks, m >= n) and
 * b(t) = b_0 + ... + b_d t^d, the coefficients x_0 .. x_d of
 * J(t) x(t) = b(t) mod t^{d+1} by block forward substitution,
 *     J_0 x_k = b_k - sum_{i=1}^{k} J_i x_{k-i},   k = 0, ..., d,
 * each in the least-squares sense with ONE QR of J_0 (Algorithm 2, every
 * tile's W kept) and Algorithm 1 on its R (diagonal tiles inverted once):
 * x_k = R^{-1} (Q^T r_k)[0:n].  The paper states this application only as
 * its motivation; the blocked solve is this library's.
 *   J: block i, limb l, entry (r, c) at J[l * psj + i * bsj + c * ldj + r]
 *      (ldj >= m, bsj >= ldj n, psj >= (d + 1) bsj); read only.
 *   b: block k, limb l, entry r at b[l * psb + k * bsb + r] (bsb >= m,
 *      psb >= (d + 1) bsb); read only.
 *   x: block k at x[l * psx + k * bsx + c] (bsx >= n, psx >= (d + 1) bsx).
 * A zero pivot of J_0's R records MDLS_ERR_SINGULAR.  Workspace:
 * mdls_toeplitz_lstsq_workspace(prec, m, n, tile) bytes.
 */
size_t mdls_toeplitz_lstsq_workspace(int prec, int64_t m, int64_t n, int tile);
int mdls_toeplitz_lstsq(int prec, int64_t m, int64_t n, int64_t d, const double* J, int64_t ldj, int64_t psj,
                        int64_t bsj, const double* b, int64_t psb, int64_t bsb, double* x, int64_t psx,
                        int64_t bsx, int tile, void* ws, size_t ws_bytes, void* stream);

/*
 * Complex multiple doubles (the paper's Section 3 remark: on complex data the
 * transpose becomes the Hermitian transpose; Section 2: real and imaginary
 * parts are kept separately).  Every complex matrix or vector is passed as
 * two arrays of the layout above, its real part and its imaginary part, with
 * one leading dimension and one plane stride for both.
 *
 * mdls_zqr -- blocked complex Householder QR (Algorithm 2 with Hermitian
 *   transposes).  Reflectors are Hermitian, H = I - beta v v^H with beta real
 *   and v(0) = 1, and map the column x to e^{i arg x0} ||x|| e1 (the sign of
 *   Golub and Van Loan's Alg. 5.1.1 replaced by the phase of x0; x0 = 0 counts
 *   as phase 0; a column with nothing below x0 is left as it is), so R's
 *   diagonal carries the phases of the reflected leading entries and R is
 *   unique for full-rank A.  A (m x n, m >= n) is overwritten by R (strictly
 *   lower part exactly zero); Q (m x m, both parts, or both NULL) receives
 *   H_1 ... H_n.  Each tile's WY form is P = I + W Y^H; the trailing update is
 *   C := C + Y (W^H C).  The WY products run as four real md products each.
 *   Workspace: mdls_zqr_workspace(prec, m, n, tile, Q != NULL) bytes.
 * mdls_zbacksub -- Algorithm 1 on a complex upper triangular R (n x n; only
 *   the upper triangle is read): inverted diagonal tiles, then the tile loop.
 *   A zero diagonal entry records MDLS_ERR_SINGULAR.  Workspace:
 *   mdls_zbacksub_workspace(prec, n, tile) bytes.
 * mdls_zlstsq -- complex least squares min ||b - A x||_2: the complex QR of
 *   [A | b] (Q^H b by the same updates, no Q formed) and mdls_zbacksub on
 *   R x = (Q^H b)[0:n].  A and b are read only.  Workspace:
 *   mdls_zlstsq_workspace(prec, m, n, tile) bytes.
 * Arguments, tiles, streams and errors as for the real calls.
 */
int mdls_zqr(int prec, int64_t m, int64_t n, double* Ar, double* Ai, int64_t lda, int64_t psa, double* Qr,
             double* Qi, int64_t ldq, int64_t psq, int tile, void* ws, size_t ws_bytes, void* stream);
size_t mdls_zqr_workspace(int prec, int64_t m, int64_t n, int tile, int want_q);
int mdls_zbacksub(int prec, int64_t n, const double* Rr, const double* Ri, int64_t ldr, int64_t psr,
                  const double* yr, const double* yi, int64_t psy, double* xr, double* xi, int64_t psx, int tile,
                  void* ws, size_t ws_bytes, void* stream);
size_t mdls_zbacksub_workspace(int prec, int64_t n, int tile);
int mdls_zlstsq(int prec, int64_t m, int64_t n, const double* Ar, const double* Ai, int64_t lda, int64_t psa,
                const double* br, const double* bi, int64_t psb, double* xr, double* xi, int64_t psx, int tile,
                void* ws, size_t ws_bytes, void* stream);
size_t mdls_zlstsq_workspace(int prec, int64_t m, int64_t n, int tile);

/*
 * mdls_vec_op -- elementwise multiple-double arithmetic on device vectors
 * (Section 1.1: the md add, mul, div of Table 1, and sqrt):
 *   op MDLS_OP_ADD: c = a + b     MDLS_OP_SUB: c = a - b
 *      MDLS_OP_MUL: c = a * b     MDLS_OP_DIV: c = a / b
 *      MDLS_OP_FMA: c = c + a * b MDLS_OP_SQRT: c = sqrt(a) (b unused)
 * count entries, limb-planar with plane strides psa, psb, psc (>= count).
 * c may alias a or b.  Division by zero and sqrt of a negative number give
 * IEEE non-finite limbs; no status is recorded.
 */
#define MDLS_OP_ADD 0
#define MDLS_OP_SUB 1
#define MDLS_OP_MUL 2
#define MDLS_OP_DIV 3
#define MDLS_OP_FMA 4
#define MDLS_OP_SQRT 5
int mdls_vec_op(int prec, int op, int64_t count, const double* a, int64_t psa, const double* b,
                int64_t psb, double* c, int64_t psc, void* stream);

/*
 * Batched least squares: many independent problems of mixed shape and
 * precision solved by one launch of a CUDA graph (row a9 of the hot path;
 * the paper solves one system at a time).
 *   mdls_problem describes one problem, exactly as the arguments of
 *   mdls_lstsq (device pointers, limb-planar layout, A and b read only, x
 *   written); tile 0 lets the autotuner choose.
 *   mdls_batched_workspace(): bytes of caller workspace for the problems
 *   (0 if one of them is invalid).
 *   mdls_batched_plan(): checks the problems, picks each tile and mode --
 *   when autotune != 0, the autotuner's choice for the size class (prec, n
 *   rounded down to a power of two, the caller's tile if fixed): the first
 *   problem of a class never seen before in this process is solved with each
 *   candidate tile (8, 16, 32 for n <= 64; 8 .. 64 for n <= 256; 16, 32, 64,
 *   128 beyond; or the caller's) in each mode (plain, split: the same
 *   accuracy) on its own buffers, timed three times (median), and the
 *   fastest pair serves the whole class; otherwise the caller's tile or a
 *   fixed rule, in plain mode -- then captures every problem's kernels into one CUDA graph
 *   (parallel branches, largest problems first, each problem with its own
 *   slice of ws and a single-block panel) and instantiates it.  Planning
 *   synchronises the device and must not run inside a stream capture.
 *   mdls_batched_launch(): one graph launch solving every problem on stream.
 *   mdls_batched_status(): waits for stream, then copies each problem's
 *   device status (MDLS_OK, MDLS_ERR_SINGULAR, ...) to status[count] (host).
 *   mdls_batched_tiles(): the tile of each problem, to tiles[count] (host).
 *   mdls_batched_modes(): the mode of each problem (MDLS_MODE_PLAIN or
 *   MDLS_MODE_SPLIT), to modes[count] (host).
 *   mdls_batched_destroy(): frees the plan (not the caller's buffers).
 * The plan keeps pointers to the problems' buffers and to ws: they must stay
 * valid and must not move while the plan is used.
 */
typedef struct {
    int prec;     /* 2, 4 or 8 limbs */
    int tile;     /* 1..256, or 0: autotuned */
    int64_t m, n; /* m >= n >= 1 */
    const double* A;
    int64_t lda, psa;
    const double* b;
    int64_t psb;
    double* x;
    int64_t psx;
} mdls_problem;

size_t mdls_batched_workspace(const mdls_problem* probs, int count);
int mdls_batched_plan(const mdls_problem* probs, int count, void* ws, size_t ws_bytes, int autotune,
                      void** plan);
int mdls_batched_launch(void* plan, void* stream);
int mdls_batched_status(void* plan, int* status, void* stream);
int mdls_batched_tiles(void* plan, int* tiles);
int mdls_batched_modes(void* plan, int* modes);
void mdls_batched_destroy(void* plan);

/*
 * mdls_lstsq_batched -- the batched least-squares solve in one call, with the
 * problem array and the per-problem status on the device.
 *   probs: DEVICE array of count mdls_problem records (device pointers
 *     inside, as for mdls_batched_plan; tile 0 = autotuned).
 *   ws: DEVICE workspace of mdls_lstsq_batched_workspace(probs, count) bytes,
 *     256-byte aligned; it holds every problem's scratch and a table of
 *     their offsets.
 *   status: DEVICE int[count]; after the call has run on stream, status[i]
 *     is problem i's status (MDLS_OK, MDLS_ERR_SINGULAR, MDLS_ERR_TIMEOUT).
 * The call reads the problem array back to the host (it synchronises
 * stream once).  The first call for a given batch (same array contents,
 * workspace, count and device) plans it as mdls_batched_plan does with the
 * autotuner on, which runs trial solves; the plan is kept in a cache of the
 * 16 most recent batches, so later calls only launch its graph and a small
 * status-gathering kernel.  Not for use inside a stream capture.
 * Returns MDLS_OK, MDLS_ERR_ARG, MDLS_ERR_PREC, MDLS_ERR_WORKSPACE or
 * MDLS_ERR_CUDA.  mdls_lstsq_batched_workspace returns 0 for an invalid batch.
 */
size_t mdls_lstsq_batched_workspace(const mdls_problem* probs, int count);
int mdls_lstsq_batched(const mdls_problem* probs, int count, void* ws, size_t ws_bytes, int* status,
                       void* stream);

/*
 * mdls_wait_check -- diagnostic of the bounded device waits (failure
 * detection).  The Householder panel runs its column blocks side by side,
 * each waiting on flags that the blocks before it publish (Section 3: the
 * columns of a tile are reduced one after the other); every such wait gives
 * up after a limit, records MDLS_ERR_TIMEOUT in the workspace status and
 * lets the kernel return, so that a lost block cannot hang the GPU.  This
 * call runs that same wait in a two-block kernel: block 1 waits for a flag
 * that block 0 publishes when publish = 1 and never publishes when
 * publish = 0.
 *   ws: device workspace of at least MDLS_WAIT_CHECK_WORKSPACE bytes,
 *   256-byte aligned (its header and the flag are cleared by the call).
 *   limit_ns: the wait's limit, 1e3 .. 1e10 ns (the library's own calls use
 *   2 s).
 * Afterwards mdls_read_status(ws) gives MDLS_ERR_TIMEOUT (publish = 0, after
 * about limit_ns) or MDLS_OK (publish = 1).  Returns MDLS_OK,
 * MDLS_ERR_WORKSPACE, MDLS_ERR_ARG or MDLS_ERR_CUDA.
 */
#define MDLS_WAIT_CHECK_WORKSPACE 512
int mdls_wait_check(void* ws, size_t ws_bytes, uint64_t limit_ns, int publish, void* stream);

/*
 * mdls_read_status -- waits for `stream`, then copies the device status word
 * of the workspace `ws` (MDLS_OK, MDLS_ERR_SINGULAR or MDLS_ERR_TIMEOUT) to
 * *status.  Returns MDLS_OK or MDLS_ERR_CUDA.
 */
int mdls_read_status(const void* ws, int* status, void* stream);

/*
 * Per-stage timing, as the paper measures its kernels (Section 4.2: every
 * launch timed with cudaEventElapsedTime, sums reported per stage of
 * Algorithms 1 and 2).  Launches are always counted per stage.
 * mdls_profile_enable(1) additionally records a CUDA event pair around every
 * launch on its stream.  mdls_profile_read() waits for those events, writes
 * up to `cap` per-stage sums (milliseconds; NULL to skip) and launch counts
 * (NULL to skip), resets them, and returns the number of stages (or a
 * negative status).  Stage indices: 0 panel, 1 compute W, 2 trailing update,
 * 3 Q accumulation, 4 invert diagonal tiles, 5 multiply with inverses,
 * 6 back substitution updates, 7 other, 8 refinement; mdls_stage_name()
 * names them.
 * The profiler is process-wide; timing is meant for one thread at a time.
 */
void mdls_profile_enable(int on);
int mdls_profile_read(double* ms, int64_t* launches, int cap);
const char* mdls_stage_name(int stage);

#ifdef __cplusplus
}
#endif
#endif /* MDLS_H */
