// Batched least squares (mdls_batched_*): many independent problems of mixed
// shape and precision solved by ONE launch of a CUDA graph.
//
// mdls_batched_plan() picks a tile per problem (the autotuner below, or the
// caller's), captures every problem's launch sequence into one graph -- the
// problems spread over parallel branches, largest first, each branch fed the
// next problem when it has the least estimated work -- and instantiates it.
// Each problem uses the single-block panel (integer digits, one block), so
// no problem ever waits on blocks of its own that the others keep off the
// SMs.  mdls_batched_launch() replays the graph on a stream.
//
// Autotuner: for every (precision, n-bucket) class not seen before (n
// buckets are powers of two), the first problem of that class is solved with
// each candidate tile (8, 16, 32 up to n = 64; 8 .. 64 up to n = 256;
// 16 .. 128 beyond) x (mode plain, split) on the problem's own buffers, timed
// with CUDA events after one warm-up (median of three), and the fastest pair
// is kept in a process-wide table for every later problem of the class.
// Both modes meet the same accuracy; split runs the WY products on the tensor
// cores and pays for digit conversions, which small problems may not repay.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/mdls.h"
#include "layout.h"
#include "profile.h"

namespace mdls {
int ls_entry_p2(int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*,
                int64_t, int, int, void*, cudaStream_t, bool);
int ls_entry_p4(int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*,
                int64_t, int, int, void*, cudaStream_t, bool);
int ls_entry_p8(int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*,
                int64_t, int, int, void*, cudaStream_t, bool);
}  // namespace mdls

using namespace mdls;

namespace {

const int kModes[] = {MDLS_MODE_PLAIN, MDLS_MODE_SPLIT};
constexpr int kBranches = 128;  // the device runs at most 128 kernels at once
constexpr int kTuneReps = 3;    // timings per candidate (median)

// Candidate tiles of the autotuner by problem width.
struct Cands {
    int t[4];
    int count;
};
Cands candidates(int64_t n) {
    if (n <= 64) return Cands{{8, 16, 32, 0}, 3};
    if (n <= 256) return Cands{{8, 16, 32, 64}, 4};
    return Cands{{16, 32, 64, 128}, 4};
}

int solve_one(const mdls_problem& p, int tile, int mode, void* ws, cudaStream_t st) {
    switch (p.prec) {
        case 2: return ls_entry_p2(p.m, p.n, p.A, p.lda, p.psa, p.b, p.psb, p.x, p.psx, tile, mode, ws, st, true);
        case 4: return ls_entry_p4(p.m, p.n, p.A, p.lda, p.psa, p.b, p.psb, p.x, p.psx, tile, mode, ws, st, true);
        default: return ls_entry_p8(p.m, p.n, p.A, p.lda, p.psa, p.b, p.psb, p.x, p.psx, tile, mode, ws, st, true);
    }
}

bool problem_ok(const mdls_problem& p) {
    return (p.prec == 2 || p.prec == 4 || p.prec == 8) && p.n >= 1 && p.m >= p.n && p.A && p.b && p.x &&
           p.lda >= p.m && p.psa >= p.lda * p.n && p.psb >= p.m && p.psx >= p.n && p.tile >= 0 &&
           p.tile <= 256;
}

// Workspace of one problem: the largest over the candidates it may run.
size_t problem_ws(const mdls_problem& p) {
    size_t best = 0;
    for (int mode : kModes) {
        if (p.tile > 0) {
            best = std::max(best, ls_layout(p.prec, p.m, p.n, norm_tile(p.tile, p.n), mode == MDLS_MODE_SPLIT).total);
            continue;
        }
        const Cands cs = candidates(p.n);
        for (int q = 0; q < cs.count; ++q) {
            const int t = norm_tile(cs.t[q], p.n);
            best = std::max(best, ls_layout(p.prec, p.m, p.n, t, mode == MDLS_MODE_SPLIT).total);
        }
    }
    return align256(best);
}

int bucket(int64_t v) {  // powers of two
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= v) ++b;
    return b;
}

std::mutex g_tune_mu;
struct Choice {
    int tile, mode;
};
std::map<std::tuple<int, int, int>, Choice> g_tune;  // (prec, n bucket, fixed tile) -> choice

int heuristic_tile(const mdls_problem& p) {
    const int t = p.n <= 64 ? 16 : (p.n <= 256 ? 32 : 64);
    return norm_tile(t, p.n);
}

Choice autotune(const mdls_problem& p, void* ws, int* rc) {
    cudaStream_t st;
    *rc = MDLS_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        *rc = MDLS_ERR_CUDA;
        return Choice{p.tile > 0 ? norm_tile(p.tile, p.n) : heuristic_tile(p), MDLS_MODE_PLAIN};
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Choice best{p.tile > 0 ? norm_tile(p.tile, p.n) : heuristic_tile(p), MDLS_MODE_PLAIN};
    float best_ms = 1e30f;
    const Cands cs = candidates(p.n);
    for (int mode : kModes) {
        int last = -1;
        for (int q = 0; q < cs.count; ++q) {
            const int t = p.tile > 0 ? norm_tile(p.tile, p.n) : norm_tile(cs.t[q], p.n);
            if (t == last) continue;
            last = t;
            if (solve_one(p, t, mode, ws, st) != MDLS_OK) continue;  // warm-up
            float reps[kTuneReps];
            bool ok = true;
            for (int r = 0; r < kTuneReps && ok; ++r) {
                cudaEventRecord(e0, st);
                ok = solve_one(p, t, mode, ws, st) == MDLS_OK;
                cudaEventRecord(e1, st);
                ok = ok && cudaEventSynchronize(e1) == cudaSuccess &&
                     cudaEventElapsedTime(&reps[r], e0, e1) == cudaSuccess;
            }
            if (!ok) continue;
            std::sort(reps, reps + kTuneReps);
            const float ms = reps[kTuneReps / 2];
            if (ms < best_ms) {
                best_ms = ms;
                best = Choice{t, mode};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    return best;
}

struct Plan {
    std::vector<mdls_problem> probs;
    std::vector<int> tiles, modes;
    std::vector<size_t> ws_off;
    char* ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

extern "C" {

size_t mdls_batched_workspace(const mdls_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (!problem_ok(probs[i])) return 0;
        total += problem_ws(probs[i]);
    }
    return total;
}

int mdls_batched_plan(const mdls_problem* probs, int count, void* ws, size_t ws_bytes, int autotune_tiles,
                      void** plan_out) {
    if (!probs || count < 1 || !plan_out) return MDLS_ERR_ARG;
    *plan_out = nullptr;
    for (int i = 0; i < count; ++i)
        if (!problem_ok(probs[i])) return probs[i].prec == 2 || probs[i].prec == 4 || probs[i].prec == 8
                                              ? MDLS_ERR_ARG
                                              : MDLS_ERR_PREC;
    const size_t need = mdls_batched_workspace(probs, count);
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return MDLS_ERR_WORKSPACE;
    Plan* P = new Plan;
    P->probs.assign(probs, probs + count);
    P->ws = static_cast<char*>(ws);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        P->ws_off.push_back(off);
        off += problem_ws(probs[i]);
    }
    const bool was_timing = profiler_pause();
    // tile and mode of every problem
    int rc = MDLS_OK;
    for (int i = 0; i < count && rc == MDLS_OK; ++i) {
        const mdls_problem& p = P->probs[i];
        Choice ch{p.tile > 0 ? norm_tile(p.tile, p.n) : heuristic_tile(p), MDLS_MODE_PLAIN};
        if (autotune_tiles) {
            const auto key = std::make_tuple(p.prec, bucket(p.n), p.tile);
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                ch = Choice{p.tile > 0 ? norm_tile(p.tile, p.n) : norm_tile(it->second.tile, p.n), it->second.mode};
            } else {
                ch = autotune(p, P->ws + P->ws_off[i], &rc);
                g_tune[key] = ch;
            }
        }
        P->tiles.push_back(ch.tile);
        P->modes.push_back(ch.mode);
    }
    // capture: problems, largest first, onto the least loaded branch
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto cost = [&](int i) {
        const mdls_problem& p = P->probs[i];
        const double pc = p.prec == 2 ? 1.0 : (p.prec == 4 ? 8.0 : 58.0);
        return pc * (double)p.m * (double)p.n * (double)p.n;
    };
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    cudaStream_t s0 = nullptr, br[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    bool capturing = false;
    if (rc == MDLS_OK && cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess) rc = MDLS_ERR_CUDA;
    for (int b = 0; b < kBranches && rc == MDLS_OK; ++b)
        if (cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming) != cudaSuccess)
            rc = MDLS_ERR_CUDA;
    if (rc == MDLS_OK && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) rc = MDLS_ERR_CUDA;
    if (rc == MDLS_OK) {
        if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MDLS_ERR_CUDA;
        else capturing = true;
    }
    if (rc == MDLS_OK && cudaEventRecord(fork, s0) != cudaSuccess) rc = MDLS_ERR_CUDA;
    double load[kBranches] = {};
    bool used[kBranches] = {};
    for (int idx = 0; idx < count && rc == MDLS_OK; ++idx) {
        const int i = order[idx];
        int b = 0;
        for (int q = 1; q < kBranches; ++q)
            if (load[q] < load[b]) b = q;
        if (!used[b]) {
            if (cudaStreamWaitEvent(br[b], fork, 0) != cudaSuccess) { rc = MDLS_ERR_CUDA; break; }
            used[b] = true;
        }
        load[b] += cost(i);
        rc = solve_one(P->probs[i], P->tiles[i], P->modes[i], P->ws + P->ws_off[i], br[b]);
    }
    for (int b = 0; b < kBranches && rc == MDLS_OK; ++b) {
        if (!used[b]) continue;
        if (cudaEventRecord(join[b], br[b]) != cudaSuccess || cudaStreamWaitEvent(s0, join[b], 0) != cudaSuccess)
            rc = MDLS_ERR_CUDA;
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s0, &g);
        if (rc == MDLS_OK && e != cudaSuccess) rc = MDLS_ERR_CUDA;
        if (rc == MDLS_OK) {
            P->graph = g;
            if (cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) rc = MDLS_ERR_CUDA;
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    for (int b = 0; b < kBranches; ++b) {
        if (br[b]) cudaStreamDestroy(br[b]);
        if (join[b]) cudaEventDestroy(join[b]);
    }
    if (fork) cudaEventDestroy(fork);
    if (s0) cudaStreamDestroy(s0);
    profiler_resume(was_timing);
    if (rc != MDLS_OK) {
        mdls_batched_destroy(P);
        return rc;
    }
    *plan_out = P;
    return MDLS_OK;
}

int mdls_batched_launch(void* plan, void* stream) {
    Plan* P = static_cast<Plan*>(plan);
    if (!P || !P->exec) return MDLS_ERR_ARG;
    // every problem's workspace header (status word) starts at zero
    return cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MDLS_OK : MDLS_ERR_CUDA;
}

int mdls_batched_status(void* plan, int* status, void* stream) {
    Plan* P = static_cast<Plan*>(plan);
    if (!P || !status) return MDLS_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MDLS_ERR_CUDA;
    for (size_t i = 0; i < P->probs.size(); ++i)
        if (cudaMemcpy(&status[i], P->ws + P->ws_off[i], sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MDLS_ERR_CUDA;
    return MDLS_OK;
}

int mdls_batched_tiles(void* plan, int* tiles) {
    Plan* P = static_cast<Plan*>(plan);
    if (!P || !tiles) return MDLS_ERR_ARG;
    for (size_t i = 0; i < P->tiles.size(); ++i) tiles[i] = P->tiles[i];
    return MDLS_OK;
}

int mdls_batched_modes(void* plan, int* modes) {
    Plan* P = static_cast<Plan*>(plan);
    if (!P || !modes) return MDLS_ERR_ARG;
    for (size_t i = 0; i < P->modes.size(); ++i) modes[i] = P->modes[i];
    return MDLS_OK;
}

void mdls_batched_destroy(void* plan) {
    Plan* P = static_cast<Plan*>(plan);
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mdls_lstsq_batched: the problem array and the per-problem status live on
// the device.  The array is read back to plan (a synchronising copy); plans
// are kept in a small cache keyed by the array's contents, the workspace and
// the count, so repeated calls on the same batch replay the same graph.
// ---------------------------------------------------------------------------
namespace {

struct CachedPlan {
    std::vector<unsigned char> key;
    void* ws;
    int dev;
    Plan* plan;
    uint64_t* offs;  // device copy of the per-problem workspace offsets (in ws)
};
std::mutex g_cache_mu;
std::vector<CachedPlan> g_cache;  // most recent last
constexpr size_t kCacheCap = 16;

__global__ void batched_status_kernel(const char* ws, const uint64_t* offs, int count, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) status[i] = *reinterpret_cast<const int*>(ws + offs[i]);
}

size_t offsets_at(size_t plan_bytes) { return align256(plan_bytes); }

}  // namespace

extern "C" size_t mdls_lstsq_batched_workspace(const mdls_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    std::vector<mdls_problem> h((size_t)count);
    if (cudaMemcpy(h.data(), probs, sizeof(mdls_problem) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess)
        return 0;
    const size_t need = mdls_batched_workspace(h.data(), count);
    if (need == 0) return 0;
    return offsets_at(need) + align256(sizeof(uint64_t) * (size_t)count);
}

extern "C" int mdls_lstsq_batched(const mdls_problem* probs, int count, void* ws, size_t ws_bytes, int* status,
                                  void* stream) {
    if (!probs || count < 1 || !status) return MDLS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<mdls_problem> h((size_t)count);
    if (cudaMemcpyAsync(h.data(), probs, sizeof(mdls_problem) * (size_t)count, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MDLS_ERR_CUDA;
    for (int i = 0; i < count; ++i)
        if (!problem_ok(h[i])) return (h[i].prec == 2 || h[i].prec == 4 || h[i].prec == 8) ? MDLS_ERR_ARG : MDLS_ERR_PREC;
    const size_t plan_bytes = mdls_batched_workspace(h.data(), count);
    const size_t need = offsets_at(plan_bytes) + align256(sizeof(uint64_t) * (size_t)count);
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return MDLS_ERR_WORKSPACE;
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<unsigned char> key(reinterpret_cast<const unsigned char*>(h.data()),
                                   reinterpret_cast<const unsigned char*>(h.data()) + sizeof(mdls_problem) * h.size());
    std::lock_guard<std::mutex> g(g_cache_mu);
    Plan* P = nullptr;
    uint64_t* offs = nullptr;
    for (size_t c = 0; c < g_cache.size(); ++c) {
        if (g_cache[c].ws == ws && g_cache[c].dev == dev && g_cache[c].key == key) {
            CachedPlan hit = g_cache[c];
            g_cache.erase(g_cache.begin() + (long)c);
            g_cache.push_back(hit);
            P = hit.plan;
            offs = hit.offs;
            break;
        }
    }
    if (!P) {
        void* handle = nullptr;
        const int rc = mdls_batched_plan(h.data(), count, ws, plan_bytes, 1, &handle);
        if (rc != MDLS_OK) return rc;
        P = static_cast<Plan*>(handle);
        offs = reinterpret_cast<uint64_t*>(static_cast<char*>(ws) + offsets_at(plan_bytes));
        std::vector<uint64_t> ho(P->ws_off.begin(), P->ws_off.end());
        if (cudaMemcpy(offs, ho.data(), sizeof(uint64_t) * ho.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            mdls_batched_destroy(P);
            return MDLS_ERR_CUDA;
        }
        if (g_cache.size() >= kCacheCap) {
            mdls_batched_destroy(g_cache.front().plan);
            g_cache.erase(g_cache.begin());
        }
        g_cache.push_back(CachedPlan{std::move(key), ws, dev, P, offs});
    }
    if (cudaGraphLaunch(P->exec, st) != cudaSuccess) return MDLS_ERR_CUDA;
    batched_status_kernel<<<(count + 127) / 128, 128, 0, st>>>(P->ws, offs, count, status);
    return cudaGetLastError() == cudaSuccess ? MDLS_OK : MDLS_ERR_CUDA;
}
