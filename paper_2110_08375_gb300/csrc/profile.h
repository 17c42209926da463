// Per-stage launch counters and optional CUDA-event timing (host only).
//
// The paper measures every kernel launch with cudaEventElapsedTime and
// reports the sums per stage of Algorithms 1 and 2 (Section 4.2 and the
// stage rows of its tables).  Each launch site of the library is wrapped in
// a StageScope: the launch is always counted; when timing is enabled an
// event pair is recorded around it on the launching stream.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdls {

enum Stage {
    ST_PANEL = 0,   // "beta, v" + "beta R^T v" + "update R"  (panel kernel)
    ST_W,           // "compute W": Y^T Y, T, W = -Y T
    ST_TRAIL,       // "YWT * C" + "R + YWTC": trailing update
    ST_QACC,        // "Q * WY^T" + "Q + QWY": accumulation of Q
    ST_INV,         // "invert diagonal tiles"
    ST_MULINV,      // "multiply with inverses"
    ST_BSUPD,       // "back substitution" (right-hand side updates)
    ST_OTHER,       // copies, identity, zeroing, elementwise ops
    ST_REFINE,      // refinement: residuals in P limbs, Q^T r and corrections
    ST_COUNT
};

void stage_begin(int stage, cudaStream_t st);
bool profiler_pause();
void profiler_resume(bool on);
void stage_end(int stage, cudaStream_t st);

struct StageScope {
    int stage;
    cudaStream_t st;
    StageScope(int s, cudaStream_t stream) : stage(s), st(stream) { stage_begin(stage, st); }
    ~StageScope() { stage_end(stage, st); }
};

}  // namespace mdls
