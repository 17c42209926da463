// Throughput probes of the arithmetic pipes the multiple-double path can use
// on GB300: FP64 (DFMA, DADD), FP32 FFMA, INT32 IMAD, and the legacy warp
// matrix instructions mma.sync for bf16 (HMMA), int8 (IMMA) and f64 (DMMA).
// Every kernel runs 8 independent dependency chains per thread (4 per warp
// for the matrix instructions) so that issue, not latency, bounds it, over a
// grid of 16 blocks of 256 threads per SM.  probe_rates() times each kernel
// with CUDA events and writes operations per second:
//   out[0] DFMA (FP64 instructions/s), out[1] DADD, out[2] FFMA, out[3] IMAD,
//   out[4] HMMA bf16 m16n8k16 (flop/s), out[5] IMMA s8 m16n8k32 (op/s),
//   out[6] DMMA f64 m8n8k4 (flop/s).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kIters = 4096;

__global__ void dfma_kernel(double* out, double s) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3 + q;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __fma_rn(a[q], s, 0.5);
    }
    double t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void dadd_kernel(double* out, double s) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3 + q;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __dadd_rn(a[q], s);
    }
    double t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void ffma_kernel(double* out, float s) {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3f + q;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __fmaf_rn(a[q], s, 0.5f);
    }
    float t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void imad_kernel(double* out, unsigned s) {
    unsigned a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x + q;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = a[q] * s + 7u;
    }
    unsigned t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t ^= a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void hmma_kernel(double* out, uint32_t seed) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = 0x3f803f80u ^ (seed * (q + 1) & 0x00010001u);  // bf16 pairs near 1
#pragma unroll
    for (int q = 0; q < 2; ++q) b[q] = 0x3f803f80u;
    float c[4][4] = {};
    for (int i = 0; i < kIters / 4; ++i) {
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(c[ch][0]), "+f"(c[ch][1]), "+f"(c[ch][2]), "+f"(c[ch][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float t = 0;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
#pragma unroll
        for (int q = 0; q < 4; ++q) t += c[ch][q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void imma_kernel(double* out, uint32_t seed) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = 0x01010101u ^ (seed * (q + 1) & 0x01000100u);
#pragma unroll
    for (int q = 0; q < 2; ++q) b[q] = 0x01010101u;
    int c[4][4] = {};
    for (int i = 0; i < kIters / 4; ++i) {
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+r"(c[ch][0]), "+r"(c[ch][1]), "+r"(c[ch][2]), "+r"(c[ch][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int t = 0;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
#pragma unroll
        for (int q = 0; q < 4; ++q) t ^= c[ch][q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void dmma_kernel(double* out, double s) {
    const double a = 1.0 + s * threadIdx.x, b = 0.5;
    double c[4][2] = {};
    for (int i = 0; i < kIters / 4; ++i) {
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[ch][0]), "+d"(c[ch][1])
                         : "d"(a), "d"(b));
    }
    double t = 0;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) t += c[ch][0] + c[ch][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

extern "C" int probe_rates(double* out, int nout) {
    if (nout < 7) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 16, threads = 256;
    const double nthreads = (double)blocks * threads;
    const double nwarps = nthreads / 32;
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto launch) {
        launch();  // warm-up
        cudaEventRecord(e0);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.0 / 1e3;
    };
    double sec;
    sec = timed([&] { dfma_kernel<<<blocks, threads>>>(buf, 0.999); });
    out[0] = nthreads * kIters * 8 / sec;
    sec = timed([&] { dadd_kernel<<<blocks, threads>>>(buf, 1e-9); });
    out[1] = nthreads * kIters * 8 / sec;
    sec = timed([&] { ffma_kernel<<<blocks, threads>>>(buf, 0.999f); });
    out[2] = nthreads * kIters * 8 / sec;
    sec = timed([&] { imad_kernel<<<blocks, threads>>>(buf, 3u); });
    out[3] = nthreads * kIters * 8 / sec;
    sec = timed([&] { hmma_kernel<<<blocks, threads>>>(buf, 12345u); });
    out[4] = nwarps * (kIters / 4) * 4 * (2.0 * 16 * 8 * 16) / sec;
    sec = timed([&] { imma_kernel<<<blocks, threads>>>(buf, 12345u); });
    out[5] = nwarps * (kIters / 4) * 4 * (2.0 * 16 * 8 * 32) / sec;
    sec = timed([&] { dmma_kernel<<<blocks, threads>>>(buf, 1e-6); });
    out[6] = nwarps * (kIters / 4) * 4 * (2.0 * 8 * 8 * 4) / sec;
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return err == cudaSuccess ? 0 : -3;
}
