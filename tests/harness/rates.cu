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
// probe_tcgen05() gives the cycles per tcgen05.mma kind::f16 (M = 128) of
// the split products' operand layout at N = 16, 64, 128, 256.
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

// tcgen05.mma (kind::f16, bf16 operands, fp32 accumulators in tensor memory,
// cta_group::1, M = 128) issued back to back by one thread per block, one
// block per SM, A and B read from shared memory in the 32-byte-swizzled
// K-major layout of the split products, rotating over 8 A tiles and 8 B
// regions so that every MMA reads fresh operands.  The issuing thread waits
// for completion on an mbarrier (bounded: 2 s of the global timer) and
// records clock64 cycles; every block frees its tensor memory before it
// returns.
static __device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
static __device__ __forceinline__ unsigned long long tc_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ __forceinline__ uint64_t tc_desc(uint32_t a) {
    return (uint64_t)((a >> 4) & 0x3FFF) | (1ull << 16) | ((uint64_t)16 << 32) | (1ull << 46) | (6ull << 61);
}

static __global__ void __launch_bounds__(128, 1) tcgen05_rate_kernel(int R, int N, unsigned long long* cycles) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;          // 8 tiles of 128 x 32 bytes
    unsigned char* B = sm + 32768;  // 8 regions of 256 x 32 bytes
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 98304);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + 98304 + 16);
    for (int i = threadIdx.x; i < 98304 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0x3f803f80u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tc_saddr(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(slot);
    if (threadIdx.x == 0) {
        const uint64_t ad = tc_desc(tc_saddr(A)), bd = tc_desc(tc_saddr(B));
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
        const unsigned long long t0 = clock64();
        for (int r = 0; r < R; ++r) {
            const uint64_t rot = (uint64_t)(r & 7);
            const uint32_t acc = r > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad + rot * 256), "l"(bd + rot * 512), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_saddr(bar))
                     : "memory");
        uint32_t ok = 0;
        const unsigned long long g0 = tc_gtimer();
        while (!ok && tc_gtimer() - g0 < 2000000000ull)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(tc_saddr(bar))
                : "memory");
        cycles[blockIdx.x] = ok ? clock64() - t0 : 0ull;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// Cycles per tcgen05.mma (the slowest block's average over R = 4096) for
// N = 16, 64, 128, 256 in out[0..3]; 0 when a block's wait gave up.
extern "C" int probe_tcgen05(double* out, int nout) {
    int sms = 0;
    if (nout < 4 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return -1;
    const size_t smem = 98304 + 64;
    if (cudaFuncSetAttribute(tcgen05_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long) * sms) != cudaSuccess) return -1;
    unsigned long long h[1024];
    const int Ns[4] = {16, 64, 128, 256};
    const int R = 4096;
    int rc = 0;
    for (int k = 0; k < 4 && rc == 0; ++k) {
        for (int w = 0; w < 2; ++w) tcgen05_rate_kernel<<<sms, 128, smem>>>(R, Ns[k], d);
        if (cudaDeviceSynchronize() != cudaSuccess) { rc = -1; break; }
        cudaMemcpy(h, d, sizeof(unsigned long long) * (sms < 1024 ? sms : 1024), cudaMemcpyDeviceToHost);
        unsigned long long mx = 0;
        for (int i = 0; i < sms && i < 1024; ++i) {
            if (h[i] == 0) rc = -2;
            mx = h[i] > mx ? h[i] : mx;
        }
        out[k] = (double)mx / R;
    }
    cudaFree(d);
    return rc;
}

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
