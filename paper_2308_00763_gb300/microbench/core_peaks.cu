// core_peaks.cu -- measured CUDA-core throughput of the GPU the filter runs on.
//
// The step kernel uses no tensor cores: its work is integer arithmetic (Philox), FP32 /
// FP64 / half2 arithmetic, special-function instructions (log, sqrt, sin/cos, exp) and
// shared-memory traffic.  This program measures the throughput of each of those units
// with long chains of independent instructions, so that the step's pipe utilisation can
// be set against measured peaks (the paper's own analysis is per pipe: its Sec. V reads
// the FP16 and XU pipe utilisation of its kernels from Nsight Compute).
//
// Each kernel runs `kChains` independent dependency chains per thread for `iters` rounds
// over a grid of (SMs x 8) CTAs of 256 threads; the result is folded into one word that is
// stored only when an impossible value appears, so nothing is optimised away.  Timing:
// CUDA events on one stream, best of `reps` launches after a warm-up launch.  Nothing
// changes clocks or any other device setting.
//
// Output: one JSON object on stdout, rates in operations (or thread instructions) per second.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#define CK(x)                                                                             \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) {                                                          \
            fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, cudaGetErrorString(e_));   \
            exit(1);                                                                      \
        }                                                                                 \
    } while (0)

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kUnroll = 16;

// FP32 fused multiply-add: 2 flops per instruction.
__global__ void k_ffma(int iters, float a, float b, uint32_t *sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.2345f) sink[0] = __float_as_uint(s);
}

// half2 fused multiply-add: 4 flops per instruction.
__global__ void k_hfma2(int iters, float a, float b, uint32_t *sink) {
    __half2 v[kChains];
    const __half2 ha = __float2half2_rn(a), hb = __float2half2_rn(b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __float2half2_rn(threadIdx.x * 1e-3f + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __hfma2(v[c], ha, hb);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += __low2float(v[c]) + __high2float(v[c]);
    if (s == -1.2345f) sink[0] = __float_as_uint(s);
}

// bfloat16x2 fused multiply-add: 4 flops per instruction.
__global__ void k_bfma2(int iters, float a, float b, uint32_t *sink) {
    __nv_bfloat162 v[kChains];
    const __nv_bfloat162 ha = __float2bfloat162_rn(a), hb = __float2bfloat162_rn(b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __float2bfloat162_rn(threadIdx.x * 1e-3f + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __hfma2(v[c], ha, hb);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += __low2float(v[c]) + __high2float(v[c]);
    if (s == -1.2345f) sink[0] = __float_as_uint(s);
}

// FP64 fused multiply-add: 2 flops per instruction.
__global__ void k_dfma(int iters, double a, double b, uint32_t *sink) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.2345) sink[0] = static_cast<uint32_t>(__double2loint(s));
}

// Special-function unit: ex2.approx (the instruction behind the fast exp of the half
// filters), one per chain step.
__global__ void k_mufu_ex2(int iters, float a, float b, uint32_t *sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = -(threadIdx.x & 7) * 0.01f - c * 0.001f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float r;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[c]));
                v[c] = r * a - b;   // stays in (-1, 0]: ex2 of it lies in (0.5, 1]
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.2345f) sink[0] = __float_as_uint(s);
}

// 32-bit integer multiply (the Philox rounds' mul.lo / mul.hi), one per chain step.
__global__ void k_imad(int iters, uint32_t a, uint32_t b, uint32_t *sink) {
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 2654435761u + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x12345678u) sink[0] = s;
}

// Integer logic and add (the Philox rounds' other half): v = (v ^ a) + b per chain step,
// two thread instructions (a logic and an add; neither folds across steps).
__global__ void k_lop3(int iters, uint32_t a, uint32_t b, uint32_t *sink) {
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 2654435761u + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = (v[c] ^ a) + b;
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x12345678u) sink[0] = s;
}

// Shared-memory loads (32-bit, conflict-free), one per chain step.
__global__ void k_lds(int iters, uint32_t a, uint32_t b, uint32_t *sink) {
    __shared__ uint32_t buf[kThreads * 2];
    for (int i = threadIdx.x; i < kThreads * 2; i += kThreads) buf[i] = (i * a + b) & (kThreads - 1);
    __syncthreads();
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (threadIdx.x + c * 32) & (kThreads - 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = buf[v[c]];
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x12345678u) sink[0] = s;
}

template <typename F>
double best_ms(F launch, int reps, cudaStream_t st) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch();   // warm-up
    CK(cudaStreamSynchronize(st));
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(a, st));
        launch();
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) best = ms;
    }
    CK(cudaGetLastError());
    CK(cudaEventDestroy(a));
    CK(cudaEventDestroy(b));
    return best;
}

int main(int argc, char **argv) {
    const int reps = argc > 1 ? atoi(argv[1]) : 5;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, dev));
    const int sms = p.multiProcessorCount;
    const int grid = sms * 8;
    uint32_t *sink = nullptr;
    CK(cudaMalloc(&sink, 16));
    cudaStream_t st;
    CK(cudaStreamCreate(&st));
    const double threads = static_cast<double>(grid) * kThreads;
    const double per_thread = static_cast<double>(kChains) * kUnroll;   // instructions per iteration

    struct Row { const char *name; double ops_per_instr; int iters; double ms; };
    Row rows[] = {{"ffma", 2.0, 4096, 0}, {"hfma2", 4.0, 4096, 0}, {"bf16x2_fma", 4.0, 4096, 0},
                  {"dfma", 2.0, 64, 0},   {"mufu_ex2", 1.0, 512, 0}, {"imad", 1.0, 4096, 0},
                  {"xor_add", 1.0, 2048, 0}, {"lds32", 1.0, 1024, 0}};
    // thread instructions per chain step of each kernel (xor_add: a logic and an add)
    const double instr_per_step[] = {1, 1, 1, 1, 1, 1, 2, 1};
    rows[0].ms = best_ms([&] { k_ffma<<<grid, kThreads, 0, st>>>(rows[0].iters, 0.999f, 1e-4f, sink); }, reps, st);
    rows[1].ms = best_ms([&] { k_hfma2<<<grid, kThreads, 0, st>>>(rows[1].iters, 0.999f, 1e-4f, sink); }, reps, st);
    rows[2].ms = best_ms([&] { k_bfma2<<<grid, kThreads, 0, st>>>(rows[2].iters, 0.999f, 1e-4f, sink); }, reps, st);
    rows[3].ms = best_ms([&] { k_dfma<<<grid, kThreads, 0, st>>>(rows[3].iters, 0.999, 1e-4, sink); }, reps, st);
    rows[4].ms = best_ms([&] { k_mufu_ex2<<<grid, kThreads, 0, st>>>(rows[4].iters, 0.5f, 0.5f, sink); }, reps, st);
    rows[5].ms = best_ms([&] { k_imad<<<grid, kThreads, 0, st>>>(rows[5].iters, 2654435761u, 12345u, sink); }, reps, st);
    rows[6].ms = best_ms([&] { k_lop3<<<grid, kThreads, 0, st>>>(rows[6].iters, 0x9E3779B9u, 0xBB67AE85u, sink); }, reps, st);
    rows[7].ms = best_ms([&] { k_lds<<<grid, kThreads, 0, st>>>(rows[7].iters, 1u, 0u, sink); }, reps, st);

    int clk_khz = 0;
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    printf("{\"device\": \"%s\", \"sms\": %d, \"attr_clock_mhz\": %.0f, \"grid\": %d, \"threads_per_cta\": %d, "
           "\"chains\": %d, \"reps\": %d, \"rates\": {",
           p.name, sms, clk_khz / 1000.0, grid, kThreads, kChains, reps);
    for (int i = 0; i < 8; ++i) {
        const double instr = threads * per_thread * rows[i].iters * instr_per_step[i];
        const double ips = instr / (rows[i].ms * 1e-3);
        printf("%s\"%s\": {\"thread_instructions_per_s\": %.6e, \"ops_per_s\": %.6e, \"ms\": %.4f, "
               "\"per_sm_per_clock_at_attr_clock\": %.3f}",
               i ? ", " : "", rows[i].name, ips, ips * rows[i].ops_per_instr, rows[i].ms,
               ips / (sms * (clk_khz * 1e3)));
    }
    printf("}}\n");
    CK(cudaFree(sink));
    CK(cudaStreamDestroy(st));
    return 0;
}
