// Micro-benchmarks of the arithmetic and atomic ceilings that bound the projection kernels on one
// GPU: FP32 FMA, FP64 FMA, INT32 ALU (add/xor) and INT32 multiply-add issue rates, and the
// throughput of scattered FP64 reductions into a grid-sized array (the flush of the projection
// adds one FP64 value per (simplex, cell) piece with a reduction to L2).
//
// Every kernel runs a fixed, bounded loop over registers (no memory traffic besides one store of
// the result so the work is kept) or, for the reductions, a bounded loop of in-range indices.
// Built by bench_peaks.py with nvcc into a small shared library of its own; C entry points take
// plain sizes and return the elapsed milliseconds measured with CUDA events (negative on error).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread (hides the pipe latency)

__global__ void __launch_bounds__(256) k_fma_f32(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma_f64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// integer ALU: one add and one xor per step and chain (two instructions)
__global__ void __launch_bounds__(256) k_alu_i32(unsigned* out, int iters, unsigned a, unsigned b) {
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 7u + (unsigned)c;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = (x[c] + a) ^ b;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// integer multiply-add
__global__ void __launch_bounds__(256) k_imad_i32(unsigned* out, int iters, unsigned a, unsigned b) {
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 5u + (unsigned)c;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Scattered FP64 reductions: thread t adds to cells of a grid of n doubles.  `run` consecutive
// cells per warp lane group (run = 1: every lane an independent pseudo-random cell; run = 32: a
// warp covers 32 consecutive cells, the pattern of the flush of one box row).  Every index is
// reduced modulo n, so every access is in range.
__global__ void __launch_bounds__(256) k_red_f64(double* grid, unsigned long long n, int per_thread, int run) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long h = (t / (unsigned long long)run) * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
#pragma unroll 1
    for (int i = 0; i < per_thread; ++i) {
        h ^= h >> 29;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 32;
        const unsigned long long cell = (h + (run > 1 ? (lane % (unsigned)run) : 0u)) % n;
        atomicAdd(grid + cell, 1.0);
    }
}

template <typename F>
float time_it(F launch, int reps) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.f;
    launch();  // warm-up
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.f;
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1.f;
    return ms / (float)reps;
}

}  // namespace

extern "C" {

// kind: 0 FP32 FMA, 1 FP64 FMA, 2 INT32 add+xor, 3 INT32 multiply-add.  Launches `blocks` blocks of
// 256 threads, each thread `iters` loop trips of 16 (kind 2: 8) steps on kChains chains.  Returns
// the milliseconds of one launch (mean of `reps`), or a negative value on a CUDA error.
// *ops_per_launch receives the arithmetic operations of one launch (an FMA counts 2, kind 2 counts
// its add and xor as 2, kind 3 its multiply-add as 2).
float peaks_alu(int kind, int blocks, int iters, int reps, double* ops_per_launch) {
    const long long threads = (long long)blocks * 256;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)threads * 8) != cudaSuccess) return -1.f;
    float ms = -1.f;
    const double steps = (double)threads * iters * (kind == 2 ? 8 : 16) * kChains;
    *ops_per_launch = 2.0 * steps;
    switch (kind) {
        case 0:
            ms = time_it([&] { k_fma_f32<<<blocks, 256>>>((float*)buf, iters, 0.999999f, 1e-7f); }, reps);
            break;
        case 1:
            ms = time_it([&] { k_fma_f64<<<blocks, 256>>>((double*)buf, iters, 0.999999, 1e-7); }, reps);
            break;
        case 2:
            ms = time_it([&] { k_alu_i32<<<blocks, 256>>>((unsigned*)buf, iters, 0x9E3779B9u, 0x7F4A7C15u); }, reps);
            break;
        case 3:
            ms = time_it([&] { k_imad_i32<<<blocks, 256>>>((unsigned*)buf, iters, 1664525u, 1013904223u); }, reps);
            break;
        default:
            break;
    }
    cudaFree(buf);
    return ms;
}

// Scattered FP64 reductions into a zeroed grid of n_cells doubles: blocks x 256 threads, each
// `per_thread` reductions; `run` as in k_red_f64.  Returns the milliseconds of one launch.
float peaks_red_f64(long long n_cells, int blocks, int per_thread, int run, int reps) {
    if (n_cells < 1 || run < 1 || run > 32) return -1.f;
    double* grid = nullptr;
    if (cudaMalloc(&grid, (size_t)n_cells * sizeof(double)) != cudaSuccess) return -1.f;
    cudaMemset(grid, 0, (size_t)n_cells * sizeof(double));
    const float ms = time_it([&] { k_red_f64<<<blocks, 256>>>(grid, (unsigned long long)n_cells, per_thread, run); },
                             reps);
    cudaFree(grid);
    return ms;
}

int peaks_device_sms(void) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    return n;
}

}  // extern "C"
