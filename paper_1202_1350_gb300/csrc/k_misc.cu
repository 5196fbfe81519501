// k_misc.cu -- field arithmetic check kernel and the field-multiply issue-rate
// microbenchmark that gives the integer-ALU roofline denominator.
#include <cuda_runtime.h>
#include "plan.h"

__global__ void k_field_mul(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x)
        out[k] = f_mul(a[k], b[k]);
}

void launch_field_mul(const u64 *a, const u64 *b, u64 *out, u64 n, cudaStream_t st)
{
    u64 blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks == 0) blocks = 1;
    k_field_mul<<<(unsigned)blocks, 256, 0, st>>>(a, b, out, n);
}

// Each thread runs CH independent chains x <- x * y + c (one product and one
// addition per step, the pattern of a fold); the products per second over the
// whole grid is the sustained field-multiply rate.
template <int VARIANT, int CH>
__global__ void __launch_bounds__(256) k_mul_rate(u64 iters, u64 *sink)
{
    u64 x[CH], y[CH];
    const u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        x[c] = (t * 0x9E3779B97F4A7C15ull + c) & FP_P;
        y[c] = ((t + 7) * 0xBF58476D1CE4E5B9ull + 3 * c) & FP_P;
        if (x[c] == FP_P) x[c] = 1;
        if (y[c] == FP_P) y[c] = 2;
    }
    for (u64 k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const u64 m = VARIANT == 0 ? f_mul(x[c], y[c]) : f_mul_wide(x[c], y[c]);
            x[c] = f_add(m, y[c]);
        }
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    if (s == 0x12345) sink[0] = s;  // keeps the chains alive
}

float run_field_mul_rate(int variant, u64 iters, int blocks, int threads, u64 *sink)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // warm-up
    if (variant == 0) k_mul_rate<0, 8><<<blocks, threads>>>(iters / 8 + 1, sink);
    else k_mul_rate<1, 8><<<blocks, threads>>>(iters / 8 + 1, sink);
    cudaEventRecord(e0);
    if (variant == 0) k_mul_rate<0, 8><<<blocks, threads>>>(iters, sink);
    else k_mul_rate<1, 8><<<blocks, threads>>>(iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}
