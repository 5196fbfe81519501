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

// The sum-check pair primitive of the product-weighted waves: per step two
// multiply-adds into 128-bit accumulators and one lazy fold (3 products).
template <int CH>
__global__ void __launch_bounds__(256) k_pair_rate(u64 iters, u64 *sink)
{
    u64 x[CH], y[CH], w[CH];
    const u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        x[c] = (t * 0x9E3779B97F4A7C15ull + c) & FP_P;
        y[c] = ((t + 7) * 0xBF58476D1CE4E5B9ull + 3 * c) & FP_P;
        w[c] = ((t + 11) * 0x94D049BB133111EBull + 5 * c) & FP_P;
    }
    u32 r0, r1;
    limbs31(0x123456789ABCDEull + t, r0, r1);
    acc128 a0, a1;
    acc_zero(a0);
    acc_zero(a1);
    u64 s = 0;
    for (u64 k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            mac(a0, w[c], x[c]);
            mac(a1, w[c], y[c]);
            const u64 f = wfold(x[c], y[c], r0, r1);
            y[c] = x[c];
            x[c] = f;
        }
        if ((k & 3) == 3) {
            s += acc_red(a0) + acc_red(a1);
            acc_zero(a0);
            acc_zero(a1);
        }
    }
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    if (s == 0x12345) sink[0] = s;
}

float run_field_mul_rate(int variant, u64 iters, int blocks, int threads, u64 *sink)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&](u64 n) {
        if (variant == 0) k_mul_rate<0, 8><<<blocks, threads>>>(n, sink);
        else if (variant == 1) k_mul_rate<1, 8><<<blocks, threads>>>(n, sink);
        else k_pair_rate<4><<<blocks, threads>>>(n, sink);
    };
    run(iters / 8 + 1);  // warm-up
    cudaEventRecord(e0);
    run(iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}
