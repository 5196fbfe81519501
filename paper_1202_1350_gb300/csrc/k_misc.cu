// k_misc.cu -- field arithmetic check kernel and the field-multiply issue-rate
// microbenchmark that gives the integer-ALU roofline denominator.
#include <cuda_runtime.h>

#include <atomic>

#include "plan.h"

namespace {
std::atomic<int> g_sms[64];
}

int device_sms()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int sms = g_sms[dev].load(std::memory_order_relaxed);
    if (sms > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
    g_sms[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

// Grid for a grid-stride loop over n items with `threads` per CTA: one CTA
// per `threads` items, at most `per_sm` CTAs per SM of the current device.
unsigned grid_for_items(u64 n, unsigned threads, unsigned per_sm)
{
    u64 b = (n + threads - 1) / threads;
    const u64 cap = (u64)device_sms() * per_sm;
    if (b > cap) b = cap;
    return b ? (unsigned)b : 1u;
}

__global__ void k_field_mul(const u64 *a, const u64 *b, u64 *out, u64 n)
{
    for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x)
        out[k] = f_mul(a[k], b[k]);
}

void launch_field_mul(const u64 *a, const u64 *b, u64 *out, u64 n, cudaStream_t st)
{
    k_field_mul<<<grid_for_items(n, 256, 8), 256, 0, st>>>(a, b, out, n);
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
// CH independent pairs per thread; MINB resident CTAs per SM the register
// allocation is sized for.
template <int CH, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pair_rate(u64 iters, u64 *sink)
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

// 32-bit integer multiply-add issue rate: CH independent chains
// x <- x y + c per thread (one multiply-add each).
template <int CH>
__global__ void __launch_bounds__(256) k_imad_rate(u64 iters, u64 *sink)
{
    u32 x[CH];
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 y = 0x9E3779B9u ^ t;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + (u32)c;
    for (u64 k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < CH; c++) asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y), "r"((u32)(2 * c + 1)));
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    if (s == 0x12345u) sink[0] = s;
}

// Exact 64x64 -> 128-bit multiply-accumulate rate (the `mac` of the sum-check
// waves): CH independent accumulators per thread.
template <int CH>
__global__ void __launch_bounds__(256) k_mac_rate(u64 iters, u64 *sink)
{
    acc128 a[CH];
    u64 x[CH];
    const u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    const u64 y = (t * 0xBF58476D1CE4E5B9ull) & FP_P;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        acc_zero(a[c]);
        x[c] = (t * 0x9E3779B97F4A7C15ull + c) & FP_P;
    }
    for (u64 k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < CH; c++) mac(a[c], x[c], y);
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= a[c].lo ^ a[c].hi;
    if (s == 0x12345) sink[0] = s;
}

namespace {

// One microbenchmark configuration: the kernel, and the units (products or
// multiply-adds) one thread does per iteration.
struct RateKernel {
    void (*fn)(u64, u64 *);
    double units_per_iter;
};

// Time `fn` over a grid of exactly one wave (every SM holding as many CTAs
// of 256 threads as fit), after a shorter warm-up launch; returns units per
// second, or a negative value on a CUDA error.
double time_rate_kernel(const RateKernel &rk, u64 iters, int sms, u64 *sink)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk.fn, 256, 0) != cudaSuccess || per_sm <= 0)
        return -1.0;
    const int blocks = sms * per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    rk.fn<<<blocks, 256>>>(iters / 8 + 1, sink);  // warm-up
    cudaEventRecord(e0);
    rk.fn<<<blocks, 256>>>(iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    return double(blocks) * 256.0 * rk.units_per_iter * double(iters) / (ms * 1e-3);
}

}  // namespace

double run_field_mul_rate(int variant, u64 iters, int sms, u64 *sink)
{
    // variant 2 (the roofline denominator) is the best of several chain counts
    // and register budgets, so that neither occupancy nor a tail wave caps it
    static const RateKernel pair[] = {
        {k_pair_rate<2, 5>, 6.0}, {k_pair_rate<2, 4>, 6.0}, {k_pair_rate<4, 4>, 12.0},
        {k_pair_rate<4, 3>, 12.0}, {k_pair_rate<8, 2>, 24.0},
    };
    switch (variant) {
    case 0: return time_rate_kernel({k_mul_rate<0, 8>, 8.0}, iters, sms, sink);
    case 1: return time_rate_kernel({k_mul_rate<1, 8>, 8.0}, iters, sms, sink);
    case 2: {
        double best = -1.0;
        for (const RateKernel &rk : pair) {
            const double r = time_rate_kernel(rk, iters, sms, sink);
            if (r < 0) return r;
            if (r > best) best = r;
        }
        return best;
    }
    case 3: return time_rate_kernel({k_imad_rate<8>, 8.0}, 4 * iters, sms, sink);
    case 4: return time_rate_kernel({k_mac_rate<8>, 8.0}, iters, sms, sink);
    default: return -1.0;
    }
}
