// field.cuh -- device arithmetic in F_p, p = 2^61 - 1 (Sec. 6.1 of the paper:
// a Mersenne prime, so reduction is shifts and masks; Sec. 5.1.4: a product
// costs a few machine multiplies).  Every value handled here is canonical,
// i.e. in [0, p).
#pragma once
#include <stdint.h>

typedef uint64_t u64;
typedef unsigned int u32;

#define FP_P 0x1FFFFFFFFFFFFFFFull

__host__ __device__ __forceinline__ u64 f_add(u64 a, u64 b)
{
    u64 s = a + b;  // < 2^62, no wrap
    return s >= FP_P ? s - FP_P : s;
}

__host__ __device__ __forceinline__ u64 f_sub(u64 a, u64 b)
{
    return a >= b ? a - b : a + (FP_P - b);
}

__host__ __device__ __forceinline__ u64 f_neg(u64 a) { return a ? FP_P - a : 0; }

// 2a - b, the value at t = 2 of the line through (0, b) and (1, a).
__host__ __device__ __forceinline__ u64 f_ext2(u64 a1, u64 a0) { return f_sub(f_add(a1, a1), a0); }

// Product with 32-bit limbs.  a = a1 2^32 + a0 with a1, b1 < 2^29 (canonical
// inputs), so
//   a b = a1 b1 2^64 + (a1 b0 + a0 b1) 2^32 + a0 b0,   mid = a1 b0 + a0 b1 < 2^62.
// Using 2^61 = 1 and 2^64 = 8 (mod p):
//   mid 2^32 = (mid >> 29) 2^61 + (mid mod 2^29) 2^32 = (mid >> 29) + (mid mod 2^29) 2^32,
//   a0 b0    = (a0 b0 mod 2^61) + (a0 b0 >> 61).
// The five terms sum to less than 3 2^61 + 2^34 < 2^63; one more fold leaves
// a value below p + 4, and one conditional subtraction makes it canonical.
__device__ __forceinline__ u64 f_mul(u64 a, u64 b)
{
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32);
    const u32 b0 = (u32)b, b1 = (u32)(b >> 32);
    const u64 lo = (u64)a0 * b0;
    const u64 mid = (u64)a1 * b0 + (u64)a0 * b1;
    const u64 hi = (u64)a1 * b1;
    u64 s = (hi << 3) + (mid >> 29) + ((mid & 0x1FFFFFFFull) << 32) + (lo & FP_P) + (lo >> 61);
    s = (s & FP_P) + (s >> 61);
    return s >= FP_P ? s - FP_P : s;
}

// Product with a full 64x64 -> 128 multiply and one Mersenne fold:
// a b = hi 2^64 + lo, (a b) mod 2^61 = lo & p, (a b) >> 61 = (hi << 3) | (lo >> 61);
// both parts are below p because a b <= (p-1)^2 < p 2^61, so one conditional
// subtraction suffices.
__device__ __forceinline__ u64 f_mul_wide(u64 a, u64 b)
{
    const u64 lo = a * b;
    const u64 hi = __umul64hi(a, b);
    u64 s = (lo & FP_P) + ((lo >> 61) | (hi << 3));
    return s >= FP_P ? s - FP_P : s;
}

// Host-side product for plan-time constants (never on the proof path).
static inline u64 h_mul(u64 a, u64 b)
{
    unsigned __int128 x = (unsigned __int128)a * b;
    u64 s = (u64)(x & FP_P) + (u64)(x >> 61);
    return s >= FP_P ? s - FP_P : s;
}

// Sum of a and b where both are canonical: lazy-free add used in reductions.
__device__ __forceinline__ u64 f_add3(u64 a, u64 b, u64 c) { return f_add(f_add(a, b), c); }

// Fermat inverse a^(p-2) (a != 0): square-and-multiply over the bits of p - 2.
__device__ __forceinline__ u64 f_inv(u64 a)
{
    u64 r = 1, b = a;
    u64 e = FP_P - 2;
    while (e) {
        if (e & 1) r = f_mul(r, b);
        b = f_mul(b, b);
        e >>= 1;
    }
    return r;
}

// 1/2 = 2^60 mod p, since 2 * 2^60 = 2^61 = 1.
#define FP_INV2 0x1000000000000000ull

// splitmix64 (Steele, Lea, Flood 2014): output number k (k >= 1) of the
// generator started at `seed` is mix(seed + k * gamma).
__device__ __forceinline__ u64 splitmix64_at(u64 seed, u64 k)
{
    u64 z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Warp-wide field sum (all 32 lanes participate).
__device__ __forceinline__ u64 warp_sum(u64 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = f_add(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---- Lazy arithmetic: values in W = [0, 2^61 + 8) ("weakly reduced"). -------
// Canonical values are in W; only transcript entries must be canonical.

// Any 64-bit x -> W, congruent mod p (2^61 = 1).
__device__ __forceinline__ u64 wred(u64 x) { return (x & FP_P) + (x >> 61); }

// W -> canonical.
__device__ __forceinline__ u64 wcanon(u64 w) { return w >= FP_P ? w - FP_P : w; }

// 128-bit accumulator of products of W values (at most 64 products).
struct acc128 {
    u64 lo, hi;
};

__device__ __forceinline__ void acc_zero(acc128 &a) { a.lo = 0; a.hi = 0; }

// a += x y (exact 128-bit multiply-add).
__device__ __forceinline__ void mac(acc128 &a, u64 x, u64 y)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(a.lo), "+l"(a.hi) : "l"(x), "l"(y));
}

// a += x (x < 2^64).
__device__ __forceinline__ void acc_add(acc128 &a, u64 x)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(a.lo), "+l"(a.hi) : "l"(x));
}

// hi 2^64 + lo -> W: 2^64 = 8 (mod p), and 8 hi = (hi >> 58) 2^61 + (8 hi mod 2^61).
__device__ __forceinline__ u64 acc_red(const acc128 &a)
{
    const u64 t = (a.lo & FP_P) + (a.lo >> 61) + ((a.hi << 3) & FP_P) + (a.hi >> 58);
    return wred(t);
}

// Product of two W values, result in W.
__device__ __forceinline__ u64 wmul(u64 x, u64 y)
{
    acc128 a;
    a.lo = x * y;
    a.hi = __umul64hi(x, y);
    return acc_red(a);
}

// u0 + r (u1 - u0) for u0, u1 in W and canonical r given as 31/30-bit limbs
// r = r1 2^31 + r0.  With d = u1 - u0 + 2p in (0, 2^63) split as d1 2^31 + d0:
//   r d + u0 = r1 d1 2^62 + (r0 d1 + r1 d0) 2^31 + (r0 d0 + u0)
// and 2^62 = 2, M 2^31 = (M >> 30) + (M mod 2^30) 2^31 (mod p).
__device__ __forceinline__ u64 wfold(u64 u0, u64 u1, u32 r0, u32 r1)
{
    const u64 d = u1 + (2 * FP_P) - u0;
    const u32 d0 = (u32)d & 0x7FFFFFFFu, d1 = (u32)(d >> 31);
    const u64 A00 = u0 + (u64)r0 * d0;
    const u64 AM = (u64)r0 * d1 + (u64)r1 * d0;
    const u64 A11 = (u64)r1 * d1;
    const u64 t = (A11 << 1) + (AM >> 30) + ((AM & 0x3FFFFFFFull) << 31) + (A00 & FP_P) + (A00 >> 61);
    return wred(t);
}

// u0 + a d for u0 in W, d < 2^62.6 (a lazy difference u1 + 2p - u0 of W
// values) and canonical a = a1 2^31 + a0: the limb scheme of wfold.
__device__ __forceinline__ u64 wlin1(u64 u0, u64 d, u32 a0, u32 a1)
{
    const u32 d0 = (u32)d & 0x7FFFFFFFu, d1 = (u32)(d >> 31);
    const u64 A00 = u0 + (u64)a0 * d0;
    const u64 AM = (u64)a0 * d1 + (u64)a1 * d0;
    const u64 A11 = (u64)a1 * d1;
    const u64 t = (A11 << 1) + (AM >> 30) + ((AM & 0x3FFFFFFFull) << 31) + (A00 & FP_P) + (A00 >> 61);
    return wred(t);
}

// u0 + a d + b e (d, e < 2^62.6; a, b canonical as 31/30-bit limbs).  Bounds:
// A00 < 2^61 + 8 + 2^63.6; AM < 2 (2^62.6 + 2^61) < 2^64; 2 A11 < 2^63.6;
// the sum t stays below 2^64.
__device__ __forceinline__ u64 wlin2(u64 u0, u64 d, u64 e, u32 a0, u32 a1, u32 b0, u32 b1)
{
    const u32 d0 = (u32)d & 0x7FFFFFFFu, d1 = (u32)(d >> 31);
    const u32 e0 = (u32)e & 0x7FFFFFFFu, e1 = (u32)(e >> 31);
    const u64 A00 = wred(u0 + (u64)a0 * d0) + (u64)b0 * e0;
    const u64 AM = (u64)a0 * d1 + (u64)a1 * d0 + (u64)b0 * e1 + (u64)b1 * e0;
    const u64 A11 = (u64)a1 * d1 + (u64)b1 * e1;
    const u64 t = (A11 << 1) + (AM >> 30) + ((AM & 0x3FFFFFFFull) << 31) + (A00 & FP_P) + (A00 >> 61);
    return wred(t);
}

__device__ __forceinline__ void limbs31(u64 r, u32 &r0, u32 &r1)
{
    r0 = (u32)r & 0x7FFFFFFFu;
    r1 = (u32)(r >> 31);
}

// Inclusive product scan over the warp (lane l gets prod_{j<=l} x_j).
__device__ __forceinline__ u64 warp_scan_mul(u64 x)
{
    const u32 lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (u32)o) x = f_mul(x, y);
    }
    return x;
}

// Inclusive suffix product scan (lane l gets prod_{j>=l} x_j).
__device__ __forceinline__ u64 warp_rscan_mul(u64 x)
{
    const u32 lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_down_sync(0xffffffffu, x, o);
        if (lane + o < 32) x = f_mul(x, y);
    }
    return x;
}

// Product over the warp of one canonical value per lane.
__device__ __forceinline__ u64 warp_prod(u64 x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = f_mul(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Warp-wide sum of one W value per lane -> W (a sum of four W values stays
// below 2^64, so reduce every two steps).
__device__ __forceinline__ u64 warp_wsum(u64 x)
{
    x += __shfl_xor_sync(0xffffffffu, x, 16);
    x += __shfl_xor_sync(0xffffffffu, x, 8);
    x = wred(x);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x = wred(x);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return wred(x);
}

// Warp-wide sums of n records of NV values in W (record q at part[q NV ..]):
// the lanes take every 32nd record, FN_U records' loads in flight per lane
// before any is added (the reductions over hundreds of per-CTA partials are
// load-latency bound).  h[t] (t < NV) = the canonical total of value t, in every lane.
#define FN_U 8
static_assert(FN_U == 8, "warp_record_sums adds its loads in two quarter-sums of four");
template <int NV>
__device__ __forceinline__ void warp_record_sums(const u64 *__restrict__ part, u32 n, u32 lane, u64 *h)
{
    u64 acc[NV];
#pragma unroll
    for (int t = 0; t < NV; t++) acc[t] = 0;
    for (u32 q0 = lane; q0 < n; q0 += 32 * FN_U) {
        u64 x[FN_U][NV];
#pragma unroll
        for (int u = 0; u < FN_U; u++) {
            const u32 q = q0 + 32 * u;
#pragma unroll
            for (int t = 0; t < NV; t++) x[u][t] = q < n ? part[(u64)q * NV + t] : 0;
        }
#pragma unroll
        for (int t = 0; t < NV; t++) {
            // four W values sum below 2^64; wred brings each quarter-sum back to W
            const u64 lo = wred(x[0][t] + x[1][t] + x[2][t] + x[3][t]);
            const u64 hi = wred(x[4][t] + x[5][t] + x[6][t] + x[7][t]);
            acc[t] = wred(acc[t] + lo + hi);
        }
    }
#pragma unroll
    for (int t = 0; t < NV; t++) h[t] = wcanon(warp_wsum(acc[t]));
}

