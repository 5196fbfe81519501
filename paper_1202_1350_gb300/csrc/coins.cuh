// coins.cuh -- the verifier's coins as functions of the seed, for any CTA
// that needs some (Sec. 3.1: the verifier's challenges are random field
// elements; here challenge c is the (c+1)-th accepted draw of splitmix64
// seeded with the proof seed, a draw equal to p being rejected).
#pragma once
#include "plan.h"

// Any rejected draw among the circuit's first nchal draws (whole CTA).
__device__ __forceinline__ bool draws_rejected(const Globals &G)
{
    bool r = false;
    for (u32 c = threadIdx.x; c < G.nchal; c += blockDim.x) r |= ((splitmix64_at(G.seed, (u64)c + 1) >> 3) == FP_P);
    return __syncthreads_or(r) != 0;
}

// Challenge c: the (c+1)-th accepted draw.
__device__ __forceinline__ u64 chal_of(const Globals &G, bool rej, u32 c)
{
    if (!rej) return splitmix64_at(G.seed, (u64)c + 1) >> 3;
    u64 k = 1;
    for (u32 got = 0;;) {
        const u64 x = splitmix64_at(G.seed, k++) >> 3;
        if (x == FP_P) continue;
        if (got == c) return x;
        got++;
    }
}

// Coordinate k of z_layer: z_0 = the first s_0 challenges; z_{i+1} =
// r1 + tau (r2 - r1) of layer i's line (r1, r2: its phase-2/3 challenges).
__device__ __forceinline__ u64 zcoord(const Globals &G, bool rej, u32 layer, u32 k)
{
    if (layer == 0) return chal_of(G, rej, k);
    const LayerDev &L = G.layers[layer - 1];
    const u32 co = L.chal_off, s = L.s, sn = L.sn;
    const u64 tau = chal_of(G, rej, co + s + 2 * sn);
    const u64 r1 = chal_of(G, rej, co + s + k), r2 = chal_of(G, rej, co + s + sn + k);
    return f_add(r1, f_mul(tau, f_sub(r2, r1)));
}

