// k_verify.cu -- verifier kernels (Sec. 2.2, Sec. 3.1, Sec. 4.1.2 of the paper).
//
// The bulk of the verifier's work is its "secret": the input's multilinear
// extension at the final random point, a sum in which every input contributes
// independently (Sec. 4.1.2), computed here as a grid-wide reduction.  The
// round checks of one layer form a short sequential chain; since each layer's
// starting claim can be read off the transcript (q_{i-1}(tau_{i-1})), all
// layers are checked concurrently, one thread per layer.  The accept bit is the
// conjunction of exactly the checks the sequential verifier makes.
#include <cuda_runtime.h>
#include "plan.h"

#define VM_NT 256

__global__ void __launch_bounds__(VM_NT) k_vmle(const EqTab tz, const u64 *x, u64 n, u64 *part, u32 *status)
{
    u64 acc = 0;
    bool bad = false;
    for (u64 k = blockIdx.x * (u64)VM_NT + threadIdx.x; k < n; k += (u64)gridDim.x * VM_NT) {
        const u64 v = x[k];
        bad |= (v >= FP_P);
        acc = f_add(acc, f_mul(eq_at(tz, k), v >= FP_P ? 0 : v));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_BAD_INPUT);
    __shared__ u64 s[VM_NT / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        u64 v = threadIdx.x < VM_NT / 32 ? s[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// Generic add~/mult~ of an explicitly wired layer at (r_P, r1, r2):
// sum over gates of eq(r_P, g) eq(r1, in1) eq(r2, in2), split by gate type.
__global__ void __launch_bounds__(VM_NT) k_vwire(Globals G, const u32 *layers_idx, u64 *wire)
{
    const u32 i = layers_idx[blockIdx.x];
    const LayerDev &L = G.layers[i];
    const u64 S = 1ull << L.s;
    u64 add = 0, mult = 0;
    for (u64 g = threadIdx.x; g < S; g += VM_NT) {
        const u64 w = f_mul(eq_at(L.trp, g), f_mul(eq_at(L.tr1, L.in1[g]), eq_at(L.tr2, L.in2[g])));
        if (L.type[g]) mult = f_add(mult, w);
        else add = f_add(add, w);
    }
    __shared__ u64 s[2][VM_NT / 32];
    add = warp_sum(add);
    mult = warp_sum(mult);
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = add;
        s[1][threadIdx.x >> 5] = mult;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        u64 a = threadIdx.x < VM_NT / 32 ? s[0][threadIdx.x] : 0;
        u64 m = threadIdx.x < VM_NT / 32 ? s[1][threadIdx.x] : 0;
        a = warp_sum(a);
        m = warp_sum(m);
        if (threadIdx.x == 0) {
            wire[2 * i] = a;
            wire[2 * i + 1] = m;
        }
    }
}

__device__ __forceinline__ u64 eq2(u64 a, u64 b)
{
    return f_add(f_mul(a, b), f_mul(f_sub(1, a), f_sub(1, b)));
}

__device__ __forceinline__ u64 eq3(u64 a, u64 b, u64 c)
{
    return f_add(f_mul(f_mul(a, b), c), f_mul(f_mul(f_sub(1, a), f_sub(1, b)), f_sub(1, c)));
}

// add~, mult~ of the structured wiring kinds at (p, w1, w2): each gate set is a
// product of per-coordinate indicator patterns, so its multilinear extension
// is the product of the matching per-coordinate factors.
__device__ void wiring_closed(u32 kind, u32 si, u32 sn, const u64 *p, const u64 *w1, const u64 *w2, u64 &add,
                              u64 &mult)
{
    add = 0;
    mult = 0;
    switch (kind) {
    case W_SQUARE: {  // g = MUL(g, g)
        u64 v = 1;
        for (u32 k = 0; k < si; k++) v = f_mul(v, eq3(p[k], w1[k], w2[k]));
        mult = v;
        break;
    }
    case W_TREE: {  // g = ADD(2g, 2g+1): w1 low bit 0, w2 low bit 1, rest = g
        u64 v = f_mul(f_sub(1, w1[0]), w2[0]);
        for (u32 k = 0; k < si; k++) v = f_mul(v, eq3(p[k], w1[k + 1], w2[k + 1]));
        add = v;
        break;
    }
    case W_F0_FIRST: {  // 2j = MUL(j, j), 2j+1 = ADD(j, j)
        u64 v = 1;
        for (u32 k = 0; k < sn; k++) v = f_mul(v, eq3(p[k + 1], w1[k], w2[k]));
        add = f_mul(p[0], v);
        mult = f_mul(f_sub(1, p[0]), v);
        break;
    }
    case W_F0_PAIR: {  // 2j = MUL(2j, 2j), 2j+1 = MUL(2j+1, 2j): in1 = g, in2 = g with low bit 0
        u64 v = f_mul(eq2(p[0], w1[0]), f_sub(1, w2[0]));
        for (u32 k = 1; k < si; k++) v = f_mul(v, eq3(p[k], w1[k], w2[k]));
        mult = v;
        break;
    }
    case W_F0_FINAL: {  // j = MUL(2j+1, 2j+1)
        u64 v = f_mul(w1[0], w2[0]);
        for (u32 k = 0; k < si; k++) v = f_mul(v, eq3(p[k], w1[k + 1], w2[k + 1]));
        mult = v;
        break;
    }
    case W_MATMULT: {  // g = (k, j, i) low to high; in1 = (k, i, 0); in2 = (j, k, 1)
        const u32 L = si / 3;
        u64 v = f_mul(f_sub(1, w1[2 * L]), w2[2 * L]);
        for (u32 b = 0; b < L; b++) {
            v = f_mul(v, eq3(p[b], w1[b], w2[L + b]));      // k bits
            v = f_mul(v, eq2(p[L + b], w2[b]));             // j bits
            v = f_mul(v, eq2(p[2 * L + b], w1[L + b]));     // i bits
        }
        mult = v;
        break;
    }
    default:
        break;
    }
}

// g(r) for the degree-2 polynomial with values g0, g1, g2 at 0, 1, 2.
__device__ __forceinline__ u64 interp3(u64 g0, u64 g1, u64 g2, u64 r)
{
    const u64 rm1 = f_sub(r, 1), rm2 = f_sub(r, 2);
    const u64 t0 = f_mul(f_mul(g0, f_mul(rm1, rm2)), FP_INV2);
    const u64 t1 = f_mul(g1, f_mul(r, rm2));
    const u64 t2 = f_mul(f_mul(g2, f_mul(r, rm1)), FP_INV2);
    return f_add(f_sub(t0, t1), t2);
}

// Value at x of the polynomial with values q[0..n] at 0..n (Lagrange form):
// weight_t = prod_{u != t}(x - u) / (t! (n-t)! (-1)^(n-t)).
__device__ u64 lagrange_at(const u64 *q, u32 n, u64 x, const u64 *invfact)
{
    u64 pre[33], suf[33];
    pre[0] = 1;
    for (u32 t = 0; t < n; t++) pre[t + 1] = f_mul(pre[t], f_sub(x, t));
    suf[n] = 1;
    for (int t = (int)n; t >= 1; t--) suf[t - 1] = f_mul(suf[t], f_sub(x, (u64)t));
    u64 acc = 0;
    for (u32 t = 0; t <= n; t++) {
        u64 w = f_mul(f_mul(pre[t], suf[t]), f_mul(invfact[t], invfact[n - t]));
        if ((n - t) & 1) w = f_neg(w);
        acc = f_add(acc, f_mul(q[t], w));
    }
    return acc;
}

#define VC_NT 1024

// All checks of the verifier, concurrently (one CTA):
//   phase 1: transcript entries canonical; claimed outputs' MLE at z_0; sum of
//            the input-MLE partials;
//   phase 2: per layer i, its starting claim (V~_0(z_0) for i = 0, else
//            q_{i-1}(tau_{i-1})), its end check claim_n = eq(z_i, r_P)[add~ (v1+v2)
//            + mult~ v1 v2] with claim_n = g_{n-1}(r_{n-1}) (or the starting
//            claim when the layer has no rounds), and for the last layer
//            q(tau) = input MLE;
//   phase 3: per round j of layer i, g_j(0) + g_j(1) = g_{j-1}(r_{j-1}) (the
//            starting claim for j = 0).
__global__ void __launch_bounds__(VC_NT) k_vcheck(Globals G, VerifyDev V, EqTab tz0, u64 S0, const u32 *round_layer,
                                                  u32 nrounds)
{
    __shared__ u64 invfact[64];
    __shared__ u64 s_red[VC_NT / 32];
    __shared__ u64 s_out_mle, s_in_mle;
    __shared__ int s_bad, s_fail;
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_bad = 0;
        s_fail = 0;
    }
    if (tid < 64) invfact[tid] = G.invfact[tid];
    // phase 1
    bool bad = false;
    for (u64 k = tid; k < V.tr_len; k += VC_NT) bad |= (V.tr[k] >= FP_P);
    u64 acc = 0;
    for (u64 b = tid; b < S0; b += VC_NT) acc = f_add(acc, f_mul(eq_at(tz0, b), V.tr[b] >= FP_P ? 0 : V.tr[b]));
    u64 acc2 = 0;
    for (u32 k = tid; k < V.mle_blocks; k += VC_NT) acc2 = f_add(acc2, V.mle_part[k]);
    __syncthreads();
    if (__any_sync(0xffffffffu, bad) && lane == 0) s_bad = 1;
    acc = warp_sum(acc);
    acc2 = warp_sum(acc2);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (tid < 32) {
        u64 v = tid < VC_NT / 32 ? s_red[tid] : 0;
        v = warp_sum(v);
        if (tid == 0) s_out_mle = v;
    }
    __syncthreads();
    if (lane == 0) s_red[warp] = acc2;
    __syncthreads();
    if (tid < 32) {
        u64 v = tid < VC_NT / 32 ? s_red[tid] : 0;
        v = warp_sum(v);
        if (tid == 0) s_in_mle = v;
    }
    __syncthreads();
    if (s_bad) goto done;
    // phase 2
    for (u32 i = tid; i < G.d; i += VC_NT) {
        const LayerDev &L = G.layers[i];
        const u32 si = L.s, sn = L.sn, n = si + 2 * sn;
        const u64 *r = G.chal + L.chal_off;
        u64 start;
        if (i == 0) {
            start = s_out_mle;
        } else {
            const LayerDev &Lp = G.layers[i - 1];
            start = lagrange_at(V.tr + Lp.tr_q, Lp.sn, G.chal[Lp.chal_off + Lp.s + 2 * Lp.sn], invfact);
        }
        V.claims[i] = start;
        u64 claim = start;
        if (n > 0) {
            const u64 *m = V.tr + L.tr_msg + 3ull * (n - 1);
            claim = interp3(m[0], m[1], m[2], r[n - 1]);
        }
        const u64 *q = V.tr + L.tr_q;
        const u64 v1 = q[0], v2 = sn ? q[1] : q[0];
        u64 add, mult;
        if (L.kind == W_EXPLICIT) {
            add = V.wire[2 * i];
            mult = V.wire[2 * i + 1];
        } else {
            wiring_closed(L.kind, si, sn, r, r + si, r + si + sn, add, mult);
        }
        const u64 expect = f_mul(G.scal[SCAL_EQZRP(i)], f_add(f_mul(add, f_add(v1, v2)), f_mul(mult, f_mul(v1, v2))));
        bool ok = (expect == claim);
        if (i + 1 == G.d) ok &= (lagrange_at(q, sn, G.chal[L.chal_off + n], invfact) == s_in_mle);
        if (!ok) atomicOr(&s_fail, 1);
    }
    __syncthreads();
    // phase 3
    for (u32 g = tid; g < nrounds; g += VC_NT) {
        const u32 i = round_layer[g] >> 8, j = round_layer[g] & 0xFF;
        const LayerDev &L = G.layers[i];
        const u64 *m = V.tr + L.tr_msg + 3ull * j;
        u64 prev;
        if (j == 0) prev = V.claims[i];
        else prev = interp3(m[-3], m[-2], m[-1], G.chal[L.chal_off + j - 1]);
        if (f_add(m[0], m[1]) != prev) atomicOr(&s_fail, 1);
    }
    __syncthreads();
done:
    if (tid == 0) {
        V.result[0] = s_in_mle;
        V.result[1] = s_out_mle;
        V.result[2] = (!s_bad && !s_fail) ? 1 : 0;
        V.result[3] = s_bad;
        if (V.accept_out) *V.accept_out = (!s_bad && !s_fail) ? 1 : 0;
    }
}

__global__ void k_init_invfact(u64 *invfact)
{
    const u32 k = threadIdx.x;
    if (k < 64) {
        u64 f = 1;
        for (u32 j = 2; j <= k; j++) f = f_mul(f, j);
        invfact[k] = f_inv(f);
    }
}

void launch_init_invfact(u64 *invfact, cudaStream_t st) { k_init_invfact<<<1, 64, 0, st>>>(invfact); }

void launch_verify(const Globals &G, const VerifyDev &V, const EqTab &tzd, const EqTab &tz0,
                   const u32 *explicit_layers, int n_explicit, cudaStream_t st)
{
    const u64 nin = 1ull << tzd.n;
    k_vmle<<<V.mle_blocks, VM_NT, 0, st>>>(tzd, V.inputs, nin, V.mle_part, G.status);
    if (n_explicit > 0) k_vwire<<<n_explicit, VM_NT, 0, st>>>(G, explicit_layers, V.wire);
    k_vcheck<<<1, VC_NT, 0, st>>>(G, V, tz0, 1ull << tz0.n, V.round_layer, V.nrounds);
}
