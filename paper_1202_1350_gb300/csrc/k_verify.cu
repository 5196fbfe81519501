// k_verify.cu -- verifier kernels (Sec. 2.2, Sec. 3.1, Sec. 4.1.2 of the paper).
//
// The bulk of the verifier's work is its "secret": the input's multilinear
// extension at the final random point, a sum in which every input contributes
// independently (Sec. 4.1.2), computed here as a grid-wide reduction whose
// CTAs derive the point from the seed themselves (so it runs beside the coin
// launch).  The round checks of one layer form a short sequential chain;
// since each layer's starting claim can be read off the transcript
// (q_{i-1}(tau_{i-1})), all layers are checked concurrently, a warp per layer,
// and every round by its own thread.  The accept bit is the conjunction of
// exactly the checks the sequential verifier makes.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "coins.cuh"

#define VM_NT 256
#define VM_MID 4  // at most 2^4 iterations per thread: a CTA covers at most 2^12 entries

// Partial sums of the two multilinear extensions the verifier needs: the
// input's at z_d (blocks [0, nin_blocks)) and the claimed outputs' at z_0 (the
// remaining blocks).  Every value contributes independently (Sec. 4.1.2);
// products accumulate exactly in 128 bits.  A CTA takes an aligned range of
// 2^lr entries and derives the point's coordinates from the seed itself, so
// the launch needs no eq table and does not wait for the coin launch:
// eq(z, i) = (coordinates above the range: per CTA) x (the low min(8, lr):
// per thread, from two 16-entry tables) x (the rest: per iteration, from a
// small table).  A non-canonical input latches ST_BAD_INPUT; a non-canonical
// output entry marks the transcript bad.
// A launch covers blocks [b0, b0 + gridDim.x) of the two ranges; src_arg,
// if given, is the source of a launch within one range (else vp's inputs and
// transcript).
__global__ void __launch_bounds__(VM_NT) k_vmle(const Globals *Gd, const VerifyPtrs *vp, u32 nd, u32 lin, u32 n0,
                                                u32 lout, u32 nin_blocks, u32 b0, const u64 *src_arg, u64 *part,
                                                u32 *status, u64 *result)
{
    const Globals &G = *Gd;
    const u32 blk = blockIdx.x + b0;
    const bool inp = blk < nin_blocks;
    const u32 nz = inp ? nd : n0, lr = inp ? lin : lout;
    const u32 b = inp ? blk : blk - nin_blocks;
    const u64 *src = src_arg ? src_arg : (inp ? vp->inputs : vp->tr);  // the claimed outputs open the transcript
    __shared__ u64 z[32], zm[32], mid[1u << VM_MID], t1[16], t2[16], bfac;
    const bool rej = draws_rejected(G);
    if (threadIdx.x < nz) {
        const u64 v = zcoord(G, rej, inp ? G.d : 0, threadIdx.x);
        z[threadIdx.x] = v;
        zm[threadIdx.x] = f_sub(1, v);
    }
    __syncthreads();
    // small factor tables, each entry a product of at most four factors:
    // t1 over coordinates [0, l1), t2 over [l1, lo), mid over [lo, lr); and
    // the CTA's factor over [lr, nz) as a warp product
    const u32 lo = lr < 8 ? lr : 8, nit = 1u << (lr - lo), l1 = lo < 4 ? lo : 4, l2 = lo - l1;
    const u32 tid = threadIdx.x;
    if (tid < 16) {
        u64 f = 1;
        for (u32 k = 0; k < l1; k++) f = f_mul(f, ((tid >> k) & 1) ? z[k] : zm[k]);
        t1[tid] = f;
    } else if (tid < 32) {
        const u32 q = tid - 16;
        u64 f = 1;
        for (u32 k = 0; k < l2; k++) f = f_mul(f, ((q >> k) & 1) ? z[l1 + k] : zm[l1 + k]);
        t2[q] = f;
    } else if (tid < 32 + nit) {
        const u32 q = tid - 32;
        u64 f = 1;
        for (u32 k = lo; k < lr; k++) f = f_mul(f, ((q >> (k - lo)) & 1) ? z[k] : zm[k]);
        mid[q] = f;
    } else if (tid >= 64 && tid < 96) {
        const u32 k = lr + (tid - 64);
        const u64 f = (k < nz) ? (((b >> (k - lr)) & 1) ? z[k] : zm[k]) : 1;
        const u64 pr = warp_prod(f);
        if (tid == 64) bfac = pr;
    }
    __syncthreads();
    acc128 acc;
    acc_zero(acc);
    bool bad = false;
    if (tid < (1u << lo)) {
        const u64 w = f_mul(f_mul(t1[tid & 15], t2[tid >> 4]), bfac);
        const u64 base = ((u64)b << lr) + tid;
        for (u32 it = 0; it < nit; it++) {
            const u64 v = src[base + ((u64)it << lo)];
            bad |= (v >= FP_P);
            mac(acc, f_mul(w, mid[it]), v >= FP_P ? 0 : v);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        if (inp) atomicOr(status, ST_BAD_INPUT);
        else atomicOr(reinterpret_cast<unsigned long long *>(&result[3]), 1ull);
    }
    __shared__ u64 s[VM_NT / 32];
    const u64 w = warp_wsum(acc_red(acc));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
        const u64 v = threadIdx.x < VM_NT / 32 ? s[threadIdx.x] : 0;
        const u64 t = warp_wsum(v);
        if (threadIdx.x == 0) part[blk] = wcanon(t);
    }
}

// Sums of a CTA's (add, mult) pair, in thread 0.
__device__ __forceinline__ void block_sum2(u64 &add, u64 &mult)
{
    __shared__ u64 s[2][VM_NT / 32];
    add = warp_sum(add);
    mult = warp_sum(mult);
    __syncthreads();  // s may still be read by an earlier call
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = add;
        s[1][threadIdx.x >> 5] = mult;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        u64 a = threadIdx.x < VM_NT / 32 ? s[0][threadIdx.x] : 0;
        u64 m = threadIdx.x < VM_NT / 32 ? s[1][threadIdx.x] : 0;
        add = warp_sum(a);
        mult = warp_sum(m);
    }
}

// Generic add~/mult~ of an explicitly wired layer at (r_P, r1, r2):
// sum over gates of eq(r_P, g) eq(r1, in1) eq(r2, in2), split by gate type.
// Each CTA sums a range of the layer's gates; the CTA that finishes a layer
// last (a counter, no waiting) adds the layer's partial sums.
__global__ void __launch_bounds__(VM_NT) k_vwire(Globals G, const VwireItem *items, VerifyDev V)
{
    const VwireItem it = items[blockIdx.x];
    const u32 i = it.layer;
    const LayerDev &L = G.layers[i];
    const u64 S = 1ull << L.s, chunk = (S + it.nblocks - 1) / it.nblocks;
    const u64 g0 = (u64)it.block * chunk, g1 = g0 + chunk < S ? g0 + chunk : S;
    u64 add = 0, mult = 0;
    for (u64 g = g0 + threadIdx.x; g < g1; g += VM_NT) {
        const u64 w = f_mul(eq_at(L.trp, g), f_mul(eq_at(L.tr1, L.in1[g]), eq_at(L.tr2, L.in2[g])));
        if (L.type[g]) mult = f_add(mult, w);
        else add = f_add(add, w);
    }
    block_sum2(add, mult);
    if (it.nblocks == 1) {
        if (threadIdx.x == 0) {
            V.wire[2 * i] = add;
            V.wire[2 * i + 1] = mult;
        }
        return;
    }
    __shared__ u32 s_last;
    if (threadIdx.x == 0) {
        V.wire_part[2 * (it.part_off + it.block)] = add;
        V.wire_part[2 * (it.part_off + it.block) + 1] = mult;
        __threadfence();
        s_last = (atomicAdd(&V.wire_ctr[i], 1u) == it.nblocks - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    add = mult = 0;
    for (u32 b = threadIdx.x; b < it.nblocks; b += VM_NT) {
        add = f_add(add, __ldcg(V.wire_part + 2 * (it.part_off + b)));
        mult = f_add(mult, __ldcg(V.wire_part + 2 * (it.part_off + b) + 1));
    }
    block_sum2(add, mult);
    if (threadIdx.x == 0) {
        V.wire[2 * i] = add;
        V.wire[2 * i + 1] = mult;
        V.wire_ctr[i] = 0;
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

// Value at x of the polynomial with values q[0..n] at 0..n (n <= 31), by the
// whole warp: lane t forms the Lagrange weight
//   prod_{u != t} (x - u) / (t! (n-t)! (-1)^(n-t))
// from warp prefix and suffix products of the factors (x - u).
__device__ u64 lagrange_warp(const u64 *q, u32 n, u64 x, const u64 *invfact)
{
    const u32 lane = threadIdx.x & 31;
    const bool in = lane <= n;
    const u64 f = in ? f_sub(x, (u64)lane) : 1;
    const u64 incl = warp_scan_mul(f);
    u64 pre = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) pre = 1;
    const u64 rincl = warp_rscan_mul(f);
    u64 suf = __shfl_down_sync(0xffffffffu, rincl, 1);
    if (lane == 31) suf = 1;
    u64 term = 0;
    if (in) {
        u64 w = f_mul(f_mul(pre, suf), f_mul(invfact[lane], invfact[n - lane]));
        if ((n - lane) & 1) w = f_neg(w);
        term = f_mul(q[lane], w);
    }
    return wcanon(warp_wsum(term));
}

// add~, mult~ at (p, w1, w2) for a structured kind, by the whole warp: lane k
// forms the factor of coordinate k, the warp multiplies them.
__device__ void wiring_warp(u32 kind, u32 si, u32 sn, const u64 *p, const u64 *w1, const u64 *w2, u64 &add,
                            u64 &mult)
{
    const u32 k = threadIdx.x & 31;
    u64 f = 1, lead = 1;
    bool is_add = false;
    switch (kind) {
    case W_SQUARE:
        if (k < si) f = eq3(p[k], w1[k], w2[k]);
        break;
    case W_TREE:
        is_add = true;
        if (k < si) f = eq3(p[k], w1[k + 1], w2[k + 1]);
        lead = f_mul(f_sub(1, w1[0]), w2[0]);
        break;
    case W_F0_FIRST:
        if (k < sn) f = eq3(p[k + 1], w1[k], w2[k]);
        break;
    case W_F0_PAIR:
        if (k >= 1 && k < si) f = eq3(p[k], w1[k], w2[k]);
        lead = f_mul(eq2(p[0], w1[0]), f_sub(1, w2[0]));
        break;
    case W_F0_FINAL:
        if (k < si) f = eq3(p[k], w1[k + 1], w2[k + 1]);
        lead = f_mul(w1[0], w2[0]);
        break;
    case W_MATMULT: {
        const u32 L = si / 3;
        if (k < L) f = f_mul(eq3(p[k], w1[k], w2[L + k]), f_mul(eq2(p[L + k], w2[k]), eq2(p[2 * L + k], w1[L + k])));
        lead = f_mul(f_sub(1, w1[2 * L]), w2[2 * L]);
        break;
    }
    default:
        break;
    }
    const u64 v = f_mul(warp_prod(f), lead);
    add = 0;
    mult = 0;
    if (kind == W_F0_FIRST) {
        add = f_mul(p[0], v);
        mult = f_mul(f_sub(1, p[0]), v);
    } else if (is_add) {
        add = v;
    } else {
        mult = v;
    }
}

#define VC_NT 256
#define VC_CL 8  // CTAs of the check launch: one thread-block cluster

// All checks of the verifier in one cluster of VC_CL CTAs; the accept bit is
// combined through the cluster's distributed shared memory (no grid-wide
// atomics).  The warps of the cluster take three kinds of item: a layer's
// starting claim with its round 0, a layer's end, and the last claim (q(tau)
// of layer d-1 = the input's MLE at z_d), all independent.  The checks: the
// layer's starting claim (for layer 0 the claimed outputs' MLE at z_0: formed
// by the warp itself when there are at most VC_OUT_INLINE outputs, else
// summed from k_vmle's partials; for layer i > 0, q_{i-1}(tau_{i-1})), round
// 0 (g_0(0) + g_0(1) = starting claim), the end of the layer
// (g_{n-1}(r_{n-1}) = eq(z_i, r_P)[add~ (v1 + v2) + mult~ v1 v2], or the
// starting claim itself when the layer has no rounds).  Every thread checks
// rounds j >= 1 (g_j(0) + g_j(1) = g_{j-1}(r_{j-1})) of a grid-stride share of
// the global rounds, and its share of the transcript entries for canonical
// form.  The
// accept bit is the conjunction of exactly the sequential verifier's checks.
// tr_arg: the transcript and accept pointer given directly (NULL: from V.vp).
__global__ void __cluster_dims__(VC_CL, 1, 1) __launch_bounds__(VC_NT)
    k_vcheck(Globals G, VerifyDev V, const u64 *tr_arg, int *accept_arg)
{
    namespace cg = cooperative_groups;
    const u64 *const tr = tr_arg ? tr_arg : V.vp->tr;
    const u32 lane = threadIdx.x & 31;
    const u32 g = blockIdx.x * VC_NT + threadIdx.x, nthreads = VC_CL * VC_NT;
    u32 fail = 0;
    // warp items: [0, d) a layer's starting claim and its round 0 (with the
    // end of the layer when it has no rounds, whose claim is the start);
    // [d, 2d) the end of layer i - d; 2d the last claim against the input's MLE
    for (u32 item = g >> 5; item <= 2 * G.d; item += nthreads >> 5) {
        if (item == 2 * G.d) {
            if (G.d == 0) continue;
            const LayerDev &L = G.layers[G.d - 1];
            const u64 fin = lagrange_warp(tr + L.tr_q, L.sn, G.chal[L.chal_off + L.s + 2 * L.sn], G.invfact);
            u64 in_mle;
            warp_record_sums<1>(V.mle_part, V.mle_blocks, lane, &in_mle);
            if (lane == 0 && fin != in_mle) fail = 1;
            continue;
        }
        const bool end_item = item >= G.d;
        const u32 i = end_item ? item - G.d : item;
        const LayerDev &L = G.layers[i];
        const u32 si = L.s, sn = L.sn, n = si + 2 * sn;
        if (end_item && n == 0) continue;  // checked with the start
        const u64 *r = G.chal + L.chal_off;
        const u64 *m = tr + L.tr_msg;
        u64 claim = 0;
        if (!end_item) {
            u64 start;
            if (i == 0) {
                if (V.mle_out_blocks == 0) {
                    // every output's eq weight a direct product over the s_0
                    // coordinates of z_0 (the first s_0 challenges)
                    u64 sum = 0;
                    for (u64 b = lane; b < G.S0; b += 32) {
                        const u64 v = tr[b];
                        u64 w = 1;
                        for (u32 k = 0; k < si; k++) w = f_mul(w, ((b >> k) & 1) ? G.chal[k] : f_sub(1, G.chal[k]));
                        sum = f_add(sum, f_mul(w, v >= FP_P ? 0 : v));  // a non-canonical entry fails the scan
                    }
                    start = warp_sum(sum);
                } else {
                    warp_record_sums<1>(V.mle_part + V.mle_blocks, V.mle_out_blocks, lane, &start);
                }
            } else {
                const LayerDev &Lp = G.layers[i - 1];
                start = lagrange_warp(tr + Lp.tr_q, Lp.sn, G.chal[Lp.chal_off + Lp.s + 2 * Lp.sn], G.invfact);
            }
            if (n > 0) {
                if (lane == 0 && f_add(m[0], m[1]) != start) fail = 1;
                continue;
            }
            claim = start;
        } else if (lane == 0) {
            const u64 *ml = m + 3ull * (n - 1);
            claim = interp3(ml[0], ml[1], ml[2], r[n - 1]);
        }
        u64 add = 0, mult = 0;
        if (L.kind == W_EXPLICIT) {
            add = V.wire[2 * i];
            mult = V.wire[2 * i + 1];
        } else {
            wiring_warp(L.kind, si, sn, r, r + si, r + si + sn, add, mult);
        }
        if (lane == 0) {
            const u64 *q = tr + L.tr_q;
            const u64 v1 = q[0], v2 = sn ? q[1] : q[0];
            const u64 expect = f_mul(G.scal[SCAL_EQZRP(i)], f_add(f_mul(add, f_add(v1, v2)), f_mul(mult, f_mul(v1, v2))));
            if (expect != claim) fail = 1;
        }
    }
    for (u32 rho = g; rho < V.nrounds; rho += nthreads) {
        const u32 i = V.round_layer[rho] >> 8, j = V.round_layer[rho] & 0xFF;
        if (j > 0) {
            const LayerDev &L = G.layers[i];
            const u64 *m = tr + L.tr_msg + 3ull * j;
            const u64 prev = interp3(m[-3], m[-2], m[-1], G.chal[L.chal_off + j - 1]);
            if (f_add(m[0], m[1]) != prev) fail = 1;
        }
    }
    for (u64 k = g; k < V.tr_len; k += nthreads)
        if (tr[k] >= FP_P) fail = 1;
    // each CTA's verdict into CTA 0's shared memory, then CTA 0 decides
    __shared__ u32 s_fail[VC_CL];
    fail = __syncthreads_or(fail);
    cg::cluster_group cluster = cg::this_cluster();
    if (threadIdx.x == 0) *cluster.map_shared_rank(&s_fail[cluster.block_rank()], 0) = fail ? 1u : 0u;
    cluster.sync();
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
        u32 bad = 0;
        for (int k = 0; k < VC_CL; k++) bad |= s_fail[k];
        const int acc = bad ? 0 : 1;
        V.result[2] = (u64)acc;
        V.result[3] = bad;
        int *const accept_out = tr_arg ? accept_arg : V.vp->accept_out;
        if (accept_out) *accept_out = acc;
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

// Per-call verifier parameters; also clears the result words (flags, accept bit).
__global__ void k_vparams(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *tr, const u64 *inputs, int *accept,
                          u64 *result)
{
    G->seed = seed;
    vp->tr = tr;
    vp->inputs = inputs;
    vp->accept_out = accept;
    for (int k = 0; k < VC_RESULT_WORDS; k++) result[k] = 0;
}

void launch_vparams(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *tr, const u64 *inputs, int *accept,
                    u64 *result, cudaStream_t st)
{
    k_vparams<<<1, 1, 0, st>>>(G, vp, seed, tr, inputs, accept, result);
}

const void *vparams_kernel() { return reinterpret_cast<const void *>(k_vparams); }

// Parameters of the verifier's input pass (seed, inputs).
__global__ void k_vparams_in(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *inputs)
{
    G->seed = seed;
    vp->inputs = inputs;
}


void launch_vparams_in(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *inputs, cudaStream_t st)
{
    k_vparams_in<<<1, 1, 0, st>>>(G, vp, seed, inputs);
}


const void *vparams_in_kernel() { return reinterpret_cast<const void *>(k_vparams_in); }


// Entries per CTA (log2) of the MLE partial sums for a point of n coordinates.
u32 vmle_log(u32 n) { return n < 11 ? n : 11; }

void launch_verify(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0, const VwireItem *wire_items,
                   int n_wire, cudaStream_t st_mle, cudaEvent_t ev_join, cudaStream_t st)
{
    // the MLE partial sums need only the seed: they run beside the coin launch
    // (st_mle forked from st before it); the checks wait for both
    k_vmle<<<V.mle_blocks + V.mle_out_blocks, VM_NT, 0, st_mle>>>(Gd, V.vp, nd, vmle_log(nd), n0, vmle_log(n0),
                                                                   V.mle_blocks, 0, nullptr, V.mle_part, G.status,
                                                                   V.result);
    cudaEventRecord(ev_join, st_mle);
    cudaStreamWaitEvent(st, ev_join, 0);
    if (n_wire > 0) k_vwire<<<n_wire, VM_NT, 0, st>>>(G, wire_items, V);
    k_vcheck<<<VC_CL, VC_NT, 0, st>>>(G, V, nullptr, nullptr);
}

void launch_verify_input(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0, cudaStream_t st)
{
    k_vmle<<<V.mle_blocks, VM_NT, 0, st>>>(Gd, V.vp, nd, vmle_log(nd), n0, vmle_log(n0), V.mle_blocks, 0, nullptr,
                                           V.mle_part, G.status, V.result);
}

void launch_verify_transcript(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0,
                              const VwireItem *wire_items, int n_wire, const u64 *tr, int *accept,
                              cudaStream_t st)
{
    if (V.mle_out_blocks > 0)
        k_vmle<<<V.mle_out_blocks, VM_NT, 0, st>>>(Gd, V.vp, nd, vmle_log(nd), n0, vmle_log(n0), V.mle_blocks,
                                                   V.mle_blocks, tr, V.mle_part, G.status, V.result);
    if (n_wire > 0) k_vwire<<<n_wire, VM_NT, 0, st>>>(G, wire_items, V);
    k_vcheck<<<VC_CL, VC_NT, 0, st>>>(G, V, tr, accept);
}
