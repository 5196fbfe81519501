// k_sc.cu -- sum-check waves of the prover (Sec. 4.1.1 of the paper: every
// message is a field sum of independent per-gate contributions; Sec. 3.1:
// messages are degree-2 polynomials given by their values at 0, 1, 2).
//
// Each sum-check instance (SCI) sums P(x) V(x) + B(x) over n variables bound
// low bit first.  Two kinds of instance:
//
//  * product-weighted (PROD): P(x) = sigma prod_m L_m(x_m) with linear factors
//    L_m(b) = c0_m (1-b) + c1_m b, B = gamma-multiple of P.  Folding P keeps the
//    product form, so P is never stored: round j's message is
//      g_j(t) = kappa_j L_j(t) h_j(t),  h_j(t) = sum_y E_j(y) V_j(t, y),
//    with kappa_j = sigma prod_{m<j} L_m(r_m), E_j(y) = prod_{m>j} L_m(y_m) and
//    V_j the value table folded with r_0..r_{j-1}; h_j is linear in t, so only
//    h_j(0), h_j(1) are summed.  Per pair of entries: two multiply-adds and one
//    fold.  Used for phase 1 of every layer (P = eq(z_i, .)) and for phase 3 of
//    TREE and SQUARE layers.
//  * general (GEN): P, V, B are tables folded every round; the message needs
//    P(t)V(t) + B(t) at t = 0, 1, 2.  Chunks sum the values at 0 and 1 and the
//    leading coefficient (P1 - P0)(V1 - V0) of each pair, which shares its
//    differences with the folds; k_final turns the three sums into the value
//    at 2.  The first wave builds P and B from the wiring on the fly (SQUARE,
//    TREE phase 2) or reads tables built by k_build23.
//
// Arithmetic is lazy: table values stay in W = [0, 2^61 + 8), products
// accumulate exactly in 128 bits and are reduced once per round per thread;
// only transcript entries are made canonical.
#include <cuda_runtime.h>

#include <algorithm>

#include "plan.h"

// --------------------------------------------------------------------------------
// Shared helpers
// --------------------------------------------------------------------------------

// Sum over the warp of 16 values per lane: afterwards lane l holds the total of
// value index l >> 1.  Inputs in W; sums are brought back to W every two
// halving steps (a sum of four W values is below 2^64).
__device__ __forceinline__ u64 warp_sum16(u64 (&v)[16])
{
    const u32 lane = threadIdx.x & 31;
#pragma unroll
    for (int step = 0; step < 4; step++) {
        const int o = 16 >> step, half = 8 >> step;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const u64 send = up ? v[i] : v[i + half];
            const u64 keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            if (step & 1) v[i] = wred(v[i]);
        }
    }
    u64 r = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
    return wred(r);
}

// Sum over the warp of 32 values per lane: afterwards lane l holds the total
// of value index l.  Inputs in W.
__device__ __forceinline__ u64 warp_sum32(u64 (&v)[32])
{
    const u32 lane = threadIdx.x & 31;
#pragma unroll
    for (int step = 0; step < 5; step++) {
        const int o = 16 >> step, half = 16 >> step;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const u64 send = up ? v[i] : v[i + half];
            const u64 keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            if (step & 1) v[i] = wred(v[i]);
        }
    }
    return wred(v[0]);
}

// (The per-wave weight tables of the PROD waves are built with the coins, in
// k_coins.cu.)


// --------------------------------------------------------------------------------
// One persistent launch for the waves of every instance: CTAs of WV_NT threads
// take tasks (one chunk of one line, PROD or GEN wave) from a shared counter,
// so the whole device stays busy until the last task; a wave whose successor
// is a single chunk runs that successor in the CTA that finishes the wave's
// last chunk (no CTA ever waits for another).
// --------------------------------------------------------------------------------

#define WV_NT 128
#define PR_SUB 16  // PROD runs of 16 entries (rounds 0..3 per run)

struct ProdSmem {
    u32 r[32][2];
    u64 Q[64];
    u64 E[256];
    u64 lvl[WV_NT / 32];
    u64 w[WV_NT / 32][32];
    u64 echunk;
};

struct GenSmem {
    u32 r[32][2];
    u64 lvl[3][WV_NT / 32];
    u64 w[WV_NT / 32][40];
    u64 hs[9][WV_NT];  // per-thread sums of in-register rounds 2..4 (kept out of registers)
};

#define LN_E 6        // line: coordinates folded per thread in registers (first wave)
#define LN_BUFA 2048  // line: shared-memory polynomial buffers (coefficients): a later
#define LN_BUFB 1024  // wave's first level is 64 pairs x <= 32 coefficients

struct LineSmem {
    u32 la[32][2], lb[32][2];  // limbs of a_k and b_k for the wave's coordinates
    u64 bufA[LN_BUFA];
    u64 bufB[LN_BUFB];
};

union WaveSmem {
    ProdSmem prod;
    GenSmem gen;
    LineSmem line;
};

// Load of a wave's input.  A first wave's input (layer values, or tables built
// by an earlier launch) is read-only for the whole launch and goes through
// L1, where the prefetch of the next run lands; a later wave's input is
// written by other CTAs of this launch and is read through L2.
__device__ __forceinline__ ulonglong2 ld_in(const ulonglong2 *p, bool ext) { return ext ? __ldg(p) : __ldcg(p); }
__device__ __forceinline__ u64 ld_in(const u64 *p, bool ext) { return ext ? __ldg(p) : __ldcg(p); }

// Bring the line holding p into L1 ahead of its load (no register cost).
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Sum of the four warps' per-warp round sums (W values).
__device__ __forceinline__ u64 cta_sum4(const u64 *a, const u64 *b, const u64 *c, const u64 *d)
{
    return wred(*a + *b + *c + *d);
}

// ---- PROD -----------------------------------------------------------------------

// Sum over the lanes l = 0 mod 2^(kk+1) of a warp (the lanes holding a
// contribution in cross round kk; the others hold 0), written by lane 0.
__device__ __forceinline__ void prod_round_sum(u64 c0, u64 c1, u32 kk, u64 *out)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if ((u32)o < (2u << kk)) break;
        c0 = wred(c0 + __shfl_xor_sync(0xffffffffu, c0, o));
        c1 = wred(c1 + __shfl_xor_sync(0xffffffffu, c1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        out[0] = c0;
        out[1] = c1;
    }
}

// Rounds off.. of a product-weighted chunk across threads.  Thread t holds
// level value t (t < na); a round pairs values 2y and 2y+1, which sit in the
// threads t = y 2^(kk+1) and t + 2^kk, and the first of them keeps the folded
// value, so rounds stay inside a warp for kk < 5 (shuffles) and continue in
// warp 0 after one exchange through shared memory.  The active thread of a
// pair contributes E_k(y) u0 and E_k(y) u1; the per-warp sums of round k go
// to sm.w[warp][2k..2k+1] (CTA-level rounds: warp 0's row, zeros elsewhere).
__device__ __forceinline__ void prod_cross(u64 uv, u32 off, u32 tid, u32 na, u32 nr, ProdSmem &sm, u32 eoff0)
{
    const u32 lane = tid & 31, warp = tid >> 5;
    // rolled: one copy of the round body keeps the kernel small
#pragma unroll 1
    for (u32 kk = 0; kk < 5; kk++) {
        const u32 k = off + kk;
        if (k < nr) {  // uniform
            const u64 u1 = __shfl_down_sync(0xffffffffu, uv, 1u << kk);
            u64 c0 = 0, c1 = 0;
            if ((tid & ((2u << kk) - 1)) == 0 && tid < na) {
                const u32 y = tid >> (kk + 1);
                const u64 w = sm.E[eoff0 - (1u << (nr - k)) + y];
                c0 = wmul(w, uv);
                c1 = wmul(w, u1);
                uv = wfold(uv, u1, sm.r[k][0], sm.r[k][1]);
            }
            prod_round_sum(c0, c1, kk, &sm.w[warp][2 * k]);
        }
    }
    if (lane == 0) {
        sm.lvl[warp] = uv;
        for (u32 k = off + 5; k < nr && k < off + 7; k++)
            if (warp) sm.w[warp][2 * k] = sm.w[warp][2 * k + 1] = 0;
    }
    __syncthreads();
    if (off + 5 < nr && warp == 0) {
        uv = (lane < WV_NT / 32) ? sm.lvl[lane] : 0;
        for (u32 kk = 5; kk < 7; kk++) {
            const u32 k = off + kk;
            if (k < nr) {
                const u64 u1 = __shfl_down_sync(0xffffffffu, uv, 1u << (kk - 5));
                const u32 t = lane << 5;  // the thread index this lane stands for
                u64 c0 = 0, c1 = 0;
                if ((t & ((2u << kk) - 1)) == 0 && t < na) {
                    const u32 y = t >> (kk + 1);
                    const u64 w = sm.E[eoff0 - (1u << (nr - k)) + y];
                    c0 = wmul(w, uv);
                    c1 = wmul(w, u1);
                    uv = wfold(uv, u1, sm.r[k][0], sm.r[k][1]);
                }
                prod_round_sum(c0, c1, kk - 5, &sm.w[0][2 * k]);
            }
        }
        if (lane == 0) sm.lvl[0] = uv;
    }
}

// Rounds 0..3 of one run of 16 entries (run `sub` of the thread's 2^e):
// pair weights Q_k(q), q = pair index + (sub << (3 - k)).
__device__ __forceinline__ u64 prod_run16(u64 (&u)[16], u32 sub, u32 e, const ProdSmem &sm, u64 (&h)[12])
{
#pragma unroll
    for (int k = 0; k < 4; k++) {
        acc128 a0, a1, b0, b1;  // two chains per value for instruction-level parallelism
        acc_zero(a0);
        acc_zero(a1);
        acc_zero(b0);
        acc_zero(b1);
        const u32 rr0 = sm.r[k][0], rr1 = sm.r[k][1];
        const u32 qoff = (1u << e) - (1u << (e - k)) + (sub << (3 - k));
#pragma unroll
        for (int q = 0; q < (8 >> k); q++) {
            const u64 w = sm.Q[qoff + q];
            const u64 u0 = u[2 * q], u1 = u[2 * q + 1];
            if (q & 1) {
                mac(b0, w, u0);
                mac(b1, w, u1);
            } else {
                mac(a0, w, u0);
                mac(a1, w, u1);
            }
            u[q] = wfold(u0, u1, rr0, rr1);
        }
        h[2 * k] = wred(h[2 * k] + acc_red(a0) + acc_red(b0));
        h[2 * k + 1] = wred(h[2 * k + 1] + acc_red(a1) + acc_red(b1));
    }
    return u[0];
}

// In-register rounds for e in 4..6: runs of 16, then rounds 4 and 5 on the
// runs' folded values.
__device__ __forceinline__ u64 prod_regs_runs(const u64 *src, u32 e, bool ext, const ProdSmem &sm, u64 (&h)[12])
{
    const u32 nruns = 1u << (e - 4);
    const u32 q4 = (1u << e) - (1u << (e - 4)), q5 = (1u << e) - 2;
    u64 f0 = 0, g0 = 0, uv = 0;
    // a rolled loop keeps the kernel small (instruction-cache bound when unrolled)
#pragma unroll 1
    for (u32 sub = 0; sub < nruns; sub++) {
        if (sub + 1 < nruns) prefetch_l1(src + (sub + 1) * PR_SUB);
        u64 u[16];
        const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(src + sub * PR_SUB);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const ulonglong2 t = ld_in(sv + q, ext);
            u[2 * q] = t.x;
            u[2 * q + 1] = t.y;
        }
        const u64 fs = prod_run16(u, sub, e, sm, h);
        if (nruns == 1) {
            uv = fs;
        } else if (sub & 1) {
            const u64 w = sm.Q[q4 + (sub >> 1)];
            h[8] = wred(h[8] + wmul(w, f0));
            h[9] = wred(h[9] + wmul(w, fs));
            const u64 g = wfold(f0, fs, sm.r[4][0], sm.r[4][1]);
            if (nruns == 2) {
                uv = g;
            } else if (sub == 1) {
                g0 = g;
            } else {
                const u64 w5 = sm.Q[q5];
                h[10] = wmul(w5, g0);
                h[11] = wmul(w5, g);
                uv = wfold(g0, g, sm.r[5][0], sm.r[5][1]);
            }
        } else {
            f0 = fs;
        }
    }
    return uv;
}

// One chunk of a PROD wave.
__device__ void prod_chunk(const Globals &G, const ProdWave &W, u32 chunk, ProdSmem &sm)
{
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 nr = W.nr, e = W.e;
    const u32 na = 1u << (nr - e);
    const u64 base = (u64)chunk << nr;
    if (tid < nr) limbs31(G.chal[W.chal_off + tid], sm.r[tid][0], sm.r[tid][1]);
    const u64 *blk = W.wblk;
    const u32 qsize = (1u << e) - 1;
    const u32 kb = e ? e - 1 : 0;
    const u32 esize = (1u << (nr - kb)) - 1;
    if (tid < qsize) sm.Q[tid] = blk[tid];
    for (u32 k = tid; k < esize; k += WV_NT) sm.E[k] = blk[qsize + k];
    if (tid == 0) {
        const u64 *olo = blk + qsize + esize;
        const u64 *ohi = olo + (1u << W.ho);
        sm.echunk = f_mul(olo[chunk & ((1u << W.ho) - 1)], ohi[chunk >> W.ho]);
    }
    __syncthreads();
    const u32 eoff0 = 1u << (nr - kb);
    u64 uv = 0;
    if (e > 0) {
        u64 h[12];
#pragma unroll
        for (int i = 0; i < 12; i++) h[i] = 0;
        if (tid < na) {
            const u64 *src = W.in + base + ((u64)tid << e);
            uv = prod_regs_runs(src, e, W.r0 == 0, sm, h);
            const u64 T = sm.E[tid];  // E_{e-1}(tid): weight of the chunk bits above the thread's run
#pragma unroll
            for (int i = 0; i < 12; i++) h[i] = wmul(T, h[i]);
        }
        u64 h16[16];
#pragma unroll
        for (int i = 0; i < 16; i++) h16[i] = (i < 12) ? h[i] : 0;
        const u64 s = warp_sum16(h16);
        if ((lane & 1) == 0 && (lane >> 1) < 2 * e) sm.w[warp][lane >> 1] = s;
    } else if (tid < na) {
        uv = ld_in(W.in + base + tid, W.r0 == 0);
    }
    prod_cross(uv, e, tid, na, nr, sm, eoff0);
    __syncthreads();
    if (tid < 2 * nr) {
        const u64 sum = wred(sm.w[0][tid] + sm.w[1][tid] + sm.w[2][tid] + sm.w[3][tid]);
        const u32 k = tid >> 1, t = tid & 1;
        W.part[((u64)k * W.nchunks + chunk) * 2 + t] = wmul(sum, sm.echunk);
    }
    if (!(W.flags & WF_LAST) && tid == 0) W.out[chunk] = sm.lvl[0];
}

// ---- GEN ------------------------------------------------------------------------

// N consecutive entries of a GEN wave's P, V, B tables at x0 (tables built
// by k_build23, or the previous wave's outputs; the first waves of SQUARE and
// TREE phase 2 form P and B themselves: sq2_run, tree2_run).
template <int N>
__device__ __forceinline__ void gen_load(const GenWave &W, u64 x0, bool hasB, u64 (&p)[N], u64 (&v)[N], u64 (&b)[N])
{
    const bool ext = W.r0 == 0;
    const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(W.inV + x0);
#pragma unroll
    for (int q = 0; q < N / 2; q++) {
        const ulonglong2 t = ld_in(sv + q, ext);
        v[2 * q] = t.x;
        v[2 * q + 1] = t.y;
    }
    const ulonglong2 *sp = reinterpret_cast<const ulonglong2 *>(W.inP + x0);
#pragma unroll
    for (int q = 0; q < N / 2; q++) {
        const ulonglong2 t = ld_in(sp + q, ext);
        p[2 * q] = t.x;
        p[2 * q + 1] = t.y;
    }
    if (hasB) {
        const ulonglong2 *sb = reinterpret_cast<const ulonglong2 *>(W.inB + x0);
#pragma unroll
        for (int q = 0; q < N / 2; q++) {
            const ulonglong2 t = ld_in(sb + q, ext);
            b[2 * q] = t.x;
            b[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; q++) b[q] = 0;
    }
}

// One general pair: the message's values at t = 0, 1 (c0, c1) and its
// leading coefficient c2 = (P1 - P0)(V1 - V0), from which the value at 2 is
// 2 c1 - c0 + 2 c2 (B is linear in t); then the folds, which share the
// differences P1 - P0, V1 - V0, B1 - B0 (lazy, below 2^62.6).
__device__ __forceinline__ void gen_pair(u64 p0, u64 p1, u64 v0, u64 v1, u64 b0, u64 b1, u32 rr0, u32 rr1,
                                         u64 &c0, u64 &c1, u64 &c2, u64 &pn, u64 &vn, u64 &bn)
{
    const u64 dp = p1 + (2 * FP_P) - p0, dv = v1 + (2 * FP_P) - v0, db = b1 + (2 * FP_P) - b0;
    c0 = wred(wmul(p0, v0) + b0);
    c1 = wred(wmul(p1, v1) + b1);
    c2 = wmul(wred(dp), wred(dv));
    pn = wlin1(p0, dp, rr0, rr1);
    vn = wlin1(v0, dv, rr0, rr1);
    bn = wlin1(b0, db, rr0, rr1);
}

// Round k on two folded triples held by one thread, summed into the
// thread's shared-memory slots hs[3j..3j+2].
__device__ __forceinline__ void gen_pair_acc(u64 p0, u64 p1, u64 v0, u64 v1, u64 b0, u64 b1, u32 rr0, u32 rr1,
                                             GenSmem &sm, u32 j, u64 &pn, u64 &vn, u64 &bn)
{
    u64 c0, c1, c2;
    gen_pair(p0, p1, v0, v1, b0, b1, rr0, rr1, c0, c1, c2, pn, vn, bn);
    const u32 t = threadIdx.x;
    sm.hs[3 * j][t] = wred(sm.hs[3 * j][t] + c0);
    sm.hs[3 * j + 1][t] = wred(sm.hs[3 * j + 1][t] + c1);
    sm.hs[3 * j + 2][t] = wred(sm.hs[3 * j + 2][t] + c2);
}

// Rounds 0..R-1 of N = 2^R entries held by one thread; adds to h[0..3R) and
// leaves the folded values in p[0], v[0], b[0].
template <int R>
__device__ __forceinline__ void gen_regs(u64 (&p)[1 << R], u64 (&v)[1 << R], u64 (&b)[1 << R], const GenSmem &sm,
                                         u64 (&h)[15])
{
#pragma unroll
    for (int k = 0; k < R; k++) {
        acc128 a0, a1, a2;
        acc_zero(a0);
        acc_zero(a1);
        acc_zero(a2);
        const u32 rr0 = sm.r[k][0], rr1 = sm.r[k][1];
#pragma unroll
        for (int q = 0; q < (1 << (R - k - 1)); q++) {
            const u64 p0 = p[2 * q], p1 = p[2 * q + 1], v0 = v[2 * q], v1 = v[2 * q + 1];
            const u64 b0 = b[2 * q], b1 = b[2 * q + 1];
            const u64 dp = p1 + (2 * FP_P) - p0, dv = v1 + (2 * FP_P) - v0, db = b1 + (2 * FP_P) - b0;
            mac(a0, p0, v0);
            mac(a1, p1, v1);
            mac(a2, wred(dp), wred(dv));  // leading coefficient (see gen_pair)
            acc_add(a0, b0);
            acc_add(a1, b1);
            p[q] = wlin1(p0, dp, rr0, rr1);
            v[q] = wlin1(v0, dv, rr0, rr1);
            b[q] = wlin1(b0, db, rr0, rr1);
        }
        h[3 * k] = wred(h[3 * k] + acc_red(a0));
        h[3 * k + 1] = wred(h[3 * k + 1] + acc_red(a1));
        h[3 * k + 2] = wred(h[3 * k + 2] + acc_red(a2));
    }
}

// Rounds 0 and 1 of the first wave of a TREE phase-2 instance on the 4
// entries at x0 (gates g = x0/2 and x0/2 + 1 of layer i).  P and B vanish at
// odd entries and P[2g] = eq(r_P, g) = w, B[2g] = w V[2g+1], so round 0 needs
// per gate only w: its message is c0 = sum w (v0 + v1), c1 = 0 and leading
// coefficient c2 = -sum w (v1 - v0), and the folds are P' = (1 - r_0) w,
// V' = V folded, B' = (1 - r_0) w v1.  The common factor 1 - r_0 of P' and B'
// is left out here: it multiplies the message of every later round of the
// instance and is applied in the final reduction.  h[2] collects the c2 sum
// with its sign flipped (restored by the caller).
__device__ __forceinline__ void tree2_run(const Globals &G, const GenWave &W, u64 x0, const GenSmem &sm,
                                          u64 (&h)[15], u64 &pn, u64 &vn, u64 &bn)
{
    const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(W.inV + x0);
    const ulonglong2 va = __ldg(sv), vb = __ldg(sv + 1);
    const EqTab &T = G.layers[W.layer].trp;
    const u64 wa = eq_at(T, x0 >> 1), wb = eq_at(T, (x0 >> 1) + 1);
    const u64 da = va.y + (2 * FP_P) - va.x, db = vb.y + (2 * FP_P) - vb.x;  // below 2^62.6
    acc128 s, t;
    acc_zero(s);
    acc_zero(t);
    mac(s, wa, va.x + va.y);  // operands below 2^62 + 16
    mac(s, wb, vb.x + vb.y);
    mac(t, wa, da);
    mac(t, wb, db);
    h[0] = wred(h[0] + acc_red(s));
    h[2] = wred(h[2] + acc_red(t));
    const u32 a0 = sm.r[0][0], a1 = sm.r[0][1];
    const u64 v0 = wlin1(va.x, da, a0, a1), v1 = wlin1(vb.x, db, a0, a1);
    const u64 b0 = wmul(wa, va.y), b1 = wmul(wb, vb.y);
    u64 c0, c1, c2;
    gen_pair(wa, wb, v0, v1, b0, b1, sm.r[1][0], sm.r[1][1], c0, c1, c2, pn, vn, bn);
    h[3] = wred(h[3] + c0);
    h[4] = wred(h[4] + c1);
    h[5] = wred(h[5] + c2);
}

// Rounds 0 and 1 of the first wave of a SQUARE phase-2 instance on the 4
// entries at x0: P[x] = eq(r_P, x) V[x] and B = 0, so the B terms drop out.
__device__ __forceinline__ void sq2_run(const Globals &G, const GenWave &W, u64 x0, const GenSmem &sm, u64 (&h)[15],
                                        u64 &pn, u64 &vn)
{
    const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(W.inV + x0);
    const ulonglong2 va = __ldg(sv), vb = __ldg(sv + 1);
    const EqTab &T = G.layers[W.layer].trp;
    u64 v[4] = {va.x, va.y, vb.x, vb.y}, p[4];
#pragma unroll
    for (int q = 0; q < 4; q++) p[q] = wmul(eq_at(T, x0 + q), v[q]);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        acc128 a0, a1, a2;
        acc_zero(a0);
        acc_zero(a1);
        acc_zero(a2);
        const u32 rr0 = sm.r[k][0], rr1 = sm.r[k][1];
#pragma unroll
        for (int q = 0; q < (2 >> k); q++) {
            const u64 p0 = p[2 * q], p1 = p[2 * q + 1], v0 = v[2 * q], v1 = v[2 * q + 1];
            const u64 dp = p1 + (2 * FP_P) - p0, dv = v1 + (2 * FP_P) - v0;
            mac(a0, p0, v0);
            mac(a1, p1, v1);
            mac(a2, wred(dp), wred(dv));
            p[q] = wlin1(p0, dp, rr0, rr1);
            v[q] = wlin1(v0, dv, rr0, rr1);
        }
        h[3 * k] = wred(h[3 * k] + acc_red(a0));
        h[3 * k + 1] = wred(h[3 * k + 1] + acc_red(a1));
        h[3 * k + 2] = wred(h[3 * k + 2] + acc_red(a2));
    }
    pn = p[0];
    vn = v[0];
}

// In-register rounds for e in 3..5: runs of 4 entries (rounds 0, 1), then
// rounds 2.. on the runs' folded triples, combined like a binary counter.
__device__ __forceinline__ void gen_regs_runs(const Globals &G, const GenWave &W, u64 x0, u32 e, bool hasB,
                                              GenSmem &sm, u64 (&h)[15], u64 &pv, u64 &vv, u64 &bv)
{
    const u32 nruns = 1u << (e - 2);
#pragma unroll
    for (int j = 0; j < 9; j++) sm.hs[j][threadIdx.x] = 0;
    u64 p0 = 0, v0 = 0, b0 = 0, p1 = 0, v1 = 0, b1 = 0, p2 = 0, v2 = 0, b2 = 0;  // pending: rounds 2, 3, 4
    u64 tp = 0, tv = 0, tb = 0;
    const bool tree2 = W.src == GS_TREE2;
    // a rolled loop keeps the kernel small (instruction-cache bound when unrolled)
#pragma unroll 1
    for (u32 sub = 0; sub < nruns; sub++) {
        if (sub + 1 < nruns) {
            const u64 xn = x0 + 4 * (sub + 1);
            prefetch_l1(W.inV + xn);
            if (W.src == GS_NONE) {
                prefetch_l1(W.inP + xn);
                if (hasB) prefetch_l1(W.inB + xn);
            }
        }
        if (tree2) {
            tree2_run(G, W, x0 + 4 * sub, sm, h, tp, tv, tb);
        } else if (W.src == GS_SQ2) {
            sq2_run(G, W, x0 + 4 * sub, sm, h, tp, tv);
            tb = 0;
        } else {
            u64 p[4], v[4], b[4];
            gen_load<4>(W, x0 + 4 * sub, hasB, p, v, b);
            gen_regs<2>(p, v, b, sm, h);
            tp = p[0];
            tv = v[0];
            tb = b[0];
        }
        if (!(sub & 1)) {  // wait for the partner run
            p0 = tp, v0 = tv, b0 = tb;
            continue;
        }
        gen_pair_acc(p0, tp, v0, tv, b0, tb, sm.r[2][0], sm.r[2][1], sm, 0, tp, tv, tb);
        if (nruns == 2) continue;
        if (!(sub & 2)) {
            p1 = tp, v1 = tv, b1 = tb;
            continue;
        }
        gen_pair_acc(p1, tp, v1, tv, b1, tb, sm.r[3][0], sm.r[3][1], sm, 1, tp, tv, tb);
        if (nruns == 4) continue;
        if (!(sub & 4)) {
            p2 = tp, v2 = tv, b2 = tb;
            continue;
        }
        gen_pair_acc(p2, tp, v2, tv, b2, tb, sm.r[4][0], sm.r[4][1], sm, 2, tp, tv, tb);
    }
    pv = tp;
    vv = tv;
    bv = tb;
    if (tree2) h[2] = wred((2 * FP_P) - h[2]);
#pragma unroll
    for (int j = 0; j < 9; j++) h[6 + j] = sm.hs[j][threadIdx.x];
}

// Sum over the lanes l = 0 mod 2^(kk+1) of a warp (the only lanes holding a
// contribution in cross round kk; the others hold 0), written by lane 0 to
// out[0..2].
__device__ __forceinline__ void gen_round_sum(u64 c0, u64 c1, u64 c2, u32 kk, u64 *out)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if ((u32)o < (2u << kk)) break;
        c0 = wred(c0 + __shfl_xor_sync(0xffffffffu, c0, o));
        c1 = wred(c1 + __shfl_xor_sync(0xffffffffu, c1, o));
        c2 = wred(c2 + __shfl_xor_sync(0xffffffffu, c2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        out[0] = c0;
        out[1] = c1;
        out[2] = c2;
    }
}

// Rounds off.. of a general chunk across threads (same placement as
// prod_cross: the first thread of each pair keeps the folded values).  The
// per-warp sums of round k go to sm.w[warp][3k..3k+2] (CTA-level rounds: warp
// 0's row, zeros in the other rows).
__device__ __forceinline__ void gen_cross(u64 &p, u64 &v, u64 &b, u32 off, u32 tid, u32 na, u32 nr, GenSmem &sm)
{
    const u32 lane = tid & 31, warp = tid >> 5;
    // rolled: one copy of the round body keeps the kernel small
#pragma unroll 1
    for (int kk = 0; kk < 5; kk++) {
        const u32 k = off + kk;
        if (k < nr) {
            const u32 d = 1u << kk;
            const u64 p1 = __shfl_down_sync(0xffffffffu, p, d);
            const u64 v1 = __shfl_down_sync(0xffffffffu, v, d);
            const u64 b1 = __shfl_down_sync(0xffffffffu, b, d);
            u64 c0 = 0, c1 = 0, c2 = 0;
            if ((tid & ((2u << kk) - 1)) == 0 && tid < na)
                gen_pair(p, p1, v, v1, b, b1, sm.r[k][0], sm.r[k][1], c0, c1, c2, p, v, b);
            gen_round_sum(c0, c1, c2, kk, &sm.w[warp][3 * k]);
        }
    }
    if (lane == 0) {
        sm.lvl[0][warp] = p;
        sm.lvl[1][warp] = v;
        sm.lvl[2][warp] = b;
        for (u32 k = off + 5; k < nr && k < off + 7; k++)
            if (warp) sm.w[warp][3 * k] = sm.w[warp][3 * k + 1] = sm.w[warp][3 * k + 2] = 0;
    }
    __syncthreads();
    if (off + 5 < nr && warp == 0) {
        const bool have = lane < WV_NT / 32;
        p = have ? sm.lvl[0][lane] : 0;
        v = have ? sm.lvl[1][lane] : 0;
        b = have ? sm.lvl[2][lane] : 0;
#pragma unroll
        for (int kk = 5; kk < 7; kk++) {
            const u32 k = off + kk;
            if (k < nr) {
                const u32 d = 1u << (kk - 5);
                const u64 p1 = __shfl_down_sync(0xffffffffu, p, d);
                const u64 v1 = __shfl_down_sync(0xffffffffu, v, d);
                const u64 b1 = __shfl_down_sync(0xffffffffu, b, d);
                const u32 t = lane << 5;
                u64 c0 = 0, c1 = 0, c2 = 0;
                if ((t & ((2u << kk) - 1)) == 0 && t < na)
                    gen_pair(p, p1, v, v1, b, b1, sm.r[k][0], sm.r[k][1], c0, c1, c2, p, v, b);
                gen_round_sum(c0, c1, c2, kk - 5, &sm.w[0][3 * k]);
            }
        }
        if (lane == 0) {
            sm.lvl[0][0] = p;
            sm.lvl[1][0] = v;
            sm.lvl[2][0] = b;
        }
    }
}

// One chunk of a GEN wave.
__device__ void gen_chunk(const Globals &G, const GenWave &W, u32 chunk, GenSmem &sm)
{
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 nr = W.nr, e = W.e;
    const u32 na = 1u << (nr - e);
    const u64 base = (u64)chunk << nr;
    const bool hasB = (W.flags & WF_HASB) != 0;
    if (tid < nr) limbs31(G.chal[W.chal_off + tid], sm.r[tid][0], sm.r[tid][1]);
    __syncthreads();
    u64 pv = 0, vv = 0, bv = 0;
    if (e > 0) {
        u64 h[15];
#pragma unroll
        for (int i = 0; i < 15; i++) h[i] = 0;
        if (tid < na) {
            const u64 x0 = base + ((u64)tid << e);
            gen_regs_runs(G, W, x0, e, hasB, sm, h, pv, vv, bv);
        }
        u64 h16[16];
#pragma unroll
        for (int i = 0; i < 16; i++) h16[i] = (i < 15) ? h[i] : 0;
        const u64 s = warp_sum16(h16);
        if ((lane & 1) == 0 && (lane >> 1) < 3 * e) sm.w[warp][lane >> 1] = s;
    } else if (tid < na) {
        const u64 x = base + tid;
        const bool ext = W.r0 == 0;
        vv = ld_in(W.inV + x, ext);
        if (W.src == GS_SQ2) {
            pv = wmul(eq_at(G.layers[W.layer].trp, x), vv);
        } else if (W.src == GS_TREE2) {
            const u64 w = (x & 1) ? 0 : eq_at(G.layers[W.layer].trp, x >> 1);
            pv = w;
            bv = (x & 1) ? 0 : wmul(w, ld_in(W.inV + x + 1, ext));
        } else {
            pv = ld_in(W.inP + x, ext);
            bv = hasB ? ld_in(W.inB + x, ext) : 0;
        }
    }
    gen_cross(pv, vv, bv, e, tid, na, nr, sm);
    __syncthreads();
    if (tid < 3 * nr) {
        const u64 sum = wred(sm.w[0][tid] + sm.w[1][tid] + sm.w[2][tid] + sm.w[3][tid]);
        const u32 k = tid / 3, t = tid % 3;
        W.part[((u64)k * W.nchunks + chunk) * 3 + t] = sum;
    }
    if (!(W.flags & WF_LAST) && tid == 0) {
        W.outP[chunk] = sm.lvl[0][0];
        W.outV[chunk] = sm.lvl[1][0];
        if (W.outB) W.outB[chunk] = sm.lvl[2][0];
    }
}

// ---- line reduction -----------------------------------------------------------------
// q(t) = V~_{i+1}(l(t)), folding V_{i+1} with coordinates a_k + b_k t in
// coefficient form (degree grows by one per folded coordinate):
//   out_c = A_c + a (B_c - A_c) + b (B_{c-1} - A_{c-1}),  c = 0 .. deg + 1.
// A first-wave chunk folds LN_E coordinates per thread in registers (2^LN_E
// consecutive entries) and the rest in shared memory; a later wave folds up
// to 7 coordinates of one polynomial per thread.

// One level of coefficient folding in registers: D+1 -> D+2 coefficients.
template <int D>
__device__ __forceinline__ void line_fold(const u64 (&A)[D + 1], const u64 (&B)[D + 1], u32 a0, u32 a1, u32 b0,
                                          u32 b1, u64 (&out)[D + 2])
{
    u64 d[D + 1];
#pragma unroll
    for (int c = 0; c <= D; c++) d[c] = B[c] + (2 * FP_P) - A[c];
    out[0] = wlin1(A[0], d[0], a0, a1);
#pragma unroll
    for (int c = 1; c <= D; c++) out[c] = wlin2(A[c], d[c], d[c - 1], a0, a1, b0, b1);
    out[D + 1] = wlin1(0, d[D], b0, b1);
}

// 8 consecutive entries -> one cubic (coordinates 0, 1, 2 of the run).
__device__ __forceinline__ void line_run8(const u64 *v, const u32 *la, const u32 *lb, u64 (&out)[4])
{
    u64 l1[4][2];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const u64 dd = v[2 * q + 1] + (2 * FP_P) - v[2 * q];
        l1[q][0] = wlin1(v[2 * q], dd, la[0], la[1]);
        l1[q][1] = wlin1(0, dd, lb[0], lb[1]);
    }
    u64 l2[2][3];
    line_fold<1>(l1[0], l1[1], la[2], la[3], lb[2], lb[3], l2[0]);
    line_fold<1>(l1[2], l1[3], la[2], la[3], lb[2], lb[3], l2[1]);
    line_fold<2>(l2[0], l2[1], la[4], la[5], lb[4], lb[5], out);
}

// Coefficient `c` of the fold of polynomials A, B (degree deg, W values).
__device__ __forceinline__ u64 line_coef(const u64 *A, const u64 *B, u32 deg, u32 c, const u32 *la, const u32 *lb)
{
    const u64 dc = (c <= deg) ? B[c] + (2 * FP_P) - A[c] : 0;
    const u64 dm = (c >= 1) ? B[c - 1] + (2 * FP_P) - A[c - 1] : 0;
    const u64 ac = (c <= deg) ? A[c] : 0;
    return wlin2(ac, dc, dm, la[0], la[1], lb[0], lb[1]);
}

// One chunk of one line wave, by the whole CTA.
__device__ void line_chunk(const Globals &G, const LineWaveDev &W, u32 chunk, LineSmem &sm)
{
    const u32 tid = threadIdx.x;
    if (tid < W.nl) {
        const u64 a = G.chal[W.a_off + W.l0 + tid];
        const u64 b = f_sub(G.chal[W.b_off + W.l0 + tid], a);
        limbs31(a, sm.la[tid][0], sm.la[tid][1]);
        limbs31(b, sm.lb[tid][0], sm.lb[tid][1]);
    }
    __syncthreads();
    u32 m, deg, k0;  // polynomials in bufA, their degree, coordinates already folded
    if (W.l0 == 0) {
        const u32 e = (W.nl >= LN_E) ? LN_E : 0;
        const u32 na = 1u << (W.nl - e);
        const u64 base = (u64)chunk << W.nl;
        if (tid < na) {
            if (e == LN_E) {
                const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(W.in + base + ((u64)tid << LN_E));
                u32 la[12], lb[12];
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    la[2 * k] = sm.la[k][0];
                    la[2 * k + 1] = sm.la[k][1];
                    lb[2 * k] = sm.lb[k][0];
                    lb[2 * k + 1] = sm.lb[k][1];
                }
                // eight runs of 8 entries (cubics over coordinates 0..2), combined
                // like a binary counter over coordinates 3, 4, 5; a rolled loop
                // keeps one copy of the run code
                u64 c0[4] = {0, 0, 0, 0}, q0[5] = {0, 0, 0, 0, 0};
                u64 s0[6] = {0, 0, 0, 0, 0, 0}, s1[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
                for (int run = 0; run < 8; run++) {
                    if (run < 7) prefetch_l1(src + 4 * (run + 1));
                    u64 v[8];
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const ulonglong2 w = __ldg(src + 4 * run + t);
                        v[2 * t] = w.x;
                        v[2 * t + 1] = w.y;
                    }
                    u64 c[4];
                    line_run8(v, la, lb, c);
                    if (!(run & 1)) {
#pragma unroll
                        for (int i = 0; i < 4; i++) c0[i] = c[i];
                        continue;
                    }
                    u64 q[5];
                    line_fold<3>(c0, c, la[6], la[7], lb[6], lb[7], q);
                    if (!(run & 2)) {
#pragma unroll
                        for (int i = 0; i < 5; i++) q0[i] = q[i];
                        continue;
                    }
                    u64 t5[6];
                    line_fold<4>(q0, q, la[8], la[9], lb[8], lb[9], t5);
#pragma unroll
                    for (int i = 0; i < 6; i++) {
                        if (run & 4) s1[i] = t5[i];
                        else s0[i] = t5[i];
                    }
                }
                u64 p[7];
                line_fold<5>(s0, s1, la[10], la[11], lb[10], lb[11], p);
#pragma unroll
                for (int c = 0; c < 7; c++) sm.bufA[tid * 7 + c] = p[c];
            } else {
                sm.bufA[tid] = __ldg(W.in + base + tid);
            }
        }
        m = na;
        deg = e;
        k0 = e;
    } else {
        // polynomials of degree l0 from the previous wave (written by other
        // CTAs of this launch when run as a tail: read through L2)
        const u32 din = W.l0, npoly = 1u << W.nl, half = npoly >> 1, C = din + 2;
        const u64 *in = W.in + ((u64)chunk << W.nl) * (din + 1);
        for (u32 idx = tid; idx < half * C; idx += WV_NT) {
            const u32 j = idx / C, c = idx - j * C;
            const u64 *A = in + (u64)(2 * j) * (din + 1), *B = A + (din + 1);
            const u64 dc = (c <= din) ? __ldcg(B + c) + (2 * FP_P) - __ldcg(A + c) : 0;
            const u64 dm = (c >= 1) ? __ldcg(B + c - 1) + (2 * FP_P) - __ldcg(A + c - 1) : 0;
            const u64 ac = (c <= din) ? __ldcg(A + c) : 0;
            sm.bufA[j * C + c] = wlin2(ac, dc, dm, sm.la[0][0], sm.la[0][1], sm.lb[0][0], sm.lb[0][1]);
        }
        m = half;
        deg = din + 1;
        k0 = 1;
    }
    __syncthreads();
    u64 *cur = sm.bufA, *nxt = sm.bufB;
    u32 k = k0;
    if (m == WV_NT && deg == LN_E && k + 5 <= W.nl) {
        // One polynomial per thread: the first five levels stay inside each
        // warp (its 32 polynomials -> 1) with no CTA barrier.  A warp works
        // in its own parts of the buffers: its level-0 inputs in bufA, then
        // alternately 256 entries of bufB and its bufA part; its result goes
        // past every warp's inputs, to bufA[1024 + warp (LN_E + 6)].
        const u32 warp = tid >> 5, lane = tid & 31;
        u64 *ownA = sm.bufA + warp * 32 * (LN_E + 1), *ownB = sm.bufB + warp * 256;
        const u64 *in = ownA;
        u32 cnt = 32, d = deg;
        for (u32 lv = 0; lv < 5; lv++, k++) {
            u64 *out = (lv == 4) ? sm.bufA + 1024 + warp * (LN_E + 6) : ((lv & 1) ? ownA : ownB);
            const u32 half = cnt >> 1, C = d + 2;
            for (u32 idx = lane; idx < half * C; idx += 32) {
                const u32 j = idx / C, c = idx - j * C;
                out[j * C + c] = line_coef(in + (2 * j) * (d + 1), in + (2 * j + 1) * (d + 1), d, c, sm.la[k], sm.lb[k]);
            }
            __syncwarp();
            in = out;
            cnt = half;
            d += 1;
        }
        __syncthreads();
        cur = sm.bufA + 1024;
        m = WV_NT / 32;
        deg = d;
    }
    for (; k < W.nl; k++) {
        const u32 half = m >> 1, C = deg + 2;
        for (u32 idx = tid; idx < half * C; idx += WV_NT) {
            const u32 j = idx / C, c = idx - j * C;
            nxt[j * C + c] =
                line_coef(cur + (2 * j) * (deg + 1), cur + (2 * j + 1) * (deg + 1), deg, c, sm.la[k], sm.lb[k]);
        }
        __syncthreads();
        u64 *t = cur;
        cur = nxt;
        nxt = t;
        m = half;
        deg += 1;
    }
    // cur[0..deg] is this chunk's polynomial
    if (!W.last) {
        u64 *out = W.out + (u64)chunk * (deg + 1);
        for (u32 c = tid; c <= deg; c += WV_NT) out[c] = cur[c];
    } else {
        // q(t) for t = 0..n by Horner; q(0) = V~_{i+1}(r1) feeds phase 3
        const u32 n = W.n;
        u64 *tr = G.tr + W.tr_q;
        for (u32 t = tid; t <= n; t += WV_NT) {
            u64 acc = cur[deg];
            for (int c = (int)deg - 1; c >= 0; c--) acc = wred(wmul(acc, (u64)t) + cur[c]);
            tr[t] = wcanon(acc);
        }
        if (tid == 0) G.scal[SCAL_V1(W.layer)] = wcanon(cur[0]);
    }
}

// ---- the persistent launch ------------------------------------------------------------

// After a chunk of a wave with a tail: count the chunk; the CTA that counts
// the last one returns true (and resets the counter for the next proof).
__device__ __forceinline__ bool wave_done(u32 *counter, u32 nchunks, u32 &s_flag)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_flag = (atomicAdd(counter, 1u) == nchunks - 1) ? 1u : 0u;
    __syncthreads();
    const bool last = s_flag != 0;
    if (last) {
        __threadfence();
        if (threadIdx.x == 0) *counter = 0;
    }
    return last;
}

extern __shared__ __align__(16) unsigned char wv_dyn[];

#ifndef WV_MINB
#define WV_MINB 4  // resident CTAs per SM the register allocation is sized for (4: 128 registers)
#endif

__global__ void __launch_bounds__(WV_NT, WV_MINB) k_waves(const Globals *Gs, const LineWaveDev *lw, const ProdWave *pw,
                                                   const GenWave *gw, const Task *tasks, int ntasks, u32 *ctr)
{
    WaveSmem &sm = *reinterpret_cast<WaveSmem *>(wv_dyn);
    __shared__ int s_task;
    __shared__ u32 s_flag;
    // the final reduction may begin its launch on SMs this launch frees as it
    // drains (it waits for the whole launch before it reads what it wrote)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (;;) {
        __syncthreads();  // the previous task is done with shared memory
        if (threadIdx.x == 0) s_task = (int)atomicAdd(&ctr[0], 1u);
        __syncthreads();
        const int ti = s_task;
        if (ti >= ntasks) break;
        const Task tk = tasks[ti];
        if (tk.type == TK_LINE) {
            const LineWaveDev &W = lw[tk.wave];
            const Globals &G = Gs[W.circ];
            line_chunk(G, W, tk.chunk, sm.line);
            if (W.tail && wave_done(W.counter, W.nchunks, s_flag)) line_chunk(G, lw[tk.wave + 1], 0, sm.line);
        } else if (tk.type == TK_PROD) {
            const ProdWave &W = pw[tk.wave];
            const Globals &G = Gs[W.circ];
            prod_chunk(G, W, tk.chunk, sm.prod);
            if ((W.flags & WF_TAIL) && wave_done(W.counter, W.nchunks, s_flag)) {
                __syncthreads();
                prod_chunk(G, pw[tk.wave + 1], 0, sm.prod);
            }
        } else {
            const GenWave &W = gw[tk.wave];
            const Globals &G = Gs[W.circ];
            gen_chunk(G, W, tk.chunk, sm.gen);
            if ((W.flags & WF_TAIL) && wave_done(W.counter, W.nchunks, s_flag)) {
                __syncthreads();
                gen_chunk(G, gw[tk.wave + 1], 0, sm.gen);
            }
        }
    }
    // the CTA that exits last resets the task counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctr[1], 1u) == gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
        }
    }
}

// Shared-memory size of the wave launch (called outside stream capture).
void waves_init()
{
    device_sms();
    cudaFuncSetAttribute(k_waves, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WaveSmem));
}

void launch_waves(const Globals *Gs, const LineWaveDev *lw, const ProdWave *pw, const GenWave *gw, const Task *tasks,
                  int ntasks, u32 *ctr, cudaStream_t st)
{
    if (ntasks <= 0) return;
    const int sms = device_sms();
    const int grid = std::min(ntasks, sms * WV_MINB);
    k_waves<<<grid, WV_NT, sizeof(WaveSmem), st>>>(Gs, lw, pw, gw, tasks, ntasks, ctr);
}

// --------------------------------------------------------------------------------
// Final reduction into the transcript.  Rounds with more than
// FINAL_WARP_MIN chunk partials (they come first in the round list) are
// summed by a warp each; the rest, the great majority in a batch of small
// circuits, by a thread each.  The round's scalars then turn the sums into
// g(0), g(1), g(2).
// --------------------------------------------------------------------------------

// The scalars a round's message needs besides its partial sums (loaded
// before the sums, so that both sets of loads are in flight together).
struct RoundScalars {
    u64 ez, ch, v1, es, kap, c0, c1;
};

// Everything but v1 (the coin launch wrote it all before the wave launch).
__device__ __forceinline__ RoundScalars round_scalars_pre(const RoundRef &R)
{
    RoundScalars S{};
    S.ez = *R.ez;
    if (R.defer || R.kind < PK_GEN_FIRST) S.ch = *R.ch;
    if (R.kind < PK_GEN_FIRST) {
        S.es = *R.esum;
        S.kap = *R.kap;
        S.c0 = R.lc[0];
        S.c1 = R.lc[1];
    }
    return S;
}

// g(0), g(1), g(2) of round R from its canonical partial sums h, written to
// the circuit's transcript.
__device__ __forceinline__ void final_round(const Globals *Gs, const RoundRef &R, const RoundScalars &S,
                                            const u64 (&h)[3])
{
    const bool gen = R.kind >= PK_GEN_FIRST;
    const u64 ez = S.ez;
    u64 g0, g1, g2;
    if (gen) {
        u64 sg = (R.kind == PK_GEN_TAB) ? 1 : ez;
        if (R.defer) sg = f_mul(sg, f_sub(1, S.ch));  // TREE phase 2: 1 - r_0 left out of P, B
        g0 = f_mul(sg, h[0]);
        g1 = f_mul(sg, h[1]);
        // h[2] is the leading coefficient: value at 2 = 2 h1 - h0 + 2 h2
        g2 = f_mul(sg, f_add(f_sub(f_add(h[1], h[1]), h[0]), f_add(h[2], h[2])));
    } else {
        const u64 v1 = S.v1, ch = S.ch, es = S.es, kap = S.kap, c0 = S.c0, c1 = S.c1;
        u64 sigma = 1, c2u = 0;
        if (R.kind == PK_TREE3) {
            sigma = f_mul(ez, f_sub(1, ch));
            c2u = v1;
        } else if (R.kind == PK_SQ3) {
            sigma = f_mul(ez, v1);
        }
        const u64 h0 = f_add(h[0], f_mul(c2u, es)), h1 = f_add(h[1], f_mul(c2u, es));
        const u64 kj = f_mul(sigma, kap);
        g0 = f_mul(kj, f_mul(c0, h0));
        g1 = f_mul(kj, f_mul(c1, h1));
        g2 = f_mul(kj, f_mul(f_sub(f_add(c1, c1), c0), f_sub(f_add(h1, h1), h0)));
    }
    u64 *tr = Gs[R.circ].tr;
    tr[R.tr_pos] = g0;
    tr[R.tr_pos + 1] = g1;
    tr[R.tr_pos + 2] = g2;
}

__global__ void __launch_bounds__(256) k_final(Globals *Gs, const RoundRef *rounds, int nrounds, int nbig,
                                               const u32 *outs, int nouts)
{
    const u32 lane = threadIdx.x & 31;
    const u64 gt = blockIdx.x * (u64)blockDim.x + threadIdx.x, nthreads = (u64)gridDim.x * blockDim.x;
    // launched early (programmatic dependence on the wave launch): the first
    // round's descriptor and coin-launch scalars are loaded before waiting
    // for the waves; v1 and the partials only after
    const u64 gw0 = gt >> 5;
    RoundRef R0{};
    RoundScalars S0{};
    if (gw0 < (u64)nbig) {
        R0 = rounds[gw0];
        if (lane == 0) S0 = round_scalars_pre(R0);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (u64 gw = gw0; gw < (u64)nbig; gw += nthreads >> 5) {
        const RoundRef R = (gw == gw0) ? R0 : rounds[gw];
        RoundScalars S{};
        if (lane == 0) {
            S = (gw == gw0) ? S0 : round_scalars_pre(R);
            if (R.kind < PK_GEN_FIRST) S.v1 = *R.v1;  // written by the layer's line reduction
        }
        u64 h[3] = {0, 0, 0};
        if (R.kind >= PK_GEN_FIRST)
            warp_record_sums<3>(R.part_pos, R.nchunks, lane, h);
        else
            warp_record_sums<2>(R.part_pos, R.nchunks, lane, h);
        if (lane == 0) final_round(Gs, R, S, h);
    }
    for (u64 t = gt; t < (u64)(nrounds - nbig); t += nthreads) {
        const RoundRef R = rounds[nbig + t];
        RoundScalars S = round_scalars_pre(R);
        if (R.kind < PK_GEN_FIRST) S.v1 = *R.v1;
        const u32 nv = R.kind >= PK_GEN_FIRST ? 3 : 2;
        u64 h[3] = {0, 0, 0};
        for (u32 q = 0; q < R.nchunks; q++)
            for (u32 v = 0; v < nv; v++) h[v] = wred(h[v] + R.part_pos[(u64)q * nv + v]);
        for (u32 v = 0; v < 3; v++) h[v] = wcanon(h[v]);
        final_round(Gs, R, S, h);
    }
    // the outputs open each transcript: a CTA per circuit (grid-stride over
    // the circuits), its threads over the outputs; the proof's in-place input
    // pointer is cleared (later evaluations read the input layer)
    for (int j = blockIdx.x; j < nouts; j += gridDim.x) {
        Globals &G = Gs[outs[j]];
        if (threadIdx.x == 0) G.in = nullptr;
        const u64 n = G.S0;
        const u64 *__restrict__ src = G.out_src;
        u64 *__restrict__ dst = G.tr;
        for (u64 x = threadIdx.x; x < n; x += blockDim.x) dst[x] = src[x];
    }
}

void launch_final(Globals *Gs, const RoundRef *rounds, int nrounds, int nbig, const u32 *outs, int nouts,
                  cudaStream_t st)
{
    const u64 warp_blocks = ((u64)nbig * 32 + 255) / 256, thread_blocks = ((u64)(nrounds - nbig) + 255) / 256;
    u64 blocks = warp_blocks > thread_blocks ? warp_blocks : thread_blocks;
    if (blocks < (u64)nouts) blocks = (u64)nouts;
    if (blocks < 64) blocks = 64;
    if (blocks > (u64)device_sms() * 8) blocks = (u64)device_sms() * 8;
    // programmatic dependence: the launch may begin while the wave launch
    // drains (k_final waits for it with griddepcontrol.wait)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_final, Gs, rounds, nrounds, nbig, outs, nouts);
}
