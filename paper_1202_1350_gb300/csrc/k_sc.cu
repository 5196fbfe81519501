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
//    P(t)V(t) at t = 0, 1, 2.  The first wave builds P and B from the wiring on
//    the fly (SQUARE, TREE phase 2) or reads tables built by k_build23.
//
// Arithmetic is lazy: table values stay in W = [0, 2^61 + 8), products
// accumulate exactly in 128 bits and are reduced once per round per thread;
// only transcript entries are made canonical.
#include <cuda_runtime.h>
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

// --------------------------------------------------------------------------------
// PROD: per-wave weight tables (computed once per proof, shared by all CTAs)
// --------------------------------------------------------------------------------

// Linear factor L_m of a product-weighted instance, from the coins.
__device__ __forceinline__ void prod_factor(const Globals &G, const SciDev &S, u32 m, u64 &c0, u64 &c1)
{
    const LayerDev &L = G.layers[S.layer];
    const u64 *rP = G.chal + L.chal_off, *r1 = rP + L.s;
    switch (S.kind) {
    case PK_PH1: {
        const u64 z = G.pts[L.z_off + m];
        c0 = f_sub(1, z);
        c1 = z;
        break;
    }
    case PK_TREE3: {
        if (m == 0) {
            c0 = 0;
            c1 = 1;
        } else {
            const u64 a = rP[m - 1], b = r1[m];
            c0 = f_mul(f_sub(1, a), f_sub(1, b));
            c1 = f_mul(a, b);
        }
        break;
    }
    default: {  // PK_SQ3
        const u64 a = rP[m], b = r1[m];
        c0 = f_mul(f_sub(1, a), f_sub(1, b));
        c1 = f_mul(a, b);
        break;
    }
    }
}

// One CTA per PROD wave.  Writes the wave's weight block
//   Q_k(q) = prod_{m=k+1}^{e-1} L_{r0+m}(bit_{m-k-1} q)      k < e          (in-thread rounds)
//   E_k(y) = prod_{m=k+1}^{nr-1} L_{r0+m}(bit_{m-k-1} y)     k = kb..nr-1   (per-thread / in-CTA rounds)
//   outer lo / hi: split table of prod_{m >= r0+nr} L_m over the chunk index,
// and, for the first wave of an SCI, its factors, kappa_j (without sigma) and
// esum_j = prod_{m>j} (c0_m + c1_m).
__global__ void __launch_bounds__(256) k_prep_prod(const Globals *Gs, const SciDev *scis, const ProdWave *waves)
{
    const ProdWave &W = waves[blockIdx.x];
    const Globals &G = Gs[W.circ];
    const SciDev &S = scis[W.sci];
    __shared__ u64 c0[32], c1[32];
    const u32 tid = threadIdx.x;
    if (tid < S.n) prod_factor(G, S, tid, c0[tid], c1[tid]);
    __syncthreads();
    if (W.r0 == 0 && tid < 32) {
        // kappa_j = prod_{m<j} L_m(r_m), esum_j = prod_{m>j} (c0_m + c1_m): warp scans
        const u32 j = tid;
        const bool in = j < S.n;
        const u64 a = in ? f_add(c0[j], f_mul(G.chal[S.chal_off + j], f_sub(c1[j], c0[j]))) : 1;
        const u64 b = in ? f_add(c0[j], c1[j]) : 1;
        u64 pre = __shfl_up_sync(0xffffffffu, warp_scan_mul(a), 1);
        u64 suf = __shfl_down_sync(0xffffffffu, warp_rscan_mul(b), 1);
        if (j == 0) pre = 1;
        if (j == 31) suf = 1;
        if (in) {
            S.Lc[2 * j] = c0[j];
            S.Lc[2 * j + 1] = c1[j];
            S.kap[j] = pre;
            S.esum[j] = suf;
        }
    }
    const u32 e = W.e, nr = W.nr, r0 = W.r0;
    u64 *blk = W.wblk;
    // Q block
    for (u32 idx = tid; idx + 1 < (1u << e); idx += blockDim.x) {
        u32 k = 0;
        while (idx >= (1u << e) - (1u << (e - k - 1))) k++;
        const u32 q = idx - ((1u << e) - (1u << (e - k)));
        u64 v = 1;
        for (u32 m = k + 1; m < e; m++) v = f_mul(v, ((q >> (m - k - 1)) & 1) ? c1[r0 + m] : c0[r0 + m]);
        blk[idx] = v;
    }
    // E block
    const u32 kb = e ? e - 1 : 0;
    u64 *E = blk + ((1u << e) - 1);
    const u32 esize = (1u << (nr - kb)) - 1;
    for (u32 idx = tid; idx < esize; idx += blockDim.x) {
        u32 k = kb;
        while (idx >= (1u << (nr - kb)) - (1u << (nr - k - 1))) k++;
        const u32 y = idx - ((1u << (nr - kb)) - (1u << (nr - k)));
        u64 v = 1;
        for (u32 m = k + 1; m < nr; m++) v = f_mul(v, ((y >> (m - k - 1)) & 1) ? c1[r0 + m] : c0[r0 + m]);
        E[idx] = v;
    }
    // outer split tables
    u64 *olo = E + esize;
    const u32 o0 = r0 + nr, no = W.no, ho = W.ho;
    u64 *ohi = olo + (1u << ho);
    for (u32 j = tid; j < (1u << ho); j += blockDim.x) {
        u64 v = 1;
        for (u32 m = 0; m < ho; m++) v = f_mul(v, ((j >> m) & 1) ? c1[o0 + m] : c0[o0 + m]);
        olo[j] = v;
    }
    for (u32 j = tid; j < (1u << (no - ho)); j += blockDim.x) {
        u64 v = 1;
        for (u32 m = 0; m < no - ho; m++) v = f_mul(v, ((j >> m) & 1) ? c1[o0 + ho + m] : c0[o0 + ho + m]);
        ohi[j] = v;
    }
}

void launch_prep_prod(const Globals *Gs, const SciDev *scis, const ProdWave *waves, int nwaves, cudaStream_t st)
{
    if (nwaves > 0) k_prep_prod<<<nwaves, 256, 0, st>>>(Gs, scis, waves);
}

// --------------------------------------------------------------------------------
// PROD waves
// --------------------------------------------------------------------------------

#define PR_NT 128
#define PR_SUB 16  // a thread's 2^PR_M entries are processed as runs of PR_SUB

// Rounds OFF.. of a product-weighted chunk across threads.  Thread t holds
// level value t (t < na); a round pairs values 2y and 2y+1, which sit in the
// threads t = y 2^(kk+1) and t + 2^kk, and the first of them keeps the folded
// value, so rounds stay inside a warp for kk < 5 (shuffles) and continue in
// warp 0 after one exchange through shared memory.  Each active thread adds
// E_k(y) u0 and E_k(y) u1 to hv[2 kk], hv[2 kk + 1].
__device__ __forceinline__ void prod_cross(u64 (&hv)[16], u64 uv, u32 off, u32 tid, u32 na, u32 nr,
                                           const u64 *s_E, u32 eoff0, const u32 (*s_r)[2], u64 *s_lvl)
{
    const u32 lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int kk = 0; kk < 5; kk++) {
        const u32 k = off + kk;
        if (k < nr) {  // uniform
            const u64 u1 = __shfl_down_sync(0xffffffffu, uv, 1u << kk);
            if ((tid & ((2u << kk) - 1)) == 0 && tid < na) {
                const u32 y = tid >> (kk + 1);
                const u64 w = s_E[eoff0 - (1u << (nr - k)) + y];
                hv[2 * kk] = wmul(w, uv);
                hv[2 * kk + 1] = wmul(w, u1);
                uv = wfold(uv, u1, s_r[k][0], s_r[k][1]);
            }
        }
    }
    if (lane == 0) s_lvl[warp] = uv;
    __syncthreads();
    if (off + 5 < nr && warp == 0) {
        uv = (lane < PR_NT / 32) ? s_lvl[lane] : 0;
#pragma unroll
        for (int kk = 5; kk < 7; kk++) {
            const u32 k = off + kk;
            if (k < nr) {
                const u64 u1 = __shfl_down_sync(0xffffffffu, uv, 1u << (kk - 5));
                const u32 t = lane << 5;  // the thread index this lane stands for
                if ((t & ((2u << kk) - 1)) == 0 && t < na) {
                    const u32 y = t >> (kk + 1);
                    const u64 w = s_E[eoff0 - (1u << (nr - k)) + y];
                    hv[2 * kk] = wmul(w, uv);
                    hv[2 * kk + 1] = wmul(w, u1);
                    uv = wfold(uv, u1, s_r[k][0], s_r[k][1]);
                }
            }
        }
        if (lane == 0) s_lvl[0] = uv;
    }
}

// Rounds 0..3 of one run of 16 entries (run index sub within the thread):
// pair weights Q_k(q), q = pair index + (sub << (3 - k)); adds the sums to
// hv[2k], hv[2k+1] and returns the folded value.
__device__ __forceinline__ u64 prod_run16(u64 (&u)[16], u32 sub, const u64 *s_Q, const u32 (*s_r)[2], u64 (&hv)[12])
{
#pragma unroll
    for (int k = 0; k < 4; k++) {
        acc128 a0, a1, b0, b1;  // two chains per value for instruction-level parallelism
        acc_zero(a0);
        acc_zero(a1);
        acc_zero(b0);
        acc_zero(b1);
        const u32 rr0 = s_r[k][0], rr1 = s_r[k][1];
        const u32 qoff = (1u << PR_M) - (1u << (PR_M - k)) + (sub << (3 - k));
#pragma unroll
        for (int q = 0; q < (8 >> k); q++) {
            const u64 w = s_Q[qoff + q];
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
        hv[2 * k] = wred(hv[2 * k] + acc_red(a0) + acc_red(b0));
        hv[2 * k + 1] = wred(hv[2 * k + 1] + acc_red(a1) + acc_red(b1));
    }
    return u[0];
}

// Sum over the CTA's warps of per-warp round sums s_w[warp][i] (W values).
__device__ __forceinline__ u64 cta_sum4(const u64 (*s_w)[32], u32 i)
{
    return wred(s_w[0][i] + s_w[1][i] + s_w[2][i] + s_w[3][i]);
}

__global__ void __launch_bounds__(PR_NT, 4) k_sc_prod(const Globals *Gs, const ProdWave *waves, const Item *items)
{
    constexpr int M = PR_M;
    __shared__ u32 s_r[32][2];
    __shared__ u64 s_Q[1 << M];
    __shared__ u64 s_E[256];
    __shared__ u64 s_lvl[PR_NT / 32];
    __shared__ u64 s_w[PR_NT / 32][32];
    __shared__ u64 s_echunk;

    const Item it = items[blockIdx.x];
    const ProdWave &W = waves[it.wave];
    const Globals &G = Gs[W.circ];
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 nr = W.nr, e = W.e, chunk = it.chunk;
    const u32 na = 1u << (nr - e);
    const u64 base = (u64)chunk << nr;
    if (tid < nr) limbs31(G.chal[W.chal_off + tid], s_r[tid][0], s_r[tid][1]);
    const u64 *blk = W.wblk;
    const u32 qsize = (1u << e) - 1;
    const u32 kb = e ? e - 1 : 0;
    const u32 esize = (1u << (nr - kb)) - 1;
    if (tid < qsize) s_Q[tid] = blk[tid];
    for (u32 k = tid; k < esize; k += PR_NT) s_E[k] = blk[qsize + k];
    if (tid == 0) {
        const u64 *olo = blk + qsize + esize;
        const u64 *ohi = olo + (1u << W.ho);
        s_echunk = f_mul(olo[chunk & ((1u << W.ho) - 1)], ohi[chunk >> W.ho]);
    }
    __syncthreads();

    const u32 eoff0 = 1u << (nr - kb);
    u64 uv = 0;  // the thread's level value after its in-register rounds
    u64 hv[16];  // cross-thread rounds: hv[2 kk + t]
#pragma unroll
    for (int i = 0; i < 16; i++) hv[i] = 0;
    if (e == M) {
        // rounds 0..M-1 in registers: four runs of 16 entries (rounds 0..3
        // each), then rounds 4 and 5 on the runs' folded values
        u64 h0[12];
#pragma unroll
        for (int i = 0; i < 12; i++) h0[i] = 0;
        if (tid < na) {
            const u64 *src = W.in + base + ((u64)tid << M);
            const u32 q4 = (1u << M) - 4, q5 = (1u << M) - 2;
            u64 f0 = 0, g0 = 0;
            // a rolled loop keeps the kernel small (instruction-cache bound when unrolled)
#pragma unroll 1
            for (u32 sub = 0; sub < 4; sub++) {
                u64 u[16];
                const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(src + sub * PR_SUB);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const ulonglong2 t = sv[q];
                    u[2 * q] = t.x;
                    u[2 * q + 1] = t.y;
                }
                const u64 fs = prod_run16(u, sub, s_Q, s_r, h0);
                if (sub & 1) {
                    // round 4 on runs (sub-1, sub); round 5 on the two results
                    const u64 w = s_Q[q4 + (sub >> 1)];
                    h0[8] = wred(h0[8] + wmul(w, f0));
                    h0[9] = wred(h0[9] + wmul(w, fs));
                    const u64 g = wfold(f0, fs, s_r[4][0], s_r[4][1]);
                    if (sub == 1) {
                        g0 = g;
                    } else {
                        const u64 w5 = s_Q[q5];
                        h0[10] = wmul(w5, g0);
                        h0[11] = wmul(w5, g);
                        uv = wfold(g0, g, s_r[5][0], s_r[5][1]);
                    }
                } else {
                    f0 = fs;
                }
            }
            const u64 T = s_E[tid];  // E_{M-1}(tid): the weight of the chunk bits above the thread's run
#pragma unroll
            for (int i = 0; i < 12; i++) h0[i] = wmul(T, h0[i]);
        }
        // per-warp sums of the in-register rounds
        u64 h16[16];
#pragma unroll
        for (int i = 0; i < 16; i++) h16[i] = (i < 12) ? h0[i] : 0;
        const u64 s = warp_sum16(h16);
        if ((lane & 1) == 0 && (lane >> 1) < 12) s_w[warp][lane >> 1] = s;
        prod_cross(hv, uv, M, tid, na, nr, s_E, eoff0, s_r, s_lvl);
    } else {
        if (tid < na) uv = W.in[base + tid];
        prod_cross(hv, uv, 0, tid, na, nr, s_E, eoff0, s_r, s_lvl);
    }
    // per-warp sums of the cross-thread rounds (after the register rounds' 12 slots when e = M)
    {
        const u64 s = warp_sum16(hv);
        const u32 o = e ? 12 : 0;
        if ((lane & 1) == 0 && (lane >> 1) < 2 * (nr - e) && (lane >> 1) < 14) s_w[warp][o + (lane >> 1)] = s;
    }
    __syncthreads();
    if (tid < 2 * nr) {
        const u64 sum = cta_sum4(s_w, tid);
        const u32 k = tid >> 1, t = tid & 1;
        W.part[((u64)k * W.nchunks + chunk) * 2 + t] = wmul(sum, s_echunk);
    }
    if (!(W.flags & WF_LAST) && tid == 0) W.out[chunk] = s_lvl[0];
}

void launch_sc_prod(const Globals *Gs, const ProdWave *waves, const Item *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_sc_prod<<<nitems, PR_NT, 0, st>>>(Gs, waves, items);
}

// --------------------------------------------------------------------------------
// GEN waves: tables P, V, B folded every round; message values at t = 0, 1, 2.
// --------------------------------------------------------------------------------

#define GN_NT 128

// P and B of the first wave for the on-the-fly kinds, for the run of 8
// entries at x0 whose V values are v[].
__device__ __forceinline__ void gen_source(const Globals &G, const GenWave &W, u64 x0, const u64 (&v)[8],
                                           u64 (&p)[8], u64 (&b)[8])
{
    const LayerDev &L = G.layers[W.layer];
    if (W.src == GS_SQ2) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
            p[q] = wmul(eq_at(L.trp, x0 + q), v[q]);
            b[q] = 0;
        }
    } else {  // GS_TREE2
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const u64 w = eq_at(L.trp, (x0 + q) >> 1);
            p[q] = w;
            b[q] = wmul(w, v[q + 1]);
            p[q + 1] = 0;
            b[q + 1] = 0;
        }
    }
}

// One general pair: message contributions at t = 0, 1, 2 and the folds.
__device__ __forceinline__ void gen_pair(u64 p0, u64 p1, u64 v0, u64 v1, u64 b0, u64 b1, u32 rr0, u32 rr1,
                                         u64 &c0, u64 &c1, u64 &c2, u64 &pn, u64 &vn, u64 &bn)
{
    c0 = wred(wmul(p0, v0) + b0);
    c1 = wred(wmul(p1, v1) + b1);
    c2 = wred(wmul(wext2(p1, p0), wext2(v1, v0)) + wext2(b1, b0));
    pn = wfold(p0, p1, rr0, rr1);
    vn = wfold(v0, v1, rr0, rr1);
    bn = wfold(b0, b1, rr0, rr1);
}

// Rounds off.. of a general chunk across threads (same placement as
// prod_cross: the first thread of each pair keeps the folded values).
__device__ __forceinline__ void gen_cross(u64 (&hv)[21], u64 &p, u64 &v, u64 &b, u32 off, u32 tid, u32 na, u32 nr,
                                          const u32 (*s_r)[2], u64 (*s_lvl)[GN_NT / 32])
{
    const u32 lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int kk = 0; kk < 5; kk++) {
        const u32 k = off + kk;
        if (k < nr) {
            const u32 d = 1u << kk;
            const u64 p1 = __shfl_down_sync(0xffffffffu, p, d);
            const u64 v1 = __shfl_down_sync(0xffffffffu, v, d);
            const u64 b1 = __shfl_down_sync(0xffffffffu, b, d);
            if ((tid & ((2u << kk) - 1)) == 0 && tid < na)
                gen_pair(p, p1, v, v1, b, b1, s_r[k][0], s_r[k][1], hv[3 * kk], hv[3 * kk + 1], hv[3 * kk + 2], p,
                         v, b);
        }
    }
    if (lane == 0) {
        s_lvl[0][warp] = p;
        s_lvl[1][warp] = v;
        s_lvl[2][warp] = b;
    }
    __syncthreads();
    if (off + 5 < nr && warp == 0) {
        const bool have = lane < GN_NT / 32;
        p = have ? s_lvl[0][lane] : 0;
        v = have ? s_lvl[1][lane] : 0;
        b = have ? s_lvl[2][lane] : 0;
#pragma unroll
        for (int kk = 5; kk < 7; kk++) {
            const u32 k = off + kk;
            if (k < nr) {
                const u32 d = 1u << (kk - 5);
                const u64 p1 = __shfl_down_sync(0xffffffffu, p, d);
                const u64 v1 = __shfl_down_sync(0xffffffffu, v, d);
                const u64 b1 = __shfl_down_sync(0xffffffffu, b, d);
                const u32 t = lane << 5;
                if ((t & ((2u << kk) - 1)) == 0 && t < na)
                    gen_pair(p, p1, v, v1, b, b1, s_r[k][0], s_r[k][1], hv[3 * kk], hv[3 * kk + 1], hv[3 * kk + 2],
                             p, v, b);
            }
        }
        if (lane == 0) {
            s_lvl[0][0] = p;
            s_lvl[1][0] = v;
            s_lvl[2][0] = b;
        }
    }
}

// Cross-thread rounds from round off, then the per-warp sums of their
// message values into s_w[warp][off * 3 ..] (after the register rounds' slots).
__device__ __forceinline__ void gen_cross_sum(u64 &p, u64 &v, u64 &b, u32 off, u32 tid, u32 na, u32 nr,
                                              const u32 (*s_r)[2], u64 (*s_lvl)[GN_NT / 32], u64 (*s_w)[40])
{
    u64 hv[32];
#pragma unroll
    for (int i = 0; i < 32; i++) hv[i] = 0;
    gen_cross(reinterpret_cast<u64(&)[21]>(hv), p, v, b, off, tid, na, nr, s_r, s_lvl);
    const u64 s = warp_sum32(hv);
    const u32 lane = tid & 31;
    if (lane < 3 * (nr - off) && lane < 21) s_w[tid >> 5][3 * off + lane] = s;
}

// Rounds 0..2 of one run of 8 entries; adds to h[0..8] and leaves the folded
// values in p[0], v[0], b[0].
__device__ __forceinline__ void gen_run8(u64 (&p)[8], u64 (&v)[8], u64 (&b)[8], const u32 (*s_r)[2], u64 (&h)[15])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        acc128 a0, a1, a2;
        acc_zero(a0);
        acc_zero(a1);
        acc_zero(a2);
        const u32 rr0 = s_r[k][0], rr1 = s_r[k][1];
#pragma unroll
        for (int q = 0; q < (4 >> k); q++) {
            const u64 p0 = p[2 * q], p1 = p[2 * q + 1], v0 = v[2 * q], v1 = v[2 * q + 1];
            const u64 b0 = b[2 * q], b1 = b[2 * q + 1];
            mac(a0, p0, v0);
            mac(a1, p1, v1);
            mac(a2, wext2(p1, p0), wext2(v1, v0));
            acc_add(a0, b0);
            acc_add(a1, b1);
            acc_add(a2, wext2(b1, b0));
            p[q] = wfold(p0, p1, rr0, rr1);
            v[q] = wfold(v0, v1, rr0, rr1);
            b[q] = wfold(b0, b1, rr0, rr1);
        }
        h[3 * k] = wred(h[3 * k] + acc_red(a0));
        h[3 * k + 1] = wred(h[3 * k + 1] + acc_red(a1));
        h[3 * k + 2] = wred(h[3 * k + 2] + acc_red(a2));
    }
}

// Round k (3 or 4) on two folded triples held by one thread.
__device__ __forceinline__ void gen_pair_acc(u64 p0, u64 p1, u64 v0, u64 v1, u64 b0, u64 b1, u32 rr0, u32 rr1,
                                             u64 *h, u64 &pn, u64 &vn, u64 &bn)
{
    u64 c0, c1, c2;
    gen_pair(p0, p1, v0, v1, b0, b1, rr0, rr1, c0, c1, c2, pn, vn, bn);
    h[0] = wred(h[0] + c0);
    h[1] = wred(h[1] + c1);
    h[2] = wred(h[2] + c2);
}

__global__ void __launch_bounds__(GN_NT, 4) k_sc_gen(const Globals *Gs, const GenWave *waves, const Item *items)
{
    constexpr int M = GN_M;
    __shared__ u32 s_r[32][2];
    __shared__ u64 s_lvl[3][GN_NT / 32];
    __shared__ u64 s_w[GN_NT / 32][40];

    const Item it = items[blockIdx.x];
    const GenWave &W = waves[it.wave];
    const Globals &G = Gs[W.circ];
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 nr = W.nr, e = W.e, chunk = it.chunk;
    const u32 na = 1u << (nr - e);
    const u64 base = (u64)chunk << nr;
    const bool hasB = (W.flags & WF_HASB) != 0;
    if (tid < nr) limbs31(G.chal[W.chal_off + tid], s_r[tid][0], s_r[tid][1]);
    __syncthreads();

    u64 pv = 0, vv = 0, bv = 0;
    if (e == M) {
        // rounds 0..4 in registers: four runs of 8 entries (rounds 0..2
        // each), round 3 on pairs of runs, round 4 on the two results
        u64 h0[15];
#pragma unroll
        for (int i = 0; i < 15; i++) h0[i] = 0;
        if (tid < na) {
            u64 fp = 0, fv = 0, fb = 0, gp = 0, gv = 0, gb = 0;
            // a rolled loop keeps the kernel small (instruction-cache bound when unrolled)
#pragma unroll 1
            for (u32 sub = 0; sub < 4; sub++) {
                u64 p[8], v[8], b[8];
                const u64 x0 = base + ((u64)tid << M) + 8 * sub;
                const ulonglong2 *sv = reinterpret_cast<const ulonglong2 *>(W.inV + x0);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const ulonglong2 t = sv[q];
                    v[2 * q] = t.x;
                    v[2 * q + 1] = t.y;
                }
                if (W.src != GS_NONE) {
                    gen_source(G, W, x0, v, p, b);
                } else {
                    const ulonglong2 *sp = reinterpret_cast<const ulonglong2 *>(W.inP + x0);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const ulonglong2 t = sp[q];
                        p[2 * q] = t.x;
                        p[2 * q + 1] = t.y;
                    }
                    if (hasB) {
                        const ulonglong2 *sb = reinterpret_cast<const ulonglong2 *>(W.inB + x0);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const ulonglong2 t = sb[q];
                            b[2 * q] = t.x;
                            b[2 * q + 1] = t.y;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; q++) b[q] = 0;
                    }
                }
                gen_run8(p, v, b, s_r, h0);
                if (sub & 1) {
                    u64 np, nv, nb;
                    gen_pair_acc(fp, p[0], fv, v[0], fb, b[0], s_r[3][0], s_r[3][1], h0 + 9, np, nv, nb);
                    if (sub == 1) {
                        gp = np;
                        gv = nv;
                        gb = nb;
                    } else {
                        gen_pair_acc(gp, np, gv, nv, gb, nb, s_r[4][0], s_r[4][1], h0 + 12, pv, vv, bv);
                    }
                } else {
                    fp = p[0];
                    fv = v[0];
                    fb = b[0];
                }
            }
        }
        u64 h16[16];
#pragma unroll
        for (int i = 0; i < 16; i++) h16[i] = (i < 15) ? h0[i] : 0;
        const u64 s = warp_sum16(h16);
        if ((lane & 1) == 0 && (lane >> 1) < 15) s_w[warp][lane >> 1] = s;
        gen_cross_sum(pv, vv, bv, M, tid, na, nr, s_r, s_lvl, s_w);
    } else {
        if (tid < na) {
            const u64 x = base + tid;
            vv = W.inV[x];
            if (W.src == GS_SQ2) {
                pv = wmul(eq_at(G.layers[W.layer].trp, x), vv);
                bv = 0;
            } else if (W.src == GS_TREE2) {
                const u64 w = (x & 1) ? 0 : eq_at(G.layers[W.layer].trp, x >> 1);
                pv = w;
                bv = (x & 1) ? 0 : wmul(w, W.inV[x + 1]);
            } else {
                pv = W.inP[x];
                bv = hasB ? W.inB[x] : 0;
            }
        }
        gen_cross_sum(pv, vv, bv, 0, tid, na, nr, s_r, s_lvl, s_w);
    }
    __syncthreads();
    if (tid < 3 * nr) {
        const u64 sum = wred(s_w[0][tid] + s_w[1][tid] + s_w[2][tid] + s_w[3][tid]);
        const u32 k = tid / 3, t = tid % 3;
        W.part[((u64)k * W.nchunks + chunk) * 3 + t] = sum;
    }
    if (!(W.flags & WF_LAST) && tid == 0) {
        W.outP[chunk] = s_lvl[0][0];
        W.outV[chunk] = s_lvl[1][0];
        if (W.outB) W.outB[chunk] = s_lvl[2][0];
    }
}

void launch_sc_gen(const Globals *Gs, const GenWave *waves, const Item *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_sc_gen<<<nitems, GN_NT, 0, st>>>(Gs, waves, items);
}

// --------------------------------------------------------------------------------
// Final reduction into the transcript: a warp per round sums the chunks'
// partials; the round's scalars turn the sums into g(0), g(1), g(2).
// --------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_final(const Globals *Gs, const SciDev *scis, const RoundRef *rounds,
                                               int nrounds, const u32 *outs, int nouts)
{
    const u32 lane = threadIdx.x & 31;
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 gw = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; gw < (u64)nrounds; gw += nwarps) {
        const RoundRef R = rounds[gw];
        const SciDev &S = scis[R.sci];
        const Globals &G = Gs[S.circ];
        const u32 nv = (S.kind >= PK_GEN_FIRST) ? 3 : 2;
        u64 h[3];
        for (u32 t = 0; t < nv; t++) {
            u64 s = 0;
            for (u32 q = lane; q < R.nchunks; q += 32) s = wred(s + R.part_pos[(u64)q * nv + t]);
            h[t] = wcanon(warp_wsum(s));
        }
        if (lane == 0) {
            const LayerDev &L = G.layers[S.layer];
            const u64 ez = G.scal[SCAL_EQZRP(S.layer)], v1 = G.scal[SCAL_V1(S.layer)];
            u64 g0, g1, g2;
            if (nv == 3) {
                const u64 sg = (S.kind == PK_GEN_TAB) ? 1 : ez;
                g0 = f_mul(sg, h[0]);
                g1 = f_mul(sg, h[1]);
                g2 = f_mul(sg, h[2]);
            } else {
                u64 sigma = 1, c2u = 0;
                if (S.kind == PK_TREE3) {
                    sigma = f_mul(ez, f_sub(1, G.chal[L.chal_off + L.s]));
                    c2u = v1;
                } else if (S.kind == PK_SQ3) {
                    sigma = f_mul(ez, v1);
                }
                const u32 j = R.j;
                const u64 es = S.esum[j];
                const u64 h0 = f_add(h[0], f_mul(c2u, es)), h1 = f_add(h[1], f_mul(c2u, es));
                const u64 kj = f_mul(sigma, S.kap[j]);
                const u64 c0 = S.Lc[2 * j], c1 = S.Lc[2 * j + 1];
                g0 = f_mul(kj, f_mul(c0, h0));
                g1 = f_mul(kj, f_mul(c1, h1));
                g2 = f_mul(kj, f_mul(f_sub(f_add(c1, c1), c0), f_sub(f_add(h1, h1), h0)));
            }
            G.tr[R.tr_pos] = g0;
            G.tr[R.tr_pos + 1] = g1;
            G.tr[R.tr_pos + 2] = g2;
        }
    }
    // the outputs open each transcript
    const u64 gid = blockIdx.x * (u64)blockDim.x + threadIdx.x, gstride = (u64)gridDim.x * blockDim.x;
    for (int j = 0; j < nouts; j++) {
        const Globals &G = Gs[outs[j]];
        const u64 n = G.S0;
        const u64 *__restrict__ src = G.layers[0].V;
        u64 *__restrict__ dst = G.tr;
        for (u64 x = gid; x < n; x += gstride) dst[x] = src[x];
    }
}

void launch_final(const Globals *Gs, const SciDev *scis, const RoundRef *rounds, int nrounds, const u32 *outs,
                  int nouts, cudaStream_t st)
{
    u64 blocks = ((u64)nrounds * 32 + 255) / 256;
    if (blocks < 64) blocks = 64;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_final<<<(unsigned)blocks, 256, 0, st>>>(Gs, scis, rounds, nrounds, outs, nouts);
}
