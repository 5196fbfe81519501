// k_pergate.cu -- the paper's per-gate prover (Sec. 4.1.1; memory access in
// Sec. 5.1.4), kept as a second prover path: same transcript as the folding
// prover, computed the way the paper's GPU prover computes it.
//
// Every message of layer i is a sum of independent per-gate contributions: in
// round k a thread per gate g (in-neighbours a, b read or computed from the
// index) adds the term of the layer polynomial whose Boolean coordinates are
// g's own bits,
//   phase 1 (bits of p):   eq(z_i, (r_<k, t, g_>k)) eq((r_<k, t), g_<=k) op(V[a], V[b])
//   phase 2 (bits of w1):  eq(z_i, r_P) eq(r_P, g) eq((r1_<j, t), a_<=j) op(V~(r1_<j, t, a_>j), V[b])
//   phase 3 (bits of w2):  eq(z_i, r_P) eq(r_P, g) eq(r1, a) eq((r2_<j, t), b_<=j) op(V~(r1), V~(r2_<j, t, b_>j))
// so each gate does a handful of field operations per round and the work of a
// layer is O(S log S).  The eq factors come from prefix tables that double
// every round (eq over the bound coordinates) and from suffix tables of z_i
// (phase 1); the partially bound values V~(r_<j, x) are the value table
// folded once per round.  Layers are independent given the coins, so round r
// of every layer runs in the same launch.  The line polynomial q(t) =
// V~_{i+1}(l(t)), t = 0..s_{i+1}, is evaluated point by point: an eq table of
// l(t) (split in two halves) dotted with V_{i+1}.
#include <cuda_runtime.h>

#include "plan.h"

#define PG_NT 256
#define PG_GPT 4  // gates (line: entries) per thread

// Sum of three W values over the CTA; thread 0 gets the totals.
__device__ __forceinline__ void cta_sum3(u64 &c0, u64 &c1, u64 &c2)
{
    __shared__ u64 s[3][PG_NT / 32];
    c0 = warp_wsum(c0);
    c1 = warp_wsum(c1);
    c2 = warp_wsum(c2);
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = c0;
        s[1][w] = c1;
        s[2][w] = c2;
    }
    __syncthreads();
    if (w == 0) {
        c0 = lane < PG_NT / 32 ? s[0][lane] : 0;
        c1 = lane < PG_NT / 32 ? s[1][lane] : 0;
        c2 = lane < PG_NT / 32 ? s[2][lane] : 0;
        c0 = warp_wsum(c0);
        c1 = warp_wsum(c1);
        c2 = warp_wsum(c2);
    }
    __syncthreads();
}

// Adds a gate's term times e_t(bit) = eq(t, bit) = (1 - bit, bit, 3 bit - 1) at
// t = 0, 1, 2 to c_t: bit 0 -> (x1, 0, -x2), bit 1 -> (0, x1, 2 x2), where x1
// is the rest of the term at t = bit and x2 at t = 2.
__device__ __forceinline__ void add_terms(u32 bit, u64 x1, u64 x2, u64 &c0, u64 &c1, u64 &c2)
{
    if (bit) {
        c1 = wred(c1 + x1);
        c2 = wred(c2 + 2 * x2);
    } else {
        c0 = wred(c0 + x1);
        c2 = wred(c2 + (2 * FP_P) - x2);
    }
}

// Setup: phase-1 suffix tables of every layer and the prefix tables' first
// entries.  suf_k (round k) holds prod_{m>k} eq(z_m, bit_{m-k-1} y) for
// y < 2^(s-k-1), stored at offset 2^(s-k-1) - 1.
__global__ void __launch_bounds__(PG_NT) k_pg_setup(const Globals *G, const PgLayer *pl, int nl)
{
    const u64 gid = blockIdx.x * (u64)PG_NT + threadIdx.x, gs = (u64)gridDim.x * PG_NT;
    for (int li = 0; li < nl; li++) {
        const PgLayer &Q = pl[li];
        const LayerDev &L = G->layers[Q.layer];
        const u64 *z = G->pts + L.z_off;
        if (gid == 0) {
            Q.preP[0] = 1;
            Q.preA[0] = 1;
            Q.preB[0] = 1;
        }
        if (Q.s == 0) continue;
        const u64 total = (1ull << Q.s) - 1;
        for (u64 e = gid; e < total; e += gs) {
            const u32 lv = 63 - __clzll(e + 1);  // table of size 2^lv
            const u32 k = Q.s - 1 - lv;
            const u64 y = e - ((1ull << lv) - 1);
            u64 v = 1;
            for (u32 m = 0; m < lv; m++) {
                const u64 zm = z[k + 1 + m];
                v = f_mul(v, ((y >> m) & 1) ? zm : f_sub(1, zm));
            }
            Q.suf[e] = v;
        }
    }
}

// Round r of every layer that has one: per-gate contributions, summed per CTA.
__global__ void __launch_bounds__(PG_NT) k_pg_gates(const Globals *G, const PgLayer *pl, const u32 *blk_layer, u32 r)
{
    const PgLayer &Q = pl[blk_layer[blockIdx.x]];
    if (r >= Q.n) return;  // uniform over the CTA
    const LayerDev &L = G->layers[Q.layer];
    const u64 S = 1ull << Q.s;
    const u64 *Vn = L.Vn;
    u64 c0 = 0, c1 = 0, c2 = 0;
    const u64 base = (u64)(blockIdx.x - Q.blk0) * (PG_NT * PG_GPT) + threadIdx.x;
    if (r < Q.s) {
        const u32 k = r;
        const u64 *suf = Q.suf + ((1ull << (Q.s - k - 1)) - 1);
        const u64 lo = (1ull << k) - 1;
#pragma unroll
        for (int q = 0; q < PG_GPT; q++) {
            const u64 g = base + (u64)q * PG_NT;
            if (g < S) {
                u64 a, b;
                u32 mul;
                gate_wiring(L, g, a, b, mul);
                const u64 x = Vn[a], y = Vn[b];
                const u64 val = mul ? wmul(x, y) : wred(x + y);
                const u64 wv = wmul(wmul(Q.preP[g & lo], suf[g >> (k + 1)]), val);
                add_terms((u32)(g >> k) & 1, wv, wv, c0, c1, c2);
            }
        }
    } else {
        const bool ph2 = r < Q.s + Q.sn;
        const u32 j = ph2 ? r - Q.s : r - Q.s - Q.sn;
        const u64 *F = (j == 0) ? Vn : ((j & 1) ? Q.fa : Q.fb);
        const u64 lo = (1ull << j) - 1;
        const u64 v1 = ph2 ? 0 : *Q.v1;
#pragma unroll
        for (int q = 0; q < PG_GPT; q++) {
            const u64 g = base + (u64)q * PG_NT;
            if (g < S) {
                u64 a, b;
                u32 mul;
                gate_wiring(L, g, a, b, mul);
                const u64 x = ph2 ? a : b;  // the in-neighbour whose bits are being bound
                const u64 h = x >> (j + 1);
                const u64 f0 = F[2 * h], f1 = F[2 * h + 1];
                const u32 bit = (u32)(x >> j) & 1;
                const u64 ft = bit ? f1 : f0, f2 = wred(2 * f1 + (2 * FP_P) - f0);
                u64 w, vt, v2;
                if (ph2) {
                    const u64 y = Vn[b];
                    w = wmul(Q.preP[g], Q.preA[a & lo]);
                    vt = mul ? wmul(ft, y) : wred(ft + y);
                    v2 = mul ? wmul(f2, y) : wred(f2 + y);
                } else {
                    w = wmul(wmul(Q.preP[g], Q.preA[a]), Q.preB[b & lo]);
                    vt = mul ? wmul(v1, ft) : wred(v1 + ft);
                    v2 = mul ? wmul(v1, f2) : wred(v1 + f2);
                }
                add_terms(bit, wmul(w, vt), wmul(w, v2), c0, c1, c2);
            }
        }
    }
    cta_sum3(c0, c1, c2);
    if (threadIdx.x == 0) {
        u64 *part = Q.part + (u64)(blockIdx.x - Q.blk0) * 3;
        part[0] = c0;
        part[1] = c1;
        part[2] = c2;
    }
}

// After round r: CTA li < nl writes layer li's round-r message (sum of the
// partials times the round's scalar factor); the other CTAs prepare round
// r + 1: the prefix table of the phase doubles with the round's challenge and
// (phases 2, 3) the value table folds with it.
__global__ void __launch_bounds__(PG_NT) k_pg_step(const Globals *G, const PgLayer *pl, int nl, u32 r)
{
    if ((int)blockIdx.x < nl) {
        const PgLayer &Q = pl[blockIdx.x];
        if (r >= Q.n) return;
        const LayerDev &L = G->layers[Q.layer];
        u64 c0 = 0, c1 = 0, c2 = 0;
        for (u32 k = threadIdx.x; k < Q.nblk; k += PG_NT) {
            c0 = wred(c0 + Q.part[3 * k]);
            c1 = wred(c1 + Q.part[3 * k + 1]);
            c2 = wred(c2 + Q.part[3 * k + 2]);
        }
        cta_sum3(c0, c1, c2);
        if (threadIdx.x == 0) {
            const u64 *rr = G->chal + L.chal_off;
            u64 f0, f1, f2;
            if (r < Q.s) {  // prod_{m<k} eq(z_m, r_m) eq(z_k, t)
                const u64 *z = G->pts + L.z_off;
                u64 cz = 1;
                for (u32 m = 0; m < r; m++) cz = f_mul(cz, f_add(f_mul(z[m], rr[m]), f_mul(f_sub(1, z[m]), f_sub(1, rr[m]))));
                const u64 zk = z[r];
                f0 = f_mul(cz, f_sub(1, zk));
                f1 = f_mul(cz, zk);
                f2 = f_mul(cz, f_sub(f_add(zk, f_add(zk, zk)), 1));
            } else {
                f0 = f1 = f2 = G->scal[SCAL_EQZRP(Q.layer)];
            }
            u64 *tr = G->tr + L.tr_msg + 3ull * r;
            tr[0] = f_mul(f0, wcanon(c0));
            tr[1] = f_mul(f1, wcanon(c1));
            tr[2] = f_mul(f2, wcanon(c2));
        }
        return;
    }
    const u64 gid = (blockIdx.x - nl) * (u64)PG_NT + threadIdx.x, gs = (u64)(gridDim.x - nl) * PG_NT;
    for (int li = 0; li < nl; li++) {
        const PgLayer &Q = pl[li];
        if (r >= Q.n) continue;
        const LayerDev &L = G->layers[Q.layer];
        const u64 ch = G->chal[L.chal_off + r];
        const u64 ch0 = f_sub(1, ch);
        u32 j;
        u64 *pre;
        if (r < Q.s) {
            j = r;
            pre = Q.preP;
        } else if (r < Q.s + Q.sn) {
            j = r - Q.s;
            pre = Q.preA;
        } else {
            j = r - Q.s - Q.sn;
            pre = Q.preB;
        }
        const u64 half = 1ull << j;
        for (u64 x = gid; x < half; x += gs) {  // in place: pairs (x, x + 2^j)
            const u64 v = pre[x];
            pre[x] = f_mul(v, ch0);
            pre[x + half] = f_mul(v, ch);
        }
        if (r < Q.s) continue;
        const u64 *F = (j == 0) ? L.Vn : ((j & 1) ? Q.fa : Q.fb);
        u64 *Fo = ((j + 1) & 1) ? Q.fa : Q.fb;
        const u64 nout = 1ull << (Q.sn - j - 1);
        u32 c0l, c1l;
        limbs31(ch, c0l, c1l);
        for (u64 y = gid; y < nout; y += gs) {
            const u64 v = wcanon(wfold(F[2 * y], F[2 * y + 1], c0l, c1l));
            Fo[y] = v;
            if (nout == 1 && r == Q.s + Q.sn - 1) *Q.v1 = v;  // V~_{i+1}(r1)
        }
    }
}

// Line polynomials: the split eq tables of l(t) = r1 + t (r2 - r1) for every
// layer and t = 0..s_{i+1}: lo_t[x] over the low h = ceil(s/2) coordinates,
// hi_t[y] over the rest, each entry a direct product.
__global__ void __launch_bounds__(PG_NT) k_pg_line_tab(const Globals *G, const PgLayer *pl, int nl)
{
    const u64 gid = blockIdx.x * (u64)PG_NT + threadIdx.x, gs = (u64)gridDim.x * PG_NT;
    for (int li = 0; li < nl; li++) {
        const PgLayer &Q = pl[li];
        const LayerDev &L = G->layers[Q.layer];
        const u32 n = Q.sn, h = (n + 1) / 2;
        const u64 nlo = 1ull << h, nhi = 1ull << (n - h), per = nlo + nhi;
        const u64 *r1 = G->chal + L.chal_off + L.s, *r2 = r1 + n;
        for (u64 e = gid; e < (u64)(n + 1) * per; e += gs) {
            const u64 t = e / per, x = e - t * per;
            const bool low = x < nlo;
            const u64 idx = low ? x : x - nlo;
            const u32 m0 = low ? 0 : h, cnt = low ? h : n - h;
            u64 v = 1;
            for (u32 m = 0; m < cnt; m++) {
                const u64 l = f_add(r1[m0 + m], f_mul(t, f_sub(r2[m0 + m], r1[m0 + m])));
                v = f_mul(v, ((idx >> m) & 1) ? l : f_sub(1, l));
            }
            Q.ltab[e] = v;
        }
    }
}

// Partial sums of q(t) = sum_x V_{i+1}[x] lo_t[x_lo] hi_t[x_hi], per CTA of
// the layer's line blocks and per t.
__global__ void __launch_bounds__(PG_NT) k_pg_line(const Globals *G, const PgLayer *pl, const u32 *lblk_layer)
{
    const PgLayer &Q = pl[lblk_layer[blockIdx.x]];
    const LayerDev &L = G->layers[Q.layer];
    const u32 n = Q.sn, h = (n + 1) / 2;
    const u64 Sn = 1ull << n, nlo = 1ull << h, per = nlo + (1ull << (n - h));
    const u64 base = (u64)(blockIdx.x - Q.lblk0) * (PG_NT * PG_GPT) + threadIdx.x;
    u64 v[PG_GPT];
#pragma unroll
    for (int q = 0; q < PG_GPT; q++) {
        const u64 x = base + (u64)q * PG_NT;
        v[q] = x < Sn ? L.Vn[x] : 0;
    }
    for (u32 t = 0; t <= n; t++) {
        const u64 *lo = Q.ltab + t * per, *hi = lo + nlo;
        acc128 acc;
        acc_zero(acc);
#pragma unroll
        for (int q = 0; q < PG_GPT; q++) {
            const u64 x = base + (u64)q * PG_NT;
            if (x < Sn) mac(acc, wmul(lo[x & (nlo - 1)], hi[x >> h]), v[q]);
        }
        u64 s = acc_red(acc), d1 = 0, d2 = 0;
        cta_sum3(s, d1, d2);
        if (threadIdx.x == 0) Q.lpart[(u64)(blockIdx.x - Q.lblk0) * (n + 1) + t] = s;
    }
}

// q(t) of every layer into the transcript, and the outputs that open it.
__global__ void __launch_bounds__(PG_NT) k_pg_line_fin(const Globals *G, const PgLayer *pl, int nl)
{
    if ((int)blockIdx.x < nl) {
        const PgLayer &Q = pl[blockIdx.x];
        const LayerDev &L = G->layers[Q.layer];
        for (u32 t = 0; t <= Q.sn; t++) {
            u64 s = 0, d1 = 0, d2 = 0;
            for (u32 k = threadIdx.x; k < Q.lnblk; k += PG_NT) s = wred(s + Q.lpart[(u64)k * (Q.sn + 1) + t]);
            cta_sum3(s, d1, d2);
            if (threadIdx.x == 0) G->tr[L.tr_q + t] = wcanon(s);
        }
        return;
    }
    const u64 S0 = G->S0;
    const u64 gid = (blockIdx.x - nl) * (u64)PG_NT + threadIdx.x, gs = (u64)(gridDim.x - nl) * PG_NT;
    for (u64 x = gid; x < S0; x += gs) G->tr[x] = G->layers[0].V[x];
}

void launch_pergate(const Globals *G, const PgLayer *pl, int nl, const u32 *blk_layer, u32 nblk,
                    const u32 *lblk_layer, u32 nlblk, u32 nrounds, cudaStream_t st)
{
    if (nl <= 0) return;
    k_pg_setup<<<304, PG_NT, 0, st>>>(G, pl, nl);
    k_pg_line_tab<<<304, PG_NT, 0, st>>>(G, pl, nl);
    for (u32 r = 0; r < nrounds; r++) {
        k_pg_gates<<<nblk, PG_NT, 0, st>>>(G, pl, blk_layer, r);
        k_pg_step<<<nl + 304, PG_NT, 0, st>>>(G, pl, nl, r);
    }
    k_pg_line<<<nlblk, PG_NT, 0, st>>>(G, pl, lblk_layer);
    k_pg_line_fin<<<nl + 64, PG_NT, 0, st>>>(G, pl, nl);
}

u32 pergate_gpt() { return PG_GPT * PG_NT; }
