// k_coins.cu -- the verifier's coins and everything derived from them alone,
// in one launch: the challenges and layer points (Sec. 3.1: z_{i+1} is the
// point the line reduction moves to), the split eq tables of those points,
// and the factor tables of the product-weighted sum-checks.
//
// Every challenge is a function of the seed (challenge c = draw c + 1 of the
// splitmix64 stream, Sec. 3.1's "verifier picks at random", made
// reproducible), so each CTA derives the challenges its job needs itself and
// no CTA waits for another.  A draw equal to p is rejected and the stream
// shifts (probability 2^-61 per draw): each CTA checks all of its circuit's
// draws and then takes the shifted sequence the slow way.
#include <cuda_runtime.h>
#include "coins.cuh"

#define CN_NT 256

// Setup role: all challenges, all points, eq(z_i, r_P) per layer.
__device__ void coins_setup(const Globals &G, bool rej)
{
    if (!rej) {
        for (u32 c = threadIdx.x; c < G.nchal; c += blockDim.x) G.chal[c] = splitmix64_at(G.seed, (u64)c + 1) >> 3;
    } else if (threadIdx.x == 0) {
        u64 k = 1;
        for (u32 c = 0; c < G.nchal; c++) {
            u64 x;
            do { x = splitmix64_at(G.seed, k++) >> 3; } while (x == FP_P);
            G.chal[c] = x;
        }
    }
    const LayerDev *L = G.layers;
    for (u32 k = threadIdx.x; k < L[0].s; k += blockDim.x) G.pts[L[0].z_off + k] = chal_of(G, rej, k);
    for (u32 qi = threadIdx.x; qi < G.nz; qi += blockDim.x) {
        const u32 i = G.zmap[qi] >> 8, k = G.zmap[qi] & 0xFF;
        G.pts[((i + 1 < G.d) ? L[i + 1].z_off : G.zd_off) + k] = zcoord(G, rej, i + 1, k);
    }
    // eq(z_i, r_P): a warp per layer, a lane per coordinate (s_i <= 30)
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (u32 i = warp; i < G.d; i += blockDim.x >> 5) {
        u64 f = 1;
        if (lane < L[i].s) {
            const u64 z = zcoord(G, rej, i, lane), rp = chal_of(G, rej, L[i].chal_off + lane);
            f = f_add(f_mul(z, rp), f_mul(f_sub(1, z), f_sub(1, rp)));
        }
        f = warp_prod(f);
        if (lane == 0) G.scal[SCAL_EQZRP(i)] = f;
    }
}

// Eq-table role: lo[j] = prod_{k<h} eq(x_k, bit_k j), hi[j] = prod_{k<n-h}
// eq(x_{h+k}, bit_k j).  Each half is a product of two sub-tables over its
// low and high coordinates, built by direct products, so every entry costs
// one product.
__device__ void coins_eq(const Globals &G, bool rej, const EqJob &J)
{
    const EqTab &t = J.t;
    __shared__ u64 x[64], xm[64];
    __shared__ u64 sub[4][256];
    for (u32 k = threadIdx.x; k < t.n; k += blockDim.x) {
        x[k] = (J.src == EQ_SRC_CHAL) ? chal_of(G, rej, J.off + k) : zcoord(G, rej, J.layer, k);
        xm[k] = f_sub(1, x[k]);
    }
    __syncthreads();
    const u32 m[2] = {t.h, t.n - t.h};
    const u32 c0[2] = {0, t.h};
    for (u32 j = 0; j < 2; j++) {
        const u32 m1 = m[j] / 2, m2 = m[j] - m1;
        for (u32 e = threadIdx.x; e < (1u << m1) + (1u << m2); e += blockDim.x) {
            const bool lowp = e < (1u << m1);
            const u32 idx = lowp ? e : e - (1u << m1);
            const u32 cnt = lowp ? m1 : m2, off = c0[j] + (lowp ? 0 : m1);
            u64 v = 1;
            for (u32 k = 0; k < cnt; k++) v = f_mul(v, ((idx >> k) & 1) ? x[off + k] : xm[off + k]);
            sub[2 * j + (lowp ? 0 : 1)][idx] = v;
        }
    }
    __syncthreads();
    u64 *dst[2] = {t.lo, t.hi};
    for (u32 j = 0; j < 2; j++) {
        const u32 m1 = m[j] / 2;
        for (u32 e = threadIdx.x; e < (1u << m[j]); e += blockDim.x)
            dst[j][e] = f_mul(sub[2 * j][e & ((1u << m1) - 1)], sub[2 * j + 1][e >> m1]);
    }
}

// Linear factor L_m of a product-weighted instance, from the coins.
__device__ void prod_factor(const Globals &G, bool rej, const SciDev &S, u32 m, u64 &c0, u64 &c1)
{
    const LayerDev &L = G.layers[S.layer];
    const u32 rP = L.chal_off, r1 = L.chal_off + L.s;
    switch (S.kind) {
    case PK_PH1: {
        const u64 z = zcoord(G, rej, S.layer, m);
        c0 = f_sub(1, z);
        c1 = z;
        break;
    }
    case PK_TREE3: {
        if (m == 0) {
            c0 = 0;
            c1 = 1;
        } else {
            const u64 a = chal_of(G, rej, rP + m - 1), b = chal_of(G, rej, r1 + m);
            c0 = f_mul(f_sub(1, a), f_sub(1, b));
            c1 = f_mul(a, b);
        }
        break;
    }
    default: {  // PK_SQ3
        const u64 a = chal_of(G, rej, rP + m), b = chal_of(G, rej, r1 + m);
        c0 = f_mul(f_sub(1, a), f_sub(1, b));
        c1 = f_mul(a, b);
        break;
    }
    }
}

// Product-weight role, one PROD wave.  Writes the wave's weight block
//   Q_k(q) = prod_{m=k+1}^{e-1} L_{r0+m}(bit_{m-k-1} q)      k < e          (in-thread rounds)
//   E_k(y) = prod_{m=k+1}^{nr-1} L_{r0+m}(bit_{m-k-1} y)     k = kb..nr-1   (per-thread / in-CTA rounds)
//   outer lo / hi: split table of prod_{m >= r0+nr} L_m over the chunk index,
// and, for the first wave of an SCI, its factors, kappa_j (without sigma) and
// esum_j = prod_{m>j} (c0_m + c1_m).
__device__ void coins_prep(const Globals &G, bool rej, const SciDev &S, const ProdWave &W)
{
    __shared__ u64 c0[32], c1[32];
    const u32 tid = threadIdx.x;
    if (tid < S.n) prod_factor(G, rej, S, tid, c0[tid], c1[tid]);
    __syncthreads();
    if (W.r0 == 0 && tid < 32) {
        // kappa_j = prod_{m<j} L_m(r_m), esum_j = prod_{m>j} (c0_m + c1_m): warp scans
        const u32 j = tid;
        const bool in = j < S.n;
        const u64 r = in ? chal_of(G, rej, S.chal_off + j) : 0;
        const u64 a = in ? f_add(c0[j], f_mul(r, f_sub(c1[j], c0[j]))) : 1;
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
    for (u32 idx = tid; idx + 1 < (1u << e); idx += blockDim.x) {  // Q block
        u32 k = 0;
        while (idx >= (1u << e) - (1u << (e - k - 1))) k++;
        const u32 q = idx - ((1u << e) - (1u << (e - k)));
        u64 v = 1;
        for (u32 m = k + 1; m < e; m++) v = f_mul(v, ((q >> (m - k - 1)) & 1) ? c1[r0 + m] : c0[r0 + m]);
        blk[idx] = v;
    }
    const u32 kb = e ? e - 1 : 0;
    u64 *E = blk + ((1u << e) - 1);
    const u32 esize = (1u << (nr - kb)) - 1;
    for (u32 idx = tid; idx < esize; idx += blockDim.x) {  // E block
        u32 k = kb;
        while (idx >= (1u << (nr - kb)) - (1u << (nr - k - 1))) k++;
        const u32 y = idx - ((1u << (nr - kb)) - (1u << (nr - k)));
        u64 v = 1;
        for (u32 m = k + 1; m < nr; m++) v = f_mul(v, ((y >> (m - k - 1)) & 1) ? c1[r0 + m] : c0[r0 + m]);
        E[idx] = v;
    }
    u64 *olo = E + esize;  // outer split tables
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

// CTAs [0, ncirc): setup of circuit blockIdx; then one per eq job; then one
// per PROD wave.
__global__ void __launch_bounds__(CN_NT) k_coins(const Globals *Gs, int ncirc, const EqJob *eqjobs, int neq,
                                                 const SciDev *scis, const ProdWave *pw)
{
    int b = blockIdx.x;
    if (b < ncirc) {
        const Globals &G = Gs[b];
        coins_setup(G, draws_rejected(G));
        return;
    }
    b -= ncirc;
    if (b < neq) {
        const EqJob J = eqjobs[b];
        const Globals &G = Gs[J.circ];
        coins_eq(G, draws_rejected(G), J);
        return;
    }
    b -= neq;
    const ProdWave &W = pw[b];
    const Globals &G = Gs[W.circ];
    coins_prep(G, draws_rejected(G), scis[W.sci], W);
}

void launch_coins(const Globals *Gs, int ncirc, const EqJob *eqjobs, int neq, const SciDev *scis,
                  const ProdWave *pw, int npw, cudaStream_t st)
{
    const int grid = ncirc + neq + npw;
    if (grid > 0) k_coins<<<grid, CN_NT, 0, st>>>(Gs, ncirc, eqjobs, neq, scis, pw);
}
