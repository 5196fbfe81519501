// k_f2sp.cu -- the special-purpose non-interactive F2 protocol (outlined in
// Sec. 3.2; prover and verifier parallelisation in Sec. 4.2; memory access in
// Sec. 5.2; GPU results in Sec. 6.3).
//
// The frequency vector a (n = v h entries) is a v x h grid, a(x, y) at
// x h + y.  Row x is the polynomial f_x of degree < h with f_x(y) = a(x, y) at
// the nodes y = 0..h-1; the proof is s(Y) = sum_x f_x(Y)^2 at Y = 0..2h-2.
// The verifier keeps f_x(r) for a secret random r, accepts iff
// s(r) = sum_x f_x(r)^2 and answers F2 = sum_{y<h} s(y).
//
// Prover.  Every row is extended to h - 1 more points independently (the
// paper's per-row transform).  With the barycentric weights of the nodes,
//   f_x(h + j) = C_j sum_y b_y / (h + j - y),  b_y = a(x, y) w_y,
//   w_y = 1 / prod_{k != y} (y - k),  C_j = prod_{k<h} (h + j - k),
// so a row's extension is a Toeplitz product of b with the table of
// inverses 1/d, d = 1..2h-2: h (h - 1) multiply-adds per row, O(n h) in all,
// done directly (no FFT).  A CTA takes SP_RB rows: their b values and the whole
// inverse table sit in shared memory (the tiles are read in shared-memory
// order, so the grid's layout in HBM never costs coalescing: Sec. 5.2's
// column-major transpose is not needed); each thread owns four extension
// points of all its CTA's rows, accumulating 128-bit products, then squares
// and sums them over the rows.  A second launch sums the CTAs' column partials.
//
// Verifier.  A streaming pass per chunk of whole rows: f_x(r) = sum_y a(x, y)
// L_y(r) with the Lagrange basis at r computed once; at the end s(r) by the
// barycentric form over the 2h - 1 proof nodes.
#include <cuda_runtime.h>

#include "plan.h"

#define SP_NT 256
#define SP_RB 4   // rows per prover CTA
#define SP_PT 4   // extension points per thread per pass
#define SP_YT 1024  // y-tile of the rows' b values in shared memory

// prod_{k < cnt, k != skip} (m - k) for a canonical m (skip = cnt: no skip).
__device__ u64 node_prod(u64 m, u64 cnt, u64 skip)
{
    u64 v = 1;
    for (u64 k = 0; k < cnt; k++)
        if (k != skip) v = f_mul(v, f_sub(m, k % FP_P));
    return v;
}

// Tables of a node count h (every entry by a direct product):
//   w[y]  = 1 / prod_{k<h, k != y} (y - k),             y < h
//   C[j]  = prod_{k<h} (h + j - k),                      j < h - 1
//   iv[d] = 1 / d,                                       d < 2h - 1 (iv[0] unused)
//   w2[y] = 1 / prod_{k<2h-1, k != y} (y - k),           y < 2h - 1
__global__ void __launch_bounds__(SP_NT) k_sp_tables(u64 h, u64 *w, u64 *C, u64 *iv, u64 *w2)
{
    const u64 n2 = 2 * h - 1;
    const u64 total = h + (h - 1) + n2 + n2;
    for (u64 e = blockIdx.x * (u64)SP_NT + threadIdx.x; e < total; e += (u64)gridDim.x * SP_NT) {
        if (e < h) {
            w[e] = f_inv(node_prod(e, h, e));
        } else if (e < 2 * h - 1) {
            const u64 j = e - h;
            C[j] = node_prod(h + j, h, h);
        } else if (e < 2 * h - 1 + n2) {
            const u64 d = e - (2 * h - 1);
            iv[d] = d ? f_inv(d) : 0;
        } else {
            const u64 y = e - (2 * h - 1 + n2);
            w2[y] = f_inv(node_prod(y, n2, y));
        }
    }
}

// Column partials of the proof for the CTA's rows: part[cta][m], m < 2h - 1
// (m < h: sum of a(x, m)^2; m = h + j: sum of f_x(h + j)^2).
__global__ void __launch_bounds__(SP_NT, 2) k_sp_prove(const u64 *a, u64 v, u64 h, const u64 *w, const u64 *C,
                                                    const u64 *iv, u64 *part, u32 *status)
{
    extern __shared__ u64 sp_dyn[];
    const u64 n2 = 2 * h - 1;
    u64 *s_iv = sp_dyn;        // 2h - 1 entries
    u64 *s_b = sp_dyn + n2;    // SP_RB x SP_YT
    const u64 x0 = (u64)blockIdx.x * SP_RB;
    const u32 nrows = (u32)((v - x0) < SP_RB ? (v - x0) : SP_RB);
    u64 *out = part + (u64)blockIdx.x * n2;
    for (u64 d = threadIdx.x; d < n2; d += SP_NT) s_iv[d] = iv[d];
    // original columns, and the canonical check of the CTA's entries
    bool bad = false;
    for (u64 y = threadIdx.x; y < h; y += SP_NT) {
        u64 s = 0;
        for (u32 r = 0; r < nrows; r++) {
            const u64 val = a[(x0 + r) * h + y];
            bad |= val >= FP_P;
            s = wred(s + wmul(val, val));
        }
        out[y] = wcanon(s);
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicOr(status, ST_BAD_INPUT);
        return;
    }
    // extension points h + j, j < h - 1, four per thread per pass
    for (u64 j0 = 0; j0 < h - 1; j0 += (u64)SP_PT * SP_NT) {
        acc128 acc[SP_RB][SP_PT];
#pragma unroll
        for (int r = 0; r < SP_RB; r++)
#pragma unroll
            for (int q = 0; q < SP_PT; q++) acc_zero(acc[r][q]);
        for (u64 y0 = 0; y0 < h; y0 += SP_YT) {
            const u64 yt = (h - y0) < SP_YT ? (h - y0) : SP_YT;
            __syncthreads();  // the previous tile is consumed
            for (u64 e = threadIdx.x; e < (u64)SP_RB * yt; e += SP_NT) {
                const u32 r = (u32)(e / yt);
                const u64 y = e - (u64)r * yt;
                s_b[r * SP_YT + y] = (r < nrows) ? f_mul(a[(x0 + r) * h + y0 + y], w[y0 + y]) : 0;
            }
            __syncthreads();
            for (u64 y = 0; y < yt; y++) {
                u64 ivq[SP_PT];
#pragma unroll
                for (int q = 0; q < SP_PT; q++) {
                    const u64 j = j0 + threadIdx.x + (u64)q * SP_NT;
                    ivq[q] = (j < h - 1) ? s_iv[h + j - (y0 + y)] : 0;  // h + j - y >= 1
                }
#pragma unroll
                for (int r = 0; r < SP_RB; r++) {
                    const u64 b = s_b[r * SP_YT + y];
#pragma unroll
                    for (int q = 0; q < SP_PT; q++) mac(acc[r][q], b, ivq[q]);
                }
                if ((y & 31) == 31) {  // 32 products of canonical values on a W value stay below 2^128
#pragma unroll
                    for (int r = 0; r < SP_RB; r++)
#pragma unroll
                        for (int q = 0; q < SP_PT; q++) {
                            acc[r][q].lo = acc_red(acc[r][q]);
                            acc[r][q].hi = 0;
                        }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < SP_PT; q++) {
            const u64 j = j0 + threadIdx.x + (u64)q * SP_NT;
            if (j >= h - 1) continue;
            const u64 cj = C[j];
            u64 s = 0;
#pragma unroll
            for (int r = 0; r < SP_RB; r++) {
                const u64 f = wmul(cj, acc_red(acc[r][q]));
                s = wred(s + wmul(f, f));
            }
            out[h + j] = wcanon(s);
        }
    }
}

// proof[m] = sum over CTAs of part[cta][m].
__global__ void __launch_bounds__(SP_NT) k_sp_reduce(const u64 *part, u32 nparts, u64 n2, u64 *proof)
{
    for (u64 m = blockIdx.x * (u64)SP_NT + threadIdx.x; m < n2; m += (u64)gridDim.x * SP_NT) {
        u64 s = 0;
        for (u32 k = 0; k < nparts; k++) s = wred(s + part[(u64)k * n2 + m]);
        proof[m] = wcanon(s);
    }
}

// Product of one canonical value per thread over the CTA (thread 0 returns it).
__device__ u64 cta_prod(u64 x)
{
    __shared__ u64 s[SP_NT / 32];
    x = warp_prod(x);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
    __syncthreads();
    u64 r = 1;
    if (threadIdx.x < 32) {
        r = threadIdx.x < SP_NT / 32 ? s[threadIdx.x] : 1;
        r = warp_prod(r);
    }
    __syncthreads();
    return r;
}

// Verifier setup (one CTA): r = the seed's first accepted draw; L[y] = L_y(r)
// over the nodes 0..h-1 and M[y] = the basis at r over 0..2h-2; rows zeroed
// by the other CTAs.  st[0] = r.
__global__ void __launch_bounds__(SP_NT) k_sp_vbegin(u64 seed, u64 v, u64 h, const u64 *w, const u64 *w2, u64 *L,
                                                     u64 *M, u64 *acc, u64 *st)
{
    if (blockIdx.x > 0) {
        for (u64 x = (blockIdx.x - 1) * (u64)SP_NT + threadIdx.x; x < v; x += (u64)(gridDim.x - 1) * SP_NT) acc[x] = 0;
        return;
    }
    u64 r = 0;
    for (u64 k = 1;; k++) {
        r = splitmix64_at(seed, k) >> 3;
        if (r != FP_P) break;
    }
    const u64 n2 = 2 * h - 1;
    // C(r) = prod_{k<h} (r - k), C2(r) = prod_{k<2h-1} (r - k)
    u64 p1 = 1, p2 = 1;
    for (u64 k = threadIdx.x; k < n2; k += SP_NT) {
        const u64 f = f_sub(r, k);
        p2 = f_mul(p2, f);
        if (k < h) p1 = f_mul(p1, f);
    }
    const u64 c1 = cta_prod(p1), c2 = cta_prod(p2);
    __shared__ u64 s_c[2];
    if (threadIdx.x == 0) {
        s_c[0] = c1;
        s_c[1] = c2;
        st[0] = r;
    }
    __syncthreads();
    for (u64 y = threadIdx.x; y < n2; y += SP_NT) {
        // r equal to a node: the basis is the indicator of that node
        const bool at = (r == y);
        const u64 inv = at ? 0 : f_inv(f_sub(r, y));
        if (y < h) L[y] = (r < h) ? (at ? 1 : 0) : f_mul(f_mul(s_c[0], w[y]), inv);
        M[y] = (r < n2) ? (at ? 1 : 0) : f_mul(f_mul(s_c[1], w2[y]), inv);
    }
}

// Streaming pass over whole rows [x0, x0 + nrows): acc[x] += sum_y a(x, y) L[y]
// (one warp per row; rows given contiguously, row x at rows[(x - x0) h]).
__global__ void __launch_bounds__(SP_NT) k_sp_vabsorb(const u64 *rows, u64 x0, u64 nrows, u64 h, const u64 *L,
                                                      u64 *acc, u32 *status)
{
    const u32 lane = threadIdx.x & 31;
    const u64 wid = (blockIdx.x * (u64)SP_NT + threadIdx.x) >> 5, nw = ((u64)gridDim.x * SP_NT) >> 5;
    for (u64 x = wid; x < nrows; x += nw) {
        const u64 *row = rows + x * h;
        acc128 s;
        acc_zero(s);
        u64 red = 0;
        bool bad = false;
        u32 k = 0;
        for (u64 y = lane; y < h; y += 32, k++) {
            const u64 val = row[y];
            bad |= val >= FP_P;
            mac(s, val >= FP_P ? 0 : val, L[y]);
            if ((k & 31) == 31) {
                red = wred(red + acc_red(s));
                acc_zero(s);
            }
        }
        const u64 t = warp_wsum(wred(red + acc_red(s)));
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_INPUT);
        if (lane == 0) acc[x0 + x] = f_add(acc[x0 + x], wcanon(t));
    }
}

// Verifier end (one CTA): res[0] = accept, res[1] = F2 answer, res[2] = s(r),
// res[3] = sum_x f_x(r)^2.
__global__ void __launch_bounds__(SP_NT) k_sp_vend(const u64 *proof, u64 v, u64 h, const u64 *M, const u64 *acc,
                                                   u64 *res)
{
    const u64 n2 = 2 * h - 1;
    u64 lhs = 0, rhs = 0, ans = 0;
    bool bad = false;
    for (u64 x = threadIdx.x; x < v; x += SP_NT) lhs = wred(lhs + wmul(acc[x], acc[x]));
    for (u64 y = threadIdx.x; y < n2; y += SP_NT) {
        const u64 s = proof[y];
        bad |= s >= FP_P;
        rhs = wred(rhs + wmul(s >= FP_P ? 0 : s, M[y]));
        if (y < h) ans = wred(ans + (s >= FP_P ? 0 : s));
    }
    __shared__ u64 sh[3][SP_NT / 32];
    lhs = warp_wsum(lhs);
    rhs = warp_wsum(rhs);
    ans = warp_wsum(ans);
    const u32 lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wv] = lhs;
        sh[1][wv] = rhs;
        sh[2][wv] = ans;
    }
    const int anybad = __syncthreads_or(bad);
    if (threadIdx.x < 32) {
        lhs = warp_wsum(lane < SP_NT / 32 ? sh[0][lane] : 0);
        rhs = warp_wsum(lane < SP_NT / 32 ? sh[1][lane] : 0);
        ans = warp_wsum(lane < SP_NT / 32 ? sh[2][lane] : 0);
        if (lane == 0) {
            lhs = wcanon(lhs);
            rhs = wcanon(rhs);
            res[0] = (!anybad && lhs == rhs) ? 1 : 0;
            res[1] = wcanon(ans);
            res[2] = rhs;
            res[3] = lhs;
        }
    }
}

size_t sp_prove_smem(u64 h) { return (size_t)(2 * h - 1 + (u64)SP_RB * SP_YT) * sizeof(u64); }
u32 sp_prove_ctas(u64 v) { return (u32)((v + SP_RB - 1) / SP_RB); }

void sp_init()
{
    cudaFuncSetAttribute(k_sp_prove, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void launch_sp_tables(u64 h, u64 *w, u64 *C, u64 *iv, u64 *w2, cudaStream_t st)
{
    k_sp_tables<<<device_sms(), SP_NT, 0, st>>>(h, w, C, iv, w2);
}

void launch_sp_prove(const u64 *a, u64 v, u64 h, const u64 *w, const u64 *C, const u64 *iv, u64 *part, u64 *proof,
                     u32 *status, cudaStream_t st)
{
    const u32 nc = sp_prove_ctas(v);
    k_sp_prove<<<nc, SP_NT, sp_prove_smem(h), st>>>(a, v, h, w, C, iv, part, status);
    k_sp_reduce<<<(unsigned)((2 * h - 1 + SP_NT - 1) / SP_NT), SP_NT, 0, st>>>(part, nc, 2 * h - 1, proof);
}

void launch_sp_vbegin(u64 seed, u64 v, u64 h, const u64 *w, const u64 *w2, u64 *L, u64 *M, u64 *acc, u64 *res,
                      cudaStream_t st)
{
    k_sp_vbegin<<<1 + device_sms(), SP_NT, 0, st>>>(seed, v, h, w, w2, L, M, acc, res);
}

void launch_sp_vabsorb(const u64 *rows, u64 x0, u64 nrows, u64 h, const u64 *L, u64 *acc, u32 *status,
                       cudaStream_t st)
{
    k_sp_vabsorb<<<grid_for_items(nrows * 32, SP_NT, 8), SP_NT, 0, st>>>(rows, x0, nrows, h, L, acc, status);
}

void launch_sp_vend(const u64 *proof, u64 v, u64 h, const u64 *M, const u64 *acc, u64 *res, cudaStream_t st)
{
    k_sp_vend<<<1, SP_NT, 0, st>>>(proof, v, h, M, acc, res);
}
