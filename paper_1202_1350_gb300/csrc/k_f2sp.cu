// k_f2sp.cu -- the special-purpose non-interactive F2 protocol (outlined in
// Sec. 3.2; prover and verifier parallelisation in Sec. 4.2; memory access in
// Sec. 5.2; GPU results in Sec. 6.3).
//
// The frequency vector a (n = v h entries) is a v x h grid, a(x, y) at
// x h + y.  Row x is the polynomial f_x of degree < h with f_x(w^y) = a(x, y),
// w a generator of the subgroup of order h of F_p^*; the proof is
// s(Y) = sum_x f_x(Y)^2 at the 2h points u^k (u of order 2h, u^2 = w).  The
// verifier keeps f_x(r) for a secret random r, accepts iff
// s(r) = sum_x f_x(r)^2 and answers F2 = sum_{k even} s(u^k).
//
// Prover (the paper's per-row transform by the Prime Factor FFT, Sec. 4.2).
// The even points u^{2y} = w^y are the nodes: s there is the column's sum of
// squares.  For the odd points u w^y: the row's coefficients are the inverse
// DFT of its values over the subgroup of order h, c_j = (1/h) sum_y a_y w^{-jy},
// and f(u w^y) = sum_j (c_j u^j) w^{jy} is a forward DFT of the twisted
// coefficients.  h = q_1 ... q_m with pairwise coprime prime powers q_i <= 61,
// so each DFT is an m-dimensional DFT with no twiddles between dimensions
// (Good-Thomas): the input index n sits at digits (n t_i mod q_i), the output
// index k at digits (k mod q_i), t_i = (h/q_i)^{-1} mod q_i, and the root of
// dimension i is w^{h/q_i}.  A CTA holds one row at a time in shared memory and
// runs each dimension as small DFTs along the innermost (contiguous) digit,
// writing that digit outermost, so after m passes the digits are back in
// order.  The host-built tables give every digit position's input slot, the
// twist factor u^j / h with the slot of the forward transform, and the index
// of every output; the CTA accumulates the squares of its rows per point and a
// second launch sums the CTAs' partials.  Work per row: 2 h (q_1 + ... + q_m)
// multiply-adds instead of the O(h^2) of a direct extension.
//
// Verifier.  f_x(r) = sum_y a(x, y) L_y(r) with the subgroup's Lagrange basis
// L_y(r) = w^y (r^h - 1) / (h (r - w^y)), streamed over whole rows; at the end
// s(r) = sum_k s_k u^k (r^{2h} - 1) / (2h (r - u^k)) over the 2h proof points
// (an indicator basis when r lies in the subgroup).
#include <cuda_runtime.h>

#include "plan.h"

#define SP_NT 256
#define SP_PNT 512  // prover CTA

// Geometry and tables of the prover's transform (device pointers; built on
// the host by vc_f2sp_create).
struct SpFft {
    u32 h, m;             // h = q_0 ... q_{m-1}
    u32 nroots;           // q_0 + ... + q_{m-1}
    u32 q[8];             // dimension sizes, innermost last
    u32 magic[8];         // ceil(2^20 / q): floor(i / q) = (i magic) >> 20 for i < 2^13
    u32 twoff[8];         // offset of dimension i's roots in fw / bw
    const u64 *fw, *bw;   // roots w_i^e and w_i^{-e}, e < q_i, per dimension
    const u32 *pin;       // input slot of index y (digits y t_i mod q_i)
    const u32 *perm;      // output slot P of the inverse DFT -> its input slot in the forward one
    const u64 *twist;     // output slot P -> u^j / h (j the index at P)
    const u32 *idx;       // output slot P -> its index j (k mod q_i digits)
};

// One pass of the multi-dimensional DFT: small DFTs of size q along the
// innermost digit (lines of q consecutive slots), output digit written
// outermost: out[k (h/q) + L] = sum_j in[L q + j] root^{jk}.
__device__ __forceinline__ void sp_pass(const u64 *in, u64 *out, u32 h, u32 q, u32 magic, const u64 *roots)
{
    const u32 lines = h / q;
    for (u32 i = threadIdx.x; i < h; i += SP_PNT) {
        const u32 L = (u32)(((u64)i * magic) >> 20), k = i - L * q;
        const u64 *src = in + L * q;
        acc128 a;
        acc_zero(a);
        u32 e = 0;
        for (u32 j = 0; j < q; j++) {  // q <= 61 products of a W value and a canonical root
            mac(a, src[j], roots[e]);
            e += k;
            if (e >= q) e -= q;
        }
        out[k * lines + L] = acc_red(a);
    }
}

// Column partials of the proof for the CTA's rows x = blockIdx.x, +gridDim.x,
// ...: part[cta][2y] = sum a(x, y)^2, part[cta][2y + 1] = sum f_x(u w^y)^2.
__global__ void __launch_bounds__(SP_PNT, 1) k_sp_prove(const u64 *a, u64 v, SpFft F, u64 *part, u32 *status)
{
    extern __shared__ u64 sp_dyn[];
    const u32 h = F.h, nt = F.nroots;
    u64 *bufA = sp_dyn, *bufB = bufA + h, *acc_e = bufB + h, *acc_o = acc_e + h, *s_fw = acc_o + h, *s_bw = s_fw + nt;
    for (u32 i = threadIdx.x; i < h; i += SP_PNT) acc_e[i] = acc_o[i] = 0;
    for (u32 i = threadIdx.x; i < nt; i += SP_PNT) {
        s_fw[i] = F.fw[i];
        s_bw[i] = F.bw[i];
    }
    bool bad = false;
    for (u64 x = blockIdx.x; x < v; x += gridDim.x) {
        __syncthreads();  // the previous row is done with the buffers
        const u64 *row = a + x * h;
        for (u32 y = threadIdx.x; y < h; y += SP_PNT) {
            u64 val = row[y];
            bad |= val >= FP_P;
            val = val >= FP_P ? 0 : val;
            bufA[__ldg(F.pin + y)] = val;
            acc_e[y] = wred(acc_e[y] + wmul(val, val));
        }
        __syncthreads();
        u64 *cur = bufA, *nxt = bufB;
        // inverse DFT: c_j (times h) at the digits of j
        for (int d = (int)F.m - 1; d >= 0; d--) {
            sp_pass(cur, nxt, h, F.q[d], F.magic[d], s_bw + F.twoff[d]);
            __syncthreads();
            u64 *t = cur; cur = nxt; nxt = t;
        }
        // twist by u^j / h, into the forward transform's input slots
        for (u32 i = threadIdx.x; i < h; i += SP_PNT) nxt[__ldg(F.perm + i)] = wmul(cur[i], __ldg(F.twist + i));
        __syncthreads();
        { u64 *t = cur; cur = nxt; nxt = t; }
        for (int d = (int)F.m - 1; d >= 0; d--) {
            sp_pass(cur, nxt, h, F.q[d], F.magic[d], s_fw + F.twoff[d]);
            __syncthreads();
            u64 *t = cur; cur = nxt; nxt = t;
        }
        // f(u w^j) at slot i, j = idx[i]: squares accumulated by slot
        for (u32 i = threadIdx.x; i < h; i += SP_PNT) {
            const u64 f = cur[i];
            acc_o[i] = wred(acc_o[i] + wmul(f, f));
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_BAD_INPUT);
    u64 *out = part + (u64)blockIdx.x * 2 * h;
    for (u32 i = threadIdx.x; i < h; i += SP_PNT) {
        out[2 * i] = wcanon(acc_e[i]);
        out[2 * __ldg(F.idx + i) + 1] = wcanon(acc_o[i]);
    }
}

// proof[k] = sum over CTAs of part[cta][k].
__global__ void __launch_bounds__(SP_NT) k_sp_reduce(const u64 *part, u32 nparts, u64 n2, u64 *proof)
{
    for (u64 m = blockIdx.x * (u64)SP_NT + threadIdx.x; m < n2; m += (u64)gridDim.x * SP_NT) {
        u64 s = 0;
        for (u32 k = 0; k < nparts; k++) s = wred(s + part[(u64)k * n2 + m]);
        proof[m] = wcanon(s);
    }
}

__device__ u64 f_pow(u64 b, u64 e)
{
    u64 r = 1;
    while (e) {
        if (e & 1) r = f_mul(r, b);
        b = f_mul(b, b);
        e >>= 1;
    }
    return r;
}

// The verifier's secret point: the seed's first accepted draw.
__device__ u64 sp_secret(u64 seed)
{
    for (u64 k = 1;; k++) {
        const u64 r = splitmix64_at(seed, k) >> 3;
        if (r != FP_P) return r;
    }
}

// Verifier setup, every CTA: r from the seed (res[0] = r, written by CTA 0);
// L[y] = L_y(r) over the nodes pw[2y] (y < h) and M[k] = the basis at r over
// the proof points pw[k] (k < 2h), grid-stride; row values zeroed.
__global__ void __launch_bounds__(SP_NT) k_sp_vbegin(u64 seed, u64 v, u64 h, u64 inv_h, const u64 *pw, u64 *L,
                                                     u64 *M, u64 *acc, u64 *res)
{
    const u64 r = sp_secret(seed);
    const u64 gt = blockIdx.x * (u64)SP_NT + threadIdx.x, nth = (u64)gridDim.x * SP_NT;
    if (gt == 0) res[0] = r;
    for (u64 x = gt; x < v; x += nth) acc[x] = 0;
    const u64 rh = f_pow(r, h), r2h = f_mul(rh, rh);
    const u64 ch = f_mul(f_sub(rh, 1), inv_h);                        // (r^h - 1) / h
    const u64 c2h = f_mul(f_mul(f_sub(r2h, 1), inv_h), FP_INV2);      // (r^2h - 1) / (2h)
    for (u64 e = gt; e < 3 * h; e += nth) {
        // e < h: node y = e (point pw[2y]); else proof point k = e - h
        const bool node = e < h;
        const u64 k = node ? 2 * e : e - h;
        const u64 pt = pw[k];
        const bool in_group = node ? (rh == 1) : (r2h == 1);
        u64 val;
        if (in_group) {
            val = (r == pt) ? 1 : 0;  // r is a point of the set: indicator basis
        } else {
            val = f_mul(f_mul(pt, node ? ch : c2h), f_inv(f_sub(r, pt)));
        }
        if (node) L[e] = val;
        else M[k] = val;
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

// Verifier end (one CTA): res[0] = accept, res[1] = F2 answer (the even
// points), res[2] = s(r), res[3] = sum_x f_x(r)^2.
__global__ void __launch_bounds__(SP_NT) k_sp_vend(const u64 *proof, u64 v, u64 h, const u64 *M, const u64 *acc,
                                                   u64 *res)
{
    const u64 n2 = 2 * h;
    u64 lhs = 0, rhs = 0, ans = 0;
    bool bad = false;
    for (u64 x = threadIdx.x; x < v; x += SP_NT) lhs = wred(lhs + wmul(acc[x], acc[x]));
    for (u64 k = threadIdx.x; k < n2; k += SP_NT) {
        const u64 s = proof[k];
        bad |= s >= FP_P;
        rhs = wred(rhs + wmul(s >= FP_P ? 0 : s, M[k]));
        if ((k & 1) == 0) ans = wred(ans + (s >= FP_P ? 0 : s));
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

size_t sp_prove_smem(u64 h, u32 nroots) { return (size_t)(4 * h + 2 * nroots) * sizeof(u64); }

u32 sp_prove_ctas(u64 v) { return (u32)(v < (u64)device_sms() ? v : (u64)device_sms()); }

void sp_init()
{
    cudaFuncSetAttribute(k_sp_prove, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void launch_sp_prove(const u64 *a, u64 v, const SpFftHost &H, u64 *part, u32 nparts, u64 *proof, u32 *status,
                     cudaStream_t st)
{
    SpFft F{};
    F.h = H.h;
    F.m = H.m;
    F.nroots = H.nroots;
    for (u32 i = 0; i < 8; i++) {
        F.q[i] = H.q[i];
        F.magic[i] = H.magic[i];
        F.twoff[i] = H.twoff[i];
    }
    F.fw = H.fw;
    F.bw = H.bw;
    F.pin = H.pin;
    F.perm = H.perm;
    F.twist = H.twist;
    F.idx = H.idx;
    k_sp_prove<<<nparts, SP_PNT, sp_prove_smem(H.h, H.nroots), st>>>(a, v, F, part, status);
    k_sp_reduce<<<(unsigned)((2 * H.h + SP_NT - 1) / SP_NT), SP_NT, 0, st>>>(part, nparts, 2 * H.h, proof);
}

void launch_sp_vbegin(u64 seed, u64 v, u64 h, u64 inv_h, const u64 *pw, u64 *L, u64 *M, u64 *acc, u64 *res,
                      cudaStream_t st)
{
    k_sp_vbegin<<<grid_for_items(3 * h > v ? 3 * h : v, SP_NT, 4), SP_NT, 0, st>>>(seed, v, h, inv_h, pw, L, M, acc,
                                                                                  res);
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
