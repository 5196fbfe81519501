// k_prove.cu -- prover kernels for the GKR/CMT protocol over F_p, p = 2^61 - 1.
//
// Paper: Thaler, Roberts, Mitzenmacher, Pfister, "Verifiable Computation with
// Massively Parallel Interactive Proofs".
//   Sec. 3.1   one iteration per layer, each touching two adjacent layers;
//   Sec. 4.1.1 every gate contributes independently to each prover message,
//              which is the field sum of the contributions (parallel reduction);
//   Sec. 5.1.4 in-neighbour indices from the gate index; coalesced accesses.
//
// The prover here folds tables instead of recomputing per-gate contributions
// from scratch each round (the folding form gives the same messages; each
// round halves the tables), and runs every layer's sum-check phases and line
// reduction concurrently, since all verifier coins follow from the seed.
#include <cuda_runtime.h>
#include "plan.h"

// --------------------------------------------------------------------------------
// Setup: verifier coins (splitmix64 stream), the layer points z_i, eq(z_i, r_P).
// --------------------------------------------------------------------------------

// Per-proof parameters of one circuit (seed, transcript pointer, and the
// inputs when the evaluation reads them in place).
__global__ void k_params(Globals *G, u64 seed, u64 *tr, const u64 *in)
{
    // the evaluation launch that follows may start now (it waits for these
    // writes before it reads them)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    G->seed = seed;
    G->tr = tr;
    G->in = in;
}

__global__ void k_params_batch(Globals *Gs, const CallParams *cp, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        Gs[j].seed = cp[j].seed;
        Gs[j].tr = cp[j].tr;
        Gs[j].in = cp[j].in_eval;
    }
}

// One CTA per chunk of a member's input copy (coalesced 16-byte moves; the
// chunks start at multiples of GATHER_CHUNK, so a chunk is 16-byte aligned
// at both ends whenever the member's buffers are).
__global__ void __launch_bounds__(256) k_gather_inputs(const CallParams *cp, const GatherChunk *chunks)
{
    const GatherChunk C = chunks[blockIdx.x];
    const u64 *src = cp[C.member].in + C.start;
    u64 *dst = C.dst;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    if (vec) {
        const u32 np = C.count / 2;
        for (u32 k = threadIdx.x; k < np; k += blockDim.x)
            reinterpret_cast<ulonglong2 *>(dst)[k] = reinterpret_cast<const ulonglong2 *>(src)[k];
        if ((C.count & 1) && threadIdx.x == 0) dst[C.count - 1] = src[C.count - 1];
    } else {
        for (u32 k = threadIdx.x; k < C.count; k += blockDim.x) dst[k] = src[k];
    }
}

void launch_gather_inputs(const CallParams *cp, const GatherChunk *chunks, int nchunks, cudaStream_t st)
{
    if (nchunks > 0) k_gather_inputs<<<nchunks, 256, 0, st>>>(cp, chunks);
}

void launch_params(Globals *G, u64 seed, u64 *tr, const u64 *in, cudaStream_t st)
{
    k_params<<<1, 1, 0, st>>>(G, seed, tr, in);
}
const void *params_kernel() { return reinterpret_cast<const void *>(k_params); }

void launch_params_batch(Globals *Gs, const CallParams *cp, int n, cudaStream_t st)
{
    if (n > 0) k_params_batch<<<(n + 255) / 256, 256, 0, st>>>(Gs, cp, n);
}


// Layer evaluation: V_i[g] = V_{i+1}[in1] op V_{i+1}[in2] (Sec. 6.2.4); an
// item covers 256 gates of one layer of one circuit.
__global__ void __launch_bounds__(256) k_eval_layer(const Globals *Gs, const LayerEval *le, const Item *items)
{
    const Item it = items[blockIdx.x];
    const LayerEval E = le[it.wave];
    const LayerDev &L = Gs[E.circ].layers[E.layer];
    const u64 g = (u64)it.chunk * 256 + threadIdx.x;
    if (g < (1ull << L.s)) {
        u64 a, b;
        u32 mul;
        gate_wiring(L, g, a, b, mul);
        const u64 x = L.Vn[a], y = L.Vn[b];
        L.V[g] = mul ? f_mul(x, y) : f_add(x, y);
    }
}

void launch_eval_layers(const Globals *Gs, const LayerEval *le, const Item *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_eval_layer<<<nitems, 256, 0, st>>>(Gs, le, items);
}

// Fused evaluation of a run of block-local layers (every structured kind but
// MATMULT): a CTA loads an aligned chunk of the run's input layer and
// evaluates it upward through the run in shared memory, writing each layer.
// Block size of layer i = chunk size * 2^(s_i - s_in); all stay <= EV_MAXB.
#ifndef EV_NT
#define EV_NT 256  // threads of an evaluation CTA
#endif
#define EV_MAXB 2048

extern __shared__ u64 ev_dyn[];

// Gate k of a block-local layer: operand positions within the block below
// and the operation.
__device__ __forceinline__ void local_gate(u32 kind, u32 k, u32 &a, u32 &b, u32 &mul)
{
    mul = 1;
    switch (kind) {
    case W_SQUARE: a = k; b = k; break;
    case W_TREE: a = 2 * k; b = 2 * k + 1; mul = 0; break;
    case W_F0_FIRST: a = k >> 1; b = k >> 1; mul = (k & 1) ? 0 : 1; break;
    case W_F0_PAIR: a = k; b = k & ~1u; break;
    default: a = 2 * k + 1; b = 2 * k + 1; break;  // W_F0_FINAL
    }
}

#define EV_LC 64  // layer descriptors cached in shared memory per launch

// Descriptor of layer i = i_hi - j of a run: from the shared cache (j < EV_LC)
// or from global memory.
struct EvLayer {
    u32 kind, s, sn;
    u64 *V;
};

// One layer of a block in shared memory, the gate kind's loop hoisted out of
// the switch.
__device__ __forceinline__ void eval_block_smem(u32 kind, const u64 *cur, u64 *nxt, u64 *__restrict__ out, u32 Bo)
{
    const u32 t = threadIdx.x;
    switch (kind) {
    case W_SQUARE:
        for (u32 k = t; k < Bo; k += EV_NT) {
            const u64 v = f_mul(cur[k], cur[k]);
            nxt[k] = v;
            out[k] = v;
        }
        break;
    case W_TREE:
        for (u32 k = t; k < Bo; k += EV_NT) {
            const u64 v = f_add(cur[2 * k], cur[2 * k + 1]);
            nxt[k] = v;
            out[k] = v;
        }
        break;
    default:
        for (u32 k = t; k < Bo; k += EV_NT) {
            u32 a, b, mul;
            local_gate(kind, k, a, b, mul);
            const u64 x = cur[a], y = cur[b];
            const u64 v = mul ? f_mul(x, y) : f_add(x, y);
            nxt[k] = v;
            out[k] = v;
        }
        break;
    }
}

// Layers whose blocks all fit in one warp (<= 64 entries in and out): warp 0
// holds the block in registers (entries l and l + 32 in lane l) and exchanges
// operands with shuffles, without block-wide barriers.  SQUARE needs no
// exchange and TREE (at most 32 outputs) only its two operands, so those take
// no multiply or shuffle they do not use.
template <class LayerFn>
__device__ __forceinline__ void eval_warp_layers(LayerFn layer, int hi, int lo, const u64 *cur, u32 B, bool chunked,
                                                 u32 chunk)
{
    const u32 lane = threadIdx.x & 31;
    u64 v0 = (lane < B) ? cur[lane] : 0, v1 = (lane + 32 < B) ? cur[lane + 32] : 0;
    for (int i = hi; i >= lo; i--) {
        const EvLayer L = layer((u32)i);
        const u32 Bo = chunked ? ((L.s >= L.sn) ? (B << (L.s - L.sn)) : (B >> (L.sn - L.s))) : (1u << L.s);
        u64 *__restrict__ out = L.V + (chunked ? (u64)chunk * Bo : 0);
        u64 nv[2];
        if (L.kind == W_SQUARE) {
            nv[0] = f_mul(v0, v0);
            nv[1] = f_mul(v1, v1);
        } else if (L.kind == W_TREE) {  // Bo <= 32: entries 2k, 2k+1 of lane k
            const u32 a = (2 * lane) & 31;
            const u64 x0 = __shfl_sync(0xffffffffu, v0, a), y0 = __shfl_sync(0xffffffffu, v0, a + 1);
            const u64 x1 = __shfl_sync(0xffffffffu, v1, a), y1 = __shfl_sync(0xffffffffu, v1, a + 1);
            nv[0] = (lane < 16) ? f_add(x0, y0) : f_add(x1, y1);
            nv[1] = 0;
        } else {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const u32 k = lane + 32 * h;
                u32 a, b, mul;
                local_gate(L.kind, k < Bo ? k : 0, a, b, mul);
                const u64 xa0 = __shfl_sync(0xffffffffu, v0, a & 31), xa1 = __shfl_sync(0xffffffffu, v1, a & 31);
                const u64 xb0 = __shfl_sync(0xffffffffu, v0, b & 31), xb1 = __shfl_sync(0xffffffffu, v1, b & 31);
                const u64 x = (a < 32) ? xa0 : xa1, y = (b < 32) ? xb0 : xb1;
                nv[h] = mul ? f_mul(x, y) : f_add(x, y);
            }
        }
        if (lane < Bo) out[lane] = nv[0];
        if (lane + 32 < Bo) out[lane + 32] = nv[1];
        v0 = (lane < Bo) ? nv[0] : 0;
        v1 = (lane + 32 < Bo) ? nv[1] : 0;
        B = Bo;
    }
}

// A chain of F0_PAIR layers (gate 2j = v_2j^2, gate 2j+1 = v_2j+1 v_2j): every
// pair of entries evolves on its own, so a thread keeps its pairs in registers
// through the whole chain, writes each layer with 16-byte stores and needs no
// barrier between the layers.  `cur` holds the block below layer hi (B
// entries); the pairs after layer lo go to `nxt`.
template <class LayerFn>
__device__ __forceinline__ void eval_pair_chain(LayerFn layer, int hi, int lo, const u64 *cur, u64 *nxt, u32 B,
                                                u32 chunk)
{
    constexpr int PP = EV_MAXB / 2 / EV_NT;  // pairs a thread holds
    const u32 np = B >> 1;
    u64 x0[PP], x1[PP];
#pragma unroll
    for (int h = 0; h < PP; h++) {
        const u32 q = threadIdx.x + h * EV_NT;
        x0[h] = (q < np) ? cur[2 * q] : 0;
        x1[h] = (q < np) ? cur[2 * q + 1] : 0;
    }
    for (int i = hi; i >= lo; i--) {
        ulonglong2 *__restrict__ out = reinterpret_cast<ulonglong2 *>(layer((u32)i).V + (u64)chunk * B);
#pragma unroll
        for (int h = 0; h < PP; h++) {
            const u32 q = threadIdx.x + h * EV_NT;
            if (q < np) {  // the shorter-latency product: the chain is latency-bound
                x1[h] = f_mul_wide(x1[h], x0[h]);
                x0[h] = f_mul_wide(x0[h], x0[h]);
                out[q] = make_ulonglong2(x0[h], x1[h]);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < PP; h++) {
        const u32 q = threadIdx.x + h * EV_NT;
        if (q < np) {
            nxt[2 * q] = x0[h];
            nxt[2 * q + 1] = x1[h];
        }
    }
}

#ifndef EV_MINB
#define EV_MINB 4  // resident evaluation CTAs per SM the register allocation is sized for
#endif

__global__ void __launch_bounds__(EV_NT, EV_MINB) k_eval_seg(const Globals *Gs, const EvalSeg *segs, const Item *items,
                                                    u32 bufsz)
{
    u64 *bufA = ev_dyn, *bufB = ev_dyn + bufsz;  // bufsz >= every block of the launch's runs and tails
    __shared__ u32 s_kind[EV_LC], s_s[EV_LC], s_sn[EV_LC];
    __shared__ u64 *s_V[EV_LC];
    __shared__ const u64 *s_in;
    const Item it = items[blockIdx.x];
    const EvalSeg S = segs[it.wave];
    const Globals &G = Gs[S.circ];
    const LayerDev *Ls = G.layers;
    u32 *const status = G.status;
    const u32 chunk = it.chunk;
    // every field the loops need, read once (stores to the layers' values
    // would otherwise force the compiler to re-read descriptors per element)
    const u32 nl = S.i_hi - S.tail_lo + 1;
    for (u32 j = threadIdx.x; j < nl && j < EV_LC; j += EV_NT) {
        const LayerDev &L = Ls[S.i_hi - j];
        s_kind[j] = L.kind;
        s_s[j] = L.s;
        s_sn[j] = L.sn;
        s_V[j] = L.V;
    }
    __shared__ u64 *s_copy;
    // launched right after the parameter write with a programmatic dependence:
    // the plan's descriptors above are static, the per-proof fields are not
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
        // a run over the input layer reads this proof's inputs in place, if
        // given, and writes them to the layer's values
        const bool inplace = G.in != nullptr && S.i_hi + 1 == G.d;
        s_in = inplace ? G.in : Ls[S.i_hi].Vn;
        s_copy = inplace ? Ls[S.i_hi].Vn : nullptr;
    }
    __syncthreads();
    auto layer = [&](u32 i) {
        const u32 j = S.i_hi - i;
        EvLayer e;
        if (j < EV_LC) {
            e.kind = s_kind[j];
            e.s = s_s[j];
            e.sn = s_sn[j];
            e.V = s_V[j];
        } else {
            const LayerDev &L = Ls[i];
            e.kind = L.kind;
            e.s = L.s;
            e.sn = L.sn;
            e.V = L.V;
        }
        return e;
    };
    u32 B = 1u << S.c;  // block size of the current (upper) layer
    constexpr int R = EV_MAXB / EV_NT;
    {
        // all loads of the chunk are issued before any store
        const u64 *__restrict__ src = s_in + ((u64)chunk << S.c);
        u64 r[R];
#pragma unroll
        for (int j = 0; j < R; j++) {
            const u32 k = threadIdx.x + j * EV_NT;
            r[j] = (k < B) ? src[k] : 0;
        }
        bool bad = false;
        u64 *const copy = s_copy ? s_copy + ((u64)chunk << S.c) : nullptr;
#pragma unroll
        for (int j = 0; j < R; j++) {
            const u32 k = threadIdx.x + j * EV_NT;
            if (k < B) {
                bad |= (r[j] >= FP_P);
                bufA[k] = r[j];
                if (copy) copy[k] = r[j];
            }
        }
        if (S.check_input && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_BAD_INPUT);
    }
    __syncthreads();
    u64 *cur = bufA, *nxt = bufB;
    int i = (int)S.i_hi;
    for (; i >= (int)S.i_lo; i--) {
        if (i == (int)S.warp_from) break;
        const EvLayer L = layer((u32)i);
        if (L.kind == W_F0_PAIR) {  // the chain of pair layers from here, in registers
            int lo = i;
            while (lo - 1 >= (int)S.i_lo && lo - 1 != (int)S.warp_from && layer((u32)(lo - 1)).kind == W_F0_PAIR) lo--;
            eval_pair_chain(layer, i, lo, cur, nxt, B, chunk);
            __syncthreads();
            u64 *t = cur; cur = nxt; nxt = t;
            i = lo;
            continue;
        }
        const u32 Bo = (L.s >= L.sn) ? (B << (L.s - L.sn)) : (B >> (L.sn - L.s));
        eval_block_smem(L.kind, cur, nxt, L.V + (u64)chunk * Bo, Bo);
        __syncthreads();
        u64 *t = cur; cur = nxt; nxt = t;
        B = Bo;
    }
    if (i >= (int)S.i_lo && threadIdx.x < 32) eval_warp_layers(layer, i, (int)S.i_lo, cur, B, true, chunk);
    if (S.tail_lo >= S.i_lo) return;
    // Last-CTA tail: every CTA publishes its writes and counts itself; the
    // last one evaluates the narrow layers below the run from the whole
    // layer i_lo (no CTA waits for another).
    __shared__ u32 s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(S.counter, 1u) == S.nchunks - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) *S.counter = 0;
    {
        // first tail layer: operands from the whole layer i_lo in global memory, all loads first
        i = (int)S.i_lo - 1;
        const EvLayer L = layer((u32)i);
        const u32 Bo = 1u << L.s;
        u64 *__restrict__ out = L.V;
        const u64 *__restrict__ vin = layer((u32)i + 1).V;
        u64 xa[R], xb[R];
#pragma unroll
        for (int j = 0; j < R; j++) {
            const u32 k = threadIdx.x + j * EV_NT;
            u32 a, b, mul;
            local_gate(L.kind, k, a, b, mul);
            xa[j] = (k < Bo) ? __ldcg(vin + a) : 0;
            xb[j] = (k < Bo) ? __ldcg(vin + b) : 0;
        }
#pragma unroll
        for (int j = 0; j < R; j++) {
            const u32 k = threadIdx.x + j * EV_NT;
            if (k < Bo) {
                u32 a, b, mul;
                local_gate(L.kind, k, a, b, mul);
                const u64 v = mul ? f_mul(xa[j], xb[j]) : f_add(xa[j], xb[j]);
                nxt[k] = v;
                out[k] = v;
            }
        }
        __syncthreads();
        u64 *t = cur; cur = nxt; nxt = t;
        B = Bo;
        i--;
    }
    for (; i >= (int)S.tail_lo; i--) {
        if (i == (int)S.tail_warp_from) break;
        const EvLayer L = layer((u32)i);
        const u32 Bo = 1u << L.s;
        eval_block_smem(L.kind, cur, nxt, L.V, Bo);
        __syncthreads();
        u64 *t = cur; cur = nxt; nxt = t;
        B = Bo;
    }
    if (i >= (int)S.tail_lo && threadIdx.x < 32) eval_warp_layers(layer, i, (int)S.tail_lo, cur, B, false, 0);
}

void launch_eval_segs(const Globals *Gs, const EvalSeg *segs, const Item *items, int nitems, u32 maxblock,
                      cudaStream_t st, bool after_params)
{
    if (maxblock > EV_MAXB) maxblock = EV_MAXB;
    if (nitems <= 0) return;
    if (!after_params) {
        k_eval_seg<<<nitems, EV_NT, 2 * maxblock * sizeof(u64), st>>>(Gs, segs, items, maxblock);
        return;
    }
    // right after k_params: a programmatic dependence lets the CTAs start and
    // read the plan's descriptors while the parameters are written
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)nitems);
    cfg.blockDim = dim3(EV_NT);
    cfg.dynamicSmemBytes = 2 * maxblock * sizeof(u64);
    cfg.stream = st;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_eval_seg, Gs, segs, items, maxblock);
}

__global__ void k_check_canonical(const u64 *x, u64 n, u32 *status)
{
    bool bad = false;
    for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x)
        bad |= (x[k] >= FP_P);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_BAD_INPUT);
}

void launch_check_canonical(const u64 *x, u64 n, u32 *status, cudaStream_t st)
{
    k_check_canonical<<<grid_for_items(n, 256, 8), 256, 0, st>>>(x, n, status);
}

// Canonical-input check inside a proof plan: an item covers 2048 inputs of
// circuit item.wave (used where the first evaluation launch does not check).
__global__ void __launch_bounds__(256) k_check_inputs(const Globals *Gs, const Item *items)
{
    const Item it = items[blockIdx.x];
    const Globals &G = Gs[it.wave];
    const LayerDev &L = G.layers[G.d - 1];
    const u64 n = 1ull << L.sn;
    bool bad = false;
    for (u64 k = (u64)it.chunk * 2048 + threadIdx.x, e = min(n, (u64)(it.chunk + 1) * 2048); k < e; k += 256)
        bad |= (L.Vn[k] >= FP_P);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(G.status, ST_BAD_INPUT);
}

void launch_check_inputs(const Globals *Gs, const Item *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_check_inputs<<<nitems, 256, 0, st>>>(Gs, items);
}

void prove_kernels_init()
{
    cudaFuncSetAttribute(k_eval_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * EV_MAXB * sizeof(u64)));
}

// --------------------------------------------------------------------------------
// Phase-2/3 tables over layer i+1, gathered per entry w (no atomics).
//   w_g = eq(z, r_P) eq(r_P, g),   u_g = w_g eq(r1, in1(g))
//   P2[w] = sum_{g: in1=w} w_g [ADD: 1, MUL: V(in2)],   B2[w] = sum_{ADD g: in1=w} w_g V(in2)
//   A2[w] = sum_{ADD g: in2=w} u_g,   M2[w] = sum_{MUL g: in2=w} u_g
//   P3 = A2 + v1 M2,   B3 = v1 A2,   v1 = V~_{i+1}(r1)
// Phase-2 message: sum P2 V + B2; phase-3 message: sum P3 V + B3.
// --------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_build23(const Globals *Gs, const BuildItem *items)
{
    const BuildItem bi = items[blockIdx.x];
    const Globals &G = Gs[bi.circ];
    const u32 i = bi.layer;
    const LayerDev &L = G.layers[i];
    const u64 w = (u64)bi.block * blockDim.x + threadIdx.x;
    const u64 Sn = 1ull << L.sn;
    const u64 ez = G.scal[SCAL_EQZRP(i)];
    const u64 v1 = G.scal[SCAL_V1(i)];
    const u64 *V = L.Vn;
    if (L.kind == W_F0_PAIR || L.kind == W_F0_FINAL) {
        // a thread per pair of entries 2q, 2q+1 (their gates share operands;
        // a thread per entry left half of each warp idle on the other path)
        const u64 q = w;
        if (2 * q >= Sn) return;
        u64 P2a, P2b, M2;
        if (L.kind == W_F0_PAIR) {  // gate 2q = v_2q^2, gate 2q+1 = v_2q+1 v_2q
            const u64 wg0 = f_mul(ez, eq_at(L.trp, 2 * q)), wg1 = f_mul(ez, eq_at(L.trp, 2 * q + 1));
            const u64 x = V[2 * q];
            P2a = f_mul(wg0, x);
            P2b = f_mul(wg1, x);
            M2 = f_add(f_mul(wg0, eq_at(L.tr1, 2 * q)), f_mul(wg1, eq_at(L.tr1, 2 * q + 1)));
        } else {  // gate q = v_2q+1^2: only entry 2q+1 is read
            const u64 wg = f_mul(ez, eq_at(L.trp, q));
            P2a = f_mul(wg, V[2 * q + 1]);
            M2 = f_mul(wg, eq_at(L.tr1, 2 * q + 1));
        }
        // PAIR: entry 2q carries the products with in1 = 2q (P2 and, with in1
        // = in2 = 2q or in1 = 2q+1, in2 = 2q, M2 at 2q); FINAL: all at 2q+1
        ulonglong2 *P2 = reinterpret_cast<ulonglong2 *>(L.P2), *P3 = reinterpret_cast<ulonglong2 *>(L.P3);
        if (L.kind == W_F0_PAIR) {
            P2[q] = make_ulonglong2(P2a, P2b);
            P3[q] = make_ulonglong2(f_mul(v1, M2), 0);
        } else {
            P2[q] = make_ulonglong2(0, P2a);
            P3[q] = make_ulonglong2(0, f_mul(v1, M2));
        }
        return;
    }
    if (w >= Sn) return;
    u64 P2 = 0, B2 = 0, A2 = 0, M2 = 0;
    switch (L.kind) {
    case W_SQUARE: {
        const u64 wg = f_mul(ez, eq_at(L.trp, w));
        P2 = f_mul(wg, V[w]);
        M2 = f_mul(wg, eq_at(L.tr1, w));
        break;
    }
    case W_TREE: {
        if ((w & 1) == 0) {
            const u64 wg = f_mul(ez, eq_at(L.trp, w >> 1));
            P2 = wg;
            B2 = f_mul(wg, V[w + 1]);
        } else {
            const u64 g = w >> 1;
            const u64 wg = f_mul(ez, eq_at(L.trp, g));
            A2 = f_mul(wg, eq_at(L.tr1, w - 1));
        }
        break;
    }
    case W_F0_FIRST: {
        const u64 wm = f_mul(ez, eq_at(L.trp, 2 * w));      // MUL gate 2w
        const u64 wa = f_mul(ez, eq_at(L.trp, 2 * w + 1));  // ADD gate 2w+1
        const u64 e1 = eq_at(L.tr1, w);
        P2 = f_add(f_mul(wm, V[w]), wa);
        B2 = f_mul(wa, V[w]);
        A2 = f_mul(wa, e1);
        M2 = f_mul(wm, e1);
        break;
    }
    case W_MATMULT: {
        const u32 Lb = L.s / 3;
        const u64 n = 1ull << Lb, msk = n - 1;
        if (w < (1ull << (2 * Lb))) {
            // gates with in1 = w: k = w mod n, i = w >> L, all j
            const u64 k = w & msk, ii = w >> Lb;
            u64 acc = 0;
            for (u64 j = 0; j < n; j++) {
                const u64 g = k | (j << Lb) | (ii << (2 * Lb));
                const u64 bidx = (1ull << (2 * Lb)) | (k << Lb) | j;
                acc = f_add(acc, f_mul(eq_at(L.trp, g), V[bidx]));
            }
            P2 = f_mul(ez, acc);
        } else {
            // gates with in2 = w: j = w mod n, k = (w >> L) mod n, all i
            const u64 j = w & msk, k = (w >> Lb) & msk;
            u64 acc = 0;
            for (u64 ii = 0; ii < n; ii++) {
                const u64 g = k | (j << Lb) | (ii << (2 * Lb));
                acc = f_add(acc, f_mul(eq_at(L.trp, g), eq_at(L.tr1, (ii << Lb) | k)));
            }
            M2 = f_mul(ez, acc);
        }
        break;
    }
    default: {  // explicit wiring, gates grouped by in1 and by in2
        // an entry read by more than BUILD_HEAVY gates is summed by a whole
        // CTA afterwards (k_build_heavy), which adds to what is written here
        const u32 a0 = L.by1_off[w], a1 = L.by1_off[w + 1];
        for (u32 q = a0; q < a1 && a1 - a0 <= BUILD_HEAVY; q++) {
            const u32 g = L.by1_g[q];
            const u64 wg = f_mul(ez, eq_at(L.trp, g));
            if (L.type[g]) {
                P2 = f_add(P2, f_mul(wg, V[L.in2[g]]));
            } else {
                P2 = f_add(P2, wg);
                B2 = f_add(B2, f_mul(wg, V[L.in2[g]]));
            }
        }
        const u32 b0 = L.by2_off[w], b1 = L.by2_off[w + 1];
        for (u32 q = b0; q < b1 && b1 - b0 <= BUILD_HEAVY; q++) {
            const u32 g = L.by2_g[q];
            const u64 ug = f_mul(f_mul(ez, eq_at(L.trp, g)), eq_at(L.tr1, L.in1[g]));
            if (L.type[g]) M2 = f_add(M2, ug);
            else A2 = f_add(A2, ug);
        }
        break;
    }
    }
    L.P2[w] = P2;
    L.P3[w] = f_add(A2, f_mul(v1, M2));
    if (L.has_add) {
        L.B2[w] = B2;
        L.B3[w] = f_mul(v1, A2);
    }
}

void launch_build23(const Globals *Gs, const BuildItem *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_build23<<<nitems, 256, 0, st>>>(Gs, items);
}

// Sums of a CTA's (x, y) pair, in thread 0.
__device__ __forceinline__ void block_sum_pair(u64 &x, u64 &y)
{
    __shared__ u64 sx[256], sy[256];
    __syncthreads();  // the arrays may still be read by an earlier call
    sx[threadIdx.x] = x;
    sy[threadIdx.x] = y;
    __syncthreads();
    for (u32 h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sx[threadIdx.x] = f_add(sx[threadIdx.x], sx[threadIdx.x + h]);
            sy[threadIdx.x] = f_add(sy[threadIdx.x], sy[threadIdx.x + h]);
        }
        __syncthreads();
    }
    x = sx[0];
    y = sy[0];
}

// One piece of the gate list of an explicit layer's entry w that more than
// BUILD_HEAVY gates read (a constant such as 1 or p - 1 feeding a whole
// layer): kind 1, the gates with in1 = w (sums for P2 and B2); kind 2, those
// with in2 = w (for A2 and M2, which enter P3 and B3).  The last piece to
// finish adds every piece's sums to what k_build23 wrote for the entry.
__global__ void __launch_bounds__(256) k_build_heavy(const Globals *Gs, const HeavyItem *items)
{
    const HeavyItem it = items[blockIdx.x];
    const Globals &G = Gs[it.circ];
    const u32 i = it.layer;
    const LayerDev &L = G.layers[i];
    const u64 w = it.w;
    const u64 ez = G.scal[SCAL_EQZRP(i)];
    const u64 *V = L.Vn;
    const u32 *off = (it.kind == 1) ? L.by1_off : L.by2_off;
    const u32 q0 = off[w] + it.piece * BUILD_PIECE, q1 = min(off[w + 1], q0 + BUILD_PIECE);
    u64 x = 0, y = 0;  // in1 lists: P2, B2 parts; in2 lists: A2, M2 parts
    if (it.kind == 1) {
        for (u32 q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const u32 g = L.by1_g[q];
            const u64 wg = f_mul(ez, eq_at(L.trp, g));
            if (L.type[g]) {
                x = f_add(x, f_mul(wg, V[L.in2[g]]));
            } else {
                x = f_add(x, wg);
                y = f_add(y, f_mul(wg, V[L.in2[g]]));
            }
        }
    } else {
        for (u32 q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const u32 g = L.by2_g[q];
            const u64 ug = f_mul(f_mul(ez, eq_at(L.trp, g)), eq_at(L.tr1, L.in1[g]));
            if (L.type[g])
                y = f_add(y, ug);
            else
                x = f_add(x, ug);
        }
    }
    block_sum_pair(x, y);
    if (it.npieces > 1) {
        __shared__ u32 s_last;
        if (threadIdx.x == 0) {
            it.part[2 * it.piece] = x;
            it.part[2 * it.piece + 1] = y;
            __threadfence();
            s_last = (atomicAdd(it.ctr, 1u) == it.npieces - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        x = y = 0;
        for (u32 q = threadIdx.x; q < it.npieces; q += blockDim.x) {
            x = f_add(x, __ldcg(it.part + 2 * q));
            y = f_add(y, __ldcg(it.part + 2 * q + 1));
        }
        block_sum_pair(x, y);
        if (threadIdx.x == 0) *it.ctr = 0;
    }
    if (threadIdx.x) return;
    if (it.kind == 1) {
        L.P2[w] = f_add(L.P2[w], x);
        if (L.has_add) L.B2[w] = f_add(L.B2[w], y);
    } else {
        const u64 v1 = G.scal[SCAL_V1(i)];
        L.P3[w] = f_add(L.P3[w], f_add(x, f_mul(v1, y)));
        if (L.has_add) L.B3[w] = f_add(L.B3[w], f_mul(v1, x));
    }
}

void launch_build_heavy(const Globals *Gs, const HeavyItem *items, int nitems, cudaStream_t st)
{
    if (nitems > 0) k_build_heavy<<<nitems, 256, 0, st>>>(Gs, items);
}

