// plan.h -- launch-plan descriptors shared by the host planner and the kernels.
//
// A proof is a fixed sequence of launches whose shapes depend only on the
// circuit's shape, so vc_circuit_create computes every descriptor once and
// uploads it; a proof only replays the plan with a new seed and new inputs.
//
// Because the verifier's coins are a function of the seed alone, every
// challenge is known before the first message is computed.  The prover uses
// this to run all d layer iterations, and within a layer its three sum-check
// phases and its line reduction, concurrently: each is an independent
// "sum-check instance" (SCI) or line job over its own tables.  The rounds of
// one SCI stay in order (each round folds the tables with its challenge).
#pragma once
#include "field.cuh"

enum : u32 {
    W_SQUARE = 0, W_TREE = 1, W_MATMULT = 2, W_F0_FIRST = 3, W_F0_PAIR = 4, W_F0_FINAL = 5,
    W_EXPLICIT = 6
};

// Split table of eq(x, .) over n coordinates: eq(x, b) = lo[b mod 2^h] * hi[b >> h]
// with h = ceil(n/2) (Sec. 4.1.1's per-gate eq factor at one product per gate).
struct EqTab {
    u64 *lo;        // 2^h entries
    u64 *hi;        // 2^(n-h) entries
    const u64 *pt;  // the point, n coordinates (device)
    u32 n, h;
};

__device__ __forceinline__ u64 eq_at(const EqTab &t, u64 b)
{
    return f_mul(t.lo[b & ((1ull << t.h) - 1)], t.hi[b >> t.h]);
}

// One layer iteration (layer i relates V_i to V_{i+1}).
struct LayerDev {
    u32 s, sn;        // s_i, s_{i+1}
    u32 kind;         // W_*
    u32 has_add;      // layer has ADD gates (else the B tables are zero)
    u32 chal_off;     // first round challenge of this layer in chal[]
    u32 z_off;        // z_i in pts[] (s_i coordinates)
    u64 *V;           // layer i values
    u64 *Vn;          // layer i+1 values
    u64 tr_msg;       // transcript offset of the layer's round values
    u64 tr_q;         // transcript offset of q(0..s_{i+1})
    EqTab tz, trp, tr1, tr2;  // eq tables of z_i, r_P, r1, r2
    u64 *P2, *B2, *P3, *B3;   // phase-2/3 tables over layer i+1 (B* NULL if !has_add)
    const unsigned char *type;  // EXPLICIT only
    const u32 *in1, *in2;
    const u32 *by1_off, *by1_g;  // gates grouped by in1: offsets [S_{i+1}+1], gate ids [S_i]
    const u32 *by2_off, *by2_g;  // gates grouped by in2
};

// In-neighbours and operation of gate g of layer i (Sec. 6.2.1 circuits):
// computed from the index for the structured kinds (a tree gate reads 2g and
// 2g+1, as in Sec. 5.1.4), read for EXPLICIT layers.
__device__ __forceinline__ void gate_wiring(const LayerDev &L, u64 g, u64 &a, u64 &b, u32 &mul)
{
    switch (L.kind) {
    case W_SQUARE: a = g; b = g; mul = 1; break;
    case W_TREE: a = 2 * g; b = 2 * g + 1; mul = 0; break;
    case W_MATMULT: {
        const u32 Lb = L.s / 3;
        const u64 n = 1ull << Lb, m = n - 1;
        const u64 k = g & m, j = (g >> Lb) & m, ii = g >> (2 * Lb);
        a = (ii << Lb) | k;
        b = (1ull << (2 * Lb)) | (k << Lb) | j;
        mul = 1;
        break;
    }
    case W_F0_FIRST: a = g >> 1; b = g >> 1; mul = (g & 1) ? 0 : 1; break;
    case W_F0_PAIR: a = g; b = g & ~1ull; mul = 1; break;
    case W_F0_FINAL: a = 2 * g + 1; b = 2 * g + 1; mul = 1; break;
    default: a = L.in1[g]; b = L.in2[g]; mul = L.type[g]; break;
    }
}

// Per-layer scalars written during a proof: scal[2 i] = eq(z_i, r_P),
// scal[2 i + 1] = V~_{i+1}(r1) (= q_i(0)).
#define SCAL_EQZRP(i) (2 * (i))
#define SCAL_V1(i) (2 * (i) + 1)

// Flags of a sum-check wave.  WF_TAIL: the next descriptor (a single chunk)
// is run by the CTA that finishes this wave's last chunk.
enum : u32 { WF_HASB = 2, WF_LAST = 4, WF_TAIL = 8 };

// Kinds of sum-check instance (SCI).  Product-weighted ones (< PK_GEN_FIRST)
// keep P = sigma prod_m L_m(x_m) implicit; general ones fold P, V, B tables.
enum : u32 {
    PK_PH1 = 0,        // phase 1 of any layer: P = eq(z_i, .), V = V_i
    PK_TREE3 = 1,      // TREE phase 3: L_0 = (0,1), L_m = eq(rP_{m-1},.) eq(r1_m,.), U = V + v1
    PK_SQ3 = 2,        // SQUARE phase 3: L_m = eq(rP_m,.) eq(r1_m,.), sigma = eq(z,rP) v1
    PK_GEN_FIRST = 8,
    PK_GEN_SQ2 = 8,    // SQUARE phase 2: P[x] = eq(rP, x) V[x] (times eq(z, rP))
    PK_GEN_TREE2 = 9,  // TREE phase 2: P[2g] = eq(rP, g), B[2g] = P[2g] V[2g+1] (times eq(z, rP))
    PK_GEN_TAB = 10    // tables built by k_build23
};

// Source of the first GEN wave's P and B.
enum : u32 { GS_NONE = 0, GS_SQ2 = 1, GS_TREE2 = 2 };

#define PR_M 6  // PROD: at most 2^6 entries per thread, folded in registers (128 threads per CTA)
#define GN_M 5  // GEN: at most 2^5 entries per thread (128 threads per CTA)
// Evaluation runs holding F0_PAIR layers take chunks of at most 2^8 input
// entries: one pair per thread of a 256-thread evaluation CTA.
#define EV_PAIR_CHUNK 8

struct SciDev {
    u32 circ;
    u32 n;         // rounds
    u32 kind;      // PK_*
    u32 layer;
    u32 chal_off;  // challenge of round k: chal[chal_off + k]
    u64 tr_off;    // transcript offset of round 0's three values
    u64 *Lc;       // PROD: factors c0_m, c1_m (2n), written by the coin launch
    u64 *kap;      // PROD: prod_{m<j} L_m(r_m)
    u64 *esum;     // PROD: prod_{m>j} (c0_m + c1_m)
};

// One wave of a PROD SCI: each CTA folds 2^nr entries (the first e rounds in
// registers, 2^e entries per thread; the rest across the CTA).
struct ProdWave {
    u32 circ;
    u32 sci;
    u32 r0, nr, e;
    u32 nchunks;
    u32 flags;
    u32 no, ho;        // coordinates beyond the chunk (r0+nr..n-1) and their split
    u32 chal_off;      // challenge of local round k: chal[chal_off + k]
    u32 pad;
    const u64 *in;     // entries of this wave's table
    u64 *out;          // one folded value per chunk (unused on the last wave)
    u64 *wblk;         // weight block: Q, E, outer lo, outer hi
    u64 *part;         // partials: part[(k * nchunks + chunk) * 2 + t]
    u32 *counter;      // chunks finished (WF_TAIL only; reset by the last)
};

// One wave of a GEN SCI.
struct GenWave {
    u32 circ;
    u32 sci;
    u32 r0, nr, e;
    u32 nchunks;
    u32 flags;
    u32 src;           // GS_* (first wave only)
    u32 layer;
    u32 chal_off;
    u32 pad;
    const u64 *inP, *inV, *inB;
    u64 *outP, *outV, *outB;
    u64 *part;         // partials: part[(k * nchunks + chunk) * 3 + t]
    u32 *counter;      // chunks finished (WF_TAIL only; reset by the last)
};

// Line reduction of layer i (q(t) = V~_{i+1}(l(t)), l(t) = r1 + t (r2 - r1)),
// computed by folding V_{i+1} with the coordinates a_k + b_k t in coefficient
// form: after folding j coordinates each entry is a polynomial of degree j.
struct LineWaveDev {
    u32 circ;
    u32 layer;
    u32 n;        // s_{i+1}
    u32 l0, nl;   // coordinates [l0, l0 + nl) folded by this wave
    u32 nchunks;
    u32 last;
    const u64 *in;  // l0 == 0: V_{i+1}; else polys [chunk][l0 + 1]
    u64 *out;       // polys [nchunks][l0 + nl + 1] (unused on the last wave)
    u32 a_off;      // a_k = chal[a_off + k] (= r1), b_k = chal[b_off + k] - a_k
    u32 b_off;
    u64 tr_q;
    u32 tail;       // the next descriptor (one chunk) is run by this wave's last CTA
    u32 pad;
    u32 *counter;   // CTAs of this wave that finished (tail only; reset by the last)
};

// Work item of a merged launch: which wave descriptor and which chunk.
struct Item {
    u32 wave;
    u32 chunk;
};

// Task of the persistent wave launch: one chunk of a line, PROD or GEN wave.
enum : u32 { TK_LINE = 0, TK_PROD = 1, TK_GEN = 2 };
struct Task {
    u32 type;
    u32 wave;   // index into the plan's line, PROD or GEN wave descriptors
    u32 chunk;
    u32 pad;
};

// Final reduction of one round: sum the chunks' partials (2 per chunk for
// PROD, 3 for GEN) and write g(0), g(1), g(2) at tr[tr_pos].  Every scalar
// the round needs is reached through its own pointer, so the loads are
// independent of one another.
struct RoundRef {
    u64 tr_pos;
    const u64 *part_pos;
    u32 nchunks;
    u32 kind;         // PK_* of the instance
    u32 circ;
    u32 sci;
    u32 j;            // round index within the SCI
    u32 defer;        // TREE phase 2, j >= 1: the message carries the factor 1 - (first challenge of the
                      // phase), left out of P and B by the first wave's round 0
    const u64 *ez;    // eq(z_i, r_P) of the layer
    const u64 *v1;    // V~_{i+1}(r1) of the layer
    const u64 *ch;    // TREE phases 2 and 3: the first challenge of phase 2
    const u64 *lc;    // PROD: c0, c1 of round j
    const u64 *kap;   // PROD: kappa_j
    const u64 *esum;  // PROD: esum_j
};

// Per-circuit globals.  Each circuit keeps one copy in device memory (and a
// batch keeps one per member); kernels find theirs through the `circ` index of
// their work descriptor.  seed and tr change per proof and are written on the
// stream by k_params (or from a parameter table for a batch) before the
// proof's launches, so a captured launch sequence can be replayed.
struct Globals {
    u64 seed;
    u32 d;
    u32 nchal;
    u64 *chal;        // nchal challenges
    u64 *pts;         // z_0 .. z_d
    u64 *scal;        // per-layer scalars (SCAL_*)
    u64 *tr;          // transcript (device)
    u32 *status;      // error flags (bit 0: non-canonical input)
    LayerDev *layers;
    u64 *invfact;     // 1/k! for k < 64 (verifier)
    const u32 *zmap;  // flattened coordinates of z_1..z_d: layer << 8 | k
    u32 nz;
    u32 zd_off;       // z_d in pts[]
    u64 S0;           // outputs
    const u64 *out_src;  // where the final reduction reads the outputs (layer 0, or a
                         // copy of it when the layer values rotate through device slots)
    const u64 *in;    // this proof's inputs when the first evaluation launch reads them
                      // in place (it also writes the input layer's values); set by
                      // k_params, cleared by k_final; NULL: the inputs are in layer d
};

// A run of block-local layers evaluated by one launch (k_eval_seg): layers
// i_hi down to i_lo, chunks of 2^c entries of layer i_hi + 1 per CTA.  The
// CTA that finishes last then evaluates layers i_lo - 1 down to tail_lo
// alone (tail_lo == i_lo: no tail); `counter` counts finished CTAs and is
// reset by the last one.
struct EvalSeg {
    u32 circ;
    u32 i_hi, i_lo;
    u32 c;
    u32 nchunks;
    u32 check_input;  // the run's input layer is the circuit's input layer
    u32 tail_lo;
    u32 warp_from;       // first run layer whose blocks all fit one warp (i_lo - 1: none)
    u32 *counter;
    u32 tail_warp_from;  // first tail layer from which all fit one warp (tail_lo - 1: none)
    u32 pad2;
};

// A layer evaluated on its own (MATMULT or EXPLICIT wiring).
struct LayerEval {
    u32 circ;
    u32 layer;
};

// Work item of k_build23: 256 entries of layer i+1's phase-2/3 tables.
struct BuildItem {
    u32 circ;
    u32 layer;
    u32 block;
    u32 pad;
};

// Parameters of one proof in a batch (written from the host each call).
struct CallParams {
    u64 seed;
    u64 *tr;
    const u64 *in;       // the member's inputs (device memory) for the gather launch
    const u64 *in_eval;  // the same when the member's first evaluation launch reads them in
                         // place (written to Globals::in), else NULL
};

// A piece of one batch member's input copy: count entries from the member's
// inputs (CallParams::in) at `start` to dst (its input layer, at `start`).
struct GatherChunk {
    u64 *dst;
    u64 start;
    u32 member;
    u32 count;
};
#define GATHER_CHUNK 2048

#define ST_BAD_INPUT 1u
#define ST_TIMEOUT 2u
#define VC_RESULT_WORDS 8  // verifier result words (device)

// ---- launch entry points (implemented in the .cu files) -------------------------
// An eq table to build and where its point comes from: challenges
// chal[off ..] (EQ_SRC_CHAL) or the point z_layer (EQ_SRC_Z).
enum : u32 { EQ_SRC_CHAL = 0, EQ_SRC_Z = 1 };
struct EqJob {
    EqTab t;
    u32 circ;
    u32 src;
    u32 off;
    u32 layer;
};

void launch_params(Globals *G, u64 seed, u64 *tr, const u64 *in, cudaStream_t st);
const void *params_kernel();   // k_params, to find its node in a captured graph
const void *vparams_kernel();  // k_vparams, likewise
void launch_params_batch(Globals *Gs, const CallParams *cp, int n, cudaStream_t st);
// Every member's inputs into its input layer, one launch (all inputs device memory).
void launch_gather_inputs(const CallParams *cp, const GatherChunk *chunks, int nchunks, cudaStream_t st);
// One launch: setup of every circuit (challenges, points, eq(z_i, r_P)),
// the eq tables and the product weights of the PROD waves.
void launch_coins(const Globals *Gs, int ncirc, const EqJob *eqjobs, int neq, const SciDev *scis,
                  const ProdWave *pw, int npw, cudaStream_t st);
void launch_eval_layers(const Globals *Gs, const LayerEval *le, const Item *items, int nitems, cudaStream_t st);
// maxblock: the largest block (entries) of any run layer or tail output in
// the launch (<= 2048); it sizes the two shared-memory buffers.
void launch_eval_segs(const Globals *Gs, const EvalSeg *segs, const Item *items, int nitems, u32 maxblock,
                      cudaStream_t st,
                      bool after_params = false);
void launch_check_canonical(const u64 *x, u64 n, u32 *status, cudaStream_t st);
void launch_check_inputs(const Globals *Gs, const Item *items, int nitems, cudaStream_t st);
void launch_build23(const Globals *Gs, const BuildItem *items, int nitems, cudaStream_t st);
// Explicit layers: an entry w of layer i+1 read by more than BUILD_HEAVY
// gates is summed after launch_build23 by npieces CTAs of up to
// BUILD_PIECE gates each (kind 1: its in1 list, 2: its in2 list); each writes
// its sums to part[2 piece ..], and the last to finish (ctr) adds them all to
// the entry's tables.
#define BUILD_HEAVY 32u
#define BUILD_PIECE 4096u
struct HeavyItem {
    u32 circ, layer, w, kind;
    u32 piece, npieces, pad0, pad1;
    u64 *part;  // 2 npieces u64
    u32 *ctr;   // zero between proofs (reset by the last piece)
};
void launch_build_heavy(const Globals *Gs, const HeavyItem *items, int nitems, cudaStream_t st);
// One persistent launch over `tasks` (ctr: two zeroed counters, left zeroed).
void launch_waves(const Globals *Gs, const LineWaveDev *lw, const ProdWave *pw, const GenWave *gw, const Task *tasks,
                  int ntasks, u32 *ctr, cudaStream_t st);
// Rounds [0, nbig) are reduced a warp each: all rounds when there are at most
// FINAL_ALL_WARPS (the warps of one full launch), else those with more than
// FINAL_WARP_MIN chunk partials; the rest a thread each.
#define FINAL_WARP_MIN 8u
#define FINAL_ALL_WARPS ((u32)device_sms() * 8u * 8u)
void launch_final(Globals *Gs, const RoundRef *rounds, int nrounds, int nbig, const u32 *outs, int nouts,
                  cudaStream_t st);
void prove_kernels_init();
void waves_init();

// verifier
// Per-call pointers of a verification, written on the stream before the
// verifier's captured launches (so that the launches can be replayed).
struct VerifyPtrs {
    const u64 *tr;      // transcript (device)
    const u64 *inputs;  // S_d inputs (device)
    int *accept_out;    // optional device int receiving the accept bit
    u64 pad;
};

struct VerifyDev {
    u32 d;
    u64 tr_len;
    const VerifyPtrs *vp;  // device
    u64 *mle_part;      // partial sums of the input MLE
    u32 mle_blocks;
    u64 *result;        // [2] accept bit, [3] a check failed (k_vcheck writes both); others unused
    u64 *wire;          // generic add~/mult~ per layer (EXPLICIT layers)
    u64 *wire_part;     // their per-CTA partial sums (two per CTA, VwireItem::part_off)
    u32 *wire_ctr;      // per layer: CTAs done (reset by the last)
    u32 mle_out_blocks; // blocks of the output-MLE partials (after the input's; 0: formed by k_vcheck)
    const u32 *round_layer;  // per global round: layer << 8 | round within layer
    u32 nrounds;
};
// One CTA's share of an explicit layer's generic wiring sum: gates
// [block, block + 1) * ceil(S_i / nblocks); partial sums at part_off + block.
struct VwireItem {
    u32 layer, block, nblocks, part_off;
};
void launch_init_invfact(u64 *invfact, cudaStream_t st);
// result: VC_RESULT_WORDS words, cleared by the launch
void launch_vparams(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *tr, const u64 *inputs, int *accept,
                    u64 *result, cudaStream_t st);
// The verifier's launches after its coin launch was issued on st: the MLE
// partial sums on st_mle (forked from st before the coins, so both run
// together), joined back into st through ev_join, then the checks.
u32 vmle_log(u32 n);
void launch_verify(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0, const VwireItem *wire_items,
                   int n_wire, cudaStream_t st_mle, cudaEvent_t ev_join, cudaStream_t st);
// The verifier in two passes.  Input pass: the input's MLE partial sums (the
// coins are launched beside it by the caller).  Transcript pass, with the
// transcript and accept pointer as arguments: the claimed outputs' MLE
// partial sums (many outputs only), add~/mult~ of explicit layers, the checks
// (the eq tables of explicit layers are launched before it by the caller).
void launch_verify_input(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0, cudaStream_t st);
void launch_verify_transcript(const Globals *Gd, const Globals &G, const VerifyDev &V, u32 nd, u32 n0,
                              const VwireItem *wire_items, int n_wire, const u64 *tr, int *accept,
                              cudaStream_t st);
void launch_vparams_in(Globals *G, VerifyPtrs *vp, u64 seed, const u64 *inputs, cudaStream_t st);
const void *vparams_in_kernel();
// Circuits with at most this many outputs have their claimed outputs' MLE
// formed inside the check launch, by one warp (more: k_vmle partial sums).
#define VC_OUT_INLINE 256u

// Per-gate prover (k_pergate.cu): one descriptor per layer.
struct PgLayer {
    u32 layer;         // i
    u32 s, sn, n;      // s_i, s_{i+1}, rounds s_i + 2 s_{i+1}
    u32 blk0, nblk;    // CTAs of the gate launches covering this layer's gates
    u32 lblk0, lnblk;  // CTAs of the line launch covering V_{i+1}
    u64 *preP;         // eq over the bound p coordinates (S_i entries; eq(r_P, .) after phase 1)
    u64 *preA, *preB;  // the same over the bound w1 / w2 coordinates (S_{i+1} each)
    u64 *suf;          // phase-1 suffix tables of z_i (S_i - 1 entries)
    u64 *fa, *fb;      // V_{i+1} folded with the bound coordinates (S_{i+1}/2, S_{i+1}/4)
    u64 *v1;           // V~_{i+1}(r1)
    u64 *part;         // per-CTA partial sums of the current round, 3 per CTA
    u64 *ltab;         // line: split eq tables of l(t), t = 0..s_{i+1}
    u64 *lpart;        // line: per-CTA partial sums, s_{i+1} + 1 per CTA
};
// Every launch of a per-gate proof after the evaluation and the coins.
void launch_pergate(const Globals *G, const PgLayer *pl, int nl, const u32 *blk_layer, u32 nblk,
                    const u32 *lblk_layer, u32 nlblk, u32 nrounds, cudaStream_t st);
u32 pergate_gpt();  // gates (and line entries) per CTA

// Special-purpose non-interactive F2 protocol (k_f2sp.cu).  The prover's
// transform (built by vc_f2sp_create): h = q_0 ... q_{m-1}, pairwise coprime
// prime powers <= 61; device tables.
struct SpFftHost {
    u32 h, m, nroots;
    u32 q[8], magic[8], twoff[8];
    const u64 *fw, *bw;      // per dimension: its root's powers and inverse powers
    const u32 *pin, *perm, *idx;
    const u64 *twist;
};
void sp_init();
size_t sp_prove_smem(u64 h, u32 nroots);
u32 sp_prove_ctas(u64 v);
void launch_sp_prove(const u64 *a, u64 v, const SpFftHost &H, u64 *part, u32 nparts, u64 *proof, u32 *status,
                     cudaStream_t st);
void launch_sp_vbegin(u64 seed, u64 v, u64 h, u64 inv_h, const u64 *pw, u64 *L, u64 *M, u64 *acc, u64 *res,
                      cudaStream_t st);
void launch_sp_vabsorb(const u64 *rows, u64 x0, u64 nrows, u64 h, const u64 *L, u64 *acc, u32 *status,
                       cudaStream_t st);
void launch_sp_vend(const u64 *proof, u64 v, u64 h, const u64 *M, const u64 *acc, u64 *res, cudaStream_t st);

// SM count of the current device (queried once per device; 1 if the query
// fails), and the grid of a grid-stride loop over n items capped at per_sm
// CTAs per SM.
int device_sms();
unsigned grid_for_items(u64 n, unsigned threads, unsigned per_sm);
void launch_field_mul(const u64 *a, const u64 *b, u64 *out, u64 n, cudaStream_t st);
double run_field_mul_rate(int variant, u64 iters, int sms, u64 *sink);
