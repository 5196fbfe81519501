// internal.h -- definitions shared by the C ABI (vc_api.cu) and the proof
// server (server.cu): device arenas, launch plans, circuit and batch handles.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "plan.h"
#include "vc.h"

constexpr u32 WV_LOG = 7;                  // log2 of the threads of a wave CTA
constexpr u32 PR_CHUNK_LOG = PR_M + WV_LOG;  // rounds of one PROD chunk (2^PR_M entries per thread)
constexpr u32 GN_CHUNK_LOG = GN_M + WV_LOG;  // rounds of one GEN chunk (2^GN_M entries per thread)
constexpr u32 LN_CHUNK0_LOG = 6 + WV_LOG;    // coordinates of a first line-wave chunk (64 entries per thread)
constexpr u32 LN_CHUNKW_LOG = WV_LOG;        // coordinates of a later line-wave chunk (one polynomial per thread)

// Tile shapes of a circuit's plan (the autotuner's knobs): rounds folded
// by a first PROD / GEN chunk, coordinates folded by a first line-wave chunk,
// the smallest evaluation chunk (log2 entries), and the size below which PROD
// instances use half-size chunks.
struct PlanConfig {
    u32 pr_chunk = PR_CHUNK_LOG;
    u32 gn_chunk = GN_CHUNK_LOG;
    u32 ln_chunk0 = LN_CHUNK0_LOG;
    u32 ev_chunk = 11;  // evaluation chunk: 2^11 inputs per CTA
    u32 pr_split = VC_SPLIT_WIDEST;  // PROD instances below 2^pr_split entries: chunks of 2^(pr_chunk - 1)
};

// Every device and page-locked host allocation of the library goes through
// these (mem.cu): they keep the process-wide budget of vc_set_memory_limit
// and fail with cudaErrorMemoryAllocation, before any CUDA call, past it.
cudaError_t lib_malloc(void **p, size_t n);
cudaError_t lib_free(void *p);
cudaError_t lib_host_alloc(void **p, size_t n, unsigned flags);
cudaError_t lib_free_host(void *p);
template <class T>
cudaError_t lib_malloc(T **p, size_t n)
{
    return lib_malloc(reinterpret_cast<void **>(p), n);
}
template <class T>
cudaError_t lib_host_alloc(T **p, size_t n, unsigned flags)
{
    return lib_host_alloc(reinterpret_cast<void **>(p), n, flags);
}

// Device slots of the wide layers of a circuit with staged values.
constexpr u32 STAGED_SLOTS = 8;
// residencies whose wide layers pass through device slots
constexpr u32 VC_VALUES_SLOTTED = VC_VALUES_STAGED | VC_VALUES_WINDOWED;

// Which layers' phase-2/3 tables are built by k_build23 (the rest are formed
// on the fly or never stored).
inline bool needs_tables(u32 kind) { return kind != W_SQUARE && kind != W_TREE; }

// Bump allocator over one device allocation (base 0: sizing pass).
struct Arena {
    uintptr_t base = 0;
    size_t off = 0;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += n * sizeof(T) + 16;
        return p;
    }
};

// Makes `d` the current device for the guard's lifetime.
struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t upload(T *dst, const std::vector<T> &src)
{
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <class T>
cudaError_t upload_async(T *dst, const std::vector<T> &src, cudaStream_t st)
{
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// The launches of one proof over a set of circuits.  Every descriptor carries
// the index (circ) of its circuit in the plan's device array of globals; the
// item lists of one evaluation step, line wave or sum-check wave hold the work
// of every circuit, so one launch serves them all.
struct Plan {
    int ncirc = 0;
    Globals *d_G = nullptr;
    std::vector<Globals> h_G;  // members' globals (merged plans: uploaded to d_G)
    std::vector<Item> checks;  // canonical-input checks (circuit, 2048-input block)
    std::vector<EqJob> eqjobs;
    std::vector<EvalSeg> segs;
    std::vector<LayerEval> levs;
    std::vector<std::vector<Item>> seg_items, lev_items;  // per evaluation step
    std::vector<u32> seg_maxblock;                         // per step: largest block of its runs
    std::vector<LineWaveDev> lw;
    std::vector<BuildItem> builds;
    std::vector<HeavyItem> heavy;  // explicit layers' entries with long gate lists (k_build_heavy)
    std::vector<SciDev> scis;
    std::vector<ProdWave> pw;
    std::vector<GenWave> gw;
    // persistent wave launches: groups A (before the wiring tables are built)
    // and B (general waves over built tables), each one launch
    std::vector<std::vector<Task>> groupsA, groupsB;
    std::vector<RoundRef> rounds;  // those with more than FINAL_WARP_MIN partials first (nbig of them)
    u32 nbig = 0;
    std::vector<u32> outs;
    // device copies
    Item *d_checks = nullptr;
    EqJob *d_eqjobs = nullptr;
    EvalSeg *d_segs = nullptr;
    LayerEval *d_levs = nullptr;
    std::vector<Item *> d_seg_items, d_lev_items;
    std::vector<Task *> d_groupsA, d_groupsB;
    u32 *d_ctr = nullptr;  // two task counters per wave launch (A groups, then B groups)
    LineWaveDev *d_lw = nullptr;
    BuildItem *d_builds = nullptr;
    HeavyItem *d_heavy = nullptr;
    SciDev *d_scis = nullptr;
    ProdWave *d_pw = nullptr;
    GenWave *d_gw = nullptr;
    RoundRef *d_rounds = nullptr;
    u32 *d_outs = nullptr;
    // execution
    cudaStream_t aux = nullptr;  // eq tables and product weights, concurrent with evaluation
    cudaStream_t cap = nullptr;  // private stream: graph capture, creation work
    cudaEvent_t ev_fork = nullptr, ev_tables = nullptr;
    cudaEvent_t ev_params = nullptr;  // a batch's parameter table was copied
    // stage events are recorded on a side branch of the graph (evs), so that
    // timing a stage adds no node between two launches (and keeps the final
    // reduction's programmatic dependence on the wave launch)
    // (one branch per stream whose stages are timed: a branch of its own
    // keeps the helper stream's marks from waiting for the main stream's)
    cudaStream_t evs = nullptr, evs_aux = nullptr;
    cudaEvent_t ev_mark = nullptr;
    struct vc_circuit *staged = nullptr;  // a single staged circuit: its own launch sequence
    cudaGraphExec_t exec = nullptr;
    // own_params: the graph's first node is the per-proof parameter write
    // (k_params), whose arguments are set on the instantiated graph before
    // each launch; the graph is kept because that update names its node
    bool own_params = false;
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t pnode = nullptr;
    cudaKernelNodeParams pkp{};
    cudaEvent_t stage_ev[2 * VC_NUM_STAGES] = {};
    bool stage_on = false;
};

struct vc_circuit {
    int device = 0;
    u32 flags = 0;                // VC_VALUES_IN_HOST_MEMORY
    bool eval_reads_inputs = false;  // the first evaluation launch can read the inputs in place
    PlanConfig cfg;
    u32 d = 0;
    std::vector<u32> s, kind, has_add;
    std::vector<std::vector<unsigned char>> ex_type;
    std::vector<std::vector<u32>> ex_in1, ex_in2;
    std::vector<std::vector<u32>> by1_off, by1_g, by2_off, by2_g;
    u64 tr_len = 0;
    u32 nchal = 0;
    u32 zd_off = 0;
    std::vector<u32> chal_off, z_off;
    std::vector<u64> tr_msg, tr_q;

    char *arena = nullptr;
    size_t arena_bytes = 0;
    char *host_vals = nullptr;  // mapped host memory of the layer values (VC_VALUES_IN_HOST_MEMORY)
    size_t host_bytes = 0;
    Globals G{};             // host copy of the circuit's globals
    Globals *d_G = nullptr;  // device copy (seed and tr written per call)
    std::vector<u64 *> V;
    u64 *d_tr = nullptr;
    u64 *d_vin = nullptr;  // VC_INPUTS_UPLOAD: the verifier's copy of page-locked host inputs
    u64 *d_result = nullptr;
    std::vector<LayerDev> L;
    LayerDev *d_layers = nullptr;
    std::vector<EqJob> eq_verify;
    EqJob *d_eq_verify = nullptr;
    u64 *partials = nullptr;
    VerifyDev Vd{};
    VerifyPtrs *d_vp = nullptr;        // per-call verifier pointers (device)
    // the verifier's own globals: coins, points and eq(z_i, r_P) in arrays of
    // its own, its status in word 1 of the status words; a verification never
    // writes what a proof on the handle reads
    Globals Gv{};
    Globals *d_Gv = nullptr;
    // vc_prove_verify: the proof and its verification in one captured graph
    // (the prover's and the verifier's parameter nodes set per call)
    cudaGraphExec_t pv_exec = nullptr;
    cudaGraph_t pv_graph = nullptr;
    cudaGraphNode_t pv_pnode = nullptr, pv_vnode = nullptr;
    cudaKernelNodeParams pv_pkp{}, pv_vkp{};
    cudaStream_t pv_vs = nullptr;  // the verifier's branch while the graph is captured
    cudaEvent_t pv_fork = nullptr, pv_join = nullptr;
    cudaGraphExec_t vexec = nullptr;   // the verifier's captured launches, parameter write first
    cudaGraph_t vgraph = nullptr;
    cudaGraphNode_t vpnode = nullptr;
    cudaKernelNodeParams vpkp{};
    // the verifier in two passes: input (coins and the input's MLE; a captured
    // graph) and transcript (everything else; plain launches)
    cudaGraphExec_t vin_exec = nullptr;
    cudaGraph_t vin_graph = nullptr;
    cudaGraphNode_t vin_node = nullptr;
    cudaKernelNodeParams vin_kp{};
    bool vin_pending = false;  // an input pass is queued and not yet consumed
    u64 vin_seed = 0;
    bool vin_sync = false;     // its inputs were host memory: the transcript pass reads the status
    std::vector<u32> explicit_layers;
    u32 *d_explicit_layers = nullptr;
    std::vector<VwireItem> vwire;  // the verifier's wiring-sum CTAs over the explicit layers
    VwireItem *d_vwire = nullptr;
    std::vector<u32> round_layer, zmap;
    u32 *d_round_layer = nullptr, *d_zmap = nullptr;
    // VC_VALUES_STAGED / VC_VALUES_WINDOWED: wide layers through W device
    // slots (V[i] = slot k mod W for the k-th wide layer), staged ones also in
    // page-locked host memory (hV); per-group task lists of the wave launches
    // (groups A and B), table builds and launch counters; a copy stream and
    // events (staged)
    std::vector<u64 *> hV;        // wide layers only (staged)
    // windowed: the proof's order of evaluations (a layer index >= 0) and
    // iteration groups run (-(g + 1))
    std::vector<int> wn_steps;
    // per layer: the evaluation step that launches it (a run of narrow layers,
    // at its first layer), -2 (inside such a run) or -1 (alone, per layer)
    std::vector<int> st_evalstep;
    std::vector<int> st_slot;     // per layer: its slot (wide layers) or -1 (kept on the device)
    u32 st_nslots = 0;            // W
    u64 st_link_bytes = 0;        // host-link bytes of one proof
    std::vector<int> st_group;    // per iteration: its group, or -1 (between narrow layers)
    std::vector<std::pair<u32, u32>> st_groups;  // first and last iteration of each group
    u64 *d_out = nullptr;  // copy of the outputs for the final reduction
    std::vector<std::vector<std::vector<Task>>> stA, stB;  // [list][wave group]: list g < ng = iteration
                                                          // group g, list ng = every iteration between
                                                          // narrow layers
    std::vector<std::vector<Task *>> d_stA, d_stB;
    std::vector<std::vector<BuildItem>> stBuild;  // [list]
    std::vector<BuildItem *> d_stBuild;
    std::vector<std::vector<Item>> stEval;  // [layer]: 256-gate blocks of k_eval_layer
    std::vector<Item *> d_stEval;
    LayerEval *d_stLev = nullptr;  // one descriptor per layer
    u32 *d_stctr = nullptr;        // two launch counters per (layer, group)
    std::vector<u32> stctr_off;    // per layer: its first counter
    cudaStream_t st_copy = nullptr;
    std::vector<cudaEvent_t> st_ev;  // per layer: evaluated, written to host, copied in, proved
    std::vector<int> eval_steps;  // >= 0: a segment; < 0: layer -step - 1 alone
    std::vector<u32> seg_maxblock;  // per segment: largest block of its run and tail
    Plan P;                       // this circuit alone (circ = 0)
    u64 *h_pinned = nullptr;      // small pinned buffer for status/result readback
    // per-gate prover (allocated on its first use)
    char *pg_arena = nullptr;
    PgLayer *d_pg = nullptr;
    u32 *d_pg_blk = nullptr, *d_pg_lblk = nullptr;
    u32 pg_nblk = 0, pg_nlblk = 0, pg_rounds = 0;
    cudaGraphExec_t pg_exec = nullptr;
};

struct vc_batch {
    int device = 0;
    std::vector<vc_circuit *> members;
    Plan P;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    CallParams *d_cp = nullptr;
    CallParams *h_cp = nullptr;  // pinned parameter table
    GatherChunk *d_gather = nullptr;  // the members' input copies, in chunks
    int ngather = 0;
};

vc_status cuda_status(cudaError_t e);
void init_device_once(int device);

// One proof of circuit c on stream st: its inputs (any memory the runtime can
// copy from) into the input layer, then its plan (resident or staged) with
// the transcript written to tr (device memory).  Asynchronous.
cudaError_t circuit_enqueue_proof(vc_circuit *c, const u64 *inputs, u64 seed, u64 *tr, cudaStream_t st);

// Host-side circuit construction: validation, offsets and the single-circuit
// plan, sized but not allocated (c->arena_bytes set).  circuit_allocate then
// takes the device memory and uploads everything.
vc_status circuit_prepare(const vc_circuit_desc *desc, int device, vc_circuit **out,
                          const PlanConfig *cfg = nullptr, u32 flags = 0);
// The tile shapes a circuit of this shape gets without explicit ones (the
// autotuned shapes of its size class, else the defaults).
PlanConfig shape_config(const vc_circuit_desc *desc);
vc_status circuit_allocate(vc_circuit *c);
void circuit_free(vc_circuit *c);

void plan_take(Plan &P, Arena &A, bool own_G);
bool plan_valid(const Plan &P);
cudaError_t plan_upload(Plan &P);                       // synchronous copies
cudaError_t plan_upload_async(Plan &P, cudaStream_t st);  // host vectors must stay unchanged until done
cudaError_t plan_resources(Plan &P);
void plan_release(Plan &P);
void plan_merge(Plan &B, const std::vector<vc_circuit *> &cs);
void enqueue_plan(Plan &P, cudaStream_t st);
void plan_drop_graph(Plan &P);
// The kernel node of `fn` in a captured graph (cudaErrorInvalidValue if none).
cudaError_t find_kernel_node(cudaGraph_t g, const void *fn, cudaGraphNode_t *node, cudaKernelNodeParams *kp);
void sort_tasks(Plan &P);
int count_launches(const Plan &P);
size_t plan_bytes(Plan &P, bool own_G);  // device bytes of the plan's descriptors

int ptr_kind(const void *p, int device, const void **mapped = nullptr);
// Status words: 0 = the prover's, 1 = the verifier's.  Queue the readback
// (and reset) of words [w0, w0 + n) on `st`; decode what was read back.
cudaError_t queue_status(vc_circuit *c, cudaStream_t st, int w0 = 0, int n = 1);
vc_status decode_status(const vc_circuit *c, int w0 = 0, int n = 1);
