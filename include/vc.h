/*
 * vc.h -- C ABI of the GB300 prover/verifier for the GKR/CMT interactive proof
 * over F_p, p = 2^61 - 1 (Thaler, Roberts, Mitzenmacher, Pfister, "Verifiable
 * Computation with Massively Parallel Interactive Proofs").
 *
 * The calls follow the paper's statement of the problem (Sec. 3.1): prover and
 * verifier agree on a layered arithmetic circuit of fan-in two; the prover
 * evaluates it, sends the outputs and then answers the verifier's random
 * challenges with polynomials; the verifier checks the answers for internal
 * consistency and finally compares the prover's last claim with one symbol of
 * the low-degree-extension encoding of the input (Sec. 2.2, Sec. 4.1.2).
 *
 * Conventions (the paper defers them to GKR/CMT; these are the readings taken):
 *   - layer 0 is the output layer, layer d the input layer; layer i has
 *     S_i = 2^{s_i} gates;
 *   - multilinear coordinate k (k >= 1) is bit k-1 of a gate index;
 *   - layer i's identity is summed over (p, w1, w2), bound in that order:
 *       V~_i(z) = sum eq(z,p) [add~_i (V~_{i+1}(w1) + V~_{i+1}(w2)) + mult~_i V~_{i+1}(w1) V~_{i+1}(w2)];
 *   - every round message is a degree-2 polynomial sent as its values at 0, 1, 2;
 *   - two claims about layer i+1 are reduced to one along l(t) = r1 + t (r2 - r1):
 *     the prover sends q(t) = V~_{i+1}(l(t)) for t = 0..s_{i+1};
 *   - the verifier's coins come from splitmix64 seeded with `seed` (a challenge
 *     is next() >> 3, redrawn while it equals p), drawn in this order: s_0
 *     output coordinates, then for each layer its s_i + 2 s_{i+1} round
 *     challenges and one line parameter tau.  Both parties replay the same
 *     stream, so the verifier's coins are fixed by the seed.
 *
 * Transcript layout (u64, every entry a canonical field element < p):
 *   [S_0 outputs]
 *   ++ for each layer i = 0..d-1:
 *        [3 (s_i + 2 s_{i+1}) round values: g_j(0), g_j(1), g_j(2) per round j]
 *        ++ [s_{i+1} + 1 line values q(0) .. q(s_{i+1})]
 *
 * Memory: every pointer argument may be host memory or CUDA device memory of
 * the circuit's device; the library detects which.  The caller owns inputs,
 * outputs and transcripts; the library owns circuits and all their device
 * scratch (allocated once by vc_circuit_create).  Device work is ordered on
 * `stream` (a cudaStream_t, NULL = the legacy default stream).
 *
 * Threads: calls on different circuit handles may run concurrently from
 * different host threads; calls on one handle must not overlap (they share
 * the handle's scratch).
 *
 * Errors: every call returns a vc_status; nothing is thrown across the ABI.
 * A verifier rejection is not an error: it is reported through *accept.
 */
#ifndef VC_H
#define VC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VC_OK = 0,
    VC_EINVAL = 1,    /* bad argument, bad circuit shape, non-canonical input */
    VC_ENOMEM = 2,    /* device or host allocation failed */
    VC_ECUDA = 3,     /* a CUDA runtime call failed */
    VC_ETIMEOUT = 4,  /* a bounded device-side wait gave up (reserved: no kernel of
                         this library waits on another, so nothing returns it) */
    VC_EBUSY = 5,     /* no free capacity (serving admission); a job already on the device */
    VC_ECANCELED = 6  /* a served job was cancelled before it reached the device */
} vc_status;

/* How layer i is wired to layer i+1 (Sec. 5.1.4: in-neighbour indices computed
 * from the gate index; Sec. 6.2.1: the benchmark circuits). */
typedef enum {
    VC_WIRE_SQUARE = 0,   /* gate g = MUL(g, g);                 s_i = s_{i+1}     */
    VC_WIRE_TREE = 1,     /* gate g = ADD(2g, 2g+1);             s_{i+1} = s_i + 1 */
    VC_WIRE_MATMULT = 2,  /* gate k + n j + n^2 i = MUL(i n + k, n^2 + k n + j);
                             s_i = 3L, s_{i+1} = 2L + 1, n = 2^L                    */
    VC_WIRE_F0_FIRST = 3, /* gate 2j = MUL(j, j), 2j+1 = ADD(j, j); s_i = s_{i+1} + 1 */
    VC_WIRE_F0_PAIR = 4,  /* gate 2j = MUL(2j, 2j), 2j+1 = MUL(2j+1, 2j); s_i = s_{i+1} */
    VC_WIRE_F0_FINAL = 5, /* gate j = MUL(2j+1, 2j+1);           s_{i+1} = s_i + 1 */
    VC_WIRE_EXPLICIT = 6  /* gate arrays supplied in vc_circuit_desc                */
} vc_wiring;

/* Layered circuit description (Sec. 3.1).  Arrays are read during
 * vc_circuit_create only and may be host memory. */
typedef struct {
    uint32_t n_layers;                 /* d >= 1: layers 0 (output) .. d (input)           */
    const uint32_t *log_width;         /* d + 1 entries, s_0 .. s_d, each <= 30             */
    const uint32_t *wiring;            /* d entries, vc_wiring of layer i -> i+1            */
    const uint8_t *const *gate_type;   /* d entries; for EXPLICIT layers: S_i bytes,
                                          0 = ADD, 1 = MUL; other entries may be NULL      */
    const uint32_t *const *in1;        /* d entries; EXPLICIT: S_i first in-neighbours     */
    const uint32_t *const *in2;        /* d entries; EXPLICIT: S_i second in-neighbours    */
} vc_circuit_desc;

typedef struct vc_circuit vc_circuit;

/* Validate a description, build the launch plan and allocate all device
 * scratch on `device`.  VC_EINVAL: widths do not fit a wiring kind, an
 * in-neighbour is out of range, or d = 0.  VC_ENOMEM: not enough device memory.
 * On success *out owns the circuit until vc_circuit_destroy. */
vc_status vc_circuit_create(const vc_circuit_desc *desc, int device, vc_circuit **out);

/* Residency of a circuit's layer values (Sec. 5.1: a circuit whose gates do
 * not fit in device memory).  With VC_VALUES_IN_HOST_MEMORY the values of
 * every layer (S_0 + ... + S_d u64, the bulk of a proof's memory) live in
 * pinned host memory mapped into the device's address space; evaluation
 * writes them and the sum-check reads them over the host link at every use
 * (the paper's copy-every-message strategy, with the link instead of copies).
 * Everything else stays in device memory and the transcript is unchanged. */
#define VC_VALUES_IN_HOST_MEMORY 1u

/* With VC_VALUES_STAGED the values of the wide layers (more than a quarter
 * of the widest) live in page-locked host memory and pass through W device
 * slots of the widest layer's size, W = floor(wide layers' values / widest
 * layer's values) clamped to [2, 8] (and to the number of wide layers), so
 * the slots never hold more than the wide layers would; narrow layers stay
 * on the device (Sec. 5.1.2, copy-once-per-layer: a layer
 * iteration needs only layers i and i+1 on the device).  A proof evaluates
 * the circuit layer by layer from the input up, writing each wide layer to
 * host memory once as soon as it is computed; then it runs every iteration
 * between narrow layers together, and the iterations that touch a wide layer
 * in order, in groups whose wide layers fit the slots, copying each group's
 * missing layers in from host memory once the slots' previous layers are no
 * longer needed.  Device memory for values: W S_max u64 plus the narrow
 * layers, instead of S_0 + ... + S_d.  Structured wirings only (EXPLICIT:
 * VC_EINVAL); such a circuit cannot join a batch (vc_batch_create:
 * VC_EINVAL) or use vc_prove_pergate (VC_EINVAL).  The transcript is
 * unchanged. */
#define VC_VALUES_STAGED 2u

/* With VC_VALUES_WINDOWED the wide layers pass through the same W device
 * slots as with VC_VALUES_STAGED, but never leave the device: since every
 * coin is known from the seed, a layer iteration can run as soon as its two
 * layers are evaluated, so a proof evaluates from the input up and, before a
 * layer overwrites a slot, runs every evaluated iteration not yet run (in one
 * merged set of launches, the narrow layers' iterations with the last set).
 * Device memory for values as with VC_VALUES_STAGED, no host memory and no
 * host-link traffic; the same restrictions (structured wirings only, no
 * batch, no vc_prove_pergate).  The transcript is unchanged. */
#define VC_VALUES_WINDOWED 8u

/* With VC_VALUES_AUTO the circuit gets device-resident values if their
 * memory can be had (from the device and within vc_set_memory_limit's cap),
 * else windowed values (VC_VALUES_WINDOWED; circuits with explicit wirings
 * skip this step), else values in mapped host memory; vc_circuit_get_info's
 * `residency` reports the choice.  VC_ENOMEM only when none fits. */
#define VC_VALUES_AUTO 4u

/* With VC_INPUTS_UPLOAD (device-resident values only: flags ==
 * VC_INPUTS_UPLOAD) page-locked host inputs given to vc_prove,
 * vc_verify_input or vc_verify are uploaded by one copy-engine transfer on
 * the call's stream (the prover's into its input layer, the verifier's into a
 * device buffer of its own, S_d more u64 of device memory) instead of being
 * read in place across the host link by the first kernel that needs them.
 * The calls stay asynchronous: the host buffer must stay unchanged until the
 * stream has passed the call.  Pageable host inputs are copied as without the
 * flag. */
#define VC_INPUTS_UPLOAD 16u

/* vc_circuit_create with residency flags (0, VC_VALUES_IN_HOST_MEMORY,
 * VC_VALUES_STAGED, VC_VALUES_WINDOWED, VC_VALUES_AUTO, or VC_INPUTS_UPLOAD;
 * VC_EINVAL for any other value; VC_ENOMEM if the device or pinned host
 * allocation fails). */
vc_status vc_circuit_create_ex(const vc_circuit_desc *desc, int device, uint32_t flags, vc_circuit **out);

/* Free the circuit and its device scratch (synchronises its device).  NULL is
 * accepted. */
vc_status vc_circuit_destroy(vc_circuit *c);

/* Transcript length in u64 for this circuit (fixed by its shape). */
vc_status vc_transcript_len(const vc_circuit *c, uint64_t *n_u64);

/* Device bytes the circuit holds (scratch + plan; layer values in host memory
 * are not counted). */
vc_status vc_circuit_bytes(const vc_circuit *c, uint64_t *bytes);

/* Layer-by-layer evaluation (Sec. 6.2.4: the prover's first step).
 * inputs: S_d canonical field elements; outputs: S_0 elements.  Synchronous:
 * returns after `outputs` is written.  VC_EINVAL if an input is >= p. */
vc_status vc_evaluate(vc_circuit *c, const uint64_t *inputs, uint64_t *outputs, void *stream);

/* Prover (Sec. 3.1, Sec. 4.1.1): evaluate the circuit on `inputs` (S_d
 * canonical elements) and write the whole transcript for the verifier coins
 * derived from `seed`.  transcript: vc_transcript_len() u64.
 * Inputs the device can address (device memory, or page-locked host memory
 * whose device address is its host address) are read in place by the first
 * evaluation launch, which writes them into the input layer; others are
 * copied first.  Either way they are read on `stream`, in stream order.
 * If `transcript` is device memory and `inputs` are read in place (device
 * memory, or page-locked host memory the device addresses) the call is
 * asynchronous with respect to the host: a non-canonical input is then
 * latched in the circuit and reported by the next vc_circuit_sync, and
 * page-locked inputs must stay unchanged until the proof is done.
 * Otherwise the call returns after the transcript is written and reports
 * VC_EINVAL itself. */
vc_status vc_prove(vc_circuit *c, const uint64_t *inputs, uint64_t seed,
                   uint64_t *transcript, void *stream);

/* The same proof computed the way the paper's GPU prover computes it
 * (Sec. 4.1.1; memory access in Sec. 5.1.4): in every round one thread per gate
 * adds that gate's independent contribution to the message, O(S log S) work
 * per layer, instead of folding tables.  The transcript is identical to
 * vc_prove's; arguments, asynchrony and errors are vc_prove's.  The first call
 * allocates the per-gate tables (about 2 S_i + 3 S_{i+1} u64 per layer;
 * VC_ENOMEM if they do not fit); they are freed with the circuit. */
vc_status vc_prove_pergate(vc_circuit *c, const uint64_t *inputs, uint64_t seed,
                           uint64_t *transcript, void *stream);

/* Wait for the circuit's queued work on `stream` and return (and clear) any
 * error latched by asynchronous calls. */
vc_status vc_circuit_sync(vc_circuit *c, void *stream);

/* Verifier (Sec. 2.2, Sec. 3.1, Sec. 4.1.2): replay the coins of `seed`,
 * check every round (g(0) + g(1) = running claim), every layer's final claim
 * against add~/mult~ at the bound point, and the last claim against the
 * input's multilinear extension at the final point.  *accept = 1 or 0.
 * A transcript entry >= p is a rejection, not an error.  If `accept`,
 * `inputs` and `transcript` are all device memory the call is asynchronous
 * (the int at `accept` is written on the stream; a non-canonical input is
 * latched for vc_circuit_sync); otherwise it returns after *accept is set and
 * reports VC_EINVAL for an input >= p itself. */
vc_status vc_verify(vc_circuit *c, const uint64_t *inputs, uint64_t seed,
                    const uint64_t *transcript, int *accept, void *stream);

/* The same verification in two passes (Sec. 2.2, Sec. 4.1.2).  The coins
 * are fixed by the seed, so the final point z_d is known before any message
 * arrives, and the verifier's one pass over the input (the input's
 * multilinear extension at z_d, the bulk of its work, in which every input
 * contributes independently) can run before or beside the proof.
 *
 * vc_verify_input queues that pass and the coins for `seed`.  `inputs` (S_d
 * canonical u64) must be device memory of the circuit's device or
 * page-locked host memory the device can address (VC_EINVAL otherwise); it
 * is read in place, so it must stay unchanged until the pass has run.  The
 * pass writes only the verifier's own scratch: its device work may run on
 * another stream concurrently with a vc_prove on the same handle (the host
 * calls themselves must not overlap, and no other call on the handle may run
 * between it and its vc_verify_transcript).  It is always asynchronous.
 *
 * vc_verify_transcript queues the rest for the same seed: the claimed
 * outputs' multilinear extension, every round and layer check, the final
 * comparison with the input pass's value.  It must be ordered after the
 * input pass on the device (same stream, or an event).  VC_EINVAL: no input
 * pass was queued since the last transcript pass or vc_verify, or it was for
 * another seed.  It is asynchronous when `transcript` and `accept` are
 * device memory and the input pass read device memory; otherwise it returns
 * after *accept is set and reports VC_EINVAL for an input >= p.  The accept
 * bit equals vc_verify's for the same arguments. */
vc_status vc_verify_input(vc_circuit *c, const uint64_t *inputs, uint64_t seed, void *stream);
vc_status vc_verify_transcript(vc_circuit *c, uint64_t seed, const uint64_t *transcript, int *accept,
                               void *stream);

/* Prove and verify in one call (Sec. 3.1's prover and verifier, the
 * verifier checking the prover's transcript): the proof as vc_prove, the
 * verifier's input pass (its coins and the inputs' multilinear extension at
 * its final point, fixed by the seed alone) beside it, and the checks of the
 * transcript after the proof, all one CUDA graph launch on `stream`.  The
 * verifier reads the inputs where the prover does: in place, or from the
 * input layer that the library's own copy filled (pageable host inputs, or
 * page-locked ones with VC_INPUTS_UPLOAD), which no launch writes.
 * transcript and accept: device or host memory.  Asynchronous (statuses
 * latched, read by vc_circuit_sync) when transcript and accept are device
 * memory and the inputs were not a pageable copy; otherwise it returns after
 * both are written.  The transcript and the accept bit equal those of
 * vc_prove followed by vc_verify.  VC_EINVAL for circuits whose values pass
 * through device slots (VC_VALUES_STAGED, VC_VALUES_WINDOWED) and for an
 * input >= p (from the call, or latched). */
vc_status vc_prove_verify(vc_circuit *c, const uint64_t *inputs, uint64_t seed, uint64_t *transcript, int *accept,
                          void *stream);

/* Stages of a proof, for timing them.  A proof runs on the caller's stream;
 * the coins, eq tables and product weights run on a helper stream owned by
 * the circuit (forked from and joined back to the caller's stream),
 * concurrently with the evaluation.  The sum-check waves and line reductions of all
 * layers run as persistent launches that take their chunks from a shared
 * task counter. */
typedef enum {
    VC_STAGE_PROOF = 0,     /* the whole proof                                           */
    VC_STAGE_TABLES = 1,    /* one launch: coins, layer points, eq(z_i, r_P), split eq
                               tables, product weights                   (helper stream) */
    VC_STAGE_EVAL = 2,      /* layer-by-layer evaluation                                  */
    VC_STAGE_WAVES = 3,     /* first persistent launch: line reductions, product-weighted
                               and on-the-fly general sum-checks (their single-chunk
                               later waves run inside it)                                */
    VC_STAGE_WAVESN = 4,    /* later persistent launches of the same kinds (wide layers) */
    VC_STAGE_BUILD = 5,     /* phase-2/3 wiring tables (MATMULT, F0, EXPLICIT layers)    */
    VC_STAGE_TABWAVES = 6,  /* general sum-checks over the built tables                  */
    VC_STAGE_FINAL = 7,     /* per-round reductions into the transcript                  */
    VC_NUM_STAGES = 8
} vc_stage;

/* Record CUDA events around the stages of every later vc_prove on this
 * circuit: events[2k] when stage k can start (the work before it is done)
 * and events[2k+1] when it has ended; a stage with no work for this circuit
 * records nothing.  `events` must hold 2 * VC_NUM_STAGES entries: cudaEvent_t
 * created on the circuit's device and owned by the caller, or NULL to skip
 * that mark (record only the stages you time: marks of one stream are
 * recorded in order, so a mark may wait for the one before it).  events ==
 * NULL turns recording off.  A proof replays a CUDA graph of its launches,
 * captured by the first vc_prove after the circuit's creation or after this
 * call; the events are event-record nodes of that graph, on side branches
 * that no launch waits for (timing a stage adds no step between launches).
 * The call must not overlap a proof in flight on the circuit (it may replace
 * the graph). */
vc_status vc_circuit_set_stage_events(vc_circuit *c, void *const *events);

/* Shape facts of a circuit. */
typedef struct {
    uint32_t n_layers;           /* d                                             */
    uint32_t n_rounds;           /* sum-check rounds over all layers              */
    uint64_t transcript_len;     /* u64 entries                                   */
    uint64_t gates;              /* non-input gates                               */
    uint64_t device_bytes;       /* scratch + plan held on the device             */
    uint32_t prove_launches;     /* kernel launches per vc_prove                  */
    uint32_t verify_launches;    /* kernel launches per vc_verify                 */
    uint32_t wave_tasks;         /* chunks in the first persistent wave launch    */
    uint32_t verify2_launches;   /* kernel launches per vc_verify_input +
                                    vc_verify_transcript                          */
    uint64_t link_bytes;         /* VC_VALUES_STAGED: layer-value bytes one
                                    vc_prove moves over the host link (each wide
                                    layer written once, plus the layers copied
                                    back in); 0 otherwise                         */
    uint32_t residency;          /* 0, VC_VALUES_IN_HOST_MEMORY, VC_VALUES_STAGED
                                    or VC_VALUES_WINDOWED: where the layer values
                                    live                                          */
    uint32_t pad;
} vc_circuit_info;

vc_status vc_circuit_get_info(const vc_circuit *c, vc_circuit_info *info);

/* Tile shapes of a circuit's launch plan: rounds folded by a first
 * product-weighted / general sum-check chunk (<= 13 / <= 12), coordinates
 * folded by a first line-reduction chunk (<= 13), the smallest evaluation
 * chunk (log2 entries, <= 11), and pr_split_log: product-weighted instances
 * of fewer than 2^pr_split_log entries use chunks half as large (they are
 * dispatched after the larger ones, so finer chunks even out the end of the
 * persistent launch; 0 = never, VC_SPLIT_WIDEST = the circuit's widest
 * layer, else <= 40).  Any choice gives the same transcript; they only
 * change speed. */
#define VC_SPLIT_WIDEST 0xFFFFFFFFu
typedef struct {
    uint32_t pr_chunk_log;
    uint32_t gn_chunk_log;
    uint32_t line_chunk_log;
    uint32_t eval_chunk_log;
    uint32_t pr_split_log;
} vc_tile_config;

/* Autotuner: times `reps` proofs of a circuit of shape `desc` (structured
 * wirings only) with candidate tile shapes (coordinate descent from the
 * current choice, on this device), records the fastest for the shape's size
 * class (depth, widest layer, its wiring kind) and returns it with its mean
 * proof time in ms.  Circuits created later in this process with a shape of
 * that class use the recorded tiles (circuits that exist keep theirs).
 * Allocates and frees scratch; synchronous. */
vc_status vc_autotune(const vc_circuit_desc *desc, int device, int reps, vc_tile_config *best, double *best_ms);

/* Autotuner for a batch: the same search, but every candidate is one tile
 * configuration for all n shapes (structured wirings only) and is timed as
 * their merged batch (vc_batch_prove, `reps` timed proofs after two untimed
 * ones, every member on zero inputs), starting from each circuit's default
 * shapes; coordinate descent until a pass improves nothing (at most two
 * passes).  The chosen configuration is recorded for the size class of every
 * shape, so circuits of these shapes created later use it, and returned with
 * the batch's mean proof time in ms.  Creates and frees the candidate
 * circuits and batches; synchronous. */
vc_status vc_autotune_batch(const vc_circuit_desc *descs, int n, int device, int reps, vc_tile_config *best,
                            double *best_ms);

/* vc_circuit_create with explicit tile shapes (VC_EINVAL outside the
 * bounds above). */
vc_status vc_circuit_create_tiles(const vc_circuit_desc *desc, int device, const vc_tile_config *tiles,
                                  vc_circuit **out);

/* The tile shapes a circuit was planned with. */
vc_status vc_circuit_get_tiles(const vc_circuit *c, vc_tile_config *tiles);

/* Batches (Sec. 6.2.3 runs many independent proofs; here they share launches).
 * A batch is a fixed set of distinct circuit handles on one device whose
 * proofs run as ONE set of merged launches: every evaluation step, line wave
 * and sum-check wave of every member is one work list, so n small proofs cost
 * about the launches of one.  A batch keeps its own launch plan and a small
 * parameter table on the device; the members keep their scratch, so a member
 * must not be used by another call while a batch proof that includes it is in
 * flight.  The first vc_batch_prove captures the launches into a CUDA graph;
 * later calls replay it. */
typedef struct vc_batch vc_batch;

/* circuits: n >= 1 distinct handles on one device (VC_EINVAL otherwise).  The
 * handles must outlive the batch. */
vc_status vc_batch_create(vc_circuit *const *circuits, int n, vc_batch **out);

/* Free the batch (synchronises its device); the members are untouched.  NULL
 * is accepted. */
vc_status vc_batch_destroy(vc_batch *b);

/* Prove every member: inputs[j], seeds[j], transcripts[j] for member j, with
 * vc_prove's pointer rules.  Asynchronous when every pointer is device memory
 * (errors latched, reported by vc_batch_sync); otherwise returns after all
 * transcripts are written and reports VC_EINVAL for a non-canonical input. */
vc_status vc_batch_prove(vc_batch *b, const uint64_t *const *inputs, const uint64_t *seeds,
                         uint64_t *const *transcripts, void *stream);

/* Wait for the batch's queued work on `stream`; return (and clear) the worst
 * error latched by any member. */
vc_status vc_batch_sync(vc_batch *b, void *stream);

typedef struct {
    uint32_t n_members;
    uint32_t prove_launches;  /* kernel launches per vc_batch_prove (all members) */
    uint64_t device_bytes;    /* plan + parameter table held by the batch         */
    uint64_t gates;           /* non-input gates over all members                 */
} vc_batch_info;

vc_status vc_batch_get_info(const vc_batch *b, vc_batch_info *info);

/* One-shot batch: vc_batch_create + vc_batch_prove + vc_batch_sync +
 * vc_batch_destroy.  Synchronous.  For repeated batches of the same circuits
 * keep a vc_batch instead (it skips the planning and the graph capture). */
vc_status vc_prove_batch(vc_circuit *const *circuits, const uint64_t *const *inputs,
                         const uint64_t *seeds, uint64_t *const *transcripts, int n,
                         void *stream);

/* Proof server (serving form of the prover; the paper has no counterpart).
 * A request loop owned by one worker thread: submitted jobs are admitted in
 * arrival order while the circuits they need fit under a device-memory cap,
 * admitted jobs are merged into launch sets (one set of merged launches for
 * all of them, as for vc_batch), and up to `max_inflight` sets run at once on
 * their own streams, so jobs that arrive while others are on the GPU are
 * admitted as slots and memory free up and their work overlaps on the device
 * (continuous batching).  Circuits are pooled by shape and stay resident
 * between jobs.  Structured wirings only (EXPLICIT layers: VC_EINVAL). */
typedef struct vc_server vc_server;

typedef struct {
    uint64_t mem_cap_bytes;  /* device bytes for resident circuits (0 = 150 GiB) */
    uint32_t max_batch;      /* jobs per launch set (0 = 16)                     */
    uint32_t max_inflight;   /* launch sets on the device at once (0 = 4, max 8) */
    uint32_t pr_split_log;   /* the server's circuits: product-weighted instances
                                below 2^pr_split_log entries use half-size chunks
                                (vc_tile_config; 0 = each circuit's own shapes) */
    uint32_t pad;
} vc_server_config;

typedef struct {
    int done;                /* 1 once the transcript is written                 */
    vc_status status;        /* the job's result (VC_EINVAL: non-canonical input) */
    uint64_t submit_ns;      /* steady-clock times: submitted, admitted, finished */
    uint64_t start_ns;
    uint64_t done_ns;
} vc_job_info;

typedef struct {
    uint64_t submitted, completed, launch_sets;
    uint64_t circuits_created, circuits_evicted;
    uint64_t held_bytes, peak_held_bytes, pending;
    uint32_t max_jobs_in_flight;
    uint32_t cancelled;      /* jobs cancelled before admission (counted in completed) */
} vc_server_stats;

/* Start a server on `device` (cfg may be NULL for the defaults). */
vc_status vc_server_create(int device, const vc_server_config *cfg, vc_server **out);

/* Finish every submitted job, then stop the worker and free everything. */
vc_status vc_server_destroy(vc_server *s);

/* Queue one proof: circuit shape `desc` (host memory, read during the call),
 * S_d canonical inputs and a transcript buffer of the shape's length, each
 * host or device memory; both must stay valid until the job is done.  Returns
 * at once with *job_id.  A shape whose circuit with device-resident values
 * exceeds the memory cap is proved with windowed values
 * (VC_VALUES_WINDOWED), alone in its launch set.  VC_EINVAL: bad shape or
 * pointer; VC_EBUSY: even with windowed values one circuit of this shape
 * exceeds the memory cap. */
vc_status vc_server_submit(vc_server *s, const vc_circuit_desc *desc, const uint64_t *inputs,
                           uint64_t seed, uint64_t *transcript, uint64_t *job_id);

/* Job state without blocking.  Once a call reports done = 1 the job is
 * forgotten (its id becomes invalid).  One consumer per job: while a
 * vc_server_wait on the job is blocked, poll and wait on it from other
 * threads return VC_EINVAL. */
vc_status vc_server_poll(vc_server *s, uint64_t job_id, vc_job_info *info);

/* Block until the job is done, report it and forget it.  VC_EINVAL for an
 * unknown id or one another thread is already waiting on. */
vc_status vc_server_wait(vc_server *s, uint64_t job_id, vc_job_info *info);

vc_status vc_server_get_stats(vc_server *s, vc_server_stats *stats);

/* Cancel a job that is still queued (not yet admitted to a launch set): it is
 * removed from the queue and completes at once with status VC_ECANCELED (a
 * poll or wait still reports it, then forgets it); its inputs and transcript
 * buffer are no longer used.  VC_EBUSY if the job is already on the device or
 * done (it then completes normally); VC_EINVAL for an unknown id. */
vc_status vc_server_cancel(vc_server *s, uint64_t job_id);

/* Library-wide memory budget (the paper has no counterpart).  Caps the bytes
 * of device memory and of page-locked host memory that this library holds at
 * once, over all circuits, batches, servers and special-purpose states of the
 * process (0 = no cap, the default).  An allocation past a cap fails before
 * any CUDA call, as a refused cudaMalloc would: the call that needed it
 * returns VC_ENOMEM and frees what it had taken, and a served job that
 * needed a new circuit completes with status VC_ENOMEM while other jobs go
 * on.  Lowering a cap below what is held frees nothing; later allocations
 * fail until enough is released.  Never fails. */
vc_status vc_set_memory_limit(uint64_t device_bytes, uint64_t pinned_bytes);

/* Bytes of device and page-locked host memory the library holds now (either
 * pointer may be NULL, not both: VC_EINVAL). */
vc_status vc_get_memory_usage(uint64_t *device_bytes, uint64_t *pinned_bytes);

/* ---- Special-purpose non-interactive F2 protocol (Sec. 3.2; Sec. 4.2;
 * Sec. 6.3).  The frequency vector a of n = v h entries is a v x h grid,
 * a(x, y) at x h + y (row-major).  Let u = 37^((p-1)/(2h)) (37 generates
 * F_p^*), so u has order 2h and w = u^2 order h.  Row x is the polynomial f_x
 * of degree < h with f_x(w^y) = a(x, y), y = 0..h-1.  The proof is
 * s(Y) = sum_x f_x(Y)^2 at the points u^k, k = 0..2h-1 (2h u64; the even
 * points are the nodes): proof length 2h words, verifier space v words.
 * The verifier keeps f_x(r) for a secret random r (drawn from its seed like
 * the GKR coins: the first accepted splitmix64 draw), accepts iff
 * s(r) = sum_x f_x(r)^2, and answers F2 = sum_{k even} s(u^k).  No
 * interaction.  Nodes of a multiplicative subgroup let the prover extend each
 * row with the Prime Factor FFT (Sec. 4.2, 5.2): h must divide (p - 1) / 2
 * with every prime-power factor at most 61, i.e. h is a product of distinct
 * members of {3 or 9, 5 or 25, 7, 11, 13, 31, 41, 61}.  Inputs must be
 * canonical (< p). */
typedef struct vc_f2sp vc_f2sp;
#define VC_F2SP_MAX_H 7000u

/* Transform tables for h and scratch for v rows on `device`.  VC_EINVAL:
 * v = 0, h > VC_F2SP_MAX_H, or h not of the form above. */
vc_status vc_f2sp_create(uint64_t v, uint64_t h, int device, vc_f2sp **out);
vc_status vc_f2sp_destroy(vc_f2sp *s);

/* Prover: proof[k] = s(u^k), k = 0..2h-1, for the v h entries at `a` (host or
 * device).  Synchronous; VC_EINVAL for an entry >= p (the proof is then
 * undefined). */
vc_status vc_f2sp_prove(vc_f2sp *s, const uint64_t *a, uint64_t *proof, void *stream);

/* Streaming verifier: begin draws r from `seed` and clears the row values;
 * absorb adds the contribution of whole rows [first_row, first_row + nrows)
 * given contiguously at `rows` (host or device; a row may be absorbed in
 * several parts as additive updates of its counts); end checks `proof`
 * (2h u64, host or device), sets *accept (1 or 0; an entry >= p is a
 * rejection) and *f2 = sum of the proof's even entries, synchronously.
 * VC_EINVAL from end if an absorbed entry was >= p.  begin and absorb are
 * asynchronous.  Device rows are read in place (keep them until end).  Host
 * rows stream through two device buffers of about 16 MB of whole rows
 * (Sec. 4.2's double buffering): each chunk is copied on the verifier's own
 * copy stream into one buffer while the previous chunk is absorbed from the
 * other, and the alternation carries over from one absorb call to the next;
 * absorb returns once the last of its rows has been copied, so the caller
 * may refill its host buffer while the absorbs run.  The buffers are
 * allocated by the first absorb of host rows (VC_ENOMEM if they cannot be). */
vc_status vc_f2sp_verify_begin(vc_f2sp *s, uint64_t seed, void *stream);
vc_status vc_f2sp_verify_absorb(vc_f2sp *s, const uint64_t *rows, uint64_t first_row, uint64_t nrows,
                                void *stream);

/* As vc_f2sp_verify_absorb, but for host rows it returns once the rows of
 * the previous absorb call have been copied (at once for the first call), so
 * the copy engine never waits for the host: a caller alternating two (or
 * more) host buffers refills the one it passed two calls ago.  The rows of
 * the last call are in use until vc_f2sp_verify_end returns.  Device rows
 * behave as with vc_f2sp_verify_absorb. */
vc_status vc_f2sp_verify_absorb_async(vc_f2sp *s, const uint64_t *rows, uint64_t first_row, uint64_t nrows,
                                      void *stream);
vc_status vc_f2sp_verify_end(vc_f2sp *s, const uint64_t *proof, uint64_t *f2, int *accept, void *stream);

/* Elementwise field product out[k] = a[k] b[k] mod p on the device (device
 * pointers, n elements, canonical inputs).  Used to check the device field
 * arithmetic.  Asynchronous. */
vc_status vc_field_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n,
                       void *stream);

/* Integer-arithmetic rate microbenchmarks (the denominators of the prover's
 * roofline; the paper has no counterpart).  Each runs `iters` steps of
 * independent dependency chains per thread over a grid of exactly one wave
 * (every SM holding as many 256-thread CTAs as fit), times the launch with
 * CUDA events after a warm-up launch, and returns units per second in *rate.
 * variant 0: canonical 32-bit-limb Mersenne product + add (8 chains; units:
 * field products); 1: canonical 64x64->128 product, fold, add (8 chains;
 * field products); 2: the product-weighted sum-check pair step of the
 * dominant kernel (two exact 128-bit multiply-adds and one lazily reduced
 * fold, counted as three field products), the best of 2, 4 and 8 pairs per
 * thread at several register budgets; 3: 32-bit integer multiply-adds (8
 * chains; units: multiply-adds); 4: exact 64x64->128-bit multiply-accumulates
 * (8 accumulators; units: multiply-accumulates).  Synchronous; VC_EINVAL for
 * another variant or iters = 0, VC_ECUDA on a CUDA error. */
vc_status vc_field_mul_rate(int device, int variant, uint64_t iters, double *rate);

/* Circuit evaluation that allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library call.  It exists for callers that cannot allocate device
 * memory, such as a process whose device memory is entirely reserved by
 * another framework's caching allocator, or code that must not trigger the
 * device-wide synchronisation a cudaMalloc or cudaFree can cause.  It has no
 * counterpart in the paper: it is vc_evaluate without a circuit handle.
 *
 * desc: the circuit shape (host memory; structured wiring kinds only, an
 * EXPLICIT layer is VC_EINVAL).  inputs: S_d canonical elements and outputs:
 * S_0 elements, both device memory of the current device (VC_EINVAL
 * otherwise).  The intermediate layers 1..d-1 are kept in one fixed device
 * array of 2^20 field elements (8 MiB); a circuit whose intermediate layers
 * need more is rejected with VC_EINVAL before any work is queued.  Every GPU on
 * which this function has run keeps that array until the process exits.
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: after a cudaDeviceReset of
 * that device it is stale, so do not call this function after one.  A CUDA
 * error already pending when it is called (left by other code) is not
 * cleared: the call returns VC_ECUDA without queuing work.  All calls
 * share the one array and it keeps the last call's contents, so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise them.
 * Synchronous: returns after `outputs` is written; VC_EINVAL if an input is
 * >= p. */
vc_status vc_evaluate_noalloc(const vc_circuit_desc *desc, const uint64_t *inputs, uint64_t *outputs,
                              void *stream);

/* Human-readable name of a status code (static string). */
const char *vc_status_string(vc_status s);

#ifdef __cplusplus
}
#endif

#endif /* VC_H */
