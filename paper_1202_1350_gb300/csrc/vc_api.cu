// vc_api.cu -- C ABI (include/vc.h): circuit validation, launch planning,
// device scratch, and the launch sequences of the prover and the verifier.
//
// Planning happens once per circuit: the widths and wiring kinds fix every
// table size, every chunk of every sum-check wave, every transcript offset and
// every challenge index, so vc_circuit_create lays all of it out in one device
// arena and uploads the descriptors.  A proof then only replays the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "plan.h"
#include "vc.h"


namespace {

constexpr u32 PR_CHUNK_LOG = PR_M + 8;  // entries folded by one PROD CTA (256 threads x 2^PR_M)
constexpr u32 GN_CHUNK_LOG = GN_M + 7;  // entries folded by one GEN CTA (128 threads x 2^GN_M)

// Which layers' phase-2/3 tables are built by k_build23 (the rest are formed
// on the fly or never stored).
static bool needs_tables(u32 kind) { return kind != W_SQUARE && kind != W_TREE; }
constexpr u32 LN_CHUNK0_LOG = 11;  // coordinates folded by the first line wave
constexpr u32 LN_CHUNKW_LOG = 9;   // coordinates folded by later line waves

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

}  // namespace

struct vc_circuit {
    int device = 0;
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

    // device arena and the descriptors that point into it
    char *arena = nullptr;
    size_t arena_bytes = 0;
    Globals G{};
    std::vector<u64 *> V;
    u64 *d_tr = nullptr;
    u64 *d_result = nullptr;
    std::vector<LayerDev> L;
    LayerDev *d_layers = nullptr;
    std::vector<EqJob> eq_prove, eq_verify;
    EqJob *d_eq_prove = nullptr, *d_eq_verify = nullptr;
    std::vector<LineWaveDev> lw;
    LineWaveDev *d_lw = nullptr;
    std::vector<std::vector<Item>> line_items;
    std::vector<Item *> d_line_items;
    std::vector<u32> build_off;
    u32 *d_build_off = nullptr;
    int build_blocks = 0;
    std::vector<SciDev> scis;
    SciDev *d_scis = nullptr;
    std::vector<ProdWave> pwaves;
    ProdWave *d_pwaves = nullptr;
    std::vector<std::vector<Item>> p_items;
    std::vector<Item *> d_p_items;
    std::vector<GenWave> gwaves;
    GenWave *d_gwaves = nullptr;
    std::vector<std::vector<Item>> g_items;
    std::vector<Item *> d_g_items;
    std::vector<RoundRef> rounds;
    RoundRef *d_rounds = nullptr;
    u64 *partials = nullptr;
    u64 n_partials = 0;
    VerifyDev Vd{};
    EqTab tzd{};
    std::vector<u32> explicit_layers;
    u32 *d_explicit_layers = nullptr;
    u64 *h_pinned = nullptr;  // small pinned buffer for status/result readback
    // evaluation steps: seg >= 0 -> eval_segs[seg]; else per-layer launch of layer (-seg - 1)
    std::vector<EvalSeg> eval_segs;
    std::vector<int> eval_steps;
    std::vector<u32> round_layer;
    u32 *d_round_layer = nullptr;
    cudaEvent_t stage_ev[2 * VC_NUM_STAGES] = {};
    bool stage_on = false;
    // helper streams and the fork/join events of a proof
    cudaStream_t aux[2] = {};
    cudaEvent_t ev_fork = nullptr, ev_tables = nullptr, ev_eval = nullptr, ev_build = nullptr, ev_prod = nullptr,
                ev_gen = nullptr;
    bool has_tab = false;
};

static vc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VC_OK : (e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA); }

// Validate the layer description against the wiring kinds (the same shape
// rules as the header's vc_wiring comments).
static bool shape_ok(u32 kind, u32 si, u32 sn)
{
    switch (kind) {
    case W_SQUARE: return si == sn;
    case W_TREE: return sn == si + 1;
    case W_MATMULT: return si % 3 == 0 && sn == 2 * (si / 3) + 1;
    case W_F0_FIRST: return si == sn + 1;
    case W_F0_PAIR: return si == sn && si >= 1;
    case W_F0_FINAL: return sn == si + 1;
    case W_EXPLICIT: return true;
    default: return false;
    }
}

static EqTab take_eq(Arena &A, const u64 *pt, u32 n)
{
    EqTab t{};
    t.n = n;
    t.h = (n + 1) / 2;
    t.pt = pt;
    t.lo = A.take<u64>(size_t(1) << t.h);
    t.hi = A.take<u64>(size_t(1) << (n - t.h));
    return t;
}

// Evaluation plan: runs of block-local layers (every kind but MATMULT and
// EXPLICIT) go to one k_eval_seg launch each; a CTA takes 2^c entries of the
// run's input layer (about 256 CTAs for wide layers) and keeps going while its
// block stays >= 32 entries (or while one CTA covers the whole layer) and
// <= 4096 entries.
static void plan_eval(vc_circuit *c)
{
    c->eval_segs.clear();
    c->eval_steps.clear();
    int i = (int)c->d - 1;
    auto local = [&](int j) { return c->kind[j] != W_MATMULT && c->kind[j] != W_EXPLICIT; };
    while (i >= 0) {
        if (!local(i)) {
            c->eval_steps.push_back(-i - 1);
            i--;
            continue;
        }
        const int s_in = (int)c->s[i + 1];
        int cl = std::min(s_in, std::max(s_in - 8, 10));
        cl = std::min(cl, 12);
        int i_lo = i + 1;
        while (true) {
            int e = cl, j = i;
            i_lo = i + 1;
            const bool whole = (cl == s_in);
            while (j >= 0 && local(j)) {
                const int ne = e + (int)c->s[j] - (int)c->s[j + 1];
                if (ne < 0 || ne > 12 || (!whole && ne < 5)) break;
                if (c->kind[j] == W_F0_PAIR && ne < 1) break;
                e = ne;
                i_lo = j;
                j--;
            }
            if (i_lo <= i || cl == 0) break;
            cl--;  // the first layer did not fit: smaller chunks
        }
        if (i_lo > i) {  // no run possible: evaluate this layer alone
            c->eval_steps.push_back(-i - 1);
            i--;
            continue;
        }
        EvalSeg S{};
        S.i_hi = (u32)i;
        S.i_lo = (u32)i_lo;
        S.c = (u32)cl;
        S.nchunks = 1u << (s_in - cl);
        S.check_input = (u32)(i + 1 == (int)c->d);
        c->eval_steps.push_back((int)c->eval_segs.size());
        c->eval_segs.push_back(S);
        i = i_lo - 1;
    }
}

static void enqueue_eval(vc_circuit *c, const Globals &G, cudaStream_t st)
{
    for (int step : c->eval_steps) {
        if (step >= 0) launch_eval_seg(G, c->eval_segs[step], st);
        else launch_eval_layer(G, c->L[-step - 1], -step - 1, st);
    }
}

// Lay out every buffer and descriptor relative to `base` (0 for sizing).
static size_t layout(vc_circuit *c, uintptr_t base)
{
    Arena A;
    A.base = base;
    const u32 d = c->d;
    auto S = [&](u32 i) { return u64(1) << c->s[i]; };

    c->V.assign(d + 1, nullptr);
    for (u32 i = 0; i <= d; i++) c->V[i] = A.take<u64>(S(i));
    Globals &G = c->G;
    G.d = d;
    G.nchal = c->nchal;
    G.chal = A.take<u64>(c->nchal + 1);
    u32 npts = 0;
    for (u32 i = 0; i <= d; i++) npts += c->s[i];
    G.pts = A.take<u64>(npts + 1);
    G.scal = A.take<u64>(2 * d + 2);
    G.status = A.take<u32>(16);
    G.invfact = A.take<u64>(64);
    c->d_result = A.take<u64>(8);
    c->d_tr = A.take<u64>(c->tr_len);

    // layers and their eq tables
    c->L.assign(d, LayerDev{});
    c->eq_prove.clear();
    c->eq_verify.clear();
    c->explicit_layers.clear();
    for (u32 i = 0; i < d; i++) {
        LayerDev &L = c->L[i];
        L.s = c->s[i];
        L.sn = c->s[i + 1];
        L.kind = c->kind[i];
        L.has_add = c->has_add[i];
        L.chal_off = c->chal_off[i];
        L.z_off = c->z_off[i];
        L.V = c->V[i];
        L.Vn = c->V[i + 1];
        L.tr_msg = c->tr_msg[i];
        L.tr_q = c->tr_q[i];
        const u64 *r = G.chal + L.chal_off;
        L.tz = take_eq(A, G.pts + L.z_off, L.s);
        L.trp = take_eq(A, r, L.s);
        L.tr1 = take_eq(A, r + L.s, L.sn);
        L.tr2 = take_eq(A, r + L.s + L.sn, L.sn);
        c->eq_prove.push_back({L.tz});
        c->eq_prove.push_back({L.trp});
        c->eq_prove.push_back({L.tr1});
        const bool tabs = needs_tables(L.kind);
        L.P2 = tabs ? A.take<u64>(S(i + 1)) : nullptr;
        L.P3 = tabs ? A.take<u64>(S(i + 1)) : nullptr;
        L.B2 = (tabs && L.has_add) ? A.take<u64>(S(i + 1)) : nullptr;
        L.B3 = (tabs && L.has_add) ? A.take<u64>(S(i + 1)) : nullptr;
        if (L.kind == W_EXPLICIT) {
            L.type = A.take<unsigned char>(S(i));
            L.in1 = A.take<u32>(S(i));
            L.in2 = A.take<u32>(S(i));
            L.by1_off = A.take<u32>(S(i + 1) + 1);
            L.by1_g = A.take<u32>(S(i));
            L.by2_off = A.take<u32>(S(i + 1) + 1);
            L.by2_g = A.take<u32>(S(i));
            c->explicit_layers.push_back(i);
            c->eq_verify.push_back({L.trp});
            c->eq_verify.push_back({L.tr1});
            c->eq_verify.push_back({L.tr2});
        }
    }
    c->tzd = take_eq(A, G.pts + c->zd_off, c->s[d]);
    c->eq_verify.push_back({c->tzd});
    c->eq_verify.push_back({c->L[0].tz});

    // line reduction waves
    c->lw.clear();
    c->line_items.clear();
    for (u32 i = 0; i < d; i++) {
        const u32 n = c->s[i + 1];
        u32 l0 = 0;
        const u64 *in = c->V[i + 1];
        for (u32 w = 0;; w++) {
            const u32 cap = (w == 0) ? LN_CHUNK0_LOG : LN_CHUNKW_LOG;
            const u32 nl = std::min(cap, n - l0);
            LineWaveDev W{};
            W.layer = i;
            W.n = n;
            W.l0 = l0;
            W.nl = nl;
            W.nchunks = u32(1) << (n - l0 - nl);
            W.last = (l0 + nl == n);
            W.in = in;
            W.out = W.last ? nullptr : A.take<u64>(size_t(W.nchunks) * (l0 + nl + 1));
            W.a_off = c->chal_off[i] + c->s[i];
            W.b_off = c->chal_off[i] + c->s[i] + n;
            W.tr_q = c->tr_q[i];
            if (c->line_items.size() <= w) c->line_items.resize(w + 1);
            const u32 idx = (u32)c->lw.size();
            c->lw.push_back(W);
            for (u32 ch = 0; ch < W.nchunks; ch++) c->line_items[w].push_back({idx, ch});
            if (W.last) break;
            in = W.out;
            l0 += nl;
        }
    }

    // phase-2/3 table builds: one thread per entry of layer i+1
    c->build_off.assign(d + 1, 0);
    for (u32 i = 0; i < d; i++)
        c->build_off[i + 1] = c->build_off[i] + (needs_tables(c->kind[i]) ? (u32)((S(i + 1) + 255) / 256) : 0);
    c->build_blocks = (int)c->build_off[d];

    // sum-check instances and their waves
    c->scis.clear();
    c->pwaves.clear();
    c->gwaves.clear();
    c->p_items.clear();
    c->g_items.clear();
    c->rounds.clear();
    u64 part_total = 0;
    for (u32 i = 0; i < d; i++) {
        const LayerDev &L = c->L[i];
        for (u32 ph = 1; ph <= 3; ph++) {
            const u32 n = (ph == 1) ? c->s[i] : c->s[i + 1];
            if (n == 0) continue;
            const u32 roff = (ph == 1) ? 0 : (ph == 2) ? c->s[i] : c->s[i] + c->s[i + 1];
            SciDev Sc{};
            Sc.n = n;
            Sc.layer = i;
            Sc.chal_off = c->chal_off[i] + roff;
            Sc.tr_off = c->tr_msg[i] + 3ull * roff;
            if (ph == 1) Sc.kind = PK_PH1;
            else if (L.kind == W_SQUARE) Sc.kind = (ph == 2) ? PK_GEN_SQ2 : PK_SQ3;
            else if (L.kind == W_TREE) Sc.kind = (ph == 2) ? PK_GEN_TREE2 : PK_TREE3;
            else Sc.kind = PK_GEN_TAB;
            const u32 sci = (u32)c->scis.size();
            const bool prod = Sc.kind < PK_GEN_FIRST;
            if (prod) {
                Sc.Lc = A.take<u64>(2 * n);
                Sc.kap = A.take<u64>(n);
                Sc.esum = A.take<u64>(n);
            }
            c->scis.push_back(Sc);
            u32 r0 = 0;
            if (prod) {
                const u64 *in = (ph == 1) ? L.V : L.Vn;
                for (u32 w = 0;; w++) {
                    const u32 nr = std::min(PR_CHUNK_LOG, n - r0);
                    ProdWave W{};
                    W.sci = sci;
                    W.r0 = r0;
                    W.nr = nr;
                    W.e = (nr >= (u32)PR_M) ? (u32)PR_M : 0;
                    W.nchunks = u32(1) << (n - r0 - nr);
                    const bool last = (r0 + nr == n);
                    W.flags = last ? WF_LAST : 0;
                    W.no = n - r0 - nr;
                    W.ho = (W.no + 1) / 2;
                    W.chal_off = Sc.chal_off + r0;
                    W.in = in;
                    W.out = last ? nullptr : A.take<u64>(W.nchunks);
                    const u32 kb = W.e ? W.e - 1 : 0;
                    W.wblk = A.take<u64>(((1u << W.e) - 1) + ((1u << (nr - kb)) - 1) + (1u << W.ho) + (1u << (W.no - W.ho)));
                    W.part = part_total;
                    for (u32 k = 0; k < nr; k++) {
                        RoundRef R{};
                        R.tr_pos = Sc.tr_off + 3ull * (r0 + k);
                        R.part_pos = part_total + u64(k) * W.nchunks * 2;
                        R.nchunks = W.nchunks;
                        R.sci = sci;
                        R.j = r0 + k;
                        c->rounds.push_back(R);
                    }
                    part_total += u64(nr) * W.nchunks * 2;
                    if (c->p_items.size() <= w) c->p_items.resize(w + 1);
                    const u32 idx = (u32)c->pwaves.size();
                    c->pwaves.push_back(W);
                    for (u32 ch = 0; ch < W.nchunks; ch++) c->p_items[w].push_back({idx, ch});
                    if (last) break;
                    in = W.out;
                    r0 += nr;
                }
            } else {
                const bool tab = Sc.kind == PK_GEN_TAB;
                const bool tabB = tab && L.has_add;
                const u64 *inP = tab ? (ph == 2 ? L.P2 : L.P3) : nullptr;
                const u64 *inB = tabB ? (ph == 2 ? L.B2 : L.B3) : nullptr;
                const u64 *inV = L.Vn;
                const bool anyB = tabB || Sc.kind == PK_GEN_TREE2;
                for (u32 w = 0;; w++) {
                    const u32 nr = std::min(GN_CHUNK_LOG, n - r0);
                    GenWave W{};
                    W.sci = sci;
                    W.r0 = r0;
                    W.nr = nr;
                    W.e = (nr >= (u32)GN_M) ? (u32)GN_M : 0;
                    W.nchunks = u32(1) << (n - r0 - nr);
                    const bool last = (r0 + nr == n);
                    W.src = (w > 0 || tab) ? GS_NONE : (Sc.kind == PK_GEN_SQ2 ? GS_SQ2 : GS_TREE2);
                    W.flags = (last ? WF_LAST : 0) | (((w > 0 && anyB) || tabB) ? WF_HASB : 0);
                    W.layer = i;
                    W.chal_off = Sc.chal_off + r0;
                    W.inP = inP;
                    W.inV = inV;
                    W.inB = inB;
                    if (!last) {
                        W.outP = A.take<u64>(W.nchunks);
                        W.outV = A.take<u64>(W.nchunks);
                        W.outB = anyB ? A.take<u64>(W.nchunks) : nullptr;
                    }
                    W.part = part_total;
                    for (u32 k = 0; k < nr; k++) {
                        RoundRef R{};
                        R.tr_pos = Sc.tr_off + 3ull * (r0 + k);
                        R.part_pos = part_total + u64(k) * W.nchunks * 3;
                        R.nchunks = W.nchunks;
                        R.sci = sci;
                        R.j = r0 + k;
                        c->rounds.push_back(R);
                    }
                    part_total += u64(nr) * W.nchunks * 3;
                    if (c->g_items.size() <= w) c->g_items.resize(w + 1);
                    const u32 idx = (u32)c->gwaves.size();
                    c->gwaves.push_back(W);
                    for (u32 ch = 0; ch < W.nchunks; ch++) c->g_items[w].push_back({idx, ch});
                    if (last) break;
                    inP = W.outP;
                    inV = W.outV;
                    inB = W.outB;
                    r0 += nr;
                }
            }
        }
    }
    c->n_partials = part_total;
    c->partials = A.take<u64>(part_total + 1);

    // verifier scratch
    const u64 Sd = S(d);
    u64 mb = (Sd + 255) / 256;
    if (mb > 152 * 4) mb = 152 * 4;
    if (mb == 0) mb = 1;
    c->Vd.mle_blocks = (u32)mb;
    c->Vd.mle_part = A.take<u64>(mb);
    c->Vd.wire = A.take<u64>(2 * d + 2);
    c->Vd.claims = A.take<u64>(d + 1);
    c->round_layer.clear();
    for (u32 i = 0; i < d; i++)
        for (u32 j = 0; j < c->s[i] + 2 * c->s[i + 1]; j++) c->round_layer.push_back((i << 8) | j);
    c->d_round_layer = A.take<u32>(c->round_layer.size() + 1);
    c->Vd.round_layer = c->d_round_layer;
    c->Vd.nrounds = (u32)c->round_layer.size();
    c->Vd.result = c->d_result;
    c->Vd.d = d;
    c->Vd.tr_len = c->tr_len;

    // descriptor arrays
    c->d_layers = A.take<LayerDev>(d);
    c->d_eq_prove = A.take<EqJob>(c->eq_prove.size());
    c->d_eq_verify = A.take<EqJob>(c->eq_verify.size());
    c->d_lw = A.take<LineWaveDev>(c->lw.size());
    c->d_line_items.assign(c->line_items.size(), nullptr);
    for (size_t w = 0; w < c->line_items.size(); w++) c->d_line_items[w] = A.take<Item>(c->line_items[w].size());
    c->d_build_off = A.take<u32>(d + 1);
    c->d_scis = A.take<SciDev>(c->scis.size() + 1);
    c->d_pwaves = A.take<ProdWave>(c->pwaves.size() + 1);
    c->d_gwaves = A.take<GenWave>(c->gwaves.size() + 1);
    c->d_p_items.assign(c->p_items.size(), nullptr);
    for (size_t w = 0; w < c->p_items.size(); w++) c->d_p_items[w] = A.take<Item>(c->p_items[w].size());
    c->d_g_items.assign(c->g_items.size(), nullptr);
    for (size_t w = 0; w < c->g_items.size(); w++) c->d_g_items[w] = A.take<Item>(c->g_items[w].size());
    c->d_rounds = A.take<RoundRef>(c->rounds.size() + 1);
    c->d_explicit_layers = A.take<u32>(c->explicit_layers.size() + 1);
    G.layers = c->d_layers;
    return A.off + 256;
}

template <class T>
static cudaError_t upload(T *dst, const std::vector<T> &src)
{
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

extern "C" vc_status vc_circuit_create(const vc_circuit_desc *desc, int device, vc_circuit **out)
{
    if (!desc || !out || desc->n_layers < 1 || desc->n_layers > 4096 || !desc->log_width || !desc->wiring)
        return VC_EINVAL;
    *out = nullptr;
    vc_circuit *c = new (std::nothrow) vc_circuit();
    if (!c) return VC_ENOMEM;
    c->device = device;
    c->d = desc->n_layers;
    const u32 d = c->d;
    c->s.assign(desc->log_width, desc->log_width + d + 1);
    c->kind.assign(desc->wiring, desc->wiring + d);
    for (u32 i = 0; i <= d; i++)
        if (c->s[i] > 30) { delete c; return VC_EINVAL; }
    c->has_add.assign(d, 0);
    c->ex_type.resize(d);
    c->ex_in1.resize(d);
    c->ex_in2.resize(d);
    c->by1_off.resize(d);
    c->by1_g.resize(d);
    c->by2_off.resize(d);
    c->by2_g.resize(d);
    for (u32 i = 0; i < d; i++) {
        const u32 si = c->s[i], sn = c->s[i + 1];
        if (!shape_ok(c->kind[i], si, sn)) { delete c; return VC_EINVAL; }
        switch (c->kind[i]) {
        case W_TREE: case W_F0_FIRST: c->has_add[i] = 1; break;
        default: break;
        }
        if (c->kind[i] == W_EXPLICIT) {
            if (!desc->gate_type || !desc->in1 || !desc->in2 || !desc->gate_type[i] || !desc->in1[i] || !desc->in2[i]) {
                delete c;
                return VC_EINVAL;
            }
            const u64 Sg = u64(1) << si, Sn = u64(1) << sn;
            c->ex_type[i].assign(desc->gate_type[i], desc->gate_type[i] + Sg);
            c->ex_in1[i].assign(desc->in1[i], desc->in1[i] + Sg);
            c->ex_in2[i].assign(desc->in2[i], desc->in2[i] + Sg);
            for (u64 g = 0; g < Sg; g++) {
                if (c->ex_type[i][g] > 1 || c->ex_in1[i][g] >= Sn || c->ex_in2[i][g] >= Sn) { delete c; return VC_EINVAL; }
                if (c->ex_type[i][g] == 0) c->has_add[i] = 1;
            }
            // gates grouped by in1 and by in2 (counting sort keeps gate order)
            auto group = [&](const std::vector<u32> &in, std::vector<u32> &off, std::vector<u32> &gs) {
                off.assign(Sn + 1, 0);
                for (u64 g = 0; g < Sg; g++) off[in[g] + 1]++;
                for (u64 w = 0; w < Sn; w++) off[w + 1] += off[w];
                gs.assign(Sg, 0);
                std::vector<u32> pos(off.begin(), off.end() - 1);
                for (u64 g = 0; g < Sg; g++) gs[pos[in[g]]++] = (u32)g;
            };
            group(c->ex_in1[i], c->by1_off[i], c->by1_g[i]);
            group(c->ex_in2[i], c->by2_off[i], c->by2_g[i]);
        }
    }
    // challenge, point and transcript offsets
    c->chal_off.assign(d, 0);
    c->z_off.assign(d, 0);
    c->tr_msg.assign(d, 0);
    c->tr_q.assign(d, 0);
    u32 ch = c->s[0], zo = 0;
    u64 tp = u64(1) << c->s[0];
    for (u32 i = 0; i < d; i++) {
        const u32 rounds = c->s[i] + 2 * c->s[i + 1];
        c->chal_off[i] = ch;
        ch += rounds + 1;
        c->z_off[i] = zo;
        zo += c->s[i];
        c->tr_msg[i] = tp;
        tp += 3ull * rounds;
        c->tr_q[i] = tp;
        tp += c->s[i + 1] + 1;
    }
    c->zd_off = zo;
    c->nchal = ch;
    c->tr_len = tp;
    plan_eval(c);

    DevGuard guard(device);
    const size_t bytes = layout(c, 0);
    cudaError_t e = cudaMalloc(&c->arena, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); delete c; return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA; }
    c->arena_bytes = bytes;
    layout(c, reinterpret_cast<uintptr_t>(c->arena));
    e = cudaMemset(c->arena, 0, bytes);
    if (e == cudaSuccess) e = upload(c->d_layers, c->L);
    if (e == cudaSuccess) e = upload(c->d_eq_prove, c->eq_prove);
    if (e == cudaSuccess) e = upload(c->d_eq_verify, c->eq_verify);
    if (e == cudaSuccess) e = upload(c->d_lw, c->lw);
    for (size_t w = 0; e == cudaSuccess && w < c->line_items.size(); w++)
        e = upload(c->d_line_items[w], c->line_items[w]);
    if (e == cudaSuccess) e = upload(c->d_build_off, c->build_off);
    if (e == cudaSuccess) e = upload(c->d_scis, c->scis);
    if (e == cudaSuccess) e = upload(c->d_pwaves, c->pwaves);
    if (e == cudaSuccess) e = upload(c->d_gwaves, c->gwaves);
    for (size_t w = 0; e == cudaSuccess && w < c->p_items.size(); w++) e = upload(c->d_p_items[w], c->p_items[w]);
    for (size_t w = 0; e == cudaSuccess && w < c->g_items.size(); w++) e = upload(c->d_g_items[w], c->g_items[w]);
    if (e == cudaSuccess) e = upload(c->d_rounds, c->rounds);
    if (e == cudaSuccess) e = upload(c->d_explicit_layers, c->explicit_layers);
    if (e == cudaSuccess) e = upload(c->d_round_layer, c->round_layer);
    if (e == cudaSuccess) {
        launch_init_invfact(c->G.invfact, 0);
        e = cudaDeviceSynchronize();
    }
    for (u32 i = 0; e == cudaSuccess && i < d; i++) {
        if (c->kind[i] != W_EXPLICIT) continue;
        const LayerDev &L = c->L[i];
        e = cudaMemcpy((void *)L.type, c->ex_type[i].data(), c->ex_type[i].size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.in1), c->ex_in1[i]);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.in2), c->ex_in2[i]);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.by1_off), c->by1_off[i]);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.by1_g), c->by1_g[i]);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.by2_off), c->by2_off[i]);
        if (e == cudaSuccess) e = upload(const_cast<u32 *>(L.by2_g), c->by2_g[i]);
    }
    if (e == cudaSuccess) e = cudaHostAlloc(&c->h_pinned, 64 * sizeof(u64), cudaHostAllocDefault);
    for (int k = 0; e == cudaSuccess && k < 2; k++) e = cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&c->ev_fork, &c->ev_tables, &c->ev_eval, &c->ev_build, &c->ev_prod, &c->ev_gen})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (const SciDev &Sc : c->scis) c->has_tab = c->has_tab || Sc.kind == PK_GEN_TAB;
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->arena) cudaFree(c->arena);
        delete c;
        return cuda_status(e);
    }
    *out = c;
    return VC_OK;
}

extern "C" vc_status vc_circuit_destroy(vc_circuit *c)
{
    if (!c) return VC_OK;
    DevGuard guard(c->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t ev : {c->ev_fork, c->ev_tables, c->ev_eval, c->ev_build, c->ev_prod, c->ev_gen})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t s : c->aux)
        if (s) cudaStreamDestroy(s);
    if (c->arena) cudaFree(c->arena);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
    return VC_OK;
}

extern "C" vc_status vc_transcript_len(const vc_circuit *c, uint64_t *n)
{
    if (!c || !n) return VC_EINVAL;
    *n = c->tr_len;
    return VC_OK;
}

extern "C" vc_status vc_circuit_bytes(const vc_circuit *c, uint64_t *bytes)
{
    if (!c || !bytes) return VC_EINVAL;
    *bytes = c->arena_bytes;
    return VC_OK;
}

// Pointer kind: 1 = device memory of `device`, 0 = host, -1 = device memory of another device.
static int ptr_kind(const void *p, int device)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == device ? 1 : -1;
    return 0;
}

static vc_status read_status_and_clear(vc_circuit *c, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(c->h_pinned, c->G.status, sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->G.status, 0, sizeof(u32), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return VC_ECUDA;
    const u32 s = *reinterpret_cast<u32 *>(c->h_pinned);
    if (s & ST_BAD_INPUT) return VC_EINVAL;
    if (s & ST_TIMEOUT) return VC_ETIMEOUT;
    return VC_OK;
}

// Enqueue evaluation + proof for inputs already in V_d; transcript -> G.tr.
static cudaError_t enqueue_prove(vc_circuit *c, u64 seed, u64 *tr, cudaStream_t st)
{
    Globals G = c->G;
    G.seed = seed;
    G.tr = tr;
    cudaStream_t sa = c->aux[0], sb = c->aux[1];
    auto mark = [&](int k, int end, cudaStream_t s) {
        if (c->stage_on) cudaEventRecord(c->stage_ev[2 * k + end], s);
    };
    mark(VC_STAGE_PROOF, 0, st);
    mark(VC_STAGE_SETUP, 0, st);
    launch_setup(G, c->zd_off, st);
    mark(VC_STAGE_SETUP, 1, st);
    cudaEventRecord(c->ev_fork, st);
    // helper A: eq tables and product weights (need the coins only)
    cudaStreamWaitEvent(sa, c->ev_fork, 0);
    mark(VC_STAGE_TABLES, 0, sa);
    launch_eqtabs(c->d_eq_prove, (int)c->eq_prove.size(), sa);
    launch_prep_prod(G, c->d_scis, c->d_pwaves, (int)c->pwaves.size(), sa);
    mark(VC_STAGE_TABLES, 1, sa);
    cudaEventRecord(c->ev_tables, sa);
    // caller's stream: evaluation
    mark(VC_STAGE_EVAL, 0, st);
    enqueue_eval(c, G, st);
    mark(VC_STAGE_EVAL, 1, st);
    cudaEventRecord(c->ev_eval, st);
    // helper A: product-weighted waves
    cudaStreamWaitEvent(sa, c->ev_eval, 0);
    for (size_t w = 0; w < c->p_items.size() || w < 2; w++) {
        if (w < 2) mark(w == 0 ? VC_STAGE_PROD0 : VC_STAGE_PRODN, 0, sa);
        if (w < c->p_items.size())
            launch_sc_prod(G, c->d_pwaves, c->d_p_items[w], (int)c->p_items[w].size(), c->partials, sa);
        if (w == 0) mark(VC_STAGE_PROD0, 1, sa);
    }
    mark(VC_STAGE_PRODN, 1, sa);
    cudaEventRecord(c->ev_prod, sa);
    // caller's stream: line reductions, then the wiring tables (they need v1 = q(0))
    mark(VC_STAGE_LINE, 0, st);
    for (size_t w = 0; w < c->line_items.size(); w++)
        launch_line_wave(G, c->d_lw, c->d_line_items[w], (int)c->line_items[w].size(), st);
    launch_build23(G, c->d_build_off, (int)c->d, c->build_blocks, st);
    mark(VC_STAGE_LINE, 1, st);
    cudaEventRecord(c->ev_build, st);
    // helper B: general waves (after the tables they read)
    cudaStreamWaitEvent(sb, c->ev_eval, 0);
    cudaStreamWaitEvent(sb, c->ev_tables, 0);
    if (c->has_tab) cudaStreamWaitEvent(sb, c->ev_build, 0);
    for (size_t w = 0; w < c->g_items.size() || w < 2; w++) {
        if (w < 2) mark(w == 0 ? VC_STAGE_GEN0 : VC_STAGE_GENN, 0, sb);
        if (w < c->g_items.size())
            launch_sc_gen(G, c->d_gwaves, c->d_g_items[w], (int)c->g_items[w].size(), c->partials, sb);
        if (w == 0) mark(VC_STAGE_GEN0, 1, sb);
    }
    mark(VC_STAGE_GENN, 1, sb);
    cudaEventRecord(c->ev_gen, sb);
    // join
    cudaStreamWaitEvent(st, c->ev_prod, 0);
    cudaStreamWaitEvent(st, c->ev_gen, 0);
    mark(VC_STAGE_FINAL, 0, st);
    launch_final(G, c->d_scis, c->d_rounds, (int)c->rounds.size(), c->partials, c->V[0], u64(1) << c->s[0], st);
    mark(VC_STAGE_FINAL, 1, st);
    mark(VC_STAGE_PROOF, 1, st);
    return cudaGetLastError();
}

extern "C" vc_status vc_prove(vc_circuit *c, const uint64_t *inputs, uint64_t seed, uint64_t *transcript,
                              void *stream)
{
    if (!c || !inputs || !transcript) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ki = ptr_kind(inputs, c->device), kt = ptr_kind(transcript, c->device);
    if (ki < 0 || kt < 0) return VC_EINVAL;
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64),
                                    ki ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return VC_ECUDA;
    e = enqueue_prove(c, seed, kt ? transcript : c->d_tr, st);
    if (e != cudaSuccess) return VC_ECUDA;
    if (!kt) {
        e = cudaMemcpyAsync(transcript, c->d_tr, c->tr_len * sizeof(u64), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    if (ki && kt) return VC_OK;
    return read_status_and_clear(c, st);
}

extern "C" vc_status vc_circuit_sync(vc_circuit *c, void *stream)
{
    if (!c) return VC_EINVAL;
    DevGuard guard(c->device);
    return read_status_and_clear(c, (cudaStream_t)stream);
}

extern "C" vc_status vc_evaluate(vc_circuit *c, const uint64_t *inputs, uint64_t *outputs, void *stream)
{
    if (!c || !inputs || !outputs) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ki = ptr_kind(inputs, c->device), ko = ptr_kind(outputs, c->device);
    if (ki < 0 || ko < 0) return VC_EINVAL;
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64),
                                    ki ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return VC_ECUDA;
    launch_check_canonical(c->V[c->d], nin, c->G.status, st);
    enqueue_eval(c, c->G, st);
    e = cudaMemcpyAsync(outputs, c->V[0], (u64(1) << c->s[0]) * sizeof(u64),
                        ko ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    return read_status_and_clear(c, st);
}

extern "C" vc_status vc_verify(vc_circuit *c, const uint64_t *inputs, uint64_t seed, const uint64_t *transcript,
                               int *accept, void *stream)
{
    if (!c || !inputs || !transcript || !accept) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ki = ptr_kind(inputs, c->device), kt = ptr_kind(transcript, c->device);
    const int ka = ptr_kind(accept, c->device);
    if (ki < 0 || kt < 0 || ka < 0) return VC_EINVAL;
    if (!ka) *accept = 0;
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaSuccess;
    const u64 *din = inputs;
    if (!ki) {
        e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64), cudaMemcpyHostToDevice, st);
        din = c->V[c->d];
    }
    const u64 *dtr = transcript;
    if (e == cudaSuccess && !kt) {
        e = cudaMemcpyAsync(c->d_tr, transcript, c->tr_len * sizeof(u64), cudaMemcpyHostToDevice, st);
        dtr = c->d_tr;
    }
    if (e != cudaSuccess) return VC_ECUDA;
    Globals G = c->G;
    G.seed = seed;
    G.tr = nullptr;
    launch_setup(G, c->zd_off, st);
    launch_eqtabs(c->d_eq_verify, (int)c->eq_verify.size(), st);
    VerifyDev Vd = c->Vd;
    Vd.tr = dtr;
    Vd.inputs = din;
    Vd.accept_out = ka ? accept : nullptr;
    launch_verify(G, Vd, c->tzd, c->L[0].tz, c->d_explicit_layers, (int)c->explicit_layers.size(), st);
    if (ka && ki && kt) return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
    e = cudaMemcpyAsync(c->h_pinned + 8, c->d_result, 4 * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    vc_status s = read_status_and_clear(c, st);
    if (s != VC_OK) return s;
    if (!ka) *accept = c->h_pinned[8 + 2] ? 1 : 0;
    return VC_OK;
}

extern "C" vc_status vc_circuit_set_stage_events(vc_circuit *c, void *const *events)
{
    if (!c) return VC_EINVAL;
    if (!events) {
        c->stage_on = false;
        return VC_OK;
    }
    for (int k = 0; k < 2 * VC_NUM_STAGES; k++) {
        if (!events[k]) return VC_EINVAL;
        c->stage_ev[k] = (cudaEvent_t)events[k];
    }
    c->stage_on = true;
    return VC_OK;
}

extern "C" vc_status vc_circuit_get_info(const vc_circuit *c, vc_circuit_info *info)
{
    if (!c || !info) return VC_EINVAL;
    vc_circuit_info I{};
    I.n_layers = c->d;
    u64 rounds = 0, gates = 0;
    for (u32 i = 0; i < c->d; i++) {
        rounds += c->s[i] + 2ull * c->s[i + 1];
        gates += u64(1) << c->s[i];
    }
    I.n_rounds = (uint32_t)rounds;
    I.transcript_len = c->tr_len;
    I.gates = gates;
    I.device_bytes = c->arena_bytes;
    // setup, eq tables, d evaluation layers, line waves, build, sum-check waves, final
    I.prove_launches = (uint32_t)(3 + c->eval_steps.size() + c->line_items.size() + (c->build_blocks > 0 ? 1 : 0) +
                                  (c->pwaves.empty() ? 0 : 1) + c->p_items.size() + c->g_items.size() +
                                  (c->eq_prove.empty() ? -1 : 0));
    I.verify_launches = (uint32_t)(3 + (c->explicit_layers.empty() ? 0 : 1) + 1);
    I.sc0_ctas = (uint32_t)((c->p_items.empty() ? 0 : c->p_items[0].size()) +
                            (c->g_items.empty() ? 0 : c->g_items[0].size()));
    *info = I;
    return VC_OK;
}

extern "C" vc_status vc_prove_batch(vc_circuit *const *circuits, const uint64_t *const *inputs,
                                    const uint64_t *seeds, uint64_t *const *transcripts, int n, void *stream)
{
    if (n < 0 || (n > 0 && (!circuits || !inputs || !seeds || !transcripts))) return VC_EINVAL;
    bool all_dev = true;
    for (int j = 0; j < n; j++) {
        vc_circuit *c = circuits[j];
        if (!c || !inputs[j] || !transcripts[j]) return VC_EINVAL;
        for (int k = 0; k < j; k++)
            if (circuits[k] == c) return VC_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int j = 0; j < n; j++) {
        vc_circuit *c = circuits[j];
        DevGuard guard(c->device);
        const int ki = ptr_kind(inputs[j], c->device), kt = ptr_kind(transcripts[j], c->device);
        if (ki < 0 || kt < 0) return VC_EINVAL;
        all_dev = all_dev && ki && kt;
        const u64 nin = u64(1) << c->s[c->d];
        cudaError_t e = cudaMemcpyAsync(c->V[c->d], inputs[j], nin * sizeof(u64),
                                        ki ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = enqueue_prove(c, seeds[j], kt ? transcripts[j] : c->d_tr, st);
        if (e == cudaSuccess && !kt)
            e = cudaMemcpyAsync(transcripts[j], c->d_tr, c->tr_len * sizeof(u64), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    if (all_dev) return VC_OK;
    vc_status worst = VC_OK;
    for (int j = 0; j < n; j++) {
        DevGuard guard(circuits[j]->device);
        vc_status s = read_status_and_clear(circuits[j], st);
        if (s != VC_OK) worst = s;
    }
    return worst;
}

extern "C" vc_status vc_field_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n, void *stream)
{
    if (!a || !b || !out) return VC_EINVAL;
    launch_field_mul(a, b, out, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}

extern "C" vc_status vc_field_mul_rate(int device, int variant, uint64_t iters, double *rate)
{
    if (!rate || iters == 0 || variant < 0 || variant > 2) return VC_EINVAL;
    DevGuard guard(device);
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return VC_ECUDA;
    u64 *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return VC_ENOMEM;
    const int threads = 256, blocks = prop.multiProcessorCount * 8;
    const float ms = run_field_mul_rate(variant, iters, blocks, threads, sink);
    cudaError_t e = cudaGetLastError();
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return VC_ECUDA;
    // variants 0, 1: 8 chains x one product per step; variant 2: 4 chains x 3 products per step
    const double per_step = (variant == 2) ? 12.0 : 8.0;
    *rate = double(blocks) * threads * per_step * double(iters) / (ms * 1e-3);
    return VC_OK;
}

extern "C" const char *vc_status_string(vc_status s)
{
    switch (s) {
    case VC_OK: return "ok";
    case VC_EINVAL: return "invalid argument";
    case VC_ENOMEM: return "out of memory";
    case VC_ECUDA: return "CUDA error";
    case VC_ETIMEOUT: return "device wait timed out";
    case VC_EBUSY: return "busy";
    default: return "unknown status";
    }
}
