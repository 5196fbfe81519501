// vc_api.cu -- C ABI (include/vc.h): circuit validation, launch planning,
// device scratch, and the launch sequences of the prover and the verifier.
//
// Planning happens once per circuit: the widths and wiring kinds fix every
// table size, every chunk of every sum-check wave, every transcript offset and
// every challenge index, so vc_circuit_create lays all of it out in one device
// arena and uploads the descriptors.  A "plan" is the list of launches of one
// proof over a set of circuits: one circuit, or the members of a batch, whose
// work items then share every launch.  The first proof of a plan captures its
// launches into a CUDA graph; later proofs replay the graph after writing the
// new seed and transcript pointer into the device-resident globals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

vc_status cuda_status(cudaError_t e)
{
    return e == cudaSuccess ? VC_OK : (e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA);
}

// Kernel attributes, set once per device.
void init_device_once(int device)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) {
        prove_kernels_init();
        waves_init();
        sp_init();
        return;
    }
    if (!done[device]) {
        prove_kernels_init();
        waves_init();
        sp_init();
        done[device] = true;
    }
}



// ---------------------------------------------------------------------------------------
// Plan construction
// ---------------------------------------------------------------------------------------

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

// Whether the first evaluation launch of a single-circuit plan is a run of
// block-local layers over the input layer (it can then read the inputs in place).
static bool first_eval_is_input_run(const Plan &P, u32 d)
{
    if (P.seg_items.empty() || P.seg_items[0].empty() || !P.lev_items[0].empty()) return false;
    for (const Item &it : P.seg_items[0])
        if (P.segs[it.wave].i_hi + 1 != d) return false;
    return true;
}

// Evaluation plan: runs of block-local layers (every kind but MATMULT and
// EXPLICIT) go to one k_eval_seg launch each; a CTA takes 2^c entries of the
// run's input layer (about 256 CTAs for wide layers) and keeps going while its
// block stays >= 32 entries (or while one CTA covers the whole layer) and
// <= 4096 entries.  Layers outside any run are evaluated alone (k_eval_layer).
// Slots of the wide layers (more than a quarter of the widest) when the
// values pass through device slots: W slots of the widest layer's size, as
// many as the wide layers' values fill (so the slots never take more device
// memory than the layers would), at least 2 (an iteration's two layers) and
// at most STAGED_SLOTS; the k-th wide layer in slot k mod W.
static void slot_plan(vc_circuit *c)
{
    const u32 d = c->d;
    u64 smax = 1, wide_sum = 0;
    u32 nwide = 0;
    for (u32 i = 0; i <= d; i++) smax = std::max(smax, u64(1) << c->s[i]);
    for (u32 i = 0; i <= d; i++)
        if (4 * (u64(1) << c->s[i]) > smax) {
            nwide++;
            wide_sum += u64(1) << c->s[i];
        }
    const u32 W = std::min<u32>(nwide, (u32)std::min<u64>(STAGED_SLOTS, std::max<u64>(2, wide_sum / smax)));
    c->st_nslots = W;
    c->st_slot.assign(d + 1, -1);
    int ord = 0;
    for (u32 i = 0; i <= d; i++)
        if (4 * (u64(1) << c->s[i]) > smax) c->st_slot[i] = ord++ % (int)W;
}

// Windowed values: evaluate from the input up; iteration i is ready once
// layer i is evaluated (layer i + 1 already is).  Before a wide layer
// overwrites its slot, every ready iteration not yet run joins one group
// (run there) if any of them reads the slot's layer.  The iterations between
// narrow layers join the last group.  Sets st_group, st_groups and wn_steps.
static void windowed_groups(vc_circuit *c)
{
    const u32 d = c->d;
    const auto wide = [&](u32 i) { return c->st_slot[i] >= 0; };
    c->st_group.assign(d, -1);
    c->st_groups.clear();
    c->wn_steps.clear();
    std::vector<int> holder(c->st_nslots, -1);
    if (wide(d)) holder[c->st_slot[d]] = (int)d;
    std::vector<u32> ready;
    auto flush = [&]() {
        if (ready.empty()) return;
        const u32 g = (u32)c->st_groups.size();
        c->st_groups.push_back({ready.back(), ready.front()});  // ready runs downward
        for (u32 j : ready) c->st_group[j] = (int)g;
        c->wn_steps.push_back(-(int)g - 1);
        ready.clear();
    };
    for (int i = (int)d - 1; i >= 0; i--) {
        if (wide((u32)i)) {
            const int L = holder[c->st_slot[i]];  // the layer it replaces
            if (L >= 0)
                for (u32 j : ready)
                    if ((int)j == L || (int)j + 1 == L) {
                        flush();
                        break;
                    }
            holder[c->st_slot[i]] = i;
        }
        c->wn_steps.push_back(i);
        if (wide((u32)i) || wide((u32)i + 1)) ready.push_back((u32)i);
    }
    flush();
    if (!c->st_groups.empty())
        for (u32 i = 0; i < d; i++)
            if (c->st_group[i] < 0) c->st_group[i] = (int)c->st_groups.size() - 1;
}

static void plan_eval(vc_circuit *c)
{
    Plan &P = c->P;
    P.segs.clear();
    P.levs.clear();
    P.checks.clear();
    c->eval_steps.clear();
    c->seg_maxblock.clear();
    int i = (int)c->d - 1;
    // values through slots: with staged values every wide layer alone (its
    // slot may have to be freed and it goes to host memory right after);
    // with windowed values runs stop where a group of iterations must run
    // first (flush[j]: before layer j is evaluated); narrow layers in runs
    const bool staged = (c->flags & VC_VALUES_STAGED) != 0;
    std::vector<char> flush(c->d + 1, 0);
    if (c->flags & VC_VALUES_SLOTTED) slot_plan(c);
    if (c->flags & VC_VALUES_WINDOWED) {
        windowed_groups(c);
        for (size_t k = 1; k < c->wn_steps.size(); k++)
            if (c->wn_steps[k] >= 0 && c->wn_steps[k - 1] < 0) flush[c->wn_steps[k]] = 1;
    }
    auto wide = [&](int j) { return (c->flags & VC_VALUES_SLOTTED) && c->st_slot[j] >= 0; };
    auto local = [&](int j) {
        return !(staged && wide(j)) && c->kind[j] != W_MATMULT && c->kind[j] != W_EXPLICIT;
    };
    while (i >= 0) {
        if (!local(i)) {
            c->eval_steps.push_back(-i - 1);
            i--;
            continue;
        }
        // chunks of 2^cl entries of the run's input layer: about 1024 CTAs for
        // wide layers, blocks of at most 2^11 entries
        const int s_in = (int)c->s[i + 1];
        int cl = std::min(s_in, std::max((int)c->cfg.ev_chunk, s_in - 10));
        cl = std::min(cl, 11);
        int i_lo = i + 1;
        u32 maxblock = 1;
        bool pairs = false;  // the run holds F0_PAIR layers
        auto grow = [&](int cl_) {
            int e = cl_, j = i;
            i_lo = i + 1;
            maxblock = 1u << cl_;
            pairs = false;
            while (j >= 0 && local(j) && !(j < i && flush[j])) {
                const int ne = e + (int)c->s[j] - (int)c->s[j + 1];
                if (ne < 0 || ne > 11) break;
                if (c->kind[j] == W_F0_PAIR && ne < 1) break;
                pairs |= c->kind[j] == W_F0_PAIR;
                e = ne;
                i_lo = j;
                maxblock = std::max(maxblock, 1u << ne);
                j--;
            }
        };
        while (true) {
            grow(cl);
            if (i_lo <= i || cl == 0) break;
            cl--;  // the first layer did not fit: smaller chunks
        }
        // pair layers run in registers, one pair per thread at most: chunks
        // of up to 2^8 entries (more CTAs, shorter chains)
        if (pairs && cl > EV_PAIR_CHUNK) {
            cl = EV_PAIR_CHUNK;
            grow(cl);
        }
        if (i_lo > i) {  // no run possible: evaluate this layer alone
            c->eval_steps.push_back(-i - 1);
            i--;
            continue;
        }
        EvalSeg S{};
        S.circ = 0;
        S.i_hi = (u32)i;
        S.i_lo = (u32)i_lo;
        S.c = (u32)cl;
        S.nchunks = 1u << (s_in - cl);
        S.check_input = (u32)(i + 1 == (int)c->d);
        // tail: narrow local layers below the run (outputs <= 2^11, first
        // input <= 2^16) go to the CTA that finishes last
        S.tail_lo = S.i_lo;
        if (S.nchunks > 1 && c->s[i_lo] <= 16)
            for (int j = i_lo - 1; j >= 0 && local(j) && !flush[j] && c->s[j] <= 11; j--) {
                S.tail_lo = (u32)j;
                maxblock = std::max(maxblock, 1u << c->s[j]);
            }
        // where the blocks start to fit one warp (<= 64 entries in and out to
        // the end of the run / tail): from there warp 0 continues alone
        {
            auto fits_from = [&](int hi, int lo, u32 Bin, bool chunked) {
                int from = lo - 1;  // none
                u32 B = Bin;
                std::vector<u32> bin(hi - lo + 2);
                for (int j = hi; j >= lo; j--) {
                    bin[hi - j] = B;
                    const int sj = (int)c->s[j], snj = (int)c->s[j + 1];
                    B = chunked ? (sj >= snj ? (B << (sj - snj)) : (B >> (snj - sj))) : (1u << sj);
                    bin[hi - j + 1] = B;
                }
                for (int j = lo; j <= hi; j++) {  // the longest suffix of layers with blocks <= 64
                    if (bin[hi - j] > 64 || bin[hi - j + 1] > 64) break;
                    from = j;
                }
                return from;
            };
            S.warp_from = (u32)fits_from(i, i_lo, 1u << cl, true);
            S.tail_warp_from = (S.tail_lo < S.i_lo) ? (u32)fits_from(i_lo - 2, (int)S.tail_lo,
                                                                      1u << c->s[i_lo - 1], false)
                                                    : S.tail_lo - 1;
        }
        c->eval_steps.push_back((int)P.segs.size());
        c->seg_maxblock.push_back(maxblock);
        P.segs.push_back(S);
        i = (int)S.tail_lo - 1;
    }
    P.seg_items.assign(c->eval_steps.size(), {});
    P.lev_items.assign(c->eval_steps.size(), {});
    P.seg_maxblock.assign(c->eval_steps.size(), 1u);
    for (size_t k = 0; k < c->eval_steps.size(); k++) {
        const int step = c->eval_steps[k];
        if (step >= 0) P.seg_maxblock[k] = c->seg_maxblock[step];
        if (step >= 0) {
            for (u32 ch = 0; ch < P.segs[step].nchunks; ch++) P.seg_items[k].push_back({(u32)step, ch});
        } else {
            const u32 layer = (u32)(-step - 1);
            const u32 idx = (u32)P.levs.size();
            P.levs.push_back({0u, layer});
            const u64 blocks = ((u64(1) << c->s[layer]) + 255) / 256;
            for (u64 b = 0; b < blocks; b++) P.lev_items[k].push_back({idx, (u32)b});
        }
    }
    // the first step checks the inputs only if it is a segment that reads them all
    if (c->eval_steps.empty() || c->eval_steps[0] < 0) {
        const u64 blocks = ((u64(1) << c->s[c->d]) + 2047) / 2048;
        for (u64 b = 0; b < blocks; b++) P.checks.push_back({0u, (u32)b});
    }
}

// Staged values: the plan's wave tasks, table builds and evaluation blocks
// split by layer iteration (each layer's launches run while only its two
// layers are on the device), with their device arrays and launch counters.
// The copies into the slots that a staged proof makes after the evaluation,
// in order: group g needs layer L, which replaces layer prev (-1: none) in
// its slot.  After the evaluation each slot holds the last wide layer
// evaluated into it; a group's wide layers missing from their slots are
// copied in before it runs.
struct StagedCopy {
    u32 group, layer;
    int prev;
};

static std::vector<StagedCopy> staged_copies(const vc_circuit &c)
{
    const u32 d = c.d;
    auto wide = [&](u32 i) { return c.st_slot[i] >= 0; };
    std::vector<int> holder(c.st_nslots, -1);
    for (int i = (int)d; i >= 0; i--)
        if (wide(i)) holder[c.st_slot[i]] = i;
    std::vector<StagedCopy> out;
    for (u32 g = 0; g < c.st_groups.size(); g++)
        for (u32 L = c.st_groups[g].first; L <= c.st_groups[g].second + 1; L++) {
            if (!wide(L) || holder[c.st_slot[L]] == (int)L) continue;
            out.push_back({g, L, holder[c.st_slot[L]]});
            holder[c.st_slot[L]] = (int)L;
        }
    return out;
}

static void staged_partition(vc_circuit *c, Arena &A)
{
    Plan &P = c->P;
    const u32 d = c->d;
    auto layer_of = [&](const Task &t) {
        return t.type == TK_LINE ? P.lw[t.wave].layer
                                 : (t.type == TK_PROD ? P.scis[P.pw[t.wave].sci].layer : P.gw[t.wave].layer);
    };
    // Iterations touching a wide layer form groups, in order, each as long as
    // its wide layers (consecutive in wide order, so in distinct slots) number
    // at most W; group g is launch list g.  Every iteration between narrow
    // layers goes to the last list (ng), run first.
    const auto wide = [&](u32 i) { return c->st_slot[i] >= 0; };
    if (c->flags & VC_VALUES_WINDOWED) {
        // groups and steps from windowed_groups (plan_eval)
    } else {
        c->st_group.assign(d, -1);
        c->st_groups.clear();
        int lo_ord = -1, hi_ord = -1;  // the current group's wide layers, by ordinal
        std::vector<int> ordinal(d + 1, -1);
        int o = 0;
        for (u32 i = 0; i <= d; i++)
            if (wide(i)) ordinal[i] = o++;
        for (u32 i = 0; i < d; i++) {
            if (!wide(i) && !wide(i + 1)) continue;
            const int a = wide(i) ? ordinal[i] : ordinal[i + 1], b = wide(i + 1) ? ordinal[i + 1] : ordinal[i];
            if (c->st_groups.empty() || std::max(hi_ord, b) - std::min(lo_ord, a) + 1 > (int)c->st_nslots) {
                c->st_groups.push_back({i, i});
                lo_ord = a;
                hi_ord = b;
            } else {
                c->st_groups.back().second = i;
                lo_ord = std::min(lo_ord, a);
                hi_ord = std::max(hi_ord, b);
            }
            c->st_group[i] = (int)c->st_groups.size() - 1;
        }
    }
    const u32 ng = (u32)c->st_groups.size();
    auto list_of = [&](u32 i) { return c->st_group[i] < 0 ? ng : (u32)c->st_group[i]; };
    auto split = [&](const std::vector<std::vector<Task>> &grp, std::vector<std::vector<std::vector<Task>>> &dst) {
        dst.assign(ng + 1, {});
        for (size_t g = 0; g < grp.size(); g++)
            for (const Task &t : grp[g]) {
                auto &v = dst[list_of(layer_of(t))];
                if (v.size() <= g) v.resize(g + 1);
                v[g].push_back(t);
            }
    };
    split(P.groupsA, c->stA);
    split(P.groupsB, c->stB);
    c->stBuild.assign(ng + 1, {});
    for (const BuildItem &b : P.builds) c->stBuild[list_of(b.layer)].push_back(b);
    c->stEval.assign(d, {});
    for (u32 i = 0; i < d; i++) {
        const u64 blocks = ((u64(1) << c->s[i]) + 255) / 256;
        for (u64 b = 0; b < blocks; b++) c->stEval[i].push_back({i, (u32)b});
    }
    c->st_evalstep.assign(d, -1);
    for (size_t k = 0; k < c->eval_steps.size(); k++) {
        const int step = c->eval_steps[k];
        if (step < 0) continue;
        const EvalSeg &S = P.segs[step];
        for (u32 j = S.tail_lo; j <= S.i_hi; j++) c->st_evalstep[j] = -2;
        c->st_evalstep[S.i_hi] = (int)k;
    }
    c->d_stLev = A.take<LayerEval>(d);
    auto take_lists = [&](auto &lists, auto &dv) {
        dv.assign(lists.size(), {});
        for (size_t i = 0; i < lists.size(); i++)
            for (auto &v : lists[i]) dv[i].push_back(A.take<Task>(v.size() + 1));
    };
    take_lists(c->stA, c->d_stA);
    take_lists(c->stB, c->d_stB);
    c->d_stBuild.assign(ng + 1, nullptr);
    c->d_stEval.assign(d, nullptr);
    for (u32 l = 0; l <= ng; l++) c->d_stBuild[l] = A.take<BuildItem>(c->stBuild[l].size() + 1);
    for (u32 i = 0; i < d; i++) c->d_stEval[i] = A.take<Item>(c->stEval[i].size() + 1);
    c->stctr_off.assign(ng + 1, 0);
    u32 nctr = 0;
    for (u32 i = 0; i <= ng; i++) {
        c->stctr_off[i] = nctr;
        nctr += 2 * (u32)(c->stA[i].size() + c->stB[i].size());
    }
    c->d_stctr = A.take<u32>(nctr + 2);  // list l's launch g: counters stctr_off[l] + 2 g, + 1
    // host-link traffic of one proof (staged): every wide layer written once,
    // plus the copies back in
    c->st_link_bytes = 0;
    if (c->flags & VC_VALUES_WINDOWED) return;
    for (u32 i = 0; i <= d; i++)
        if (wide(i)) c->st_link_bytes += (u64(1) << c->s[i]) * sizeof(u64);
    for (const StagedCopy &k : staged_copies(*c)) c->st_link_bytes += (u64(1) << c->s[k.layer]) * sizeof(u64);
}

static cudaError_t staged_upload(vc_circuit *c)
{
    std::vector<LayerEval> lev(c->d);
    for (u32 i = 0; i < c->d; i++) lev[i] = {0u, i};
    cudaError_t e = upload(c->d_stLev, lev);
    for (size_t i = 0; e == cudaSuccess && i < c->stA.size(); i++)
        for (size_t g = 0; e == cudaSuccess && g < c->stA[i].size(); g++) e = upload(c->d_stA[i][g], c->stA[i][g]);
    for (size_t i = 0; e == cudaSuccess && i < c->stB.size(); i++)
        for (size_t g = 0; e == cudaSuccess && g < c->stB[i].size(); g++) e = upload(c->d_stB[i][g], c->stB[i][g]);
    for (size_t l = 0; e == cudaSuccess && l < c->stBuild.size(); l++) e = upload(c->d_stBuild[l], c->stBuild[l]);
    for (u32 i = 0; e == cudaSuccess && i < c->d; i++) e = upload(c->d_stEval[i], c->stEval[i]);
    u32 nctr = 0;
    for (size_t l = 0; l < c->stA.size(); l++) nctr += 2 * (u32)(c->stA[l].size() + c->stB[l].size());
    if (e == cudaSuccess) e = cudaMemset(c->d_stctr, 0, sizeof(u32) * (nctr + 2));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->st_copy, cudaStreamNonBlocking);
    c->st_ev.assign(4 * (c->d + 1), nullptr);
    for (cudaEvent_t &ev : c->st_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    return e;
}

// Lay out every buffer and descriptor relative to `base` (0 for sizing) and
// fill the circuit's single-circuit plan (circ = 0).
static size_t layout(vc_circuit *c, uintptr_t base, uintptr_t hbase)
{
    Arena A;
    A.base = base;
    const u32 d = c->d;
    auto S = [&](u32 i) { return u64(1) << c->s[i]; };
    Plan &P = c->P;

    // layer values: device memory, or host memory mapped into the device's
    // address space (read and written by the kernels over the host link)
    Arena H;
    H.base = hbase;
    const bool host = (c->flags & VC_VALUES_IN_HOST_MEMORY) != 0;
    const bool staged = (c->flags & VC_VALUES_SLOTTED) != 0;
    const bool windowed = (c->flags & VC_VALUES_WINDOWED) != 0;  // no host copies
    c->V.assign(d + 1, nullptr);
    c->hV.assign(staged ? d + 1 : 0, nullptr);
    if (staged) {
        // wide layers (more than a quarter of the widest) in page-locked host
        // memory, passing through W device slots of the widest layer's size
        // (the k-th wide layer in slot k mod W); narrow layers stay on the
        // device.  W: as many slots as the wide layers' values fill, so the
        // slots never take more device memory than the layers would, at
        // least 2 (an iteration's two layers) and at most STAGED_SLOTS
        // (slot_plan, called by plan_eval, chose W and each wide layer's slot)
        u64 smax = 1;
        for (u32 i = 0; i <= d; i++) smax = std::max(smax, S(i));
        const u32 W = c->st_nslots;
        std::vector<u64 *> slot(W);
        for (u32 k = 0; k < W; k++) slot[k] = A.take<u64>(smax);
        for (u32 i = 0; i <= d; i++) {
            if (c->st_slot[i] >= 0) {
                c->V[i] = slot[c->st_slot[i]];
                if (!windowed) c->hV[i] = H.take<u64>(S(i));
            } else {
                c->V[i] = A.take<u64>(S(i));
            }
        }
        c->d_out = A.take<u64>(S(0));
    } else {
        for (u32 i = 0; i <= d; i++) c->V[i] = host ? H.take<u64>(S(i)) : A.take<u64>(S(i));
    }
    c->host_bytes = (host || (staged && !windowed)) ? H.off + 256 : 0;
    Globals &G = c->G;
    G = Globals{};
    G.d = d;
    G.nchal = c->nchal;
    G.chal = A.take<u64>(c->nchal + 1);
    u32 npts = 0;
    for (u32 i = 0; i <= d; i++) npts += c->s[i];
    G.pts = A.take<u64>(npts + 1);
    G.scal = A.take<u64>(2 * d + 2);
    G.status = A.take<u32>(16);
    G.invfact = A.take<u64>(64);
    G.zd_off = c->zd_off;
    G.S0 = S(0);
    G.out_src = staged ? c->d_out : c->V[0];
    c->d_G = A.take<Globals>(1);
    P.d_G = c->d_G;
    c->d_result = A.take<u64>(VC_RESULT_WORDS);
    c->d_tr = A.take<u64>(c->tr_len);
    c->d_vin = (c->flags & VC_INPUTS_UPLOAD) ? A.take<u64>(S(d)) : nullptr;
    G.tr = c->d_tr;

    for (EvalSeg &Sg : P.segs) Sg.counter = A.take<u32>(1);

    // layers and their eq tables
    c->L.assign(d, LayerDev{});
    P.eqjobs.clear();
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
        P.eqjobs.push_back({L.tz, 0u, EQ_SRC_Z, 0u, i});
        P.eqjobs.push_back({L.trp, 0u, EQ_SRC_CHAL, L.chal_off, 0u});
        P.eqjobs.push_back({L.tr1, 0u, EQ_SRC_CHAL, L.chal_off + L.s, 0u});
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
            c->eq_verify.push_back({L.trp, 0u, EQ_SRC_CHAL, L.chal_off, 0u});
            c->eq_verify.push_back({L.tr1, 0u, EQ_SRC_CHAL, L.chal_off + L.s, 0u});
            c->eq_verify.push_back({L.tr2, 0u, EQ_SRC_CHAL, L.chal_off + L.s + L.sn, 0u});
        }
    }

    // Waves.  A wave is one launch's share of an instance: chunks of 2^nr
    // entries (2^nl coordinates for the line reduction).  A wave followed by a
    // single-chunk wave gets WF_TAIL / tail: its last CTA runs the successor,
    // whose descriptor follows directly.  Every other wave is a task list of
    // a persistent launch: group A[g] (g = waves before it in its instance)
    // or, for general waves over tables built by k_build23, group B[g].
    P.lw.clear();
    P.groupsA.clear();
    P.groupsB.clear();
    auto add_tasks = [&](bool groupB, u32 g, u32 type, u32 idx, u32 nchunks) {
        auto &grp = groupB ? P.groupsB : P.groupsA;
        if (grp.size() <= g) grp.resize(g + 1);
        for (u32 ch = 0; ch < nchunks; ch++) grp[g].push_back({type, idx, ch, 0u});
    };
    for (u32 i = 0; i < d; i++) {
        const u32 n = c->s[i + 1];
        u32 l0 = 0, g = 0;
        const u64 *in = c->V[i + 1];
        bool tail = false;
        for (u32 w = 0;; w++) {
            const u32 cap = (w == 0) ? c->cfg.ln_chunk0 : LN_CHUNKW_LOG;
            const u32 nl = std::min(cap, n - l0);
            LineWaveDev W{};
            W.circ = 0;
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
            const u32 idx = (u32)P.lw.size();
            if (!W.last && (n - l0 - nl) <= LN_CHUNKW_LOG) {  // the next wave is one chunk
                W.tail = 1;
                W.counter = A.take<u32>(1);
            }
            P.lw.push_back(W);
            if (!tail) add_tasks(false, g++, TK_LINE, idx, W.nchunks);
            tail = W.tail != 0;
            if (W.last) break;
            in = W.out;
            l0 += nl;
        }
    }

    // phase-2/3 table builds: one thread per entry of layer i+1, and a CTA
    // per entry of an explicit layer that more than BUILD_HEAVY gates read
    P.builds.clear();
    P.heavy.clear();
    for (u32 i = 0; i < d; i++) {
        if (!needs_tables(c->kind[i])) continue;
        // F0 pair and final layers: a thread per pair of entries of layer i+1
        const bool pairs = c->kind[i] == W_F0_PAIR || c->kind[i] == W_F0_FINAL;
        const u64 blocks = ((pairs ? S(i + 1) / 2 : S(i + 1)) + 255) / 256;
        for (u64 b = 0; b < blocks; b++) P.builds.push_back({0u, i, (u32)b, 0u});
        if (c->kind[i] != W_EXPLICIT) continue;
        for (u64 w = 0; w < S(i + 1); w++)
            for (u32 kind = 1; kind <= 2; kind++) {
                const auto &off = (kind == 1) ? c->by1_off[i] : c->by2_off[i];
                const u32 n = off[w + 1] - off[w];
                if (n <= BUILD_HEAVY) continue;
                const u32 np = (n + BUILD_PIECE - 1) / BUILD_PIECE;
                u64 *part = A.take<u64>(2 * (u64)np);
                u32 *ctr = A.take<u32>(1);
                for (u32 q = 0; q < np; q++) P.heavy.push_back({0u, i, (u32)w, kind, q, np, 0u, 0u, part, ctr});
            }
    }

    // sum-check instances and their waves; all partial sums go to one buffer
    P.scis.clear();
    P.pw.clear();
    P.gw.clear();
    P.rounds.clear();
    std::vector<u64> pw_off, gw_off, round_off;
    u64 part_total = 0;
    u32 smax = 0;
    for (u32 i = 0; i <= d; i++) smax = std::max(smax, c->s[i]);
    for (u32 i = 0; i < d; i++) {
        const LayerDev &L = c->L[i];
        for (u32 ph = 1; ph <= 3; ph++) {
            const u32 n = (ph == 1) ? c->s[i] : c->s[i + 1];
            if (n == 0) continue;
            const u32 roff = (ph == 1) ? 0 : (ph == 2) ? c->s[i] : c->s[i] + c->s[i + 1];
            SciDev Sc{};
            Sc.circ = 0;
            Sc.n = n;
            Sc.layer = i;
            Sc.chal_off = c->chal_off[i] + roff;
            Sc.tr_off = c->tr_msg[i] + 3ull * roff;
            if (ph == 1) Sc.kind = PK_PH1;
            else if (L.kind == W_SQUARE) Sc.kind = (ph == 2) ? PK_GEN_SQ2 : PK_SQ3;
            else if (L.kind == W_TREE) Sc.kind = (ph == 2) ? PK_GEN_TREE2 : PK_TREE3;
            else Sc.kind = PK_GEN_TAB;
            const u32 sci = (u32)P.scis.size();
            const bool prod = Sc.kind < PK_GEN_FIRST;
            if (prod) {
                Sc.Lc = A.take<u64>(2 * n);
                Sc.kap = A.take<u64>(n);
                Sc.esum = A.take<u64>(n);
            }
            P.scis.push_back(Sc);
            const u32 nv = prod ? 2 : 3;
            // smaller PROD instances (dispatched after the larger ones) use
            // half-size chunks, which evens out the end of the launch
            const u32 split = (c->cfg.pr_split == VC_SPLIT_WIDEST) ? smax : c->cfg.pr_split;
            const u32 C = prod ? ((n < split && c->cfg.pr_chunk > 1) ? c->cfg.pr_chunk - 1 : c->cfg.pr_chunk)
                               : c->cfg.gn_chunk;
            const u32 M = prod ? (u32)PR_M : (u32)GN_M;
            const bool tab = Sc.kind == PK_GEN_TAB;
            const bool tabB = tab && L.has_add;
            const bool anyB = tabB || Sc.kind == PK_GEN_TREE2;
            const u64 *inP = tab ? (ph == 2 ? L.P2 : L.P3) : nullptr;
            const u64 *inB = tabB ? (ph == 2 ? L.B2 : L.B3) : nullptr;
            const u64 *inV = (ph == 1) ? L.V : L.Vn;
            // TREE phase 2 with a first wave in registers: its round 0 leaves
            // the factor 1 - r_0 out of P and B (applied per round by k_final)
            const bool defer = Sc.kind == PK_GEN_TREE2 && std::min(C, n) > WV_LOG;
            u32 r0 = 0, g = 0;
            bool tail = false;
            for (u32 w = 0;; w++) {
                const u32 nr = std::min(C, n - r0);
                const u32 nchunks = u32(1) << (n - r0 - nr);
                const bool last = (r0 + nr == n);
                // entries per thread: all WV threads busy, at most 2^M each; the
                // register phase works on runs (16 entries PROD, 4 GEN), so a
                // wave of more than WV threads' entries takes at least one run
                const u32 run = prod ? 4u : 2u;
                const u32 e = nr > WV_LOG ? std::min(M, std::max(run, nr - WV_LOG)) : 0u;
                const bool has_tail = !last && (n - r0 - nr) <= C;  // the next wave is one chunk
                for (u32 k = 0; k < nr; k++) {
                    RoundRef R{};
                    R.tr_pos = Sc.tr_off + 3ull * (r0 + k);
                    R.nchunks = nchunks;
                    R.kind = Sc.kind;
                    R.circ = 0;
                    R.sci = sci;
                    R.j = r0 + k;
                    R.defer = (defer && R.j >= 1) ? 1u : 0u;
                    R.ez = G.scal + SCAL_EQZRP(i);
                    R.v1 = G.scal + SCAL_V1(i);
                    R.ch = G.chal + c->chal_off[i] + c->s[i];
                    if (prod) {
                        R.lc = Sc.Lc + 2 * R.j;
                        R.kap = Sc.kap + R.j;
                        R.esum = Sc.esum + R.j;
                    }
                    round_off.push_back(part_total + u64(k) * nchunks * nv);
                    P.rounds.push_back(R);
                }
                u32 idx;
                if (prod) {
                    ProdWave W{};
                    W.circ = 0;
                    W.sci = sci;
                    W.r0 = r0;
                    W.nr = nr;
                    W.e = e;
                    W.nchunks = nchunks;
                    W.flags = (last ? WF_LAST : 0) | (has_tail ? WF_TAIL : 0);
                    W.no = n - r0 - nr;
                    W.ho = (W.no + 1) / 2;
                    W.chal_off = Sc.chal_off + r0;
                    W.in = inV;
                    W.out = last ? nullptr : A.take<u64>(nchunks);
                    const u32 kb = W.e ? W.e - 1 : 0;
                    W.wblk = A.take<u64>(((1u << W.e) - 1) + ((1u << (nr - kb)) - 1) + (1u << W.ho) +
                                         (1u << (W.no - W.ho)));
                    W.counter = has_tail ? A.take<u32>(1) : nullptr;
                    pw_off.push_back(part_total);
                    idx = (u32)P.pw.size();
                    P.pw.push_back(W);
                    inV = W.out;
                } else {
                    GenWave W{};
                    W.circ = 0;
                    W.sci = sci;
                    W.r0 = r0;
                    W.nr = nr;
                    W.e = e;
                    W.nchunks = nchunks;
                    W.src = (w > 0 || tab) ? GS_NONE : (Sc.kind == PK_GEN_SQ2 ? GS_SQ2 : GS_TREE2);
                    W.flags = (last ? WF_LAST : 0) | (((w > 0 && anyB) || tabB) ? WF_HASB : 0) |
                              (has_tail ? WF_TAIL : 0);
                    W.layer = i;
                    W.chal_off = Sc.chal_off + r0;
                    W.inP = inP;
                    W.inV = inV;
                    W.inB = inB;
                    if (!last) {
                        W.outP = A.take<u64>(nchunks);
                        W.outV = A.take<u64>(nchunks);
                        W.outB = anyB ? A.take<u64>(nchunks) : nullptr;
                    }
                    W.counter = has_tail ? A.take<u32>(1) : nullptr;
                    gw_off.push_back(part_total);
                    idx = (u32)P.gw.size();
                    P.gw.push_back(W);
                    inP = W.outP;
                    inV = W.outV;
                    inB = W.outB;
                }
                if (!tail) add_tasks(tab, g++, prod ? TK_PROD : TK_GEN, idx, nchunks);
                tail = has_tail;
                part_total += u64(nr) * nchunks * nv;
                if (last) break;
                r0 += nr;
            }
        }
    }
    c->partials = A.take<u64>(part_total + 1);
    for (size_t k = 0; k < P.pw.size(); k++) P.pw[k].part = c->partials + pw_off[k];
    for (size_t k = 0; k < P.gw.size(); k++) P.gw[k].part = c->partials + gw_off[k];
    for (size_t k = 0; k < P.rounds.size(); k++) P.rounds[k].part_pos = c->partials + round_off[k];
    P.outs.assign(1, 0u);
    sort_tasks(P);

    // verifier scratch
    // MLE partial sums: one CTA per 2^vmle_log(s) entries
    const u64 mb = u64(1) << (c->s[d] - vmle_log(c->s[d]));
    const u64 mbo = u64(1) << (c->s[0] - vmle_log(c->s[0]));
    c->Vd.mle_blocks = (u32)mb;
    c->Vd.mle_out_blocks = S(0) <= VC_OUT_INLINE ? 0u : (u32)mbo;  // few outputs: formed in the check launch
    c->Vd.mle_part = A.take<u64>(mb + mbo);
    c->Vd.wire = A.take<u64>(2 * d + 2);
    // the verifier's wiring sums: about 4096 gates per CTA, at most 1024 CTAs a layer
    c->vwire.clear();
    u32 nparts = 0;
    for (u32 i : c->explicit_layers) {
        const u32 nb = (u32)std::min<u64>(1024, std::max<u64>(1, S(i) / 4096));
        for (u32 b = 0; b < nb; b++) c->vwire.push_back({i, b, nb, nparts});
        nparts += nb;
    }
    c->Vd.wire_part = A.take<u64>(2 * (u64)nparts + 2);
    c->Vd.wire_ctr = A.take<u32>(d + 1);
    c->d_vwire = A.take<VwireItem>(c->vwire.size() + 1);
    c->round_layer.clear();
    for (u32 i = 0; i < d; i++)
        for (u32 j = 0; j < c->s[i] + 2 * c->s[i + 1]; j++) c->round_layer.push_back((i << 8) | j);
    c->d_round_layer = A.take<u32>(c->round_layer.size() + 1);
    c->Vd.round_layer = c->d_round_layer;
    c->Vd.nrounds = (u32)c->round_layer.size();
    c->zmap.clear();
    for (u32 i = 0; i < d; i++)
        for (u32 k = 0; k < c->s[i + 1]; k++) c->zmap.push_back((i << 8) | k);
    c->d_zmap = A.take<u32>(c->zmap.size() + 1);
    G.zmap = c->d_zmap;
    G.nz = (u32)c->zmap.size();
    c->Vd.result = c->d_result;
    c->Vd.d = d;
    c->Vd.tr_len = c->tr_len;
    c->Vd.vp = c->d_vp = A.take<VerifyPtrs>(1);

    // descriptor arrays
    c->d_layers = A.take<LayerDev>(d);
    G.layers = c->d_layers;
    c->d_eq_verify = A.take<EqJob>(c->eq_verify.size());
    c->d_explicit_layers = A.take<u32>(c->explicit_layers.size() + 1);

    // the verifier's globals (everything else shared, read-only for it)
    Globals &Gv = c->Gv;
    Gv = G;
    Gv.chal = A.take<u64>(c->nchal + 1);
    Gv.pts = A.take<u64>(npts + 1);
    Gv.scal = A.take<u64>(2 * d + 2);
    Gv.status = G.status + 1;
    Gv.tr = nullptr;
    c->d_Gv = A.take<Globals>(1);
    if (staged) staged_partition(c, A);
    return A.off;
}

// Device arrays for a plan's descriptors, carved from an arena (own_G: the
// plan holds its own array of globals, as a batch does).
void plan_take(Plan &P, Arena &A, bool own_G)
{
    if (own_G) P.d_G = A.take<Globals>(P.ncirc);
    P.d_checks = A.take<Item>(P.checks.size() + 1);
    P.d_eqjobs = A.take<EqJob>(P.eqjobs.size() + 1);
    P.d_segs = A.take<EvalSeg>(P.segs.size() + 1);
    P.d_levs = A.take<LayerEval>(P.levs.size() + 1);
    auto items = [&](std::vector<std::vector<Item>> &v, std::vector<Item *> &dv) {
        dv.assign(v.size(), nullptr);
        for (size_t k = 0; k < v.size(); k++) dv[k] = A.take<Item>(v[k].size() + 1);
    };
    items(P.seg_items, P.d_seg_items);
    items(P.lev_items, P.d_lev_items);
    auto tasks = [&](std::vector<std::vector<Task>> &v, std::vector<Task *> &dv) {
        dv.assign(v.size(), nullptr);
        for (size_t k = 0; k < v.size(); k++) dv[k] = A.take<Task>(v[k].size() + 1);
    };
    tasks(P.groupsA, P.d_groupsA);
    tasks(P.groupsB, P.d_groupsB);
    P.d_ctr = A.take<u32>(2 * (P.groupsA.size() + P.groupsB.size()) + 2);
    P.d_lw = A.take<LineWaveDev>(P.lw.size() + 1);
    P.d_builds = A.take<BuildItem>(P.builds.size() + 1);
    P.d_heavy = A.take<HeavyItem>(P.heavy.size() + 1);
    P.d_scis = A.take<SciDev>(P.scis.size() + 1);
    P.d_pw = A.take<ProdWave>(P.pw.size() + 1);
    P.d_gw = A.take<GenWave>(P.gw.size() + 1);
    P.d_rounds = A.take<RoundRef>(P.rounds.size() + 1);
    P.d_outs = A.take<u32>(P.outs.size() + 1);
}

// Host-side consistency check of a plan before any of it reaches the device:
// every item names an existing descriptor and one of its chunks, every
// descriptor an existing circuit and sum-check instance.
bool plan_valid(const Plan &P)
{
    const u32 nc = (u32)P.ncirc;
    for (const Item &it : P.checks)
        if (it.wave >= nc) return false;
    for (const EqJob &J : P.eqjobs)
        if (J.circ >= nc || J.t.n > 30 || (J.src != EQ_SRC_CHAL && J.src != EQ_SRC_Z)) return false;
    for (const EvalSeg &S : P.segs)
        if (S.circ >= nc) return false;
    for (const LayerEval &E : P.levs)
        if (E.circ >= nc) return false;
    for (size_t k = 0; k < P.lw.size(); k++) {
        const LineWaveDev &W = P.lw[k];
        if (W.circ >= nc) return false;
        if (W.tail && (k + 1 >= P.lw.size() || P.lw[k + 1].nchunks != 1 || P.lw[k + 1].layer != W.layer ||
                       P.lw[k + 1].circ != W.circ || P.lw[k + 1].l0 != W.l0 + W.nl || !W.counter))
            return false;
    }
    for (const BuildItem &b : P.builds)
        if (b.circ >= nc) return false;
    for (const HeavyItem &b : P.heavy)
        if (b.circ >= nc || (b.kind != 1 && b.kind != 2) || b.piece >= b.npieces || !b.part || !b.ctr) return false;
    for (const SciDev &S : P.scis)
        if (S.circ >= nc) return false;
    for (size_t k = 0; k < P.pw.size(); k++) {
        const ProdWave &W = P.pw[k];
        if (W.circ >= nc || W.sci >= P.scis.size() || P.scis[W.sci].circ != W.circ) return false;
        if (W.nr > PR_CHUNK_LOG || W.e > (u32)PR_M || W.e > W.nr || W.nr - W.e > WV_LOG || (W.e && W.e < 4))
            return false;
        if ((W.flags & WF_TAIL) && (k + 1 >= P.pw.size() || P.pw[k + 1].nchunks != 1 || P.pw[k + 1].sci != W.sci ||
                                    P.pw[k + 1].r0 != W.r0 + W.nr || !W.counter))
            return false;
    }
    for (size_t k = 0; k < P.gw.size(); k++) {
        const GenWave &W = P.gw[k];
        if (W.circ >= nc || W.sci >= P.scis.size() || P.scis[W.sci].circ != W.circ) return false;
        if (W.nr > GN_CHUNK_LOG || W.e > (u32)GN_M || W.e > W.nr || W.nr - W.e > WV_LOG || (W.e && W.e < 2))
            return false;
        if ((W.flags & WF_TAIL) && (k + 1 >= P.gw.size() || P.gw[k + 1].nchunks != 1 || P.gw[k + 1].sci != W.sci ||
                                    P.gw[k + 1].r0 != W.r0 + W.nr || !W.counter))
            return false;
    }
    for (const LineWaveDev &W : P.lw)
        if (W.nl > (W.l0 ? LN_CHUNKW_LOG : LN_CHUNK0_LOG) || W.n > 30) return false;
    for (const RoundRef &R : P.rounds)
        if (R.sci >= P.scis.size() || R.j >= P.scis[R.sci].n || R.circ >= nc || P.scis[R.sci].circ != R.circ ||
            !R.ez || !R.v1 || !R.ch || (R.kind < PK_GEN_FIRST && (!R.lc || !R.kap || !R.esum)))
            return false;
    for (u32 o : P.outs)
        if (o >= nc) return false;
    for (const auto &v : P.seg_items)
        for (const Item &it : v)
            if (it.wave >= P.segs.size() || it.chunk >= P.segs[it.wave].nchunks) return false;
    for (const auto &v : P.lev_items)
        for (const Item &it : v)
            if (it.wave >= P.levs.size()) return false;
    auto task_ok = [&](const Task &t) {
        switch (t.type) {
        case TK_LINE: return t.wave < P.lw.size() && t.chunk < P.lw[t.wave].nchunks;
        case TK_PROD: return t.wave < P.pw.size() && t.chunk < P.pw[t.wave].nchunks;
        case TK_GEN: return t.wave < P.gw.size() && t.chunk < P.gw[t.wave].nchunks;
        default: return false;
        }
    };
    for (const auto *grp : {&P.groupsA, &P.groupsB})
        for (const auto &v : *grp)
            for (const Task &t : v)
                if (!task_ok(t)) return false;
    return P.seg_items.size() == P.d_seg_items.size() && P.lev_items.size() == P.d_lev_items.size() &&
           P.groupsA.size() == P.d_groupsA.size() && P.groupsB.size() == P.d_groupsB.size();
}

// Task order inside a launch: line chunks first (their tails are the
// longest serial work), then general, then product-weighted; within a kind,
// chunks of larger waves first.
void sort_tasks(Plan &P)
{
    // the final reduction takes every round a warp each while one launch has
    // a warp for each; beyond that the rounds with many partials a warp each,
    // the rest a thread each
    if (P.rounds.size() <= FINAL_ALL_WARPS) {
        P.nbig = (u32)P.rounds.size();
    } else {
        auto many = [](const RoundRef &R) { return R.nchunks > FINAL_WARP_MIN; };
        P.nbig = (u32)(std::stable_partition(P.rounds.begin(), P.rounds.end(), many) - P.rounds.begin());
    }
    auto rank = [&](const Task &t) { return t.type == TK_LINE ? 0 : (t.type == TK_GEN ? 1 : 2); };
    auto entries = [&](const Task &t) {  // the wave's whole size: larger waves first
        return t.type == TK_LINE ? (u64(P.lw[t.wave].nchunks) << P.lw[t.wave].nl)
                                 : (t.type == TK_PROD ? (u64(P.pw[t.wave].nchunks) << P.pw[t.wave].nr)
                                                      : (u64(P.gw[t.wave].nchunks) << P.gw[t.wave].nr));
    };
    for (auto *grp : {&P.groupsA, &P.groupsB})
        for (auto &v : *grp)
            std::stable_sort(v.begin(), v.end(), [&](const Task &a, const Task &b) {
                const int ra = rank(a), rb = rank(b);
                if (ra != rb) return ra < rb;
                return entries(a) > entries(b);
            });
}

cudaError_t plan_upload(Plan &P)
{
    if (!plan_valid(P)) return cudaErrorInvalidValue;
    cudaError_t e = upload(P.d_checks, P.checks);
    if (e == cudaSuccess) e = upload(P.d_eqjobs, P.eqjobs);
    if (e == cudaSuccess) e = upload(P.d_segs, P.segs);
    if (e == cudaSuccess) e = upload(P.d_levs, P.levs);
    auto items = [&](std::vector<std::vector<Item>> &v, std::vector<Item *> &dv) {
        for (size_t k = 0; e == cudaSuccess && k < v.size(); k++) e = upload(dv[k], v[k]);
    };
    items(P.seg_items, P.d_seg_items);
    items(P.lev_items, P.d_lev_items);
    for (size_t k = 0; e == cudaSuccess && k < P.groupsA.size(); k++) e = upload(P.d_groupsA[k], P.groupsA[k]);
    for (size_t k = 0; e == cudaSuccess && k < P.groupsB.size(); k++) e = upload(P.d_groupsB[k], P.groupsB[k]);
    if (e == cudaSuccess) e = cudaMemset(P.d_ctr, 0, sizeof(u32) * (2 * (P.groupsA.size() + P.groupsB.size()) + 2));
    if (e == cudaSuccess) e = upload(P.d_lw, P.lw);
    if (e == cudaSuccess) e = upload(P.d_builds, P.builds);
    if (e == cudaSuccess) e = upload(P.d_heavy, P.heavy);
    if (e == cudaSuccess) e = upload(P.d_scis, P.scis);
    if (e == cudaSuccess) e = upload(P.d_pw, P.pw);
    if (e == cudaSuccess) e = upload(P.d_gw, P.gw);
    if (e == cudaSuccess) e = upload(P.d_rounds, P.rounds);
    if (e == cudaSuccess) e = upload(P.d_outs, P.outs);
    return e;
}

cudaError_t plan_upload_async(Plan &P, cudaStream_t st)
{
    if (!plan_valid(P)) return cudaErrorInvalidValue;
    cudaError_t e = upload_async(P.d_G, P.h_G, st);
    if (e == cudaSuccess) e = upload_async(P.d_checks, P.checks, st);
    if (e == cudaSuccess) e = upload_async(P.d_eqjobs, P.eqjobs, st);
    if (e == cudaSuccess) e = upload_async(P.d_segs, P.segs, st);
    if (e == cudaSuccess) e = upload_async(P.d_levs, P.levs, st);
    auto items = [&](std::vector<std::vector<Item>> &v, std::vector<Item *> &dv) {
        for (size_t k = 0; e == cudaSuccess && k < v.size(); k++) e = upload_async(dv[k], v[k], st);
    };
    items(P.seg_items, P.d_seg_items);
    items(P.lev_items, P.d_lev_items);
    for (size_t k = 0; e == cudaSuccess && k < P.groupsA.size(); k++)
        e = upload_async(P.d_groupsA[k], P.groupsA[k], st);
    for (size_t k = 0; e == cudaSuccess && k < P.groupsB.size(); k++)
        e = upload_async(P.d_groupsB[k], P.groupsB[k], st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(P.d_ctr, 0, sizeof(u32) * (2 * (P.groupsA.size() + P.groupsB.size()) + 2), st);
    if (e == cudaSuccess) e = upload_async(P.d_lw, P.lw, st);
    if (e == cudaSuccess) e = upload_async(P.d_builds, P.builds, st);
    if (e == cudaSuccess) e = upload_async(P.d_heavy, P.heavy, st);
    if (e == cudaSuccess) e = upload_async(P.d_scis, P.scis, st);
    if (e == cudaSuccess) e = upload_async(P.d_pw, P.pw, st);
    if (e == cudaSuccess) e = upload_async(P.d_gw, P.gw, st);
    if (e == cudaSuccess) e = upload_async(P.d_rounds, P.rounds, st);
    if (e == cudaSuccess) e = upload_async(P.d_outs, P.outs, st);
    return e;
}

size_t plan_bytes(Plan &P, bool own_G)
{
    Arena A;
    plan_take(P, A, own_G);
    return A.off + 256;
}

cudaError_t plan_resources(Plan &P)
{
    cudaError_t e = cudaStreamCreateWithFlags(&P.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.evs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.evs_aux, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&P.ev_fork, &P.ev_tables, &P.ev_params, &P.ev_mark})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

void plan_drop_graph(Plan &P)
{
    if (P.exec) cudaGraphExecDestroy(P.exec);
    if (P.graph) cudaGraphDestroy(P.graph);
    P.exec = nullptr;
    P.graph = nullptr;
    P.pnode = nullptr;
}

void plan_release(Plan &P)
{
    plan_drop_graph(P);
    for (cudaEvent_t *ev : {&P.ev_fork, &P.ev_tables, &P.ev_params, &P.ev_mark}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    for (cudaStream_t *s : {&P.aux, &P.cap, &P.evs, &P.evs_aux}) {
        if (*s) cudaStreamDestroy(*s);
        *s = nullptr;
    }
}

// Merge the single-circuit plans of `cs` into one plan: every descriptor keeps
// its circuit's buffers and gets circ = the member's index; the item lists of
// the same evaluation step, line wave or sum-check wave are concatenated.
// Steps of different circuits are independent, and the steps of one circuit
// keep their order, so each merged launch is valid for every member.
void plan_merge(Plan &B, const std::vector<vc_circuit *> &cs)
{
    B = Plan{};
    B.ncirc = (int)cs.size();
    auto grow = [](std::vector<std::vector<Item>> &dst, size_t n) {
        if (dst.size() < n) dst.resize(n);
    };
    auto append = [](std::vector<std::vector<Item>> &dst, const std::vector<std::vector<Item>> &src, u32 off) {
        for (size_t k = 0; k < src.size(); k++)
            for (Item it : src[k]) dst[k].push_back({it.wave + off, it.chunk});
    };
    for (size_t j = 0; j < cs.size(); j++) {
        const Plan &P = cs[j]->P;
        const u32 cj = (u32)j;
        const u32 oseg = (u32)B.segs.size(), olev = (u32)B.levs.size(), olw = (u32)B.lw.size();
        const u32 osci = (u32)B.scis.size(), opw = (u32)B.pw.size(), ogw = (u32)B.gw.size();
        for (Item it : P.checks) B.checks.push_back({cj, it.chunk});
        for (EqJob J : P.eqjobs) {
            J.circ = cj;
            B.eqjobs.push_back(J);
        }
        for (EvalSeg S : P.segs) {
            S.circ = cj;
            B.segs.push_back(S);
        }
        for (LayerEval E : P.levs) {
            E.circ = cj;
            B.levs.push_back(E);
        }
        grow(B.seg_items, P.seg_items.size());
        grow(B.lev_items, P.lev_items.size());
        if (B.seg_maxblock.size() < P.seg_maxblock.size()) B.seg_maxblock.resize(P.seg_maxblock.size(), 1u);
        for (size_t k = 0; k < P.seg_maxblock.size(); k++)
            B.seg_maxblock[k] = std::max(B.seg_maxblock[k], P.seg_maxblock[k]);
        append(B.seg_items, P.seg_items, oseg);
        append(B.lev_items, P.lev_items, olev);
        for (LineWaveDev W : P.lw) {
            W.circ = cj;
            B.lw.push_back(W);
        }
        auto tasks = [&](std::vector<std::vector<Task>> &dst, const std::vector<std::vector<Task>> &src) {
            if (dst.size() < src.size()) dst.resize(src.size());
            for (size_t k = 0; k < src.size(); k++)
                for (Task t : src[k]) {
                    t.wave += (t.type == TK_LINE) ? olw : (t.type == TK_PROD ? opw : ogw);
                    dst[k].push_back(t);
                }
        };
        tasks(B.groupsA, P.groupsA);
        tasks(B.groupsB, P.groupsB);
        for (BuildItem b : P.builds) {
            b.circ = cj;
            B.builds.push_back(b);
        }
        for (HeavyItem b : P.heavy) {
            b.circ = cj;
            B.heavy.push_back(b);
        }
        for (SciDev Sc : P.scis) {
            Sc.circ = cj;
            B.scis.push_back(Sc);
        }
        for (ProdWave W : P.pw) {
            W.circ = cj;
            W.sci += osci;
            B.pw.push_back(W);
        }
        for (GenWave W : P.gw) {
            W.circ = cj;
            W.sci += osci;
            B.gw.push_back(W);
        }
        for (RoundRef R : P.rounds) {
            R.sci += osci;
            R.circ = cj;
            B.rounds.push_back(R);
        }
        B.outs.push_back(cj);
        B.h_G.push_back(cs[j]->G);
    }
    sort_tasks(B);
}

// ---------------------------------------------------------------------------------------
// Proof launch sequence
// ---------------------------------------------------------------------------------------

// The launches of one proof of every circuit of the plan, after the globals
// hold the call's seeds.  `st` checks and evaluates the circuit; the helper
// stream, forked from `st` at the start, runs the coin launch (challenges,
// points, eq tables, product weights: none depends on the circuit's values);
// `st` then waits for it and runs the persistent wave launches (line
// reductions, product-weighted and general sum-checks), the wiring tables and
// the general waves over them where the circuit has such layers, and the
// final reduction.
void enqueue_plan(Plan &P, cudaStream_t st)
{
    cudaStream_t sa = P.aux;
    const Globals *Gs = P.d_G;
    // stage events become event-record nodes of the captured graph, on a
    // branch (P.evs) that depends on the point of `s` where the stage starts
    // or ends but that no launch depends on
    bool marked = false, marked_aux = false;
    auto mark = [&](int k, int end, cudaStream_t s) {
        if (!(P.stage_on && P.stage_ev[2 * k + end])) return;
        const bool aux = s == P.aux;
        cudaStream_t b = aux ? P.evs_aux : P.evs;
        cudaEventRecord(P.ev_mark, s);
        cudaStreamWaitEvent(b, P.ev_mark, 0);
        cudaEventRecordWithFlags(P.stage_ev[2 * k + end], b, cudaEventRecordExternal);
        (aux ? marked_aux : marked) = true;
    };
    auto any_tasks = [](const std::vector<std::vector<Task>> &g, size_t from) {
        for (size_t k = from; k < g.size(); k++)
            if (!g[k].empty()) return true;
        return false;
    };
    const bool has_wavesn = any_tasks(P.groupsA, 1), has_build = !P.builds.empty(),
               has_tabwaves = any_tasks(P.groupsB, 0);
    const size_t nA = P.groupsA.size();
    auto waves = [&](std::vector<Task> &tasks, Task *d_tasks, size_t g) {
        launch_waves(Gs, P.d_lw, P.d_pw, P.d_gw, d_tasks, (int)tasks.size(), P.d_ctr + 2 * g, st);
    };
    mark(VC_STAGE_PROOF, 0, st);
    if (P.own_params) launch_params(P.d_G, 0, nullptr, nullptr, st);  // arguments set per launch
    // helper stream: coins, points, eq tables and product weights (they do not
    // depend on the circuit's values), concurrently with the evaluation; the
    // evaluation, the longer of the two, is put into the graph first
    cudaEventRecord(P.ev_fork, st);
    mark(VC_STAGE_EVAL, 0, st);
    for (size_t k = 0; k < P.seg_items.size(); k++) {
        launch_eval_segs(Gs, P.d_segs, P.d_seg_items[k], (int)P.seg_items[k].size(), P.seg_maxblock[k], st,
                         P.own_params && k == 0);
        launch_eval_layers(Gs, P.d_levs, P.d_lev_items[k], (int)P.lev_items[k].size(), st);
    }
    // inputs not checked by an evaluation segment: the check only latches a
    // status read after the proof, so it need not delay the evaluation
    launch_check_inputs(Gs, P.d_checks, (int)P.checks.size(), st);
    mark(VC_STAGE_EVAL, 1, st);
    cudaStreamWaitEvent(sa, P.ev_fork, 0);
    mark(VC_STAGE_TABLES, 0, sa);
    launch_coins(Gs, P.ncirc, P.d_eqjobs, (int)P.eqjobs.size(), P.d_scis, P.d_pw, (int)P.pw.size(), sa);
    mark(VC_STAGE_TABLES, 1, sa);
    cudaEventRecord(P.ev_tables, sa);
    cudaStreamWaitEvent(st, P.ev_tables, 0);
    // line reductions, product-weighted and on-the-fly general waves
    mark(VC_STAGE_WAVES, 0, st);
    if (nA) waves(P.groupsA[0], P.d_groupsA[0], 0);
    mark(VC_STAGE_WAVES, 1, st);
    if (has_wavesn) {
        mark(VC_STAGE_WAVESN, 0, st);
        for (size_t g = 1; g < nA; g++) waves(P.groupsA[g], P.d_groupsA[g], g);
        mark(VC_STAGE_WAVESN, 1, st);
    }
    // wiring tables (they need q(0) of every line reduction), then their waves
    if (has_build) {
        mark(VC_STAGE_BUILD, 0, st);
        launch_build23(Gs, P.d_builds, (int)P.builds.size(), st);
        launch_build_heavy(Gs, P.d_heavy, (int)P.heavy.size(), st);
        mark(VC_STAGE_BUILD, 1, st);
    }
    if (has_tabwaves) {
        mark(VC_STAGE_TABWAVES, 0, st);
        for (size_t g = 0; g < P.groupsB.size(); g++) waves(P.groupsB[g], P.d_groupsB[g], nA + g);
        mark(VC_STAGE_TABWAVES, 1, st);
    }
    mark(VC_STAGE_FINAL, 0, st);
    launch_final(P.d_G, P.d_rounds, (int)P.rounds.size(), (int)P.nbig, P.d_outs, (int)P.outs.size(), st);
    mark(VC_STAGE_FINAL, 1, st);
    mark(VC_STAGE_PROOF, 1, st);
    // the branches join the stream at the end
    for (int k = 0; k < 2; k++)
        if (k ? marked_aux : marked) {
            cudaEventRecord(P.ev_mark, k ? P.evs_aux : P.evs);
            cudaStreamWaitEvent(st, P.ev_mark, 0);
        }
}

cudaError_t find_kernel_node(cudaGraph_t g, const void *fn, cudaGraphNode_t *node, cudaKernelNodeParams *kp)
{
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) e = cudaGraphGetNodes(g, nodes.data(), &n);
    for (size_t k = 0; e == cudaSuccess && k < n; k++) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[k], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p{};
        e = cudaGraphKernelNodeGetParams(nodes[k], &p);
        if (e == cudaSuccess && p.func == fn) {
            *node = nodes[k];
            *kp = p;
            kp->kernelParams = nullptr;  // owned by the node; each update passes its own
            kp->extra = nullptr;
            return cudaSuccess;
        }
    }
    return e == cudaSuccess ? cudaErrorInvalidValue : e;
}

// Capture what `enqueue` puts on a stream into an instantiated graph; with
// `fn`, also find that kernel's node (the graph is then kept in *keep).
template <class F>
static cudaError_t capture_graph(cudaStream_t cap, F enqueue, cudaGraphExec_t *exec, const void *fn,
                                 cudaGraph_t *keep, cudaGraphNode_t *node, cudaKernelNodeParams *kp)
{
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    enqueue(cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess && fn) e = find_kernel_node(g, fn, node, kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) *exec = nullptr;
    if (e == cudaSuccess && fn)
        *keep = g;
    else if (g)
        cudaGraphDestroy(g);
    return e;
}

// Set the arguments of a graph's parameter node for its next launch (launches
// already queued keep theirs).
static cudaError_t set_node_args(cudaGraphExec_t exec, cudaGraphNode_t node, cudaKernelNodeParams kp, void **args)
{
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphExecKernelNodeSetParams(exec, node, &kp);
}

// Run the plan on `st`: replay its CUDA graph (captured on first use, and
// again after the stage events change).  A plan with its own parameter node
// gets (seed, tr, in) through it.
// The launches and copies of one proof of a circuit with staged values
// (Sec. 5.1.2, copy-once-per-layer).  Narrow layers stay on the device; wide
// layers pass through three slots.  Evaluation runs layer by layer from the
// input up; each wide layer is written to host memory on the copy stream as
// soon as it is computed, and a wide layer reuses a slot only after the host
// copy of the slot's previous layer is done.  Then every iteration between
// narrow layers runs in one merged set of launches, and the iterations that
// touch a wide layer run one after the other in order, each on its two
// layers: a wide layer missing from its slot is copied in from host memory,
// ahead of time (while the previous iteration runs) when the slot's previous
// layer is no longer needed by then.  Coins and the final reduction are
// those of the resident plan.
// Evaluation of layer i in a proof with values through slots: a wide layer
// alone; a run of narrow layers in one launch, at its first layer.
static void eval_layer(vc_circuit &c, u32 i, cudaStream_t st)
{
    Plan &P = c.P;
    const int k = c.st_evalstep[i];
    if (k >= 0)
        launch_eval_segs(P.d_G, P.d_segs, P.d_seg_items[k], (int)P.seg_items[k].size(), P.seg_maxblock[k], st);
    else if (k == -1)
        launch_eval_layers(P.d_G, c.d_stLev, c.d_stEval[i], (int)c.stEval[i].size(), st);
}

static void enqueue_staged(vc_circuit &c, cudaStream_t st)
{
    Plan &P = c.P;
    const Globals *Gs = P.d_G;
    const u32 d = c.d;
    cudaStream_t sa = P.aux, cp = c.st_copy;
    enum { EVALUATED = 0, ON_HOST = 1, COPIED_IN = 2, PROVED = 3 };
    auto ev = [&](u32 i, int k) { return c.st_ev[4 * i + k]; };
    auto bytes = [&](u32 i) { return (u64(1) << c.s[i]) * sizeof(u64); };
    auto wide = [&](u32 i) { return c.st_slot[i] >= 0; };
    auto run_list = [&](u32 l) {  // the launches of list l (a group of iterations, or the narrow ones)
        for (size_t g = 0; g < c.stA[l].size(); g++)
            launch_waves(Gs, P.d_lw, P.d_pw, P.d_gw, c.d_stA[l][g], (int)c.stA[l][g].size(),
                         c.d_stctr + c.stctr_off[l] + 2 * g, st);
        if (!c.stBuild[l].empty()) launch_build23(Gs, c.d_stBuild[l], (int)c.stBuild[l].size(), st);
        for (size_t g = 0; g < c.stB[l].size(); g++)
            launch_waves(Gs, P.d_lw, P.d_pw, P.d_gw, c.d_stB[l][g], (int)c.stB[l][g].size(),
                         c.d_stctr + c.stctr_off[l] + 2 * (c.stA[l].size() + g), st);
    };
    launch_params(P.d_G, 0, nullptr, nullptr, st);  // arguments set per launch
    cudaEventRecord(P.ev_fork, st);
    cudaStreamWaitEvent(sa, P.ev_fork, 0);
    launch_coins(Gs, P.ncirc, P.d_eqjobs, (int)P.eqjobs.size(), P.d_scis, P.d_pw, (int)P.pw.size(), sa);
    cudaEventRecord(P.ev_tables, sa);
    // evaluation; holder[s] = the wide layer in slot s (-1: none yet)
    std::vector<int> holder(c.st_nslots, -1);
    auto to_host = [&](u32 i) {
        cudaEventRecord(ev(i, EVALUATED), st);
        cudaStreamWaitEvent(cp, ev(i, EVALUATED), 0);
        cudaMemcpyAsync(c.hV[i], c.V[i], bytes(i), cudaMemcpyDeviceToHost, cp);
        cudaEventRecord(ev(i, ON_HOST), cp);
    };
    launch_check_inputs(Gs, P.d_checks, (int)P.checks.size(), st);  // the inputs are in layer d
    if (wide(d)) {
        holder[c.st_slot[d]] = (int)d;
        to_host(d);
    }
    for (int i = (int)d - 1; i >= 0; i--) {
        if (wide(i)) {
            const int sl = c.st_slot[i];
            if (holder[sl] >= 0) cudaStreamWaitEvent(st, ev(holder[sl], ON_HOST), 0);
            holder[sl] = i;
        }
        eval_layer(c, (u32)i, st);
        if (wide(i)) to_host(i);
    }
    // the outputs for the final reduction (layer 0's slot may be reused)
    cudaMemcpyAsync(c.d_out, c.V[0], bytes(0), cudaMemcpyDeviceToDevice, st);
    cudaStreamWaitEvent(st, P.ev_tables, 0);
    run_list((u32)c.st_groups.size());  // every iteration between narrow layers
    // the groups of iterations touching a wide layer, in order: the group's
    // wide layers missing from their slots are copied in once the group that
    // last used the slot's layer is done (its PROVED event, recorded at its
    // first iteration)
    auto last_use = [&](int L) { return L < (int)d ? L : (int)d - 1; };
    const std::vector<StagedCopy> copies = staged_copies(c);
    size_t k = 0;
    for (u32 g = 0; g < c.st_groups.size(); g++) {
        for (; k < copies.size() && copies[k].group == g; k++) {
            const u32 L = copies[k].layer;
            if (copies[k].prev >= 0) {
                const int pg = c.st_group[last_use(copies[k].prev)];
                cudaStreamWaitEvent(cp, ev(c.st_groups[pg].first, PROVED), 0);
            }
            cudaMemcpyAsync(c.V[L], c.hV[L], bytes(L), cudaMemcpyHostToDevice, cp);
            cudaEventRecord(ev(L, COPIED_IN), cp);
            cudaStreamWaitEvent(st, ev(L, COPIED_IN), 0);
        }
        run_list(g);
        cudaEventRecord(ev(c.st_groups[g].first, PROVED), st);
    }
    cudaEventRecord(ev(d, PROVED), cp);  // join the copy stream
    cudaStreamWaitEvent(st, ev(d, PROVED), 0);
    launch_final(P.d_G, P.d_rounds, (int)P.rounds.size(), (int)P.nbig, P.d_outs, (int)P.outs.size(), st);
}

// Windowed values: one stream evaluates from the input up and runs each
// group of iterations where the plan placed it (before the layer that
// overwrites a slot one of them reads), so stream order alone keeps every
// slot's layer until its last reader is done; the coins run beside the
// evaluation, and the first group waits for them.
static void enqueue_windowed(vc_circuit &c, cudaStream_t st)
{
    Plan &P = c.P;
    const Globals *Gs = P.d_G;
    cudaStream_t sa = P.aux;
    auto run_list = [&](u32 l) {
        for (size_t g = 0; g < c.stA[l].size(); g++)
            launch_waves(Gs, P.d_lw, P.d_pw, P.d_gw, c.d_stA[l][g], (int)c.stA[l][g].size(),
                         c.d_stctr + c.stctr_off[l] + 2 * g, st);
        if (!c.stBuild[l].empty()) launch_build23(Gs, c.d_stBuild[l], (int)c.stBuild[l].size(), st);
        for (size_t g = 0; g < c.stB[l].size(); g++)
            launch_waves(Gs, P.d_lw, P.d_pw, P.d_gw, c.d_stB[l][g], (int)c.stB[l][g].size(),
                         c.d_stctr + c.stctr_off[l] + 2 * (c.stA[l].size() + g), st);
    };
    launch_params(P.d_G, 0, nullptr, nullptr, st);  // arguments set per launch
    cudaEventRecord(P.ev_fork, st);
    cudaStreamWaitEvent(sa, P.ev_fork, 0);
    launch_coins(Gs, P.ncirc, P.d_eqjobs, (int)P.eqjobs.size(), P.d_scis, P.d_pw, (int)P.pw.size(), sa);
    cudaEventRecord(P.ev_tables, sa);
    launch_check_inputs(Gs, P.d_checks, (int)P.checks.size(), st);  // the inputs are in layer d
    bool coins = false;
    for (int step : c.wn_steps) {
        if (step >= 0) {
            eval_layer(c, (u32)step, st);
            // the outputs for the transcript, while layer 0 is in its slot
            if (step == 0) cudaMemcpyAsync(c.d_out, c.V[0], (u64(1) << c.s[0]) * sizeof(u64), cudaMemcpyDeviceToDevice, st);
            continue;
        }
        if (!coins) {
            cudaStreamWaitEvent(st, P.ev_tables, 0);
            coins = true;
        }
        run_list((u32)(-step - 1));
    }
    if (!coins) cudaStreamWaitEvent(st, P.ev_tables, 0);
    run_list((u32)c.st_groups.size());  // iterations between narrow layers not placed in a group
    launch_final(P.d_G, P.d_rounds, (int)P.rounds.size(), (int)P.nbig, P.d_outs, (int)P.outs.size(), st);
}

static cudaError_t plan_launch(Plan &P, cudaStream_t st, u64 seed = 0, u64 *tr = nullptr,
                               const u64 *in = nullptr)
{
    cudaError_t e = cudaSuccess;
    if (!P.exec) {
        e = capture_graph(P.cap,
                          [&](cudaStream_t cs) {
                              if (!P.staged)
                                  enqueue_plan(P, cs);
                              else if (P.staged->flags & VC_VALUES_WINDOWED)
                                  enqueue_windowed(*P.staged, cs);
                              else
                                  enqueue_staged(*P.staged, cs);
                          },
                          &P.exec,
                          P.own_params ? params_kernel() : nullptr, &P.graph, &P.pnode, &P.pkp);
        if (e != cudaSuccess) {
            plan_drop_graph(P);
            return e;
        }
    }
    if (P.own_params) {
        Globals *G = P.d_G;
        void *args[4] = {&G, &seed, &tr, &in};
        e = set_node_args(P.exec, P.pnode, P.pkp, args);
        if (e != cudaSuccess) return e;
    }
    return cudaGraphLaunch(P.exec, st);
}

// Kernel launches of one proof (the parameter write included).
int count_launches(const Plan &P)
{
    int n = 2;  // parameters; coins, eq tables and product weights
    n += !P.checks.empty();
    for (size_t k = 0; k < P.seg_items.size(); k++) n += (!P.seg_items[k].empty()) + (!P.lev_items[k].empty());
    for (const auto &v : P.groupsA) n += !v.empty();
    n += !P.builds.empty();
    n += !P.heavy.empty();
    for (const auto &v : P.groupsB) n += !v.empty();
    return n + 1;  // final
}

cudaError_t circuit_enqueue_proof(vc_circuit *c, const u64 *inputs, u64 seed, u64 *tr, cudaStream_t st)
{
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = plan_launch(c->P, st, seed, tr, nullptr);
    return e;
}

// ---------------------------------------------------------------------------------------
// Circuits
// ---------------------------------------------------------------------------------------

// ---- tile-shape autotuning -------------------------------------------------------
// Size class of a circuit: depth, widest layer, and that layer's wiring kind.
static std::vector<u32> size_class(const vc_circuit_desc *desc)
{
    u32 smax = 0, kmax = 0;
    for (u32 i = 0; i < desc->n_layers; i++)
        if (desc->log_width[i] >= smax) {
            smax = desc->log_width[i];
            kmax = desc->wiring[i];
        }
    return {desc->n_layers, smax, kmax};
}

static std::mutex g_tune_mu;
static std::map<std::vector<u32>, PlanConfig> g_tuned;  // size class -> fastest measured tile shapes

static bool config_ok(const PlanConfig &f)
{
    return f.pr_chunk >= 1 && f.pr_chunk <= PR_CHUNK_LOG && f.gn_chunk >= 1 && f.gn_chunk <= GN_CHUNK_LOG &&
           f.ln_chunk0 >= 1 && f.ln_chunk0 <= LN_CHUNK0_LOG && f.ev_chunk >= 1 && f.ev_chunk <= 11 &&
           (f.pr_split <= 40 || f.pr_split == VC_SPLIT_WIDEST);
}

PlanConfig shape_config(const vc_circuit_desc *desc)
{
    PlanConfig f;
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned.find(size_class(desc));
    if (it != g_tuned.end()) f = it->second;
    return f;
}

vc_status circuit_prepare(const vc_circuit_desc *desc, int device, vc_circuit **out, const PlanConfig *cfg,
                          u32 flags)
{
    if (flags != 0 && flags != VC_VALUES_IN_HOST_MEMORY && flags != VC_VALUES_STAGED && flags != VC_VALUES_WINDOWED &&
        flags != VC_INPUTS_UPLOAD)
        return VC_EINVAL;
    if (!desc || !out || desc->n_layers < 1 || desc->n_layers > 4096 || !desc->log_width || !desc->wiring)
        return VC_EINVAL;
    *out = nullptr;
    if (cfg && !config_ok(*cfg)) return VC_EINVAL;
    vc_circuit *c = new (std::nothrow) vc_circuit();
    if (!c) return VC_ENOMEM;
    c->cfg = cfg ? *cfg : shape_config(desc);
    c->device = device;
    c->flags = flags;
    c->d = desc->n_layers;
    const u32 d = c->d;
    c->s.assign(desc->log_width, desc->log_width + d + 1);
    c->kind.assign(desc->wiring, desc->wiring + d);
    for (u32 i = 0; i <= d; i++)
        if (c->s[i] > 30) {
            delete c;
            return VC_EINVAL;
        }
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
        if (!shape_ok(c->kind[i], si, sn) || ((flags & VC_VALUES_SLOTTED) && c->kind[i] == W_EXPLICIT)) {
            delete c;
            return VC_EINVAL;
        }
        if (c->kind[i] == W_TREE || c->kind[i] == W_F0_FIRST) c->has_add[i] = 1;
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
                if (c->ex_type[i][g] > 1 || c->ex_in1[i][g] >= Sn || c->ex_in2[i][g] >= Sn) {
                    delete c;
                    return VC_EINVAL;
                }
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
    c->P.ncirc = 1;
    c->P.own_params = true;
    c->P.staged = (flags & VC_VALUES_SLOTTED) ? c : nullptr;
    // values through slots: the proof copies the inputs into their layer first
    c->eval_reads_inputs = !(flags & VC_VALUES_SLOTTED) && first_eval_is_input_run(c->P, c->d);
    Arena A;
    A.off = layout(c, 0, 0);
    plan_take(c->P, A, false);
    c->arena_bytes = A.off + 256;
    *out = c;
    return VC_OK;
}

void circuit_free(vc_circuit *c)
{
    if (!c) return;
    for (cudaGraphExec_t x : {c->vexec, c->vin_exec, c->pv_exec})
        if (x) cudaGraphExecDestroy(x);
    for (cudaGraph_t g : {c->vgraph, c->vin_graph, c->pv_graph})
        if (g) cudaGraphDestroy(g);
    for (cudaEvent_t ev : {c->pv_fork, c->pv_join})
        if (ev) cudaEventDestroy(ev);
    if (c->pv_vs) cudaStreamDestroy(c->pv_vs);
    if (c->pg_exec) cudaGraphExecDestroy(c->pg_exec);
    if (c->pg_arena) lib_free(c->pg_arena);
    for (cudaEvent_t ev : c->st_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->st_copy) cudaStreamDestroy(c->st_copy);
    plan_release(c->P);
    if (c->arena) lib_free(c->arena);
    if (c->host_vals) lib_free_host(c->host_vals);
    if (c->h_pinned) lib_free_host(c->h_pinned);
    delete c;
}

vc_status circuit_allocate(vc_circuit *c)
{
    const u32 d = c->d;
    const size_t bytes = c->arena_bytes;
    DevGuard guard(c->device);
    init_device_once(c->device);
    cudaError_t e = lib_malloc(&c->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->arena = nullptr;
        return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA;
    }
    uintptr_t hbase = 0;
    const bool staged = (c->flags & VC_VALUES_SLOTTED) != 0;
    if (c->host_bytes) {
        // mapped for kernels reading the values in place; staged values are
        // only copied, by address on the host
        void *dp = nullptr;
        e = lib_host_alloc(&c->host_vals, c->host_bytes,
                           staged ? cudaHostAllocDefault : (cudaHostAllocMapped | cudaHostAllocPortable));
        if (e == cudaSuccess && !staged) e = cudaHostGetDevicePointer(&dp, c->host_vals, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA;
        }
        memset(c->host_vals, 0, c->host_bytes);
        hbase = reinterpret_cast<uintptr_t>(staged ? static_cast<void *>(c->host_vals) : dp);
    }
    {
        Arena A;
        A.base = reinterpret_cast<uintptr_t>(c->arena);
        A.off = layout(c, A.base, hbase);
        plan_take(c->P, A, false);
    }
    e = cudaMemset(c->arena, 0, bytes);
    if (e == cudaSuccess) e = upload(c->d_layers, c->L);
    if (e == cudaSuccess) e = upload(c->d_eq_verify, c->eq_verify);
    if (e == cudaSuccess) e = upload(c->d_explicit_layers, c->explicit_layers);
    if (e == cudaSuccess) e = upload(c->d_vwire, c->vwire);
    if (e == cudaSuccess) e = upload(c->d_round_layer, c->round_layer);
    if (e == cudaSuccess) e = upload(c->d_zmap, c->zmap);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_G, &c->G, sizeof(Globals), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_Gv, &c->Gv, sizeof(Globals), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = plan_upload(c->P);
    if (e == cudaSuccess && staged) e = staged_upload(c);
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
    if (e == cudaSuccess) e = plan_resources(c->P);
    if (e == cudaSuccess) {
        // on a private stream: creation does not wait for other work on the device
        launch_init_invfact(c->G.invfact, c->P.cap);
        e = cudaStreamSynchronize(c->P.cap);
    }
    if (e == cudaSuccess) e = lib_host_alloc(&c->h_pinned, 64 * sizeof(u64), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    return VC_OK;
}

extern "C" vc_status vc_circuit_create(const vc_circuit_desc *desc, int device, vc_circuit **out)
{
    return vc_circuit_create_ex(desc, device, 0, out);
}

extern "C" vc_status vc_circuit_create_ex(const vc_circuit_desc *desc, int device, uint32_t flags, vc_circuit **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    if (flags == VC_VALUES_AUTO) {
        // device-resident values, else windowed ones, else mapped host
        // memory: the first whose memory can be had
        vc_status st = vc_circuit_create_ex(desc, device, 0, out);
        if (st != VC_ENOMEM) return st;
        st = vc_circuit_create_ex(desc, device, VC_VALUES_WINDOWED, out);
        if (st != VC_ENOMEM && st != VC_EINVAL) return st;  // VC_EINVAL: explicit wirings are not windowed
        return vc_circuit_create_ex(desc, device, VC_VALUES_IN_HOST_MEMORY, out);
    }
    vc_circuit *c = nullptr;
    vc_status st = circuit_prepare(desc, device, &c, nullptr, flags);
    if (st != VC_OK) return st;
    st = circuit_allocate(c);
    if (st != VC_OK) {
        DevGuard guard(device);
        circuit_free(c);
        return st;
    }
    *out = c;
    return VC_OK;
}

extern "C" vc_status vc_circuit_destroy(vc_circuit *c)
{
    if (!c) return VC_OK;
    DevGuard guard(c->device);
    cudaDeviceSynchronize();
    circuit_free(c);
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

// Pointer kind: 1 = device memory of `device`, 0 = host, -1 = device memory of
// another device.  With `mapped`: for page-locked host memory that the current
// device can address, its device address (else NULL).
int ptr_kind(const void *p, int device, const void **mapped)
{
    if (mapped) *mapped = nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == device ? 1 : -1;
    // (only where the device address is the host address, as under unified addressing)
    if (mapped && a.type == cudaMemoryTypeHost && a.devicePointer == p) *mapped = p;
    return 0;
}

cudaError_t queue_status(vc_circuit *c, cudaStream_t st, int w0, int n)
{
    u32 *h = reinterpret_cast<u32 *>(c->h_pinned) + w0;
    cudaError_t e = cudaMemcpyAsync(h, c->G.status + w0, n * sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->G.status + w0, 0, n * sizeof(u32), st);
    return e;
}

vc_status decode_status(const vc_circuit *c, int w0, int n)
{
    u32 s = 0;
    for (int k = 0; k < n; k++) s |= reinterpret_cast<const u32 *>(c->h_pinned)[w0 + k];
    if (s & ST_BAD_INPUT) return VC_EINVAL;
    if (s & ST_TIMEOUT) return VC_ETIMEOUT;
    return VC_OK;
}

static vc_status read_status_and_clear(vc_circuit *c, cudaStream_t st, int w0 = 0, int n = 1)
{
    cudaError_t e = queue_status(c, st, w0, n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return VC_ECUDA;
    return decode_status(c, w0, n);
}

extern "C" vc_status vc_prove(vc_circuit *c, const uint64_t *inputs, uint64_t seed, uint64_t *transcript,
                              void *stream)
{
    if (!c || !inputs || !transcript) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const void *mapped = nullptr;
    const int ki = ptr_kind(inputs, c->device, &mapped), kt = ptr_kind(transcript, c->device);
    if (ki < 0 || kt < 0) return VC_EINVAL;
    // inputs the device can address are read in place by the first evaluation
    // launch (which writes the input layer); otherwise they are copied first,
    // as are page-locked host inputs of a circuit that uploads them
    const bool upload = (c->flags & VC_INPUTS_UPLOAD) && ki == 0 && mapped;
    const u64 *in = nullptr;
    if (c->eval_reads_inputs && !upload) in = ki ? inputs : static_cast<const u64 *>(mapped);
    cudaError_t e = cudaSuccess;
    if (!in) {
        const u64 nin = u64(1) << c->s[c->d];
        e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64), cudaMemcpyDefault, st);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    e = plan_launch(c->P, st, seed, kt ? transcript : c->d_tr, in);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    if (!kt) {
        e = cudaMemcpyAsync(transcript, c->d_tr, c->tr_len * sizeof(u64), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    if (kt && (ki || in || upload)) return VC_OK;  // no pageable input copy: asynchronous, status latched
    return read_status_and_clear(c, st);
}

// ---- the per-gate prover: device state and its launch sequence ---------------------

static vc_status pergate_prepare(vc_circuit *c)
{
    if (c->pg_arena) return VC_OK;
    const u32 d = c->d, gpc = pergate_gpt();
    std::vector<PgLayer> pl(d);
    std::vector<u32> blk, lblk;
    u32 rounds = 0;
    auto blocks = [&](u64 n) { return u32((n + gpc - 1) / gpc); };
    for (u32 i = 0; i < d; i++) {
        PgLayer &Q = pl[i];
        Q = PgLayer{};
        Q.layer = i;
        Q.s = c->s[i];
        Q.sn = c->s[i + 1];
        Q.n = Q.s + 2 * Q.sn;
        rounds = std::max(rounds, Q.n);
        Q.blk0 = (u32)blk.size();
        Q.nblk = blocks(u64(1) << Q.s);
        blk.insert(blk.end(), Q.nblk, i);
        Q.lblk0 = (u32)lblk.size();
        Q.lnblk = blocks(u64(1) << Q.sn);
        lblk.insert(lblk.end(), Q.lnblk, i);
    }
    // one allocation: sizing pass (base 0), then the real one
    auto carve = [&](Arena &A) {
        for (u32 i = 0; i < d; i++) {
            PgLayer &Q = pl[i];
            const u64 S = u64(1) << Q.s, Sn = u64(1) << Q.sn;
            const u32 h = (Q.sn + 1) / 2;
            Q.preP = A.take<u64>(S);
            Q.preA = A.take<u64>(Sn);
            Q.preB = A.take<u64>(Sn);
            Q.suf = A.take<u64>(S);
            Q.fa = A.take<u64>(std::max<u64>(1, Sn / 2));
            Q.fb = A.take<u64>(std::max<u64>(1, Sn / 4));
            Q.v1 = A.take<u64>(1);
            Q.part = A.take<u64>(3ull * Q.nblk);
            Q.ltab = A.take<u64>(u64(Q.sn + 1) * ((u64(1) << h) + (u64(1) << (Q.sn - h))));
            Q.lpart = A.take<u64>(u64(Q.sn + 1) * Q.lnblk);
        }
        c->d_pg = A.take<PgLayer>(d);
        c->d_pg_blk = A.take<u32>(blk.size());
        c->d_pg_lblk = A.take<u32>(lblk.size());
    };
    Arena A0;
    carve(A0);
    char *mem = nullptr;
    if (lib_malloc(&mem, A0.off) != cudaSuccess) {
        cudaGetLastError();
        return VC_ENOMEM;
    }
    Arena A;
    A.base = reinterpret_cast<uintptr_t>(mem);
    carve(A);
    cudaError_t e = upload(c->d_pg, pl);
    if (e == cudaSuccess) e = upload(c->d_pg_blk, blk);
    if (e == cudaSuccess) e = upload(c->d_pg_lblk, lblk);
    if (e != cudaSuccess) {
        lib_free(mem);
        return VC_ECUDA;
    }
    c->pg_arena = mem;
    c->pg_nblk = (u32)blk.size();
    c->pg_nlblk = (u32)lblk.size();
    c->pg_rounds = rounds;
    return VC_OK;
}

// Evaluation, the coins (challenges, points, eq(z_i, r_P)) and the per-gate
// rounds, captured once per circuit.
static cudaError_t pergate_launch(vc_circuit *c, cudaStream_t st)
{
    Plan &P = c->P;
    if (!c->pg_exec) {
        cudaError_t e = cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        launch_check_inputs(P.d_G, P.d_checks, (int)P.checks.size(), P.cap);
        for (size_t k = 0; k < P.seg_items.size(); k++) {
            launch_eval_segs(P.d_G, P.d_segs, P.d_seg_items[k], (int)P.seg_items[k].size(), P.seg_maxblock[k], P.cap);
            launch_eval_layers(P.d_G, P.d_levs, P.d_lev_items[k], (int)P.lev_items[k].size(), P.cap);
        }
        launch_coins(P.d_G, 1, nullptr, 0, nullptr, nullptr, 0, P.cap);
        launch_pergate(P.d_G, c->d_pg, (int)c->d, c->d_pg_blk, c->pg_nblk, c->d_pg_lblk, c->pg_nlblk, c->pg_rounds,
                       P.cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(P.cap, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e;
        }
        e = cudaGraphInstantiate(&c->pg_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->pg_exec = nullptr;
            return e;
        }
    }
    return cudaGraphLaunch(c->pg_exec, st);
}

extern "C" vc_status vc_prove_pergate(vc_circuit *c, const uint64_t *inputs, uint64_t seed, uint64_t *transcript,
                                      void *stream)
{
    if (!c || !inputs || !transcript) return VC_EINVAL;
    if (c->flags & VC_VALUES_SLOTTED) return VC_EINVAL;  // reads every layer in place
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ki = ptr_kind(inputs, c->device), kt = ptr_kind(transcript, c->device);
    if (ki < 0 || kt < 0) return VC_EINVAL;
    vc_status s = pergate_prepare(c);
    if (s != VC_OK) return s;
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64),
                                    cudaMemcpyDefault, st);
    if (e != cudaSuccess) return VC_ECUDA;
    launch_params(c->d_G, seed, kt ? transcript : c->d_tr, nullptr, st);
    e = pergate_launch(c, st);
    if (e == cudaSuccess) e = cudaGetLastError();
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
    return read_status_and_clear(c, (cudaStream_t)stream, 0, 2);  // the prover's and the verifier's words
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
                                    cudaMemcpyDefault, st);
    if (e != cudaSuccess) return VC_ECUDA;
    launch_check_canonical(c->V[c->d], nin, c->G.status, st);
    const Plan &P = c->P;
    for (size_t k = 0; k < P.seg_items.size(); k++) {
        launch_eval_segs(P.d_G, P.d_segs, P.d_seg_items[k], (int)P.seg_items[k].size(), P.seg_maxblock[k], st);
        launch_eval_layers(P.d_G, P.d_levs, P.d_lev_items[k], (int)P.lev_items[k].size(), st);
    }
    e = cudaMemcpyAsync(outputs, c->V[0], (u64(1) << c->s[0]) * sizeof(u64),
                        cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    return read_status_and_clear(c, st);
}

// The transcript on the device for the verifier: in place, or copied into
// the handle's transcript buffer.
static cudaError_t verifier_transcript(vc_circuit *c, const uint64_t *transcript, int kt, cudaStream_t st,
                                       const u64 **dtr)
{
    *dtr = transcript;
    if (kt) return cudaSuccess;
    *dtr = c->d_tr;
    return cudaMemcpyAsync(c->d_tr, transcript, c->tr_len * sizeof(u64), cudaMemcpyHostToDevice, st);
}

// After a verifier launch: asynchronous return, or wait for the accept bit
// and the verifier's status word.
static vc_status verifier_finish(vc_circuit *c, bool async, int ka, int *accept, cudaStream_t st)
{
    if (async) return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
    cudaError_t e = cudaMemcpyAsync(c->h_pinned + 8, c->d_result, 4 * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    vc_status s = read_status_and_clear(c, st, 1, 1);
    if (s != VC_OK) return s;
    if (!ka) *accept = c->h_pinned[8 + 2] ? 1 : 0;
    return VC_OK;
}

extern "C" vc_status vc_verify(vc_circuit *c, const uint64_t *inputs, uint64_t seed, const uint64_t *transcript,
                               int *accept, void *stream)
{
    if (!c || !inputs || !transcript || !accept) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const void *mapped = nullptr;
    const int ki = ptr_kind(inputs, c->device, &mapped), kt = ptr_kind(transcript, c->device);
    const int ka = ptr_kind(accept, c->device);
    if (ki < 0 || kt < 0 || ka < 0) return VC_EINVAL;
    if (!ka) *accept = 0;
    c->vin_pending = false;  // this call reuses the input pass's scratch
    const u64 nin = u64(1) << c->s[c->d];
    cudaError_t e = cudaSuccess;
    // the input MLE reads the inputs once: in place when the device can address
    // them, else from a copy (page-locked ones of a circuit that uploads its
    // inputs into the verifier's own buffer)
    const bool upload = (c->flags & VC_INPUTS_UPLOAD) && ki == 0 && mapped;
    const u64 *din = ki ? inputs : upload ? nullptr : static_cast<const u64 *>(mapped);
    if (upload) {
        e = cudaMemcpyAsync(c->d_vin, inputs, nin * sizeof(u64), cudaMemcpyHostToDevice, st);
        din = c->d_vin;
    } else if (!din) {
        e = cudaMemcpyAsync(c->V[c->d], inputs, nin * sizeof(u64), cudaMemcpyDefault, st);
        din = c->V[c->d];
    }
    const u64 *dtr = nullptr;
    if (e == cudaSuccess) e = verifier_transcript(c, transcript, kt, st, &dtr);
    if (e != cudaSuccess) return VC_ECUDA;
    // the verifier's launches are one captured graph; its first node writes
    // the per-call pointers and seed, with arguments set before each launch
    if (!c->vexec) {
        auto enqueue = [&](cudaStream_t cs) {
            launch_vparams(c->d_Gv, c->d_vp, 0, nullptr, nullptr, nullptr, c->d_result, cs);
            cudaEventRecord(c->P.ev_fork, cs);
            cudaStreamWaitEvent(c->P.aux, c->P.ev_fork, 0);
            launch_coins(c->d_Gv, 1, c->d_eq_verify, (int)c->eq_verify.size(), nullptr, nullptr, 0, cs);
            launch_verify(c->d_Gv, c->Gv, c->Vd, c->s[c->d], c->s[0], c->d_vwire, (int)c->vwire.size(),
                          c->P.aux, c->P.ev_tables, cs);
        };
        e = capture_graph(c->P.cap, enqueue, &c->vexec, vparams_kernel(), &c->vgraph, &c->vpnode, &c->vpkp);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    {
        Globals *G = c->d_Gv;
        VerifyPtrs *vp = c->d_vp;
        int *acc_out = ka ? accept : nullptr;
        u64 *res = c->d_result;
        void *args[7] = {&G, &vp, &seed, &dtr, &din, &acc_out, &res};
        e = set_node_args(c->vexec, c->vpnode, c->vpkp, args);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(c->vexec, st);
    if (e != cudaSuccess) return VC_ECUDA;
    return verifier_finish(c, ka && (ki || upload) && kt, ka, accept, st);
}

extern "C" vc_status vc_verify_input(vc_circuit *c, const uint64_t *inputs, uint64_t seed, void *stream)
{
    if (!c || !inputs) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const void *mapped = nullptr;
    const int ki = ptr_kind(inputs, c->device, &mapped);
    // the pass reads its inputs in place, or page-locked ones of a circuit
    // that uploads its inputs from the verifier's own copy
    const bool upload = (c->flags & VC_INPUTS_UPLOAD) && ki == 0 && mapped;
    const u64 *din = ki > 0 ? inputs : upload ? c->d_vin : static_cast<const u64 *>(mapped);
    if (ki < 0 || !din) return VC_EINVAL;
    cudaError_t e = cudaSuccess;
    if (upload) {
        e = cudaMemcpyAsync(c->d_vin, inputs, (u64(1) << c->s[c->d]) * sizeof(u64), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    if (!c->vin_exec) {
        auto enqueue = [&](cudaStream_t cs) {
            launch_vparams_in(c->d_Gv, c->d_vp, 0, nullptr, cs);
            cudaEventRecord(c->P.ev_fork, cs);
            cudaStreamWaitEvent(c->P.aux, c->P.ev_fork, 0);
            launch_verify_input(c->d_Gv, c->Gv, c->Vd, c->s[c->d], c->s[0], c->P.aux);
            cudaEventRecord(c->P.ev_tables, c->P.aux);
            launch_coins(c->d_Gv, 1, nullptr, 0, nullptr, nullptr, 0, cs);
            cudaStreamWaitEvent(cs, c->P.ev_tables, 0);
        };
        e = capture_graph(c->P.cap, enqueue, &c->vin_exec, vparams_in_kernel(), &c->vin_graph, &c->vin_node,
                          &c->vin_kp);
        if (e != cudaSuccess) return VC_ECUDA;
    }
    Globals *G = c->d_Gv;
    VerifyPtrs *vp = c->d_vp;
    void *args[4] = {&G, &vp, &seed, &din};
    e = set_node_args(c->vin_exec, c->vin_node, c->vin_kp, args);
    if (e == cudaSuccess) e = cudaGraphLaunch(c->vin_exec, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    c->vin_pending = true;
    c->vin_seed = seed;
    c->vin_sync = ki == 0 && !upload;
    return VC_OK;
}

extern "C" vc_status vc_verify_transcript(vc_circuit *c, uint64_t seed, const uint64_t *transcript, int *accept,
                                          void *stream)
{
    if (!c || !transcript || !accept) return VC_EINVAL;
    if (!c->vin_pending || c->vin_seed != seed) return VC_EINVAL;
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int kt = ptr_kind(transcript, c->device), ka = ptr_kind(accept, c->device);
    if (kt < 0 || ka < 0) return VC_EINVAL;
    c->vin_pending = false;
    if (!ka) *accept = 0;
    const u64 *dtr = nullptr;
    cudaError_t e = verifier_transcript(c, transcript, kt, st, &dtr);
    if (e != cudaSuccess) return VC_ECUDA;
    // plain launches with the per-call pointers as arguments (one launch for
    // structured circuits): nothing to capture, nothing to write first
    launch_coins(c->d_Gv, 0, c->d_eq_verify, (int)c->eq_verify.size(), nullptr, nullptr, 0, st);
    launch_verify_transcript(c->d_Gv, c->Gv, c->Vd, c->s[c->d], c->s[0], c->d_vwire, (int)c->vwire.size(), dtr,
                             ka ? accept : nullptr, st);
    return verifier_finish(c, ka && kt && !c->vin_sync, ka, accept, st);
}

// The proof and its verification as one graph: the verifier's branch (its
// parameters, coins and eq tables, and the inputs' MLE at its final point,
// all fixed by the seed) forks at the start and runs beside the proof; the
// checks of the transcript follow the proof's final reduction and join the
// branch.  Parameters: the prover's k_params node and the verifier's
// k_vparams node, set before each launch.
static cudaError_t pv_capture(vc_circuit *c)
{
    cudaError_t e = cudaSuccess;
    if (!c->pv_vs) e = cudaStreamCreateWithFlags(&c->pv_vs, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->pv_fork) e = cudaEventCreateWithFlags(&c->pv_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !c->pv_join) e = cudaEventCreateWithFlags(&c->pv_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    cudaStream_t cs = c->P.cap;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    // the proof's launches are captured first, so that the graph starts them
    // ahead of the verifier's branch, which forks from the start
    cudaEventRecord(c->pv_fork, cs);
    enqueue_plan(c->P, cs);
    cudaStreamWaitEvent(c->pv_vs, c->pv_fork, 0);
    launch_vparams(c->d_Gv, c->d_vp, 0, nullptr, nullptr, nullptr, c->d_result, c->pv_vs);
    launch_coins(c->d_Gv, 1, c->d_eq_verify, (int)c->eq_verify.size(), nullptr, nullptr, 0, c->pv_vs);
    launch_verify_input(c->d_Gv, c->Gv, c->Vd, c->s[c->d], c->s[0], c->pv_vs);
    cudaEventRecord(c->pv_join, c->pv_vs);
    cudaStreamWaitEvent(cs, c->pv_join, 0);
    // transcript and accept pointer from the verifier's parameters
    launch_verify_transcript(c->d_Gv, c->Gv, c->Vd, c->s[c->d], c->s[0], c->d_vwire, (int)c->vwire.size(), nullptr,
                             nullptr, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = find_kernel_node(g, params_kernel(), &c->pv_pnode, &c->pv_pkp);
    if (e == cudaSuccess) e = find_kernel_node(g, vparams_kernel(), &c->pv_vnode, &c->pv_vkp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->pv_exec, g, 0);
    if (e != cudaSuccess) {
        c->pv_exec = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return e;
    }
    c->pv_graph = g;
    return cudaSuccess;
}

extern "C" vc_status vc_prove_verify(vc_circuit *c, const uint64_t *inputs, uint64_t seed, uint64_t *transcript,
                                     int *accept, void *stream)
{
    if (!c || !inputs || !transcript || !accept) return VC_EINVAL;
    if (c->P.staged || !c->P.own_params) return VC_EINVAL;  // values through device slots: vc_prove, vc_verify
    DevGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const void *mapped = nullptr;
    const int ki = ptr_kind(inputs, c->device, &mapped), kt = ptr_kind(transcript, c->device);
    const int ka = ptr_kind(accept, c->device);
    if (ki < 0 || kt < 0 || ka < 0) return VC_EINVAL;
    if (!ka) *accept = 0;
    c->vin_pending = false;  // this call reuses the input pass's scratch
    // the prover's inputs as in vc_prove; the verifier reads them where the
    // prover does: in place, or in the input layer the library's copy filled
    // (no launch writes that layer then)
    const bool upload = (c->flags & VC_INPUTS_UPLOAD) && ki == 0 && mapped;
    const u64 *in = nullptr;
    if (c->eval_reads_inputs && !upload) in = ki ? inputs : static_cast<const u64 *>(mapped);
    cudaError_t e = cudaSuccess;
    if (!in)
        e = cudaMemcpyAsync(c->V[c->d], inputs, (u64(1) << c->s[c->d]) * sizeof(u64), cudaMemcpyDefault, st);
    const u64 *din = in ? in : ki > 0 ? inputs : c->V[c->d];
    if (e == cudaSuccess && !c->pv_exec) e = pv_capture(c);
    u64 *tr = kt ? transcript : c->d_tr;
    const u64 *trc = tr;
    int *acc = ka ? accept : nullptr;
    Globals *G = c->P.d_G, *Gv = c->d_Gv;
    VerifyPtrs *vp = c->d_vp;
    u64 *res = c->d_result;
    void *pargs[4] = {&G, &seed, &tr, &in};
    void *vargs[7] = {&Gv, &vp, &seed, &trc, &din, &acc, &res};
    if (e == cudaSuccess) e = set_node_args(c->pv_exec, c->pv_pnode, c->pv_pkp, pargs);
    if (e == cudaSuccess) e = set_node_args(c->pv_exec, c->pv_vnode, c->pv_vkp, vargs);
    if (e == cudaSuccess) e = cudaGraphLaunch(c->pv_exec, st);
    if (e == cudaSuccess && !kt)
        e = cudaMemcpyAsync(transcript, c->d_tr, c->tr_len * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    if (kt && ka && (ki || in || upload)) return VC_OK;  // asynchronous, statuses latched
    const vc_status s = read_status_and_clear(c, st);
    if (s != VC_OK) return s;
    return verifier_finish(c, false, ka, accept, st);
}

extern "C" vc_status vc_circuit_set_stage_events(vc_circuit *c, void *const *events)
{
    if (!c) return VC_EINVAL;
    DevGuard guard(c->device);
    if (c->P.exec) {  // the events are part of the captured graph: capture again
        plan_drop_graph(c->P);
    }
    if (c->pv_exec) {  // and of the proof-and-verification graph
        cudaGraphExecDestroy(c->pv_exec);
        cudaGraphDestroy(c->pv_graph);
        c->pv_exec = nullptr;
        c->pv_graph = nullptr;
    }
    c->P.stage_on = events != nullptr;
    if (events)
        for (int k = 0; k < 2 * VC_NUM_STAGES; k++) c->P.stage_ev[k] = (cudaEvent_t)events[k];
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
    I.prove_launches = (uint32_t)count_launches(c->P);
    // parameters, coins and eq tables, input/output MLE, wiring (EXPLICIT only), checks
    I.verify_launches = (uint32_t)(4 + (c->explicit_layers.empty() ? 0 : 1));
    // input pass: parameters, coins, input MLE; transcript pass: eq tables
    // and wiring (EXPLICIT only), output MLE (many outputs only), checks
    I.verify2_launches = (uint32_t)(4 + (c->explicit_layers.empty() ? 0 : 2) + (c->Vd.mle_out_blocks ? 1 : 0));
    I.wave_tasks = (uint32_t)(c->P.groupsA.empty() ? 0 : c->P.groupsA[0].size());
    I.residency = c->flags & ~VC_INPUTS_UPLOAD;
    I.link_bytes = c->P.staged ? c->st_link_bytes : 0;
    *info = I;
    return VC_OK;
}

// Mean time of `reps` proofs of a circuit of shape `desc` built with tiles `f`
// (inputs all zero, device buffers, after two warm-up proofs).
static vc_status time_config(const vc_circuit_desc *desc, int device, const PlanConfig &f, int reps, u64 *din,
                             u64 *dtr, cudaStream_t st, double *ms)
{
    vc_circuit *c = nullptr;
    vc_status s = circuit_prepare(desc, device, &c, &f);
    if (s != VC_OK) return s;
    s = circuit_allocate(c);
    if (s == VC_OK) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int k = 0; k < 2 && s == VC_OK; k++) s = vc_prove(c, din, 1 + k, dtr, st);
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && s == VC_OK; k++) s = vc_prove(c, din, 10 + k, dtr, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess && s == VC_OK) s = VC_ECUDA;
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s == VC_OK) s = read_status_and_clear(c, st);
    }
    cudaStreamSynchronize(st);
    circuit_free(c);
    return s;
}

extern "C" vc_status vc_autotune(const vc_circuit_desc *desc, int device, int reps, vc_tile_config *best,
                                 double *best_ms)
{
    if (!desc || !desc->log_width || !desc->wiring || desc->n_layers < 1 || reps < 1) return VC_EINVAL;
    for (u32 i = 0; i < desc->n_layers; i++)
        if (desc->wiring[i] == W_EXPLICIT) return VC_EINVAL;  // tuned per structured shape
    DevGuard guard(device);
    init_device_once(device);
    const u64 nin = u64(1) << desc->log_width[desc->n_layers];
    vc_circuit *probe = nullptr;
    vc_status s = circuit_prepare(desc, device, &probe, nullptr);
    if (s != VC_OK) return s;
    const u64 trl = probe->tr_len;
    PlanConfig cur = probe->cfg;
    circuit_free(probe);
    u64 *din = nullptr, *dtr = nullptr;
    cudaStream_t st = nullptr;
    if (lib_malloc(&din, nin * sizeof(u64)) != cudaSuccess || lib_malloc(&dtr, trl * sizeof(u64)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (din) lib_free(din);
        if (dtr) lib_free(dtr);
        return VC_ENOMEM;
    }
    cudaMemsetAsync(din, 0, nin * sizeof(u64), st);
    double cur_ms = 0;
    s = time_config(desc, device, cur, reps, din, dtr, st, &cur_ms);
    // coordinate descent over the five knobs (split: below the widest layer,
    // below half of its size, never)
    u32 smax = 0;
    for (u32 i = 0; i <= desc->n_layers; i++) smax = std::max(smax, desc->log_width[i]);
    const u32 cand[5][4] = {{11, 12, 13, 0}, {10, 11, 12, 0}, {11, 12, 13, 0}, {8, 9, 10, 11},
                            {VC_SPLIT_WIDEST, smax ? smax - 1 : 0, 0, VC_SPLIT_WIDEST}};
    const int ncand[5] = {3, 3, 3, 4, 3};
    for (int knob = 0; knob < 5 && s == VC_OK; knob++)
        for (int j = 0; j < ncand[knob]; j++) {
            PlanConfig f = cur;
            u32 *field = knob == 0 ? &f.pr_chunk : knob == 1 ? &f.gn_chunk : knob == 2 ? &f.ln_chunk0
                       : knob == 3 ? &f.ev_chunk : &f.pr_split;
            if (*field == cand[knob][j]) continue;
            *field = cand[knob][j];
            double ms = 0;
            s = time_config(desc, device, f, reps, din, dtr, st, &ms);
            if (s == VC_OK && ms < 0.98 * cur_ms) {
                cur = f;
                cur_ms = ms;
            }
        }
    lib_free(din);
    lib_free(dtr);
    cudaStreamDestroy(st);
    if (s != VC_OK) return s;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tuned[size_class(desc)] = cur;
    }
    if (best) *best = {cur.pr_chunk, cur.gn_chunk, cur.ln_chunk0, cur.ev_chunk, cur.pr_split};
    if (best_ms) *best_ms = cur_ms;
    return VC_OK;
}

// Mean time of `reps` proofs of a merged batch of circuits of shapes
// descs[0..n) built with tile shapes f (after two untimed proofs; the first
// captures the batch's graph).  Every member reads the same zero inputs.
static vc_status time_batch_config(const vc_circuit_desc *descs, int n, int device, const PlanConfig &f, int reps,
                                   const u64 *din, cudaStream_t st, double *ms)
{
    std::vector<vc_circuit *> cs(n, nullptr);
    vc_status s = VC_OK;
    u64 trl = 0;
    for (int j = 0; j < n && s == VC_OK; j++) {
        s = circuit_prepare(&descs[j], device, &cs[j], &f);
        if (s == VC_OK) s = circuit_allocate(cs[j]);
        if (s == VC_OK) trl += cs[j]->tr_len;
    }
    vc_batch *b = nullptr;
    u64 *dtr = nullptr;
    if (s == VC_OK) s = vc_batch_create(cs.data(), n, &b);
    if (s == VC_OK && lib_malloc(&dtr, trl * sizeof(u64)) != cudaSuccess) {
        cudaGetLastError();
        s = VC_ENOMEM;
    }
    if (s == VC_OK) {
        std::vector<const uint64_t *> ins(n, din);
        std::vector<uint64_t *> trs(n);
        std::vector<uint64_t> seeds(n);
        u64 off = 0;
        for (int j = 0; j < n; j++) {
            trs[j] = dtr + off;
            off += cs[j]->tr_len;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = VC_ECUDA;
        for (int k = 0; k < 2 + reps && s == VC_OK; k++) {
            if (k == 2) cudaEventRecord(e0, st);
            for (int j = 0; j < n; j++) seeds[j] = 1000u * k + j + 1;
            s = vc_batch_prove(b, ins.data(), seeds.data(), trs.data(), st);
        }
        if (s == VC_OK) {
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = VC_ECUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            *ms = t / reps;
        }
        if (s == VC_OK) s = vc_batch_sync(b, st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    cudaStreamSynchronize(st);
    if (b) vc_batch_destroy(b);
    if (dtr) lib_free(dtr);
    for (vc_circuit *c : cs)
        if (c) circuit_free(c);
    return s;
}

extern "C" vc_status vc_autotune_batch(const vc_circuit_desc *descs, int n, int device, int reps,
                                       vc_tile_config *best, double *best_ms)
{
    if (!descs || n < 1 || reps < 1) return VC_EINVAL;
    u64 nin = 0;
    u32 smax = 0;
    for (int j = 0; j < n; j++) {
        const vc_circuit_desc &D = descs[j];
        if (!D.log_width || !D.wiring || D.n_layers < 1 || D.n_layers > 4096) return VC_EINVAL;
        for (u32 i = 0; i < D.n_layers; i++)
            if (D.wiring[i] == W_EXPLICIT || D.log_width[i] > 30) return VC_EINVAL;
        if (D.log_width[D.n_layers] > 30) return VC_EINVAL;
        nin = std::max(nin, u64(1) << D.log_width[D.n_layers]);
        for (u32 i = 0; i <= D.n_layers; i++) smax = std::max(smax, D.log_width[i]);
    }
    DevGuard guard(device);
    init_device_once(device);
    u64 *din = nullptr;
    cudaStream_t st = nullptr;
    if (lib_malloc(&din, nin * sizeof(u64)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (din) lib_free(din);
        return VC_ENOMEM;
    }
    cudaMemsetAsync(din, 0, nin * sizeof(u64), st);
    PlanConfig cur;  // every member's default tile shapes
    double cur_ms = 0;
    vc_status s = time_batch_config(descs, n, device, cur, reps, din, st, &cur_ms);
    // coordinate descent over the knobs, one configuration for every member,
    // timed on the merged batch itself (the split threshold below the widest
    // layer of the batch, below 2^13 and 2^11, or never)
    const u32 cand[5][4] = {{11, 12, 13, 0}, {10, 11, 12, 0}, {11, 12, 13, 0}, {8, 9, 10, 11},
                            {VC_SPLIT_WIDEST, 13, 11, smax ? smax - 1 : 0}};
    const int ncand[5] = {3, 3, 3, 4, 4};
    for (int pass = 0; pass < 2 && s == VC_OK; pass++) {
        bool moved = false;
        for (int knob = 0; knob < 5 && s == VC_OK; knob++)
            for (int j = 0; j < ncand[knob]; j++) {
                PlanConfig f = cur;
                u32 *field = knob == 0 ? &f.pr_chunk : knob == 1 ? &f.gn_chunk : knob == 2 ? &f.ln_chunk0
                           : knob == 3 ? &f.ev_chunk : &f.pr_split;
                if (*field == cand[knob][j]) continue;
                *field = cand[knob][j];
                double ms = 0;
                s = time_batch_config(descs, n, device, f, reps, din, st, &ms);
                if (s == VC_OK && ms < 0.98 * cur_ms) {
                    cur = f;
                    cur_ms = ms;
                    moved = true;
                }
            }
        if (!moved) break;
    }
    lib_free(din);
    cudaStreamDestroy(st);
    if (s != VC_OK) return s;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        for (int j = 0; j < n; j++) g_tuned[size_class(&descs[j])] = cur;
    }
    if (best) *best = {cur.pr_chunk, cur.gn_chunk, cur.ln_chunk0, cur.ev_chunk, cur.pr_split};
    if (best_ms) *best_ms = cur_ms;
    return VC_OK;
}

extern "C" vc_status vc_circuit_create_tiles(const vc_circuit_desc *desc, int device, const vc_tile_config *tiles,
                                            vc_circuit **out)
{
    if (!out || !tiles) return VC_EINVAL;
    *out = nullptr;
    PlanConfig f;
    f.pr_chunk = tiles->pr_chunk_log;
    f.gn_chunk = tiles->gn_chunk_log;
    f.ln_chunk0 = tiles->line_chunk_log;
    f.ev_chunk = tiles->eval_chunk_log;
    f.pr_split = tiles->pr_split_log;
    vc_circuit *c = nullptr;
    vc_status st = circuit_prepare(desc, device, &c, &f);
    if (st != VC_OK) return st;
    st = circuit_allocate(c);
    if (st != VC_OK) {
        DevGuard guard(device);
        circuit_free(c);
        return st;
    }
    *out = c;
    return VC_OK;
}

extern "C" vc_status vc_circuit_get_tiles(const vc_circuit *c, vc_tile_config *tiles)
{
    if (!c || !tiles) return VC_EINVAL;
    *tiles = {c->cfg.pr_chunk, c->cfg.gn_chunk, c->cfg.ln_chunk0, c->cfg.ev_chunk, c->cfg.pr_split};
    return VC_OK;
}

// ---------------------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------------------

extern "C" vc_status vc_batch_create(vc_circuit *const *circuits, int n, vc_batch **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    if (n <= 0 || !circuits) return VC_EINVAL;
    for (int j = 0; j < n; j++) {
        if (!circuits[j] || circuits[j]->device != circuits[0]->device || (circuits[j]->flags & VC_VALUES_SLOTTED))
            return VC_EINVAL;
        for (int k = 0; k < j; k++)
            if (circuits[k] == circuits[j]) return VC_EINVAL;
    }
    vc_batch *b = new (std::nothrow) vc_batch();
    if (!b) return VC_ENOMEM;
    b->device = circuits[0]->device;
    b->members.assign(circuits, circuits + n);
    DevGuard guard(b->device);
    plan_merge(b->P, b->members);
    // the input copies of members whose first evaluation launch cannot read
    // device inputs in place, as chunks of one gather launch
    std::vector<GatherChunk> gather;
    for (int j = 0; j < n; j++) {
        vc_circuit *c = b->members[j];
        if (c->eval_reads_inputs) continue;
        const u64 nin = u64(1) << c->s[c->d];
        for (u64 s0 = 0; s0 < nin; s0 += GATHER_CHUNK)
            gather.push_back({c->V[c->d] + s0, s0, (u32)j, (u32)std::min<u64>(GATHER_CHUNK, nin - s0)});
    }
    b->ngather = (int)gather.size();
    size_t bytes = 0;
    {
        Arena A;
        plan_take(b->P, A, true);
        A.take<CallParams>(n);
        A.take<GatherChunk>(gather.size());
        bytes = A.off + 256;
    }
    cudaError_t e = lib_malloc(&b->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA;
    }
    b->arena_bytes = bytes;
    {
        Arena A;
        A.base = reinterpret_cast<uintptr_t>(b->arena);
        plan_take(b->P, A, true);
        b->d_cp = A.take<CallParams>(n);
        b->d_gather = A.take<GatherChunk>(gather.size());
    }
    e = upload(b->P.d_G, b->P.h_G);
    if (e == cudaSuccess) e = upload(b->d_gather, gather);
    if (e == cudaSuccess) e = plan_upload(b->P);
    if (e == cudaSuccess) e = lib_host_alloc(&b->h_cp, n * sizeof(CallParams), cudaHostAllocDefault);
    if (e == cudaSuccess) e = plan_resources(b->P);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_release(b->P);
        if (b->h_cp) lib_free_host(b->h_cp);
        lib_free(b->arena);
        delete b;
        return cuda_status(e);
    }
    *out = b;
    return VC_OK;
}

extern "C" vc_status vc_batch_destroy(vc_batch *b)
{
    if (!b) return VC_OK;
    DevGuard guard(b->device);
    cudaDeviceSynchronize();
    plan_release(b->P);
    if (b->arena) lib_free(b->arena);
    if (b->h_cp) lib_free_host(b->h_cp);
    delete b;
    return VC_OK;
}

extern "C" vc_status vc_batch_prove(vc_batch *b, const uint64_t *const *inputs, const uint64_t *seeds,
                                    uint64_t *const *transcripts, void *stream)
{
    if (!b || !inputs || !seeds || !transcripts) return VC_EINVAL;
    DevGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->members.size();
    std::vector<int> kt(n);
    bool all_dev = true, all_in_dev = true;
    for (int j = 0; j < n; j++) {
        vc_circuit *c = b->members[j];
        if (!inputs[j] || !transcripts[j]) return VC_EINVAL;
        const int ki = ptr_kind(inputs[j], c->device);
        kt[j] = ptr_kind(transcripts[j], c->device);
        if (ki < 0 || kt[j] < 0) return VC_EINVAL;
        all_dev = all_dev && ki && kt[j];
        all_in_dev = all_in_dev && ki;
    }
    // the pinned parameter table is rewritten only after the previous call's copy of it finished
    if (cudaEventSynchronize(b->P.ev_params) != cudaSuccess) return VC_ECUDA;
    for (int j = 0; j < n; j++) {
        vc_circuit *c = b->members[j];
        if (!all_in_dev) {  // host inputs: one copy per member
            const u64 nin = u64(1) << c->s[c->d];
            if (cudaMemcpyAsync(c->V[c->d], inputs[j], nin * sizeof(u64), cudaMemcpyDefault, st) != cudaSuccess)
                return VC_ECUDA;
        }
        b->h_cp[j].seed = seeds[j];
        b->h_cp[j].tr = kt[j] ? transcripts[j] : c->d_tr;
        b->h_cp[j].in = inputs[j];
        b->h_cp[j].in_eval = (all_in_dev && c->eval_reads_inputs) ? inputs[j] : nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_cp, b->h_cp, n * sizeof(CallParams), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->P.ev_params, st);
    if (e != cudaSuccess) return VC_ECUDA;
    // device inputs: read in place by the first evaluation launch, or copied
    // by one gather launch (members whose first evaluation step cannot)
    if (all_in_dev) launch_gather_inputs(b->d_cp, b->d_gather, b->ngather, st);
    launch_params_batch(b->P.d_G, b->d_cp, n, st);
    e = plan_launch(b->P, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return VC_ECUDA;
    for (int j = 0; j < n; j++) {
        if (kt[j]) continue;
        vc_circuit *c = b->members[j];
        if (cudaMemcpyAsync(transcripts[j], c->d_tr, c->tr_len * sizeof(u64), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return VC_ECUDA;
    }
    if (all_dev) return VC_OK;
    return vc_batch_sync(b, stream);
}

extern "C" vc_status vc_batch_sync(vc_batch *b, void *stream)
{
    if (!b) return VC_EINVAL;
    DevGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    for (vc_circuit *c : b->members)
        if (queue_status(c, st) != cudaSuccess) return VC_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return VC_ECUDA;
    vc_status worst = VC_OK;
    for (vc_circuit *c : b->members) {
        const vc_status s = decode_status(c);
        if (s != VC_OK) worst = s;
    }
    return worst;
}

extern "C" vc_status vc_batch_get_info(const vc_batch *b, vc_batch_info *info)
{
    if (!b || !info) return VC_EINVAL;
    vc_batch_info I{};
    I.n_members = (uint32_t)b->members.size();
    I.prove_launches = (uint32_t)count_launches(b->P);
    I.device_bytes = b->arena_bytes;
    u64 gates = 0;
    for (const vc_circuit *c : b->members)
        for (u32 i = 0; i < c->d; i++) gates += u64(1) << c->s[i];
    I.gates = gates;
    *info = I;
    return VC_OK;
}

extern "C" vc_status vc_prove_batch(vc_circuit *const *circuits, const uint64_t *const *inputs,
                                    const uint64_t *seeds, uint64_t *const *transcripts, int n, void *stream)
{
    if (n < 0 || (n > 0 && (!circuits || !inputs || !seeds || !transcripts))) return VC_EINVAL;
    if (n == 0) return VC_OK;
    vc_batch *b = nullptr;
    vc_status s = vc_batch_create(circuits, n, &b);
    if (s != VC_OK) return s;
    s = vc_batch_prove(b, inputs, seeds, transcripts, stream);
    if (s == VC_OK) s = vc_batch_sync(b, stream);
    vc_batch_destroy(b);
    return s;
}

// ---------------------------------------------------------------------------------------
// Field arithmetic checks
// ---------------------------------------------------------------------------------------

extern "C" vc_status vc_field_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n, void *stream)
{
    if (!a || !b || !out) return VC_EINVAL;
    launch_field_mul(a, b, out, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}

extern "C" vc_status vc_field_mul_rate(int device, int variant, uint64_t iters, double *rate)
{
    if (!rate || iters == 0 || variant < 0 || variant > 4) return VC_EINVAL;
    DevGuard guard(device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return VC_ECUDA;
    u64 *sink = nullptr;
    if (lib_malloc(&sink, 64) != cudaSuccess) return VC_ENOMEM;
    const double r = run_field_mul_rate(variant, iters, sms, sink);
    lib_free(sink);
    if (r <= 0) return VC_ECUDA;
    *rate = r;
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
    case VC_ECANCELED: return "cancelled";
    default: return "unknown status";
    }
}
