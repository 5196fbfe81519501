// server.cu -- proof server: a request loop with admission by device memory
// and continuous batching (vc_server_* in include/vc.h).
//
// Jobs are queued by vc_server_submit from any host thread.  One worker
// thread per server owns all device work: it admits queued jobs in arrival
// order while the circuits they need fit under the memory cap, merges the
// admitted jobs' launch plans into one launch set (one launch per evaluation
// step and sum-check wave for all of them), and issues it on one of several
// launch slots, each with its own streams.  Jobs that arrive while earlier
// sets run are admitted into the next free slot, so their work overlaps on
// the device.  Circuits are pooled by shape and stay resident (tables,
// scratch, plan) between jobs; a job holds its circuit from admission to
// completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

u64 now_ns()
{
    return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct ShapeKey {
    std::vector<u32> widths, kinds;
    bool operator<(const ShapeKey &o) const
    {
        return widths != o.widths ? widths < o.widths : kinds < o.kinds;
    }
};

struct Shape {
    u64 bytes = 0;                     // device bytes of one circuit of this shape
    bool staged = false;               // resident values exceed the cap: values through device
                                       // slots (windowed), jobs run alone
    u64 tr_len = 0, n_in = 0;
    std::vector<vc_circuit *> idle;    // allocated, not in use
    u32 live = 0;                      // allocated (idle or in use)
    u64 last_used = 0;
};

struct Job {
    u64 id = 0;
    ShapeKey key;
    Shape *shape = nullptr;
    const u64 *inputs = nullptr;
    u64 seed = 0;
    u64 *transcript = nullptr;
    bool in_dev = false, tr_dev = false;
    vc_circuit *c = nullptr;
    u64 t_submit = 0, t_start = 0, t_done = 0;
    vc_status status = VC_OK;
    bool done = false;
    bool claimed = false;  // a vc_server_wait owns the job (one consumer per job)
    u64 stage_off = 0;  // offset of the job's transcript in the slot's pinned staging buffer
};

// One in-flight launch set.
struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    Plan P;
    char *dev = nullptr;
    size_t dev_cap = 0;
    CallParams *h_cp = nullptr;
    size_t cp_cap = 0;
    u64 *h_stage = nullptr;  // pinned staging of host transcripts
    size_t stage_cap = 0;
    std::vector<Job *> jobs;
    bool busy = false;
};

}  // namespace

struct vc_server;
static vc_status server_prepare(const vc_server *s, const vc_circuit_desc *desc, vc_circuit **out,
                                u32 flags = 0);

struct vc_server {
    int device = 0;
    u64 cap = 0;
    u32 max_batch = 16, max_inflight = 4;
    u32 pr_split = 0;  // 0: each circuit's own tile shapes
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<u64, Job *> jobs;
    std::map<ShapeKey, Shape> shapes;
    u64 held = 0, peak_held = 0;
    u64 next_id = 1;
    bool stop = false;
    std::vector<Slot> slots;
    std::thread worker;
    vc_server_stats stats{};
    u32 in_flight = 0;
};

namespace {

// Take an idle circuit of the job's shape, or allocate one under the cap
// (evicting idle circuits of other shapes, least recently used first).
// Called by the worker with the lock held; allocation happens under it.
enum Acq { ACQ_OK, ACQ_WAIT, ACQ_FAIL };

Acq acquire(vc_server *s, Job *j, vc_circuit **out)
{
    Shape &sh = *j->shape;
    if (!sh.idle.empty()) {
        *out = sh.idle.back();
        sh.idle.pop_back();
        return ACQ_OK;
    }
    while (s->held + sh.bytes > s->cap) {
        Shape *victim = nullptr;
        for (auto &kv : s->shapes)
            if (&kv.second != &sh && !kv.second.idle.empty() &&
                (!victim || kv.second.last_used < victim->last_used))
                victim = &kv.second;
        if (!victim) return ACQ_WAIT;  // wait for running jobs to release memory
        vc_circuit *c = victim->idle.back();
        victim->idle.pop_back();
        victim->live--;
        s->held -= victim->bytes;
        cudaDeviceSynchronize();  // cudaFree would synchronise anyway
        circuit_free(c);
        s->stats.circuits_evicted++;
    }
    vc_circuit_desc d{};
    d.n_layers = (u32)j->key.kinds.size();
    d.log_width = j->key.widths.data();
    d.wiring = j->key.kinds.data();
    vc_circuit *c = nullptr;
    if (server_prepare(s, &d, &c, sh.staged ? VC_VALUES_WINDOWED : 0u) != VC_OK) return ACQ_FAIL;
    if (circuit_allocate(c) != VC_OK) {
        circuit_free(c);
        return ACQ_FAIL;
    }
    sh.live++;
    s->held += sh.bytes;
    s->peak_held = std::max(s->peak_held, s->held);
    s->stats.circuits_created++;
    *out = c;
    return ACQ_OK;
}

template <class T>
bool ensure_pinned(T *&p, size_t &cap, size_t n)
{
    if (n <= cap) return true;
    const size_t want = std::max(n, cap * 2);
    if (p) lib_free_host(p);
    p = nullptr;
    cap = 0;
    if (lib_host_alloc(&p, want * sizeof(T), cudaHostAllocDefault) != cudaSuccess) return false;
    cap = want;
    return true;
}

// A job whose values pass through device slots: its circuit's own launch
// sequence on the slot's stream (it cannot be merged with others).
vc_status launch_staged(Slot &sl)
{
    Job *j = sl.jobs[0];
    vc_circuit *c = j->c;
    if (!j->tr_dev) {
        j->stage_off = 0;
        if (!ensure_pinned(sl.h_stage, sl.stage_cap, (size_t)j->shape->tr_len)) return VC_ENOMEM;
    }
    if (circuit_enqueue_proof(c, j->inputs, j->seed, j->tr_dev ? j->transcript : c->d_tr, sl.st) != cudaSuccess)
        return VC_ECUDA;
    if (!j->tr_dev && cudaMemcpyAsync(sl.h_stage, c->d_tr, j->shape->tr_len * sizeof(u64), cudaMemcpyDeviceToHost,
                                      sl.st) != cudaSuccess)
        return VC_ECUDA;
    if (queue_status(c, sl.st) != cudaSuccess) return VC_ECUDA;
    if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return VC_ECUDA;
    return cudaGetLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}

// Issue one launch set for the slot's jobs (circuits assigned).
vc_status launch(vc_server *s, Slot &sl)
{
    if (sl.jobs.size() == 1 && sl.jobs[0]->shape->staged) return launch_staged(sl);
    std::vector<vc_circuit *> cs;
    for (Job *j : sl.jobs) cs.push_back(j->c);
    // merged plan; the slot's streams and events are kept across sets
    Plan res = sl.P;
    plan_merge(sl.P, cs);
    sl.P.aux = res.aux;
    sl.P.cap = res.cap;
    sl.P.ev_fork = res.ev_fork;
    sl.P.ev_tables = res.ev_tables;
    sl.P.ev_params = res.ev_params;
    const int n = (int)cs.size();
    const size_t need = plan_bytes(sl.P, true) + (size_t)n * sizeof(CallParams) + 512;
    if (need > sl.dev_cap) {
        if (sl.dev) {
            cudaStreamSynchronize(sl.st);
            lib_free(sl.dev);
        }
        sl.dev = nullptr;
        sl.dev_cap = 0;
        const size_t want = std::max(need, (size_t)16 << 20);
        if (lib_malloc(&sl.dev, want) != cudaSuccess) {
            cudaGetLastError();
            return VC_ENOMEM;
        }
        sl.dev_cap = want;
    }
    Arena A;
    A.base = reinterpret_cast<uintptr_t>(sl.dev);
    plan_take(sl.P, A, true);
    CallParams *d_cp = A.take<CallParams>(n);
    if (!ensure_pinned(sl.h_cp, sl.cp_cap, (size_t)n)) return VC_ENOMEM;
    u64 stage = 0;
    for (Job *j : sl.jobs)
        if (!j->tr_dev) {
            j->stage_off = stage;
            stage += j->shape->tr_len;
        }
    if (stage && !ensure_pinned(sl.h_stage, sl.stage_cap, (size_t)stage)) return VC_ENOMEM;
    if (plan_upload_async(sl.P, sl.st) != cudaSuccess) return VC_ECUDA;
    for (int k = 0; k < n; k++) {
        Job *j = sl.jobs[k];
        vc_circuit *c = j->c;
        if (cudaMemcpyAsync(c->V[c->d], j->inputs, j->shape->n_in * sizeof(u64), cudaMemcpyDefault, sl.st) !=
            cudaSuccess)
            return VC_ECUDA;
        sl.h_cp[k].seed = j->seed;
        sl.h_cp[k].tr = j->tr_dev ? j->transcript : c->d_tr;
        sl.h_cp[k].in = nullptr;
        sl.h_cp[k].in_eval = nullptr;  // the server copies every job's inputs into its input layer
    }
    if (cudaMemcpyAsync(d_cp, sl.h_cp, n * sizeof(CallParams), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
        return VC_ECUDA;
    launch_params_batch(sl.P.d_G, d_cp, n, sl.st);
    enqueue_plan(sl.P, sl.st);
    for (Job *j : sl.jobs) {
        vc_circuit *c = j->c;
        if (!j->tr_dev &&
            cudaMemcpyAsync(sl.h_stage + j->stage_off, c->d_tr, j->shape->tr_len * sizeof(u64),
                            cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
            return VC_ECUDA;
        if (queue_status(c, sl.st) != cudaSuccess) return VC_ECUDA;
    }
    if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return VC_ECUDA;
    if (cudaGetLastError() != cudaSuccess) return VC_ECUDA;
    return VC_OK;
}

// Completion of a slot's set: results to the callers, circuits back to the pool.
void finish(vc_server *s, Slot &sl, vc_status launch_status)
{
    const u64 t = now_ns();
    std::lock_guard<std::mutex> g(s->mu);
    for (Job *j : sl.jobs) {
        if (launch_status == VC_OK && !j->tr_dev)
            std::memcpy(j->transcript, sl.h_stage + j->stage_off, j->shape->tr_len * sizeof(u64));
        j->status = (launch_status != VC_OK) ? launch_status : decode_status(j->c);
        j->t_done = t;
        j->done = true;
        j->shape->idle.push_back(j->c);
        j->shape->last_used = t;
        j->c = nullptr;
        s->stats.completed++;
    }
    s->in_flight -= (u32)sl.jobs.size();
    sl.jobs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
}

void worker_main(vc_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        // completions
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish(s, sl, q == cudaSuccess ? VC_OK : VC_ECUDA);
            progressed = true;
        }
        // admission into a free slot
        Slot *free_slot = nullptr;
        for (Slot &sl : s->slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        bool any_busy = false;
        for (Slot &sl : s->slots) any_busy = any_busy || sl.busy;
        if (free_slot) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->pending.empty() && !any_busy) break;
            const u64 t = now_ns();
            while (!s->pending.empty() && free_slot->jobs.size() < s->max_batch) {
                Job *j = s->pending.front();
                // a job with staged values runs alone in its slot
                if (!free_slot->jobs.empty() && (j->shape->staged || free_slot->jobs[0]->shape->staged)) break;
                vc_circuit *c = nullptr;
                const Acq a = acquire(s, j, &c);
                if (a == ACQ_WAIT && (any_busy || !free_slot->jobs.empty())) break;  // memory frees up later
                s->pending.pop_front();
                if (a != ACQ_OK) {  // cannot be served (allocation failed, nothing left to wait for)
                    j->status = VC_ENOMEM;
                    j->t_start = j->t_done = t;
                    j->done = true;
                    s->stats.completed++;
                    s->cv_done.notify_all();
                    continue;
                }
                j->c = c;
                j->t_start = t;
                free_slot->jobs.push_back(j);
                if (j->shape->staged) break;
            }
            if (!free_slot->jobs.empty()) {
                s->in_flight += (u32)free_slot->jobs.size();
                s->stats.max_jobs_in_flight = std::max(s->stats.max_jobs_in_flight, s->in_flight);
                s->stats.launch_sets++;
                free_slot->busy = true;
                lk.unlock();
                const vc_status st = launch(s, *free_slot);
                if (st != VC_OK) {
                    cudaStreamSynchronize(free_slot->st);
                    cudaGetLastError();
                    finish(s, *free_slot, st);
                }
                progressed = true;
            } else if (!any_busy) {
                // nothing running: sleep until a submission arrives
                if (s->stop && s->pending.empty()) break;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace

// A circuit for the server: its shape's tile shapes, with the server's split
// threshold if one was configured.
static vc_status server_prepare(const vc_server *s, const vc_circuit_desc *desc, vc_circuit **out, u32 flags)
{
    if (!s->pr_split) return circuit_prepare(desc, s->device, out, nullptr, flags);
    PlanConfig f = shape_config(desc);
    f.pr_split = s->pr_split;
    return circuit_prepare(desc, s->device, out, &f, flags);
}

extern "C" vc_status vc_server_create(int device, const vc_server_config *cfg, vc_server **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    if (cfg && cfg->pr_split_log > 40) return VC_EINVAL;
    vc_server *s = new (std::nothrow) vc_server();
    if (!s) return VC_ENOMEM;
    s->device = device;
    s->cap = (cfg && cfg->mem_cap_bytes) ? cfg->mem_cap_bytes : (u64)150 << 30;
    s->max_batch = (cfg && cfg->max_batch) ? cfg->max_batch : 16;
    s->max_inflight = (cfg && cfg->max_inflight) ? cfg->max_inflight : 4;
    if (s->max_inflight > 8) s->max_inflight = 8;
    s->pr_split = cfg ? cfg->pr_split_log : 0;
    DevGuard guard(device);
    init_device_once(device);
    s->slots.resize(s->max_inflight);
    cudaError_t e = cudaSuccess;
    for (Slot &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = plan_resources(sl.P);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Slot &sl : s->slots) {
            plan_release(sl.P);
            if (sl.st) cudaStreamDestroy(sl.st);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        delete s;
        return cuda_status(e);
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return VC_OK;
}

extern "C" vc_status vc_server_destroy(vc_server *s)
{
    if (!s) return VC_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    DevGuard guard(s->device);
    cudaDeviceSynchronize();
    for (Slot &sl : s->slots) {
        plan_release(sl.P);
        if (sl.dev) lib_free(sl.dev);
        if (sl.h_cp) lib_free_host(sl.h_cp);
        if (sl.h_stage) lib_free_host(sl.h_stage);
        cudaStreamDestroy(sl.st);
        cudaEventDestroy(sl.done);
    }
    for (auto &kv : s->shapes)
        for (vc_circuit *c : kv.second.idle) circuit_free(c);
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return VC_OK;
}

extern "C" vc_status vc_server_submit(vc_server *s, const vc_circuit_desc *desc, const uint64_t *inputs,
                                      uint64_t seed, uint64_t *transcript, uint64_t *job_id)
{
    if (!s || !desc || !inputs || !transcript || !job_id || !desc->log_width || !desc->wiring ||
        desc->n_layers < 1 || desc->n_layers > 4096)
        return VC_EINVAL;
    ShapeKey key;
    key.widths.assign(desc->log_width, desc->log_width + desc->n_layers + 1);
    key.kinds.assign(desc->wiring, desc->wiring + desc->n_layers);
    for (u32 k : key.kinds)
        if (k == W_EXPLICIT) return VC_EINVAL;  // the server takes structured wirings only
    const int ki = ptr_kind(inputs, s->device), kt = ptr_kind(transcript, s->device);
    if (ki < 0 || kt < 0) return VC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->shapes.find(key);
    if (it == s->shapes.end()) {
        vc_circuit *c = nullptr;
        const vc_status st = server_prepare(s, desc, &c);
        if (st != VC_OK) return st;
        Shape sh;
        sh.bytes = c->arena_bytes;
        sh.tr_len = c->tr_len;
        sh.n_in = u64(1) << c->s[c->d];
        circuit_free(c);  // host-only object
        if (sh.bytes > s->cap) {
            // too large to keep every layer on the device: pass the wide
            // layers through device slots, each iteration run while its two
            // layers are there (windowed values), if that fits
            vc_circuit *cs = nullptr;
            if (server_prepare(s, desc, &cs, VC_VALUES_WINDOWED) == VC_OK) {
                sh.bytes = cs->arena_bytes;
                sh.staged = true;
                circuit_free(cs);
            }
        }
        it = s->shapes.emplace(key, sh).first;
    }
    if (it->second.bytes > s->cap) return VC_EBUSY;
    Job *j = new (std::nothrow) Job();
    if (!j) return VC_ENOMEM;
    j->id = s->next_id++;
    j->key = key;
    j->shape = &it->second;
    j->inputs = inputs;
    j->seed = seed;
    j->transcript = transcript;
    j->in_dev = ki == 1;
    j->tr_dev = kt == 1;
    j->t_submit = now_ns();
    s->jobs[j->id] = j;
    s->pending.push_back(j);
    s->stats.submitted++;
    *job_id = j->id;
    s->cv_work.notify_one();
    return VC_OK;
}

static void fill_info(const Job *j, vc_job_info *info)
{
    info->done = j->done ? 1 : 0;
    info->status = j->done ? j->status : VC_OK;
    info->submit_ns = j->t_submit;
    info->start_ns = j->t_start;
    info->done_ns = j->t_done;
}

extern "C" vc_status vc_server_poll(vc_server *s, uint64_t job_id, vc_job_info *info)
{
    if (!s || !info) return VC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || it->second->claimed) return VC_EINVAL;
    fill_info(it->second, info);
    if (it->second->done) {
        delete it->second;
        s->jobs.erase(it);
    }
    return VC_OK;
}

extern "C" vc_status vc_server_wait(vc_server *s, uint64_t job_id, vc_job_info *info)
{
    if (!s || !info) return VC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || it->second->claimed) return VC_EINVAL;
    Job *j = it->second;
    j->claimed = true;  // no other poll or wait can take (and free) the job meanwhile
    s->cv_done.wait(lk, [&] { return j->done; });
    fill_info(j, info);
    s->jobs.erase(job_id);
    delete j;
    return VC_OK;
}

extern "C" vc_status vc_server_cancel(vc_server *s, uint64_t job_id)
{
    if (!s) return VC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return VC_EINVAL;
    Job *j = it->second;
    auto q = std::find(s->pending.begin(), s->pending.end(), j);
    if (q == s->pending.end()) return VC_EBUSY;  // admitted (on the device) or done
    s->pending.erase(q);
    j->status = VC_ECANCELED;
    j->t_start = j->t_done = now_ns();
    j->done = true;
    s->stats.completed++;
    s->stats.cancelled++;
    s->cv_done.notify_all();
    return VC_OK;
}

extern "C" vc_status vc_server_get_stats(vc_server *s, vc_server_stats *st)
{
    if (!s || !st) return VC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->stats;
    st->held_bytes = s->held;
    st->peak_held_bytes = s->peak_held;
    st->pending = (u64)s->pending.size();
    return VC_OK;
}
