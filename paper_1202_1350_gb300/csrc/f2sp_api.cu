// f2sp_api.cu -- C ABI of the special-purpose non-interactive F2 protocol
// (declarations and contracts in include/vc.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

struct vc_f2sp {
    int device = 0;
    u64 v = 0, h = 0;
    char *mem = nullptr;
    SpFftHost F{};                                            // prover's transform (device tables)
    u64 *pw = nullptr;                                        // u^k, k < 2h (the proof points)
    u64 inv_h = 0;
    u64 *L = nullptr, *M = nullptr, *acc = nullptr;           // verifier state
    u64 *part = nullptr, *proof = nullptr, *res = nullptr;    // prover partials, staging, results
    u32 nparts = 0;
    u32 *status = nullptr;
    u64 *a_stage = nullptr;  // the prover's host inputs are staged here (allocated on first use)
    u64 *h_res = nullptr;    // pinned: results and status readback
    // the verifier's host rows stream through two device buffers of
    // `chunk_rows` rows on their own copy stream: chunk j is copied into
    // buffer j % 2 while chunk j - 1 is absorbed from the other (allocated on
    // first use; the alternation carries over between absorb calls)
    u64 *rbuf[2] = {};
    u64 chunk_rows = 0;
    int next_buf = 0;
    cudaStream_t rcopy = nullptr;
    cudaEvent_t copied[2] = {}, absorbed[2] = {};
    cudaEvent_t call_copied[2] = {};  // absorb call k's last copy: call_copied[k % 2]
    u64 ncalls = 0;
};

namespace {

u64 h_pow(u64 b, u64 e)
{
    u64 r = 1;
    while (e) {
        if (e & 1) r = h_mul(r, b);
        b = h_mul(b, b);
        e >>= 1;
    }
    return r;
}

u64 h_inv(u64 a) { return h_pow(a, FP_P - 2); }

// The factors of h for the prime-factor transform: pairwise coprime prime
// powers, each a divisor of p - 1 and at most 61 (so that a length-q DFT sums
// at most 61 exact products in 128 bits).  False if h has another factor.
bool sp_factor(u64 h, std::vector<u32> &q)
{
    static const u32 primes[] = {3, 5, 7, 11, 13, 31, 41, 61};
    q.clear();
    for (u32 pr : primes) {
        u32 pp = 1;
        while (h % pr == 0) {
            h /= pr;
            pp *= pr;
        }
        if (pp > 1) {
            if (pp > 61 || (FP_P - 1) % pp != 0) return false;
            q.push_back(pp);
        }
    }
    return h == 1 && q.size() <= 8;
}

}  // namespace

static vc_status sp_status(vc_f2sp *s, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(s->h_res, s->res, 4 * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res + 4, s->status, sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    const u32 stv = (u32)(s->h_res[4] & 0xFFFFFFFFu);
    if (stv) {
        cudaMemsetAsync(s->status, 0, sizeof(u32), st);
        cudaStreamSynchronize(st);
        return VC_EINVAL;
    }
    return VC_OK;
}

extern "C" vc_status vc_f2sp_create(uint64_t v, uint64_t h, int device, vc_f2sp **out)
{
    if (!out) return VC_EINVAL;
    *out = nullptr;
    std::vector<u32> q;
    if (v < 1 || h < 1 || h > VC_F2SP_MAX_H || v > (uint64_t(1) << 40) / h || (FP_P - 1) % (2 * h) != 0 ||
        !sp_factor(h, q))
        return VC_EINVAL;
    DevGuard guard(device);
    init_device_once(device);
    vc_f2sp *s = new (std::nothrow) vc_f2sp();
    if (!s) return VC_ENOMEM;
    s->device = device;
    s->v = v;
    s->h = h;
    // the transform's geometry: dimension d has size q[d]; slot = sum of
    // digit_d stride_d, the last dimension innermost
    const u32 m = (u32)q.size();
    std::vector<u32> stride(m), N(m), t(m);
    u32 nroots = 0;
    for (int d = (int)m - 1; d >= 0; d--) stride[d] = (d == (int)m - 1) ? 1 : stride[d + 1] * q[d + 1];
    SpFftHost &F = s->F;
    F.h = (u32)h;
    F.m = m;
    for (u32 d = 0; d < m; d++) {
        N[d] = (u32)(h / q[d]);
        t[d] = 0;
        while ((u64)N[d] * t[d] % q[d] != 1 % q[d]) t[d]++;  // (h / q_d)^{-1} mod q_d
        F.q[d] = q[d];
        F.magic[d] = ((1u << 20) + q[d] - 1) / q[d];
        F.twoff[d] = nroots;
        nroots += q[d];
    }
    F.nroots = nroots;
    s->nparts = sp_prove_ctas(v);
    const u64 n2 = 2 * h;
    u32 *d_pin = nullptr, *d_perm = nullptr, *d_idx = nullptr;
    u64 *d_fw = nullptr, *d_bw = nullptr, *d_twist = nullptr;
    auto carve = [&](Arena &A) {
        d_pin = A.take<u32>(h);
        d_perm = A.take<u32>(h);
        d_idx = A.take<u32>(h);
        d_twist = A.take<u64>(h);
        d_fw = A.take<u64>(nroots + 1);
        d_bw = A.take<u64>(nroots + 1);
        s->pw = A.take<u64>(n2);
        s->L = A.take<u64>(h);
        s->M = A.take<u64>(n2);
        s->acc = A.take<u64>(v);
        s->part = A.take<u64>((u64)s->nparts * n2);
        s->proof = A.take<u64>(n2);
        s->res = A.take<u64>(4);
        s->status = A.take<u32>(1);
    };
    Arena A0;
    carve(A0);
    cudaError_t e = lib_malloc(&s->mem, A0.off);
    if (e == cudaSuccess) {
        Arena A;
        A.base = reinterpret_cast<uintptr_t>(s->mem);
        carve(A);
        e = cudaMemset(s->mem, 0, A0.off);
    }
    if (e == cudaSuccess) {
        // tables (exact host arithmetic): u generates the subgroup of order
        // 2h, w = u^2 the one of order h; root of dimension d = w^{h / q_d}
        const u64 u = h_pow(37, (FP_P - 1) / n2), w = h_mul(u, u);
        s->inv_h = h_inv(h);
        std::vector<u64> pw(n2), fw(nroots + 1, 0), bw(nroots + 1, 0), twist(h);
        std::vector<u32> pin(h), perm(h), idx(h);
        u64 tpow = 1;
        for (u64 k = 0; k < n2; k++, tpow = h_mul(tpow, u)) pw[k] = tpow;
        for (u32 d = 0; d < m; d++) {
            const u64 root = h_pow(w, N[d]), iroot = h_inv(root);
            u64 f = 1, b = 1;
            for (u32 e2 = 0; e2 < q[d]; e2++, f = h_mul(f, root), b = h_mul(b, iroot)) {
                fw[F.twoff[d] + e2] = f;
                bw[F.twoff[d] + e2] = b;
            }
        }
        auto slot_of_input = [&](u64 y) {  // digits y t_d mod q_d
            u64 p = 0;
            for (u32 d = 0; d < m; d++) p += ((y * t[d]) % q[d]) * stride[d];
            return (u32)p;
        };
        for (u64 y = 0; y < h; y++) pin[y] = slot_of_input(y);
        for (u64 P = 0; P < h; P++) {  // output slot: digits k_d = j mod q_d; j by CRT
            u64 j = 0;
            for (u32 d = 0; d < m; d++) {
                const u64 kd = (P / stride[d]) % q[d];
                j = (j + kd * N[d] % h * t[d]) % h;
            }
            idx[P] = (u32)j;
            perm[P] = slot_of_input(j);
            twist[P] = h_mul(pw[j], s->inv_h);
        }
        e = upload(d_pin, pin);
        if (e == cudaSuccess) e = upload(d_perm, perm);
        if (e == cudaSuccess) e = upload(d_idx, idx);
        if (e == cudaSuccess) e = upload(d_twist, twist);
        if (e == cudaSuccess) e = upload(d_fw, fw);
        if (e == cudaSuccess) e = upload(d_bw, bw);
        if (e == cudaSuccess) e = upload(s->pw, pw);
        F.fw = d_fw;
        F.bw = d_bw;
        F.pin = d_pin;
        F.perm = d_perm;
        F.idx = d_idx;
        F.twist = d_twist;
    }
    if (e == cudaSuccess) e = lib_host_alloc(&s->h_res, 8 * sizeof(u64), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->mem) lib_free(s->mem);
        if (s->h_res) lib_free_host(s->h_res);
        delete s;
        return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA;
    }
    *out = s;
    return VC_OK;
}

extern "C" vc_status vc_f2sp_destroy(vc_f2sp *s)
{
    if (!s) return VC_OK;
    DevGuard guard(s->device);
    cudaDeviceSynchronize();
    if (s->mem) lib_free(s->mem);
    if (s->a_stage) lib_free(s->a_stage);
    if (s->h_res) lib_free_host(s->h_res);
    for (int b = 0; b < 2; b++) {
        if (s->rbuf[b]) lib_free(s->rbuf[b]);
        if (s->copied[b]) cudaEventDestroy(s->copied[b]);
        if (s->absorbed[b]) cudaEventDestroy(s->absorbed[b]);
        if (s->call_copied[b]) cudaEventDestroy(s->call_copied[b]);
    }
    if (s->rcopy) cudaStreamDestroy(s->rcopy);
    delete s;
    return VC_OK;
}

// Rows per streaming chunk: about 8 MB, whole rows, at most v.
#ifndef SP_CHUNK_LOG
#define SP_CHUNK_LOG 21  // streaming chunks of about 2^SP_CHUNK_LOG entries (16 MB)
#endif
static u64 sp_chunk_rows(u64 v, u64 h)
{
    const u64 rows = std::max<u64>(1, (u64(1) << SP_CHUNK_LOG) / h);
    return std::min(rows, v);
}

static vc_status sp_stream_prepare(vc_f2sp *s)
{
    if (s->rcopy) return VC_OK;
    const u64 rows = sp_chunk_rows(s->v, s->h);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; b++) e = lib_malloc((void **)&s->rbuf[b], rows * s->h * sizeof(u64));
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        e = cudaEventCreateWithFlags(&s->copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->absorbed[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->call_copied[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->rcopy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (int b = 0; b < 2; b++) {
            if (s->rbuf[b]) lib_free(s->rbuf[b]);
            if (s->copied[b]) cudaEventDestroy(s->copied[b]);
            if (s->absorbed[b]) cudaEventDestroy(s->absorbed[b]);
            if (s->call_copied[b]) cudaEventDestroy(s->call_copied[b]);
            s->rbuf[b] = nullptr;
            s->copied[b] = s->absorbed[b] = s->call_copied[b] = nullptr;
        }
        s->rcopy = nullptr;
        return e == cudaErrorMemoryAllocation ? VC_ENOMEM : VC_ECUDA;
    }
    s->chunk_rows = rows;
    return VC_OK;
}

// Device copy of n u64 at p: p itself, or the staging buffer after a copy.
static const u64 *sp_device_input(vc_f2sp *s, const uint64_t *p, u64 n, cudaStream_t st, vc_status *err)
{
    *err = VC_OK;
    const int k = ptr_kind(p, s->device);
    if (k < 0) {
        *err = VC_EINVAL;
        return nullptr;
    }
    if (k == 1) return p;
    if (!s->a_stage && lib_malloc(&s->a_stage, s->v * s->h * sizeof(u64)) != cudaSuccess) {
        cudaGetLastError();
        s->a_stage = nullptr;
        *err = VC_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(s->a_stage, p, n * sizeof(u64), cudaMemcpyDefault, st) != cudaSuccess) {
        *err = VC_ECUDA;
        return nullptr;
    }
    return s->a_stage;
}

extern "C" vc_status vc_f2sp_prove(vc_f2sp *s, const uint64_t *a, uint64_t *proof, void *stream)
{
    if (!s || !a || !proof) return VC_EINVAL;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ptr_kind(proof, s->device) < 0) return VC_EINVAL;
    vc_status err;
    const u64 *da = sp_device_input(s, a, s->v * s->h, st, &err);
    if (!da) return err;
    launch_sp_prove(da, s->v, s->F, s->part, s->nparts, s->proof, s->status, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(proof, s->proof, 2 * s->h * sizeof(u64), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_status(e);
    return sp_status(s, st);
}

extern "C" vc_status vc_f2sp_verify_begin(vc_f2sp *s, uint64_t seed, void *stream)
{
    if (!s) return VC_EINVAL;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    launch_sp_vbegin(seed, s->v, s->h, s->inv_h, s->pw, s->L, s->M, s->acc, s->res, st);
    return cuda_status(cudaGetLastError());
}

// One absorb call.  Host rows: returns once the rows of this call (wait_own)
// or of the previous call (otherwise) have been copied to the device.
static vc_status sp_absorb(vc_f2sp *s, const uint64_t *rows, uint64_t first_row, uint64_t nrows, void *stream,
                           bool wait_own)
{
    if (!s || !rows || first_row > s->v || nrows > s->v - first_row) return VC_EINVAL;
    if (nrows == 0) return VC_OK;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int k = ptr_kind(rows, s->device);
    if (k < 0) return VC_EINVAL;
    if (k == 1) {
        launch_sp_vabsorb(rows, first_row, nrows, s->h, s->L, s->acc, s->status, st);
        return cuda_status(cudaGetLastError());
    }
    // host rows: double-buffered (Sec. 4.2): the copy of each chunk waits
    // only for the absorb that last read its buffer, so it overlaps the
    // absorb of the chunk before it
    const vc_status ps = sp_stream_prepare(s);
    if (ps != VC_OK) return ps;
    const u64 h = s->h;
    cudaError_t e = cudaSuccess;
    for (u64 r = 0; r < nrows && e == cudaSuccess; r += s->chunk_rows) {
        const u64 m = std::min(s->chunk_rows, nrows - r);
        const int b = s->next_buf;
        s->next_buf ^= 1;
        e = cudaStreamWaitEvent(s->rcopy, s->absorbed[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->rbuf[b], rows + r * h, m * h * sizeof(u64), cudaMemcpyHostToDevice, s->rcopy);
        if (e == cudaSuccess) e = cudaEventRecord(s->copied[b], s->rcopy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->copied[b], 0);
        if (e == cudaSuccess) {
            launch_sp_vabsorb(s->rbuf[b], first_row + r, m, h, s->L, s->acc, s->status, st);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->absorbed[b], st);
    }
    // the rows have been read when the call's last copy is done: the caller
    // may refill that buffer then while the absorbs run on
    const u64 call = s->ncalls++;
    if (e == cudaSuccess) e = cudaEventRecord(s->call_copied[call & 1], s->rcopy);
    if (e == cudaSuccess && wait_own) e = cudaEventSynchronize(s->call_copied[call & 1]);
    if (e == cudaSuccess && !wait_own && call > 0) e = cudaEventSynchronize(s->call_copied[(call - 1) & 1]);
    return cuda_status(e);
}

extern "C" vc_status vc_f2sp_verify_absorb(vc_f2sp *s, const uint64_t *rows, uint64_t first_row, uint64_t nrows,
                                           void *stream)
{
    return sp_absorb(s, rows, first_row, nrows, stream, true);
}

extern "C" vc_status vc_f2sp_verify_absorb_async(vc_f2sp *s, const uint64_t *rows, uint64_t first_row,
                                                 uint64_t nrows, void *stream)
{
    return sp_absorb(s, rows, first_row, nrows, stream, false);
}

extern "C" vc_status vc_f2sp_verify_end(vc_f2sp *s, const uint64_t *proof, uint64_t *f2, int *accept, void *stream)
{
    if (!s || !proof || !f2 || !accept) return VC_EINVAL;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    const u64 n2 = 2 * s->h;
    const int kp = ptr_kind(proof, s->device);
    if (kp < 0) return VC_EINVAL;
    cudaError_t e = cudaSuccess;
    const u64 *dp = proof;
    if (kp == 0) {
        e = cudaMemcpyAsync(s->proof, proof, n2 * sizeof(u64), cudaMemcpyHostToDevice, st);
        dp = s->proof;
    }
    if (e == cudaSuccess) {
        launch_sp_vend(dp, s->v, s->h, s->M, s->acc, s->res, st);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_status(e);
    const vc_status r = sp_status(s, st);
    if (r != VC_OK) return r;
    *accept = (int)s->h_res[0];
    *f2 = s->h_res[1];
    return VC_OK;
}
