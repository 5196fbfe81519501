// f2sp_api.cu -- C ABI of the special-purpose non-interactive F2 protocol
// (declarations and contracts in include/vc.h).
#include <cuda_runtime.h>

#include <new>

#include "internal.h"

struct vc_f2sp {
    int device = 0;
    u64 v = 0, h = 0;
    char *mem = nullptr;
    u64 *w = nullptr, *C = nullptr, *iv = nullptr, *w2 = nullptr;  // node tables
    u64 *L = nullptr, *M = nullptr, *acc = nullptr;                 // verifier state
    u64 *part = nullptr, *proof = nullptr, *res = nullptr;          // prover partials, staging, results
    u32 *status = nullptr;
    u64 *a_stage = nullptr;  // host inputs are staged here (allocated on first use)
    u64 *h_res = nullptr;    // pinned: results and status readback
};

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
    if (v < 1 || h < 1 || h > VC_F2SP_MAX_H || v > (uint64_t(1) << 40) / h) return VC_EINVAL;
    DevGuard guard(device);
    init_device_once(device);
    vc_f2sp *s = new (std::nothrow) vc_f2sp();
    if (!s) return VC_ENOMEM;
    s->device = device;
    s->v = v;
    s->h = h;
    const u64 n2 = 2 * h - 1, nc = sp_prove_ctas(v);
    auto carve = [&](Arena &A) {
        s->w = A.take<u64>(h);
        s->C = A.take<u64>(h);
        s->iv = A.take<u64>(n2);
        s->w2 = A.take<u64>(n2);
        s->L = A.take<u64>(h);
        s->M = A.take<u64>(n2);
        s->acc = A.take<u64>(v);
        s->part = A.take<u64>(nc * n2);
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
    if (e == cudaSuccess) e = lib_host_alloc(&s->h_res, 8 * sizeof(u64), cudaHostAllocDefault);
    if (e == cudaSuccess) {
        launch_sp_tables(h, s->w, s->C, s->iv, s->w2, 0);
        e = cudaDeviceSynchronize();
    }
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
    delete s;
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
    launch_sp_prove(da, s->v, s->h, s->w, s->C, s->iv, s->part, s->proof, s->status, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(proof, s->proof, (2 * s->h - 1) * sizeof(u64), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_status(e);
    return sp_status(s, st);
}

extern "C" vc_status vc_f2sp_verify_begin(vc_f2sp *s, uint64_t seed, void *stream)
{
    if (!s) return VC_EINVAL;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    launch_sp_vbegin(seed, s->v, s->h, s->w, s->w2, s->L, s->M, s->acc, s->res, st);
    return cuda_status(cudaGetLastError());
}

extern "C" vc_status vc_f2sp_verify_absorb(vc_f2sp *s, const uint64_t *rows, uint64_t first_row, uint64_t nrows,
                                           void *stream)
{
    if (!s || !rows || first_row > s->v || nrows > s->v - first_row) return VC_EINVAL;
    if (nrows == 0) return VC_OK;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    vc_status err;
    const u64 *dr = sp_device_input(s, rows, nrows * s->h, st, &err);
    if (!dr) return err;
    launch_sp_vabsorb(dr, first_row, nrows, s->h, s->L, s->acc, s->status, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && dr == s->a_stage) e = cudaStreamSynchronize(st);  // the stage is reused
    return cuda_status(e);
}

extern "C" vc_status vc_f2sp_verify_end(vc_f2sp *s, const uint64_t *proof, uint64_t *f2, int *accept, void *stream)
{
    if (!s || !proof || !f2 || !accept) return VC_EINVAL;
    DevGuard guard(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    const u64 n2 = 2 * s->h - 1;
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
