// noalloc.cu -- circuit evaluation that allocates no device memory.
//
// For callers that cannot call cudaMalloc: for example a process whose device
// memory is already reserved in full by another framework's caching
// allocator, or code that must not trigger the device-wide synchronisation
// that cudaMalloc/cudaFree can cause.  The caller passes the circuit shape,
// the inputs and the outputs; the intermediate layers go to a fixed array in
// device memory that this file declares, so nothing is allocated per call.
#include <cuda_runtime.h>

#include <mutex>

#include "field.cuh"
#include "vc.h"

unsigned grid_for_items(u64 n, unsigned threads, unsigned per_sm);  // k_misc.cu

// Intermediate-layer capacity in field elements (8 MiB), plus one status slot.
#define NOALLOC_MAX_VALUES (1u << 20)

static __device__ __align__(256) u64 g_noalloc_scratch[NOALLOC_MAX_VALUES + 32];

namespace {

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current.  In host code the array's name only stands in
// for the symbol; a kernel must receive the address found here.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
u64 *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int device, u64 **out)
{
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<u64 *>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

bool shape_fits(u32 kind, u32 si, u32 sn)
{
    switch (kind) {
    case VC_WIRE_SQUARE: return si == sn;
    case VC_WIRE_TREE: return sn == si + 1;
    case VC_WIRE_MATMULT: return si % 3 == 0 && sn == 2 * (si / 3) + 1;
    case VC_WIRE_F0_FIRST: return si == sn + 1;
    case VC_WIRE_F0_PAIR: return si == sn && si >= 1;
    case VC_WIRE_F0_FINAL: return sn == si + 1;
    default: return false;  // explicit wiring needs device copies of its arrays
    }
}

}  // namespace

// One layer of a structured-wiring circuit: V[g] = Vn[in1(g)] op Vn[in2(g)].
__global__ void __launch_bounds__(256) k_eval_noalloc(u32 kind, u32 s, const u64 *Vn, u64 *V)
{
    const u64 S = 1ull << s;
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < S; g += (u64)gridDim.x * blockDim.x) {
        u64 a, b;
        bool mul = true;
        switch (kind) {
        case VC_WIRE_SQUARE: a = g; b = g; break;
        case VC_WIRE_TREE: a = 2 * g; b = 2 * g + 1; mul = false; break;
        case VC_WIRE_MATMULT: {
            const u32 L = s / 3;
            const u64 m = (1ull << L) - 1;
            const u64 k = g & m, j = (g >> L) & m, i = g >> (2 * L);
            a = (i << L) | k;
            b = (1ull << (2 * L)) | (k << L) | j;
            break;
        }
        case VC_WIRE_F0_FIRST: a = g >> 1; b = g >> 1; mul = (g & 1) == 0; break;
        case VC_WIRE_F0_PAIR: a = g; b = g & ~1ull; break;
        default: a = 2 * g + 1; b = 2 * g + 1; break;  // VC_WIRE_F0_FINAL
        }
        const u64 x = Vn[a], y = Vn[b];
        V[g] = mul ? f_mul(x, y) : f_add(x, y);
    }
}

__global__ void k_noalloc_check(const u64 *x, u64 n, u64 *status)
{
    bool bad = false;
    for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x)
        bad |= (x[k] >= FP_P);
    if (bad) atomicOr(reinterpret_cast<unsigned long long *>(status), 1ull);
}

static unsigned grid_for(u64 n) { return grid_for_items(n, 256, 16); }

extern "C" vc_status vc_evaluate_noalloc(const vc_circuit_desc *desc, const uint64_t *inputs, uint64_t *outputs,
                                         void *stream)
{
    if (!desc || !inputs || !outputs || !desc->log_width || !desc->wiring) return VC_EINVAL;
    const u32 d = desc->n_layers;
    if (d < 1 || d > 4096) return VC_EINVAL;
    u64 need = 0;
    for (u32 i = 0; i <= d; i++)
        if (desc->log_width[i] > 30) return VC_EINVAL;
    for (u32 i = 0; i < d; i++) {
        if (!shape_fits(desc->wiring[i], desc->log_width[i], desc->log_width[i + 1])) return VC_EINVAL;
        if (i >= 1) need += 1ull << desc->log_width[i];
    }
    if (need > NOALLOC_MAX_VALUES) return VC_EINVAL;  // intermediate layers exceed the fixed array

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return VC_ECUDA;
    // an error left pending by other code stays for its owner to read; the
    // error checks below then see only this call's own calls and launches
    if (cudaPeekAtLastError() != cudaSuccess) return VC_ECUDA;
    for (const void *p : {static_cast<const void *>(inputs), static_cast<const void *>(outputs)}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return VC_EINVAL;
        }
        if (a.type != cudaMemoryTypeDevice || a.device != device) return VC_EINVAL;
    }
    u64 *scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return VC_ECUDA;
    u64 *status = scratch + NOALLOC_MAX_VALUES;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The array keeps the previous call's contents: the status slot must start at 0.
    if (cudaMemsetAsync(status, 0, sizeof(u64), st) != cudaSuccess) return VC_ECUDA;
    const u64 nin = 1ull << desc->log_width[d];
    k_noalloc_check<<<grid_for(nin), 256, 0, st>>>(inputs, nin, status);
    // Layer i+1 lives at scratch + off(i+1); layer d is the caller's inputs,
    // layer 0 the caller's outputs.
    u64 off_next = need;
    const u64 *src = inputs;
    for (int i = (int)d - 1; i >= 0; i--) {
        u64 *dst;
        if (i == 0) {
            dst = outputs;
        } else {
            off_next -= 1ull << desc->log_width[i];
            dst = scratch + off_next;
        }
        k_eval_noalloc<<<grid_for(1ull << desc->log_width[i]), 256, 0, st>>>(desc->wiring[i], desc->log_width[i],
                                                                             src, dst);
        src = dst;
    }
    if (cudaGetLastError() != cudaSuccess) return VC_ECUDA;
    u64 h_status = 0;
    if (cudaMemcpyAsync(&h_status, status, sizeof(u64), cudaMemcpyDeviceToHost, st) != cudaSuccess) return VC_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return VC_ECUDA;
    return h_status ? VC_EINVAL : VC_OK;
}
