// tetra_dos_noalloc: tetra_dos without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// DOS: code that runs under a host framework which owns every device
// allocation through its own pool and forbids raw cudaMalloc, code with a hard
// device-memory budget fixed before it starts, or a latency-sensitive loop in
// which a cudaMalloc / cudaFree (which may synchronise the device) is not
// acceptable. For them this entry point takes the kernel's scratch memory from
// a fixed array that is part of the library image instead of from a workspace
// argument. The caller still passes inputs and outputs.
#include <mutex>

#include <cudaTypedefs.h>

#include "tetra_internal.cuh"

namespace tetra {

namespace {

// Scratch of the allocation-free entry point: the status words and the int64
// per-CTA partial DOS of tetra_dos. It is a static device array, so every GPU
// that loads libtetra holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the array's device address and the context it was looked up in.
// A device reset destroys the context (and the address with it); the next
// call sees a different current context and looks the address up again.
void *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

PFN_cuCtxGetCurrent_v4000 ctx_fn() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    });
    return fn;
}

// Device address of the scratch array on `device`, which the caller has made
// current with cudaSetDevice (so its primary context is current).
// In host code the array's name only stands for the device symbol, so the
// address is fetched with cudaGetSymbolAddress, once per device and context.
// `lookup` false: return the cached address only (nullptr if none).
tetra_status_t scratch_address(int device, void **ptr, bool lookup) {
    if (device < 0 || device >= kMaxDevices) return TETRA_EUNSUPPORTED;
    CUcontext ctx = nullptr;
    auto fn = ctx_fn();
    if (!fn || fn(&ctx) != CUDA_SUCCESS || !ctx) return TETRA_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[device] || g_scratch_ctx[device] != ctx) {
        g_scratch_ptr[device] = nullptr;
        if (!lookup) {
            *ptr = nullptr;
            return TETRA_OK;
        }
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TETRA_ECUDA;
        g_scratch_ptr[device] = p;
        g_scratch_ctx[device] = ctx;
    }
    *ptr = g_scratch_ptr[device];
    return TETRA_OK;
}

}  // namespace

}  // namespace tetra

extern "C" tetra_status_t tetra_dos_noalloc(tetra_plan_t plan, const float *eps, const void *w,
                                            const float *omega, float *dos, cudaStream_t stream) {
    if (!plan || !eps || !w || !omega || !dos) return TETRA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(eps) & 15u) || (reinterpret_cast<uintptr_t>(w) & 15u))
        return TETRA_EINVAL;
    // Same kernels as tetra_dos; only the number of persistent CTAs is lowered
    // when their int64 partials would not fit the fixed scratch. The result does
    // not depend on that number (exact integer accumulation).
    tetra::Plan q = *plan;
    while (q.grid_x > 1 && tetra::dos_forward_workspace(q) > tetra::kNoAllocScratchBytes) --q.grid_x;
    if (tetra::dos_forward_workspace(q) > tetra::kNoAllocScratchBytes) return TETRA_ENOMEM;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    void *scratch = nullptr;
    const tetra_status_t st = tetra::scratch_address(plan->device, &scratch, true);
    if (st != TETRA_OK) return st;
    return tetra::launch_dos_forward(q, eps, w, omega, dos, scratch, tetra::kNoAllocScratchBytes,
                                     stream);
}

extern "C" tetra_status_t tetra_noalloc_status(int device, cudaStream_t stream) {
    const tetra::DeviceGuard dg(device);
    if (!dg.ok()) return TETRA_ECUDA;
    void *scratch = nullptr;
    const tetra_status_t st = tetra::scratch_address(device, &scratch, false);
    if (st != TETRA_OK) return st;
    if (!scratch) return TETRA_OK;   // no tetra_dos_noalloc call on this device and context yet
    return tetra_workspace_status(scratch, stream);
}
