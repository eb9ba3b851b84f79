// Internal declarations shared by the libtetra translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include "../../include/tetra.h"

// ---------------------------------------------------------------- plan
// Host-side plan: the problem description and the launch geometry chosen for it.
struct tetra_plan_s {
    tetra_desc_t d;
    int device;
    int sm_count;
    size_t smem_optin;
    int z0, z1;                 // cube planes [z0, z1)
    int eps_stride, w_stride;   // elements per point
    int nx, ny, nz;             // padded extents
    int wbytes;                 // bytes per weight element
    // forward-kernel geometry
    int BX, BY, BZ;             // box of cubes
    int nbx, nby, nbz, n_boxes;
    int chunk_w, n_chunks;      // energy chunking of the shared-memory tile
    int grid_x;                 // persistent CTAs per energy chunk
    int threads;
    int fixed_bits;             // fixed-point fraction bits (see dos.cu)
    int flush_bits;             // a tile block is flushed once its bound reaches 2^flush_bits
    int items_per_box;          // work units per box: (pair, band) in point mode, (tetrahedron, band) in bin mode
    int tile_stride;            // ints per energy in the shared tile
    int tile_copies;            // copies of the tile (bin mode: lanes spread over them)
    size_t smem_bytes;
};

// Host-side plan of a batch of independent models evaluated by one launch of
// the forward kernel: per-model plans with a common box shape. The persistent
// CTAs take (model, box) work items from a global counter at run time.
namespace tetra {
constexpr int kMaxBatch = 64;
}  // namespace tetra
struct tetra_batch_plan_s {
    int n_models;
    int device;
    tetra_plan_s models[tetra::kMaxBatch];   // common box shape, one energy chunk each
    int big;                                 // model with the most energies
    int chunk_w;                             // energies per shared tile (= max n_omega)
    size_t smem_bytes;
    int grid_x;                              // persistent CTAs
    int total_boxes;                         // work items of the whole batch
    int box_base[tetra::kMaxBatch];          // first global work index of each model
};

namespace tetra {

// ---------------------------------------------------------------- status flags
// The first bytes of every workspace hold device-side status bits.
enum : int { kFlagTimeout = 1, kFlagRange = 2, kFlagConfig = 4 };
constexpr size_t kStatusBytes = 256;
constexpr size_t kQueueOffset = 64;   // batched launches: work counter inside the status bytes

using Plan = ::tetra_plan_s;

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for an mbarrier phase with a wall-clock limit. Returns false (and sets
// the timeout flag) when the limit passes; the caller then stops using the
// buffer the barrier guards.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            if (status) atomicOr(status, kFlagTimeout);
            return false;
        }
        __nanosleep(64);
    }
}

// 4-D tiled TMA load into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// NORB orbital weights of one (point, band) as FP32: 16-byte loads when a
// point's row fills whole vectors, scalars (zero beyond n_orb) otherwise.
template <int NORB, typename WT>
__device__ __forceinline__ void load_weights(const WT *src, int n_orb, float (&b)[NORB]) {
    constexpr int VEC = 16 / sizeof(WT);
    if (NORB % VEC == 0 && n_orb == NORB) {
#pragma unroll
        for (int v = 0; v < NORB / VEC; ++v) {
            const uint4 q = reinterpret_cast<const uint4 *>(src)[v];
            const WT *e = reinterpret_cast<const WT *>(&q);
#pragma unroll
            for (int j = 0; j < VEC; ++j) b[v * VEC + j] = to_f32<WT>(e[j]);
        }
    } else {
#pragma unroll
        for (int s = 0; s < NORB; ++s) b[s] = (s < n_orb) ? to_f32<WT>(src[s]) : 0.f;
    }
}

// ---------------------------------------------------------------- host helpers
// Makes `device` current for the lifetime of the guard and restores the
// caller's current device afterwards, so an entry point leaves the calling
// thread's device as it found it.
class DeviceGuard {
  public:
    // cudaSetDevice is called even when `device` is already current: it also
    // makes the device's primary context current on the calling thread.
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev_) != cudaSuccess) return;
        ok_ = cudaSetDevice(device) == cudaSuccess;
        switched_ = ok_ && prev_ != device;
    }
    ~DeviceGuard() {
        if (switched_) cudaSetDevice(prev_);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
    bool ok() const { return ok_; }

  private:
    int prev_ = 0;
    bool ok_ = false;
    bool switched_ = false;
};

tetra_status_t encode_point_map(CUtensorMap *map, const void *base, CUtensorMapDataType dtype,
                                int elem_bytes, int stride_elems, int nx, int ny, int nz,
                                int box_x, int box_y, int box_z);

int norb_template(int n_orb);

// Launchers implemented in dos.cu / eig.cu.
tetra_status_t launch_dos_forward(const Plan &P, const float *eps, const void *w,
                                  const float *omega, float *dos, void *ws, size_t ws_bytes,
                                  cudaStream_t stream);
size_t dos_forward_workspace(const Plan &P);
using BatchPlan = ::tetra_batch_plan_s;
tetra_status_t launch_dos_batched(const BatchPlan &B, const float *const *eps, const void *const *w,
                                  const float *const *omega, float *const *dos, void *ws,
                                  size_t ws_bytes, cudaStream_t stream);
size_t dos_batched_workspace(const BatchPlan &B);
tetra_status_t plan_init(Plan &P, const tetra_desc_t &d, int device, const int box[3], int ctas_per_sm);
void default_box(const tetra_desc_t &d, int box[3]);
tetra_status_t launch_dos_backward(const Plan &P, const float *eps, const void *w,
                                   const float *omega, const float *grad_dos, float *grad_eps,
                                   float *grad_w, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t dos_backward_workspace(const Plan &P);
tetra_status_t launch_eig(const Plan &P, const tetra_model_t *m, float *eps, void *w,
                          cudaStream_t stream);
tetra_status_t launch_pair_bands(const Plan &P, const float *eps, const int q[3], float kT, float mu,
                                 const Plan &Q, float *eps_p, float *w_p, cudaStream_t stream);
tetra_status_t launch_eig_backward(const Plan &P, const tetra_model_t *m, const float *geps,
                                   const float *gw, float *gparams, void *ws, size_t ws_bytes,
                                   cudaStream_t stream);
size_t eig_backward_workspace(const Plan &P, int n_R);

}  // namespace tetra
