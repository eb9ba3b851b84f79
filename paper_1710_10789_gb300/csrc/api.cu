// C ABI of libtetra: plans, layouts, argument checks and dispatch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include <cudaTypedefs.h>

#include "tetra_internal.cuh"

namespace tetra {

namespace {

int round_up(int a, int m) { return (a + m - 1) / m * m; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int env_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

// 4-D map over a point-major array: dims (stride, nx, ny, nz); box
// (stride, box_x, box_y, box_z) so one load brings every band of a box of points.
tetra_status_t encode_point_map(CUtensorMap *map, const void *base, CUtensorMapDataType dtype,
                                int elem_bytes, int stride_elems, int nx, int ny, int nz,
                                int box_x, int box_y, int box_z) {
    auto fn = encode_fn();
    if (!fn) return TETRA_ECUDA;
    cuuint64_t dims[4] = {(cuuint64_t)stride_elems, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[3] = {(cuuint64_t)stride_elems * elem_bytes,
                             (cuuint64_t)stride_elems * elem_bytes * nx,
                             (cuuint64_t)stride_elems * elem_bytes * nx * ny};
    cuuint32_t box[4] = {(cuuint32_t)stride_elems, (cuuint32_t)std::min(box_x, nx),
                         (cuuint32_t)std::min(box_y, ny), (cuuint32_t)std::min(box_z, nz)};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(map, dtype, 4, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TETRA_OK : TETRA_EINVAL;
}

// Chooses the box shape, energy chunking and grid of the forward kernel.
static tetra_status_t plan_geometry(Plan &P) {
    const tetra_desc_t &d = P.d;
    // box sides are powers of two (items are decoded with shifts)
    auto pow2_floor = [](int v) { int p = 1; while (2 * p <= v) p *= 2; return p; };
    P.BX = pow2_floor(std::max(1, std::min(env_int("TETRA_BOX_X", 4), d.n1)));
    P.BY = pow2_floor(std::max(1, std::min(env_int("TETRA_BOX_Y", 4), d.n2)));
    // at most ~1536 (tetrahedron, band) items per box keeps the per-item
    // fixed-point cap of the int32 tile (2^30 / items) above typical values
    const int bz_default = std::max(1, std::min(4, 1536 / (96 * d.n_bands)));
    P.BZ = pow2_floor(std::max(1, std::min(env_int("TETRA_BOX_Z", bz_default), P.z1 - P.z0)));
    if (P.BX < 1 || P.BY < 1 || P.BZ < 1) return TETRA_EINVAL;
    P.nbx = (d.n1 + P.BX - 1) / P.BX;
    P.nby = (d.n2 + P.BY - 1) / P.BY;
    P.nbz = (P.z1 - P.z0 + P.BZ - 1) / P.BZ;
    P.n_boxes = P.nbx * P.nby * P.nbz;
    const size_t npts = (size_t)(P.BX + 1) * (P.BY + 1) * (P.BZ + 1);
    const size_t e_off = (npts * P.eps_stride * 4 + 127) & ~size_t(127);
    const size_t stage = (e_off + npts * P.w_stride * P.wbytes + 127) & ~size_t(127);
    P.items_per_box = 6 * P.BX * P.BY * P.BZ * d.n_bands;
    if (P.items_per_box > 65535) return TETRA_EUNSUPPORTED;
    P.tile_stride = tetra::norb_template(d.n_orb) + 1;
    // two TMA stages, per-item sort arrays, histogram, mbarriers, alignment
    // slack and the kernel's static variables
    const size_t n_classes = (P.items_per_box + 95) / 96;
    const size_t fixed = 2 * stage + 7 * (size_t)P.items_per_box + 16 + (2 * 256 + 64 * n_classes) * 4 + 32 +
                         1024 + 512 + 64;
    // per energy: int tile row, cached energy, 1/width (bin mode), block bound share
    const size_t per_w = 4 * (size_t)(P.tile_stride + 1 + (d.mode == TETRA_BIN ? 1 : 0)) + 1;
    if (fixed + per_w * 64 > P.smem_optin) return TETRA_EUNSUPPORTED;
    int cw = (int)std::min<size_t>((P.smem_optin - fixed - 8) / per_w, (size_t)d.n_omega);
    P.n_chunks = (d.n_omega + cw - 1) / cw;
    P.chunk_w = (d.n_omega + P.n_chunks - 1) / P.n_chunks;
    P.smem_bytes = fixed + per_w * P.chunk_w + 8;
    P.threads = 512;
    const int ctas = std::max(1, env_int("TETRA_CTAS_PER_SM", 1)) * P.sm_count;
    P.grid_x = std::max(1, std::min(P.n_boxes, (ctas + P.n_chunks - 1) / P.n_chunks));
    // Fixed-point fraction bits. A DOS value is a sum of N contributions of
    // size ~2^F / K units (K = energies per tetrahedron window), each rounded
    // with an unbiased dithered error below one unit, so its relative error is
    // about sqrt(K n_omega / n_items) / 2^(F+1). Take F so that this stays
    // below 5e-6 for the worst case K = n_omega; items whose bound exceeds the
    // int32 tile cap go through the exact 64-bit path instead.
    {
        const double items = 6.0 * d.n1 * d.n2 * (double)(P.z1 - P.z0) * d.n_bands;
        const double need = 1e5 * d.n_omega / std::sqrt(items);
        int F = (int)std::ceil(std::log2(std::max(need, 1.0)));
        F = std::max(17, std::min(28, F));
        P.fixed_bits = env_int("TETRA_FIXED_BITS", F);
    }
    return TETRA_OK;
}

}  // namespace tetra

using tetra::Plan;

extern "C" {

tetra_status_t tetra_plan(tetra_plan_t *plan, const tetra_desc_t *desc, int device) {
    if (!plan || !desc) return TETRA_EINVAL;
    *plan = nullptr;
    const tetra_desc_t &d = *desc;
    if (d.n1 < 1 || d.n2 < 1 || d.n3 < 1 || d.n1 > 4096 || d.n2 > 4096 || d.n3 > 4096)
        return TETRA_EINVAL;
    if (d.n_bands < 1 || d.n_bands > 64 || d.n_orb < 1 || d.n_orb > 16 || d.n_omega < 1)
        return TETRA_EINVAL;
    if (d.mode != TETRA_POINT && d.mode != TETRA_BIN) return TETRA_EINVAL;
    if (d.weight_dtype != TETRA_F32 && d.weight_dtype != TETRA_F16 && d.weight_dtype != TETRA_BF16)
        return TETRA_EINVAL;
    int z0 = d.z_begin, z1 = d.z_end;
    if (z0 == 0 && z1 == 0) z1 = d.n3;
    if (z0 < 0 || z1 > d.n3 || z0 >= z1) return TETRA_EINVAL;
    Plan *P = new (std::nothrow) Plan();
    if (!P) return TETRA_ENOMEM;
    P->d = d;
    P->device = device;
    P->z0 = z0;
    P->z1 = z1;
    P->nx = d.n1 + 1;
    P->ny = d.n2 + 1;
    P->nz = d.n3 + 1;
    P->wbytes = d.weight_dtype == TETRA_F32 ? 4 : 2;
    P->eps_stride = tetra::round_up(d.n_bands, 4);
    const int align = 16 / P->wbytes;
    int ws = tetra::round_up(d.n_bands * d.n_orb, align);
    if ((ws * P->wbytes) % 128 == 0) ws += align;   // spread points over smem banks
    P->w_stride = ws;
    if (P->w_stride > 256 || P->eps_stride > 256) {
        delete P;
        return TETRA_EUNSUPPORTED;
    }
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        delete P;
        return TETRA_ECUDA;
    }
    P->sm_count = sms;
    P->smem_optin = (size_t)optin;
    tetra_status_t st = tetra::plan_geometry(*P);
    if (st != TETRA_OK) {
        delete P;
        return st;
    }
    *plan = P;
    return TETRA_OK;
}

tetra_status_t tetra_plan_destroy(tetra_plan_t plan) {
    delete plan;
    return TETRA_OK;
}

tetra_status_t tetra_layout(tetra_plan_t plan, tetra_layout_t *L) {
    if (!plan || !L) return TETRA_EINVAL;
    L->nx = plan->nx;
    L->ny = plan->ny;
    L->nz = plan->nz;
    L->eps_stride = plan->eps_stride;
    L->w_stride = plan->w_stride;
    const size_t pts = (size_t)plan->nx * plan->ny * plan->nz;
    L->eps_elems = pts * plan->eps_stride;
    L->w_elems = pts * plan->w_stride;
    return TETRA_OK;
}

size_t tetra_workspace_bytes(tetra_plan_t plan) {
    if (!plan) return 0;
    size_t a = tetra::dos_forward_workspace(*plan);
    if (plan->d.mode == TETRA_BIN) a = std::max(a, tetra::dos_backward_workspace(*plan));
    return a;
}

tetra_status_t tetra_dos(tetra_plan_t plan, const float *eps, const void *w, const float *omega,
                         float *dos, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !eps || !w || !omega || !dos || !ws) return TETRA_EINVAL;
    if (!tetra::aligned16(eps) || !tetra::aligned16(w) || !tetra::aligned16(ws)) return TETRA_EINVAL;
    if (ws_bytes < tetra::dos_forward_workspace(*plan)) return TETRA_ENOMEM;
    if (cudaSetDevice(plan->device) != cudaSuccess) return TETRA_ECUDA;
    return tetra::launch_dos_forward(*plan, eps, w, omega, dos, ws, ws_bytes, stream);
}

tetra_status_t tetra_dos_backward(tetra_plan_t plan, const float *eps, const void *w,
                                  const float *omega, const float *grad_dos, float *grad_eps,
                                  float *grad_w, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !eps || !w || !omega || !grad_dos || !grad_eps || !grad_w || !ws) return TETRA_EINVAL;
    if (plan->d.mode != TETRA_BIN) return TETRA_EUNSUPPORTED;
    if (!tetra::aligned16(eps) || !tetra::aligned16(w) || !tetra::aligned16(ws)) return TETRA_EINVAL;
    if (ws_bytes < tetra::dos_backward_workspace(*plan)) return TETRA_ENOMEM;
    if (cudaSetDevice(plan->device) != cudaSuccess) return TETRA_ECUDA;
    return tetra::launch_dos_backward(*plan, eps, w, omega, grad_dos, grad_eps, grad_w, ws,
                                      ws_bytes, stream);
}

tetra_status_t tetra_eig(tetra_plan_t plan, const tetra_model_t *model, float *eps, void *w,
                         cudaStream_t stream) {
    if (!plan || !model || !eps || !w) return TETRA_EINVAL;
    if (!tetra::aligned16(eps) || !tetra::aligned16(w)) return TETRA_EINVAL;
    if (cudaSetDevice(plan->device) != cudaSuccess) return TETRA_ECUDA;
    return tetra::launch_eig(*plan, model, eps, w, stream);
}

size_t tetra_eig_workspace_bytes(tetra_plan_t plan, int n_R) {
    if (!plan) return 0;
    return tetra::eig_backward_workspace(*plan, n_R);
}

tetra_status_t tetra_eig_backward(tetra_plan_t plan, const tetra_model_t *model,
                                  const float *grad_eps, const float *grad_w, float *grad_params,
                                  void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !model || !grad_eps || !grad_w || !grad_params || !ws) return TETRA_EINVAL;
    if (!tetra::aligned16(ws)) return TETRA_EINVAL;
    if (ws_bytes < tetra::eig_backward_workspace(*plan, model->n_R)) return TETRA_ENOMEM;
    if (cudaSetDevice(plan->device) != cudaSuccess) return TETRA_ECUDA;
    return tetra::launch_eig_backward(*plan, model, grad_eps, grad_w, grad_params, ws, ws_bytes,
                                      stream);
}

tetra_status_t tetra_workspace_status(const void *ws, cudaStream_t stream) {
    if (!ws) return TETRA_EINVAL;
    int flags = 0;
    if (cudaMemcpyAsync(&flags, ws, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return TETRA_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return TETRA_ECUDA;
    if (flags & tetra::kFlagTimeout) return TETRA_ETIMEOUT;
    if (flags & tetra::kFlagRange) return TETRA_ERANGE;
    if (flags & tetra::kFlagConfig) return TETRA_ECUDA;
    return TETRA_OK;
}

const char *tetra_strerror(tetra_status_t s) {
    switch (s) {
        case TETRA_OK: return "TETRA_OK";
        case TETRA_EINVAL: return "TETRA_EINVAL: invalid argument";
        case TETRA_EUNSUPPORTED: return "TETRA_EUNSUPPORTED: not supported by this build";
        case TETRA_ECUDA: return "TETRA_ECUDA: CUDA runtime error";
        case TETRA_ENOMEM: return "TETRA_ENOMEM: workspace too small or allocation failed";
        case TETRA_ETIMEOUT: return "TETRA_ETIMEOUT: device wait hit its limit";
        case TETRA_ERANGE: return "TETRA_ERANGE: value outside the fixed-point range";
    }
    return "TETRA_UNKNOWN";
}

const char *tetra_version(void) { return "0.1.0"; }

}  // extern "C"
