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

int pow2_floor(int v) {
    int p = 1;
    while (2 * p <= v) p *= 2;
    return p;
}

// Default box of cubes for a band count: 4 x 4 x BZ with at most ~1536 work
// items per box (a work item is a (tetrahedron pair, band) with up to 8
// orbitals, a (tetrahedron, band) with more), which keeps the per-item
// fixed-point cap of the int32 tile (2^30 / items) above typical values.
void default_box(const tetra_desc_t &d, int box[3]) {
    const bool pairs = tetra::norb_template(d.n_orb) <= 8;
    const int per_cube = (pairs ? 3 : 6) * std::max(1, d.n_bands);
    box[0] = env_int("TETRA_BOX_X", 4);
    box[1] = env_int("TETRA_BOX_Y", 4);
    box[2] = env_int("TETRA_BOX_Z", std::max(1, std::min(4, 1536 / (16 * per_cube))));
}

// Chooses the box shape, energy chunking and grid of the forward kernel. Box
// sides are powers of two (items are decoded with shifts), clipped to the grid.
static tetra_status_t plan_geometry(Plan &P, const int box[3], int ctas_per_sm) {
    const tetra_desc_t &d = P.d;
    P.BX = pow2_floor(std::max(1, std::min(box[0], d.n1)));
    P.BY = pow2_floor(std::max(1, std::min(box[1], d.n2)));
    P.BZ = pow2_floor(std::max(1, std::min(box[2], P.z1 - P.z0)));
    if (P.BX < 1 || P.BY < 1 || P.BZ < 1) return TETRA_EINVAL;
    P.nbx = (d.n1 + P.BX - 1) / P.BX;
    P.nby = (d.n2 + P.BY - 1) / P.BY;
    P.nbz = (P.z1 - P.z0 + P.BZ - 1) / P.BZ;
    P.n_boxes = P.nbx * P.nby * P.nbz;
    const size_t npts = (size_t)(P.BX + 1) * (P.BY + 1) * (P.BZ + 1);
    // TMA slots (128-byte multiples): two of a box's energies, one of its weights
    const size_t e_stage = (npts * P.eps_stride * 4 + 127) & ~size_t(127);
    const size_t w_stage = (npts * P.w_stride * P.wbytes + 127) & ~size_t(127);
    // up to 8 orbitals: one item per face-sharing tetrahedron pair (3 per
    // cube); more: one item per tetrahedron (6 per cube)
    const bool pairs = tetra::norb_template(d.n_orb) <= 8;
    P.items_per_box = (pairs ? 3 : 6) * P.BX * P.BY * P.BZ * d.n_bands;
    if (P.items_per_box > 65535) return TETRA_EUNSUPPORTED;
    P.tile_stride = tetra::norb_template(d.n_orb) + 1;
    // TMA slots, per-item sort arrays, length histogram and cursors, three
    // mbarriers, alignment slack, the kernel's static variables and the tile's
    // extra row
    const size_t fixed = 2 * e_stage + w_stage + 6 * (size_t)P.items_per_box + 16 + 2 * 256 * 4 + 40 + 1024 +
                         512 + 128 + 4 * (size_t)P.tile_stride;
    // per energy: int tile row, cached energy, 1/width (bin mode), block bound share
    // (integrated mode: plus a row of per-orbital step sums)
    const size_t per_w = 4 * (size_t)(P.tile_stride + 1 + (d.mode == TETRA_BIN ? 1 : 0) +
                                      (d.mode == TETRA_INTEGRATED ? P.tile_stride - 1 : 0)) + 1;
    if (fixed + per_w * 64 > P.smem_optin) return TETRA_EUNSUPPORTED;
    int cw = (int)std::min<size_t>((P.smem_optin - fixed - 8) / per_w, (size_t)d.n_omega);
    P.n_chunks = (d.n_omega + cw - 1) / cw;
    P.chunk_w = (d.n_omega + P.n_chunks - 1) / P.n_chunks;
    P.smem_bytes = fixed + per_w * P.chunk_w + 8;
    // Bin mode: neighbouring pairs of a band tend to fall into the same bin,
    // so a warp's tile adds hit the same addresses; up to 8 copies of the
    // tile (as shared memory allows), one per lane residue, spread them.
    // Each copy has its own block bounds (4 bytes per 64 energies).
    P.tile_copies = 1;
    if (d.mode == TETRA_BIN && pairs) {
        const size_t copy = 4 * (size_t)P.tile_stride * (P.chunk_w + 1) + 4 * (size_t)((P.chunk_w + 63) / 64);
        const size_t room = P.smem_optin > P.smem_bytes ? P.smem_optin - P.smem_bytes : 0;
        P.tile_copies = (int)std::min<size_t>(8, 1 + room / copy);
        P.smem_bytes += (size_t)(P.tile_copies - 1) * copy;
    }
    P.threads = pairs ? 384 : 512;
    const int ctas = std::max(1, ctas_per_sm) * P.sm_count;
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
        // integrated occupation: a tetrahedron's full weight V_T/V_G is 2^18
        // units (per-item rounding below 2e-6 of it, and a box's items stay
        // under the int32 tile's per-item cap)
        if (d.mode == TETRA_INTEGRATED) F = 18;
        P.fixed_bits = env_int("TETRA_FIXED_BITS", F);
    }
    // tile blocks are flushed at a bound of 2^30 (a lower value, for tests of
    // the flush path, from TETRA_FLUSH_BITS)
    P.flush_bits = std::max(8, std::min(30, env_int("TETRA_FLUSH_BITS", 30)));
    return TETRA_OK;
}

// Validates a description and fills a plan for it (box shape given).
tetra_status_t plan_init(Plan &P, const tetra_desc_t &d, int device, const int box[3], int ctas_per_sm) {
    if (d.n1 < 1 || d.n2 < 1 || d.n3 < 1 || d.n1 > 4096 || d.n2 > 4096 || d.n3 > 4096)
        return TETRA_EINVAL;
    if (d.n_bands < 1 || d.n_bands > 64 || d.n_orb < 1 || d.n_orb > 16 || d.n_omega < 1)
        return TETRA_EINVAL;
    if (d.mode != TETRA_POINT && d.mode != TETRA_BIN && d.mode != TETRA_INTEGRATED) return TETRA_EINVAL;
    if (d.weight_dtype != TETRA_F32 && d.weight_dtype != TETRA_F16 && d.weight_dtype != TETRA_BF16)
        return TETRA_EINVAL;
    int z0 = d.z_begin, z1 = d.z_end;
    if (z0 == 0 && z1 == 0) z1 = d.n3;
    if (z0 < 0 || z1 > d.n3 || z0 >= z1) return TETRA_EINVAL;
    P = Plan();
    P.d = d;
    P.device = device;
    P.z0 = z0;
    P.z1 = z1;
    P.nx = d.n1 + 1;
    P.ny = d.n2 + 1;
    P.nz = d.n3 + 1;
    P.wbytes = d.weight_dtype == TETRA_F32 ? 4 : 2;
    P.eps_stride = round_up(d.n_bands, 4);
    const int align = 16 / P.wbytes;
    int ws = round_up(d.n_bands * d.n_orb, align);
    if ((ws * P.wbytes) % 128 == 0) ws += align;   // spread points over smem banks
    P.w_stride = ws;
    if (P.w_stride > 256 || P.eps_stride > 256) return TETRA_EUNSUPPORTED;
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return TETRA_ECUDA;
    P.sm_count = sms;
    P.smem_optin = (size_t)optin;
    return plan_geometry(P, box, ctas_per_sm);
}

}  // namespace tetra

using tetra::Plan;

extern "C" {

tetra_status_t tetra_plan(tetra_plan_t *plan, const tetra_desc_t *desc, int device) {
    if (!plan || !desc) return TETRA_EINVAL;
    *plan = nullptr;
    int box[3];
    tetra::default_box(*desc, box);
    Plan *P = new (std::nothrow) Plan();
    if (!P) return TETRA_ENOMEM;
    tetra_status_t st = tetra::plan_init(*P, *desc, device, box, tetra::env_int("TETRA_CTAS_PER_SM", 1));
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
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_dos_forward(*plan, eps, w, omega, dos, ws, ws_bytes, stream);
}

tetra_status_t tetra_dos_backward(tetra_plan_t plan, const float *eps, const void *w,
                                  const float *omega, const float *grad_dos, float *grad_eps,
                                  float *grad_w, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !eps || !w || !omega || !grad_dos || !grad_eps || !grad_w || !ws) return TETRA_EINVAL;
    if (plan->d.mode != TETRA_BIN) return TETRA_EUNSUPPORTED;
    if (!tetra::aligned16(eps) || !tetra::aligned16(w) || !tetra::aligned16(ws)) return TETRA_EINVAL;
    if (ws_bytes < tetra::dos_backward_workspace(*plan)) return TETRA_ENOMEM;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_dos_backward(*plan, eps, w, omega, grad_dos, grad_eps, grad_w, ws,
                                      ws_bytes, stream);
}

tetra_status_t tetra_eig(tetra_plan_t plan, const tetra_model_t *model, float *eps, void *w,
                         cudaStream_t stream) {
    if (!plan || !model || !eps || !w) return TETRA_EINVAL;
    if (!tetra::aligned16(eps) || !tetra::aligned16(w)) return TETRA_EINVAL;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
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
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_eig_backward(*plan, model, grad_eps, grad_w, grad_params, ws, ws_bytes,
                                      stream);
}

tetra_status_t tetra_plan_batched(tetra_batch_plan_t *plan, const tetra_desc_t *descs, int n_models,
                                  const tetra_tune_t *tune, int device) {
    if (!plan || !descs) return TETRA_EINVAL;
    *plan = nullptr;
    if (n_models < 1 || n_models > tetra::kMaxBatch) return TETRA_EINVAL;
    const tetra_desc_t &d0 = descs[0];
    if (d0.mode == TETRA_INTEGRATED) return TETRA_EUNSUPPORTED;   // single-model plans only
    for (int m = 1; m < n_models; ++m) {
        const tetra_desc_t &d = descs[m];
        if (d.n_bands != d0.n_bands || d.n_orb != d0.n_orb || d.mode != d0.mode ||
            d.weight_dtype != d0.weight_dtype)
            return TETRA_EINVAL;
    }
    tetra_tune_t t = {0, 0, 0, 0};
    if (tune) t = *tune;
    int box[3];
    tetra::default_box(d0, box);
    if (t.box_x > 0) box[0] = t.box_x;
    if (t.box_y > 0) box[1] = t.box_y;
    if (t.box_z > 0) box[2] = t.box_z;
    // one box shape for the whole batch: clipped to the smallest grid
    for (int m = 0; m < n_models; ++m) {
        const tetra_desc_t &d = descs[m];
        if (d.n1 < 1 || d.n2 < 1 || d.n3 < 1) return TETRA_EINVAL;
        const int zb = d.z_begin, ze = (d.z_begin == 0 && d.z_end == 0) ? d.n3 : d.z_end;
        box[0] = std::min(box[0], d.n1);
        box[1] = std::min(box[1], d.n2);
        box[2] = std::min(box[2], std::max(1, ze - zb));
    }
    for (int i = 0; i < 3; ++i) box[i] = tetra::pow2_floor(std::max(1, box[i]));
    const int ctas_per_sm = t.ctas_per_sm > 0 ? t.ctas_per_sm : 1;
    tetra_batch_plan_s *B = new (std::nothrow) tetra_batch_plan_s();
    if (!B) return TETRA_ENOMEM;
    auto fail = [&](tetra_status_t s) {
        delete B;
        return s;
    };
    B->n_models = n_models;
    B->device = device;
    B->big = 0;
    for (int m = 0; m < n_models; ++m) {
        tetra_status_t st = tetra::plan_init(B->models[m], descs[m], device, box, ctas_per_sm);
        if (st != TETRA_OK) return fail(st);
        if (descs[m].n_omega > descs[B->big].n_omega) B->big = m;
    }
    // the largest energy grid must fit one shared tile (no energy chunks)
    const Plan &Pb = B->models[B->big];
    if (Pb.n_chunks != 1) return fail(TETRA_EUNSUPPORTED);
    B->chunk_w = Pb.chunk_w;
    B->smem_bytes = Pb.smem_bytes;
    // work items: every box of every model, models in order; the CTAs claim
    // them at run time
    long total = 0;
    for (int m = 0; m < n_models; ++m) {
        B->box_base[m] = (int)total;
        total += B->models[m].n_boxes;
        if (total > (1L << 30)) return fail(TETRA_EUNSUPPORTED);
    }
    B->total_boxes = (int)total;
    B->grid_x = (int)std::max<long>(1, std::min<long>(total, (long)ctas_per_sm * Pb.sm_count));
    *plan = B;
    return TETRA_OK;
}

tetra_status_t tetra_batch_plan_destroy(tetra_batch_plan_t plan) {
    delete plan;
    return TETRA_OK;
}

tetra_status_t tetra_batch_layout(tetra_batch_plan_t plan, int model, tetra_layout_t *layout) {
    if (!plan || model < 0 || model >= plan->n_models) return TETRA_EINVAL;
    return tetra_layout(&plan->models[model], layout);
}

size_t tetra_batch_workspace_bytes(tetra_batch_plan_t plan) {
    if (!plan) return 0;
    return tetra::dos_batched_workspace(*plan);
}

tetra_status_t tetra_batch_info(tetra_batch_plan_t plan, int *box, int *grid, int *n_slots) {
    if (!plan) return TETRA_EINVAL;
    if (box) {
        box[0] = plan->models[0].BX;
        box[1] = plan->models[0].BY;
        box[2] = plan->models[0].BZ;
    }
    if (grid) *grid = plan->grid_x;
    if (n_slots) *n_slots = plan->n_models;
    return TETRA_OK;
}

tetra_status_t tetra_dos_batched(tetra_batch_plan_t plan, const float *const *eps, const void *const *w,
                                 const float *const *omega, float *const *dos, void *ws,
                                 size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !eps || !w || !omega || !dos || !ws) return TETRA_EINVAL;
    if (!tetra::aligned16(ws)) return TETRA_EINVAL;
    for (int m = 0; m < plan->n_models; ++m) {
        if (!eps[m] || !w[m] || !omega[m] || !dos[m]) return TETRA_EINVAL;
        if (!tetra::aligned16(eps[m]) || !tetra::aligned16(w[m])) return TETRA_EINVAL;
    }
    if (ws_bytes < tetra::dos_batched_workspace(*plan)) return TETRA_ENOMEM;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_dos_batched(*plan, eps, w, omega, dos, ws, ws_bytes, stream);
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
