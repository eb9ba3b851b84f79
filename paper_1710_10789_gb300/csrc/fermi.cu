// Fermi level from the integrated orbital occupation (TETRA_INTEGRATED mode of
// the forward kernel): bracketing by repeated 64-point evaluations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kFermiPoints = 64;

// Order-preserving map of a float to an unsigned int (for atomic min / max).
__device__ __forceinline__ unsigned ordered(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float unordered(unsigned u) {
    const unsigned v = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    float f;
    memcpy(&f, &v, sizeof f);
    return f;
}

// Minimum and maximum band energy over the plan's points (bands < nb).
__global__ void band_range_kernel(const float *eps, long n_pts, int stride, int nb, unsigned *mm) {
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_pts * nb; i += (long)gridDim.x * blockDim.x) {
        const long p = i / nb;
        const int n = (int)(i - p * nb);
        const unsigned o = ordered(eps[p * stride + n]);
        lo = min(lo, o);
        hi = max(hi, o);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

// kFermiPoints equidistant energies on [lo, hi] (both end points included).
__global__ void fill_grid_kernel(float *om, float lo, float hi) {
    const int i = threadIdx.x;
    if (i < kFermiPoints)
        om[i] = (i == kFermiPoints - 1) ? hi : lo + (hi - lo) * ((float)i / (float)(kFermiPoints - 1));
}

// Occupation summed over orbitals, at each of the grid's energies.
__global__ void sum_orbitals_kernel(const float *dos, int n_orb, float *tot) {
    const int i = threadIdx.x;
    if (i < kFermiPoints) {
        float t = 0.f;
        for (int s = 0; s < n_orb; ++s) t += dos[s * kFermiPoints + i];
        tot[i] = t;
    }
}

// The 64-energy integrated-mode plan of a plan (same grid, box and orbitals).
tetra_status_t integrated_plan(const Plan &P, Plan &Q) {
    tetra_desc_t d = P.d;
    d.mode = TETRA_INTEGRATED;
    d.n_omega = kFermiPoints;
    const int box[3] = {P.BX, P.BY, P.BZ};
    return plan_init(Q, d, P.device, box, std::max(1, P.grid_x / std::max(1, P.sm_count)));
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

size_t fermi_workspace(const Plan &P) {
    Plan Q;
    if (integrated_plan(P, Q) != TETRA_OK) return 0;
    return align256(dos_forward_workspace(Q)) + align256(sizeof(float) * kFermiPoints) +
           align256(sizeof(float) * (size_t)P.d.n_orb * kFermiPoints) + align256(sizeof(float) * kFermiPoints) + 256;
}

tetra_status_t fermi_level(const Plan &P, const float *eps, const void *w, double n_electrons, float *ef,
                           void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (P.z0 != 0 || P.z1 != P.d.n3) return TETRA_EUNSUPPORTED;   // the count needs the whole grid
    Plan Q;
    tetra_status_t st = integrated_plan(P, Q);
    if (st != TETRA_OK) return st;
    if (ws_bytes < fermi_workspace(P)) return TETRA_ENOMEM;
    unsigned char *b = static_cast<unsigned char *>(ws);
    void *fws = b;
    const size_t fws_bytes = align256(dos_forward_workspace(Q));
    float *om = reinterpret_cast<float *>(b + fws_bytes);
    float *dos = reinterpret_cast<float *>(b + fws_bytes + align256(sizeof(float) * kFermiPoints));
    float *tot = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(dos) +
                                           align256(sizeof(float) * (size_t)P.d.n_orb * kFermiPoints));
    unsigned *mm = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(tot) +
                                                align256(sizeof(float) * kFermiPoints));
    // bracket: the band range
    const unsigned init[2] = {0xFFFFFFFFu, 0u};
    if (cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, stream) != cudaSuccess) return TETRA_ECUDA;
    const long n_pts = (long)P.nx * P.ny * P.nz;
    band_range_kernel<<<4 * P.sm_count, 256, 0, stream>>>(eps, n_pts, P.eps_stride, P.d.n_bands, mm);
    unsigned hmm[2];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return TETRA_ECUDA;
    float lo = unordered(hmm[0]), hi = unordered(hmm[1]);
    if (!(lo <= hi)) return TETRA_EINVAL;
    if (hi == lo) hi = std::nextafter(lo, INFINITY);
    float h_tot[kFermiPoints];
    for (int round = 0; round < 64; ++round) {
        fill_grid_kernel<<<1, kFermiPoints, 0, stream>>>(om, lo, hi);
        if (cudaGetLastError() != cudaSuccess) return TETRA_ECUDA;
        st = launch_dos_forward(Q, eps, w, om, dos, fws, fws_bytes, stream);
        if (st != TETRA_OK) return st;
        sum_orbitals_kernel<<<1, kFermiPoints, 0, stream>>>(dos, P.d.n_orb, tot);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return TETRA_ECUDA;
        // N is non-decreasing: the first grid energy with N >= n_electrons
        if (round == 0 && (n_electrons < 0.0 || n_electrons > (double)h_tot[kFermiPoints - 1] * (1.0 + 1e-6)))
            return TETRA_EINVAL;
        int j = 0;
        while (j < kFermiPoints - 1 && (double)h_tot[j] < n_electrons) ++j;
        const float step = (hi - lo) / (float)(kFermiPoints - 1);
        const float nlo = (j == 0) ? lo : lo + step * (float)(j - 1);
        const float nhi = (j == kFermiPoints - 1) ? hi : lo + step * (float)j;
        // FP32 resolution reached: the bracket no longer shrinks
        if (!(nhi - nlo < hi - lo) || nhi <= std::nextafter(nlo, INFINITY)) {
            lo = nlo;
            hi = nhi;
            break;
        }
        lo = nlo;
        hi = nhi;
    }
    *ef = 0.5f * (lo + hi);
    return TETRA_OK;
}

}  // namespace tetra

extern "C" size_t tetra_fermi_workspace_bytes(tetra_plan_t plan) {
    if (!plan) return 0;
    return tetra::fermi_workspace(*plan);
}

extern "C" tetra_status_t tetra_fermi_level(tetra_plan_t plan, const float *eps, const void *w, double n_electrons,
                                            float *ef, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !eps || !w || !ef || !ws) return TETRA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(eps) & 15u) || (reinterpret_cast<uintptr_t>(w) & 15u) ||
        (reinterpret_cast<uintptr_t>(ws) & 15u))
        return TETRA_EINVAL;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::fermi_level(*plan, eps, w, n_electrons, ef, ws, ws_bytes, stream);
}
