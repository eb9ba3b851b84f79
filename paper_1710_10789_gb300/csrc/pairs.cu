// Transition bands of the bare susceptibility at momentum q: for every grid
// point k and band pair (n, m), energy eps_m(k+q) - eps_n(k) and weight
// f(eps_n(k)) - f(eps_m(k+q)) (Fermi-Dirac occupation). Their tetrahedron DOS,
// evaluated by tetra_dos on a plan with n_bands^2 bands, is the spectral part
// of the bare Lindhard function (the extension to susceptibilities the paper
// names; both differences are linear inside a tetrahedron by the method's own
// interpolation).
#include "tetra_internal.cuh"

namespace tetra {

namespace {

__device__ __forceinline__ float occupation(float e, float mu, float inv_kT) {
    return 0.5f * (1.0f - tanhf(0.5f * (e - mu) * inv_kT));
}

// One thread per padded point of the pair plan's layout (halo included).
template <int NB>
__global__ void pair_bands_kernel(const float *eps, int eps_stride, int n1, int n2, int n3, int nx, int ny,
                                  int qx, int qy, int qz, float mu, float inv_kT, long n_pts,
                                  float *eps_p, int eps_stride_p, float *w_p, int w_stride_p) {
    const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (p >= n_pts) return;
    const int px = (int)(p % nx), py = (int)((p / nx) % ny), pz = (int)(p / ((long)nx * ny));
    const int x = px % n1, y = py % n2, z = pz % n3;
    const long pk = x + (long)nx * (y + (long)ny * z);
    const int xq = (x + qx) % n1, yq = (y + qy) % n2, zq = (z + qz) % n3;
    const long pkq = xq + (long)nx * (yq + (long)ny * zq);
    float ek[NB], ekq[NB], fk[NB], fkq[NB];
#pragma unroll
    for (int n = 0; n < NB; ++n) {
        ek[n] = eps[pk * eps_stride + n];
        ekq[n] = eps[pkq * eps_stride + n];
        fk[n] = occupation(ek[n], mu, inv_kT);
        fkq[n] = occupation(ekq[n], mu, inv_kT);
    }
    float *eo = eps_p + p * eps_stride_p;
    float *wo = w_p + p * w_stride_p;
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            eo[n * NB + m] = ekq[m] - ek[n];
            wo[n * NB + m] = fk[n] - fkq[m];
        }
}

template <int NB>
cudaError_t launch_nb(const Plan &P, const Plan &Q, const float *eps, const int q[3], float mu, float inv_kT,
                      float *eps_p, float *w_p, cudaStream_t stream) {
    const long n_pts = (long)Q.nx * Q.ny * Q.nz;
    const int threads = 128;
    const long blocks = (n_pts + threads - 1) / threads;
    pair_bands_kernel<NB><<<(unsigned)blocks, threads, 0, stream>>>(
        eps, P.eps_stride, P.d.n1, P.d.n2, P.d.n3, P.nx, P.ny, q[0], q[1], q[2], mu, inv_kT, n_pts, eps_p,
        Q.eps_stride, w_p, Q.w_stride);
    return cudaGetLastError();
}

int reduce_q(int a, int n) {
    const int m = a % n;
    return m < 0 ? m + n : m;
}

}  // namespace

tetra_status_t launch_pair_bands(const Plan &P, const float *eps, const int q_in[3], float kT, float mu,
                                 const Plan &Q, float *eps_p, float *w_p, cudaStream_t stream) {
    const int nb = P.d.n_bands;
    if (Q.d.n1 != P.d.n1 || Q.d.n2 != P.d.n2 || Q.d.n3 != P.d.n3) return TETRA_EINVAL;
    if (Q.d.n_bands != nb * nb || Q.d.n_orb != 1 || Q.d.weight_dtype != TETRA_F32) return TETRA_EINVAL;
    if (P.z0 != 0 || P.z1 != P.d.n3 || Q.z0 != 0 || Q.z1 != Q.d.n3) return TETRA_EUNSUPPORTED;
    if (!(kT > 0.f) || !(kT < 1e30f)) return TETRA_EINVAL;
    const int q[3] = {reduce_q(q_in[0], P.d.n1), reduce_q(q_in[1], P.d.n2), reduce_q(q_in[2], P.d.n3)};
    const float inv_kT = 1.0f / kT;
    cudaError_t e;
    switch (nb) {
        case 1: e = launch_nb<1>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 2: e = launch_nb<2>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 3: e = launch_nb<3>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 4: e = launch_nb<4>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 5: e = launch_nb<5>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 6: e = launch_nb<6>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 7: e = launch_nb<7>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        case 8: e = launch_nb<8>(P, Q, eps, q, mu, inv_kT, eps_p, w_p, stream); break;
        default: return TETRA_EUNSUPPORTED;
    }
    return e == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace tetra

extern "C" tetra_status_t tetra_pair_bands(tetra_plan_t plan, const float *eps, const int q[3], float kT, float mu,
                                           tetra_plan_t pair_plan, float *eps_pairs, float *w_pairs,
                                           cudaStream_t stream) {
    if (!plan || !pair_plan || !eps || !q || !eps_pairs || !w_pairs) return TETRA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(eps) & 15u) || (reinterpret_cast<uintptr_t>(eps_pairs) & 15u) ||
        (reinterpret_cast<uintptr_t>(w_pairs) & 15u))
        return TETRA_EINVAL;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_pair_bands(*plan, eps, q, kT, mu, *pair_plan, eps_pairs, w_pairs, stream);
}
