// Batched Hermitian eigensolver for tight-binding Hamiltonians on the k-grid
// (Sec. II.A: H(k) of Eq. (1) diagonalised point by point; orbital weights
// b = |a|^2 of Eq. (3)), writing band energies and orbital weights directly in
// the tetra layout, halo points included.
//
// One thread owns one k-point: it builds H(k) = diag(onsite) +
// sum_r [t_r e^{ik.R_r} + h.c.] from the model staged in shared memory,
// reduces it to real tridiagonal form by Householder reflections and
// diagonalises that by implicit-shift QR, with H, the reflectors, the
// accumulated rotations and the tridiagonal in registers (all indices
// compile-time after unrolling), forms each eigenvector by applying the
// reflectors to a column of the rotations, then sorts the eigenpairs with a
// transposition network and stores eps_n and |V_sn|^2.
#include "eig_common.cuh"

namespace tetra {

namespace {

using namespace eigdetail;

template <int N, typename WT>
__global__ void __launch_bounds__(kEigThreads) tetra_eig_kernel(const EigArgs A) {
    __shared__ float s_on[N];
    __shared__ float4 s_hop[kMaxR * n_upper<N>()];
    __shared__ int s_R[3 * kMaxR];
    stage_model<N>(A.params, A.R, A.n_R, A.n1, A.n2, A.n3, s_on, s_hop, s_R);
    __syncthreads();
    const long P = (long)A.nx * A.ny * A.nz;
    const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (q >= P) return;
    const long p = q + (long)A.z_off * A.nx * A.ny;   // padded point index
    const int px = (int)(p % A.nx), py = (int)((p / A.nx) % A.ny), pz = (int)(p / ((long)A.nx * A.ny));
    const int x = px % A.n1, y = py % A.n2, z = pz % A.n3;

    Herm<N> M;
    {
        Mat<N> H;   // upper triangle of H(k)
        build_h<N>(H, s_on, s_hop, s_R, A.n_R, x, y, z, A.n1, A.n2, A.n3);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                M.ar[i][j] = H.hr[j][i];
                M.ai[i][j] = (i == j) ? 0.f : -H.hi[j][i];
            }
    }
    float ev[N];
    float W[N][N];   // W[n][s] = |V_sn|^2
    if constexpr (N == 1) {
        ev[0] = M.ar[0][0];
        W[0][0] = 1.f;
    } else {
        householder_tridiag<N>(M);
        tridiag_qr<N>(M);
#pragma unroll
        for (int n = 0; n < N; ++n) {
            ev[n] = M.d[n];
            float vr[N], vi[N];
            eigvec_column<N>(M, n, vr, vi);
#pragma unroll
            for (int s = 0; s < N; ++s) W[n][s] = vr[s] * vr[s] + vi[s] * vi[s];
        }
    }
    // eigenvalues and weights, sorted ascending (odd-even transposition network)
#pragma unroll
    for (int round = 0; round < N; ++round)
#pragma unroll
        for (int a = (round & 1); a + 1 < N; a += 2) {
            const bool sw = ev[a + 1] < ev[a];
            const float lo = sw ? ev[a + 1] : ev[a], hi = sw ? ev[a] : ev[a + 1];
            ev[a] = lo; ev[a + 1] = hi;
#pragma unroll
            for (int s = 0; s < N; ++s) {
                const float u = W[a][s], v = W[a + 1][s];
                W[a][s] = sw ? v : u;
                W[a + 1][s] = sw ? u : v;
            }
        }
    // Stores: 16-byte vectors when a point's values fill whole vectors (the
    // layout's point strides are multiples of 16 bytes), scalars otherwise.
    float *eo = A.eps + p * A.eps_stride;
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int n = 0; n < N; n += 4)
            *reinterpret_cast<float4 *>(eo + n) = make_float4(ev[n], ev[n + 1], ev[n + 2], ev[n + 3]);
    } else {
#pragma unroll
        for (int n = 0; n < N; ++n) eo[n] = ev[n];
    }
    WT *wo = static_cast<WT *>(A.w) + p * A.w_stride;
    constexpr int VEC = 16 / sizeof(WT);
    if (A.n_orb_out < N) {
        // projection on the first n_orb_out orbitals only: w[n][s], s < n_orb_out
#pragma unroll
        for (int n = 0; n < N; ++n)
#pragma unroll
            for (int s = 0; s < N; ++s)
                if (s < A.n_orb_out) wo[n * A.n_orb_out + s] = from_f32<WT>(W[n][s]);
    } else if constexpr ((N * N) % VEC == 0) {
#pragma unroll
        for (int v = 0; v < N * N / VEC; ++v) {
            uint4 q;
            WT *e = reinterpret_cast<WT *>(&q);
#pragma unroll
            for (int j = 0; j < VEC; ++j) e[j] = from_f32<WT>(W[(v * VEC + j) / N][(v * VEC + j) % N]);
            reinterpret_cast<uint4 *>(wo)[v] = q;
        }
    } else {
#pragma unroll
        for (int n = 0; n < N; ++n)
#pragma unroll
            for (int s = 0; s < N; ++s) wo[n * N + s] = from_f32<WT>(W[n][s]);
    }
}

template <int N>
cudaError_t launch_n(const Plan &P, const EigArgs &A, cudaStream_t stream) {
    const long pts = (long)A.nx * A.ny * A.nz;
    const int grid = (int)((pts + kEigThreads - 1) / kEigThreads);
    switch (P.d.weight_dtype) {
        case TETRA_F16: tetra_eig_kernel<N, __half><<<grid, kEigThreads, 0, stream>>>(A); break;
        case TETRA_BF16: tetra_eig_kernel<N, __nv_bfloat16><<<grid, kEigThreads, 0, stream>>>(A); break;
        default: tetra_eig_kernel<N, float><<<grid, kEigThreads, 0, stream>>>(A); break;
    }
    return cudaGetLastError();
}

}  // namespace

tetra_status_t launch_eig(const Plan &P, const tetra_model_t *m, float *eps, void *w,
                          cudaStream_t stream) {
    if (!m || !m->params || (m->n_R > 0 && !m->R) || !eps || !w) return TETRA_EINVAL;
    if (m->n_orb < 1 || m->n_orb > 8 || m->n_orb != P.d.n_bands || P.d.n_orb > m->n_orb)
        return TETRA_EUNSUPPORTED;
    if (m->n_R < 0 || m->n_R > kMaxR) return TETRA_EINVAL;
    EigArgs A;
    A.n1 = P.d.n1; A.n2 = P.d.n2; A.n3 = P.d.n3;
    A.nx = P.nx; A.ny = P.ny;
    // a slab plan needs the points of its cube planes z0 .. z1 (upper halo included)
    A.z_off = P.z0;
    A.nz = P.z1 - P.z0 + 1;
    A.n_R = m->n_R;
    A.eps_stride = P.eps_stride; A.w_stride = P.w_stride; A.n_orb_out = P.d.n_orb;
    A.params = m->params; A.R = m->R; A.eps = eps; A.w = w;
    cudaError_t e;
    switch (m->n_orb) {
        case 1: e = launch_n<1>(P, A, stream); break;
        case 2: e = launch_n<2>(P, A, stream); break;
        case 3: e = launch_n<3>(P, A, stream); break;
        case 4: e = launch_n<4>(P, A, stream); break;
        case 5: e = launch_n<5>(P, A, stream); break;
        case 6: e = launch_n<6>(P, A, stream); break;
        case 7: e = launch_n<7>(P, A, stream); break;
        default: e = launch_n<8>(P, A, stream); break;
    }
    return e == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace tetra
