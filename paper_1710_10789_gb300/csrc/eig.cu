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
// compile-time after unrolling), ranks the eigenvalues, and stores each
// eigenvalue and the squared moduli of its eigenvector (formed by applying the
// reflectors to a column of the rotations) at its place in ascending order.
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
        build_h<N>(H, s_on, s_hop, s_R, A.n_R, x, y, z, grid3(A.n1, A.n2, A.n3));
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                M.ar[i][j] = H.hr[j][i];
                M.ai[i][j] = (i == j) ? 0.f : -H.hi[j][i];
            }
    }
    float *eo = A.eps + p * A.eps_stride;
    WT *wo = static_cast<WT *>(A.w) + p * A.w_stride;
    if constexpr (N == 1) {
        eo[0] = M.ar[0][0];
        wo[0] = from_f32<WT>(1.f);
        return;
    } else {
        householder_tridiag<N>(M);
        tridiag_qr<N>(M);
        // place of each eigenpair in ascending order; equal eigenvalues keep
        // their column order (a NaN counts as +inf, so the places stay a
        // permutation whatever the input)
        float key[N];
        int rank[N];
#pragma unroll
        for (int j = 0; j < N; ++j) key[j] = isnan(M.d[j]) ? INFINITY : M.d[j];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            int r = 0;
#pragma unroll
            for (int i = 0; i < N; ++i) r += (key[i] < key[j]) || (key[i] == key[j] && i < j);
            rank[j] = r;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) eo[rank[j]] = M.d[j];
        // weights |V_sn|^2 of eigenvector n, stored as band row rank[n]: whole
        // 16-byte vectors when a row fills them (the point strides are
        // multiples of 16 bytes), scalars otherwise. The columns are formed in
        // a loop that is not unrolled (one copy of the reflector code: the
        // unrolled solver does not fit the instruction cache), reading G and
        // the ranks from this thread's slice of shared memory.
        extern __shared__ float s_g[];   // [N * N + N][blockDim.x]
        const int ts = blockDim.x;
        float *gs = s_g + threadIdx.x;
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) gs[(r * N + c) * ts] = M.g[r][c];
#pragma unroll
        for (int j = 0; j < N; ++j) gs[(N * N + j) * ts] = __int_as_float(rank[j]);
        constexpr int VEC = 16 / sizeof(WT);
#pragma unroll 1
        for (int n = 0; n < N; ++n) {
            float vr[N], vi[N], b[N];
#pragma unroll
            for (int r = 0; r < N; ++r) {
                const float g = gs[(r * N + n) * ts];
                vr[r] = M.sr[r] * g;
                vi[r] = M.si[r] * g;
            }
            apply_reflectors<N>(M, vr, vi);
            const int rk = __float_as_int(gs[(N * N + n) * ts]);
#pragma unroll
            for (int s = 0; s < N; ++s) b[s] = vr[s] * vr[s] + vi[s] * vi[s];
            if (A.n_orb_out < N) {
                // projection on the first n_orb_out orbitals only
#pragma unroll
                for (int s = 0; s < N; ++s)
                    if (s < A.n_orb_out) wo[rk * A.n_orb_out + s] = from_f32<WT>(b[s]);
            } else if constexpr (N % VEC == 0) {
                uint4 *row = reinterpret_cast<uint4 *>(wo + rk * N);
#pragma unroll
                for (int v = 0; v < N / VEC; ++v) {
                    uint4 q;
                    WT *e = reinterpret_cast<WT *>(&q);
#pragma unroll
                    for (int j = 0; j < VEC; ++j) e[j] = from_f32<WT>(b[v * VEC + j]);
                    row[v] = q;
                }
            } else {
#pragma unroll
                for (int s = 0; s < N; ++s) wo[rk * N + s] = from_f32<WT>(b[s]);
            }
        }
    }
}

template <int N>
cudaError_t launch_n(const Plan &P, const EigArgs &A, cudaStream_t stream) {
    const long pts = (long)A.nx * A.ny * A.nz;
    const int grid = (int)((pts + kEigThreads - 1) / kEigThreads);
    const size_t smem = N > 1 ? sizeof(float) * (N * N + N) * kEigThreads : 0;
    auto go = [&](auto kfn) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kfn<<<grid, kEigThreads, smem, stream>>>(A);
        return cudaGetLastError();
    };
    switch (P.d.weight_dtype) {
        case TETRA_F16: return go(tetra_eig_kernel<N, __half>);
        case TETRA_BF16: return go(tetra_eig_kernel<N, __nv_bfloat16>);
        default: return go(tetra_eig_kernel<N, float>);
    }
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
