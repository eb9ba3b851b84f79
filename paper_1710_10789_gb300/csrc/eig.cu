// Batched Hermitian eigensolver for tight-binding Hamiltonians on the k-grid
// (Sec. II.A: H(k) of Eq. (1) diagonalised point by point; orbital weights
// b = |a|^2 of Eq. (3)), writing band energies and orbital weights directly in
// the tetra layout, halo points included.
//
// One thread owns one k-point: it builds H(k) = diag(onsite) +
// sum_r [t_r e^{ik.R_r} + h.c.] from the model staged in shared memory, runs
// cyclic complex Jacobi sweeps with the upper triangle of H and the full
// eigenvector matrix in registers (all indices compile-time after unrolling),
// then sorts the eigenpairs with a transposition network and stores
// eps_n and |V_sn|^2.
#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kEigThreads = 128;
constexpr int kMaxR = 32;

struct EigArgs {
    int n1, n2, n3, nx, ny, nz;
    int n_R;
    int eps_stride, w_stride, n_orb_out;
    const float *params;
    const int *R;
    float *eps;
    void *w;
};

template <int N>
struct Mat {
    float hr[N][N], hi[N][N];   // upper triangle of H used (i <= j)
    float vr[N][N], vi[N][N];   // eigenvectors in columns
    float skip;                 // couplings at or below this are dropped unrotated
};

// Full-matrix element H_kp from upper-triangle storage (k != p).
template <int N>
__device__ __forceinline__ void hget(const Mat<N> &M, int k, int p, float &re, float &im) {
    if (k < p) { re = M.hr[k][p]; im = M.hi[k][p]; }
    else { re = M.hr[p][k]; im = -M.hi[p][k]; }
}
template <int N>
__device__ __forceinline__ void hset(Mat<N> &M, int k, int p, float re, float im) {
    if (k < p) { M.hr[k][p] = re; M.hi[k][p] = im; }
    else { M.hr[p][k] = re; M.hi[p][k] = -im; }
}

// Jacobi rotation zeroing H_pq (p < q): H <- U^H H U, V <- V U with
// U_pp = c, U_pq = s, U_qp = -s e^{-i phi}, U_qq = c e^{-i phi}, H_pq = |h| e^{i phi}.
template <int N, int p, int q>
__device__ __forceinline__ bool rotate(Mat<N> &M) {
    const float hr = M.hr[p][q], hi = M.hi[p][q];
    const float h2 = hr * hr + hi * hi;
    const float ha = sqrtf(h2);
    const float a = M.hr[p][p], b = M.hr[q][q];
    // coupling at the FP32 rounding level of ||H||: drop it, no rotation
    if (ha <= M.skip) {
        M.hr[p][q] = 0.f;
        M.hi[p][q] = 0.f;
        return false;
    }
    const float ihs = 1.0f / ha;
    const float er = hr * ihs, ei = -hi * ihs;   // e^{-i phi}
    const float tau = (b - a) * 0.5f * ihs;
    const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
    const float c = rsqrtf(fmaf(t, t, 1.0f));
    const float s = t * c;
    M.hr[p][p] = a - t * ha;
    M.hr[q][q] = b + t * ha;
    M.hr[p][q] = 0.f;
    M.hi[p][q] = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (k == p || k == q) continue;
        float xr, xi, yr, yi;
        hget(M, k, p, xr, xi);
        hget(M, k, q, yr, yi);
        const float zr = er * yr - ei * yi, zi = er * yi + ei * yr;   // e^{-i phi} H_kq
        hset(M, k, p, c * xr - s * zr, c * xi - s * zi);
        hset(M, k, q, s * xr + c * zr, s * xi + c * zi);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float xr = M.vr[i][p], xi = M.vi[i][p];
        const float yr = M.vr[i][q], yi = M.vi[i][q];
        const float zr = er * yr - ei * yi, zi = er * yi + ei * yr;
        M.vr[i][p] = c * xr - s * zr; M.vi[i][p] = c * xi - s * zi;
        M.vr[i][q] = s * xr + c * zr; M.vi[i][q] = s * xi + c * zi;
    }
    return true;
}

template <int N, int p, int q>
struct Sweep {
    // one cyclic sweep over all pairs; returns whether any rotation was applied
    __device__ __forceinline__ static bool run(Mat<N> &M) {
        bool any = rotate<N, p, q>(M);
        if constexpr (q + 1 < N) any |= Sweep<N, p, q + 1>::run(M);
        else if constexpr (p + 2 < N) any |= Sweep<N, p + 1, p + 2>::run(M);
        return any;
    }
};

template <int N>
__device__ __forceinline__ float offdiag2(const Mat<N> &M) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i + 1; j < N; ++j) s += M.hr[i][j] * M.hr[i][j] + M.hi[i][j] * M.hi[i][j];
    return s;
}

template <int N>
__device__ __forceinline__ void jacobi(Mat<N> &M) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) { M.vr[i][j] = (i == j) ? 1.f : 0.f; M.vi[i][j] = 0.f; }
    if constexpr (N > 1) {
        float fro = 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i) fro += M.hr[i][i] * M.hr[i][i];
        fro += 2.f * offdiag2(M);
        // couplings below the FP32 resolution of ||H|| are dropped unrotated; the
        // 1e-18 floor keeps |h|^2 out of the denormal range, where |h| (and with
        // it the phase h*/|h| of the rotation) would lose accuracy
        M.skip = 6e-8f * sqrtf(fro) + 1e-18f;
        // cyclic sweeps until the squared off-diagonal norm is below 1e-14 of
        // ||H||^2 (FP32 rounding level; convergence is quadratic), at most 12
        const float tol = 1e-14f * fro + 1e-30f;
        for (int sweep = 0; sweep < 12; ++sweep) {
            if (offdiag2(M) <= tol) break;
            Sweep<N, 0, 1>::run(M);
        }
    }
}

template <int N, typename WT>
__global__ void __launch_bounds__(kEigThreads) tetra_eig_kernel(const EigArgs A) {
    __shared__ float s_par[N + 2 * kMaxR * N * N];
    __shared__ int s_R[3 * kMaxR];
    const int npar = N + 2 * A.n_R * N * N;
    for (int i = threadIdx.x; i < npar; i += blockDim.x) s_par[i] = A.params[i];
    for (int i = threadIdx.x; i < 3 * A.n_R; i += blockDim.x) s_R[i] = A.R[i];
    __syncthreads();
    const long P = (long)A.nx * A.ny * A.nz;
    const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int px = (int)(p % A.nx), py = (int)((p / A.nx) % A.ny), pz = (int)(p / ((long)A.nx * A.ny));
    const int x = px % A.n1, y = py % A.n2, z = pz % A.n3;

    Mat<N> M;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) { M.hr[i][j] = (i == j) ? s_par[i] : 0.f; M.hi[i][j] = 0.f; }
    const float *tre = s_par + N;
    const float *tim = s_par + N + A.n_R * N * N;
    for (int r = 0; r < A.n_R; ++r) {
        // phase 2 pi k.R reduced exactly: m_i = (x_i R_i) mod n_i
        auto md = [](long a, int n) { long m = a % n; return m < 0 ? m + n : m; };
        const long m0 = md((long)x * s_R[3 * r], A.n1);
        const long m1 = md((long)y * s_R[3 * r + 1], A.n2);
        const long m2 = md((long)z * s_R[3 * r + 2], A.n3);
        float frac = (float)m0 / A.n1 + (float)m1 / A.n2 + (float)m2 / A.n3;
        float sn, cs;
        sincospif(2.0f * frac, &sn, &cs);
        const float *Tr = tre + r * N * N, *Ti = tim + r * N * N;
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i; j < N; ++j) {
                // t_ij e^{i th} + conj(t_ji) e^{-i th}
                const float ar = Tr[i * N + j], ai = Ti[i * N + j];
                const float br = Tr[j * N + i], bi = Ti[j * N + i];
                M.hr[i][j] += (ar * cs - ai * sn) + (br * cs - bi * sn);
                M.hi[i][j] += (ar * sn + ai * cs) - (br * sn + bi * cs);
            }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) M.hi[i][i] = 0.f;
    jacobi<N>(M);

    // eigenvalues and weights, sorted ascending (odd-even transposition network)
    float ev[N];
    float W[N][N];   // W[n][s] = |V_sn|^2
#pragma unroll
    for (int n = 0; n < N; ++n) {
        ev[n] = M.hr[n][n];
#pragma unroll
        for (int s = 0; s < N; ++s) W[n][s] = M.vr[s][n] * M.vr[s][n] + M.vi[s][n] * M.vi[s][n];
    }
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
    float *eo = A.eps + p * A.eps_stride;
#pragma unroll
    for (int n = 0; n < N; ++n) eo[n] = ev[n];
    WT *wo = static_cast<WT *>(A.w) + p * A.w_stride;
#pragma unroll
    for (int n = 0; n < N; ++n)
#pragma unroll
        for (int s = 0; s < N; ++s) wo[n * N + s] = from_f32<WT>(W[n][s]);
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
    if (m->n_orb < 1 || m->n_orb > 8 || m->n_orb != P.d.n_bands || m->n_orb != P.d.n_orb)
        return TETRA_EUNSUPPORTED;
    if (m->n_R < 0 || m->n_R > kMaxR) return TETRA_EINVAL;
    EigArgs A;
    A.n1 = P.d.n1; A.n2 = P.d.n2; A.n3 = P.d.n3;
    A.nx = P.nx; A.ny = P.ny; A.nz = P.nz;
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
