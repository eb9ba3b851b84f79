// Adjoint of tetra_eig (not in the paper): dL/d(model parameters) from
// dL/deps_n(k) and dL/db_{n,s}(k), b_{n,s} = |V_{s n}|^2.
//
// Per k-point (first-order perturbation theory of the Hermitian eigenproblem):
//   d eps_n  = <n| dH |n>                               (Hellmann-Feynman)
//   d V_n    = sum_{m != n} V_m <m| dH |n> F_nm,  F_nm = 1/(eps_n - eps_m)
// so that dL = Re sum_ij dH_ij Q_ij with
//   Q = conj(V) (diag(geps) + 2 B) V^T,  B_mn = F_nm sum_s gw_{n s} conj(V_sn) V_sm.
// F_nm is formed in FP64 and regularised as d / (d^2 + eta^2), d = eps_n - eps_m,
// eta = 1e-8 eV, so near-degenerate pairs stay finite. With H(k) = diag(onsite)
// + sum_r [t_r e^{ik.R_r} + h.c.]:
//   dL/d onsite_i = Re sum_k Q_ii,
//   dL/d Re t_r   = Re sum_k e^{ik.R_r} (Q + Q^H),   dL/d Im t_r = -Im (same).
// Each persistent block accumulates its k-points in a fixed order (FP32 over
// one block step of 64 k-points, FP64 across steps); a second kernel adds the
// block partials in FP64 in block order (deterministic).
#include "eig_common.cuh"

namespace tetra {

namespace {

using namespace eigdetail;

constexpr int kBT = 64;   // k-points per block iteration
constexpr double kEta = 1e-8;

struct EigBwdArgs {
    int n1, n2, n3, nx, ny, n_R;
    int eps_stride, w_stride;
    const float *params;
    const int *R;
    const float *geps, *gw;
    double *partial;   // [gridDim.x][n_out]
    int n_out;
};

template <int N>
__global__ void __launch_bounds__(kBT) tetra_eig_bwd_kernel(const EigBwdArgs A) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float s_on[N];
    __shared__ float4 s_hop[kMaxR * n_upper<N>()];
    __shared__ int s_R[3 * kMaxR];
    constexpr int NN2 = 2 * N * N;   // complex N x N as (re, im) pairs
    float *Vs = sm;                  // [kBT][NN2]  eigenvectors V[s][j]
    float *Is = Vs + kBT * NN2;      // [kBT][NN2]  inner, later Q + Q^H
    float *Xs = Is + kBT * NN2;      // [kBT][NN2]  inner V^T
    float *Ph = Xs + kBT * NN2;      // [kBT][2 n_R] e^{ik.R}
    double *acc = reinterpret_cast<double *>(Ph + kBT * 2 * kMaxR);   // [n_out] block sums
    const int tid = threadIdx.x;
    stage_model<N>(A.params, A.R, A.n_R, A.n1, A.n2, A.n3, s_on, s_hop, s_R);
    __syncthreads();
    const long nk = (long)A.n1 * A.n2 * A.n3;
    const Grid3 g3 = grid3(A.n1, A.n2, A.n3);
    // outputs owned by this thread: o = tid, tid + kBT, ... (accumulated in acc[o])
    for (int o = tid; o < A.n_out; o += kBT) acc[o] = 0.0;
    float *V = Vs + tid * NN2, *In = Is + tid * NN2, *X = Xs + tid * NN2, *ph = Ph + tid * 2 * A.n_R;

    for (long k0 = (long)blockIdx.x * kBT; k0 < nk; k0 += (long)gridDim.x * kBT) {
        const long k = k0 + tid;
        const bool live = k < nk;
        if (live) {
            const int x = (int)(k % A.n1), y = (int)((k / A.n1) % A.n2), z = (int)(k / ((long)A.n1 * A.n2));
            // the forward's eigensolver (Householder + implicit QR), so the
            // eigenvectors are the ones the forward's weights came from
            Herm<N> M;
            {
                Mat<N> H;
                build_h<N>(H, s_on, s_hop, s_R, A.n_R, x, y, z, g3);
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int j = 0; j <= i; ++j) {
                        M.ar[i][j] = H.hr[j][i];
                        M.ai[i][j] = (i == j) ? 0.f : -H.hi[j][i];
                    }
            }
            float lam[N];
            if constexpr (N == 1) {
                lam[0] = M.ar[0][0];
                V[0] = 1.f;
                V[1] = 0.f;
            } else {
                householder_tridiag<N>(M);
                tridiag_qr<N>(M);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    lam[j] = M.d[j];
                    float vr[N], vi[N];
                    eigvec_column<N>(M, j, vr, vi);
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        V[2 * (s * N + j)] = vr[s];
                        V[2 * (s * N + j) + 1] = vi[s];
                    }
                }
            }
            // sorted band index of each eigenvector column (ties keep column
            // order, as the forward's stable transposition sort does)
            int rank[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                int r = 0;
#pragma unroll
                for (int i = 0; i < N; ++i) r += (lam[i] < lam[j]) || (lam[i] == lam[j] && i < j);
                rank[j] = r;
            }
            const long p = x + (long)A.nx * (y + (long)A.ny * z);
            float ge[N];
#pragma unroll
            for (int j = 0; j < N; ++j) ge[j] = A.geps[p * A.eps_stride + rank[j]];
            // S = inner + inner^H with inner = diag(geps) + 2 B, B_mn = F_nm A_nm,
            // A_nm = sum_s gw_ns conj(V_sn) V_sm; F is antisymmetric, so
            // S_nn = 2 geps_n and, for m != n,
            // S_mn = 2 F_nm sum_s (gw_ns - gw_ms) conj(V_sn) V_sm,  S_nm = conj(S_mn).
            // Then Q + Q^H = conj(V) S V^T, a Hermitian product: only i <= j formed.
            // gw of band n (column order) and orbital s, staged in X until Y
            // overwrites it
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const float *g = A.gw + p * A.w_stride + (long)rank[n] * N;
#pragma unroll
                for (int s = 0; s < N; ++s) X[n * N + s] = g[s];
            }
#pragma unroll
            for (int n = 0; n < N; ++n) {
                In[2 * (n * N + n)] = 2.f * ge[n];
                In[2 * (n * N + n) + 1] = 0.f;
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    float ar = 0.f, ai = 0.f;
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        const float vnr = V[2 * (s * N + n)], vni = V[2 * (s * N + n) + 1];
                        const float vmr = V[2 * (s * N + m)], vmi = V[2 * (s * N + m) + 1];
                        const float dg = X[n * N + s] - X[m * N + s];
                        // conj(V_sn) V_sm
                        ar = fmaf(dg, vnr * vmr + vni * vmi, ar);
                        ai = fmaf(dg, vnr * vmi - vni * vmr, ai);
                    }
                    const double d = (double)lam[n] - (double)lam[m];
                    const float F2 = 2.f * (float)(d / (d * d + kEta * kEta));
                    In[2 * (m * N + n)] = F2 * ar;   // S_mn
                    In[2 * (m * N + n) + 1] = F2 * ai;
                    In[2 * (n * N + m)] = F2 * ar;   // S_nm = conj(S_mn)
                    In[2 * (n * N + m) + 1] = -F2 * ai;
                }
            }
            // Y = S V^T : Y_mj = sum_n S_mn V_jn
#pragma unroll
            for (int m = 0; m < N; ++m)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    float xr = 0.f, xi = 0.f;
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        const float ir = In[2 * (m * N + n)], ii = In[2 * (m * N + n) + 1];
                        const float vr = V[2 * (j * N + n)], vi = V[2 * (j * N + n) + 1];
                        xr = fmaf(ir, vr, fmaf(-ii, vi, xr));
                        xi = fmaf(ir, vi, fmaf(ii, vr, xi));
                    }
                    X[2 * (m * N + j)] = xr;
                    X[2 * (m * N + j) + 1] = xi;
                }
            // Z = conj(V) Y = Q + Q^H into In (i <= j, mirrored; real diagonal)
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = i; j < N; ++j) {
                    float zr = 0.f, zi = 0.f;
#pragma unroll
                    for (int m = 0; m < N; ++m) {
                        const float vr = V[2 * (i * N + m)], vi = -V[2 * (i * N + m) + 1];
                        const float yr = X[2 * (m * N + j)], yi = X[2 * (m * N + j) + 1];
                        zr = fmaf(vr, yr, fmaf(-vi, yi, zr));
                        zi = fmaf(vr, yi, fmaf(vi, yr, zi));
                    }
                    In[2 * (i * N + j)] = zr;
                    In[2 * (i * N + j) + 1] = (i == j) ? 0.f : zi;
                    if (i != j) {
                        In[2 * (j * N + i)] = zr;
                        In[2 * (j * N + i) + 1] = -zi;
                    }
                }
            for (int r = 0; r < A.n_R; ++r) phase(s_R + 3 * r, x, y, z, g3, ph[2 * r + 1], ph[2 * r]);
        } else {
            for (int i = 0; i < NN2; ++i) In[i] = 0.f;
            for (int r = 0; r < 2 * A.n_R; ++r) ph[r] = 0.f;
        }
        __syncthreads();
        // block sums over the kBT k-points, in thread order: FP32 within the
        // block step, added to the FP64 accumulator once per step (FP64
        // arithmetic is slow on this GPU; 64 FP32 terms keep ~1e-6 relative)
        for (int o = tid; o < A.n_out; o += kBT) {
            float s = 0.f;
            if (o < N) {
                for (int t = 0; t < kBT; ++t) s += Is[t * NN2 + 2 * (o * N + o)];
                s *= 0.5f;
            } else {
                const int q = o - N;
                const int half = A.n_R * N * N;
                const bool im = q >= half;
                const int qq = im ? q - half : q;
                const int r = qq / (N * N), ij = qq - r * N * N;
                // Re: c zr - sn zi; Im (negated): -(sn zr + c zi)
                for (int t = 0; t < kBT; ++t) {
                    const float c = Ph[t * 2 * A.n_R + 2 * r], sn = Ph[t * 2 * A.n_R + 2 * r + 1];
                    const float zr = Is[t * NN2 + 2 * ij], zi = Is[t * NN2 + 2 * ij + 1];
                    const float a = im ? -sn : c, b = im ? -c : -sn;
                    s = fmaf(a, zr, fmaf(b, zi, s));
                }
            }
            acc[o] += (double)s;
        }
        __syncthreads();
    }
    for (int o = tid; o < A.n_out; o += kBT) A.partial[(long)blockIdx.x * A.n_out + o] = acc[o];
}

__global__ void tetra_eig_bwd_reduce(const double *partial, int n_blocks, int n_out, float *out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    double s = 0.0;
    for (int b = 0; b < n_blocks; ++b) s += partial[(long)b * n_out + o];
    out[o] = (float)s;
}

template <int N>
cudaError_t launch_n(const EigBwdArgs &A, int grid, cudaStream_t stream) {
    const size_t smem = (size_t)kBT * (3 * 2 * N * N + 2 * kMaxR) * sizeof(float) +
                        (size_t)A.n_out * sizeof(double);
    auto kfn = tetra_eig_bwd_kernel<N>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kfn<<<grid, kBT, smem, stream>>>(A);
    return cudaGetLastError();
}

int bwd_grid(const Plan &P) {
    const long nk = (long)P.d.n1 * P.d.n2 * P.d.n3;
    const long blocks = (nk + kBT - 1) / kBT;
    return (int)std::min<long>(blocks, 2L * P.sm_count);
}

}  // namespace

size_t eig_backward_workspace(const Plan &P, int n_R) {
    const int N = P.d.n_bands;
    const int n_out = N + 2 * n_R * N * N;
    return kStatusBytes + sizeof(double) * (size_t)bwd_grid(P) * n_out;
}

tetra_status_t launch_eig_backward(const Plan &P, const tetra_model_t *m, const float *geps,
                                   const float *gw, float *gparams, void *ws, size_t ws_bytes,
                                   cudaStream_t stream) {
    if (!m->params || (m->n_R > 0 && !m->R)) return TETRA_EINVAL;
    if (m->n_orb < 1 || m->n_orb > 8 || m->n_orb != P.d.n_bands || m->n_orb != P.d.n_orb)
        return TETRA_EUNSUPPORTED;
    if (m->n_R < 0 || m->n_R > kMaxR) return TETRA_EINVAL;
    if (ws_bytes < eig_backward_workspace(P, m->n_R)) return TETRA_ENOMEM;
    EigBwdArgs A;
    A.n1 = P.d.n1; A.n2 = P.d.n2; A.n3 = P.d.n3; A.nx = P.nx; A.ny = P.ny; A.n_R = m->n_R;
    A.eps_stride = P.eps_stride; A.w_stride = P.w_stride;
    A.params = m->params; A.R = m->R; A.geps = geps; A.gw = gw;
    A.n_out = m->n_orb + 2 * m->n_R * m->n_orb * m->n_orb;
    A.partial = reinterpret_cast<double *>(static_cast<unsigned char *>(ws) + kStatusBytes);
    if (cudaMemsetAsync(ws, 0, kStatusBytes, stream) != cudaSuccess) return TETRA_ECUDA;
    const int grid = bwd_grid(P);
    cudaError_t e;
    switch (m->n_orb) {
        case 1: e = launch_n<1>(A, grid, stream); break;
        case 2: e = launch_n<2>(A, grid, stream); break;
        case 3: e = launch_n<3>(A, grid, stream); break;
        case 4: e = launch_n<4>(A, grid, stream); break;
        case 5: e = launch_n<5>(A, grid, stream); break;
        case 6: e = launch_n<6>(A, grid, stream); break;
        case 7: e = launch_n<7>(A, grid, stream); break;
        default: e = launch_n<8>(A, grid, stream); break;
    }
    if (e != cudaSuccess) return TETRA_ECUDA;
    tetra_eig_bwd_reduce<<<(A.n_out + 127) / 128, 128, 0, stream>>>(A.partial, grid, A.n_out, gparams);
    return cudaGetLastError() == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace tetra
