// Adjoint of tetra_eig (not in the paper): dL/d(model parameters) from
// dL/deps_n(k) and dL/db_{n,s}(k), b_{n,s} = |V_{s n}|^2.
//
// Per k-point (first-order perturbation theory of the Hermitian eigenproblem):
//   d eps_n  = <n| dH |n>                               (Hellmann-Feynman)
//   d V_n    = sum_{m != n} V_m <m| dH |n> F_nm,  F_nm = 1/(eps_n - eps_m)
// so that dL = Re sum_ij dH_ij Q_ij with
//   Q = conj(V) (diag(geps) + 2 B) V^T,  B_mn = F_nm sum_s gw_{n s} conj(V_sn) V_sm.
// F_nm is regularised as d / (d^2 + eta^2), d = eps_n - eps_m, eta = 1e-8 eV,
// so near-degenerate pairs stay finite; for those (|d| < kNearDeg) it is
// formed in FP64, for the rest in FP32 (their 1/d is far from any
// cancellation). With H(k) = diag(onsite) + sum_r [t_r e^{ik.R_r} + h.c.]:
//   dL/d onsite_i = Re sum_k Q_ii,
//   dL/d Re t_r   = Re sum_k e^{ik.R_r} (Q + Q^H),   dL/d Im t_r = -Im (same).
// Each persistent block takes kBT k-points per step, one per thread, and adds
// them into its FP64 accumulators in a fixed order (FP32 sums over kChunk
// k-points in between); a second kernel adds the block partials in FP64 in
// block order (deterministic).
//
// Shared memory per thread: one row of 2 N^2 + 1 floats (an odd stride, so
// the rows of a warp fall in different banks), real parts in [0, N^2) and
// imaginary parts in [N^2, 2 N^2). It holds in turn the rotations G of the QR
// phase (G_rn in the real slot of V_rn), the eigenvectors V (V_sn at s N + n;
// column n written over the G column it was formed from), and Z = Q + Q^H
// (Z_ij, i <= j, at j N + i: column j written over row j of V once that row is
// in registers). Beside it the 2 n_R phases e^{ik.R_r}. At 8 orbitals and 7
// lattice vectors a 128-thread block takes about 85 KB, so two blocks share an
// SM.
#include "eig_common.cuh"

namespace tetra {

namespace {

using namespace eigdetail;

constexpr int kBT = 128;     // k-points per block step
constexpr int kChunk = 32;   // k-points summed in FP32 before an FP64 add
constexpr int kRB = 4;       // lattice vectors per reduction pass of a thread
constexpr float kEta2 = 1e-16f;   // eta^2, eta = 1e-8 eV
constexpr double kEta = 1e-8;
constexpr float kNearDeg = 1e-4f; // eV: pairs this close take F_nm in FP64

struct EigBwdArgs {
    int n1, n2, n3, nx, ny, n_R;
    int eps_stride, w_stride;
    const float *params;
    const int *R;
    const float *geps, *gw;
    double *partial;   // [gridDim.x][n_out]
    int n_out;
};

// 2 F_nm in FP64 for a near-degenerate pair; one copy of the code, called
// from the unrolled pair loop (inline, its 28 FP64 divisions would crowd the
// instruction cache).
__device__ __noinline__ float twice_f_fp64(float en, float em) {
    const double dd = (double)en - (double)em;
    return (float)(2.0 * dd / (dd * dd + kEta * kEta));
}

template <int N>
__host__ __device__ constexpr int row_floats() { return 2 * N * N + 1; }

// Dynamic shared memory: FP64 accumulators [n_out], the staged hoppings
// [n_R][n_upper], the per-thread rows [kBT][2 N^2 + 1], the phases
// [kBT][2 n_R] (byte offsets).
struct BwdSmem {
    size_t hop, z, ph, total;
};
template <int N>
__host__ __device__ inline BwdSmem bwd_smem(int n_R, int n_out) {
    BwdSmem L;
    L.hop = ((size_t)n_out * sizeof(double) + 15) / 16 * 16;
    L.z = L.hop + (size_t)n_R * n_upper<N>() * sizeof(float4);
    L.ph = L.z + (size_t)kBT * row_floats<N>() * sizeof(float);
    L.total = L.ph + (size_t)kBT * 2 * n_R * sizeof(float);
    return L;
}

template <int N>
__global__ void __launch_bounds__(kBT, 2) tetra_eig_bwd_kernel(const EigBwdArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float s_on[N];
    __shared__ int s_R[3 * kMaxR];
    constexpr int NN = N * N;
    constexpr int RF = row_floats<N>();
    const BwdSmem L = bwd_smem<N>(A.n_R, A.n_out);
    double *acc = reinterpret_cast<double *>(smraw);
    float4 *s_hop = reinterpret_cast<float4 *>(smraw + L.hop);
    float *Zs = reinterpret_cast<float *>(smraw + L.z);
    float *Ph = reinterpret_cast<float *>(smraw + L.ph);
    const int tid = threadIdx.x;
    const int PS = 2 * A.n_R;
    stage_model<N>(A.params, A.R, A.n_R, A.n1, A.n2, A.n3, s_on, s_hop, s_R);
    // outputs: o < N on-site, then Re and Im parts of every (r, i, j)
    for (int o = tid; o < A.n_out; o += kBT) acc[o] = 0.0;
    __syncthreads();
    const long nk = (long)A.n1 * A.n2 * A.n3;
    const Grid3 g3 = grid3(A.n1, A.n2, A.n3);
    float *row = Zs + tid * RF;
    float *ph = Ph + tid * PS;

    for (long k0 = (long)blockIdx.x * kBT; k0 < nk; k0 += (long)gridDim.x * kBT) {
        const long k = k0 + tid;
        if (k < nk) {
            const int x = (int)(k % A.n1), y = (int)((k / A.n1) % A.n2), z = (int)(k / ((long)A.n1 * A.n2));
            float lam[N];
            if constexpr (N == 1) {
                Mat<1> H;
                build_h<1>(H, s_on, s_hop, s_R, A.n_R, x, y, z, g3);
                lam[0] = H.hr[0][0];
                row[0] = 1.f;
                row[1] = 0.f;
            } else {
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
                householder_tridiag<N>(M);
                tridiag_qr<N>(M);
#pragma unroll
                for (int j = 0; j < N; ++j) lam[j] = M.d[j];
#pragma unroll
                for (int r = 0; r < N; ++r)
#pragma unroll
                    for (int c = 0; c < N; ++c) row[r * N + c] = M.g[r][c];
                // eigenvector columns in a loop that is not unrolled (one copy
                // of the reflector code), each over the G column it came from
#pragma unroll 1
                for (int n = 0; n < N; ++n) {
                    float vr[N], vi[N];
#pragma unroll
                    for (int r = 0; r < N; ++r) {
                        const float g = row[r * N + n];
                        vr[r] = M.sr[r] * g;
                        vi[r] = M.si[r] * g;
                    }
                    apply_reflectors<N>(M, vr, vi);
#pragma unroll
                    for (int r = 0; r < N; ++r) {
                        row[r * N + n] = vr[r];
                        row[NN + r * N + n] = vi[r];
                    }
                }
            }
            // sorted band index of each eigenvector column (ties keep column
            // order, as the forward's ranking does)
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
            const float *gwp = A.gw + p * A.w_stride;
            // S = inner + inner^H with inner = diag(geps) + 2 B, B_mn = F_nm A_nm,
            // A_nm = sum_s gw_ns conj(V_sn) V_sm; F is antisymmetric, so
            // S_nn = 2 geps_n and, for m < n,
            // S_mn = 2 F_nm sum_s (gw_ns - gw_ms) conj(V_sn) V_sm,  S_nm = conj(S_mn).
            float sr[N][N], si[N][N];   // S_mn for m < n
#pragma unroll
            for (int n = 0; n < N; ++n)
#pragma unroll
                for (int m = 0; m < n; ++m) { sr[m][n] = 0.f; si[m][n] = 0.f; }
#pragma unroll 1
            for (int s = 0; s < N; ++s) {
                float vr[N], vi[N], g[N];
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    vr[n] = row[s * N + n];
                    vi[n] = row[NN + s * N + n];
                    g[n] = gwp[rank[n] * N + s];   // gw of band n (column order), orbital s
                }
#pragma unroll
                for (int n = 0; n < N; ++n)
#pragma unroll
                    for (int m = 0; m < n; ++m) {
                        const float dg = g[n] - g[m];
                        // conj(V_sn) V_sm
                        sr[m][n] = fmaf(dg, vr[n] * vr[m] + vi[n] * vi[m], sr[m][n]);
                        si[m][n] = fmaf(dg, vr[n] * vi[m] - vi[n] * vr[m], si[m][n]);
                    }
            }
#pragma unroll
            for (int n = 0; n < N; ++n)
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    const float d = lam[n] - lam[m];
                    float F2 = 2.f * __fdividef(d, fmaf(d, d, kEta2));
                    // FP64 only in a warp that has a near-degenerate pair here
                    // (a vote, so the rare FP64 path is not evaluated for all)
                    if (__any_sync(__activemask(), fabsf(d) < kNearDeg) && fabsf(d) < kNearDeg)
                        F2 = twice_f_fp64(lam[n], lam[m]);
                    sr[m][n] *= F2;
                    si[m][n] *= F2;
                }
            // Q + Q^H = conj(V) S V^T, Hermitian: Z_ij for i <= j only. Column j
            // (last first): y = S (row j of V)^T, Z_ij = sum_m conj(V_im) y_m.
#pragma unroll 1
            for (int j = N - 1; j >= 0; --j) {
                float vjr[N], vji[N], yr[N], yi[N];
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    vjr[n] = row[j * N + n];
                    vji[n] = row[NN + j * N + n];
                }
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    float ar = 2.f * ge[m] * vjr[m], ai = 2.f * ge[m] * vji[m];
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        if (n == m) continue;
                        const float s_r = m < n ? sr[m][n] : sr[n][m];
                        const float s_i = m < n ? si[m][n] : -si[n][m];
                        ar = fmaf(s_r, vjr[n], fmaf(-s_i, vji[n], ar));
                        ai = fmaf(s_r, vji[n], fmaf(s_i, vjr[n], ai));
                    }
                    yr[m] = ar;
                    yi[m] = ai;
                }
                // Z_jj from the registers (real), then Z_ij for i < j from rows
                // i of V, which later columns no longer need
                {
                    float zr = 0.f;
#pragma unroll
                    for (int m = 0; m < N; ++m) zr = fmaf(vjr[m], yr[m], fmaf(vji[m], yi[m], zr));
                    row[j * N + j] = zr;
                    row[NN + j * N + j] = 0.f;
                }
#pragma unroll 1
                for (int i = 0; i < j; ++i) {
                    float zr = 0.f, zi = 0.f;
#pragma unroll
                    for (int m = 0; m < N; ++m) {
                        const float vr = row[i * N + m], vi = -row[NN + i * N + m];
                        zr = fmaf(vr, yr[m], fmaf(-vi, yi[m], zr));
                        zi = fmaf(vr, yi[m], fmaf(vi, yr[m], zi));
                    }
                    row[j * N + i] = zr;
                    row[NN + j * N + i] = zi;
                }
            }
            for (int r = 0; r < A.n_R; ++r) phase(s_R + 3 * r, x, y, z, g3, ph[2 * r + 1], ph[2 * r]);
        } else {
            for (int i = 0; i < 2 * NN; ++i) row[i] = 0.f;
            for (int r = 0; r < PS; ++r) ph[r] = 0.f;
        }
        __syncthreads();
        // block sums over the kBT k-points, in k-point order: FP32 over
        // kChunk k-points, FP64 beyond (FP64 arithmetic is slow on this GPU)
        if (tid < N) {
            double s = 0.0;
            for (int c0 = 0; c0 < kBT; c0 += kChunk) {
                float f = 0.f;
                for (int t = c0; t < c0 + kChunk; ++t) f += Zs[t * RF + tid * N + tid];
                s += (double)f;
            }
            acc[tid] += 0.5 * s;   // Re Q_ii = Z_ii / 2
        }
        {
            // P threads per matrix entry (i, j); thread (ij, q) takes the
            // lattice vectors r = q, q + P, ..., kRB of them per pass.
            // Re output: c Re Z - s Im Z; Im output: -(s Re Z + c Im Z), with
            // Z_ij = conj(Z_ji) read from the stored triangle for i > j.
            constexpr int P = kBT / NN;
            if (tid < P * NN) {
                const int ij = tid % NN, q = tid / NN;
                const int i = ij / N, j = ij - i * N;
                const int slot = i <= j ? j * N + i : i * N + j;
                const float zsg = i <= j ? 1.f : -1.f;
                const int half = A.n_R * NN;
                for (int r0 = q; r0 < A.n_R; r0 += kRB * P) {
                    double dre[kRB], dim[kRB];
#pragma unroll
                    for (int b = 0; b < kRB; ++b) { dre[b] = 0.0; dim[b] = 0.0; }
                    for (int c0 = 0; c0 < kBT; c0 += kChunk) {
                        float fre[kRB], fim[kRB];
#pragma unroll
                        for (int b = 0; b < kRB; ++b) { fre[b] = 0.f; fim[b] = 0.f; }
                        for (int t = c0; t < c0 + kChunk; ++t) {
                            const float zr = Zs[t * RF + slot], zi = zsg * Zs[t * RF + NN + slot];
                            const float2 *pt = reinterpret_cast<const float2 *>(Ph + t * PS);
#pragma unroll
                            for (int b = 0; b < kRB; ++b) {
                                const int r = r0 + b * P;
                                if (r < A.n_R) {
                                    const float2 cs = pt[r];   // (cos, sin)
                                    fre[b] = fmaf(cs.x, zr, fmaf(-cs.y, zi, fre[b]));
                                    fim[b] = fmaf(-cs.y, zr, fmaf(-cs.x, zi, fim[b]));
                                }
                            }
                        }
#pragma unroll
                        for (int b = 0; b < kRB; ++b) { dre[b] += (double)fre[b]; dim[b] += (double)fim[b]; }
                    }
#pragma unroll
                    for (int b = 0; b < kRB; ++b) {
                        const int r = r0 + b * P;
                        if (r < A.n_R) {
                            acc[N + r * NN + ij] += dre[b];
                            acc[N + half + r * NN + ij] += dim[b];
                        }
                    }
                }
            }
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
    const size_t smem = bwd_smem<N>(A.n_R, A.n_out).total;
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
