// Device code shared by the eigensolver and its adjoint: H(k) of the
// tight-binding model (Eq. (1) in hopping form) and cyclic complex Jacobi.
#pragma once
#include "tetra_internal.cuh"

namespace tetra {
namespace eigdetail {

constexpr int kEigThreads = 128;
constexpr int kMaxR = 32;

struct EigArgs {
    int n1, n2, n3, nx, ny;
    int z_off, nz;   // padded planes z_off .. z_off + nz - 1 are computed
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

// e^{i k.R} at grid point (x, y, z): 2 pi k.R reduced exactly with integer
// arithmetic, m_i = (x_i R_i) mod n_i, before the single-precision sin/cos.
__device__ __forceinline__ void phase(const int *R, int x, int y, int z, int n1, int n2, int n3,
                                      float &sn, float &cs) {
    auto md = [](long a, int n) { long m = a % n; return m < 0 ? m + n : m; };
    const long m0 = md((long)x * R[0], n1);
    const long m1 = md((long)y * R[1], n2);
    const long m2 = md((long)z * R[2], n3);
    const float frac = (float)m0 / n1 + (float)m1 / n2 + (float)m2 / n3;
    sincospif(2.0f * frac, &sn, &cs);
}

// H(k) at grid point (x, y, z) from the model staged in shared memory
// (s_par: onsite[N], Re t[n_R][N][N], Im t[n_R][N][N]; s_R: R[n_R][3]);
// upper triangle into M.
template <int N>
__device__ __forceinline__ void build_h(Mat<N> &M, const float *s_par, const int *s_R, int n_R,
                                        int x, int y, int z, int n1, int n2, int n3) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) { M.hr[i][j] = (i == j) ? s_par[i] : 0.f; M.hi[i][j] = 0.f; }
    const float *tre = s_par + N;
    const float *tim = s_par + N + n_R * N * N;
    for (int r = 0; r < n_R; ++r) {
        float sn, cs;
        phase(s_R + 3 * r, x, y, z, n1, n2, n3, sn, cs);
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
}

}  // namespace eigdetail
}  // namespace tetra
