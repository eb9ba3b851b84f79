// Device code shared by the eigensolver and its adjoint: H(k) of the
// tight-binding model (Eq. (1) in hopping form) and a Hermitian eigensolver
// (Householder reduction to real tridiagonal form, implicit-shift QR).
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
};

// Lattice vector component reduced to [0, n): staged once per block so that
// the phase needs only 32-bit products below n^2 <= 2^24.
__device__ __forceinline__ int reduce_mod(int a, int n) {
    const int m = a % n;
    return m < 0 ? m + n : m;
}

// e^{i k.R} at grid point (x, y, z) for R given reduced mod (n1, n2, n3):
// 2 pi k.R is reduced exactly with integer arithmetic, m_i = (x_i R_i) mod n_i,
// before the single-precision sin/cos.
__device__ __forceinline__ void phase(const int *R, int x, int y, int z, int n1, int n2, int n3,
                                      float &sn, float &cs) {
    const int m0 = (x * R[0]) % n1;
    const int m1 = (y * R[1]) % n2;
    const int m2 = (z * R[2]) % n3;
    const float frac = (float)m0 / n1 + (float)m1 / n2 + (float)m2 / n3;
    sincospif(2.0f * frac, &sn, &cs);
}

// H(k) at grid point (x, y, z) from the model staged in shared memory
// (s_par: onsite[N], Re t[n_R][N][N], Im t[n_R][N][N]; s_R: R[n_R][3] reduced
// mod (n1, n2, n3));
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

namespace tetra {
namespace eigdetail {

// Hermitian eigensolver by Householder reduction to real tridiagonal form and
// implicit-shift QR (Wilkinson shift), eigenvectors accumulated. Every array
// index is a compile-time constant after unrolling, so the matrices live in
// registers; only the QR iteration counts are data-dependent (runtime loops
// around fixed-size code).
template <int N>
struct Herm {
    float ar[N][N], ai[N][N];   // lower triangle of A used (i >= j)
    float qr[N][N], qi[N][N];   // unitary Q, A = Q T Q^H; then the eigenvectors (columns)
    float g[N][N];              // real orthogonal G of the QR phase, T = G diag(d) G^T
    float d[N], e[N];           // real tridiagonal T: diagonal, sub-diagonal e[0..N-2]
};

// A (lower triangle) -> d, e real and Q with A = Q T Q^H.
// Step k reflects x = A[k+1..N-1][k] onto alpha e_1 with H = I - 2 u u^H,
// alpha = -(x_0/|x_0|) |x| (no cancellation in v_0 = x_0 - alpha), applies
// A <- H A H to the trailing block as A -= 2 (u w^H + w u^H), w = p - (u^H p) u,
// p = A u, and Q <- Q H. Columns whose entries below the sub-diagonal are at
// the FP32 resolution of ||A|| are left as they are (those entries dropped).
template <int N>
__device__ __forceinline__ void householder_tridiag(Herm<N> &M) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) { M.qr[i][j] = (i == j) ? 1.f : 0.f; M.qi[i][j] = 0.f; }
    float fro = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        fro = fmaf(M.ar[i][i], M.ar[i][i], fro);
#pragma unroll
        for (int j = 0; j < i; ++j) fro += 2.f * (M.ar[i][j] * M.ar[i][j] + M.ai[i][j] * M.ai[i][j]);
    }
    const float drop2 = 3.6e-15f * fro + 1e-36f;   // (6e-8 ||A||_F)^2
    float er[N], ei[N];
#pragma unroll
    for (int k = 0; k + 2 < N; ++k) {
        float sig = 0.f;
#pragma unroll
        for (int j = k + 2; j < N; ++j) sig += M.ar[j][k] * M.ar[j][k] + M.ai[j][k] * M.ai[j][k];
        const float x0r = M.ar[k + 1][k], x0i = M.ai[k + 1][k];
        const float ax0 = sqrtf(x0r * x0r + x0i * x0i);
        const bool act = sig > drop2;
        const float xn = sqrtf(ax0 * ax0 + sig);
        const float ia = ax0 > 0.f ? 1.f / ax0 : 0.f;
        const float phr = ax0 > 0.f ? x0r * ia : 1.f, phi = ax0 > 0.f ? x0i * ia : 0.f;
        const float t0 = ax0 + xn;
        const float iv = act ? rsqrtf(t0 * t0 + sig) : 0.f;
        er[k] = act ? -phr * xn : x0r;
        ei[k] = act ? -phi * xn : x0i;
        // u over indices k+1 .. N-1 (stored at position i)
        float ur[N], ui[N];
        ur[k + 1] = phr * t0 * iv;
        ui[k + 1] = phi * t0 * iv;
#pragma unroll
        for (int j = k + 2; j < N; ++j) { ur[j] = M.ar[j][k] * iv; ui[j] = M.ai[j][k] * iv; }
        // p = A_s u (A_s Hermitian, lower storage)
        float pr[N], pi[N];
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int j = k + 1; j < N; ++j) {
                float a_r, a_i;   // A[i][j]
                if (i >= j) { a_r = M.ar[i][j]; a_i = M.ai[i][j]; }
                else { a_r = M.ar[j][i]; a_i = -M.ai[j][i]; }
                if (i == j) a_i = 0.f;
                sr = fmaf(a_r, ur[j], fmaf(-a_i, ui[j], sr));
                si = fmaf(a_r, ui[j], fmaf(a_i, ur[j], si));
            }
            pr[i] = sr;
            pi[i] = si;
        }
        float K = 0.f;   // Re(u^H p)
#pragma unroll
        for (int i = k + 1; i < N; ++i) K = fmaf(ur[i], pr[i], fmaf(ui[i], pi[i], K));
        float wr[N], wi[N];
#pragma unroll
        for (int i = k + 1; i < N; ++i) { wr[i] = fmaf(-K, ur[i], pr[i]); wi[i] = fmaf(-K, ui[i], pi[i]); }
        // A_s -= 2 (u w^H + w u^H), lower triangle
#pragma unroll
        for (int i = k + 1; i < N; ++i)
#pragma unroll
            for (int j = k + 1; j <= i; ++j) {
                // u_i conj(w_j) + w_i conj(u_j)
                const float cr = ur[i] * wr[j] + ui[i] * wi[j] + wr[i] * ur[j] + wi[i] * ui[j];
                const float ci = ui[i] * wr[j] - ur[i] * wi[j] + wi[i] * ur[j] - wr[i] * ui[j];
                M.ar[i][j] = fmaf(-2.f, cr, M.ar[i][j]);
                if (i != j) M.ai[i][j] = fmaf(-2.f, ci, M.ai[i][j]);
            }
        // Q[:, k+1..] <- Q[:, k+1..] (I - 2 u u^H)
#pragma unroll
        for (int r = 0; r < N; ++r) {
            float tr = 0.f, ti = 0.f;   // (Q u)_r
#pragma unroll
            for (int j = k + 1; j < N; ++j) {
                tr = fmaf(M.qr[r][j], ur[j], fmaf(-M.qi[r][j], ui[j], tr));
                ti = fmaf(M.qr[r][j], ui[j], fmaf(M.qi[r][j], ur[j], ti));
            }
#pragma unroll
            for (int j = k + 1; j < N; ++j) {
                // Q_rj -= 2 t_r conj(u_j)
                M.qr[r][j] = fmaf(-2.f, tr * ur[j] + ti * ui[j], M.qr[r][j]);
                M.qi[r][j] = fmaf(-2.f, ti * ur[j] - tr * ui[j], M.qi[r][j]);
            }
        }
    }
    if constexpr (N > 1) {
        er[N - 2] = M.ar[N - 1][N - 2];
        ei[N - 2] = M.ai[N - 1][N - 2];
    }
#pragma unroll
    for (int k = 0; k < N; ++k) M.d[k] = M.ar[k][k];
    // unitary diagonal scaling that makes the sub-diagonal real and >= 0:
    // delta_{k+1} = delta_k e_k / |e_k|, Q <- Q diag(delta)
    float dr = 1.f, di = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (k > 0) {
#pragma unroll
            for (int r = 0; r < N; ++r) {
                const float a = M.qr[r][k], b = M.qi[r][k];
                M.qr[r][k] = a * dr - b * di;
                M.qi[r][k] = a * di + b * dr;
            }
        }
        if (k + 1 < N) {
            const float ae = sqrtf(er[k] * er[k] + ei[k] * ei[k]);
            const float ie = ae > 0.f ? 1.f / ae : 0.f;
            const float cr = ae > 0.f ? er[k] * ie : 1.f, ci = ae > 0.f ? ei[k] * ie : 0.f;
            const float nr = dr * cr - di * ci, ni = dr * ci + di * cr;
            dr = nr;
            di = ni;
            M.e[k] = ae;
        }
    }
}

// Implicit-shift QR on the real tridiagonal (d, e), the real rotations
// accumulated into G (started at the identity; the eigenvectors of H are the
// columns of Q G, formed once at the end). Deflation from the bottom: the
// block [l, m] with m = N-1 .. 1 and l the first row below the last
// negligible sub-diagonal entry; each step chases the bulge of one
// Wilkinson-shifted QR step down the block with Givens rotations
// R = [[c, s], [-s, c]] (T <- R^T T R, G <- G R).
template <int N>
__device__ __forceinline__ void tridiag_qr(Herm<N> &M) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) M.g[i][j] = (i == j) ? 1.f : 0.f;
    constexpr float kTol = 1.1920929e-07f;   // 2^-23
    float nrm = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) nrm = fmaxf(nrm, fabsf(M.d[k]));
#pragma unroll
    for (int k = 0; k + 1 < N; ++k) nrm = fmaxf(nrm, fabsf(M.e[k]));
    const float floor_ = 1e-30f * nrm + 1e-36f;
#pragma unroll
    for (int m = N - 1; m >= 1; --m) {
        for (int it = 0; it < 30; ++it) {
            if (fabsf(M.e[m - 1]) <= fmaf(kTol, fabsf(M.d[m - 1]) + fabsf(M.d[m]), floor_)) break;
            int l = 0;
#pragma unroll
            for (int j = 0; j + 1 < m; ++j)
                if (fabsf(M.e[j]) <= fmaf(kTol, fabsf(M.d[j]) + fabsf(M.d[j + 1]), floor_)) l = j + 1;
            const float dl = 0.5f * (M.d[m - 1] - M.d[m]);
            const float em = M.e[m - 1];
            const float hyp = sqrtf(fmaf(dl, dl, em * em));
            const float mu = M.d[m] - em * em / (dl + copysignf(hyp, dl));
            float g = 0.f;
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const bool act = k >= l;
                const float x = (k == l) ? M.d[k] - mu : (k > 0 ? M.e[k - 1] : 0.f);
                const float z = (k == l) ? M.e[k] : g;
                const float r2 = fmaf(x, x, z * z);
                const bool rot = act && r2 > 0.f;
                const float ir = rot ? rsqrtf(r2) : 0.f;
                const float c = rot ? x * ir : 1.f;
                const float s = rot ? -z * ir : 0.f;
                if (k > 0 && act && k > l) M.e[k - 1] = r2 * ir;
                const float a = M.d[k], b = M.d[k + 1], ee = M.e[k];
                const float cc = c * c, ss = s * s, cs = c * s;
                M.d[k] = fmaf(cc, a, fmaf(-2.f * cs, ee, ss * b));
                M.d[k + 1] = fmaf(ss, a, fmaf(2.f * cs, ee, cc * b));
                M.e[k] = fmaf(cs, a - b, (cc - ss) * ee);
                if (k + 1 < m) {
                    const float f = M.e[k + 1];
                    g = -s * f;
                    M.e[k + 1] = c * f;
                }
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    const float x = M.g[r][k], y = M.g[r][k + 1];
                    M.g[r][k] = fmaf(c, x, -s * y);
                    M.g[r][k + 1] = fmaf(s, x, c * y);
                }
            }
        }
    }
    // eigenvectors: Q <- Q G
#pragma unroll
    for (int r = 0; r < N; ++r) {
        float vr[N], vi[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                sr = fmaf(M.qr[r][k], M.g[k][n], sr);
                si = fmaf(M.qi[r][k], M.g[k][n], si);
            }
            vr[n] = sr;
            vi[n] = si;
        }
#pragma unroll
        for (int n = 0; n < N; ++n) {
            M.qr[r][n] = vr[n];
            M.qi[r][n] = vi[n];
        }
    }
}

}  // namespace eigdetail
}  // namespace tetra
