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

// (a b) mod n for 0 <= a, b < n <= 4096: the product is below 2^24, exact in
// FP32, so the quotient taken from a float product is off by at most one and
// the remainder is corrected into [0, n).
__device__ __forceinline__ int mulmod(int a, int b, int n, float inv_n) {
    const int ab = a * b;
    int m = ab - n * __float2int_rz(__int2float_rn(ab) * inv_n);
    m = m < 0 ? m + n : m;
    return m >= n ? m - n : m;
}

// Grid extents and their reciprocals, for the phases.
struct Grid3 {
    int n1, n2, n3;
    float i1, i2, i3;
};
__device__ __forceinline__ Grid3 grid3(int n1, int n2, int n3) {
    return Grid3{n1, n2, n3, 1.f / n1, 1.f / n2, 1.f / n3};
}

// e^{i k.R} at grid point (x, y, z) for R given reduced mod (n1, n2, n3):
// 2 pi k.R is reduced exactly with integer arithmetic, m_i = (x_i R_i) mod n_i,
// before the single-precision sin/cos.
__device__ __forceinline__ void phase(const int *R, int x, int y, int z, const Grid3 &g, float &sn,
                                      float &cs) {
    const int m0 = mulmod(x, R[0], g.n1, g.i1);
    const int m1 = mulmod(y, R[1], g.n2, g.i2);
    const int m2 = mulmod(z, R[2], g.n3, g.i3);
    const float frac = (float)m0 * g.i1 + (float)m1 * g.i2 + (float)m2 * g.i3;
    sincospif(2.0f * frac, &sn, &cs);
}

// Upper-triangle entries (i <= j) of an N x N matrix, row by row.
template <int N>
__host__ __device__ constexpr int n_upper() { return N * (N + 1) / 2; }

// The model as build_h reads it, staged in shared memory by every thread of
// the block: s_on[N] on-site energies; s_hop[n_R][n_upper] per hopping r and
// upper-triangle pair (i, j) the sums and differences of t_ij and t_ji,
// {Re(t_ij + t_ji), Im(t_ij + t_ji), Re(t_ij - t_ji), Im(t_ij - t_ji)}
// (params: onsite[N], Re t[n_R][N][N], Im t[n_R][N][N]); s_R[n_R][3] the
// lattice vectors reduced mod (n1, n2, n3).
template <int N>
__device__ __forceinline__ void stage_model(const float *params, const int *R, int n_R, int n1,
                                            int n2, int n3, float *s_on, float4 *s_hop, int *s_R) {
    constexpr int NP = n_upper<N>();
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_on[i] = params[i];
    const float *tre = params + N, *tim = params + N + n_R * N * N;
    for (int idx = threadIdx.x; idx < n_R * NP; idx += blockDim.x) {
        const int r = idx / NP;
        int i = 0, rem = idx - r * NP;
        while (rem >= N - i) { rem -= N - i; ++i; }
        const int j = i + rem;
        const float ar = tre[r * N * N + i * N + j], ai = tim[r * N * N + i * N + j];
        const float br = tre[r * N * N + j * N + i], bi = tim[r * N * N + j * N + i];
        s_hop[idx] = make_float4(ar + br, ai + bi, ar - br, ai - bi);
    }
    for (int i = threadIdx.x; i < 3 * n_R; i += blockDim.x)
        s_R[i] = reduce_mod(R[i], i % 3 == 0 ? n1 : (i % 3 == 1 ? n2 : n3));
}

// H(k) at grid point (x, y, z) from the staged model (stage_model), upper
// triangle into M. Term r adds t_ij e^{i th} + conj(t_ji) e^{-i th}
// = (S_re c - S_im s) + i (D_re s + D_im c), th = k.R_r, S = t_ij + t_ji,
// D = t_ij - t_ji.
template <int N>
__device__ __forceinline__ void build_h(Mat<N> &M, const float *s_on, const float4 *s_hop,
                                        const int *s_R, int n_R, int x, int y, int z,
                                        const Grid3 &g) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i; j < N; ++j) { M.hr[i][j] = (i == j) ? s_on[i] : 0.f; M.hi[i][j] = 0.f; }
    for (int r = 0; r < n_R; ++r) {
        float sn, cs;
        phase(s_R + 3 * r, x, y, z, g, sn, cs);
        const float4 *h = s_hop + r * n_upper<N>();
#pragma unroll
        for (int i = 0, q = 0; i < N; ++i)
#pragma unroll
            for (int j = i; j < N; ++j, ++q) {
                const float4 t = h[q];
                M.hr[i][j] = fmaf(t.x, cs, fmaf(-t.y, sn, M.hr[i][j]));
                M.hi[i][j] = fmaf(t.z, sn, fmaf(t.w, cs, M.hi[i][j]));
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
    float ur[N][N], ui[N][N];   // reflector k (k <= N-3) in row k, entries k+1 .. N-1
    float sr[N], si[N];         // unitary diagonal scaling delta
    float g[N][N];              // real orthogonal G of the QR phase, T = G diag(d) G^T
    float d[N], e[N];           // real tridiagonal T: diagonal, sub-diagonal e[0..N-2]
    float qr[N][N], qi[N][N];   // eigenvectors (columns), when formed by eigenvectors()
};

// A (lower triangle) -> d, e real and Q = H_0 H_1 ... H_{N-3} diag(delta) with
// A = Q T Q^H; the reflectors H_k = I - 2 u_k u_k^H and delta are kept, Q is
// not formed. Step k reflects x = A[k+1..N-1][k] onto alpha e_1,
// alpha = -(x_0/|x_0|) |x| (no cancellation in v_0 = x_0 - alpha), and applies
// A <- H A H to the trailing block as A -= 2 (u w^H + w u^H), w = p - (u^H p) u,
// p = A u. Columns whose entries below the sub-diagonal are at the FP32
// resolution of ||A|| are left as they are (those entries dropped; u_k = 0).
template <int N>
__device__ __forceinline__ void householder_tridiag(Herm<N> &M) {
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
#pragma unroll
        for (int j = k + 1; j < N; ++j) { M.ur[k][j] = ur[j]; M.ui[k][j] = ui[j]; }
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
    }
    if constexpr (N > 1) {
        er[N - 2] = M.ar[N - 1][N - 2];
        ei[N - 2] = M.ai[N - 1][N - 2];
    }
#pragma unroll
    for (int k = 0; k < N; ++k) M.d[k] = M.ar[k][k];
    // unitary diagonal scaling that makes the sub-diagonal real and >= 0:
    // delta_0 = 1, delta_{k+1} = delta_k e_k / |e_k|
    float dr = 1.f, di = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        M.sr[k] = dr;
        M.si[k] = di;
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
// columns of Q G, formed by eigvec_column). Deflation from the bottom: the
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
}

// x <- H_0 (H_1 (... H_{N-3} x)): the reflectors applied last to first as
// x <- x - 2 u (u^H x).
template <int N>
__device__ __forceinline__ void apply_reflectors(const Herm<N> &M, float (&xr)[N], float (&xi)[N]) {
#pragma unroll
    for (int k = N - 3; k >= 0; --k) {
        float tr = 0.f, ti = 0.f;   // u^H x
#pragma unroll
        for (int j = k + 1; j < N; ++j) {
            tr = fmaf(M.ur[k][j], xr[j], fmaf(M.ui[k][j], xi[j], tr));
            ti = fmaf(M.ur[k][j], xi[j], fmaf(-M.ui[k][j], xr[j], ti));
        }
        tr *= 2.f;
        ti *= 2.f;
#pragma unroll
        for (int j = k + 1; j < N; ++j) {
            xr[j] = fmaf(-M.ur[k][j], tr, fmaf(M.ui[k][j], ti, xr[j]));
            xi[j] = fmaf(-M.ur[k][j], ti, fmaf(-M.ui[k][j], tr, xi[j]));
        }
    }
}

// Eigenvector n of H: column n of Q G = H_0 (H_1 (... H_{N-3} (diag(delta) G e_n))).
template <int N>
__device__ __forceinline__ void eigvec_column(const Herm<N> &M, int n, float (&xr)[N], float (&xi)[N]) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
        xr[r] = M.sr[r] * M.g[r][n];
        xi[r] = M.si[r] * M.g[r][n];
    }
    apply_reflectors<N>(M, xr, xi);
}

// All eigenvectors into M.qr / M.qi (column n = eigenvector of d[n]).
template <int N>
__device__ __forceinline__ void eigenvectors(Herm<N> &M) {
#pragma unroll
    for (int n = 0; n < N; ++n) {
        float xr[N], xi[N];
        eigvec_column<N>(M, n, xr, xi);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            M.qr[r][n] = xr[r];
            M.qi[r][n] = xi[r];
        }
    }
}

}  // namespace eigdetail
}  // namespace tetra
