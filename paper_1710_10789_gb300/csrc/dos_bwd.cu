// Adjoint of the bin-mode DOS (not in the paper): given g = dL/dDOS[s][i] for
// DOS_s[i] = sum_{T,n} sum_l b_{l,s} [w_l(e_{i+1}) - w_l(e_i)] / (e_{i+1} - e_i),
// computes dL/db and dL/deps at every k-point.
//
// One thread owns one (grid point, band): it visits the 24 tetrahedra that
// have the point as a corner (in a fixed order, so the float sums are
// deterministic without atomics), re-sorts each one and, for every bin the
// tetrahedron overlaps, evaluates the corner weights of Sec. II.C together
// with their derivatives with respect to the four sorted corner energies by
// forward-mode dual numbers (value + 4 tangents) carried through the paper's
// formulas. The point then collects
//   dL/db_{p,s}  += g_si dW_l(p)/dE_i
//   dL/deps_p    += sum_s g_si sum_l b_{l,s} dW_l/de_{l(p)}      (bin averages)
#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kBwdThreads = 128;

// value and derivatives with respect to the 4 sorted corner energies
struct D4 {
    float v, d[4];
};
__device__ __forceinline__ D4 dconst(float v) { D4 r; r.v = v; r.d[0] = r.d[1] = r.d[2] = r.d[3] = 0.f; return r; }
__device__ __forceinline__ D4 operator+(const D4 &a, const D4 &b) { D4 r; r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
__device__ __forceinline__ D4 operator-(const D4 &a, const D4 &b) { D4 r; r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
__device__ __forceinline__ D4 operator*(const D4 &a, const D4 &b) { D4 r; r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
__device__ __forceinline__ D4 operator*(float s, const D4 &a) { D4 r; r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = s * a.d[k]; return r; }
__device__ __forceinline__ D4 operator/(const D4 &a, const D4 &b) {
    const float ib = 1.0f / b.v;
    D4 r; r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}

// Corner weights w_l(E) (Sec. II.C, all five cases) with derivatives with
// respect to the sorted corner energies; f = V_T/(4 V_G). Regions are taken
// half-open as in the forward kernel.
__device__ void weights_dual(const float e[4], float E, float f, D4 w[4]) {
    D4 E1 = dconst(e[0]), E2 = dconst(e[1]), E3 = dconst(e[2]), E4 = dconst(e[3]);
    E1.d[0] = 1.f; E2.d[1] = 1.f; E3.d[2] = 1.f; E4.d[3] = 1.f;
    const D4 EE = dconst(E);
    if (E <= e[0]) {
        for (int l = 0; l < 4; ++l) w[l] = dconst(0.f);
    } else if (E >= e[3]) {
        for (int l = 0; l < 4; ++l) w[l] = dconst(f);
    } else if (E <= e[1]) {
        const D4 E21 = E2 - E1, E31 = E3 - E1, E41 = E4 - E1, x = EE - E1;
        const D4 C = f * (x * x * x) / (E21 * E31 * E41);
        const D4 S = dconst(1.f) / E21 + dconst(1.f) / E31 + dconst(1.f) / E41;
        w[0] = C * (dconst(4.f) - x * S);
        w[1] = C * x / E21;
        w[2] = C * x / E31;
        w[3] = C * x / E41;
    } else if (E <= e[2]) {
        const D4 E31 = E3 - E1, E41 = E4 - E1, E32 = E3 - E2, E42 = E4 - E2;
        const D4 a = EE - E1, bq = EE - E2, c = E3 - EE, dd = E4 - EE;
        const D4 C1 = f * (a * a) / (E31 * E41);
        const D4 C2 = f * (a * bq * c) / (E31 * E32 * E41);
        const D4 C3 = f * (bq * bq * dd) / (E32 * E41 * E42);
        w[0] = C1 + (C1 + C2) * c / E31 + (C1 + C2 + C3) * dd / E41;
        w[1] = C1 + C2 + C3 + (C2 + C3) * c / E32 + C3 * dd / E42;
        w[2] = (C1 + C2) * a / E31 + (C2 + C3) * bq / E32;
        w[3] = (C1 + C2 + C3) * a / E41 + C3 * bq / E42;
    } else {
        const D4 E41 = E4 - E1, E42 = E4 - E2, E43 = E4 - E3, y = E4 - EE;
        const D4 C = f * (y * y * y) / (E41 * E42 * E43);
        const D4 S = dconst(1.f) / E41 + dconst(1.f) / E42 + dconst(1.f) / E43;
        w[0] = dconst(f) - C * y / E41;
        w[1] = dconst(f) - C * y / E42;
        w[2] = dconst(f) - C * y / E43;
        w[3] = dconst(f) - C * (dconst(4.f) - S * y);
    }
}

// Table I corner labels minus one.
__constant__ int c_tab[6][4] = {{0, 1, 2, 5}, {1, 2, 3, 5}, {0, 2, 4, 5},
                                {2, 3, 5, 7}, {2, 4, 5, 6}, {2, 5, 6, 7}};

struct BwdArgs {
    int n1, n2, n3, nx, ny, nz, nb, n_orb, n_bins;
    int eps_stride, w_stride;
    float f;   // V_T / (4 V_G)
    const float *eps;
    const void *w;
    const float *edges;      // n_bins + 1
    const float *grad_dos;   // [n_orb][n_bins]
    float *geps, *gw;
};

template <int NORB, typename WT>
__global__ void __launch_bounds__(kBwdThreads) tetra_dos_bwd_kernel(const BwdArgs A) {
    const long P = (long)A.nx * A.ny * A.nz;
    const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (gid >= P * A.nb) return;
    const int n = (int)(gid % A.nb);
    const long p = gid / A.nb;
    const int px = (int)(p % A.nx), py = (int)((p / A.nx) % A.ny), pz = (int)(p / ((long)A.nx * A.ny));
    const WT *W = static_cast<const WT *>(A.w);
    float *ge = A.geps + p * A.eps_stride + n;
    float *gw = A.gw + p * A.w_stride + (long)n * A.n_orb;
    if (n == 0) {   // the point's padding entries are written too (zeros)
        for (int i = A.nb; i < A.eps_stride; ++i) A.geps[p * A.eps_stride + i] = 0.f;
        for (int i = A.nb * A.n_orb; i < A.w_stride; ++i) A.gw[p * A.w_stride + i] = 0.f;
    }
    if (px >= A.n1 || py >= A.n2 || pz >= A.n3) {   // halo copy: no own gradient
        *ge = 0.f;
        for (int s = 0; s < A.n_orb; ++s) gw[s] = 0.f;
        return;
    }
    const float om0 = A.edges[0];
    const float inv_de = (float)A.n_bins / (A.edges[A.n_bins] - om0);
    float acc_e = 0.f;
    float acc_w[NORB];
#pragma unroll
    for (int s = 0; s < NORB; ++s) acc_w[s] = 0.f;
    // the point is corner c of the cube whose origin is (point - offset(c))
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const int cx = (px - dx + A.n1) % A.n1, cy = (py - dy + A.n2) % A.n2, cz = (pz - dz + A.n3) % A.n3;
        for (int t = 0; t < 6; ++t) {
            int my = -1;
#pragma unroll
            for (int q = 0; q < 4; ++q) if (c_tab[t][q] == c) my = q;
            if (my < 0) continue;
            float e[4];
            int pt[4], slot[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cc = c_tab[t][q];
                const int x = cx + (cc & 1), y = cy + ((cc >> 1) & 1), z = cz + ((cc >> 2) & 1);
                pt[q] = x + A.nx * (y + A.ny * z);   // padded layout holds the periodic images
                e[q] = A.eps[(long)pt[q] * A.eps_stride + n];
                slot[q] = q;
            }
            // sort corners by energy, carrying their Table-I slot (stable for ties)
#pragma unroll
            for (int i = 1; i < 4; ++i)
#pragma unroll
                for (int j = i; j > 0; --j)
                    if (e[j] < e[j - 1]) {
                        const float te = e[j]; e[j] = e[j - 1]; e[j - 1] = te;
                        const int ts = slot[j]; slot[j] = slot[j - 1]; slot[j - 1] = ts;
                    }
            int r_my = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) if (slot[r] == my) r_my = r;
            // bins whose weight difference can be non-zero
            int lo = (int)floorf(fminf(fmaxf((e[0] - om0) * inv_de, -2.f), (float)A.n_bins + 2.f));
            int hi = (int)ceilf(fminf(fmaxf((e[3] - om0) * inv_de, -2.f), (float)A.n_bins + 2.f));
            lo = min(max(lo, 0), A.n_bins);
            hi = max(min(hi, A.n_bins - 1), -1);
            while (lo > 0 && A.edges[lo] > e[0]) --lo;
            while (lo < A.n_bins && A.edges[lo + 1] <= e[0]) ++lo;
            while (hi < A.n_bins - 1 && (A.edges[hi + 1] < e[3] || A.edges[hi + 1] <= e[0])) ++hi;
            while (hi >= 0 && !(A.edges[hi] < e[3] || A.edges[hi] <= e[0])) --hi;
            if (lo > hi) continue;
            // orbital weights of the four corners, in sorted order
            float b[4][NORB];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s = 0; s < NORB; ++s)
                    b[r][s] = (s < A.n_orb) ? to_f32<WT>(W[(long)pt[slot[r]] * A.w_stride + (long)n * A.n_orb + s]) : 0.f;
            D4 wl[4], wu[4];
            weights_dual(e, A.edges[lo], A.f, wl);
            for (int i = lo; i <= hi; ++i) {
                weights_dual(e, A.edges[i + 1], A.f, wu);
                const float iw = 1.0f / (A.edges[i + 1] - A.edges[i]);
                // dW_l/dE-bin for this corner, and sum_l b_l dW_l/de_{r_my}
                const float dWmy = (wu[r_my].v - wl[r_my].v) * iw;
#pragma unroll
                for (int s = 0; s < NORB; ++s) {
                    if (s >= A.n_orb) continue;
                    const float g = A.grad_dos[(long)s * A.n_bins + i];
                    acc_w[s] = fmaf(g, dWmy, acc_w[s]);
                    float de = 0.f;
#pragma unroll
                    for (int r = 0; r < 4; ++r) de = fmaf(b[r][s], wu[r].d[r_my] - wl[r].d[r_my], de);
                    acc_e = fmaf(g * iw, de, acc_e);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) wl[r] = wu[r];
            }
        }
    }
    *ge = acc_e;
#pragma unroll
    for (int s = 0; s < NORB; ++s) if (s < A.n_orb) gw[s] = acc_w[s];
}

template <int NORB>
cudaError_t launch_bwd_n(const Plan &P, const BwdArgs &A, cudaStream_t stream) {
    const long total = (long)A.nx * A.ny * A.nz * A.nb;
    const int grid = (int)((total + kBwdThreads - 1) / kBwdThreads);
    switch (P.d.weight_dtype) {
        case TETRA_F16: tetra_dos_bwd_kernel<NORB, __half><<<grid, kBwdThreads, 0, stream>>>(A); break;
        case TETRA_BF16: tetra_dos_bwd_kernel<NORB, __nv_bfloat16><<<grid, kBwdThreads, 0, stream>>>(A); break;
        default: tetra_dos_bwd_kernel<NORB, float><<<grid, kBwdThreads, 0, stream>>>(A); break;
    }
    return cudaGetLastError();
}

}  // namespace

size_t dos_backward_workspace(const Plan &) { return kStatusBytes; }

tetra_status_t launch_dos_backward(const Plan &P, const float *eps, const void *w,
                                   const float *omega, const float *grad_dos, float *grad_eps,
                                   float *grad_w, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (ws_bytes < kStatusBytes) return TETRA_ENOMEM;
    if (P.z0 != 0 || P.z1 != P.d.n3) return TETRA_EUNSUPPORTED;   // whole grid only
    BwdArgs A;
    A.n1 = P.d.n1; A.n2 = P.d.n2; A.n3 = P.d.n3; A.nx = P.nx; A.ny = P.ny; A.nz = P.nz;
    A.nb = P.d.n_bands; A.n_orb = P.d.n_orb; A.n_bins = P.d.n_omega;
    A.eps_stride = P.eps_stride; A.w_stride = P.w_stride;
    A.f = (float)(0.25 / (6.0 * (double)P.d.n1 * (double)P.d.n2 * (double)P.d.n3));
    A.eps = eps; A.w = w; A.edges = omega; A.grad_dos = grad_dos; A.geps = grad_eps; A.gw = grad_w;
    if (cudaMemsetAsync(ws, 0, kStatusBytes, stream) != cudaSuccess) return TETRA_ECUDA;
    cudaError_t e;
    const int no = P.d.n_orb;
    if (no <= 1) e = launch_bwd_n<1>(P, A, stream);
    else if (no <= 2) e = launch_bwd_n<2>(P, A, stream);
    else if (no <= 4) e = launch_bwd_n<4>(P, A, stream);
    else if (no <= 8) e = launch_bwd_n<8>(P, A, stream);
    else e = launch_bwd_n<16>(P, A, stream);
    return e == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace tetra
