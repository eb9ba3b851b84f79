// Adjoint of the bin-mode DOS (not in the paper): given g = dL/dDOS[s][i] for
// DOS_s[i] = sum_{T,n} sum_l b_{l,s} [w_l(e_{i+1}) - w_l(e_i)] / (e_{i+1} - e_i),
// computes dL/db and dL/deps at every k-point.
//
// One thread owns one (grid point, band): it visits the 24 tetrahedra that
// have the point as a corner (in a fixed order, so the float sums are
// deterministic without atomics), re-sorts each one and, for every bin the
// tetrahedron overlaps, evaluates the corner weights of Sec. II.C together
// with their derivatives with respect to the energy of the thread's own corner
// (forward mode, one tangent, carried through the paper's formulas with the
// reciprocal energy differences formed once per tetrahedron). The point then collects
//   dL/db_{p,s}  += g_si dW_l(p)/dE_i
//   dL/deps_p    += sum_s g_si sum_l b_{l,s} dW_l/de_{l(p)}      (bin averages)
#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kBwdThreads = 128;

// A value and its derivative along one direction: the energy of the sorted
// corner that holds the thread's own grid point (forward-mode AD with one
// tangent; the other three corner energies are constants).
struct F1 {
    float v, d;
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1{a.v * b.v, fmaf(a.d, b.v, a.v * b.d)}; }
__device__ __forceinline__ F1 operator*(float s, F1 a) { return F1{s * a.v, s * a.d}; }
__device__ __forceinline__ F1 operator-(float s, F1 a) { return F1{s - a.v, -a.d}; }

// Per-tetrahedron constants: the sorted corner energies with their tangents
// (1 for the differentiated corner, 0 otherwise) and the reciprocal energy
// differences 1/E_ab with theirs (d(1/x) = -dx/x^2). A difference that is
// not positive gets 0: no region that reads it is ever entered then (the
// regions are half-open, so every executed branch has positive denominators).
struct TetD {
    F1 e1, e2, e3, e4;
    F1 r21, r31, r41, r32, r42, r43;
};
__device__ __forceinline__ F1 rcp_diff(F1 a, F1 b) {   // 1 / (a - b)
    const float x = a.v - b.v;
    const float r = x > 0.f ? __fdividef(1.0f, x) : 0.f;
    return F1{r, -(a.d - b.d) * r * r};
}
__device__ __forceinline__ void tetd_setup(TetD &T, const float e[4], int r_my) {
    T.e1 = F1{e[0], r_my == 0 ? 1.f : 0.f};
    T.e2 = F1{e[1], r_my == 1 ? 1.f : 0.f};
    T.e3 = F1{e[2], r_my == 2 ? 1.f : 0.f};
    T.e4 = F1{e[3], r_my == 3 ? 1.f : 0.f};
    T.r21 = rcp_diff(T.e2, T.e1); T.r31 = rcp_diff(T.e3, T.e1); T.r41 = rcp_diff(T.e4, T.e1);
    T.r32 = rcp_diff(T.e3, T.e2); T.r42 = rcp_diff(T.e4, T.e2); T.r43 = rcp_diff(T.e4, T.e3);
}

// Corner weights w_l(E) (Sec. II.C, all five cases) with their derivatives
// along the tangent of T; f = V_T/(4 V_G). Regions are taken half-open as in
// the forward kernel.
__device__ __forceinline__ void weights_tan(const TetD &T, float E, float f, F1 w[4]) {
    if (E <= T.e1.v) {
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] = F1{0.f, 0.f};
    } else if (E >= T.e4.v) {
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] = F1{f, 0.f};
    } else if (E <= T.e2.v) {
        const F1 x = E - T.e1;
        const F1 C = f * (((x * x) * x) * ((T.r21 * T.r31) * T.r41));
        const F1 S = T.r21 + T.r31 + T.r41;
        const F1 Cx = C * x;
        w[0] = C * (4.f - x * S);
        w[1] = Cx * T.r21;
        w[2] = Cx * T.r31;
        w[3] = Cx * T.r41;
    } else if (E <= T.e3.v) {
        const F1 a = E - T.e1, bq = E - T.e2, c = T.e3 - F1{E, 0.f}, dd = T.e4 - F1{E, 0.f};
        const F1 r3141 = T.r31 * T.r41;
        const F1 C1 = f * ((a * a) * r3141);
        const F1 C2 = f * (((a * bq) * c) * (r3141 * T.r32));
        const F1 C3 = f * (((bq * bq) * dd) * ((T.r32 * T.r41) * T.r42));
        const F1 C12 = C1 + C2, C23 = C2 + C3, C123 = C12 + C3;
        w[0] = C1 + (C12 * c) * T.r31 + (C123 * dd) * T.r41;
        w[1] = C123 + (C23 * c) * T.r32 + (C3 * dd) * T.r42;
        w[2] = (C12 * a) * T.r31 + (C23 * bq) * T.r32;
        w[3] = (C123 * a) * T.r41 + (C3 * bq) * T.r42;
    } else {
        const F1 y = T.e4 - F1{E, 0.f};
        const F1 C = f * (((y * y) * y) * ((T.r41 * T.r42) * T.r43));
        const F1 S = T.r41 + T.r42 + T.r43;
        const F1 Cy = C * y;
        w[0] = f - Cy * T.r41;
        w[1] = f - Cy * T.r42;
        w[2] = f - Cy * T.r43;
        w[3] = f - C * (4.f - S * y);
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
    int staged;              // grad_dos, edges and 1/widths copied to shared memory
};

// Shared-memory bytes of the staged bin data, or 0 when it does not fit the
// budget that keeps three 128-thread blocks per SM.
inline size_t bwd_stage_bytes(int n_orb, int n_bins) {
    const size_t b = sizeof(float) * ((size_t)n_orb * n_bins + 2 * (size_t)n_bins + 1);
    return b <= 64 * 1024 ? b : 0;
}

template <int NORB, typename WT>
__global__ void __launch_bounds__(kBwdThreads) tetra_dos_bwd_kernel(const BwdArgs A) {
    extern __shared__ float s_bins[];   // staged: grad_dos, edges, 1/widths
    const float *gd = A.grad_dos, *ed = A.edges, *siw = nullptr;
    if (A.staged) {
        const int ng = A.n_orb * A.n_bins;
        for (int i = threadIdx.x; i < ng; i += blockDim.x) s_bins[i] = A.grad_dos[i];
        for (int i = threadIdx.x; i <= A.n_bins; i += blockDim.x) s_bins[ng + i] = A.edges[i];
        for (int i = threadIdx.x; i < A.n_bins; i += blockDim.x)
            s_bins[ng + A.n_bins + 1 + i] = 1.0f / (A.edges[i + 1] - A.edges[i]);
        __syncthreads();
        gd = s_bins;
        ed = s_bins + ng;
        siw = s_bins + ng + A.n_bins + 1;
    }
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
    const float om0 = ed[0];
    const float inv_de = (float)A.n_bins / (ed[A.n_bins] - om0);
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
            while (lo > 0 && ed[lo] > e[0]) --lo;
            while (lo < A.n_bins && ed[lo + 1] <= e[0]) ++lo;
            while (hi < A.n_bins - 1 && (ed[hi + 1] < e[3] || ed[hi + 1] <= e[0])) ++hi;
            while (hi >= 0 && !(ed[hi] < e[3] || ed[hi] <= e[0])) --hi;
            if (lo > hi) continue;
            // orbital weights of the four corners, in sorted order
            float b[4][NORB];
#pragma unroll
            for (int r = 0; r < 4; ++r)
                load_weights<NORB, WT>(W + (long)pt[slot[r]] * A.w_stride + (long)n * A.n_orb, A.n_orb, b[r]);
            TetD TD;
            tetd_setup(TD, e, r_my);
            // the own corner's weight, selected without a runtime register index
            auto own = [&](const F1 (&w)[4]) {
                return r_my == 0 ? w[0].v : r_my == 1 ? w[1].v : r_my == 2 ? w[2].v : w[3].v;
            };
            F1 wl[4], wu[4];
            weights_tan(TD, ed[lo], A.f, wl);
            for (int i = lo; i <= hi; ++i) {
                weights_tan(TD, ed[i + 1], A.f, wu);
                const float iw = siw ? siw[i] : 1.0f / (ed[i + 1] - ed[i]);
                // dW_l/dE-bin for this corner, and sum_l b_l dW_l/de_{r_my}
                const float dWmy = (own(wu) - own(wl)) * iw;
                float dw[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) dw[r] = wu[r].d - wl[r].d;
#pragma unroll
                for (int s = 0; s < NORB; ++s) {
                    if (s >= A.n_orb) continue;
                    const float g = gd[(long)s * A.n_bins + i];
                    acc_w[s] = fmaf(g, dWmy, acc_w[s]);
                    float de = 0.f;
#pragma unroll
                    for (int r = 0; r < 4; ++r) de = fmaf(b[r][s], dw[r], de);
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
    const size_t smem = A.staged ? bwd_stage_bytes(A.n_orb, A.n_bins) : 0;
    auto go = [&](auto kfn) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kfn<<<grid, kBwdThreads, smem, stream>>>(A);
        return cudaGetLastError();
    };
    switch (P.d.weight_dtype) {
        case TETRA_F16: return go(tetra_dos_bwd_kernel<NORB, __half>);
        case TETRA_BF16: return go(tetra_dos_bwd_kernel<NORB, __nv_bfloat16>);
        default: return go(tetra_dos_bwd_kernel<NORB, float>);
    }
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
    A.staged = bwd_stage_bytes(A.n_orb, A.n_bins) > 0;
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
