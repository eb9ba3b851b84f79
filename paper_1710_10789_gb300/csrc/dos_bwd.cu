// Adjoint of the bin-mode DOS (not in the paper): given g = dL/dDOS[s][i] for
// DOS_s[i] = sum_{T,n} sum_l b_{l,s} [w_l(e_{i+1}) - w_l(e_i)] / (e_{i+1} - e_i),
// computes dL/db and dL/deps at every k-point.
//
// One thread owns one (cube, band). For each of the cube's six tetrahedra it
// sorts the corners once and, for every bin the tetrahedron overlaps,
// evaluates the corner weights of Sec. II.C together with their derivatives
// along all four corner energies (forward mode with four tangents; the six
// reciprocal energy differences and their tangents are formed once per
// tetrahedron, so the paper's formulas run on multiplies only). Then
//   dL/db_{l,s}  += g_si dW_l/dE_i                                (bin averages)
//   dL/de_r      += sum_i (1/width_i) sum_l [sum_s g_si b_{l,s}] d(dW_l)/de_r
// for the sorted corners l, r, added into the cube's eight corner
// accumulators (thread-private shared memory). Cubes are processed in eight
// launches, one per parity class of the cube origin (x, y, z mod 2): two
// cubes of one class share no point of the padded layout (the layout holds
// the periodic images x = n1 etc. as separate points), so each class adds its
// corner sums to the gradient arrays without atomics. A last pass folds the
// periodic images onto the interior points. Every sum runs in a fixed order,
// so the result is deterministic.
//
// The kernel is bound by the latency of its loads and branches, not by its
// arithmetic: three blocks per SM (168 registers) hide more of it than two.
// To fit that register count, the third weight case runs through the first
// case's code on the mirrored tetrahedron, which also keeps a warp whose
// lanes sit in both outer cases on one path.
#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kBwdThreads = 128;

// A value and its derivatives along the four sorted corner energies.
struct F4 {
    float v, d[4];
};
__device__ __forceinline__ F4 operator+(const F4 &a, const F4 &b) {
    return F4{a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2], a.d[3] + b.d[3]}};
}
__device__ __forceinline__ F4 operator-(const F4 &a, const F4 &b) {
    return F4{a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2], a.d[3] - b.d[3]}};
}
__device__ __forceinline__ F4 operator*(const F4 &a, const F4 &b) {
    F4 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < 4; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
    return r;
}
__device__ __forceinline__ F4 operator*(float s, const F4 &a) {
    return F4{s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2], s * a.d[3]}};
}
__device__ __forceinline__ F4 operator-(float s, const F4 &a) {
    return F4{s - a.v, {-a.d[0], -a.d[1], -a.d[2], -a.d[3]}};
}
__device__ __forceinline__ F4 konst(float v) { return F4{v, {0.f, 0.f, 0.f, 0.f}}; }

// Per-tetrahedron constants: the sorted corner energies with their tangents
// (unit vectors) and the reciprocal energy differences 1/E_ab with theirs
// (d(1/x) = -dx/x^2). A difference that is not positive gets 0: no region
// that reads it is ever entered then (the regions are half-open, so every
// executed branch has positive denominators).
struct TetD {
    F4 e1, e2, e3, e4;
    F4 r21, r31, r41, r32, r42, r43;
};
__device__ __forceinline__ F4 rcp_diff(const F4 &a, const F4 &b) {   // 1 / (a - b)
    const float x = a.v - b.v;
    const float r = x > 0.f ? __fdividef(1.0f, x) : 0.f;
    const float r2 = r * r;
    return F4{r, {-(a.d[0] - b.d[0]) * r2, -(a.d[1] - b.d[1]) * r2, -(a.d[2] - b.d[2]) * r2,
                  -(a.d[3] - b.d[3]) * r2}};
}
__device__ __forceinline__ void tetd_setup(TetD &T, const float e[4]) {
    T.e1 = F4{e[0], {1.f, 0.f, 0.f, 0.f}};
    T.e2 = F4{e[1], {0.f, 1.f, 0.f, 0.f}};
    T.e3 = F4{e[2], {0.f, 0.f, 1.f, 0.f}};
    T.e4 = F4{e[3], {0.f, 0.f, 0.f, 1.f}};
    T.r21 = rcp_diff(T.e2, T.e1); T.r31 = rcp_diff(T.e3, T.e1); T.r41 = rcp_diff(T.e4, T.e1);
    T.r32 = rcp_diff(T.e3, T.e2); T.r42 = rcp_diff(T.e4, T.e2); T.r43 = rcp_diff(T.e4, T.e3);
}

// Corner weights w_l(E) (Sec. II.C, all five cases) with their derivatives
// along the four corner energies; f = V_T/(4 V_G). Regions are taken
// half-open as in the forward kernel.
__device__ __forceinline__ void weights4(const TetD &T, float E, float f, F4 w[4]) {
    if (E <= T.e1.v) {
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] = konst(0.f);
    } else if (E >= T.e4.v) {
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] = konst(f);
    } else if (E > T.e2.v && E <= T.e3.v) {
        const F4 a = konst(E) - T.e1, bq = konst(E) - T.e2, c = T.e3 - konst(E), dd = T.e4 - konst(E);
        const F4 r3141 = T.r31 * T.r41;
        const F4 C1 = f * ((a * a) * r3141);
        const F4 C2 = f * (((a * bq) * c) * (r3141 * T.r32));
        const F4 C3 = f * (((bq * bq) * dd) * ((T.r32 * T.r41) * T.r42));
        const F4 C12 = C1 + C2, C23 = C2 + C3, C123 = C12 + C3;
        w[0] = C1 + (C12 * c) * T.r31 + (C123 * dd) * T.r41;
        w[1] = C123 + (C23 * c) * T.r32 + (C3 * dd) * T.r42;
        w[2] = (C12 * a) * T.r31 + (C23 * bq) * T.r32;
        w[3] = (C123 * a) * T.r41 + (C3 * bq) * T.r42;
    } else {
        // E1 < E <= E2, or E3 < E < E4 as the first case of the mirrored
        // tetrahedron (energies -E4 <= -E3 <= -E2 <= -E1 at -E: distance
        // E4 - E, reciprocals 1/E43, 1/E42, 1/E41), whose weights are f minus
        // the original's in reverse corner order
        const bool mir = E > T.e2.v;
        const F4 x = mir ? T.e4 - konst(E) : konst(E) - T.e1;
        const F4 ra = mir ? T.r43 : T.r21, rb = mir ? T.r42 : T.r31;
        const F4 C = f * (((x * x) * x) * ((ra * rb) * T.r41));
        const F4 S = ra + rb + T.r41;
        const F4 Cx = C * x;
        const F4 u0 = C * (4.f - x * S), u1 = Cx * ra, u2 = Cx * rb, u3 = Cx * T.r41;
        w[0] = mir ? f - u3 : u0;
        w[1] = mir ? f - u2 : u1;
        w[2] = mir ? f - u1 : u2;
        w[3] = mir ? f - u0 : u3;
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
// 64 KB budget.
inline size_t bwd_stage_bytes(int n_orb, int n_bins) {
    const size_t b = sizeof(float) * ((size_t)n_orb * n_bins + 2 * (size_t)n_bins + 1);
    return b <= 64 * 1024 ? b : 0;
}

// Thread-private corner accumulators: (1 + n_orb) values for each of the
// cube's 8 corners, interleaved over the block's threads.
inline size_t bwd_scratch_bytes(int n_orb) { return sizeof(float) * (1 + (size_t)n_orb) * 8 * kBwdThreads; }

template <int NORB, typename WT>
__global__ void __launch_bounds__(kBwdThreads, 3) tetra_dos_bwd_kernel(const BwdArgs A, int px, int py, int pz) {
    extern __shared__ float s_mem[];
    const int ng = A.n_orb * A.n_bins;
    const size_t stage = A.staged ? (size_t)ng + 2 * (size_t)A.n_bins + 1 : 0;
    float *scr = s_mem + ((stage + 3) & ~size_t(3));   // [(1 + n_orb) * 8][blockDim]
    const float *gd = A.grad_dos, *ed = A.edges, *siw = nullptr;
    if (A.staged) {
        for (int i = threadIdx.x; i < ng; i += blockDim.x) s_mem[i] = A.grad_dos[i];
        for (int i = threadIdx.x; i <= A.n_bins; i += blockDim.x) s_mem[ng + i] = A.edges[i];
        for (int i = threadIdx.x; i < A.n_bins; i += blockDim.x)
            s_mem[ng + A.n_bins + 1 + i] = 1.0f / (A.edges[i + 1] - A.edges[i]);
        __syncthreads();
        gd = s_mem;
        ed = s_mem + ng;
        siw = s_mem + ng + A.n_bins + 1;
    }
    // cubes of this parity class: x = px, px + 2, ... < n1 (same for y, z)
    const int cxn = (A.n1 - px + 1) >> 1, cyn = (A.n2 - py + 1) >> 1, czn = (A.n3 - pz + 1) >> 1;
    const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (gid >= (long)cxn * cyn * czn * A.nb) return;
    const int n = (int)(gid % A.nb);
    const long cube = gid / A.nb;
    const int x = px + 2 * (int)(cube % cxn), y = py + 2 * (int)((cube / cxn) % cyn),
              z = pz + 2 * (int)(cube / ((long)cxn * cyn));
    const WT *W = static_cast<const WT *>(A.w);
    const int nv = 1 + A.n_orb;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int v = 0; v < nv * 8; ++v) scr[v * nt + tid] = 0.f;
    const float om0 = ed[0];
    const float inv_de = (float)A.n_bins / (ed[A.n_bins] - om0);
    for (int t = 0; t < 6; ++t) {
        float e[4];
        int pt[4], slot[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = c_tab[t][q];
            pt[q] = (x + (cc & 1)) + A.nx * ((y + ((cc >> 1) & 1)) + A.ny * (z + ((cc >> 2) & 1)));
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
        tetd_setup(TD, e);
        float acc_e[4] = {0.f, 0.f, 0.f, 0.f};
        float acc_w[4][NORB];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < NORB; ++s) acc_w[r][s] = 0.f;
        F4 wl[4], wu[4];
        weights4(TD, ed[lo], A.f, wl);
        for (int i = lo; i <= hi; ++i) {
            weights4(TD, ed[i + 1], A.f, wu);
            const float iw = siw ? siw[i] : 1.0f / (ed[i + 1] - ed[i]);
            float dW[4], h[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int l = 0; l < 4; ++l) dW[l] = (wu[l].v - wl[l].v) * iw;
#pragma unroll
            for (int s = 0; s < NORB; ++s) {
                if (s >= A.n_orb) continue;
                const float g = gd[(long)s * A.n_bins + i];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    acc_w[l][s] = fmaf(g, dW[l], acc_w[l][s]);
                    h[l] = fmaf(g, b[l][s], h[l]);
                }
            }
            // d(bin DOS contribution)/d(sorted corner energy r)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float de = 0.f;
#pragma unroll
                for (int l = 0; l < 4; ++l) de = fmaf(h[l], wu[l].d[r] - wl[l].d[r], de);
                acc_e[r] = fmaf(iw, de, acc_e[r]);
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) wl[l] = wu[l];
        }
        // add the sorted corners' sums to the cube-corner accumulators
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int c = c_tab[t][slot[r]];
            scr[(0 * 8 + c) * nt + tid] += acc_e[r];
#pragma unroll
            for (int s = 0; s < NORB; ++s)
                if (s < A.n_orb) scr[((1 + s) * 8 + c) * nt + tid] += acc_w[r][s];
        }
    }
    // this class's cubes share no point: plain read-modify-write
    for (int c = 0; c < 8; ++c) {
        const long p = (x + (c & 1)) + (long)A.nx * ((y + ((c >> 1) & 1)) + (long)A.ny * (z + (c >> 2)));
        A.geps[p * A.eps_stride + n] += scr[(0 * 8 + c) * nt + tid];
        float *gwp = A.gw + p * A.w_stride + (long)n * A.n_orb;
        for (int s = 0; s < A.n_orb; ++s) gwp[s] += scr[((1 + s) * 8 + c) * nt + tid];
    }
}

// Folds the periodic images (x = n1, y = n2, z = n3 in the padded layout) onto
// the interior point they copy and zeroes them: one thread per (interior
// point on a face x = 0, y = 0 or z = 0, band), images added in a fixed order.
// The face points are enumerated plane by plane: x = 0; y = 0 with x >= 1;
// z = 0 with x, y >= 1.
__global__ void tetra_dos_bwd_fold(const BwdArgs A) {
    const long fa = (long)A.n2 * A.n3, fb = (long)(A.n1 - 1) * A.n3, fc = (long)(A.n1 - 1) * (A.n2 - 1);
    const long gid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (gid >= (fa + fb + fc) * A.nb) return;
    const int n = (int)(gid % A.nb);
    long k = gid / A.nb;
    int x, y, z;
    if (k < fa) {                      // plane x = 0
        x = 0; y = (int)(k % A.n2); z = (int)(k / A.n2);
    } else if ((k -= fa) < fb) {       // plane y = 0, x >= 1
        x = 1 + (int)(k % (A.n1 - 1)); y = 0; z = (int)(k / (A.n1 - 1));
    } else {                           // plane z = 0, x, y >= 1
        k -= fb;
        x = 1 + (int)(k % (A.n1 - 1)); y = 1 + (int)(k / (A.n1 - 1)); z = 0;
    }
    const int mx = x == 0 ? 2 : 1, my = y == 0 ? 2 : 1, mz = z == 0 ? 2 : 1;
    const long p0 = x + (long)A.nx * (y + (long)A.ny * z);
    float se = A.geps[p0 * A.eps_stride + n];
    for (int iz = 0; iz < mz; ++iz)
        for (int iy = 0; iy < my; ++iy)
            for (int ix = 0; ix < mx; ++ix) {
                if (ix == 0 && iy == 0 && iz == 0) continue;
                const long q = (x + ix * A.n1) + (long)A.nx * ((y + iy * A.n2) + (long)A.ny * (z + iz * A.n3));
                se += A.geps[q * A.eps_stride + n];
                A.geps[q * A.eps_stride + n] = 0.f;
            }
    A.geps[p0 * A.eps_stride + n] = se;
    for (int s = 0; s < A.n_orb; ++s) {
        float sw = A.gw[p0 * A.w_stride + (long)n * A.n_orb + s];
        for (int iz = 0; iz < mz; ++iz)
            for (int iy = 0; iy < my; ++iy)
                for (int ix = 0; ix < mx; ++ix) {
                    if (ix == 0 && iy == 0 && iz == 0) continue;
                    const long q = (x + ix * A.n1) + (long)A.nx * ((y + iy * A.n2) + (long)A.ny * (z + iz * A.n3));
                    float *gq = A.gw + q * A.w_stride + (long)n * A.n_orb + s;
                    sw += *gq;
                    *gq = 0.f;
                }
        A.gw[p0 * A.w_stride + (long)n * A.n_orb + s] = sw;
    }
}

template <int NORB>
cudaError_t launch_bwd_n(const Plan &P, const BwdArgs &A, cudaStream_t stream) {
    const size_t stage = A.staged ? bwd_stage_bytes(A.n_orb, A.n_bins) : 0;
    const size_t smem = ((stage + 15) & ~size_t(15)) + bwd_scratch_bytes(A.n_orb);
    auto go = [&](auto kfn) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        for (int cls = 0; cls < 8; ++cls) {
            const int px = cls & 1, py = (cls >> 1) & 1, pz = cls >> 2;
            const long cubes = (long)((A.n1 - px + 1) >> 1) * ((A.n2 - py + 1) >> 1) * ((A.n3 - pz + 1) >> 1);
            const long total = cubes * A.nb;
            if (total == 0) continue;
            const int grid = (int)((total + kBwdThreads - 1) / kBwdThreads);
            kfn<<<grid, kBwdThreads, smem, stream>>>(A, px, py, pz);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        const long face = ((long)A.n2 * A.n3 + (long)(A.n1 - 1) * A.n3 + (long)(A.n1 - 1) * (A.n2 - 1)) * A.nb;
        tetra_dos_bwd_fold<<<(int)((face + 255) / 256), 256, 0, stream>>>(A);
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
    // the parity classes add into the arrays: start from zero (halo and
    // padding entries stay zero)
    const size_t pts = (size_t)P.nx * P.ny * P.nz;
    if (cudaMemsetAsync(grad_eps, 0, sizeof(float) * pts * P.eps_stride, stream) != cudaSuccess ||
        cudaMemsetAsync(grad_w, 0, sizeof(float) * pts * P.w_stride, stream) != cudaSuccess)
        return TETRA_ECUDA;
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
