// Spectral function of the bare susceptibility at T = 0 by exact
// double-band clipping of every tetrahedron: the extension to
// susceptibilities that arXiv:1710.10789 names for its method (abstract,
// Conclusions), here with step occupations.
//
//   S(q, w) = sum_{n,m} (1/V_G) int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
//                                 delta(w - (e_m(k+q) - e_n(k))),
//   Im chi0(q, w + i0) = -pi S(q, w).
//
// Inside a tetrahedron the method interpolates every band linearly, so
// a = e_n - mu, c = e_m(k+q) - mu and the transition energy D = c - a are
// linear there. The occupation difference is +1 on {a < 0 < c}, -1 on
// {c < 0 < a} and 0 elsewhere; each region is the tetrahedron cut by two
// planes. A cut by one plane keeps a corner tetrahedron, a wedge or a prism,
// each split into at most three tetrahedra; the second cut splits those
// again. Over a sub-tetrahedron of volume fraction nu, D is linear and its
// distribution is nu * g(w), g the normalised density of a linear function on
// a tetrahedron (the total of Sec. II.C's corner weight derivatives divided
// by V_T / V_G), or nu * [G(w_hi) - G(w_lo)] / (w_hi - w_lo) as a bin average.
//
// One thread per (cube, tetrahedron) runs over the band pairs in a loop that
// is not unrolled (the unrolled 64-pair loop overflowed the instruction
// cache); a pair whose regions are empty (band n nowhere occupied or band m
// nowhere empty for the +1 region, and the converse for -1) is skipped from
// four corner minima and maxima. The clipping only queues the kept
// sub-tetrahedra (sorted transition energies, amplitude, dither key) in a
// per-warp queue in shared memory; between band pairs, once the queue holds
// kDrainAt entries, all 32 lanes drain it, one sub-tetrahedron per lane, so
// the per-energy work is not serialised behind the lanes' different clip
// paths. Contributions are rounded once to integers of a fixed-point unit
// (a dither hashed from the contribution's identity makes the rounding
// unbiased) and added with 64-bit integer atomics into a per-CTA shared
// tile, then summed over CTAs in fixed order: the result does not depend on
// the schedule or on the order in which queues are drained.
#include <atomic>

#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr int kSpecThreads = 128;
constexpr int kSpecWarps = kSpecThreads / 32;
constexpr int kSpecBlocksPerSM = 4;
constexpr int kSpecBits = 26;   // fixed-point fraction bits of the unit below
constexpr int kQueueCap = 256;  // sub-tetrahedra per warp queue
constexpr int kDrainAt = 64;    // a queue this full is drained before the next band pair

// Table I (corner labels minus one, label c at offset (c&1, (c>>1)&1, (c>>2)&1)).
__constant__ int kSpecTable[6][4] = {{0, 1, 2, 5}, {1, 2, 3, 5}, {0, 2, 4, 5},
                                     {2, 3, 5, 7}, {2, 4, 5, 6}, {2, 5, 6, 7}};

// A point of the parent tetrahedron: three barycentric coordinates (the
// fourth is implied) and the two linear fields a and c.
struct P5 {
    float l0, l1, l2, a, c;
};

__device__ __forceinline__ P5 cut(const P5 &u, const P5 &v, float su, float sv) {
    const float t = su / (su - sv);
    return {fmaf(t, v.l0 - u.l0, u.l0), fmaf(t, v.l1 - u.l1, u.l1), fmaf(t, v.l2 - u.l2, u.l2),
            fmaf(t, v.a - u.a, u.a), fmaf(t, v.c - u.c, u.c)};
}

// Field a clip keeps the negative side of: 0 -> a, 1 -> -a, 2 -> c, 3 -> -c.
__device__ __forceinline__ float field(const P5 &p, int which) {
    const float v = (which < 2) ? p.a : p.c;
    return (which & 1) ? -v : v;
}

__device__ __forceinline__ void cswap5(P5 &x, P5 &y, float &sx, float &sy) {
    if (sy < sx) {
        const P5 t = x;
        x = y;
        y = t;
        const float ts = sx;
        sx = sy;
        sy = ts;
    }
}

// One sub-tetrahedron waiting in a warp's queue: its sorted transition
// energies, amplitude sign * nu * scale and dither key.
struct SubTet {
    float d0, d1, d2, d3, amp;
    uint32_t key;
};

// Constants of a launch that the sub-tetrahedron accumulation needs.
struct SpecArgs {
    const float *om;        // shared: energies (point) or bin edges (bin)
    long long *tile;        // shared: int64 accumulators per energy / bin
    int n_om;               // energies or bins
    int mode;               // TETRA_POINT or TETRA_BIN
    float scale;            // V_T/V_G over the fixed-point unit
    int *status;
    float om0, om_last;     // first and last grid energy (edge)
    float inv_de;           // 1 / mean spacing, for the index estimates
    SubTet *q;              // shared: this warp's queue [kQueueCap]
    int *qn;                // shared: its fill count
};

// Normalised density g and cumulative G of a linear function with sorted
// corner values d0 <= d1 <= d2 <= d3 at w (reciprocals precomputed).
struct Lin {
    float d0, d1, d2, d3;
    float k1, k2a, k2b, k3;   // g = k1 x^2 | k2a (d21 + 2x - k2b x^2) | k3 y^2
    float g2c;                     // G case 2: (d21^2 + 3 d21 x + 3 x^2 - k2b x^3) * g2c
};

// (All three pieces are evaluated and one is selected: the lanes of a warp
// walk different sub-tetrahedra, so a branch per piece would diverge.)
__device__ __forceinline__ float lin_g(const Lin &L, float w) {
    const float x1 = w - L.d0, x2 = w - L.d1, y = L.d3 - w;
    const float g1 = L.k1 * x1 * x1;
    const float g2 = L.k2a * fmaf(-L.k2b * x2, x2, fmaf(2.f, x2, L.d1 - L.d0));
    const float g3 = L.k3 * y * y;
    const float g = (w <= L.d1) ? g1 : ((w <= L.d2) ? g2 : g3);
    return (w > L.d0 && w < L.d3) ? g : 0.f;
}

__device__ __forceinline__ float lin_G(const Lin &L, float w) {
    const float x1 = w - L.d0, x2 = w - L.d1, y = L.d3 - w, d21 = L.d1 - L.d0;
    const float G1 = L.k1 * (1.f / 3.f) * x1 * x1 * x1;
    const float G2 = L.g2c * (d21 * d21 + x2 * (3.f * d21 + x2 * (3.f - L.k2b * x2)));
    const float G3 = 1.f - L.k3 * (1.f / 3.f) * y * y * y;
    const float G = (w <= L.d1) ? G1 : ((w <= L.d2) ? G2 : G3);
    return !(w > L.d0) ? 0.f : (!(w < L.d3) ? 1.f : G);
}

// Mean spacing of the energy grid (or bin width), the scale of the
// fixed-point unit unit = (V_T/V_G) / de * 2^-26; the same expression in the
// kernel and in the reduction.
__device__ __forceinline__ double mean_spacing(const float *om, int n_om, int mode) {
    const int spacings = mode == TETRA_BIN ? n_om : n_om - 1;
    double de = spacings > 0 ? ((double)om[spacings] - (double)om[0]) / spacings : 1.0;
    return de > 0.0 ? de : 1.0;
}

__device__ __forceinline__ float hash_dither(uint32_t key) {
    uint32_t h = key * 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f;
}

// First index i in [0, n) with om[i] > x (or n), from the index a uniform
// grid would give (om0 + i / inv_de), corrected against the grid itself, so
// any ascending grid gives the exact index.
__device__ __forceinline__ int upper_index(const float *om, int n, float x, float om0, float inv_de) {
    const float e = fminf(fmaxf((x - om0) * inv_de, -1.f), (float)n + 1.f);
    int i = min(max((int)ceilf(e), 0), n);
    while (i > 0 && om[i - 1] > x) --i;
    while (i < n && !(om[i] > x)) ++i;
    return i;
}

// First index i in [0, n) with om[i] >= x (or n), as upper_index.
__device__ __forceinline__ int lower_index(const float *om, int n, float x, float om0, float inv_de) {
    const float e = fminf(fmaxf((x - om0) * inv_de, -1.f), (float)n + 1.f);
    int i = min(max((int)ceilf(e), 0), n);
    while (i > 0 && om[i - 1] >= x) --i;
    while (i < n && !(om[i] >= x)) ++i;
    return i;
}

// Adds one sub-tetrahedron's distribution of D to the tile.
__device__ void deposit(const SubTet &T, const SpecArgs &S) {
    Lin L;
    L.d0 = T.d0; L.d1 = T.d1; L.d2 = T.d2; L.d3 = T.d3;
    const float d21 = T.d1 - T.d0, d31 = T.d2 - T.d0, d41 = T.d3 - T.d0;
    const float d32 = T.d2 - T.d1, d42 = T.d3 - T.d1, d43 = T.d3 - T.d2;
    L.k1 = d21 > 0.f ? 3.f / (d21 * d31 * d41) : 0.f;
    L.k2a = (d31 > 0.f) ? 3.f / (d31 * d41) : 0.f;
    L.k2b = (d32 > 0.f && d42 > 0.f) ? (d31 + d42) / (d32 * d42) : 0.f;
    L.k3 = d43 > 0.f ? 3.f / (d41 * d42 * d43) : 0.f;
    L.g2c = (d31 > 0.f) ? 1.f / (d31 * d41) : 0.f;
    int i0, i1;   // indices [i0, i1)
    if (S.mode == TETRA_BIN) {
        i0 = max(0, upper_index(S.om, S.n_om + 1, T.d0, S.om0, S.inv_de) - 1);   // bins with upper edge > d0
        i1 = min(S.n_om, upper_index(S.om, S.n_om + 1, T.d3, S.om0, S.inv_de));   // and lower edge <= d3
    } else {
        i0 = upper_index(S.om, S.n_om, T.d0, S.om0, S.inv_de);
        i1 = lower_index(S.om, S.n_om, T.d3, S.om0, S.inv_de);
    }
    const float dith = hash_dither(T.key);
    float Gp = (S.mode == TETRA_BIN && i0 < i1) ? lin_G(L, S.om[i0]) : 0.f;
    for (int i = i0; i < i1; ++i) {
        float v;
        if (S.mode == TETRA_BIN) {
            const float Gn = lin_G(L, S.om[i + 1]);
            v = (Gn - Gp) / (S.om[i + 1] - S.om[i]);
            Gp = Gn;
        } else {
            v = lin_g(L, S.om[i]);
        }
        const float x = fmaf(T.amp, v, dith);
        long long qv;
        if (fabsf(x) < 4194304.f) {
            // round to nearest even by adding 1.5 * 2^23 (exact below 2^22):
            // the same integer as the 64-bit conversion, without the FP64
            // pipe that conversion runs on
            qv = __float_as_int(x + 12582912.f) - 0x4B400000;
        } else if (fabsf(x) < 4.0e18f) {
            qv = __float2ll_rn(x);
        } else {
            atomicOr(S.status, kFlagRange);
            qv = 0;
        }
        if (qv) atomicAdd(reinterpret_cast<unsigned long long *>(&S.tile[i]), static_cast<unsigned long long>(qv));
    }
}

// Queues sign * nu * (distribution of D) of one sub-tetrahedron in this
// warp's queue (or adds it at once when the queue is full).
__device__ __noinline__ void accumulate(P5 v0, P5 v1, P5 v2, P5 v3, float sign, uint32_t key,
                                        const SpecArgs S) {
    const float u00 = v0.l0 - v3.l0, u01 = v0.l1 - v3.l1, u02 = v0.l2 - v3.l2;
    const float u10 = v1.l0 - v3.l0, u11 = v1.l1 - v3.l1, u12 = v1.l2 - v3.l2;
    const float u20 = v2.l0 - v3.l0, u21 = v2.l1 - v3.l1, u22 = v2.l2 - v3.l2;
    const float nu = fabsf(u00 * (u11 * u22 - u12 * u21) - u01 * (u10 * u22 - u12 * u20) +
                           u02 * (u10 * u21 - u11 * u20));
    if (!(nu > 0.f)) return;
    float d[4] = {v0.c - v0.a, v1.c - v1.a, v2.c - v2.a, v3.c - v3.a};
#define SPEC_CS(i, j) { const float lo_ = fminf(d[i], d[j]), hi_ = fmaxf(d[i], d[j]); d[i] = lo_; d[j] = hi_; }
    SPEC_CS(0, 1) SPEC_CS(2, 3) SPEC_CS(0, 2) SPEC_CS(1, 3) SPEC_CS(1, 2)
#undef SPEC_CS
    // a flat transition energy is a delta: measure zero in point mode, its
    // whole weight in the bin that holds it in bin mode
    if (S.mode != TETRA_BIN && !(d[3] > d[0])) return;
    // no grid energy (bin) in reach
    if (d[3] < S.om[0] || d[0] > S.om_last) return;
    const SubTet T{d[0], d[1], d[2], d[3], sign * nu * S.scale, key};
    const int slot = atomicAdd(S.qn, 1);
    if (slot < kQueueCap) S.q[slot] = T;
    else deposit(T, S);
}

// Every lane of the warp takes queued sub-tetrahedra in turn; the queue is
// empty afterwards. Called by all 32 lanes together.
__device__ __forceinline__ void drain(const SpecArgs &S, int lane) {
    __syncwarp();
    const int n = min(*S.qn, kQueueCap);
    for (int e = lane; e < n; e += 32) deposit(S.q[e], S);
    __syncwarp();
    if (lane == 0) *S.qn = 0;
    __syncwarp();
}

// Cuts tetrahedron (v0..v3) to {field(which) < 0} and accumulates the kept
// sub-tetrahedra (second and last cut).
__device__ __noinline__ void clip_second(P5 v0, P5 v1, P5 v2, P5 v3, int which, float sign, uint32_t key,
                                         const SpecArgs S) {
    float s0 = field(v0, which), s1 = field(v1, which), s2 = field(v2, which), s3 = field(v3, which);
    cswap5(v0, v1, s0, s1);
    cswap5(v2, v3, s2, s3);
    cswap5(v0, v2, s0, s2);
    cswap5(v1, v3, s1, s3);
    cswap5(v1, v2, s1, s2);
    const int k = (s0 < 0.f) + (s1 < 0.f) + (s2 < 0.f) + (s3 < 0.f);
    if (k == 0) return;
    if (k == 4) {
        accumulate(v0, v1, v2, v3, sign, key * 4u, S);
    } else if (k == 1) {
        accumulate(v0, cut(v0, v1, s0, s1), cut(v0, v2, s0, s2), cut(v0, v3, s0, s3), sign, key * 4u, S);
    } else if (k == 3) {
        const P5 p0 = cut(v0, v3, s0, s3), p1 = cut(v1, v3, s1, s3), p2 = cut(v2, v3, s2, s3);
        accumulate(v0, v1, v2, p0, sign, key * 4u, S);
        accumulate(v1, v2, p0, p1, sign, key * 4u + 1u, S);
        accumulate(v2, p0, p1, p2, sign, key * 4u + 2u, S);
    } else {
        const P5 p02 = cut(v0, v2, s0, s2), p03 = cut(v0, v3, s0, s3);
        const P5 p12 = cut(v1, v2, s1, s2), p13 = cut(v1, v3, s1, s3);
        accumulate(v0, p02, p03, v1, sign, key * 4u, S);
        accumulate(p02, p03, v1, p12, sign, key * 4u + 1u, S);
        accumulate(p03, v1, p12, p13, sign, key * 4u + 2u, S);
    }
}

// One region of one (tetrahedron, band pair): first cut by `first`, then
// every kept tetrahedron by `second`.
__device__ __noinline__ void region(P5 v0, P5 v1, P5 v2, P5 v3, int first, int second, float sign,
                                    uint32_t key, const SpecArgs S) {
    float s0 = field(v0, first), s1 = field(v1, first), s2 = field(v2, first), s3 = field(v3, first);
    cswap5(v0, v1, s0, s1);
    cswap5(v2, v3, s2, s3);
    cswap5(v0, v2, s0, s2);
    cswap5(v1, v3, s1, s3);
    cswap5(v1, v2, s1, s2);
    const int k = (s0 < 0.f) + (s1 < 0.f) + (s2 < 0.f) + (s3 < 0.f);
    if (k == 0) return;
    if (k == 4) {
        clip_second(v0, v1, v2, v3, second, sign, key * 4u, S);
    } else if (k == 1) {
        clip_second(v0, cut(v0, v1, s0, s1), cut(v0, v2, s0, s2), cut(v0, v3, s0, s3), second, sign, key * 4u, S);
    } else if (k == 3) {
        const P5 p0 = cut(v0, v3, s0, s3), p1 = cut(v1, v3, s1, s3), p2 = cut(v2, v3, s2, s3);
        clip_second(v0, v1, v2, p0, second, sign, key * 4u, S);
        clip_second(v1, v2, p0, p1, second, sign, key * 4u + 1u, S);
        clip_second(v2, p0, p1, p2, second, sign, key * 4u + 2u, S);
    } else {
        const P5 p02 = cut(v0, v2, s0, s2), p03 = cut(v0, v3, s0, s3);
        const P5 p12 = cut(v1, v2, s1, s2), p13 = cut(v1, v3, s1, s3);
        clip_second(v0, p02, p03, v1, second, sign, key * 4u, S);
        clip_second(p02, p03, v1, p12, second, sign, key * 4u + 1u, S);
        clip_second(p03, v1, p12, p13, second, sign, key * 4u + 2u, S);
    }
}

template <int NB>
__global__ void __launch_bounds__(kSpecThreads, kSpecBlocksPerSM)
    spectral_t0_kernel(const float *eps, int eps_stride, int n1, int n2, int n3, int nx, int ny, int z0, int z1,
                       int qx, int qy, int qz, float mu, const float *omega, int n_om, int mode,
                       long long *partials, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    SubTet *queues = reinterpret_cast<SubTet *>(smem);                         // [warps][kQueueCap]
    int *qcount = reinterpret_cast<int *>(queues + kSpecWarps * kQueueCap);    // [warps]
    long long *tile = reinterpret_cast<long long *>(qcount + 2 * kSpecWarps); // 8-byte aligned
    float *om = reinterpret_cast<float *>(tile + n_om);
    const int n_edges = (mode == TETRA_BIN) ? n_om + 1 : n_om;
    for (int i = threadIdx.x; i < n_om; i += blockDim.x) tile[i] = 0;
    for (int i = threadIdx.x; i < n_edges; i += blockDim.x) om[i] = omega[i];
    if (threadIdx.x < kSpecWarps) qcount[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // V_T/V_G in fixed-point units: de * 2^26
    const double de = mean_spacing(om, n_om, mode);
    const float scale = (float)ldexp(de, kSpecBits);
    const float om_lo = om[0], om_hi = om[n_edges - 1];
    const SpecArgs S{om, tile, n_om, mode, scale, status, om_lo, om_hi, (float)(1.0 / de),
                     queues + warp * kQueueCap, qcount + warp};
    // energy range of the grid: a band pair whose transition energies over a
    // tetrahedron miss it contributes nothing (the clipped regions' values
    // lie between the corner minimum and maximum); the +1 region has positive
    // transition energies, the -1 region negative ones
    const long n_items = 6L * n1 * n2 * (long)(z1 - z0);
    const long stride = (long)gridDim.x * blockDim.x;
    // whole warps step through the items together (the queue is drained by
    // all 32 lanes); a lane past the end takes part without items
    for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_items; base += stride) {
        const long it = base + lane;
        const bool valid = it < n_items;
        float a[4][NB], c[4][NB];   // indexed by band at run time below
        if (valid) {
            const int t = (int)(it % 6);
            const long cube = it / 6;
            const int x = (int)(cube % n1), y = (int)((cube / n1) % n2), z = z0 + (int)(cube / ((long)n1 * n2));
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int cl = kSpecTable[t][v];
                const int xx = x + (cl & 1), yy = y + ((cl >> 1) & 1), zz = z + (cl >> 2);
                // the point itself: the layout's halo covers xx = n1 etc.
                const long p = xx + (long)nx * (yy + (long)ny * zz);
                // the point shifted by q, reduced into the grid
                // (xx <= n1 and 0 <= qx < n1, so one subtraction reduces it)
                int sx = xx + qx, sy = yy + qy, sz = zz + qz;
                sx -= (sx >= n1) ? n1 : 0;
                sy -= (sy >= n2) ? n2 : 0;
                sz -= (sz >= n3) ? n3 : 0;
                const long pq = sx + (long)nx * (sy + (long)ny * sz);
#pragma unroll
                for (int n = 0; n < NB; ++n) {
                    a[v][n] = eps[p * eps_stride + n] - mu;
                    c[v][n] = eps[pq * eps_stride + n] - mu;
                }
            }
        }
        // per band: some corner occupied (an), some corner empty (ap); the
        // same for the bands at k + q (cn: occupied, cp: empty)
        uint32_t an = 0, ap = 0, cn = 0, cp = 0, a_all = 0, c_all = 0;
        if (valid) {
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                const float amin = fminf(fminf(a[0][n], a[1][n]), fminf(a[2][n], a[3][n]));
                const float amax = fmaxf(fmaxf(a[0][n], a[1][n]), fmaxf(a[2][n], a[3][n]));
                const float cmin = fminf(fminf(c[0][n], c[1][n]), fminf(c[2][n], c[3][n]));
                const float cmax = fmaxf(fmaxf(c[0][n], c[1][n]), fmaxf(c[2][n], c[3][n]));
                an |= (amin < 0.f ? 1u : 0u) << n;
                ap |= (amax > 0.f ? 1u : 0u) << n;
                cn |= (cmin < 0.f ? 1u : 0u) << n;
                cp |= (cmax > 0.f ? 1u : 0u) << n;
                a_all |= (amax < 0.f ? 1u : 0u) << n;   // occupied at every corner
                c_all |= (cmin > 0.f ? 1u : 0u) << n;   // empty at every corner
            }
        }
        // band pairs in a loop that is not unrolled (one copy of the code);
        // the queue is drained between pairs once it holds kDrainAt entries
#pragma unroll 1
        for (int pr = 0; pr < NB * NB; ++pr) {
            // lane 0's count, read after every push of the previous pair and
            // before any of this one: the same decision in every lane
            __syncwarp();
            const int queued = __shfl_sync(0xffffffffu, *S.qn, 0);
            if (queued >= kDrainAt) drain(S, lane);
            const int n = pr / NB, m = pr - (pr / NB) * NB;
            bool plus = ((an >> n) & 1u) && ((cp >> m) & 1u);
            bool minus = ((ap >> n) & 1u) && ((cn >> m) & 1u);
            if (!plus && !minus) continue;
            const float d0 = c[0][m] - a[0][n], d1 = c[1][m] - a[1][n];
            const float d2 = c[2][m] - a[2][n], d3 = c[3][m] - a[3][n];
            const float dlo = fminf(fminf(d0, d1), fminf(d2, d3)), dhi = fmaxf(fmaxf(d0, d1), fmaxf(d2, d3));
            if (dhi < om_lo || dlo > om_hi) continue;
            plus = plus && om_hi > 0.f;
            minus = minus && om_lo < 0.f;
            if (!plus && !minus) continue;
            const P5 v0{1.f, 0.f, 0.f, a[0][n], c[0][m]};
            const P5 v1{0.f, 1.f, 0.f, a[1][n], c[1][m]};
            const P5 v2{0.f, 0.f, 1.f, a[2][n], c[2][m]};
            const P5 v3{0.f, 0.f, 0.f, a[3][n], c[3][m]};
            const uint32_t key = ((uint32_t)it * (uint32_t)(NB * NB) + (uint32_t)(n * NB + m)) * 2u;
            // band n occupied and band m empty at every corner: the +1
            // region is the whole tetrahedron (the same sub-tetrahedron and
            // dither key the two cuts would produce)
            if (((a_all >> n) & 1u) && ((c_all >> m) & 1u)) {
                accumulate(v0, v1, v2, v3, 1.f, key * 16u, S);
                continue;
            }
            // +1 on {a < 0, c > 0}; -1 on {a > 0, c < 0}
            if (plus) region(v0, v1, v2, v3, 0, 3, 1.f, key, S);
            if (minus) region(v0, v1, v2, v3, 1, 2, -1.f, key + 1u, S);
        }
    }
    drain(S, lane);
    __syncthreads();
    long long *dst = partials + (long)blockIdx.x * n_om;
    for (int i = threadIdx.x; i < n_om; i += blockDim.x) dst[i] = tile[i];
}

// S[i] = unit * sum over CTAs (fixed order) of the int64 partials.
__global__ void spectral_reduce_kernel(const long long *partials, int grid, int n_om, int mode, const float *omega,
                                       double vtvg, float *S) {
    const double unit = vtvg / mean_spacing(omega, n_om, mode) * ldexp(1.0, -kSpecBits);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_om; i += gridDim.x * blockDim.x) {
        long long acc = 0;
        for (int b = 0; b < grid; ++b) acc += partials[(long)b * n_om + i];
        S[i] = (float)((double)acc * unit);
    }
}

// persistent blocks, as many as fit an SM at the register bound
int spectral_grid(const Plan &P) { return kSpecBlocksPerSM * P.sm_count; }

size_t spectral_smem(int n_om, int mode) {
    return sizeof(SubTet) * kSpecWarps * kQueueCap + sizeof(int) * 2 * kSpecWarps + sizeof(long long) * (size_t)n_om +
           sizeof(float) * (size_t)(mode == TETRA_BIN ? n_om + 1 : n_om);
}

template <int NB>
cudaError_t launch_spectral_nb(const Plan &P, const float *eps, const int q[3], float mu, const float *omega,
                               int n_om, int mode, long long *partials, int *status, int grid,
                               size_t smem, cudaStream_t stream) {
    auto k = spectral_t0_kernel<NB>;
    static std::atomic<int> opted[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || opted[dev].load() < (int)smem) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) {
            int cur = opted[dev].load();
            while (cur < (int)smem && !opted[dev].compare_exchange_weak(cur, (int)smem)) {
            }
        }
    }
    k<<<grid, kSpecThreads, smem, stream>>>(eps, P.eps_stride, P.d.n1, P.d.n2, P.d.n3, P.nx, P.ny, P.z0, P.z1,
                                           q[0], q[1], q[2], mu, omega, n_om, mode, partials, status);
    return cudaGetLastError();
}

int mod_q(int a, int n) {
    const int m = a % n;
    return m < 0 ? m + n : m;
}

}  // namespace

size_t spectral_t0_workspace(const Plan &P, int n_om) {
    return kStatusBytes + sizeof(long long) * (size_t)spectral_grid(P) * (size_t)n_om;
}

tetra_status_t launch_spectral_t0(const Plan &P, const float *eps, const int q_in[3], float mu, int mode, int n_om,
                                  const float *omega, float *S, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (n_om < 1 || (mode != TETRA_POINT && mode != TETRA_BIN)) return TETRA_EINVAL;
    if (P.d.n_bands > 8) return TETRA_EUNSUPPORTED;
    // the bands at k + q come from every plane of the grid
    if (P.z0 != 0 || P.z1 != P.d.n3) return TETRA_EUNSUPPORTED;
    const size_t smem = spectral_smem(n_om, mode);
    if (smem > P.smem_optin) return TETRA_EUNSUPPORTED;
    if (ws_bytes < spectral_t0_workspace(P, n_om)) return TETRA_ENOMEM;
    const double vtvg = 1.0 / (6.0 * (double)P.d.n1 * (double)P.d.n2 * (double)P.d.n3);
    const int q[3] = {mod_q(q_in[0], P.d.n1), mod_q(q_in[1], P.d.n2), mod_q(q_in[2], P.d.n3)};
    const int grid = spectral_grid(P);
    int *status = reinterpret_cast<int *>(ws);
    long long *partials = reinterpret_cast<long long *>(static_cast<unsigned char *>(ws) + kStatusBytes);
    if (cudaMemsetAsync(ws, 0, kStatusBytes, stream) != cudaSuccess) return TETRA_ECUDA;
    cudaError_t e;
    switch (P.d.n_bands) {
        case 1: e = launch_spectral_nb<1>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 2: e = launch_spectral_nb<2>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 3: e = launch_spectral_nb<3>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 4: e = launch_spectral_nb<4>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 5: e = launch_spectral_nb<5>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 6: e = launch_spectral_nb<6>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 7: e = launch_spectral_nb<7>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        default: e = launch_spectral_nb<8>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
    }
    if (e != cudaSuccess) return TETRA_ECUDA;
    spectral_reduce_kernel<<<(n_om + 255) / 256, 256, 0, stream>>>(partials, grid, n_om, mode, omega, vtvg, S);
    return cudaGetLastError() == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace tetra

extern "C" size_t tetra_spectral_t0_workspace_bytes(tetra_plan_t plan, int n_omega) {
    if (!plan || n_omega < 1) return 0;
    return tetra::spectral_t0_workspace(*plan, n_omega);
}

extern "C" tetra_status_t tetra_spectral_t0(tetra_plan_t plan, const float *eps, const int q[3], float mu, int mode,
                                            int n_omega, const float *omega, float *S, void *ws, size_t ws_bytes,
                                            cudaStream_t stream) {
    if (!plan || !eps || !q || !omega || !S || !ws) return TETRA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(eps) & 15u) || (reinterpret_cast<uintptr_t>(ws) & 15u)) return TETRA_EINVAL;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_spectral_t0(*plan, eps, q, mu, mode, n_omega, omega, S, ws, ws_bytes, stream);
}
