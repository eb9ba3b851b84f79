// Bare susceptibility at T = 0 by exact double-band clipping of every
// tetrahedron: the extension to susceptibilities that arXiv:1710.10789 names
// for its method (abstract, Conclusions), here with step occupations.
//
//   S(q, w) = sum_{n,m} (1/V_G) int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
//                                 delta(w - (e_m(k+q) - e_n(k))),
//   Im chi0(q, w + i0) = -pi S(q, w),
//   Re chi0(q, w) = sum_{n,m} (1/V_G) P int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
//                                             / (w - e_m(k+q) + e_n(k)).
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
//
// The real part runs the same clipping with KIND = kKindRe: every
// sub-tetrahedron reaches every energy (its principal-value average of
// 1/(w - D), below), so the sub-tetrahedra are kept in per-lane segments and
// the whole warp evaluates them, lane by lane in a fixed order, at all
// energies (each lane owning every 32nd energy).
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
// the real part of chi0 (kKindRe) next to the spectral function (kKindS)
constexpr int kKindS = 0, kKindRe = 1;
constexpr int kReBlocksPerSM = 3;
constexpr int kSubPerPair = 18;  // sub-tetrahedra one (tetrahedron, band pair) can give: 2 regions x 3 x 3
constexpr int kReFlush = 64;     // entries summed in FP32 before the per-warp sums go to the tile
constexpr int kReMom = 12;       // highest moment of the far-field series
constexpr int kRePiece = 15;     // highest term of a density piece's own series

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

// One sub-tetrahedron of the real part in its lane's segment: sorted
// transition energies and amplitude.
struct ReSeg {
    float d0, d1, d2, d3, amp;
};

// Far-field set-up of one entry as the warp's lanes read it (16 words):
// mean c, (4 R)^2, amplitude, segment slot, moments mu_0 and mu_2..mu_kReMom
// (mu_1 vanishes about the mean).
struct __align__(16) ReStage {
    float c, far2, amp;
    int loc;
    float mu0, mu[kReMom - 1];
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
    int *qn;                // shared: its fill count (real part: this lane's)
    float *racc;            // shared, real part: this warp's FP32 sums per energy
    ReSeg *rq;              // shared, real part: this lane's segment [kSubPerPair]
    ReStage *stage;         // shared, real part: this warp's set-ups [32]
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
// warp's queue (or adds it at once when the queue is full). Real part: in
// this lane's own segment, in the order the clipping produces them.
template <int KIND>
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
    if constexpr (KIND == kKindRe) {
        // every sub-tetrahedron reaches every energy (a flat one as 1/(w - d))
        const int slot = (*S.qn)++;
        S.rq[slot] = ReSeg{d[0], d[1], d[2], d[3], sign * nu * S.scale};
        return;
    }
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
template <int KIND>
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
        accumulate<KIND>(v0, v1, v2, v3, sign, key * 4u, S);
    } else if (k == 1) {
        accumulate<KIND>(v0, cut(v0, v1, s0, s1), cut(v0, v2, s0, s2), cut(v0, v3, s0, s3), sign, key * 4u, S);
    } else if (k == 3) {
        const P5 p0 = cut(v0, v3, s0, s3), p1 = cut(v1, v3, s1, s3), p2 = cut(v2, v3, s2, s3);
        accumulate<KIND>(v0, v1, v2, p0, sign, key * 4u, S);
        accumulate<KIND>(v1, v2, p0, p1, sign, key * 4u + 1u, S);
        accumulate<KIND>(v2, p0, p1, p2, sign, key * 4u + 2u, S);
    } else {
        const P5 p02 = cut(v0, v2, s0, s2), p03 = cut(v0, v3, s0, s3);
        const P5 p12 = cut(v1, v2, s1, s2), p13 = cut(v1, v3, s1, s3);
        accumulate<KIND>(v0, p02, p03, v1, sign, key * 4u, S);
        accumulate<KIND>(p02, p03, v1, p12, sign, key * 4u + 1u, S);
        accumulate<KIND>(p03, v1, p12, p13, sign, key * 4u + 2u, S);
    }
}

// One region of one (tetrahedron, band pair): first cut by `first`, then
// every kept tetrahedron by `second`.
template <int KIND>
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
        clip_second<KIND>(v0, v1, v2, v3, second, sign, key * 4u, S);
    } else if (k == 1) {
        clip_second<KIND>(v0, cut(v0, v1, s0, s1), cut(v0, v2, s0, s2), cut(v0, v3, s0, s3), second, sign, key * 4u, S);
    } else if (k == 3) {
        const P5 p0 = cut(v0, v3, s0, s3), p1 = cut(v1, v3, s1, s3), p2 = cut(v2, v3, s2, s3);
        clip_second<KIND>(v0, v1, v2, p0, second, sign, key * 4u, S);
        clip_second<KIND>(v1, v2, p0, p1, second, sign, key * 4u + 1u, S);
        clip_second<KIND>(v2, p0, p1, p2, second, sign, key * 4u + 2u, S);
    } else {
        const P5 p02 = cut(v0, v2, s0, s2), p03 = cut(v0, v3, s0, s3);
        const P5 p12 = cut(v1, v2, s1, s2), p13 = cut(v1, v3, s1, s3);
        clip_second<KIND>(v0, p02, p03, v1, second, sign, key * 4u, S);
        clip_second<KIND>(p02, p03, v1, p12, second, sign, key * 4u + 1u, S);
        clip_second<KIND>(p03, v1, p12, p13, second, sign, key * 4u + 2u, S);
    }
}

// ---- real part: P<1/(w - D)> of one sub-tetrahedron at every energy ----
//
// Re chi0(q, w) adds sign * nu * P<1/(w - D)> for every sub-tetrahedron; the
// average is the principal-value integral of D's density g against
// 1/(w - x). g is a quadratic spline on the sorted corner values d0..d3 with
// Bernstein coefficients (0, 0, G1) on [d0, d1], (G1, 3/d41, G2) on [d1, d2]
// and (G2, 0, 0) on [d2, d3], G1 = 3 d21/(d31 d41) = g(d1), G2 = 3 d43/(d41
// d42) = g(d2). Far from the sub-tetrahedron (|w - c| > 4 R, c the mean of
// the corner values, R the largest |d_k - c|) the average is the moment
// series sum_n mu_n / (w - c)^(n+1), mu_n = <(D - c)^n> = 6 n!/(n+3)!
// h_n(d - c) (h_n the complete homogeneous symmetric polynomial), whose
// terms shrink by 1/4 or more. Near it each piece [a, b] (h = b - a,
// s = (w - a)/h) gives, within 3/2 of its own centre,
//   p(s) [ln|w - a| - ln|w - b|] + b0 (3/2 - s) + b1 (2s - 1) - b2 (s + 1/2),
// p the piece's polynomial continued to t = s, and beyond that its own
// moment series in 1/(s - 1/2) (a thin piece far from w, where the closed
// form would cancel). At a knot the two pieces meeting there drop their
// equal-and-opposite ln|w - knot| terms.
// Far-field data of a sub-tetrahedron: mean c of its corner values, (4 R)^2
// and the moments mu_0..mu_kReMom about c.
struct ReFar {
    float c, far2;
    float mu[kReMom + 1];
};

__device__ __forceinline__ void re_far_setup(const ReSeg &T, ReFar &F) {
    F.c = 0.25f * ((T.d0 + T.d1) + (T.d2 + T.d3));
    const float e[4] = {T.d0 - F.c, T.d1 - F.c, T.d2 - F.c, T.d3 - F.c};
    const float R = fmaxf(-e[0], e[3]);
    F.far2 = 16.f * R * R;
    // h_n(e) from prod_k 1 / (1 - e_k t), one factor at a time
    float h[kReMom + 1];
    h[0] = 1.f;
#pragma unroll
    for (int n = 1; n <= kReMom; ++n) h[n] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int n = 1; n <= kReMom; ++n) h[n] = fmaf(e[k], h[n - 1], h[n]);
#pragma unroll
    for (int n = 0; n <= kReMom; ++n) F.mu[n] = h[n] * (6.f / (float)((n + 1) * (n + 2) * (n + 3)));
}

// int_0^1 p(t) / (s - t) dt for a piece with Bernstein coefficients b0..b2.
__device__ __forceinline__ float re_piece(float b0, float b1, float b2, float a, float rh, float La, float Lb,
                                          float w) {
    if (rh == 0.f) return 0.f;
    const float s = (w - a) * rh, up = s - 0.5f;
    if (fabsf(up) >= 1.5f) {
        // p = A + B tau + C tau^2, tau = t - 1/2; moments of tau^k over
        // [-1/2, 1/2]: 2^-k / (k + 1) for even k, 0 for odd k
        const float A = 0.25f * (b0 + 2.f * b1 + b2), B = b2 - b0, C = b0 - 2.f * b1 + b2;
        const float v = 1.f / up;
        float acc = 0.f;
#pragma unroll
        for (int j = kRePiece; j >= 0; --j) {
            float m;
            if (j % 2 == 0)
                m = A * (ldexpf(1.f, -j) / (float)(j + 1)) + C * (ldexpf(1.f, -(j + 2)) / (float)(j + 3));
            else
                m = B * (ldexpf(1.f, -(j + 1)) / (float)(j + 2));
            acc = fmaf(acc, v, m);
        }
        return acc * v;
    }
    const float t1 = 1.f - s;
    const float ps = fmaf(b0 * t1, t1, fmaf(2.f * b1 * s, t1, b2 * s * s));
    return fmaf(ps, La - Lb, fmaf(b0, 1.5f - s, fmaf(b1, 2.f * s - 1.f, -b2 * (s + 0.5f))));
}

__device__ __forceinline__ float re_log(float w, float d) { return (w == d) ? 0.f : __logf(fabsf(w - d)); }

// P<1/(w - D)> within four half-widths of the sub-tetrahedron (or for a
// flat one): the three density pieces.
__device__ float re_near(const ReSeg &T, float w) {
    const float d21 = T.d1 - T.d0, d31 = T.d2 - T.d0, d41 = T.d3 - T.d0;
    const float d32 = T.d2 - T.d1, d42 = T.d3 - T.d1, d43 = T.d3 - T.d2;
    if (!(d41 > 0.f)) return (w == T.d0) ? 0.f : 1.f / (w - T.d0);
    const float G1 = d31 > 0.f ? __fdividef(3.f * d21, d31 * d41) : 0.f;
    const float G2 = d42 > 0.f ? __fdividef(3.f * d43, d41 * d42) : 0.f;
    const float mid = __fdividef(3.f, d41);
    const float r1 = d21 > 0.f ? __fdividef(1.f, d21) : 0.f;
    const float r2 = d32 > 0.f ? __fdividef(1.f, d32) : 0.f;
    const float r3 = d43 > 0.f ? __fdividef(1.f, d43) : 0.f;
    const float L0 = re_log(w, T.d0), L1 = re_log(w, T.d1), L2 = re_log(w, T.d2), L3 = re_log(w, T.d3);
    return re_piece(0.f, 0.f, G1, T.d0, r1, L0, L1, w) + re_piece(G1, mid, G2, T.d1, r2, L1, L2, w) +
           re_piece(G2, 0.f, 0.f, T.d2, r3, L2, L3, w);
}

// The moment series with terms mu_0..mu_K at v = 1/(w - c), four energies at once.
template <int K>
__device__ __forceinline__ void re_series4(const float (&mu)[kReMom + 1], const float (&v)[4], float (&r)[4]) {
    float acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = mu[K];
#pragma unroll
    for (int n = K - 1; n >= 0; --n)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fmaf(acc[k], v[k], mu[n]);
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = acc[k] * v[k];
}

// Adds the per-warp FP32 sums to the tile (one rounding per energy and
// flush) and clears them. Every lane owns the energies lane, lane + 32, ...
__device__ __forceinline__ void re_flush(const SpecArgs &S, int lane) {
    __syncwarp();
    for (int i = lane; i < S.n_om; i += 32) {
        const float x = S.racc[i];
        S.racc[i] = 0.f;
        if (fabsf(x) < 4.0e18f) {
            const long long qv = __float2ll_rn(x);
            if (qv) atomicAdd(reinterpret_cast<unsigned long long *>(&S.tile[i]), static_cast<unsigned long long>(qv));
        } else {
            atomicOr(S.status, kFlagRange);
        }
    }
    __syncwarp();
}

// The warp takes the sub-tetrahedra its lanes queued for the last band
// pair in lane order (a fixed order: the FP32 sums are reproducible), up to
// 32 at a time: each lane sets up one entry's far field into the warp's
// staging area; then every lane runs over its energies (lane, lane + 32,
// lane + 64, lane + 96 of each chunk of 128) and, for each staged entry in
// order, adds its average there into four register sums, which go to the
// warp's FP32 sums once per chunk. Series terms (truncation below 2^-23 of
// the leading 1/(w - c), terms shrinking by R/|w - c|): 6 when the warp's 128
// energies are all beyond 16 R, 8 beyond 8 R, 13 beyond 4 R; nearer, the
// density pieces.
__device__ __forceinline__ void re_process(const SpecArgs &S, const ReSeg *wq, int *wn, int lane,
                                           int &since_flush) {
    constexpr unsigned kAll = 0xffffffffu;
    __syncwarp();
    const int mine = wn[lane];
    // exclusive prefix of the lanes' counts
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kAll, incl, d);
        if (lane >= d) incl += y;
    }
    const int start = incl - mine, total = __shfl_sync(kAll, incl, 31);
    for (int base = 0; base < total; base += 32) {
        // this lane's entry: the last lane whose segment starts at or before it
        const int e = base + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int cand = src + step;
            if (__shfl_sync(kAll, start, cand) <= e) src = cand;
        }
        const int src_start = __shfl_sync(kAll, start, src);
        if (e < total) {
            const int loc = src * kSubPerPair + (e - src_start);
            const ReSeg T = wq[loc];
            ReFar F;
            re_far_setup(T, F);
            ReStage &st = S.stage[lane];
            st.c = F.c; st.far2 = F.far2; st.amp = T.amp; st.loc = loc; st.mu0 = F.mu[0];
#pragma unroll
            for (int n = 2; n <= kReMom; ++n) st.mu[n - 2] = F.mu[n];
        }
        __syncwarp();
        const int n_here = min(32, total - base);
        for (int c0 = 0; c0 < S.n_om; c0 += 128) {
            float w[4], sum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = S.om[min(c0 + lane + 32 * k, S.n_om - 1)];
            for (int j = 0; j < n_here; ++j) {
                const ReStage &st = S.stage[j];
                float mu[kReMom + 1];
                mu[0] = st.mu0;
                mu[1] = 0.f;
#pragma unroll
                for (int n = 2; n <= kReMom; ++n) mu[n] = st.mu[n - 2];
                float v[4], r[4];
                float umin = INFINITY;
                bool lane_far = true;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float u = w[k] - st.c;
                    v[k] = __fdividef(1.f, u);
                    if (c0 + lane + 32 * k < S.n_om) {
                        umin = fminf(umin, u * u);
                        lane_far = lane_far && (u * u > st.far2);
                    }
                }
                // the warp's nearest energy (non-negative floats order as integers)
                const float wmin = __uint_as_float(__reduce_min_sync(kAll, __float_as_uint(umin)));
                const float R2 = st.far2 * (1.f / 16.f);
                if (R2 * 256.f < wmin) {
                    re_series4<5>(mu, v, r);
                } else if (R2 * 64.f < wmin) {
                    re_series4<7>(mu, v, r);
                } else if (lane_far) {
                    re_series4<kReMom>(mu, v, r);
                } else {
                    const ReSeg T = wq[st.loc];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float u = w[k] - st.c;
                        if (u * u > st.far2) {
                            float p = mu[kReMom];
#pragma unroll
                            for (int n = kReMom - 1; n >= 0; --n) p = fmaf(p, v[k], mu[n]);
                            r[k] = p * v[k];
                        } else {
                            r[k] = re_near(T, w[k]);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) sum[k] = fmaf(st.amp, r[k], sum[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = c0 + lane + 32 * k;
                if (i < S.n_om) S.racc[i] += sum[k];
            }
        }
        __syncwarp();
        since_flush += n_here;
        if (since_flush >= kReFlush) {
            re_flush(S, lane);
            since_flush = 0;
        }
    }
    __syncwarp();
    wn[lane] = 0;
    __syncwarp();
}

template <int KIND>
__host__ __device__ constexpr int queue_entries() { return KIND == kKindS ? kQueueCap : 32 * kSubPerPair; }
template <int KIND>
__host__ __device__ constexpr int queue_counts() { return KIND == kKindS ? 2 : 32; }

template <int KIND>
__host__ __device__ constexpr size_t queue_entry_bytes() { return KIND == kKindS ? sizeof(SubTet) : sizeof(ReSeg); }

// S: queues, counts, tile, energies. Real part: lane segments, counts,
// staged set-ups, FP32 sums, tile, energies.
template <int KIND>
size_t spec_smem_bytes(int n_om, int mode) {
    return queue_entry_bytes<KIND>() * kSpecWarps * queue_entries<KIND>() +
           sizeof(int) * kSpecWarps * queue_counts<KIND>() +
           (KIND == kKindRe ? sizeof(ReStage) * kSpecWarps * 32 + sizeof(float) * kSpecWarps * (size_t)n_om : 0) +
           sizeof(long long) * (size_t)n_om + sizeof(float) * (size_t)(mode == TETRA_BIN ? n_om + 1 : n_om);
}

template <int NB, int KIND>
__global__ void __launch_bounds__(kSpecThreads, KIND == kKindS ? kSpecBlocksPerSM : kReBlocksPerSM)
    spectral_t0_kernel(const float *eps, int eps_stride, int n1, int n2, int n3, int nx, int ny, int z0, int z1,
                       int qx, int qy, int qz, float mu, const float *omega, int n_om, int mode,
                       long long *partials, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int QW = queue_entries<KIND>(), QC = queue_counts<KIND>();
    unsigned char *qraw = smem;                                             // [warps][QW] entries
    int *qcount = reinterpret_cast<int *>(qraw + queue_entry_bytes<KIND>() * kSpecWarps * QW);   // [warps][QC]
    ReStage *stage = reinterpret_cast<ReStage *>(qcount + kSpecWarps * QC); // real part: [warps][32]
    float *racc = reinterpret_cast<float *>(stage + (KIND == kKindRe ? kSpecWarps * 32 : 0));   // [warps][n_om]
    long long *tile = reinterpret_cast<long long *>(racc + (KIND == kKindRe ? kSpecWarps * n_om : 0));
    float *om = reinterpret_cast<float *>(tile + n_om);
    const int n_edges = (mode == TETRA_BIN) ? n_om + 1 : n_om;
    for (int i = threadIdx.x; i < n_om; i += blockDim.x) tile[i] = 0;
    for (int i = threadIdx.x; i < n_edges; i += blockDim.x) om[i] = omega[i];
    for (int i = threadIdx.x; i < kSpecWarps * QC; i += blockDim.x) qcount[i] = 0;
    if constexpr (KIND == kKindRe)
        for (int i = threadIdx.x; i < kSpecWarps * n_om; i += blockDim.x) racc[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // V_T/V_G in fixed-point units: de * 2^26
    const double de = mean_spacing(om, n_om, mode);
    const float scale = (float)ldexp(de, kSpecBits);
    const float om_lo = om[0], om_hi = om[n_edges - 1];
    SubTet *wq = reinterpret_cast<SubTet *>(qraw) + warp * QW;   // S
    ReSeg *wr = reinterpret_cast<ReSeg *>(qraw) + warp * QW;     // real part
    int *wn = qcount + warp * QC;
    const SpecArgs S{om, tile, n_om, mode, scale, status, om_lo, om_hi, (float)(1.0 / de), wq,
                     KIND == kKindS ? wn : wn + lane, racc + warp * n_om, wr + lane * kSubPerPair,
                     stage + warp * 32};
    int since_flush = 0;   // real part: entries in the per-warp FP32 sums
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
            if constexpr (KIND == kKindS) {
                // lane 0's count, read after every push of the previous pair
                // and before any of this one: the same decision in every lane
                __syncwarp();
                const int queued = __shfl_sync(0xffffffffu, *S.qn, 0);
                if (queued >= kDrainAt) drain(S, lane);
            } else {
                re_process(S, wr, wn, lane, since_flush);   // the previous pair's sub-tetrahedra
            }
            const int n = pr / NB, m = pr - (pr / NB) * NB;
            bool plus = ((an >> n) & 1u) && ((cp >> m) & 1u);
            bool minus = ((ap >> n) & 1u) && ((cn >> m) & 1u);
            if (!plus && !minus) continue;
            if constexpr (KIND == kKindS) {
                const float d0 = c[0][m] - a[0][n], d1 = c[1][m] - a[1][n];
                const float d2 = c[2][m] - a[2][n], d3 = c[3][m] - a[3][n];
                const float dlo = fminf(fminf(d0, d1), fminf(d2, d3)), dhi = fmaxf(fmaxf(d0, d1), fmaxf(d2, d3));
                if (dhi < om_lo || dlo > om_hi) continue;
                plus = plus && om_hi > 0.f;
                minus = minus && om_lo < 0.f;
                if (!plus && !minus) continue;
            }
            const P5 v0{1.f, 0.f, 0.f, a[0][n], c[0][m]};
            const P5 v1{0.f, 1.f, 0.f, a[1][n], c[1][m]};
            const P5 v2{0.f, 0.f, 1.f, a[2][n], c[2][m]};
            const P5 v3{0.f, 0.f, 0.f, a[3][n], c[3][m]};
            const uint32_t key = ((uint32_t)it * (uint32_t)(NB * NB) + (uint32_t)(n * NB + m)) * 2u;
            // band n occupied and band m empty at every corner: the +1
            // region is the whole tetrahedron (the same sub-tetrahedron and
            // dither key the two cuts would produce)
            if (((a_all >> n) & 1u) && ((c_all >> m) & 1u)) {
                accumulate<KIND>(v0, v1, v2, v3, 1.f, key * 16u, S);
                continue;
            }
            // +1 on {a < 0, c > 0}; -1 on {a > 0, c < 0}
            if (plus) region<KIND>(v0, v1, v2, v3, 0, 3, 1.f, key, S);
            if (minus) region<KIND>(v0, v1, v2, v3, 1, 2, -1.f, key + 1u, S);
        }
    }
    if constexpr (KIND == kKindS) {
        drain(S, lane);
    } else {
        re_process(S, wr, wn, lane, since_flush);
        re_flush(S, lane);
    }
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
template <int KIND>
int spectral_grid(const Plan &P) { return (KIND == kKindS ? kSpecBlocksPerSM : kReBlocksPerSM) * P.sm_count; }

template <int NB, int KIND>
cudaError_t launch_spectral_nb(const Plan &P, const float *eps, const int q[3], float mu, const float *omega,
                               int n_om, int mode, long long *partials, int *status, int grid,
                               size_t smem, cudaStream_t stream) {
    auto k = spectral_t0_kernel<NB, KIND>;
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

template <int KIND>
size_t spectral_workspace(const Plan &P, int n_om) {
    return kStatusBytes + sizeof(long long) * (size_t)spectral_grid<KIND>(P) * (size_t)n_om;
}

template <int KIND>
tetra_status_t launch_spectral(const Plan &P, const float *eps, const int q_in[3], float mu, int mode, int n_om,
                               const float *omega, float *S, void *ws, size_t ws_bytes, cudaStream_t stream) {
    if (n_om < 1 || (mode != TETRA_POINT && mode != TETRA_BIN)) return TETRA_EINVAL;
    if (P.d.n_bands > 8) return TETRA_EUNSUPPORTED;
    // the bands at k + q come from every plane of the grid
    if (P.z0 != 0 || P.z1 != P.d.n3) return TETRA_EUNSUPPORTED;
    const size_t smem = spec_smem_bytes<KIND>(n_om, mode);
    if (smem > P.smem_optin) return TETRA_EUNSUPPORTED;
    if (ws_bytes < spectral_workspace<KIND>(P, n_om)) return TETRA_ENOMEM;
    const double vtvg = 1.0 / (6.0 * (double)P.d.n1 * (double)P.d.n2 * (double)P.d.n3);
    const int q[3] = {mod_q(q_in[0], P.d.n1), mod_q(q_in[1], P.d.n2), mod_q(q_in[2], P.d.n3)};
    const int grid = spectral_grid<KIND>(P);
    int *status = reinterpret_cast<int *>(ws);
    long long *partials = reinterpret_cast<long long *>(static_cast<unsigned char *>(ws) + kStatusBytes);
    if (cudaMemsetAsync(ws, 0, kStatusBytes, stream) != cudaSuccess) return TETRA_ECUDA;
    cudaError_t e;
    switch (P.d.n_bands) {
        case 1: e = launch_spectral_nb<1, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 2: e = launch_spectral_nb<2, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 3: e = launch_spectral_nb<3, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 4: e = launch_spectral_nb<4, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 5: e = launch_spectral_nb<5, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 6: e = launch_spectral_nb<6, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        case 7: e = launch_spectral_nb<7, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
        default: e = launch_spectral_nb<8, KIND>(P, eps, q, mu, omega, n_om, mode, partials, status, grid, smem, stream); break;
    }
    if (e != cudaSuccess) return TETRA_ECUDA;
    spectral_reduce_kernel<<<(n_om + 255) / 256, 256, 0, stream>>>(partials, grid, n_om, mode, omega, vtvg, S);
    return cudaGetLastError() == cudaSuccess ? TETRA_OK : TETRA_ECUDA;
}

}  // namespace

size_t spectral_t0_workspace(const Plan &P, int n_om) { return spectral_workspace<kKindS>(P, n_om); }

tetra_status_t launch_spectral_t0(const Plan &P, const float *eps, const int q_in[3], float mu, int mode, int n_om,
                                  const float *omega, float *S, void *ws, size_t ws_bytes, cudaStream_t stream) {
    return launch_spectral<kKindS>(P, eps, q_in, mu, mode, n_om, omega, S, ws, ws_bytes, stream);
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

extern "C" size_t tetra_chi0_real_t0_workspace_bytes(tetra_plan_t plan, int n_omega) {
    if (!plan || n_omega < 1) return 0;
    return tetra::spectral_workspace<tetra::kKindRe>(*plan, n_omega);
}

extern "C" tetra_status_t tetra_chi0_real_t0(tetra_plan_t plan, const float *eps, const int q[3], float mu,
                                             int n_omega, const float *omega, float *R, void *ws, size_t ws_bytes,
                                             cudaStream_t stream) {
    if (!plan || !eps || !q || !omega || !R || !ws) return TETRA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(eps) & 15u) || (reinterpret_cast<uintptr_t>(ws) & 15u)) return TETRA_EINVAL;
    const tetra::DeviceGuard dg(plan->device);
    if (!dg.ok()) return TETRA_ECUDA;
    return tetra::launch_spectral<tetra::kKindRe>(*plan, eps, q, mu, TETRA_POINT, n_omega, omega, R, ws, ws_bytes,
                                                  stream);
}
