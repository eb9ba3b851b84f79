// Forward kernel of the linear tetrahedron orbital-resolved DOS
// (arXiv:1710.10789, Sec. II.C weights, Eqs. (8)-(9)) for sm_103a.
//
// Work decomposition
//  * The cube grid [0,n1) x [0,n2) x [z0,z1) is cut into boxes of BX*BY*BZ
//    cubes. A persistent CTA walks a sequence of boxes and, for each, has the
//    box's (BX+1)(BY+1)(BZ+1) corner points of all bands (energies and orbital
//    weights, tetra layout) copied into shared memory by two 4-D TMA loads:
//    the energies double buffered across boxes, the weights (read only by the
//    walks) in one slot loaded behind the next box's window pass. One model: boxes blockIdx.x, blockIdx.x +
//    gridDim.x, ... (blockIdx.y = energy chunk). A batch of models: each CTA
//    claims the next (model, box) item from a global counter (models in
//    order), so the work stays balanced whatever the models' costs; when the
//    model changes the CTA flushes its tile into that model's int64
//    accumulator with integer atomics and reloads the energy grid.
//  * One thread handles one (tetrahedron, band) item: it reads the four corner
//    energies, sorts them with a 5-comparator network carrying the corner
//    positions (Sec. II.C sorts E1 <= E2 <= E3 <= E4), reads the orbital
//    weights in sorted order, and visits only the energies strictly inside
//    (E1, E4) (bins overlapping it in bin mode); all others get zero weight.
//  * Up to 8 orbitals (every mode): the item is a pair of tetrahedra sharing
//    a face (Table I's six form three such pairs). Their windows overlap
//    heavily, so one walk over the union of the two windows adds both
//    tetrahedra's contributions at each energy before touching the shared
//    tile: about half the shared-memory traffic of one tetrahedron each.
//    (Integrated mode: each tetrahedron adds its weights below its own E4
//    and puts its own saturation step.)
//  * Items of a box are ranked by window length (counting sort), so the 32
//    lanes of a warp walk windows of nearly equal length.
//  * Each visited energy adds sum_l b_{l,s} dw_l to the CTA's tile for every
//    orbital s (Eq. (8)).
//
// Accumulation: exact fixed point, no float atomics anywhere
//  * Contributions are scaled by 1/u, u = (V_T/V_G) / dE * 2^-F (dE = mean
//    grid spacing, F = fixed_bits), rounded to integers and added with integer
//    shared-memory atomics into an int32 tile [energies][n_orb + 1]. Integer
//    addition is associative, so the tile does not depend on thread order.
//  * The rounding adds 1.5 * 2^23 in FP32 and the tile receives the raw bit
//    pattern, i.e. the integer plus the constant bias M = 0x4B400000. The
//    extra column of each tile row counts (as differences: +1 at a window's
//    first energy, -1 after its last) how many adds the row received, so a
//    row's value is recovered modulo 2^32 as raw - count * M when it is
//    flushed.
//  * A per-item bound q_max (|b| <= Bmax of the box, and the tetrahedron DOS
//    is at most 3/E41 of V_T/V_G) decides between this fast path and a 64-bit
//    global integer path for rare near-flat tetrahedra. The sum of q_max over
//    processed items bounds every tile entry; the tile is flushed into the
//    CTA's int64 partial in global memory before it could overflow.
//  * tetra_dos_reduce sums the per-CTA int64 partials (exact) and scales by u;
//    for a batch, each model's accumulator is scaled.
#include <atomic>
#include <memory>
#include <new>

#include "tetra_internal.cuh"

namespace tetra {

namespace {

constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23: float + kMagic rounds to an integer
constexpr int kMagicBits = 0x4B400000;  // bit pattern of kMagic
constexpr uint32_t kSmemAlign = 1024;
// Work unit, threads per CTA and registers per thread. Point mode with up to
// 8 orbitals walks face-sharing tetrahedron pairs, holding two tetrahedra's
// weights and constants in registers; 16 orbitals would not fit, so there, as
// in bin mode, a unit is one tetrahedron. Each of the SM's four
// sub-partitions has 16K registers for its warps: 12 warps (3 per
// sub-partition) can use 168 registers per thread, 16 warps 128.
template <int MODE, int NORB>
struct Cfg {
    static constexpr bool pairs = NORB <= 8;
    static constexpr int threads = pairs ? 384 : 512;
    static constexpr int max_regs = pairs ? 168 : 128;
    static constexpr int units_per_cube = pairs ? 3 : 6;
};
constexpr int kMaxThreads = 512;
constexpr int kKBins = 256;     // window-length histogram bins (K >= 255 share one)

// Table I, corner labels minus one; label c sits at offset (c&1, (c>>1)&1, (c>>2)&1).
// Packed 3 bits per corner, 12 bits per tetrahedron, so that lanes holding
// different tetrahedra decode their corners from an immediate instead of
// serialising on divergent constant-memory reads.
constexpr int kTableI[6][4] = {{0, 1, 2, 5}, {1, 2, 3, 5}, {0, 2, 4, 5},
                               {2, 3, 5, 7}, {2, 4, 5, 6}, {2, 5, 6, 7}};
constexpr uint32_t pack_tet(int t) {
    return (uint32_t)(kTableI[t][0] | kTableI[t][1] << 3 | kTableI[t][2] << 6 | kTableI[t][3] << 9);
}
constexpr uint64_t kTetLo = (uint64_t)pack_tet(0) | (uint64_t)pack_tet(1) << 12 | (uint64_t)pack_tet(2) << 24 |
                            (uint64_t)pack_tet(3) << 36 | (uint64_t)pack_tet(4) << 48;
constexpr uint32_t kTetHi = pack_tet(5);
__device__ __forceinline__ uint32_t tet_code(int t) {
    return t < 5 ? (uint32_t)(kTetLo >> (12 * t)) & 0xFFFu : kTetHi;
}

// Table I's tetrahedra as three face-sharing pairs: (1st, 2nd), (3rd, 5th),
// (4th, 6th). Per pair five corner labels minus one: the three corners of the
// shared face, the corner only in the first tetrahedron, the corner only in
// the second. First tetrahedron = slots {0,1,2,3}, second = slots {0,1,2,4}.
constexpr int kPair[3][5] = {{1, 2, 5, 0, 3}, {2, 4, 5, 0, 6}, {2, 5, 7, 3, 6}};
constexpr uint32_t pack_pair(int p) {
    return (uint32_t)(kPair[p][0] | kPair[p][1] << 3 | kPair[p][2] << 6 | kPair[p][3] << 9 |
                      kPair[p][4] << 12);
}
constexpr uint64_t kPairCode = (uint64_t)pack_pair(0) | (uint64_t)pack_pair(1) << 16 |
                               (uint64_t)pack_pair(2) << 32;
__device__ __forceinline__ uint32_t pair_code(int p) { return (uint32_t)(kPairCode >> (16 * p)) & 0x7FFFu; }

// Launch constants shared by every model of a launch.
struct FwdArgs {
    int nb, n_orb;
    int BX, BY, BZ;
    int lbx, lby, lbz;   // log2 of the box sides (powers of two)
    int eps_stride, w_stride;
    uint32_t e_box_bytes, w_box_bytes;   // TMA bytes of a box's energies / weights
    uint32_t e_stage, w_stage;           // their shared-memory slots (128-byte multiples)
    int chunk_w;         // energies per shared tile (largest model of a batch)
    int tile_copies;     // copies of the tile; lane l of a bin-mode pair adds into copy l % tile_copies
    int items_per_box;   // items per box: (pair, band) in point mode, (tetrahedron, band) otherwise
    int fast_cap;
    unsigned flush_at;   // a 64-energy block is flushed once its bound reaches this
    long long *G;        // int64 partials, [slot][n_orb][chunk_w]
    long long *Gs;       // integrated mode: int64 partial step sums, [slot][n_orb][chunk_w]
    int *status;
    int *queue;          // batched: next unclaimed (model, box) work item
};

// Fixed-point unit, identical in every kernel that uses it. The DOS modes
// scale with the mean energy spacing (their values are per energy); the
// integrated occupation is dimensionless, so its unit does not depend on the
// grid (a narrow grid, as in a Fermi-level search, keeps full resolution).
__device__ __forceinline__ double fixed_unit(const float *omega, int n_omega, int mode, double vtvg,
                                             int bits) {
    double de;
    if (mode == TETRA_INTEGRATED)
        de = 1.0;
    else if (mode != TETRA_BIN)
        de = n_omega > 1 ? ((double)omega[n_omega - 1] - (double)omega[0]) / (n_omega - 1) : 1.0;
    else
        de = ((double)omega[n_omega] - (double)omega[0]) / n_omega;
    if (!(de > 0.0)) de = 1.0;
    return vtvg / de * ldexp(1.0, -bits);
}

__device__ __forceinline__ void cswap(float &ea, float &eb, int &pa, int &pb) {
    const bool s = eb < ea;
    const float lo = s ? eb : ea, hi = s ? ea : eb;
    const int plo = s ? pb : pa, phi = s ? pa : pb;
    ea = lo; eb = hi; pa = plo; pb = phi;
}

// One rounded contribution added to the CTA's int64 partial (global 64-bit
// integer atomics): the path of the rare items whose bound does not fit the
// int32 tile. acc holds the dithered value; the same single rounding to
// nearest as the tile path.
__device__ __forceinline__ void deposit_one(float acc, long long *g, int *status) {
    if (fabsf(acc) < 9.0e18f) {
        const long long q = __float2ll_rn(acc);
        if (q != 0) atomicAdd(reinterpret_cast<unsigned long long *>(g), static_cast<unsigned long long>(q));
    } else {
        atomicOr(status, kFlagRange);
    }
}

__device__ __forceinline__ void sort4(float (&e)[4], int (&p)[4]) {
    cswap(e[0], e[1], p[0], p[1]);
    cswap(e[2], e[3], p[2], p[3]);
    cswap(e[0], e[2], p[0], p[2]);
    cswap(e[1], e[3], p[1], p[3]);
    cswap(e[1], e[2], p[1], p[2]);
}

// Dither offset in [-1/2, 1/2) for one (tetrahedron, band) item, hashed from its
// global identity so it does not depend on the launch shape.
__device__ __forceinline__ float item_dither(uint32_t key) {
    uint32_t h = key * 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f;
}

// floor(a / d) for 0 <= a and 0 < d below 2^24: a float quotient corrected
// by one step (the TMA issue at the end of a box sits on every thread's path
// to the next barrier, so it avoids integer division).
__device__ __forceinline__ int fdivq(int a, int d) {
    int q = (int)__fdividef((float)a, (float)d);
    q -= (q * d > a) ? 1 : 0;
    q += ((q + 1) * d <= a) ? 1 : 0;
    return q;
}

__device__ __forceinline__ float safe_rcp(float x) { return x > 0.f ? __fdividef(1.0f, x) : 0.f; }

// Per-item constants of the weight formulas, in fixed-point units.
struct Tet {
    float e1, e2, e3, e4;
    float r21, r31, r41, r32, r42, r43;
    float P1, S1, P3, S3, k1, k2, k3, fq;
};

__device__ __forceinline__ void tet_setup(Tet &T, float e1, float e2, float e3, float e4, float fq) {
    T.e1 = e1; T.e2 = e2; T.e3 = e3; T.e4 = e4;
    T.r21 = safe_rcp(e2 - e1); T.r31 = safe_rcp(e3 - e1); T.r41 = safe_rcp(e4 - e1);
    T.r32 = safe_rcp(e3 - e2); T.r42 = safe_rcp(e4 - e2); T.r43 = safe_rcp(e4 - e3);
    T.P1 = 4.f * fq * T.r21 * T.r31 * T.r41;
    T.S1 = T.r21 + T.r31 + T.r41;
    T.P3 = 4.f * fq * T.r41 * T.r42 * T.r43;
    T.S3 = T.r41 + T.r42 + T.r43;
    T.k1 = fq * T.r31 * T.r41;
    T.k2 = fq * T.r31 * T.r32 * T.r41;
    T.k3 = fq * T.r32 * T.r41 * T.r42;
    T.fq = fq;
}

// Point-mode constants of one item, for a branch-free evaluation of the four
// corner derivatives dw_l/dE at any E strictly inside (E1, E4):
//  * cases E1 < E <= E2 and E3 < E < E4 share one mirrored form: with
//    v = E - E1 (or E4 - E), g = P v^2, the apex corner (1, or 4) gets
//    g (3 - v S) and the other three g v / E_j1 (or g v / E_4j);
//  * in E2 < E <= E3 every dw_l is a cubic in t = E - E2, evaluated by
//    Horner from coefficients expanded from the printed C1, C2, C3 forms.
// e2c is the upper end of the first case: E2, or the float just below E4 when
// E2 = E4 (then no energy below E4 may take the first case's form).
struct TetP {
    float e1, e2, e3, e4, e2c;
    float P1, S1, r21, r31, r41;
    float P3, S3, r42, r43;
    float c[4][4];   // c[l][m]: coefficient of t^m in dw_l (case E2 < E <= E3)
};

__device__ __forceinline__ void tetp_setup(TetP &T, float e1, float e2, float e3, float e4, float fq) {
    T.e1 = e1; T.e2 = e2; T.e3 = e3; T.e4 = e4;
    T.e2c = (e2 < e4) ? e2 : nextafterf(e4, -INFINITY);
    const float A = e2 - e1, B = e3 - e2, C = e4 - e2;
    T.r21 = safe_rcp(A); T.r31 = safe_rcp(e3 - e1); T.r41 = safe_rcp(e4 - e1);
    const float r32 = safe_rcp(B);
    T.r42 = safe_rcp(C); T.r43 = safe_rcp(e4 - e3);
    T.P1 = 4.f * fq * T.r21 * T.r31 * T.r41;
    T.S1 = T.r21 + T.r31 + T.r41;
    T.P3 = 4.f * fq * T.r41 * T.r42 * T.r43;
    T.S3 = T.r41 + T.r42 + T.r43;
    const float r31 = T.r31, r41 = T.r41, r42 = T.r42;
    const float k1 = fq * r31 * r41, k2 = fq * r31 * r32 * r41, k3 = fq * r32 * r41 * r42;
    const float k1r31 = k1 * r31, k1r41 = k1 * r41, k2r31 = k2 * r31, k2r41 = k2 * r41;
    const float k2r32 = k2 * r32, k3r41 = k3 * r41, k3r32 = k3 * r32, k3r42 = k3 * r42;
    T.c[0][0] = -A * (A * (k1r31 + k1r41) - B * B * k2r31 - B * C * k2r41 - 2.f * B * k1r31 -
                      2.f * C * k1r41 - 2.f * k1);
    T.c[0][1] = -2.f * (2.f * A * B * k2r31 + A * B * k2r41 + A * C * k2r41 + 2.f * A * k1r31 +
                        2.f * A * k1r41 - B * B * k2r31 - B * C * k2r41 - B * k1r31 -
                        C * C * k3r41 - C * k1r41 - k1);
    T.c[0][2] = -3.f * (-A * k2r31 - A * k2r41 + 2.f * B * k2r31 + B * k2r41 + C * k2r41 +
                        2.f * C * k3r41 + k1r31 + k1r41);
    T.c[0][3] = 4.f * (k2r31 + k2r41 + k3r41);
    T.c[1][0] = A * (B * B * k2r32 + B * k2 + 2.f * k1);
    T.c[1][1] = -2.f * (2.f * A * B * k2r32 + A * k2 - B * B * k2r32 - B * C * k3r32 - B * k2 -
                        C * C * k3r42 - C * k3 - k1);
    T.c[1][2] = 3.f * (A * k2r32 - 2.f * B * k2r32 - B * k3r32 - C * k3r32 - 2.f * C * k3r42 - k2 - k3);
    T.c[1][3] = 4.f * (k2r32 + k3r32 + k3r42);
    T.c[2][0] = A * A * r31 * (B * k2 + 3.f * k1);
    T.c[2][1] = 2.f * A * (-A * k2r31 + 2.f * B * k2r31 + B * k2r32 + 3.f * k1r31);
    T.c[2][2] = 3.f * (-2.f * A * k2r31 - A * k2r32 + B * k2r31 + B * k2r32 + C * k3r32 + k1r31);
    T.c[2][3] = -4.f * (k2r31 + k2r32 + k3r32);
    T.c[3][0] = A * A * r41 * (B * k2 + 3.f * k1);
    T.c[3][1] = 2.f * A * r41 * (-A * k2 + 2.f * B * k2 + C * k3 + 3.f * k1);
    T.c[3][2] = 3.f * (-2.f * A * k2r41 - A * k3r41 + B * k2r41 + C * k3r41 + C * k3r42 + k1r41);
    T.c[3][3] = -4.f * (k2r41 + k3r41 + k3r42);
}

// Valid at any E: outside (E1, E4) the clamped distance v = 0 makes every
// derivative exactly zero (E >= E4 always takes the E4 - E form). At E = E3
// the third case's form is used (equal to the second's by continuity). The
// two mirrored forms give, in sorted corner order, (apex, u r21, u r31, u r41)
// for the first case and (u r41, u r42, u r43, apex) for the third, so the
// first and last outputs swap apex and u r41 and the middle two pick their
// reciprocal: fewer selects than choosing every parameter first.
// LEAN (the single-model kernel): the first case tested against the stored
// e2c, and the mirrored forms' outputs picked as above. Otherwise (the
// batched kernel, which has no register to spare for the leaner form: it
// spilled there) the same values from the five selected parameters of the
// case and one test E <= E2 and E < E4 (the same set as E <= e2c).
template <bool LEAN = true>
__device__ __forceinline__ void tetp_dw(const TetP &T, float E, float d[4]) {
    const bool in1 = LEAN ? E <= T.e2c : (E <= T.e2 && E < T.e4);
    const bool in3 = !in1 && E >= T.e3;
    const float v = fmaxf(in1 ? E - T.e1 : T.e4 - E, 0.f);
    const float P = in1 ? T.P1 : T.P3;
    const float S = in1 ? T.S1 : T.S3;
    const float g = P * v * v;
    const float apex = g * fmaf(-v, S, 3.f);
    const float u = g * v;
    float m0, m1, m2, m3;
    if constexpr (LEAN) {
        const float u41 = u * T.r41;
        m0 = in1 ? apex : u41;
        m1 = u * (in1 ? T.r21 : T.r42);
        m2 = u * (in1 ? T.r31 : T.r43);
        m3 = in1 ? u41 : apex;
    } else {
        const float ra = in1 ? T.r21 : T.r41, rb = in1 ? T.r31 : T.r42, rc = in1 ? T.r41 : T.r43;
        const float o1 = u * ra, o2 = u * rb, o3 = u * rc;
        m0 = in1 ? apex : o1;
        m1 = in1 ? o1 : o2;
        m2 = in1 ? o2 : o3;
        m3 = in1 ? o3 : apex;
    }
    const float t = E - T.e2;
    float h[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) h[l] = fmaf(fmaf(fmaf(T.c[l][3], t, T.c[l][2]), t, T.c[l][1]), t, T.c[l][0]);
    const bool in2 = !in1 && !in3;
    d[0] = in2 ? h[0] : m0;
    d[1] = in2 ? h[1] : m1;
    d[2] = in2 ? h[2] : m2;
    d[3] = in2 ? h[3] : m3;
}

// w_l(E) for any E (Sec. II.C, all five cases), sorted corners.
template <bool OPEN = false>
__device__ __forceinline__ void tet_weights(const Tet &T, float E, float w[4]) {
    if (E <= T.e1) {
        w[0] = w[1] = w[2] = w[3] = 0.f;
    } else if (E >= T.e4) {
        // saturated; OPEN: zero, the saturated part being added elsewhere
        w[0] = w[1] = w[2] = w[3] = OPEN ? 0.f : T.fq;
    } else if (E <= T.e2) {
        const float x = E - T.e1;
        const float C = 0.25f * T.P1 * x * x * x;
        w[0] = C * fmaf(-x, T.S1, 4.f);
        const float cx = C * x;
        w[1] = cx * T.r21; w[2] = cx * T.r31; w[3] = cx * T.r41;
    } else if (E <= T.e3) {
        const float a = E - T.e1, bq = E - T.e2, c = T.e3 - E, dd = T.e4 - E;
        const float C1 = T.k1 * a * a;
        const float C2 = T.k2 * a * bq * c;
        const float C3 = T.k3 * bq * bq * dd;
        const float S12 = C1 + C2, S23 = C2 + C3, S123 = S12 + C3;
        w[0] = C1 + S12 * c * T.r31 + S123 * dd * T.r41;
        w[1] = S123 + S23 * c * T.r32 + C3 * dd * T.r42;
        w[2] = S12 * a * T.r31 + S23 * bq * T.r32;
        w[3] = S123 * a * T.r41 + C3 * bq * T.r42;
    } else {
        const float y = T.e4 - E;
        const float C = 0.25f * T.P3 * y * y * y;
        const float cy = C * y;
        w[0] = T.fq - cy * T.r41; w[1] = T.fq - cy * T.r42; w[2] = T.fq - cy * T.r43;
        w[3] = T.fq - C * fmaf(-y, T.S3, 4.f);
    }
}

// Adds one energy's contribution of an item directly to the CTA's int64
// partial (global integer atomics): the path of the rare items whose bound
// does not fit the int32 tile. Same dithered single rounding as the tile path:
// round(c + delta - 1/2) with delta in [0,1) hashed from the item.
template <int NORB>
__device__ __forceinline__ void deposit_slow(const float (&b)[4][NORB], const float d[4], int n_orb,
                                             float dith, long long *gcol, int g_stride, int *status) {
#pragma unroll
    for (int s = 0; s < NORB; ++s) {
        if (s < n_orb) {
            float acc = fmaf(b[0][s], d[0], dith);
            acc = fmaf(b[1][s], d[1], acc);
            acc = fmaf(b[2][s], d[2], acc);
            acc = fmaf(b[3][s], d[3], acc);
            if (fabsf(acc) < 9.0e18f) {
                const long long q = __float2ll_rn(acc);
                if (q != 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(gcol + (long)s * g_stride),
                              static_cast<unsigned long long>(q));
            } else {
                atomicOr(status, kFlagRange);
            }
        }
    }
}

// Energy window of one item, as global indices clipped to this CTA's chunk
// [w0, w0+wc): point mode, energies strictly inside (e1, e4); bin mode, bins
// whose weight difference can be non-zero (upper edge > e1, and lower edge
// < e4 or <= e1). The estimate from the mean spacing is corrected against the
// cached grid, so any ascending grid gives the exact window.
template <int MODE>
__device__ __forceinline__ void item_window(float e1, float e4, const float *om, int w0, int wc,
                                            float om0, float inv_de, int n_omega, int &lo, int &hi) {
    const float flo = fminf(fmaxf((e1 - om0) * inv_de, -2.f), (float)n_omega + 2.f);
    const float fhi = fminf(fmaxf((e4 - om0) * inv_de, -2.f), (float)n_omega + 2.f);
    if (MODE != TETRA_BIN) {
        lo = min(max((int)floorf(flo) + 1, w0), w0 + wc);
        hi = max(min((int)ceilf(fhi) - 1, w0 + wc - 1), w0 - 1);
        while (lo > w0 && om[lo - 1 - w0] > e1) --lo;
        while (lo < w0 + wc && om[lo - w0] <= e1) ++lo;
        while (hi < w0 + wc - 1 && om[hi + 1 - w0] < e4) ++hi;
        while (hi >= w0 && om[hi - w0] >= e4) --hi;
    } else {
        lo = min(max((int)floorf(flo), w0), w0 + wc);
        hi = max(min((int)ceilf(fhi), w0 + wc - 1), w0 - 1);
        while (lo > w0 && om[lo - w0] > e1) --lo;
        while (lo < w0 + wc && om[lo + 1 - w0] <= e1) ++lo;
        while (hi < w0 + wc - 1 && (om[hi + 1 - w0] < e4 || om[hi + 1 - w0] <= e1)) ++hi;
        while (hi >= w0 && !(om[hi - w0] < e4 || om[hi - w0] <= e1)) --hi;
    }
}

// One model of a launch: grid, energy grid and where its partial sums go.
struct ModelP {
    int n1, n2, n3, z0, z1, nbx, nby, n_boxes, n_omega;
    int fixed_bits;
    int box_base;    // first global work index of the model (batched launches)
    double vtvg;
    const float *omega;
};

struct MapPair {   // CUtensorMap is 128-byte aligned
    CUtensorMap e, w;
};

// Per-launch model table, passed by value (kernel parameter space).
template <int MAXM>
struct Batch {
    MapPair maps[MAXM];
    ModelP m[MAXM];
    int n_models;
    int total_work;   // batched: (model, box) items of the launch
};

template <int NORB, typename WT, int MODE, int MAXM>
__global__ void __maxnreg__((Cfg<MODE, NORB>::max_regs))
    tetra_dos_fwd_kernel(const __grid_constant__ Batch<MAXM> B, const FwdArgs A) {
    // tile row: NORB orbitals + the row's add count (differences); the odd
    // row length also spreads consecutive rows over the shared-memory banks
    constexpr int TS = NORB + 1;
    constexpr int CNT = NORB;
    extern __shared__ unsigned char smem_raw[];
    // TMA destinations need an aligned base; the dynamic area starts after the
    // static variables, so align it here (the host reserves kSmemAlign bytes).
    unsigned char *smem = smem_raw + ((kSmemAlign - (smem_u32(smem_raw) & (kSmemAlign - 1))) &
                                      (kSmemAlign - 1));
    const int tid = threadIdx.x;
    const int chunk = blockIdx.y;   // energy chunk (single-model launches)
    // shared memory carve-up
    // energies of two boxes (pass A of box k+1 needs no weights) and the
    // weights of one box, refilled after pass B and loaded while the next
    // box's pass A and ranking run
    unsigned char *estage[2] = {smem, smem + A.e_stage};
    unsigned char *wstage = smem + 2 * A.e_stage;
    int *tile = reinterpret_cast<int *>(wstage + A.w_stage);   // [copies][chunk_w + 1][TS]
    // (copies only for single-model bin-mode pairs; elsewhere one, known at
    // compile time: the batched kernel measured faster without them)
    constexpr bool kCopies = MODE == TETRA_BIN && Cfg<MODE, NORB>::pairs && MAXM == 1;
    const int n_copies = kCopies ? A.tile_copies : 1, copy_ints = TS * (A.chunk_w + 1);
    // integrated mode: per-orbital sums of the saturated weights of the items
    // whose E4 lies between energy j-1 and j, [chunk_w][NORB] (plain integers)
    int *stile = tile + copy_ints * n_copies;
    float *om = reinterpret_cast<float *>(stile + (MODE == TETRA_INTEGRATED ? NORB * A.chunk_w : 0));
    float *iw = om + A.chunk_w + 1;                                   // 1/bin width (bin mode)
    unsigned *blk_bound = reinterpret_cast<unsigned *>(iw + (MODE == TETRA_BIN ? A.chunk_w : 0));
    const int n_blk = (A.chunk_w + 63) >> 6;
    // (one set of block bounds per tile copy: copy c's bounds at c * n_blk)
    short *s_lo = reinterpret_cast<short *>(blk_bound + n_blk * n_copies);   // window start - w0
    unsigned short *s_K = reinterpret_cast<unsigned short *>(s_lo + A.items_per_box);
    unsigned short *s_list = s_K + A.items_per_box;                 // items sorted by K
    int *khist = reinterpret_cast<int *>(
        (reinterpret_cast<uintptr_t>(s_list + A.items_per_box) + 15) & ~uintptr_t(15));
    int *kcursor = khist + kKBins;           // rank cursors per window length
    uint64_t *mbar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(kcursor + kKBins) + 15) & ~uintptr_t(15));
    __shared__ float red_f[kMaxThreads / 32];
    __shared__ int s_wsum[kMaxThreads / 32];
    __shared__ int s_abort, s_active, s_slot;
    __shared__ int s_cdelta[8];   // staged-box point offset of cube corner c
    __shared__ int n_issued[3];   // TMA loads issued per mbarrier (thread 0 keeps them)

    // self-check of the shared-memory carve-up against the launch's dynamic size
    {
        const uintptr_t need = reinterpret_cast<uintptr_t>(mbar + 3) - reinterpret_cast<uintptr_t>(smem_raw);
        const bool bad = need > dynamic_smem_bytes() || (smem_u32(estage[0]) & 127u) != 0 ||
                         (A.e_stage & 127u) != 0 || (A.w_stage & 127u) != 0 || A.e_box_bytes > A.e_stage ||
                         A.w_box_bytes > A.w_stage || (smem_u32(mbar) & 7u) != 0 || A.items_per_box > 65535;
        if (bad) {
            if (tid == 0) atomicOr(A.status, kFlagConfig);
            return;
        }
    }
    if (tid < 8)
        s_cdelta[tid] = (tid & 1) + (A.BX + 1) * (((tid >> 1) & 1) + (A.BY + 1) * (tid >> 2));
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&mbar[0], 1);   // energies, stage 0
        mbar_init(&mbar[1], 1);   // energies, stage 1
        mbar_init(&mbar[2], 1);   // weights
        n_issued[0] = n_issued[1] = n_issued[2] = 0;
        fence_mbar_init();
    }

    // Work sequence of this CTA: item k -> (model, box). Single model: boxes
    // blockIdx.x, blockIdx.x + gridDim.x, ... Batched: thread 0 claims global
    // items (models in order, boxes within a model) from a counter, two steps
    // ahead, so every CTA stays busy until the batch is done; the claim for
    // step k+2 is issued when step k starts and decoded when step k ends (its
    // latency hidden behind the box), and s_wm / s_wb hold the decoded
    // (model, box) of steps k .. k+2 (model -1: no more work).
    __shared__ int s_wm[4], s_wb[4];
    int claim_m = 0;   // thread 0: model of its last claim (claims only grow)
    auto store_claim = [&](int k, int g) {   // thread 0 only
        if (g >= B.total_work) {
            s_wm[k & 3] = -1;
            return;
        }
        while (claim_m + 1 < B.n_models && B.m[claim_m + 1].box_base <= g) ++claim_m;
        s_wm[k & 3] = claim_m;
        s_wb[k & 3] = g - B.m[claim_m].box_base;
    };
    auto work = [&](int k, int &mi, int &box) -> bool {
        if (MAXM == 1) {
            mi = 0;
            box = blockIdx.x + k * gridDim.x;
            return box < B.m[0].n_boxes;
        }
        mi = s_wm[k & 3];
        box = s_wb[k & 3];
        return mi >= 0;
    };
    // energies of work item k (already claimed) into energy stage stg
    auto issue_e = [&](int k, int stg) {   // thread 0 only
        int mi, box;
        if (!work(k, mi, box)) return;
        const ModelP &Mk = B.m[mi];
        const int bq = fdivq(box, Mk.nbx), iz = fdivq(bq, Mk.nby), ix = box - bq * Mk.nbx, iy = bq - iz * Mk.nby;
        ++n_issued[stg];
        mbar_arrive_expect_tx(&mbar[stg], A.e_box_bytes);
        tma_load_4d(estage[stg], &B.maps[mi].e, 0, ix * A.BX, iy * A.BY, Mk.z0 + iz * A.BZ, &mbar[stg]);
    };
    // weights of work item k (already claimed) into the weight stage
    auto issue_w = [&](int k) {   // thread 0 only
        int mi, box;
        if (!work(k, mi, box)) return;
        const ModelP &Mk = B.m[mi];
        const int bq = fdivq(box, Mk.nbx), iz = fdivq(bq, Mk.nby), ix = box - bq * Mk.nbx, iy = bq - iz * Mk.nby;
        ++n_issued[2];
        mbar_arrive_expect_tx(&mbar[2], A.w_box_bytes);
        tma_load_4d(wstage, &B.maps[mi].w, 0, ix * A.BX, iy * A.BY, Mk.z0 + iz * A.BZ, &mbar[2]);
    };
    __syncthreads();
    // prologue: energies of the first two work items, weights of the first
    if (tid == 0) {
        if (MAXM > 1) {
            store_claim(0, atomicAdd(A.queue, 1));
            store_claim(1, atomicAdd(A.queue, 1));
        }
        issue_e(0, 0);
        issue_e(1, 1);
        issue_w(0);
    }
    int g_next = 0;   // thread 0: the claim in flight (step k+2)
    __syncthreads();

    const int PX = A.BX + 1, PY = A.BY + 1;
    const int ncube = A.BX * A.BY * A.BZ;   // a power of two
    const int lcube = A.lbx + A.lby + A.lbz;

    // state of the model whose boxes are being accumulated
    int cur = -1, w0 = 0, wc = 0;
    double u = 1.0;
    float fq = 0.f, om0 = 0.f, inv_de = 0.f, max_iw = 0.f;
    long long *Gc = A.G;
    // The count column of rows 0..wc: differences (as the walks update it)
    // to per-row add counts by a block-wide inclusive scan, and back. Each
    // warp scans a segment of rows; segment totals are combined through
    // shared memory. Called by every thread of the CTA.
    auto counts_from_diffs = [&](int *tile) {
        const int nw = (int)(blockDim.x >> 5), warp = tid >> 5, lane = tid & 31;
        const int nr = wc + 1;
        const int seg = ((nr + nw - 1) / nw + 31) & ~31;
        const int r0 = warp * seg, r1 = min(r0 + seg, nr);
        int carry = 0;
        for (int r = r0; r < r1; r += 32) {
            const int rr = r + lane;
            int x = rr < r1 ? tile[rr * TS + CNT] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            x += carry;
            if (rr < r1) tile[rr * TS + CNT] = x;
            carry = __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) s_wsum[warp] = carry;
        __syncthreads();
        int off = 0;
        for (int w2 = 0; w2 < warp; ++w2) off += s_wsum[w2];
        if (off != 0)
            for (int rr = r0 + lane; rr < r1; rr += 32) tile[rr * TS + CNT] += off;
        __syncthreads();
    };
    auto diffs_from_counts = [&](int *tile) {
        const int nw = (int)(blockDim.x >> 5), warp = tid >> 5, lane = tid & 31;
        const int nr = wc + 1;
        const int seg = ((nr + nw - 1) / nw + 31) & ~31;
        const int r0 = warp * seg, r1 = min(r0 + seg, nr);
        // the count before the segment belongs to another warp: read it first
        const int prev0 = (r0 > 0 && r0 < r1) ? tile[(r0 - 1) * TS + CNT] : 0;
        __syncthreads();
        if (r1 > r0) {
            // chunks last to first, so each chunk's predecessor is still a count
            for (int r = r0 + (((r1 - r0 - 1) >> 5) << 5); r >= r0; r -= 32) {
                const int rr = r + lane;
                const int x = rr < r1 ? tile[rr * TS + CNT] : 0;
                int pv = __shfl_up_sync(0xffffffffu, x, 1);
                if (lane == 0) pv = (r == r0) ? prev0 : tile[(r - 1) * TS + CNT];
                if (rr < r1) tile[rr * TS + CNT] = x - pv;
            }
        }
        __syncthreads();
    };
    // Value of a tile entry since its last flush: raw sum minus count * M
    // (modulo 2^32; the bounds keep the true value below 2^31 in magnitude).
    auto entry_value = [&](const int *tile, int j, int s) -> int {
        const unsigned n_add = (unsigned)tile[j * TS + CNT];
        return (int)((unsigned)tile[j * TS + s] - n_add * (unsigned)kMagicBits);
    };
    // the entry's value summed over the tile's copies
    auto entry_total = [&](int j, int s) -> int {
        int v = 0;
        for (int c = 0; c < n_copies; ++c) v += entry_value(tile + c * copy_ints, j, s);
        return v;
    };
    // moves the int32 tile of the current model into its int64 partial slot
    long long *Gsc = A.Gs;
    auto flush_tile = [&]() {
        for (int c = 0; c < n_copies; ++c) counts_from_diffs(tile + c * copy_ints);
        for (int i = tid; i < A.n_orb * wc; i += blockDim.x) {
            const int s = i / wc, j = i - s * wc;
            const int v = entry_total(j, s);
            if (v)
                atomicAdd(reinterpret_cast<unsigned long long *>(Gc + (long)s * A.chunk_w + j),
                          static_cast<unsigned long long>(static_cast<long long>(v)));
            if (MODE == TETRA_INTEGRATED) {
                const int sv = stile[j * NORB + s];
                if (sv)
                    atomicAdd(reinterpret_cast<unsigned long long *>(Gsc + (long)s * A.chunk_w + j),
                              static_cast<unsigned long long>(static_cast<long long>(sv)));
            }
        }
    };

    for (int k = 0;; ++k) {
        int mi, box;
        if (!work(k, mi, box)) break;
        if (MAXM > 1 && tid == 0) g_next = atomicAdd(A.queue, 1);
        const ModelP &M = B.m[mi];
        if (mi != cur) {
            // switch model: flush the previous one, reset the tile, cache the energy grid
            if (cur >= 0) flush_tile();
            __syncthreads();
            cur = mi;
            w0 = (MAXM == 1) ? chunk * A.chunk_w : 0;
            wc = min(A.chunk_w, M.n_omega - w0);
            // partial slot: one per (energy chunk, CTA) for a single model, one
            // per model for a batch (CTAs flush into it with integer atomics)
            const long slot = (MAXM == 1) ? (long)chunk * gridDim.x + blockIdx.x : (long)mi;
            Gc = A.G + slot * (long)A.n_orb * A.chunk_w;
            if (MODE == TETRA_INTEGRATED) Gsc = A.Gs + slot * (long)A.n_orb * A.chunk_w;
            for (int i = tid; i < copy_ints * n_copies; i += blockDim.x) tile[i] = 0;
            if (MODE == TETRA_INTEGRATED)
                for (int i = tid; i < NORB * A.chunk_w; i += blockDim.x) stile[i] = 0;
            for (int i = tid; i < n_blk * n_copies; i += blockDim.x) blk_bound[i] = 0;
            const int n_om = (MODE != TETRA_BIN) ? wc : wc + 1;
            for (int i = tid; i < n_om; i += blockDim.x) om[i] = M.omega[w0 + i];
            __syncthreads();
            if (MODE == TETRA_BIN)
                for (int i = tid; i < wc; i += blockDim.x) iw[i] = 1.0f / (om[i + 1] - om[i]);
            u = fixed_unit(M.omega, M.n_omega, MODE, M.vtvg, M.fixed_bits);
            fq = (float)(0.25 * M.vtvg / u);   // V_T/(4 V_G) in fixed-point units
            om0 = M.omega[0];
            const float omN = (MODE != TETRA_BIN) ? M.omega[M.n_omega - 1] : M.omega[M.n_omega];
            inv_de = (MODE != TETRA_BIN) ? (M.n_omega > 1 ? (float)(M.n_omega - 1) / (omN - om0) : 0.f)
                                           : (float)M.n_omega / (omN - om0);
            if (MODE == TETRA_BIN) {
                // the narrowest bin of the whole grid bounds every bin contribution
                max_iw = 0.f;
                for (int i = tid; i < M.n_omega; i += blockDim.x)
                    max_iw = fmaxf(max_iw, 1.0f / (M.omega[i + 1] - M.omega[i]));
                for (int o = 16; o; o >>= 1) max_iw = fmaxf(max_iw, __shfl_xor_sync(0xffffffffu, max_iw, o));
                if ((tid & 31) == 0) red_f[tid >> 5] = max_iw;
                __syncthreads();
                max_iw = 0.f;
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) max_iw = fmaxf(max_iw, red_f[i]);
            }
            __syncthreads();
        }
        const int st = k & 1;
        for (int i = tid; i < kKBins; i += blockDim.x) khist[i] = 0;
        if (tid == 0) s_slot = 0;
        const bool ok = mbar_wait_bounded(&mbar[st], (k >> 1) & 1, A.status);
        if (__syncthreads_or(!ok)) {
            s_abort = 1;
            break;
        }
        const float *Es = reinterpret_cast<const float *>(estage[st]);
        const WT *Ws = reinterpret_cast<const WT *>(wstage);
        const int ix = box % M.nbx, iy = (box / M.nbx) % M.nby, iz = box / (M.nbx * M.nby);
        const int gx0 = ix * A.BX, gy0 = iy * A.BY, gz0 = M.z0 + iz * A.BZ;
        const int lane = tid & 31, warp = tid >> 5, nwarp = (int)(blockDim.x >> 5);


        // Pass A: window of every item (corner min / max only) and a histogram
        // of its length K, so that pass B can hand items of similar length to
        // the same warp. The integers an item adds do not depend on which thread
        // adds them, so the grouping cannot change the result.
        // Each thread takes up to four items at once: their windows are
        // independent, so the corner loads and window searches of the four
        // overlap instead of running one after another.
        {
            constexpr int U = 4;
            const int stride_w = nwarp * 32;
            for (int base0 = warp * 32; base0 < A.items_per_box; base0 += stride_w * U) {
                int Ku[U], lou[U];
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const int it = base0 + uu * stride_w + lane;
                    // integrated mode: an item also counts when only its step (the
                    // first energy at or above E4) lies in the chunk; items off the
                    // grid get lo = w0 + wc, which makes them inactive
                    int K = 0, lo = (MODE == TETRA_INTEGRATED) ? w0 + wc : 0;
                    if (it < A.items_per_box) {
                        constexpr bool PAIRS = Cfg<MODE, NORB>::pairs;
                        constexpr int UPC = Cfg<MODE, NORB>::units_per_cube;
                        const int cube = it & (ncube - 1);
                        const int rest = it >> lcube;
                        const int t = rest % UPC, n = rest / UPC;
                        const int cx = cube & (A.BX - 1), cy = (cube >> A.lbx) & (A.BY - 1), cz = cube >> (A.lbx + A.lby);
                        if (gx0 + cx < M.n1 && gy0 + cy < M.n2 && gz0 + cz < M.z1) {
                            // a pair's window is the union of its two tetrahedra's:
                            // the window of the min / max over its five corners
                            float e1 = 3.0e38f, e4 = -3.0e38f;
                            const uint32_t code = PAIRS ? pair_code(t) : tet_code(t);
                            const int p0 = cx + PX * (cy + PY * cz);
#pragma unroll
                            for (int q = 0; q < (PAIRS ? 5 : 4); ++q) {
                                const int p = p0 + s_cdelta[(code >> (3 * q)) & 7];
                                const float ev = Es[p * A.eps_stride + n];
                                e1 = fminf(e1, ev);
                                e4 = fmaxf(e4, ev);
                            }
                            int hi;
                            item_window<MODE>(e1, e4, om, w0, wc, om0, inv_de, M.n_omega, lo, hi);
                            K = max(0, hi - lo + 1);
                        }
                    }
                    Ku[uu] = K;
                    lou[uu] = lo;
                }
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const int it = base0 + uu * stride_w + lane;
                    const int K = Ku[uu], lo = lou[uu];
                    if (it < A.items_per_box) {
                        s_lo[it] = (short)(lo - w0);
                        s_K[it] = (unsigned short)K;
                    }
                    const bool act = it < A.items_per_box && (K > 0 || (MODE == TETRA_INTEGRATED && lo + K < w0 + wc));
                    if constexpr (MODE == TETRA_INTEGRATED && Cfg<MODE, NORB>::pairs) {
                        // items with an empty window (only a step: every tetrahedron
                        // below the chunk) all count in bin 0, one add per warp
                        const unsigned zm = __ballot_sync(0xffffffffu, act && K == 0);
                        if (act && K > 0) atomicAdd(&khist[min(K, kKBins - 1)], 1);
                        if (zm && lane == __ffs(zm) - 1) atomicAdd(&khist[0], __popc(zm));
                    } else {
                        if (act) atomicAdd(&khist[min(K, kKBins - 1)], 1);
                    }
                }
            }
        }
        __syncthreads();
        // Items ranked by window length K: an exclusive scan of the K histogram
        // gives each length its first rank; an item's rank = first rank + its
        // place among items of equal K (atomic cursor; items of equal K are
        // interchangeable).
        if (tid < 32) {
            constexpr int PER = kKBins / 32;
            int v[PER], sum = 0;
#pragma unroll
            for (int j = 0; j < PER; ++j) { v[j] = khist[tid * PER + j]; sum += v[j]; }
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (tid >= o) x += y;
            }
            int run = x - sum;
#pragma unroll
            for (int j = 0; j < PER; ++j) { kcursor[tid * PER + j] = run; run += v[j]; }
            if (tid == 31) s_active = x;
        }
        __syncthreads();
        for (int base = warp * 32; base < A.items_per_box; base += nwarp * 32) {
            const int it = base + lane;
            const int K = it < A.items_per_box ? (int)s_K[it] : 0;
            const bool act = it < A.items_per_box &&
                             (K > 0 || (MODE == TETRA_INTEGRATED && s_lo[it] + K < wc));
            if constexpr (MODE == TETRA_INTEGRATED && Cfg<MODE, NORB>::pairs) {
                // empty windows: consecutive ranks from one cursor add per warp
                const unsigned zm = __ballot_sync(0xffffffffu, act && K == 0);
                if (act && K > 0) s_list[atomicAdd(&kcursor[min(K, kKBins - 1)], 1)] = (unsigned short)it;
                if (zm) {
                    const int lead = __ffs(zm) - 1;
                    int zb = 0;
                    if (lane == lead) zb = atomicAdd(&kcursor[0], __popc(zm));
                    zb = __shfl_sync(0xffffffffu, zb, lead);
                    if (act && K == 0) s_list[zb + __popc(zm & ((1u << lane) - 1u))] = (unsigned short)it;
                }
            } else {
                if (act) s_list[atomicAdd(&kcursor[min(K, kKBins - 1)], 1)] = (unsigned short)it;
            }
        }
        // the box's weights (loaded while pass A and the ranking ran), and
        // Bmax = max |w| over them (all of the box, padding included, so it
        // bounds every orbital weight an item can read)
        const bool okw = mbar_wait_bounded(&mbar[2], k & 1, A.status);
        float bmax = 0.f;
        if (okw) {
            const int n16 = (int)(A.w_box_bytes >> 4);
            const uint4 *src = reinterpret_cast<const uint4 *>(wstage);
            for (int i = tid; i < n16; i += blockDim.x) {
                const uint4 v = src[i];
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (sizeof(WT) == 4) {
                        bmax = fmaxf(bmax, fabsf(__uint_as_float(wv[q])));
                    } else {
                        const WT lo = *reinterpret_cast<const WT *>(&wv[q]);
                        const WT hi = *(reinterpret_cast<const WT *>(&wv[q]) + 1);
                        bmax = fmaxf(bmax, fmaxf(fabsf(to_f32<WT>(lo)), fabsf(to_f32<WT>(hi))));
                    }
                }
            }
        }
        for (int o = 16; o; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        if (lane == 0) red_f[warp] = bmax;
        if (__syncthreads_or(!okw)) {
            s_abort = 1;
            break;
        }
        bmax = 0.f;
        for (int i = 0; i < nwarp; ++i) bmax = fmaxf(bmax, red_f[i]);
        const int n_active = s_active;
        const int n_slots = (n_active + 31) >> 5;

        // Pass B: slot q holds the 32 items of ranks 32q .. 32q+31 (nearly equal
        // window length, so a warp's lanes finish together). Warps claim slots
        // longest windows first (a shared counter), which balances the warps'
        // work before the end-of-box barrier.
        for (;;) {
            int claim = 0;
            if (lane == 0) claim = atomicAdd(&s_slot, 1);
            claim = __shfl_sync(0xffffffffu, claim, 0);
            if (claim >= n_slots) break;
            const int pos = (n_slots - 1 - claim) * 32 + lane;
            const bool valid = pos < n_active;
            const int it = valid ? (int)s_list[pos] : 0;
            const int cube = it & (ncube - 1);
            const int rest = it >> lcube;
            const int cx = cube & (A.BX - 1), cy = (cube >> A.lbx) & (A.BY - 1), cz = cube >> (A.lbx + A.lby);
            const int p0 = cx + PX * (cy + PY * cz);
            const int lo = valid ? w0 + s_lo[it] : w0;
            const int hi = valid ? lo + s_K[it] - 1 : w0 - 1;
            const uint32_t gcube = (uint32_t)(gx0 + cx) +
                                   (uint32_t)M.n1 * ((uint32_t)(gy0 + cy) + (uint32_t)M.n2 * (uint32_t)(gz0 + cz));
            if constexpr (Cfg<MODE, NORB>::pairs) {
                // integrated mode: the lanes that hold an item, for the warp sums of
                // the steps on the chunk's first energy
                const unsigned vmask = (MODE == TETRA_INTEGRATED) ? __ballot_sync(0xffffffffu, valid) : 0u;
                if (!valid) continue;
                // ---- a pair of tetrahedra sharing a face, walked over the union window
                const int pr = rest % 3, n = rest / 3;
                const uint32_t code = pair_code(pr);
                float ea[4], eb[4];
                int pa[4], pb[4];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    pa[q] = pb[q] = p0 + s_cdelta[(code >> (3 * q)) & 7];
                    ea[q] = eb[q] = Es[pa[q] * A.eps_stride + n];
                }
                pa[3] = p0 + s_cdelta[(code >> 9) & 7];
                pb[3] = p0 + s_cdelta[(code >> 12) & 7];
                ea[3] = Es[pa[3] * A.eps_stride + n];
                eb[3] = Es[pb[3] * A.eps_stride + n];
                sort4(ea, pa);
                sort4(eb, pb);
                float ba[4][NORB], bb[4][NORB];
#pragma unroll
                for (int r4 = 0; r4 < 4; ++r4) {
                    load_weights<NORB, WT>(Ws + (long)pa[r4] * A.w_stride + n * A.n_orb, A.n_orb, ba[r4]);
                    load_weights<NORB, WT>(Ws + (long)pb[r4] * A.w_stride + n * A.n_orb, A.n_orb, bb[r4]);
                }
                const float dith = item_dither((gcube * 3u + (uint32_t)pr) * (uint32_t)A.nb + (uint32_t)n);
                if constexpr (MODE == TETRA_INTEGRATED) {
                    // Occupation: the walk over the union window adds each
                    // tetrahedron's weights below its own E4 (zero at and above
                    // it); from its step, the first energy at or above its E4,
                    // the saturated weights fq sum_l b_l enter the step tile.
                    // Every corner weight is at most V_T/(4 V_G): the pair adds
                    // at most 8 fq Bmax to any entry.
                    const float qmax = bmax * 8.f * fq * 1.01f;
                    const bool fast = qmax < (float)A.fast_cap;
                    int loa, hia, lob, hib;
                    item_window<MODE>(ea[0], ea[3], om, w0, wc, om0, inv_de, M.n_omega, loa, hia);
                    item_window<MODE>(eb[0], eb[3], om, w0, wc, om0, inv_de, M.n_omega, lob, hib);
                    // the first energy with saturated weights: at or above E4 and
                    // above E1 (a flat tetrahedron, E1 = E4, is empty at E = E1)
                    const int hsa = max(hia + 1, loa), hsb = max(hib + 1, lob);
                    const bool stepa = hsa < w0 + wc, stepb = hsb < w0 + wc;
                    // steps on the chunk's first energy (there go the steps of all
                    // tetrahedra below the chunk) are summed over the warp first
                    const bool firsta = fast && stepa && hsa == w0, firstb = fast && stepb && hsb == w0;
                    const unsigned qbnd = fast ? (unsigned)qmax + 2u : 0u;
                    if (fast) {
                        if (hi >= lo) {
                            for (int bk = (lo - w0) >> 6; bk <= ((hi - w0) >> 6); ++bk) atomicAdd(&blk_bound[bk], qbnd);
                            atomicAdd(&tile[(lo - w0) * TS + CNT], 1);
                            atomicAdd(&tile[(hi + 1 - w0) * TS + CNT], -1);
                        }
                        if (stepa && !firsta) atomicAdd(&blk_bound[(hsa - w0) >> 6], qbnd);
                        if (stepb && !firstb) atomicAdd(&blk_bound[(hsb - w0) >> 6], qbnd);
                    }
                    Tet TA, TB;
                    tet_setup(TA, ea[0], ea[1], ea[2], ea[3], fq);
                    tet_setup(TB, eb[0], eb[1], eb[2], eb[3], fq);
                    float sa[NORB], sb[NORB];   // saturated contributions fq sum_l b_{l,s}
#pragma unroll
                    for (int s = 0; s < NORB; ++s) {
                        sa[s] = fq * ((ba[0][s] + ba[1][s]) + (ba[2][s] + ba[3][s]));
                        sb[s] = fq * ((bb[0][s] + bb[1][s]) + (bb[2][s] + bb[3][s]));
                    }
                    if (__any_sync(vmask, firsta || firstb)) {
                        // the warp's first-energy steps (a tetrahedron whose step is
                        // there adds nothing in the window): integer sums, one add per orbital
                        const bool lead = lane == __ffs(vmask) - 1;
                        const unsigned bsum = __reduce_add_sync(vmask, (firsta ? qbnd : 0u) + (firstb ? qbnd : 0u));
                        if (lead && bsum) atomicAdd(&blk_bound[0], bsum);
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            const int v = (firsta ? __float_as_int(sa[s] + dith + kMagic) - kMagicBits : 0) +
                                          (firstb ? __float_as_int(sb[s] + dith + kMagic) - kMagicBits : 0);
                            const int tot = __reduce_add_sync(vmask, v);
                            if (lead && tot) atomicAdd(&stile[s], tot);
                        }
                    }
                    if (fast) {
                        const int K = hi - lo + 1;
                        int i = lo + ((lane * max(K, 1)) >> 5);
                        for (int j = 0; j < K; ++j) {
                            float wa[4], wb[4];
                            tet_weights<true>(TA, om[i - w0], wa);
                            tet_weights<true>(TB, om[i - w0], wb);
                            int *col = tile + (i - w0) * TS;
#pragma unroll
                            for (int s = 0; s < NORB; ++s) {
                                float acc = fmaf(ba[0][s], wa[0], dith);
                                acc = fmaf(ba[1][s], wa[1], acc);
                                acc = fmaf(ba[2][s], wa[2], acc);
                                acc = fmaf(ba[3][s], wa[3], acc);
                                acc = fmaf(bb[0][s], wb[0], acc);
                                acc = fmaf(bb[1][s], wb[1], acc);
                                acc = fmaf(bb[2][s], wb[2], acc);
                                acc = fmaf(bb[3][s], wb[3], acc);
                                atomicAdd(col + s, __float_as_int(acc + kMagic));
                            }
                            i = (i == hi) ? lo : i + 1;
                        }
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            if (stepa && !firsta)
                                atomicAdd(&stile[(hsa - w0) * NORB + s], __float_as_int(sa[s] + dith + kMagic) - kMagicBits);
                            if (stepb && !firstb)
                                atomicAdd(&stile[(hsb - w0) * NORB + s], __float_as_int(sb[s] + dith + kMagic) - kMagicBits);
                        }
                    } else {
                        for (int i = lo; i <= hi; ++i) {
                            float wa[4], wb[4];
                            tet_weights<true>(TA, om[i - w0], wa);
                            tet_weights<true>(TB, om[i - w0], wb);
#pragma unroll
                            for (int s = 0; s < NORB; ++s) {
                                if (s >= A.n_orb) continue;
                                float acc = fmaf(ba[0][s], wa[0], dith);
                                acc = fmaf(ba[1][s], wa[1], acc);
                                acc = fmaf(ba[2][s], wa[2], acc);
                                acc = fmaf(ba[3][s], wa[3], acc);
                                acc = fmaf(bb[0][s], wb[0], acc);
                                acc = fmaf(bb[1][s], wb[1], acc);
                                acc = fmaf(bb[2][s], wb[2], acc);
                                acc = fmaf(bb[3][s], wb[3], acc);
                                deposit_one(acc, Gc + (long)s * A.chunk_w + (i - w0), A.status);
                            }
                        }
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            if (s >= A.n_orb) continue;
                            if (stepa) deposit_one(sa[s] + dith, Gsc + (long)s * A.chunk_w + (hsa - w0), A.status);
                            if (stepb) deposit_one(sb[s] + dith, Gsc + (long)s * A.chunk_w + (hsb - w0), A.status);
                        }
                    }
                    continue;
                }
                if constexpr (MODE == TETRA_BIN) {
                    // Bin averages: each tetrahedron's weight step over the bin
                    // divided by its width (zero below E1; above E4 the weights
                    // are saturated and their steps vanish), bins walked in
                    // order so each upper edge's weights serve the next bin.
                    float qmax = bmax * 8.f * fq * max_iw * 1.01f;
                    if (!(ea[3] > ea[0]) || !(eb[3] > eb[0])) qmax = 3.0e38f;
                    const bool fast = qmax < (float)A.fast_cap;
                    // this lane's copy of the tile and of its block bounds (the
                    // copies are summed when flushed)
                    const int cp = n_copies > 1 ? lane % n_copies : 0;
                    int *tl = tile + cp * copy_ints;
                    unsigned *bl = blk_bound + cp * n_blk;
                    if (fast && hi >= lo) {
                        const unsigned qbnd = (unsigned)qmax + 2u;
                        for (int bk = (lo - w0) >> 6; bk <= ((hi - w0) >> 6); ++bk) atomicAdd(&bl[bk], qbnd);
                        atomicAdd(&tl[(lo - w0) * TS + CNT], 1);
                        atomicAdd(&tl[(hi + 1 - w0) * TS + CNT], -1);
                    }
                    Tet TA, TB;
                    tet_setup(TA, ea[0], ea[1], ea[2], ea[3], fq);
                    tet_setup(TB, eb[0], eb[1], eb[2], eb[3], fq);
                    float wpa[4], wpb[4];
                    tet_weights(TA, om[lo - w0], wpa);
                    tet_weights(TB, om[lo - w0], wpb);
                    int *col = tl + (lo - w0) * TS;
                    for (int i = lo; i <= hi; ++i, col += TS) {
                        float wna[4], wnb[4], da[4], db[4];
                        tet_weights(TA, om[i + 1 - w0], wna);
                        tet_weights(TB, om[i + 1 - w0], wnb);
                        const float sc = iw[i - w0];
#pragma unroll
                        for (int r4 = 0; r4 < 4; ++r4) {
                            da[r4] = (wna[r4] - wpa[r4]) * sc;
                            wpa[r4] = wna[r4];
                            db[r4] = (wnb[r4] - wpb[r4]) * sc;
                            wpb[r4] = wnb[r4];
                        }
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            if (!fast && s >= A.n_orb) continue;
                            float acc = fmaf(ba[0][s], da[0], dith);
                            acc = fmaf(ba[1][s], da[1], acc);
                            acc = fmaf(ba[2][s], da[2], acc);
                            acc = fmaf(ba[3][s], da[3], acc);
                            acc = fmaf(bb[0][s], db[0], acc);
                            acc = fmaf(bb[1][s], db[1], acc);
                            acc = fmaf(bb[2][s], db[2], acc);
                            acc = fmaf(bb[3][s], db[3], acc);
                            if (fast)
                                atomicAdd(col + s, __float_as_int(acc + kMagic));
                            else
                                deposit_one(acc, Gc + (long)s * A.chunk_w + (i - w0), A.status);
                        }
                    }
                    continue;
                }
                // bound on every |contribution| of the pair, in fixed-point units:
                // the tetrahedron DOS is at most 3/E41 of V_T/V_G; a flat
                // tetrahedron (E1 = E4) contributes nothing in point mode
                const float qa = (ea[3] > ea[0]) ? bmax * 4.f * fq * 3.1f * safe_rcp(ea[3] - ea[0]) : 0.f;
                const float qb = (eb[3] > eb[0]) ? bmax * 4.f * fq * 3.1f * safe_rcp(eb[3] - eb[0]) : 0.f;
                const float qmax = qa + qb;
                const bool fast = qmax < (float)A.fast_cap;
                if (fast) {
                    const unsigned qbnd = (unsigned)qmax + 2u;
                    for (int bk = (lo - w0) >> 6; bk <= ((hi - w0) >> 6); ++bk) atomicAdd(&blk_bound[bk], qbnd);
                    atomicAdd(&tile[(lo - w0) * TS + CNT], 1);
                    atomicAdd(&tile[(hi + 1 - w0) * TS + CNT], -1);
                }
                TetP TA, TB;
                tetp_setup(TA, ea[0], ea[1], ea[2], ea[3], fq);
                tetp_setup(TB, eb[0], eb[1], eb[2], eb[3], fq);
                // both tetrahedra's corner derivatives at E (zero outside a
                // tetrahedron's own window (E1, E4), see tetp_dw)
                auto both = [&](float E, float (&da)[4], float (&db)[4]) {
                    tetp_dw<MAXM == 1>(TA, E, da);
                    tetp_dw<MAXM == 1>(TB, E, db);
                };
                if (fast) {
                    // lane-dependent start, wrapping walk (see below)
                    const int K = hi - lo + 1;
                    int i = lo + ((lane * K) >> 5);
                    for (int j = 0; j < K; ++j) {
                        float da[4], db[4];
                        both(om[i - w0], da, db);
                        int *col = tile + (i - w0) * TS;
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            float acc = fmaf(ba[0][s], da[0], dith);
                            acc = fmaf(ba[1][s], da[1], acc);
                            acc = fmaf(ba[2][s], da[2], acc);
                            acc = fmaf(ba[3][s], da[3], acc);
                            acc = fmaf(bb[0][s], db[0], acc);
                            acc = fmaf(bb[1][s], db[1], acc);
                            acc = fmaf(bb[2][s], db[2], acc);
                            acc = fmaf(bb[3][s], db[3], acc);
                            atomicAdd(col + s, __float_as_int(acc + kMagic));
                        }
                        i = (i == hi) ? lo : i + 1;
                    }
                } else {
                    for (int i = lo; i <= hi; ++i) {
                        float da[4], db[4];
                        both(om[i - w0], da, db);
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            if (s >= A.n_orb) continue;
                            float acc = fmaf(ba[0][s], da[0], dith);
                            acc = fmaf(ba[1][s], da[1], acc);
                            acc = fmaf(ba[2][s], da[2], acc);
                            acc = fmaf(ba[3][s], da[3], acc);
                            acc = fmaf(bb[0][s], db[0], acc);
                            acc = fmaf(bb[1][s], db[1], acc);
                            acc = fmaf(bb[2][s], db[2], acc);
                            acc = fmaf(bb[3][s], db[3], acc);
                            deposit_one(acc, Gc + (long)s * A.chunk_w + (i - w0), A.status);
                        }
                    }
                }
                continue;
            }
            const int t = rest % 6, n = rest / 6;
            float e[4];
            int p[4];
            const uint32_t code = tet_code(t);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                p[q] = p0 + s_cdelta[(code >> (3 * q)) & 7];
                e[q] = Es[p[q] * A.eps_stride + n];
            }
            sort4(e, p);
            float b[4][NORB];
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4)
                load_weights<NORB, WT>(Ws + (long)p[r4] * A.w_stride + n * A.n_orb, A.n_orb, b[r4]);
            // per-item bound on every |contribution|, in fixed-point units (the
            // tetrahedron DOS is at most 3/E41 of V_T/V_G; a bin average at most
            // its weight step over the narrowest bin)
            // (integrated mode: every corner weight is at most V_T/(4 V_G))
            float qmax = (MODE == TETRA_POINT) ? bmax * 4.f * fq * 3.1f * safe_rcp(e[3] - e[0])
                         : (MODE == TETRA_BIN) ? bmax * 4.f * fq * max_iw * 1.01f
                                               : bmax * 4.f * fq * 1.01f;
            if (!(e[3] > e[0]) && MODE != TETRA_INTEGRATED) qmax = 3.0e38f;
            const bool fast = qmax < (float)A.fast_cap;
            const float dith = item_dither((gcube * 6u + (uint32_t)t) * (uint32_t)A.nb + (uint32_t)n);
            if (!valid) continue;
            // integrated mode: the first energy at or above E4, where the item's
            // saturated weights enter the step tile (none if beyond the grid)
            const int hs = hi + 1;
            const bool step = MODE == TETRA_INTEGRATED && hs < w0 + wc;
            // Bookkeeping of the tile: every entry of blocks lo/64 .. hi/64 may
            // receive at most qmax from this item, and rows lo .. hi each receive
            // one add per orbital.
            if (fast) {
                const unsigned qbnd = (unsigned)qmax + 2u;
                if (hi >= lo) {
                    for (int bk = (lo - w0) >> 6; bk <= ((hi - w0) >> 6); ++bk) atomicAdd(&blk_bound[bk], qbnd);
                    atomicAdd(&tile[(lo - w0) * TS + CNT], 1);
                    atomicAdd(&tile[(hi + 1 - w0) * TS + CNT], -1);
                }
                if (step) atomicAdd(&blk_bound[(hs - w0) >> 6], qbnd);
            }
            if constexpr (MODE == TETRA_INTEGRATED) {
                Tet T;
                tet_setup(T, e[0], e[1], e[2], e[3], fq);
                float bsum[NORB];   // saturated contribution: fq sum_l b_{l,s}
#pragma unroll
                for (int s = 0; s < NORB; ++s) bsum[s] = fq * ((b[0][s] + b[1][s]) + (b[2][s] + b[3][s]));
                if (fast) {
                    const int K = hi - lo + 1;
                    int i = lo + ((lane * max(K, 1)) >> 5);
                    for (int j = 0; j < K; ++j) {
                        float wl[4];
                        tet_weights(T, om[i - w0], wl);
                        int *col = tile + (i - w0) * TS;
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            float acc = fmaf(b[0][s], wl[0], dith);
                            acc = fmaf(b[1][s], wl[1], acc);
                            acc = fmaf(b[2][s], wl[2], acc);
                            acc = fmaf(b[3][s], wl[3], acc);
                            atomicAdd(col + s, __float_as_int(acc + kMagic));
                        }
                        i = (i == hi) ? lo : i + 1;
                    }
                    if (step) {
#pragma unroll
                        for (int s = 0; s < NORB; ++s)
                            atomicAdd(&stile[(hs - w0) * NORB + s], __float_as_int(bsum[s] + dith + kMagic) - kMagicBits);
                    }
                } else {
                    for (int i = lo; i <= hi; ++i) {
                        float wl[4];
                        tet_weights(T, om[i - w0], wl);
                        deposit_slow<NORB>(b, wl, A.n_orb, dith, Gc + (i - w0), A.chunk_w, A.status);
                    }
                    if (step) {
#pragma unroll
                        for (int s = 0; s < NORB; ++s)
                            if (s < A.n_orb) deposit_one(bsum[s] + dith, Gsc + (long)s * A.chunk_w + (hs - w0), A.status);
                    }
                }
                continue;
            }
            if constexpr (MODE == TETRA_POINT) {
                TetP TP;
                tetp_setup(TP, e[0], e[1], e[2], e[3], fq);
                if (fast) {
                    // The walk over the window starts at a lane-dependent offset
                    // and wraps: lanes whose windows coincide then add to
                    // different tile rows at each step instead of serialising on
                    // the same addresses. The sum does not depend on the order.
                    const int K = hi - lo + 1;
                    int i = lo + ((lane * K) >> 5);
                    for (int j = 0; j < K; ++j) {
                        float d[4];
                        tetp_dw<MAXM == 1>(TP, om[i - w0], d);
                        int *col = tile + (i - w0) * TS;
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            float acc = fmaf(b[0][s], d[0], dith);
                            acc = fmaf(b[1][s], d[1], acc);
                            acc = fmaf(b[2][s], d[2], acc);
                            acc = fmaf(b[3][s], d[3], acc);
                            atomicAdd(col + s, __float_as_int(acc + kMagic));
                        }
                        i = (i == hi) ? lo : i + 1;
                    }
                } else {
                    for (int i = lo; i <= hi; ++i) {
                        float d[4];
                        tetp_dw<MAXM == 1>(TP, om[i - w0], d);
                        deposit_slow<NORB>(b, d, A.n_orb, dith, Gc + (i - w0), A.chunk_w, A.status);
                    }
                }
            } else {
                Tet T;
                tet_setup(T, e[0], e[1], e[2], e[3], fq);
                float wp[4];
                tet_weights(T, om[lo - w0], wp);
                int *col = tile + (lo - w0) * TS;
                for (int i = lo; i <= hi; ++i, col += TS) {
                    float wn[4], d[4];
                    tet_weights(T, om[i + 1 - w0], wn);
                    const float sc = iw[i - w0];
#pragma unroll
                    for (int r4 = 0; r4 < 4; ++r4) { d[r4] = (wn[r4] - wp[r4]) * sc; wp[r4] = wn[r4]; }
                    if (fast) {
#pragma unroll
                        for (int s = 0; s < NORB; ++s) {
                            float acc = fmaf(b[0][s], d[0], dith);
                            acc = fmaf(b[1][s], d[1], acc);
                            acc = fmaf(b[2][s], d[2], acc);
                            acc = fmaf(b[3][s], d[3], acc);
                            atomicAdd(col + s, __float_as_int(acc + kMagic));
                        }
                    } else {
                        deposit_slow<NORB>(b, d, A.n_orb, dith, Gc + (i - w0), A.chunk_w, A.status);
                    }
                }
            }
        }
        __syncthreads();   // every thread is done reading both slots and adding to the tile
        // refill: energies of work item k+2 into this energy stage, weights of k+1
        if (tid == 0) {
            fence_proxy_async_smem();
            if (MAXM > 1) store_claim(k + 2, g_next);
            issue_e(k + 2, st);
            issue_w(k + 1);
        }
        // A block whose bound reached flush_at is moved into the CTA's int64
        // partial before the next box: one box adds less than 2^30 - 2^20 to any
        // entry (per-unit cap x units per box), so entries stay below 2^31.
        // A flushed entry is reset to count * M, the raw value of zero.
        if constexpr (MAXM > 1) {
            // (the batched kernel: one tile copy; this form measured faster there)
            const bool mine = tid < n_blk && blk_bound[tid] >= A.flush_at;
            if (__syncthreads_or(mine)) {
                counts_from_diffs(tile);
                for (int bk = 0; bk < n_blk; ++bk) {
                    if (blk_bound[bk] < A.flush_at) continue;   // uniform: every thread reads the same value
                    const int j0 = bk << 6, jn = min(64, wc - j0);
                    for (int i = tid; i < A.n_orb * 64; i += blockDim.x) {
                        const int s = i >> 6, j = i & 63;
                        if (j >= jn) continue;
                        const int v = entry_value(tile, j0 + j, s);
                        if (v) {
                            atomicAdd(reinterpret_cast<unsigned long long *>(Gc + (long)s * A.chunk_w + j0 + j),
                                      static_cast<unsigned long long>(static_cast<long long>(v)));
                            tile[(j0 + j) * TS + s] = (int)((unsigned)tile[(j0 + j) * TS + CNT] * (unsigned)kMagicBits);
                        }
                    }
                }
                __syncthreads();
                diffs_from_counts(tile);
                if (tid < n_blk && blk_bound[tid] >= A.flush_at) blk_bound[tid] = 0;
                __syncthreads();
            }
            continue;
        }
        bool mine = false;
        for (int i = tid; i < n_blk * n_copies; i += blockDim.x) mine = mine || blk_bound[i] >= A.flush_at;
        if (__syncthreads_or(mine)) {
            for (int c = 0; c < n_copies; ++c) {
                const unsigned *bc = blk_bound + c * n_blk;
                bool any = false;   // uniform: every thread reads the same values
                for (int bk = 0; bk < n_blk; ++bk) any = any || bc[bk] >= A.flush_at;
                if (!any) continue;
                int *tc = tile + c * copy_ints;
                counts_from_diffs(tc);
                for (int bk = 0; bk < n_blk; ++bk) {
                    if (bc[bk] < A.flush_at) continue;   // uniform
                    const int j0 = bk << 6, jn = min(64, wc - j0);
                    for (int i = tid; i < A.n_orb * 64; i += blockDim.x) {
                        const int s = i >> 6, j = i & 63;
                        if (j >= jn) continue;
                        const int v = entry_value(tc, j0 + j, s);
                        if (v) {
                            atomicAdd(reinterpret_cast<unsigned long long *>(Gc + (long)s * A.chunk_w + j0 + j),
                                      static_cast<unsigned long long>(static_cast<long long>(v)));
                            tc[(j0 + j) * TS + s] = (int)((unsigned)tc[(j0 + j) * TS + CNT] * (unsigned)kMagicBits);
                        }
                        if (MODE == TETRA_INTEGRATED) {
                            int *se = &stile[(j0 + j) * NORB + s];
                            if (*se) {
                                atomicAdd(reinterpret_cast<unsigned long long *>(Gsc + (long)s * A.chunk_w + j0 + j),
                                          static_cast<unsigned long long>(static_cast<long long>(*se)));
                                *se = 0;
                            }
                        }
                    }
                }
                __syncthreads();
                diffs_from_counts(tc);
            }
            for (int i = tid; i < n_blk * n_copies; i += blockDim.x)
                if (blk_bound[i] >= A.flush_at) blk_bound[i] = 0;
            __syncthreads();
        }
    }
    __syncthreads();
    if (s_abort) {
        // a TMA wait timed out: wait (bounded) for copies still in flight, then leave
        if (tid == 0) {
            for (int b = 0; b < 3; ++b)
                if (n_issued[b] > 0)
                    mbar_wait_bounded(&mbar[b], (uint32_t)(n_issued[b] - 1) & 1u, nullptr, 100000000ull);
        }
        return;
    }
    if (cur >= 0) flush_tile();
}

// Single model: dos[s][w0+j] = u * sum over CTAs of the int64 partials (exact).
__global__ void tetra_dos_reduce_kernel(const long long *G, int grid_x, int n_orb, int n_omega,
                                        int chunk_w, int mode, const float *omega, double vtvg,
                                        int bits, float *dos) {
    const double u = fixed_unit(omega, n_omega, mode, vtvg, bits);
    const long total = (long)n_orb * n_omega;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / n_omega), i = (int)(idx - (long)s * n_omega);
        const int chunk = i / chunk_w, j = i - chunk * chunk_w;
        const long long *g = G + ((long)chunk * grid_x * n_orb + s) * chunk_w + j;
        long long acc = 0;
        for (int c = 0; c < grid_x; ++c) acc += g[(long)c * n_orb * chunk_w];
        dos[idx] = (float)((double)acc * u);
    }
}

// Integrated mode: block (s, c) = orbital s, energy chunk c. A chunk's CTAs
// put the steps of every tetrahedron below the chunk on its first energy, so
// the running sum of the step partials starts afresh in each chunk:
// dos[s][w0 + j] = u * (sum over CTAs of the window partials at j + the
// running sum over j' <= j of the chunk's step partials), exact int64
// arithmetic up to the scaling.
__global__ void tetra_dos_reduce_integrated(const long long *G, const long long *Gs, int grid_x, int n_orb,
                                            int n_omega, int chunk_w, const float *omega, double vtvg,
                                            int bits, float *dos) {
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    const int s = blockIdx.x, chunk = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (int)(blockDim.x >> 5);
    const int w0 = chunk * chunk_w, wc = min(chunk_w, n_omega - w0);
    const long cta_stride = (long)n_orb * chunk_w;
    const long first = ((long)chunk * grid_x * n_orb + s) * chunk_w;
    const double u = fixed_unit(omega, n_omega, TETRA_INTEGRATED, vtvg, bits);
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < wc; base += blockDim.x) {
        const int j = base + tid;
        long long wsum = 0, ssum = 0;
        if (j < wc) {
            for (int c = 0; c < grid_x; ++c) {
                const long off = first + c * cta_stride + j;
                wsum += G[off];
                ssum += Gs[off];
            }
        }
        long long x = ssum;   // inclusive scan over the block
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        long long off = s_carry;
        for (int w2 = 0; w2 < warp; ++w2) off += s_warp[w2];
        x += off;
        if (j < wc) dos[(long)s * n_omega + w0 + j] = (float)((double)(wsum + x) * u);
        __syncthreads();
        if (tid == 0) {
            long long tot = 0;
            for (int w2 = 0; w2 < nw; ++w2) tot += s_warp[w2];
            s_carry += tot;
        }
        __syncthreads();
    }
}

// Batched: model blockIdx.y scales its int64 accumulator (slot = model).
struct BatchOut {
    float *dos[kMaxBatch];
};
__global__ void tetra_dos_reduce_batched(const __grid_constant__ Batch<kMaxBatch> B, const BatchOut O,
                                         const long long *G, int n_orb, int chunk_w, int mode) {
    const ModelP &M = B.m[blockIdx.y];
    const double u = fixed_unit(M.omega, M.n_omega, mode, M.vtvg, M.fixed_bits);
    const long total = (long)n_orb * M.n_omega;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / M.n_omega), i = (int)(idx - (long)s * M.n_omega);
        const long long g = G[((long)blockIdx.y * n_orb + s) * chunk_w + i];
        O.dos[blockIdx.y][idx] = (float)((double)g * u);
    }
}

template <int NORB, typename WT, int MODE, int MAXM>
cudaError_t launch_t(size_t smem, dim3 grid, const Batch<MAXM> &Bt, const FwdArgs &A,
                     cudaStream_t stream) {
    auto k = tetra_dos_fwd_kernel<NORB, WT, MODE, MAXM>;
    // The shared-memory opt-in is set once per device and size, so that a
    // launch inside a CUDA-graph capture makes no attribute call.
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
    k<<<grid, Cfg<MODE, NORB>::threads, smem, stream>>>(Bt, A);
    return cudaGetLastError();
}

template <int NORB, int MODE, int MAXM>
cudaError_t launch_wt(int wdtype, size_t smem, dim3 grid, const Batch<MAXM> &Bt, const FwdArgs &A,
                      cudaStream_t stream) {
    switch (wdtype) {
        case TETRA_F16: return launch_t<NORB, __half, MODE, MAXM>(smem, grid, Bt, A, stream);
        case TETRA_BF16: return launch_t<NORB, __nv_bfloat16, MODE, MAXM>(smem, grid, Bt, A, stream);
        default: return launch_t<NORB, float, MODE, MAXM>(smem, grid, Bt, A, stream);
    }
}

template <int MODE, int MAXM>
cudaError_t launch_norb(int n_orb, int wdtype, size_t smem, dim3 grid, const Batch<MAXM> &Bt,
                        const FwdArgs &A, cudaStream_t stream) {
    if (n_orb <= 1) return launch_wt<1, MODE, MAXM>(wdtype, smem, grid, Bt, A, stream);
    if (n_orb <= 2) return launch_wt<2, MODE, MAXM>(wdtype, smem, grid, Bt, A, stream);
    if (n_orb <= 4) return launch_wt<4, MODE, MAXM>(wdtype, smem, grid, Bt, A, stream);
    if (n_orb <= 8) return launch_wt<8, MODE, MAXM>(wdtype, smem, grid, Bt, A, stream);
    return launch_wt<16, MODE, MAXM>(wdtype, smem, grid, Bt, A, stream);
}

// Launch constants shared by all models of a plan (box geometry, strides).
void fill_common(const Plan &P, FwdArgs &A) {
    A.nb = P.d.n_bands; A.n_orb = P.d.n_orb;
    A.BX = P.BX; A.BY = P.BY; A.BZ = P.BZ;
    A.lbx = __builtin_ctz(P.BX); A.lby = __builtin_ctz(P.BY); A.lbz = __builtin_ctz(P.BZ);
    A.eps_stride = P.eps_stride; A.w_stride = P.w_stride;
    const uint32_t npts = (uint32_t)(P.BX + 1) * (P.BY + 1) * (P.BZ + 1);
    A.e_box_bytes = npts * P.eps_stride * 4u;
    A.w_box_bytes = npts * P.w_stride * (uint32_t)P.wbytes;
    // every TMA destination starts on a 128-byte boundary
    A.e_stage = (A.e_box_bytes + 127u) & ~127u;
    A.w_stage = (A.w_box_bytes + 127u) & ~127u;
    A.chunk_w = P.chunk_w;
    A.tile_copies = P.tile_copies;
    A.items_per_box = P.items_per_box;
    A.flush_at = 1u << P.flush_bits;
    long cap = ((1L << 30) - (1L << 20)) / A.items_per_box;
    if (cap > (1L << 21)) cap = 1L << 21;
    A.fast_cap = (int)cap;
}

ModelP model_of(const Plan &P, const float *omega) {
    ModelP m;
    m.n1 = P.d.n1; m.n2 = P.d.n2; m.n3 = P.d.n3; m.z0 = P.z0; m.z1 = P.z1;
    m.nbx = P.nbx; m.nby = P.nby; m.n_boxes = P.n_boxes; m.n_omega = P.d.n_omega;
    m.fixed_bits = P.fixed_bits;
    m.box_base = 0;
    m.vtvg = 1.0 / (6.0 * (double)P.d.n1 * (double)P.d.n2 * (double)P.d.n3);
    m.omega = omega;
    return m;
}

tetra_status_t encode_maps(const Plan &P, const float *eps, const void *w, MapPair &mp) {
    const CUtensorMapDataType wdt = P.d.weight_dtype == TETRA_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                    : P.d.weight_dtype == TETRA_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    tetra_status_t st = encode_point_map(&mp.e, eps, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P.eps_stride,
                                         P.nx, P.ny, P.nz, P.BX + 1, P.BY + 1, P.BZ + 1);
    if (st != TETRA_OK) return st;
    return encode_point_map(&mp.w, w, wdt, P.wbytes, P.w_stride, P.nx, P.ny, P.nz, P.BX + 1,
                            P.BY + 1, P.BZ + 1);
}

}  // namespace

int norb_template(int n_orb) {
    return n_orb <= 1 ? 1 : n_orb <= 2 ? 2 : n_orb <= 4 ? 4 : n_orb <= 8 ? 8 : 16;
}

size_t dos_forward_workspace(const Plan &P) {
    // integrated mode: a second array of the same size for the step sums
    const size_t parts = sizeof(long long) * (size_t)P.n_chunks * P.grid_x * P.d.n_orb * (size_t)P.chunk_w;
    return kStatusBytes + (P.d.mode == TETRA_INTEGRATED ? 2 : 1) * parts;
}

tetra_status_t launch_dos_forward(const Plan &P, const float *eps, const void *w,
                                  const float *omega, float *dos, void *ws, size_t ws_bytes,
                                  cudaStream_t stream) {
    const size_t need = dos_forward_workspace(P);
    if (ws_bytes < need) return TETRA_ENOMEM;
    static thread_local Batch<1> Bt;   // 0.3 KB of tensor maps + model constants
    Bt.n_models = 1;
    Bt.total_work = P.n_boxes;
    tetra_status_t st = encode_maps(P, eps, w, Bt.maps[0]);
    if (st != TETRA_OK) return st;
    Bt.m[0] = model_of(P, omega);
    FwdArgs A;
    fill_common(P, A);
    A.status = reinterpret_cast<int *>(ws);
    A.queue = nullptr;
    A.G = reinterpret_cast<long long *>(static_cast<unsigned char *>(ws) + kStatusBytes);
    A.Gs = A.G + (size_t)P.n_chunks * P.grid_x * P.d.n_orb * (size_t)P.chunk_w;
    cudaError_t e = cudaMemsetAsync(ws, 0, need, stream);
    if (e != cudaSuccess) return TETRA_ECUDA;
    const dim3 grid(P.grid_x, P.n_chunks);
    const int mode = P.d.mode;
    e = mode == TETRA_POINT ? launch_norb<TETRA_POINT, 1>(P.d.n_orb, P.d.weight_dtype, P.smem_bytes, grid, Bt, A, stream)
        : mode == TETRA_BIN ? launch_norb<TETRA_BIN, 1>(P.d.n_orb, P.d.weight_dtype, P.smem_bytes, grid, Bt, A, stream)
                            : launch_norb<TETRA_INTEGRATED, 1>(P.d.n_orb, P.d.weight_dtype, P.smem_bytes, grid, Bt,
                                                               A, stream);
    if (e != cudaSuccess) return TETRA_ECUDA;
    if (mode == TETRA_INTEGRATED) {
        const dim3 rgrid(P.d.n_orb, P.n_chunks);
        tetra_dos_reduce_integrated<<<rgrid, 256, 0, stream>>>(A.G, A.Gs, P.grid_x, P.d.n_orb, P.d.n_omega,
                                                               P.chunk_w, omega, Bt.m[0].vtvg, P.fixed_bits,
                                                               dos);
        if (cudaGetLastError() != cudaSuccess) return TETRA_ECUDA;
        return TETRA_OK;
    }
    const long total = (long)P.d.n_orb * P.d.n_omega;
    const int rb = 256;
    const int rg = (int)std::min<long>((total + rb - 1) / rb, 4L * P.sm_count);
    tetra_dos_reduce_kernel<<<rg, rb, 0, stream>>>(A.G, P.grid_x, P.d.n_orb, P.d.n_omega,
                                                   P.chunk_w, P.d.mode, omega, Bt.m[0].vtvg,
                                                   P.fixed_bits, dos);
    if (cudaGetLastError() != cudaSuccess) return TETRA_ECUDA;
    return TETRA_OK;
}

size_t dos_batched_workspace(const BatchPlan &B) {
    return kStatusBytes + sizeof(long long) * (size_t)B.n_models * B.models[0].d.n_orb * (size_t)B.chunk_w;
}

tetra_status_t launch_dos_batched(const BatchPlan &BP, const float *const *eps, const void *const *w,
                                  const float *const *omega, float *const *dos, void *ws,
                                  size_t ws_bytes, cudaStream_t stream) {
    const size_t need = dos_batched_workspace(BP);
    if (ws_bytes < need) return TETRA_ENOMEM;
    std::unique_ptr<Batch<kMaxBatch>> Bt(new (std::nothrow) Batch<kMaxBatch>());
    std::unique_ptr<BatchOut> O(new (std::nothrow) BatchOut());
    if (!Bt || !O) return TETRA_ENOMEM;
    Bt->n_models = BP.n_models;
    Bt->total_work = BP.total_boxes;
    for (int m = 0; m < BP.n_models; ++m) {
        const Plan &P = BP.models[m];
        tetra_status_t st = encode_maps(P, eps[m], w[m], Bt->maps[m]);
        if (st != TETRA_OK) return st;
        ModelP mp = model_of(P, omega[m]);
        mp.box_base = BP.box_base[m];
        Bt->m[m] = mp;
        O->dos[m] = dos[m];
    }
    const Plan &P0 = BP.models[BP.big];
    FwdArgs A;
    fill_common(P0, A);
    A.chunk_w = BP.chunk_w;
    A.status = reinterpret_cast<int *>(ws);
    A.queue = reinterpret_cast<int *>(static_cast<unsigned char *>(ws) + kQueueOffset);
    A.G = reinterpret_cast<long long *>(static_cast<unsigned char *>(ws) + kStatusBytes);
    A.Gs = nullptr;
    cudaError_t e = cudaMemsetAsync(ws, 0, need, stream);   // status, counter, accumulators
    if (e != cudaSuccess) return TETRA_ECUDA;
    const dim3 grid(BP.grid_x, 1);
    const int n_orb = P0.d.n_orb, wdt = P0.d.weight_dtype;
    e = (P0.d.mode == TETRA_POINT)
            ? launch_norb<TETRA_POINT, kMaxBatch>(n_orb, wdt, BP.smem_bytes, grid, *Bt, A, stream)
            : launch_norb<TETRA_BIN, kMaxBatch>(n_orb, wdt, BP.smem_bytes, grid, *Bt, A, stream);
    if (e != cudaSuccess) return TETRA_ECUDA;
    const long total = (long)n_orb * BP.chunk_w;
    const int rb = 256;
    const int rg = (int)std::max<long>(1, std::min<long>((total + rb - 1) / rb, 64));
    tetra_dos_reduce_batched<<<dim3(rg, BP.n_models), rb, 0, stream>>>(*Bt, *O, A.G, n_orb,
                                                                        BP.chunk_w, P0.d.mode);
    if (cudaGetLastError() != cudaSuccess) return TETRA_ECUDA;
    return TETRA_OK;
}

}  // namespace tetra
