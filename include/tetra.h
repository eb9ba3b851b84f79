/*
 * tetra.h - C ABI of libtetra, a GB300 (sm_103a) implementation of the linear
 * tetrahedron method for the orbital-resolved density of states
 * (D. Guterding, H. O. Jeschke, "An efficient GPU algorithm for
 * tetrahedron-based Brillouin-zone integration", arXiv:1710.10789).
 *
 * General conventions
 *  - Every entry point returns a tetra_status_t; nothing is thrown across the
 *    ABI. Argument errors are reported synchronously, before any work is
 *    enqueued. Work is enqueued on the given CUDA stream and runs
 *    asynchronously; errors raised on the device (a wait that timed out, a
 *    value outside the representable range) are recorded in the workspace and
 *    returned by tetra_workspace_status().
 *  - All array arguments are DEVICE pointers owned by the caller, except where
 *    a parameter says "host". The library never frees caller memory. Outputs
 *    are overwritten, never accumulated into.
 *  - Results are deterministic: the same plan, inputs and workspace size give
 *    bit-identical outputs. The DOS is accumulated in exact 64-bit fixed point,
 *    so it is also independent of the launch shape.
 *
 * k-grid and the padded point-major layout ("tetra layout")
 *  - The k-grid is periodic and Gamma-centred with n1 x n2 x n3 points,
 *    k = 2 pi (x/n1, y/n2, z/n3) in reciprocal-lattice units (Sec. IV.A uses
 *    N x N x 10 grids). Every point is the origin of one elemental cube, which
 *    is split into the six tetrahedra of Table I around its 3-6 diagonal; cube
 *    corner label c = 1 + dx + 2 dy + 4 dz for the offset (dx, dy, dz).
 *  - Band energies and orbital weights are stored per grid point, with one
 *    periodic halo plane in each direction: P = (n1+1)(n2+1)(n3+1) points,
 *    point index p = x + (n1+1) (y + (n2+1) z) for x <= n1, y <= n2, z <= n3,
 *    holding the data of k-point (x mod n1, y mod n2, z mod n3).
 *      eps: float, eps[p * eps_stride + n]                  (band n)
 *      w  : F32/F16/BF16, w[p * w_stride + n * n_orb + s]  (band n, orbital s)
 *    with the strides reported by tetra_layout(). Both arrays must be 16-byte
 *    aligned. Bands are sorted ascending at each point (Sec. II.A diagonalises
 *    H(k) point by point), and w = |a^s_n(k)|^2 of Eq. (3).
 */
#ifndef TETRA_H
#define TETRA_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TETRA_OK = 0,
    TETRA_EINVAL = 1,        /* bad argument (null pointer, size, alignment)      */
    TETRA_EUNSUPPORTED = 2,  /* valid request this build does not support         */
    TETRA_ECUDA = 3,         /* a CUDA runtime call failed                        */
    TETRA_ENOMEM = 4,        /* workspace too small / allocation failed           */
    TETRA_ETIMEOUT = 5,      /* a device-side wait hit its iteration limit        */
    TETRA_ERANGE = 6         /* a contribution exceeded the fixed-point range     */
} tetra_status_t;

enum { TETRA_POINT = 0, TETRA_BIN = 1, TETRA_INTEGRATED = 2 };
enum { TETRA_F32 = 0, TETRA_F16 = 1, TETRA_BF16 = 2 };

/* Problem description of one DOS evaluation. */
typedef struct {
    int n1, n2, n3;     /* k-grid size, each >= 1                                   */
    int n_bands;        /* bands per k-point, 1..64                                 */
    int n_orb;          /* orbitals, 1..16 (Sec. III.B: up to 16 orbitals)          */
    int n_omega;        /* energies (TETRA_POINT, TETRA_INTEGRATED) or bins (TETRA_BIN), >= 1 */
    int mode;           /* TETRA_POINT: rho_s(E) at energies, Eq. (9);
                           TETRA_BIN: bin averages of rho_s over consecutive edges;
                           TETRA_INTEGRATED: occupation n_s(E) up to each energy */
    int weight_dtype;   /* storage type of w: TETRA_F32, TETRA_F16, TETRA_BF16      */
    int z_begin, z_end; /* cube planes [z_begin, z_end) to integrate (a k-slab, for
                           splitting one grid over several calls or devices);
                           0, 0 means the whole grid                                */
} tetra_desc_t;

/* Element strides of the tetra layout for a plan. */
typedef struct {
    int nx, ny, nz;       /* padded extents n1+1, n2+1, n3+1                        */
    int eps_stride;       /* floats per point in eps                                */
    int w_stride;         /* elements per point in w                                */
    size_t eps_elems;     /* total floats of eps  = nx*ny*nz*eps_stride             */
    size_t w_elems;       /* total elements of w  = nx*ny*nz*w_stride               */
} tetra_layout_t;

typedef struct tetra_plan_s *tetra_plan_t;

/* Creates a plan for desc on CUDA device `device` (host call; reads device
 * properties, picks the box shape and grid of the kernels). The plan owns only
 * host memory. Returns TETRA_EINVAL for an invalid desc. */
tetra_status_t tetra_plan(tetra_plan_t *plan, const tetra_desc_t *desc, int device);

/* Destroys a plan (host memory only). Safe on NULL. */
tetra_status_t tetra_plan_destroy(tetra_plan_t plan);

/* Layout strides the plan expects (host call). */
tetra_status_t tetra_layout(tetra_plan_t plan, tetra_layout_t *layout);

/* Bytes of device workspace tetra_dos / tetra_dos_backward need (host call). */
size_t tetra_workspace_bytes(tetra_plan_t plan);

/* Orbital-resolved DOS by the linear tetrahedron method (Sec. II.C, Eqs. (8)-(9)).
 *   eps, w : band energies and orbital weights in the tetra layout.
 *   omega  : TETRA_POINT, TETRA_INTEGRATED: n_omega ascending energies E_i.
 *            TETRA_BIN:   n_omega + 1 ascending bin edges.
 *            Any ascending grid is correct; equidistant grids (Sec. IV.A) are
 *            fastest.
 *   dos    : [n_orb][n_omega] float, overwritten.
 *            TETRA_POINT: dos[s][i] = sum_{T,n} sum_l b_{n,l,s} dw_l/dE (E_i).
 *            TETRA_BIN:   dos[s][i] = sum_{T,n} sum_l b_{n,l,s}
 *                           [w_l(e_{i+1}) - w_l(e_i)] / (e_{i+1} - e_i).
 *            TETRA_INTEGRATED: dos[s][i] = sum_{T,n} sum_l b_{n,l,s} w_l(E_i),
 *                           the occupation of orbital s per spin up to E_i
 *                           (Eq. (2) with the step function as occupation;
 *                           not in the paper, which integrates the DOS only).
 *                           Grids longer than one shared-memory tile (about
 *                           2400 energies for 8 orbitals) run as several
 *                           energy chunks; every value is the same integer sum
 *                           as in a plan over that energy alone.
 *            Normalised per spin and orbital: with unitary weights the bin
 *            DOS of each orbital integrates to 1, and n_s(E) rises from 0 to 1.
 *   ws     : device workspace of at least tetra_workspace_bytes(plan) bytes,
 *            16-byte aligned; contents on entry are ignored.
 * Returns TETRA_EINVAL for null/misaligned pointers or ws_bytes too small. */
tetra_status_t tetra_dos(tetra_plan_t plan, const float *eps, const void *w,
                         const float *omega, float *dos, void *ws, size_t ws_bytes,
                         cudaStream_t stream);

/* tetra_dos without a workspace argument, for callers that cannot allocate
 * device memory where they need a DOS: code under a host framework that owns
 * all device allocations through its own pool, code whose device-memory budget
 * is fixed before it starts, or a latency-sensitive loop that must not call
 * cudaMalloc / cudaFree. The paper has no counterpart; it is a library
 * convenience.
 *   Scratch: a static device array of 32 MiB inside libtetra (held on every
 *   GPU that loads the library until the process exits). The call allocates
 *   nothing. If the plan's per-CTA partial sums do not fit, fewer persistent
 *   CTAs are used (same result, bit for bit); if they do not fit even with one
 *   CTA, returns TETRA_ENOMEM. With one CTA the scratch holds
 *     256 + m * 8 * n_orb * n_chunks * ceil(n_omega / n_chunks)  bytes,
 *   m = 2 in TETRA_INTEGRATED mode and 1 otherwise, where n_chunks is the
 *   number of shared-memory energy tiles of the plan (1 up to about 4300
 *   energies for 8 orbitals and 8 bands in F32).
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture. The address is kept with the device's context;
 *   after a device reset the next call looks it up again.
 *   Sharing: every call on a device uses the same array, and the call clears
 *   what it needs before use. Calls whose kernels overlap on the GPU (different
 *   streams, or host threads) race on the array and give wrong results;
 *   serialise them. The array keeps the last call's contents, including its
 *   device-side status words: read them with tetra_noalloc_status().
 * Arguments and results are those of tetra_dos. */
tetra_status_t tetra_dos_noalloc(tetra_plan_t plan, const float *eps, const void *w,
                                 const float *omega, float *dos, cudaStream_t stream);

/* Device-side status of the last tetra_dos_noalloc call on `device`, read
 * from the front of its static scratch array (synchronises `stream`, which
 * must be a stream of `device` or 0). TETRA_OK, TETRA_ETIMEOUT or
 * TETRA_ERANGE, as tetra_workspace_status() gives for tetra_dos; TETRA_OK if
 * no tetra_dos_noalloc call has run on the device yet. Not in the paper. */
tetra_status_t tetra_noalloc_status(int device, cudaStream_t stream);

/* Adjoint of tetra_dos in TETRA_BIN mode (not in the paper; the derivative of
 * its bin-averaged DOS). Given grad_dos = dL/d dos [n_orb][n_omega], writes
 *   grad_eps = dL/d eps (float, tetra layout, eps_stride)
 *   grad_w   = dL/d w   (float, tetra layout with w_stride; F32 even when w
 *                        is stored in F16/BF16)
 * Interior points receive the full derivative with respect to the value of
 * that k-point; halo points (x == n1 or y == n2 or z == n3) and the layout's
 * padding entries are set to 0 (both arrays are overwritten completely).
 * Returns TETRA_EUNSUPPORTED for a TETRA_POINT plan. */
tetra_status_t tetra_dos_backward(tetra_plan_t plan, const float *eps, const void *w,
                                  const float *omega, const float *grad_dos,
                                  float *grad_eps, float *grad_w, void *ws,
                                  size_t ws_bytes, cudaStream_t stream);

/* Tight-binding model in device memory, the hopping form of Eq. (1):
 *   H(k) = diag(onsite) + sum_r [ t_r e^{i k.R_r} + t_r^dagger e^{-i k.R_r} ].
 * params: onsite[n_orb] followed by Re t[n_R][n_orb][n_orb] and then
 *         Im t[n_R][n_orb][n_orb] (float; row index = first orbital index).
 * R: int[n_R][3] lattice vectors. */
typedef struct {
    int n_orb;            /* 1..8 for tetra_eig                                     */
    int n_R;              /* number of independent lattice vectors, 0..32           */
    const float *params;  /* device, n_orb + 2 n_R n_orb^2 floats                   */
    const int *R;         /* device, 3 n_R ints                                     */
} tetra_model_t;

/* Band energies and orbital weights of a tight-binding model on the plan's
 * grid (Sec. II.A: diagonalisation of H(k) point by point), written directly
 * in the tetra layout. A batched Hermitian eigensolver on the GPU (Householder
 * reduction to real tridiagonal form, implicit-shift QR), one k-point per
 * thread; bands ascending, w[n][s] = |V_{s n}|^2 stored in the plan's weight_dtype.
 * Requires plan n_bands == model n_orb <= 8 and plan n_orb <= model n_orb: a
 * plan with fewer orbitals than the model gets the weights of the model's
 * first n_orb orbitals (a projection on an orbital subset, as the paper's
 * five Fe-d orbitals of its eight-orbital model). Halo points are written too. For
 * a slab plan (z_begin, z_end) only the point planes z_begin .. z_end (the
 * corners of its cubes) are written; the rest of eps and w is left as is. */
tetra_status_t tetra_eig(tetra_plan_t plan, const tetra_model_t *model, float *eps, void *w,
                         cudaStream_t stream);

/* Derivative of a loss through tetra_eig to the model parameters (not in the
 * paper): given dL/d eps and dL/d w in the tetra layout (float; halo entries
 * ignored), writes grad_params (same packing as model->params, float).
 * Eigenvector derivatives use F_nm = d/(d^2 + eta^2), d = e_n - e_m,
 * eta = 1e-8 eV, in FP64 for near-degenerate pairs (|d| < 1e-4 eV) and in
 * FP32 for the rest. Deterministic: fixed
 * summation order over k-points and blocks. Needs
 * tetra_eig_workspace_bytes(plan) bytes of workspace. */
tetra_status_t tetra_eig_backward(tetra_plan_t plan, const tetra_model_t *model,
                                  const float *grad_eps, const float *grad_w,
                                  float *grad_params, void *ws, size_t ws_bytes,
                                  cudaStream_t stream);
size_t tetra_eig_workspace_bytes(tetra_plan_t plan, int n_R);

/* ---------------------------------------------------------------- batches
 * Many independent DOS problems in ONE launch of the forward kernel (not in
 * the paper, which evaluates one model at a time; Secs. III-IV). Each model has
 * its own k-grid, energy grid and data; all share n_bands, n_orb, mode and
 * weight_dtype. The persistent CTAs claim (model, box) work items from a
 * global counter, so uneven models keep every SM busy; each model's result is
 * summed in exact integers, so it equals what tetra_dos gives for it bit for
 * bit (same fixed-point bits), whatever the schedule.
 * Every argument of tetra_dos_batched travels in kernel parameters, so the
 * call can be captured in a CUDA graph and replayed with the same pointers. */
#define TETRA_MAX_BATCH 64

typedef struct tetra_batch_plan_s *tetra_batch_plan_t;

/* Launch-shape choices (e.g. from an autotuner); zero fields take the default. */
typedef struct {
    int box_x, box_y, box_z; /* cubes per box side (rounded down to powers of two
                                and clipped to the smallest grid); default 4,4,4
                                for 8 bands and up to 8 orbitals, 4,4,2 for 8
                                bands and 9 to 16 orbitals                         */
    int ctas_per_sm;         /* persistent CTAs per SM, default 1                  */
} tetra_tune_t;

/* Plans a batch of n_models (1..TETRA_MAX_BATCH) descriptions (host array).
 * tune may be NULL. Returns TETRA_EINVAL if the descriptions differ in n_bands,
 * n_orb, mode or weight_dtype or one is invalid, TETRA_EUNSUPPORTED if the
 * largest n_omega does not fit one shared-memory tile (about 4300 energies, or
 * 3900 bins, for 8 orbitals and 8 bands in F32 with the default box). The plan
 * owns only host memory. */
tetra_status_t tetra_plan_batched(tetra_batch_plan_t *plan, const tetra_desc_t *descs, int n_models,
                                  const tetra_tune_t *tune, int device);
tetra_status_t tetra_batch_plan_destroy(tetra_batch_plan_t plan);

/* Layout strides of model `model` (host call). */
tetra_status_t tetra_batch_layout(tetra_batch_plan_t plan, int model, tetra_layout_t *layout);

/* Bytes of device workspace tetra_dos_batched needs (host call). */
size_t tetra_batch_workspace_bytes(tetra_batch_plan_t plan);

/* Chosen launch shape (host call): box[3] cubes per box side, grid = persistent
 * CTAs, n_slots = int64 accumulators (one per model). Any output may be NULL. */
tetra_status_t tetra_batch_info(tetra_batch_plan_t plan, int *box, int *grid, int *n_slots);

/* DOS of every model of the batch (Sec. II.C, Eqs. (8)-(9), as tetra_dos).
 *   eps, w, omega, dos: HOST arrays of n_models DEVICE pointers; model m uses
 *   eps[m], w[m] in its tetra layout, omega[m] (n_omega or n_omega + 1 values)
 *   and writes dos[m] ([n_orb][n_omega] of its description).
 *   ws: at least tetra_batch_workspace_bytes(plan) bytes, 16-byte aligned.
 * The host arrays are read during the call only. */
tetra_status_t tetra_dos_batched(tetra_batch_plan_t plan, const float *const *eps, const void *const *w,
                                 const float *const *omega, float *const *dos, void *ws,
                                 size_t ws_bytes, cudaStream_t stream);

/* Fermi level of the plan's bands: the energy E_F at which the occupation
 * summed over the plan's orbitals, N(E) = sum_s n_s(E) (TETRA_INTEGRATED mode
 * of tetra_dos: Eq. (2) with the step function as occupation, Sec. II.C
 * corner weights), equals n_electrons per spin. With unitary weights of all
 * orbitals (tetra_eig with plan n_orb = n_bands) N counts the states below E,
 * from 0 to n_bands. Not in the paper (which evaluates the DOS only).
 *   eps, w : as for tetra_dos, for any plan mode (the plan's grid, bands,
 *            orbitals and weight dtype are used).
 *   n_electrons : target count per spin, in [0, N(max eps)].
 *   ef     : host float, the result.
 *   ws     : device workspace of at least tetra_fermi_workspace_bytes(plan)
 *            bytes, 16-byte aligned.
 * Method: the band minimum and maximum bracket E_F; each round evaluates N at
 * 64 equidistant energies of the bracket in one TETRA_INTEGRATED launch and
 * keeps the sub-interval where N crosses n_electrons, until the bracket is at
 * the FP32 resolution of the energies (about six rounds). Synchronises
 * `stream` once per round. Returns TETRA_EINVAL for null/misaligned pointers
 * or n_electrons outside [0, N(max eps)], TETRA_ENOMEM if ws_bytes is too
 * small, TETRA_EUNSUPPORTED for a slab plan (the count needs the whole grid). */
size_t tetra_fermi_workspace_bytes(tetra_plan_t plan);
tetra_status_t tetra_fermi_level(tetra_plan_t plan, const float *eps, const void *w, double n_electrons,
                                 float *ef, void *ws, size_t ws_bytes, cudaStream_t stream);

/* Transition bands of the bare susceptibility at momentum q (the extension
 * to susceptibilities the paper names as future work; not in the paper).
 * For every point k of the plan's grid and band pair (n, m), stored as band
 * j = n * n_bands + m of pair_plan:
 *   eps_pairs : eps_m(k + q) - eps_n(k),
 *   w_pairs   : f(eps_n(k)) - f(eps_m(k + q)),  f(e) = 1 / (1 + e^{(e - mu)/kT}).
 * tetra_dos on pair_plan (point mode, energies w) then gives the spectral
 * function S(q, w) = sum_{n,m} int [f_n(k) - f_m(k+q)] delta(w - eps_m(k+q)
 * + eps_n(k)) dk / V_G of the bare Lindhard function, Im chi0(q, w + i0) =
 * -pi S(q, w): both differences are linear inside a tetrahedron by the
 * method's own interpolation. Only the spectral (imaginary) part is provided.
 *   plan      : the bands (n_bands <= 8), eps in its tetra layout.
 *   q         : integer grid vector (q_i in units of 2 pi / n_i), any sign.
 *   kT, mu    : temperature (> 0) and chemical potential, in energy units.
 *   pair_plan : same grid, n_bands = plan n_bands^2, n_orb = 1, TETRA_F32;
 *               eps_pairs / w_pairs in its tetra layout (halo points written).
 * Returns TETRA_EINVAL for mismatched plans, kT <= 0, null or misaligned
 * pointers, TETRA_EUNSUPPORTED for slab plans or n_bands > 8. */
tetra_status_t tetra_pair_bands(tetra_plan_t plan, const float *eps, const int q[3], float kT, float mu,
                                tetra_plan_t pair_plan, float *eps_pairs, float *w_pairs, cudaStream_t stream);

/* Spectral function of the bare susceptibility at T = 0 (the extension to
 * susceptibilities the paper names as future work; not in the paper):
 *   S(q, w) = sum_{n,m} (1/V_G) int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
 *                                  delta(w - e_m(k+q) + e_n(k)),
 *   Im chi0(q, w + i0) = -pi S(q, w),
 * with every band linear inside each tetrahedron (the method's
 * interpolation) and the step occupations clipped exactly: in each
 * tetrahedron the regions {e_n < mu < e_m(k+q)} (+1) and
 * {e_m(k+q) < mu < e_n} (-1) are cut into sub-tetrahedra over which the
 * transition energy is linear.
 *   plan    : the bands (n_bands <= 8; n_orb, weight_dtype and mode unused),
 *             eps in its tetra layout; whole-grid plans only.
 *   q       : integer grid vector (q_i in units of 2 pi / n_i), any sign.
 *   mu      : chemical potential (energy units of eps).
 *   mode    : TETRA_POINT: S at n_omega ascending energies omega[i];
 *             TETRA_BIN: bin averages over n_omega bins, omega holds the
 *             n_omega + 1 ascending edges.
 *   S       : [n_omega] float, overwritten.
 *   ws      : at least tetra_spectral_t0_workspace_bytes(plan, n_omega)
 *             bytes, 16-byte aligned.
 * Exact integer accumulation: the result does not depend on the launch.
 * Returns TETRA_EINVAL for null/misaligned pointers or a bad mode,
 * TETRA_EUNSUPPORTED for n_bands > 8, slab plans, or n_omega beyond one
 * shared-memory tile (about 17000 energies); device-side TETRA_ERANGE
 * (tetra_workspace_status) for a contribution beyond the 64-bit range. */
size_t tetra_spectral_t0_workspace_bytes(tetra_plan_t plan, int n_omega);
tetra_status_t tetra_spectral_t0(tetra_plan_t plan, const float *eps, const int q[3], float mu, int mode,
                                 int n_omega, const float *omega, float *S, void *ws, size_t ws_bytes,
                                 cudaStream_t stream);

/* Real part of the T = 0 bare susceptibility (the Lindhard-type extension of
 * the method, abstract and Conclusions) at grid vector q:
 *   Re chi0(q, w) = sum_{n,m} (1/V_G) P int dk [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
 *                                          / (w - e_m(k+q) + e_n(k)),
 * the Hilbert transform of tetra_spectral_t0's S (chi0 = int S(w')/(w - w' + i0) dw').
 * Same clipping into sub-tetrahedra as tetra_spectral_t0; each sub-tetrahedron
 * of volume fraction nu adds sign * nu * P<1/(w - D)>, the principal-value
 * average of 1/(w - D) over it (D linear there): a moment series beyond four
 * half-widths of its D range, the closed form of its density's three
 * quadratic pieces (logarithms) nearer. Every sub-tetrahedron reaches every
 * energy, so the cost grows with n_omega x sub-tetrahedra.
 *   plan, eps, q, mu : as tetra_spectral_t0 (whole-grid plan, n_bands <= 8).
 *   omega   : [n_omega] float, device, the energies (eV); any order.
 *   R       : [n_omega] float, overwritten.
 *   ws      : at least tetra_chi0_real_t0_workspace_bytes(plan, n_omega)
 *             bytes, 16-byte aligned.
 * The sub-tetrahedra of a warp are summed in FP32 in a fixed order (64 at a
 * time) and added to exact 64-bit integer tiles: reproducible for a given
 * plan and device, not bitwise independent of the launch shape. Returns
 * TETRA_EINVAL for null/misaligned pointers, TETRA_EUNSUPPORTED for
 * n_bands > 8, slab plans or n_omega beyond about 6000 (shared memory);
 * device-side TETRA_ERANGE (tetra_workspace_status) for a sum beyond the
 * 64-bit range. */
size_t tetra_chi0_real_t0_workspace_bytes(tetra_plan_t plan, int n_omega);
tetra_status_t tetra_chi0_real_t0(tetra_plan_t plan, const float *eps, const int q[3], float mu,
                                  int n_omega, const float *omega, float *R, void *ws, size_t ws_bytes,
                                  cudaStream_t stream);

/* Device-side status recorded in a workspace by the last call that used it
 * (synchronises `stream`). TETRA_OK, TETRA_ETIMEOUT or TETRA_ERANGE. The
 * fixed-point accumulation of tetra_dos raises TETRA_ERANGE (and leaves that
 * contribution out) when one contribution exceeds the 64-bit range: in point
 * mode a nearly flat tetrahedron (energy spread below ~1e-12 eV for typical
 * grids) with a grid energy inside its window, whose DOS there is ~3/E41. */
tetra_status_t tetra_workspace_status(const void *ws, cudaStream_t stream);

/* Human-readable name of a status. */
const char *tetra_strerror(tetra_status_t status);

/* Library version, e.g. "0.1.0". */
const char *tetra_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TETRA_H */
