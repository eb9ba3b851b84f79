"""GPU parity of tetra_dos against the FP64 oracle (called through the C ABI).

Bar: max |dos_gpu - dos_oracle| <= 2e-5 * max |dos_oracle| for FP32 weights
on identical inputs (the FP32 values the GPU reads, widened to FP64 for the
oracle). FP16/BF16 runs give the oracle the same rounded weights, so the same
bar applies to the kernel itself.
"""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import energy_window, from_layout, sc_problem, tb_problem, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def T():
    import paper_1710_10789_gb300 as T
    T.build()
    assert torch.cuda.is_available()
    return T


def run_gpu(T, eps, w, n, omega, mode="point", wdtype="f32", z_range=None, n_omega=None):
    n1, n2, n3 = n
    nb, no = eps.shape[1], w.shape[2]
    nw = len(omega) - 1 if mode == "bin" else len(omega)
    plan = T.Plan(n1, n2, n3, nb, no, nw, mode=mode, weight_dtype=wdtype, z_range=z_range)
    L = plan.layout
    npw = {"f32": np.float32, "f16": np.float16, "bf16": np.float32}[wdtype]
    E, W = to_layout(eps, w, n1, n2, n3, L.eps_stride, L.w_stride, npw)
    dev = torch.device("cuda")
    Et = torch.from_numpy(E).to(dev)
    Wt = torch.from_numpy(W).to(dev)
    if wdtype == "bf16":
        Wt = Wt.to(torch.bfloat16)
    om = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev)
    out = plan.dos(Et, Wt, om)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    return out.cpu().numpy().astype(np.float64), plan, Et, Wt, om


def assert_parity(g, r, tol=TOL):
    err = np.max(np.abs(g - r))
    scale = np.max(np.abs(r))
    assert scale > 0
    assert err <= tol * scale, f"max err {err:.3e} vs {tol * scale:.3e} (max {scale:.3e})"
    return err / scale


def rounded_weights(w, wdtype):
    if wdtype == "f16":
        return w.astype(np.float16).astype(np.float64)
    if wdtype == "bf16":
        return torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    return w.astype(np.float64)


# ---------------------------------------------------------------- small cases, dense oracle
def test_simple_cubic_16_point_mode(T):
    """Single band SC NN tight binding, 16^3, 401 energies on [-6.5, 6.5]."""
    _, eps, w = sc_problem(16)
    omega = tbgen.uniform_grid(-6.5, 6.5, 401)
    g, *_ = run_gpu(T, eps, w, (16, 16, 16), omega)
    r = oracle.dos(eps, w, 16, 16, 16, omega.astype(np.float64), nthreads=NTHREADS)
    assert_parity(g, r)


@pytest.mark.parametrize("wdtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", ["point", "bin"])
def test_tb8_small_grid(T, mode, wdtype):
    n = (10, 9, 11)   # ragged: partial boxes in every direction
    _, eps, w = tb_problem(0, n)
    omega = energy_window(eps, 301 if mode == "point" else 121)
    g, *_ = run_gpu(T, eps, w, n, omega, mode=mode, wdtype=wdtype)
    r = oracle.dos(eps, rounded_weights(w, wdtype), *n, omega.astype(np.float64), mode=mode,
                   nthreads=NTHREADS)
    assert_parity(g, r)


@pytest.mark.parametrize("n_orb,nb", [(1, 1), (2, 2), (3, 3), (5, 5), (4, 7)])
def test_orbital_and_band_counts(T, n_orb, nb):
    n = (6, 7, 5)
    rng = np.random.default_rng(n_orb * 10 + nb)
    nk = np.prod(n)
    eps = np.sort(rng.normal(0, 1.5, (nk, nb)), axis=1).astype(np.float32)
    w = rng.uniform(0, 1, (nk, nb, n_orb)).astype(np.float32)
    omega = energy_window(eps, 97)
    g, *_ = run_gpu(T, eps, w, n, omega)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), nthreads=NTHREADS)
    assert_parity(g, r)


def test_sixteen_orbitals_and_energy_chunking(T):
    """n_orb = 16 and enough energies that the shared tile is split into chunks."""
    n = (6, 6, 6)
    rng = np.random.default_rng(16)
    nk = np.prod(n)
    eps = np.sort(rng.normal(0, 2, (nk, 4)), axis=1).astype(np.float32)
    w = rng.uniform(0, 1, (nk, 4, 16)).astype(np.float32)
    omega = energy_window(eps, 5000)
    g, plan, *_ = run_gpu(T, eps, w, n, omega)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), nthreads=NTHREADS)
    assert_parity(g, r)


def test_energy_grid_outside_bands_gives_zero(T):
    _, eps, w = tb_problem(1, (5, 5, 5))
    omega = tbgen.uniform_grid(float(eps.max()) + 1.0, float(eps.max()) + 3.0, 50)
    g, *_ = run_gpu(T, eps, w, (5, 5, 5), omega)
    assert np.all(g == 0.0)


def test_flat_band_point_and_bin(T):
    """A dispersionless band: point DOS is zero off the level (measure zero on
    the level itself); bin DOS puts the whole weight into the bin holding it."""
    n = (4, 4, 4)
    nk = 64
    eps = np.full((nk, 1), 0.3, np.float32)
    w = np.ones((nk, 1, 1), np.float32)
    omega = tbgen.uniform_grid(-1, 1, 41)
    g, *_ = run_gpu(T, eps, w, n, omega)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64))
    np.testing.assert_array_equal(g, r)
    edges = tbgen.bin_edges(-1, 1, 20)
    g, *_ = run_gpu(T, eps, w, n, edges, mode="bin")
    r = oracle.dos(eps, w, *n, edges.astype(np.float64), mode="bin")
    assert_parity(g, r)
    np.testing.assert_allclose((g[0] * np.diff(edges.astype(np.float64))).sum(), 1.0, rtol=1e-6)


def test_partly_flat_bands_every_mode(T):
    """Bands flat over part of the grid: face-sharing pairs then hold one flat
    and one dispersive tetrahedron (the bin-mode pair takes the exact 64-bit
    path, the integrated pair puts two steps), next to fully flat and fully
    dispersive pairs. Point, bin and integrated mode against the oracle."""
    n = (8, 7, 6)
    x, y, z = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    x, y, z = (a.transpose(2, 1, 0).ravel() for a in (x, y, z))   # k = x + n1 (y + n2 z)
    c = np.cos(2 * np.pi * x / n[0]) + 0.5 * np.cos(2 * np.pi * y / n[1]) + 0.3 * np.cos(2 * np.pi * z / n[2])
    # exactly flat where c <= 0.2 (values within 1e-3 of the level snapped onto
    # it: a window of width ~1e-17 with a grid energy inside would make the
    # point DOS exceed the fixed-point range, which the kernel reports as
    # TETRA_ERANGE instead of computing)
    flat = np.where(c - 0.2 > 1e-3, c - 0.2, 0.0)
    eps = np.stack([flat, np.full(c.shape, 0.7), c], axis=1).astype(np.float32)
    w = np.random.default_rng(5).uniform(0.1, 1.0, (eps.shape[0], 3, 2)).astype(np.float32)
    omega = tbgen.uniform_grid(-1.9, 2.0, 79)
    g, *_ = run_gpu(T, eps, w, n, omega)
    assert_parity(g, oracle.dos(eps, w, *n, omega.astype(np.float64)))
    edges = tbgen.bin_edges(-1.95, 2.05, 40)
    g, *_ = run_gpu(T, eps, w, n, edges, mode="bin")
    r = oracle.dos(eps, w, *n, edges.astype(np.float64), mode="bin")
    assert_parity(g, r)
    g, *_ = run_gpu(T, eps, w, n, omega, mode="integrated")
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), mode="integrated")
    assert_parity(g, r)


def test_flat_band_level_on_a_bin_edge(T):
    n = (3, 3, 3)
    eps = np.full((27, 1), 0.25, np.float32)
    w = np.ones((27, 1, 1), np.float32)
    edges = np.array([-1, -0.5, 0, 0.25, 0.5, 1.0], np.float32)
    g, *_ = run_gpu(T, eps, w, n, edges, mode="bin")
    r = oracle.dos(eps, w, *n, edges.astype(np.float64), mode="bin")
    np.testing.assert_allclose(g, r, rtol=1e-6, atol=1e-7)


def test_single_energy_point(T):
    _, eps, w = tb_problem(2, (6, 6, 6))
    omega = np.array([0.1], np.float32)
    g, *_ = run_gpu(T, eps, w, (6, 6, 6), omega)
    r = oracle.dos(eps, w, 6, 6, 6, omega.astype(np.float64))
    assert_parity(g, r)


def test_nonuniform_grid_is_still_exact(T):
    _, eps, w = tb_problem(3, (7, 6, 5))
    rng = np.random.default_rng(0)
    omega = np.sort(rng.uniform(eps.min() - 0.1, eps.max() + 0.1, 173)).astype(np.float32)
    g, *_ = run_gpu(T, eps, w, (7, 6, 5), omega)
    r = oracle.dos(eps, w, 7, 6, 5, omega.astype(np.float64))
    assert_parity(g, r)


def test_bin_mode_sum_rule_on_gpu(T):
    n = (12, 12, 12)
    _, eps, w = tb_problem(4, n)
    edges = tbgen.bin_edges(float(eps.min()) - 0.1, float(eps.max()) + 0.1, 200)
    g, *_ = run_gpu(T, eps, w, n, edges, mode="bin")
    integral = (g * np.diff(edges.astype(np.float64))[None, :]).sum(1)
    # sum_n |c_sn|^2 = 1 up to the FP32 rounding of the inputs
    np.testing.assert_allclose(integral, 1.0, atol=2e-5)


def test_bitwise_determinism_and_launch_shape_independence(T, monkeypatch):
    n = (14, 13, 12)
    _, eps, w = tb_problem(5, n)
    omega = energy_window(eps, 500)
    g1, *_ = run_gpu(T, eps, w, n, omega)
    g2, *_ = run_gpu(T, eps, w, n, omega)
    assert np.array_equal(g1, g2)
    monkeypatch.setenv("TETRA_BOX_X", "3")
    monkeypatch.setenv("TETRA_BOX_Y", "5")
    monkeypatch.setenv("TETRA_BOX_Z", "2")
    monkeypatch.setenv("TETRA_CTAS_PER_SM", "1")
    g3, *_ = run_gpu(T, eps, w, n, omega)
    assert np.array_equal(g1, g3)


@pytest.mark.parametrize("mode", ["point", "bin"])
def test_tile_flushes_leave_the_bits_unchanged(T, monkeypatch, mode):
    """Blocks of the shared tile are moved into the int64 partials when their
    bound passes 2^flush_bits (2^30 normally). With a low threshold every
    box flushes; integer accumulation makes the result bit-identical, which
    checks the raw-sum / add-count bookkeeping of the flush."""
    n = (20, 18, 16)
    _, eps, w = tb_problem(8, n)
    omega = energy_window(eps, 700 if mode == "point" else 301)   # bin mode: edges
    g1, *_ = run_gpu(T, eps, w, n, omega, mode=mode)
    monkeypatch.setenv("TETRA_FLUSH_BITS", "10")
    g2, *_ = run_gpu(T, eps, w, n, omega, mode=mode)
    assert np.array_equal(g1, g2)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), mode=mode, nthreads=NTHREADS)
    assert_parity(g2, r)


def test_z_slabs_add_up_to_the_whole(T, monkeypatch):
    """Splitting the grid into k-slabs (the unit of multi-device sharding):
    with a common fixed-point unit every item contributes the same integers,
    so the slab sum equals the single call up to the final float rounding."""
    n = (8, 8, 10)
    _, eps, w = tb_problem(6, n)
    omega = energy_window(eps, 200)
    monkeypatch.setenv("TETRA_FIXED_BITS", "20")
    full, *_ = run_gpu(T, eps, w, n, omega)
    parts = sum(run_gpu(T, eps, w, n, omega, z_range=zr)[0] for zr in [(0, 3), (3, 7), (7, 10)])
    assert_parity(parts, full, tol=1e-6)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64))
    assert_parity(parts, r)


# ---------------------------------------------------------------- full-size configurations
def test_tb8_64cube_2000_energies_sampled(T):
    """8-orbital synthetic model, 64^3 grid (1.57M tetrahedra), 2000 energies:
    the GPU result at every energy vs the oracle at a sample of 24 energies."""
    n = (64, 64, 64)
    _, eps, w = tb_problem(0, n)
    omega = energy_window(eps, 2000)
    g, *_ = run_gpu(T, eps, w, n, omega)
    idx = np.linspace(0, 1999, 24).astype(int)
    r = oracle.dos(eps, w, *n, omega[idx].astype(np.float64), nthreads=NTHREADS)
    err = np.max(np.abs(g[:, idx] - r))
    assert err <= TOL * np.max(np.abs(g)), err


def test_synthetic_256cube_4000_energies_sampled(T):
    """256^3 grid (100.7M tetrahedra), 8 bands x 8 orbitals, 4000 energies, in
    the launch configuration the benchmark times; oracle at 4 energies."""
    n = (256, 256, 256)
    eps, w = tbgen.synthetic_bands(7, *n, 8, 8)
    eps = eps.astype(np.float32)
    w = w.astype(np.float32)
    omega = energy_window(eps, 4000)
    g, _, Et, Wt, _ = run_gpu(T, eps, w, n, omega)
    idx = np.array([700, 1500, 2600, 3300])
    r = oracle.dos(eps, w, *n, omega[idx].astype(np.float64), nthreads=NTHREADS)
    err = np.max(np.abs(g[:, idx] - r))
    assert err <= TOL * np.max(np.abs(g)), err
    # per-orbital sum rule at full size, exact in bin mode: over a window that
    # holds every band, the integral of DOS_s is the k-average of
    # sum_n w[k, n, s] (each k-point is a corner of 24 tetrahedra of volume
    # V_G / (6 N)). (A Riemann sum of the point DOS is not exact: near-flat
    # tetrahedra give spikes narrower than the energy spacing.)
    edges = tbgen.bin_edges(float(omega[0]), float(omega[-1]), 4000)
    bplan = T.Plan(*n, 8, 8, 4000, mode="bin")
    gb = bplan.dos(Et, Wt, torch.from_numpy(edges).to(Et.device)).cpu().numpy().astype(np.float64)
    assert bplan.status() == T.TETRA_OK
    integral = (gb * np.diff(edges.astype(np.float64))[None, :]).sum(1)
    np.testing.assert_allclose(integral, w.astype(np.float64).sum(1).mean(0), rtol=1e-4)


def test_slabs_of_one_model_on_separate_plans(T):
    """The k-slab split of one model (paper_1710_10789_gb300.shard): each slab
    computes its own eigen-data and DOS; the rank-ordered sum matches the
    whole-grid DOS within the parity bar, and the oracle."""
    import paper_1710_10789_gb300.shard as shard
    from helpers import model_arrays

    n = (12, 10, 9)
    model = tbgen.tb_model(17, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    pt, Rt = torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev)
    whole = T.Plan(*n, 8, 8, 700)
    eps, w = whole.eig(pt, Rt)
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    om = torch.from_numpy(tbgen.uniform_grid(lo, hi, 700)).to(dev)
    full = whole.dos(eps, w, om).cpu().numpy().astype(np.float64)
    parts = []
    for z0, z1 in shard.slab_ranges(n[2], 4):
        plan = T.Plan(*n, 8, 8, 700, z_range=(z0, z1))
        e_s, w_s = plan.eig(pt, Rt)
        parts.append(plan.dos(e_s, w_s, om))
    total = shard.combine_slabs(torch, parts).cpu().numpy().astype(np.float64)
    assert_parity(total, full)
    E_h, W_h = from_layout(eps.cpu().numpy(), w.cpu().numpy(), *n, 8, 8)
    r = oracle.dos(E_h, W_h, *n, om.cpu().numpy().astype(np.float64), nthreads=NTHREADS)
    assert_parity(total, r)


def test_paper_shape_five_projected_orbitals(T):
    """The paper's benchmark shape (Sec. IV: 60 x 60 x 10 k-grid, 8 bands, the
    DOS projected on 5 of the 8 orbitals, 1024 energies), on the synthetic
    8-orbital model: GPU eigensolver writing the first 5 orbitals' weights,
    then the DOS, against the oracle on the same FP32 eigen-data."""
    from helpers import model_arrays

    n = (60, 60, 10)
    model = tbgen.tb_model(21, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 5, 1024)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    om = torch.from_numpy(tbgen.uniform_grid(lo, hi, 1024)).to(dev)
    g = plan.dos(eps, w, om).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    E_h, W_h = from_layout(eps.cpu().numpy(), w.cpu().numpy(), *n, 8, 5)
    r = oracle.dos(E_h, W_h, *n, om.cpu().numpy().astype(np.float64), nthreads=NTHREADS)
    assert g.shape == (5, 1024)
    assert_parity(g, r)


@pytest.mark.parametrize("how", ["swap_xz", "invert"])
def test_gpu_invariant_under_maps_of_the_triangulation(T, how):
    """Swapping the x and z axes, or inverting k, maps Table I's
    triangulation onto itself with every tetrahedron's corners in another
    order: the GPU's DOS of the relabelled grid equals the original within
    the parity bar (not bit for bit: the rounding dither is keyed to the
    tetrahedron's place in its cube, which the map changes)."""
    from test_oracle_pins import grid_map
    n = (12, 10, 12)
    _, eps, w = tb_problem(9, n)
    omega = energy_window(eps, 300)
    g0, *_ = run_gpu(T, eps, w, n, omega)
    g1, *_ = run_gpu(T, grid_map(eps, n, how), grid_map(w, n, how), n, omega)
    assert_parity(g1, g0)
