"""GPU integrated orbital occupation n_s(E) (tetra_dos in TETRA_INTEGRATED mode)
and the Fermi level (tetra_fermi_level) against the FP64 oracle, on identical
inputs (the FP32 values the GPU reads, widened for the oracle).

Bar: max |n_gpu - n_oracle| <= 2e-5 * max |n_oracle| (the DOS parity bar);
Fermi levels within 1e-4 eV (FP32 energies; N(E) carries FP32 rounding)."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import energy_window, from_layout, model_arrays, sc_problem, tb_problem, to_layout

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


def gpu_inputs(T, eps, w, n, n_omega, mode="integrated"):
    plan = T.Plan(*n, eps.shape[1], w.shape[2], n_omega, mode=mode)
    L = plan.layout
    E, W = to_layout(eps, w, *n, L.eps_stride, L.w_stride, np.float32)
    dev = torch.device("cuda")
    return plan, torch.from_numpy(E).to(dev), torch.from_numpy(W).to(dev)


def run(T, eps, w, n, omega):
    plan, Et, Wt = gpu_inputs(T, eps, w, n, len(omega))
    om = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(Et.device)
    out = plan.dos(Et, Wt, om)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    return out.cpu().numpy().astype(np.float64)


def parity(g, r, tol=TOL):
    err = np.max(np.abs(g - r))
    assert err <= tol * np.max(np.abs(r)), (err, np.max(np.abs(r)))


def test_integrated_occupation_matches_oracle_beyond_both_band_edges(T):
    n = (10, 9, 11)   # ragged boxes in every direction
    _, eps, w = tb_problem(0, n)
    omega = tbgen.uniform_grid(float(eps.min()) - 1.0, float(eps.max()) + 1.0, 401)
    g = run(T, eps, w, n, omega)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), mode="integrated", nthreads=NTHREADS)
    parity(g, r)
    # below every band nothing, above every band the k-average of sum_n b_sn
    assert np.all(g[:, 0] == 0.0)
    np.testing.assert_allclose(g[:, -1], w.astype(np.float64).sum(1).mean(0), rtol=1e-5)


def test_integrated_grid_inside_the_bands_and_a_single_energy(T):
    n = (8, 7, 6)
    _, eps, w = tb_problem(2, n)
    omega = energy_window(eps, 150, pad=-0.5)   # starts above the lowest band bottom
    g = run(T, eps, w, n, omega)
    r = oracle.dos(eps, w, *n, omega.astype(np.float64), mode="integrated", nthreads=NTHREADS)
    parity(g, r)
    one = np.array([0.5 * (eps.min() + eps.max())], np.float32)
    g1 = run(T, eps, w, n, one)
    r1 = oracle.dos(eps, w, *n, one.astype(np.float64), mode="integrated", nthreads=NTHREADS)
    parity(g1, r1)


def test_integrated_flushes_leave_the_bits_unchanged(T, monkeypatch):
    n = (16, 14, 12)
    _, eps, w = tb_problem(9, n)
    omega = energy_window(eps, 600)
    g1 = run(T, eps, w, n, omega)
    g2 = run(T, eps, w, n, omega)
    assert np.array_equal(g1, g2)
    monkeypatch.setenv("TETRA_FLUSH_BITS", "10")
    g3 = run(T, eps, w, n, omega)
    assert np.array_equal(g1, g3)


def test_integrated_64cube_sampled(T):
    n = (64, 64, 64)
    _, eps, w = tb_problem(0, n)
    omega = energy_window(eps, 1500)
    g = run(T, eps, w, n, omega)
    idx = np.linspace(0, 1499, 12).astype(int)
    r = oracle.dos(eps, w, *n, omega[idx].astype(np.float64), mode="integrated", nthreads=NTHREADS)
    assert np.max(np.abs(g[:, idx] - r)) <= TOL * np.max(np.abs(g))


def test_integrated_grid_of_several_energy_chunks(T):
    """6000 energies with 8 orbitals span three shared-memory tiles. Each chunk
    puts the full step of every tetrahedron below it on its first energy, so
    every value is the same integer sum as in a plan over any slice of the grid
    that contains it (the fixed-point unit of this mode does not depend on the
    grid), and the chunked result matches the oracle at sampled energies."""
    n = (12, 10, 9)
    _, eps, w = tb_problem(3, n)
    omega = energy_window(eps, 6000, pad=0.3)
    g = run(T, eps, w, n, omega)
    for a, b in [(0, 1700), (1700, 3900), (3900, 6000), (1999, 2002), (4321, 4322)]:
        assert np.array_equal(g[:, a:b], run(T, eps, w, n, omega[a:b])), (a, b)
    idx = np.unique(np.concatenate([np.linspace(0, 5999, 19).astype(int), [1999, 2000, 2001, 3999, 4000]]))
    r = oracle.dos(eps, w, *n, omega[idx].astype(np.float64), mode="integrated", nthreads=NTHREADS)
    parity(g[:, idx], r)
    np.testing.assert_allclose(g[:, -1], w.astype(np.float64).sum(1).mean(0), rtol=1e-5)
    # occupations do not decrease with E (up to one fixed-point rounding per item)
    assert np.min(np.diff(g, axis=1)) >= -1e-6 * np.max(g)
    # a non-uniform grid of several chunks (spacing growing towards the top)
    x = np.linspace(0.0, 1.0, 5000)
    lo, hi = float(eps.min()) - 0.2, float(eps.max()) + 0.2
    om2 = (lo + (hi - lo) * (0.3 * x + 0.7 * x ** 3)).astype(np.float32)
    g2 = run(T, eps, w, n, om2)
    idx2 = np.linspace(0, 4999, 17).astype(int)
    r2 = oracle.dos(eps, w, *n, om2[idx2].astype(np.float64), mode="integrated", nthreads=NTHREADS)
    parity(g2[:, idx2], r2)


@pytest.mark.parametrize("n_electrons", [0.37, 2.0, 5.25])
def test_fermi_level_matches_oracle(T, n_electrons):
    n = (12, 11, 10)
    _, eps, w = tb_problem(4, n)
    plan, Et, Wt = gpu_inputs(T, eps, w, n, 16, mode="point")
    ef = plan.fermi_level(Et, Wt, n_electrons)
    ef_ref = oracle.fermi_level(eps.astype(np.float64), *n, n_electrons, nthreads=NTHREADS)
    assert abs(ef - ef_ref) < 1e-4, (ef, ef_ref)
    # orbital occupations at E_F add up to the electron count
    occ = run(T, eps, w, n, np.array([ef], np.float32))[:, 0]
    assert abs(occ.sum() - n_electrons) < 2e-4 * max(1.0, n_electrons)


def test_simple_cubic_half_filling_on_gpu(T):
    _, eps, w = sc_problem(16)
    plan, Et, Wt = gpu_inputs(T, eps, w, (16, 16, 16), 16, mode="point")
    assert abs(plan.fermi_level(Et, Wt, 0.5)) < 1e-5


def test_fermi_level_from_the_gpu_eigensolver(T):
    """Model -> tetra_eig -> tetra_fermi_level, against the oracle on the
    eigen-data the GPU produced."""
    n = (14, 12, 10)
    model = tbgen.tb_model(5, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 8, 64)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    ef = plan.fermi_level(eps, w, 3.5)
    E_h, _ = from_layout(eps.cpu().numpy(), w.cpu().numpy(), *n, 8, 8)
    ef_ref = oracle.fermi_level(E_h.astype(np.float64), *n, 3.5, nthreads=NTHREADS)
    assert abs(ef - ef_ref) < 1e-4, (ef, ef_ref)
