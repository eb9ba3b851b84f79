"""GPU parity on the benchmark's own inputs (Sec. II.A eigen-data into
Eqs. (8)-(9)): the seeded 8-orbital model on the 256^3 grid, its eigen-data
from the GPU eigensolver (tetra_eig), 4000 energies on [eps_min - 0.1,
eps_max + 0.1], point mode, in the launch configuration bench.py times.

The oracle evaluates the same eigen-data (the values the kernel reads,
widened to FP64) at energies spread over the band range, cube slab by cube
slab. Bars:
  * FP32 weights, and FP16 / BF16 weights with the oracle fed the same
    rounded weights: 2e-5 * max |DOS| (the kernel on identical inputs).
  * FP16 / BF16 weights against the oracle on the unrounded (FP32) weights:
    the storage error of the weights, reported and bounded by the relative
    rounding unit of the storage type (2^-11 FP16, 2^-8 BF16): every
    contribution is a non-negative combination of the weights, so a relative
    error u of each weight moves the DOS by at most u * DOS.
  * End to end on the 64^3 grid, 2000 energies: GPU eigensolver + DOS against
    LAPACK (FP64) + the oracle; reported, and bounded by the effect of the
    FP32 eigensolver's eigenvalue error (see the test).
"""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import model_arrays

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


def oracle_dos_layout(E, W, n, nb, no, energies, slab=16):
    """Oracle point DOS of eigen-data held in the tetra layout (numpy arrays
    of the padded point grid), cube slab by cube slab: planes z0 .. z1 of the
    layout form a grid of z1 - z0 + 1 planes whose first z1 - z0 cube planes
    are the slab's cubes (no periodic wrap in z is needed); the oracle's
    volume factor 1/(6 n1 n2 n3') is rescaled to the full n3."""
    n1, n2, n3 = n
    out = np.zeros((no, len(energies)))
    for z0 in range(0, n3, slab):
        z1 = min(z0 + slab, n3)
        nz = z1 - z0 + 1
        e = np.ascontiguousarray(E[z0:z1 + 1, :n2, :n1, :nb], dtype=np.float64).reshape(-1, nb)
        w = np.ascontiguousarray(W[z0:z1 + 1, :n2, :n1, :nb * no], dtype=np.float64).reshape(-1, nb, no)
        part = oracle.dos(e, w, n1, n2, nz, np.asarray(energies, np.float64), z_range=(0, z1 - z0),
                          nthreads=NTHREADS)
        out += part * (nz / n3)
    return out


def bench_problem(T, wdtype, n=256, nw=4000):
    """Model, eigen-data (GPU) and energy grid exactly as bench.py builds them."""
    dev = torch.device("cuda")
    p, R = model_arrays(tbgen.tb_model(0, n_orb=8))
    plan = T.Plan(n, n, n, 8, 8, nw, weight_dtype=wdtype)
    eps, w = plan.empty_inputs()
    plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev), eps, w)
    torch.cuda.synchronize()
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    omega = torch.from_numpy(tbgen.uniform_grid(lo, hi, nw)).to(dev)
    return plan, eps, w, omega


SAMPLE = np.linspace(150, 3850, 12).round().astype(int)


@pytest.fixture(scope="module")
def f32_reference(T):
    """FP32 run of the benchmark configuration and the oracle on its inputs."""
    plan, eps, w, omega = bench_problem(T, "f32")
    g = plan.dos(eps, w, omega)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    E = eps.cpu().numpy()
    W = w.cpu().numpy()
    om = omega.cpu().numpy()
    r = oracle_dos_layout(E, W, (256,) * 3, 8, 8, om[SAMPLE])
    out = {"gpu": g.cpu().numpy().astype(np.float64), "oracle": r, "E": E, "W": W, "omega": om}
    del eps, w, plan
    torch.cuda.empty_cache()
    return out


def test_benchmark_inputs_f32(f32_reference):
    g, r = f32_reference["gpu"][:, SAMPLE], f32_reference["oracle"]
    err = np.max(np.abs(g - r)) / np.max(np.abs(r))
    print(f"256^3 benchmark inputs, FP32 weights, {len(SAMPLE)} energies: max rel err {err:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("wdtype,unit", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_benchmark_inputs_reduced_precision(T, f32_reference, wdtype, unit):
    plan, eps, w, omega = bench_problem(T, wdtype)
    # the eigensolver computes in FP32 whatever the storage type: same energies
    assert np.array_equal(eps.cpu().numpy(), f32_reference["E"])
    g = plan.dos(eps, w, omega)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    g = g.cpu().numpy().astype(np.float64)[:, SAMPLE]
    Wr = w.to(torch.float32).cpu().numpy()
    del w
    # (1) the kernel on identical (rounded) inputs
    r_rounded = oracle_dos_layout(f32_reference["E"], Wr, (256,) * 3, 8, 8, f32_reference["omega"][SAMPLE])
    err = np.max(np.abs(g - r_rounded)) / np.max(np.abs(r_rounded))
    # (2) against the FP64 oracle on the unrounded (FP32) weights
    r = f32_reference["oracle"]
    err_storage = np.max(np.abs(g - r)) / np.max(np.abs(r))
    print(f"256^3 benchmark inputs, {wdtype} weights: parity {err:.2e}, "
          f"error against the oracle on unrounded weights {err_storage:.2e}")
    assert err <= TOL
    assert err_storage <= unit + 2 * TOL


def test_end_to_end_64cube(T):
    """GPU eigensolver + DOS against LAPACK eigh (FP64) + the oracle on the
    8-orbital model, 64^3 grid, 2000 energies. The FP32 eigensolver's
    eigenvalues are within ~1e-5 eV of LAPACK (test_gpu_eig); a shift de of
    the four corner energies of a tetrahedron moves its point DOS by about
    |d rho_T/dE| de ~ 6 de / E41^2 of V_T/V_G, i.e. a relative change
    ~2 de / E41 of its contribution. Tetrahedra of the 64^3 grid have E41 of
    order 0.1 eV, so each contribution moves by ~2e-4 relative at most, and
    these shifts are uncorrelated between tetrahedra; the bound 1e-3 * max
    leaves room for the narrowest tetrahedra near band extrema."""
    n = 64
    nw = 2000
    dev = torch.device("cuda")
    model = tbgen.tb_model(0, n_orb=8)
    p, R = model_arrays(model)
    plan = T.Plan(n, n, n, 8, 8, nw)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    omega = tbgen.uniform_grid(lo, hi, nw)
    g = plan.dos(eps, w, torch.from_numpy(omega).to(dev))
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    g = g.cpu().numpy().astype(np.float64)
    # FP64 reference: the FP32-rounded parameters (what the GPU sees) in LAPACK
    m64 = oracle.params_to_model(p.astype(np.float64), model)
    e64, w64 = oracle.eig(m64, n, n, n)
    idx = np.arange(5, nw, 25)
    r = oracle.dos(e64, w64, n, n, n, omega[idx].astype(np.float64), nthreads=NTHREADS)
    err = np.max(np.abs(g[:, idx] - r)) / np.max(np.abs(r))
    print(f"64^3 end to end (GPU eig + DOS vs LAPACK + oracle), {len(idx)} energies: max rel err {err:.2e}")
    assert err <= 1e-3
