"""T = 0 spectral function of the bare susceptibility on the GPU
(tetra_spectral_t0, exact double-band clipping of every tetrahedron) against
the FP64 oracle (oracle.spectral_t0) on the same FP32 band energies widened
to FP64. Bar: 2e-5 * max |S| as for the DOS; the clipping runs in FP32, and
the thinnest sub-tetrahedra carry weights proportional to their volume, so
the rounding of a cut moves a value by a relative ~1e-6 of the largest
contributions at most."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import model_arrays, tb_problem, to_layout

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


def gpu_spectral(T, eps, n, q, mu, omega, mode):
    nb = eps.shape[1]
    plan = T.Plan(*n, nb, 1, 16)
    L = plan.layout
    E, _ = to_layout(eps, np.zeros((eps.shape[0], nb, 1), np.float32), *n, L.eps_stride, L.w_stride)
    dev = torch.device("cuda")
    Et = torch.from_numpy(E).to(dev)
    om = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev)
    s = plan.spectral_t0(Et, q, mu, om, mode=mode)
    torch.cuda.synchronize()
    assert plan.spectral_status() == T.TETRA_OK
    return s.cpu().numpy().astype(np.float64), plan, Et, om


@pytest.mark.parametrize("mode", ["point", "bin"])
@pytest.mark.parametrize("q", [(0, 0, 0), (3, 0, 0), (-2, 5, 1)])
def test_spectral_t0_against_oracle(T, q, mode):
    n = (10, 9, 8)
    _, eps, _ = tb_problem(3, n)
    mu = float(np.median(eps))
    omega = tbgen.bin_edges(-3.0, 3.0, 240) if mode == "bin" else tbgen.uniform_grid(-3.0, 3.0, 241)
    g, *_ = gpu_spectral(T, eps, n, q, mu, omega, mode)
    r = oracle.spectral_t0(eps.astype(np.float64), *n, q, mu, omega.astype(np.float64), mode=mode,
                           nthreads=NTHREADS)
    scale = np.max(np.abs(r))
    assert scale > 0
    err = np.max(np.abs(g - r)) / scale
    print(f"q={q} {mode}: max rel err {err:.2e}")
    assert err <= TOL


def test_spectral_t0_sum_rule_sign_and_determinism(T):
    """Bin mode over every transition energy integrates to zero (the occupied
    volumes of band n and of the shifted band m agree); S >= 0 above zero
    energy and <= 0 below; two calls give the same bits."""
    n = (8, 8, 6)
    _, eps, _ = tb_problem(5, n)
    mu = float(np.median(eps))
    span = float(eps.max() - eps.min()) + 0.5
    edges = tbgen.bin_edges(-span, span, 400)
    g, plan, Et, om = gpu_spectral(T, eps, n, (2, 3, 1), mu, edges, "bin")
    total = float((g * np.diff(edges.astype(np.float64))).sum())
    pos = float((np.clip(g, 0, None) * np.diff(edges.astype(np.float64))).sum())
    assert abs(total) <= 1e-5 * pos, (total, pos)
    mid = 0.5 * (edges[1:] + edges[:-1]).astype(np.float64)
    width = float(edges[1] - edges[0])
    assert np.all(g[mid > width] >= -1e-6 * g.max()) and np.all(g[mid < -width] <= 1e-6 * g.max())
    again = plan.spectral_t0(Et, (2, 3, 1), mu, om, mode="bin").cpu().numpy().astype(np.float64)
    assert np.array_equal(again, g)


def test_spectral_t0_from_the_model_at_64cube(T):
    """Model -> tetra_eig -> Fermi level of 4 electrons -> S(q, w) at T = 0
    for q = (16, 0, 0) on 400 energies in [0, 4] eV; the oracle at a sample
    of energies on the GPU's band energies."""
    n = (64, 64, 64)
    model = tbgen.tb_model(0, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 8, 16)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    omega = tbgen.uniform_grid(0.0, 4.0, 400)
    s = plan.spectral_t0(eps, (16, 0, 0), mu, torch.from_numpy(omega).to(dev)).cpu().numpy().astype(np.float64)
    assert plan.spectral_status() == T.TETRA_OK
    E = eps.cpu().numpy()[:64, :64, :64, :8].reshape(-1, 8).astype(np.float64)
    idx = np.linspace(5, 395, 8).astype(int)
    r = oracle.spectral_t0(E, *n, (16, 0, 0), mu, omega[idx].astype(np.float64), nthreads=NTHREADS)
    err = np.max(np.abs(s[idx] - r)) / np.max(np.abs(s))
    print(f"64^3 T=0 spectral function, 8 energies: max rel err {err:.2e}")
    assert err <= TOL
