"""Real part of the T = 0 bare susceptibility on the GPU (tetra_chi0_real_t0)
against the FP64 oracle (oracle.chi0_real_t0) on the same FP32 band energies
widened to FP64.

Bar, from the FP32 arithmetic: each sub-tetrahedron's principal-value
average is good to a few u = 2^-24 of its magnitude (moment series truncated
below 4^-13, logarithms to ~2^-21 absolute), the averages are summed 64 at a
time in FP32 and the sums added exactly; the result carries the FP32 error of
terms of both signs, whose sum of magnitudes exceeds |Re chi0| by at most a
few hundred on these grids: 1e-4 of max |Re chi0| bounds it, far below what a
dropped region or a wrong sign (O(1) of the result) would give."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import model_arrays, tb_problem, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def T():
    import paper_1710_10789_gb300 as T
    T.build()
    assert torch.cuda.is_available()
    return T


def gpu_real(T, eps, n, q, mu, omega):
    nb = eps.shape[1]
    plan = T.Plan(*n, nb, 1, 16)
    L = plan.layout
    E, _ = to_layout(eps, np.zeros((eps.shape[0], nb, 1), np.float32), *n, L.eps_stride, L.w_stride)
    dev = torch.device("cuda")
    Et = torch.from_numpy(E).to(dev)
    om = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev)
    r = plan.chi0_real_t0(Et, q, mu, om)
    torch.cuda.synchronize()
    assert plan.spectral_status() == T.TETRA_OK
    return r.cpu().numpy().astype(np.float64), plan, Et, om


@pytest.mark.parametrize("q", [(0, 0, 0), (3, 0, 0), (-2, 5, 1)])
def test_chi0_real_against_oracle(T, q):
    n = (10, 9, 8)
    _, eps, _ = tb_problem(3, n)
    mu = float(np.median(eps))
    omega = np.concatenate([tbgen.uniform_grid(-3.0, 3.0, 97), [-25.0, -9.5, 7.25, 40.0]]).astype(np.float32)
    g, *_ = gpu_real(T, eps, n, q, mu, omega)
    r = oracle.chi0_real_t0(eps.astype(np.float64), *n, q, mu, omega.astype(np.float64), nthreads=NTHREADS)
    scale = np.max(np.abs(r))
    err = np.max(np.abs(g - r)) / scale
    print(f"q={q}: max |Re chi0 GPU - oracle| / max = {err:.2e}")
    assert err <= TOL


def test_chi0_real_symmetry_reproducibility_and_kramers_kronig(T):
    """Re chi0(-q, -w) = Re chi0(q, w); two calls give the same bits; and the
    GPU's real part is the Hilbert transform of the GPU's own exact bin
    averages of S (to the binning error)."""
    n = (8, 8, 6)
    _, eps, _ = tb_problem(5, n)
    mu = float(np.median(eps))
    q = (2, 3, 1)
    w = np.array([-2.1, -0.7, 0.03, 0.8, 1.9, 3.3], np.float32)
    g, plan, Et, om = gpu_real(T, eps, n, q, mu, w)
    again = plan.chi0_real_t0(Et, q, mu, om).cpu().numpy().astype(np.float64)
    assert np.array_equal(again, g)
    gm = plan.chi0_real_t0(Et, tuple(-v for v in q), mu, -om).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gm - g)) <= TOL * np.max(np.abs(g))
    span = float(eps.max() - eps.min()) + 0.5
    edges = np.linspace(-span, span, 6001).astype(np.float32)
    s = plan.spectral_t0(Et, q, mu, torch.from_numpy(edges).to(Et.device), mode="bin").cpu().numpy().astype(np.float64)
    e64 = edges.astype(np.float64)
    lo, hi = e64[:-1], e64[1:]
    kk = np.array([np.sum(s * np.log(np.abs((x - lo) / (x - hi)))) for x in w.astype(np.float64)])
    assert np.max(np.abs(g - kk)) <= 3e-3 * np.max(np.abs(g)), (g, kk)


def test_chi0_real_from_the_model_at_64cube(T):
    """Model -> tetra_eig -> Fermi level of 4 electrons -> Re chi0(q, w) at
    T = 0, q = (16, 0, 0), 400 energies on [0, 4] eV (the benchmark's
    workload); the oracle at 6 of them on the GPU's band energies."""
    n = (64, 64, 64)
    model = tbgen.tb_model(0, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 8, 16)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    omega = tbgen.uniform_grid(0.0, 4.0, 400)
    r = plan.chi0_real_t0(eps, (16, 0, 0), mu, torch.from_numpy(omega).to(dev)).cpu().numpy().astype(np.float64)
    assert plan.spectral_status() == T.TETRA_OK
    E = eps.cpu().numpy()[:64, :64, :64, :8].reshape(-1, 8).astype(np.float64)
    idx = np.linspace(3, 396, 6).astype(int)
    ref = oracle.chi0_real_t0(E, *n, (16, 0, 0), mu, omega[idx].astype(np.float64), nthreads=NTHREADS)
    err = np.max(np.abs(r[idx] - ref)) / np.max(np.abs(ref))
    print(f"64^3 Re chi0 at 6 energies: max rel err {err:.2e}")
    assert err <= TOL


def test_chi0_real_near_the_energy_limit_and_beyond(T):
    """6000 energies (near the shared-memory limit of about 6300: the per-warp
    FP32 sums hold every energy) against the oracle at sampled energies; one
    energy more than fits is refused with TETRA_EUNSUPPORTED before any
    launch; and the T = 0 spectral function is refused the same way beyond
    its own limit."""
    n = (6, 5, 4)
    _, eps, _ = tb_problem(3, n)
    mu = float(np.median(eps))
    omega = tbgen.uniform_grid(-4.0, 4.0, 6000)
    g, plan, Et, _ = gpu_real(T, eps, n, (1, 2, 0), mu, omega)
    idx = np.linspace(0, 5999, 9).astype(int)
    r = oracle.chi0_real_t0(eps.astype(np.float64), *n, (1, 2, 0), mu, omega[idx].astype(np.float64),
                            nthreads=NTHREADS)
    assert np.max(np.abs(g[idx] - r)) <= TOL * np.max(np.abs(r))
    dev = Et.device
    big = torch.from_numpy(tbgen.uniform_grid(-4.0, 4.0, 7000)).to(dev)
    with pytest.raises(T.TetraError) as ex:
        plan.chi0_real_t0(Et, (1, 2, 0), mu, big)
    assert ex.value.status == T.TETRA_EUNSUPPORTED
    huge = torch.from_numpy(tbgen.uniform_grid(-4.0, 4.0, 20000)).to(dev)
    with pytest.raises(T.TetraError) as ex:
        plan.spectral_t0(Et, (1, 2, 0), mu, huge)
    assert ex.value.status == T.TETRA_EUNSUPPORTED
