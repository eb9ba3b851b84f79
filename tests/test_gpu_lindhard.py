"""Spectral function of the bare susceptibility on the GPU: tetra_pair_bands
(transition energies and occupation differences at momentum q) against the
oracle's definition, then tetra_dos on the pair bands against the oracle DOS
of the same pair bands (the FP32 values the GPU wrote, widened)."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import from_layout, model_arrays, tb_problem, to_layout

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


def spectral(T, eps, w, n, q, kT, mu, omega):
    nb = eps.shape[1]
    plan = T.Plan(*n, nb, w.shape[2], 16)
    E, W = to_layout(eps, w, *n, plan.layout.eps_stride, plan.layout.w_stride, np.float32)
    dev = torch.device("cuda")
    Et = torch.from_numpy(E).to(dev)
    pplan = T.Plan(*n, nb * nb, 1, len(omega))
    ep, wp = plan.pair_bands(Et, q, kT, mu, pplan)
    om = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev)
    s = pplan.dos(ep, wp, om)
    torch.cuda.synchronize()
    assert pplan.status() == T.TETRA_OK
    Dp, Wp = from_layout(ep.cpu().numpy(), wp.cpu().numpy(), *n, nb * nb, 1)
    return s.cpu().numpy().astype(np.float64)[0], Dp, Wp


@pytest.mark.parametrize("q", [(0, 0, 0), (3, 0, 0), (-2, 5, 1)])
def test_pair_bands_and_spectral_function(T, q):
    n = (10, 9, 8)
    _, eps, w = tb_problem(3, n)
    kT, mu = 0.05, float(np.median(eps))
    omega = tbgen.uniform_grid(-3.0, 3.0, 241)
    s, Dp, Wp = spectral(T, eps, w, n, q, kT, mu, omega)
    d_ref, w_ref = oracle.pair_bands(eps.astype(np.float64), *n, q, kT, mu)
    assert np.max(np.abs(Dp - d_ref)) <= 2e-6 * np.abs(eps).max()
    assert np.max(np.abs(Wp - w_ref)) <= 1e-6
    r = oracle.dos(Dp, Wp, *n, omega.astype(np.float64), nthreads=NTHREADS)[0]
    assert np.max(np.abs(s - r)) <= TOL * np.max(np.abs(r))


def test_spectral_function_from_the_model_at_64cube(T):
    """Model -> tetra_eig -> Fermi level of 4 electrons -> pair bands at
    q = (16, 0, 0) -> S(q, w) on 400 energies; the oracle at a sample of
    energies on the GPU's pair bands."""
    n = (64, 64, 64)
    model = tbgen.tb_model(0, n_orb=8)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 8, 16)
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    omega = tbgen.uniform_grid(0.0, 4.0, 400)
    pplan = T.Plan(*n, 64, 1, 400)
    ep, wp = plan.pair_bands(eps, (16, 0, 0), 0.025, mu, pplan)
    s = pplan.dos(ep, wp, torch.from_numpy(omega).to(dev)).cpu().numpy().astype(np.float64)[0]
    assert pplan.status() == T.TETRA_OK
    Dp, Wp = from_layout(ep.cpu().numpy(), wp.cpu().numpy(), *n, 64, 1)
    idx = np.linspace(5, 395, 8).astype(int)
    r = oracle.dos(Dp, Wp, *n, omega[idx].astype(np.float64), nthreads=NTHREADS)[0]
    assert np.max(np.abs(s[idx] - r)) <= TOL * np.max(np.abs(s))
