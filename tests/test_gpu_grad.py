"""GPU adjoints against the FP64 oracle: bin-DOS backward (tetra_dos_backward),
eigensolver backward (tetra_eig_backward) and the full chain hoppings -> DOS
(autograd) against central finite differences of the FP64 oracle chain."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import from_layout, model_arrays, rounded_model, tb_problem, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def T():
    import paper_1710_10789_gb300 as T
    T.build()
    return T


def run_dos_backward(T, eps, w, n, edges, g):
    n1, n2, n3 = n
    nb, no = eps.shape[1], w.shape[2]
    plan = T.Plan(n1, n2, n3, nb, no, len(edges) - 1, mode="bin")
    L = plan.layout
    E, W = to_layout(eps, w, n1, n2, n3, L.eps_stride, L.w_stride)
    dev = torch.device("cuda")
    Et, Wt = torch.from_numpy(E).to(dev), torch.from_numpy(W).to(dev)
    ge, gw = plan.dos_backward(Et, Wt, torch.from_numpy(edges).to(dev),
                               torch.from_numpy(g.astype(np.float32)).to(dev))
    torch.cuda.synchronize()
    ge, gw = ge.cpu().numpy(), gw.cpu().numpy()
    # halo entries are zero
    assert np.all(ge[n3] == 0) and np.all(ge[:, n2] == 0) and np.all(ge[:, :, n1] == 0)
    return from_layout(ge, gw, n1, n2, n3, nb, no)


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("case", ["random", "tb8"])
def test_dos_backward_matches_oracle(T, case):
    if case == "random":
        n = (5, 4, 6)
        rng = np.random.default_rng(3)
        nk = np.prod(n)
        eps = np.sort(rng.normal(0, 1.0, (nk, 3)), axis=1).astype(np.float32)
        w = rng.uniform(0, 1, (nk, 3, 2)).astype(np.float32)
    else:
        n = (8, 7, 6)
        _, eps, w = tb_problem(9, n)
    edges = tbgen.bin_edges(float(eps.min()) - 0.2, float(eps.max()) + 0.2, 40)
    g = np.random.default_rng(4).normal(0, 1, (w.shape[2], 40))
    ge, gw = run_dos_backward(T, eps, w, n, edges, g)
    re, rw = oracle.dos_bin_grad(eps, w, *n, edges.astype(np.float64), g)
    assert rel_err(gw, rw) < 2e-5
    assert rel_err(ge, re) < 5e-4


def test_eig_backward_matches_oracle(T):
    n = (6, 5, 4)
    model = tbgen.tb_model(21, n_orb=8)
    m64 = rounded_model(model)
    rng = np.random.default_rng(7)
    nk = np.prod(n)
    geps = rng.normal(0, 1, (nk, 8))
    gw = rng.normal(0, 1, (nk, 8, 8))
    plan = T.Plan(*n, 8, 8, 16)
    L = plan.layout
    GE, GW = to_layout(geps, gw, *n, L.eps_stride, L.w_stride)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    g = plan.eig_backward(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev),
                          torch.from_numpy(GE).to(dev), torch.from_numpy(GW).to(dev))
    torch.cuda.synchronize()
    ref = oracle.eig_backward(m64, *n, geps, gw)
    # FP32 eigenvectors: compare against the largest entry
    assert rel_err(g.cpu().numpy().astype(np.float64), ref) < 2e-3


def chain_loss_oracle(params, model, n, edges, target):
    m = oracle.params_to_model(params, model)
    e, w = oracle.eig(m, *n)
    d = oracle.dos(e, w, *n, edges, mode="bin", nthreads=NTHREADS)
    return float(((d - target) ** 2).sum())


@pytest.mark.parametrize("n,nbins,ndir", [((10, 10, 10), 120, 3), ((64, 64, 64), 200, 1)])
def test_hopping_gradient_through_the_chain(T, n, nbins, ndir):
    """Config 'differentiation': loss = sum (bin DOS - target)^2 with the target
    from a second seeded model; gradient with respect to the 150 fitted real
    parameters vs central differences of the FP64 oracle chain along random
    directions in that subset."""
    from paper_1710_10789_gb300.autograd import model_dos

    model = tbgen.tb_model(0, n_orb=8)
    target_model = tbgen.tb_model(1, n_orb=8)
    et, wt = oracle.eig(target_model, *n)
    edges = tbgen.bin_edges(float(et.min()) - 0.1, float(et.max()) + 0.1, nbins)
    e64 = edges.astype(np.float64)
    target = oracle.dos(et, wt, *n, e64, mode="bin", nthreads=NTHREADS)
    p32, R = model_arrays(model)
    idx = tbgen.fit_parameter_subset(0, 150, p32.size)
    dev = torch.device("cuda")
    plan = T.Plan(*n, 8, 8, nbins, mode="bin")
    params = torch.from_numpy(p32).to(dev).requires_grad_(True)
    Rt = torch.from_numpy(R).to(dev)
    dos = model_dos(params, Rt, torch.from_numpy(edges).to(dev), plan)
    loss = ((dos.double() - torch.from_numpy(target).to(dev)) ** 2).sum()
    loss.backward()
    grad = params.grad.cpu().numpy().astype(np.float64)
    p64 = p32.astype(np.float64)
    rng = np.random.default_rng(11)
    h = 1e-4
    for _ in range(ndir):
        v = np.zeros_like(p64)
        v[idx] = rng.normal(0, 1, idx.size)
        v /= np.linalg.norm(v)
        fd = (chain_loss_oracle(p64 + h * v, model, n, e64, target) -
              chain_loss_oracle(p64 - h * v, model, n, e64, target)) / (2 * h)
        an = float(grad @ v)
        assert abs(an - fd) <= 2e-2 * abs(fd) + 1e-6, (an, fd)
