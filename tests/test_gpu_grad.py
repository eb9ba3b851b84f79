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


# Bounds from the FP32 arithmetic (u = 2^-24), each well above the measured
# error and far below the size of a real mistake (a dropped term or a wrong
# sign moves a gradient by O(1) of its largest entry):
#  * DOS adjoint, weights: differences of FP32 corner weights at bin edges,
#    each weight O(V_T/4V_G) with error ~4u of it; the difference is smaller
#    than the weights by about (bin width)/E41, so its relative error is
#    ~4u E41/width ~ 1e-6 on the test grids (bins ~0.6 eV, E41 ~ 1-3 eV).
DOS_W_TOL = 1e-5
#  * DOS adjoint, energies: the tangents carry 1/(E_j - E_i) factors whose
#    terms cancel when two corner energies nearly coincide, so a few more
#    digits are lost than for the weights.
DOS_E_TOL = 1e-4
#  * eigensolver adjoint: FP32 eigenvectors are accurate to ~u |H| / gap
#    (|H| ~ 5 eV, gaps ~0.3 eV: ~1e-6); the 1/(e_n - e_m) factors are formed
#    in FP64 and regularised, so near-degenerate pairs do not amplify it.
EIG_TOL = 2e-5


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
    print(f"dos backward ({case}): grad_w {rel_err(gw, rw):.2e}, grad_eps {rel_err(ge, re):.2e}")
    assert rel_err(gw, rw) < DOS_W_TOL
    assert rel_err(ge, re) < DOS_E_TOL


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
    err = rel_err(g.cpu().numpy().astype(np.float64), ref)
    print(f"eig backward: {err:.2e}")
    assert err < EIG_TOL


def chain_loss_oracle(params, model, n, edges, target):
    m = oracle.params_to_model(params, model)
    e, w = oracle.eig(m, *n)
    d = oracle.dos(e, w, *n, edges, mode="bin", nthreads=NTHREADS)
    return float(((d - target) ** 2).sum())


# Error budget of the chain gradient: the FP32 eigensolver adjoint is good to
# EIG_TOL of the largest entry of the parameter gradient, the FP32 forward DOS
# to 2e-5 of its maximum and the DOS adjoint to DOS_W_TOL / DOS_E_TOL; chained,
# every component of the gradient is within CHAIN_TOL * max|gradient| of the
# exact one, and a directional derivative g.v (|v| = 1) within
# CHAIN_TOL * |g_subset|_2. The
# finite differences of the FP64 oracle chain carry their own error: the loss
# is only once continuously differentiable (its second derivative jumps when
# a corner energy crosses a bin edge or a case boundary), so the central
# difference is compared with Richardson's extrapolation from steps h and h/2
# and their difference is added to the bound.
CHAIN_TOL = 5e-5


def chain_setup(T, n, nbins):
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
    return model, p32.astype(np.float64), idx, grad, e64, target


def richardson(f, h):
    """Central difference of f at 0 with steps h and h/2: (extrapolated value,
    error estimate)."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3, abs(d2 - d1)


@pytest.mark.parametrize("n,nbins", [((10, 10, 10), 120), ((64, 64, 64), 200)])
def test_hopping_gradient_through_the_chain(T, n, nbins):
    """Config 'differentiation': loss = sum (bin DOS - target)^2 with the target
    from a second seeded model; gradient with respect to the 150 fitted real
    parameters against finite differences of the FP64 oracle chain along four
    random directions in that subset."""
    model, p64, idx, grad, e64, target = chain_setup(T, n, nbins)
    gnorm = np.linalg.norm(grad[idx])
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(4):
        v = np.zeros_like(p64)
        v[idx] = rng.normal(0, 1, idx.size)
        v /= np.linalg.norm(v)
        fd, fd_err = richardson(lambda h: chain_loss_oracle(p64 + h * v, model, n, e64, target), 2e-4)
        an = float(grad @ v)
        worst = max(worst, (abs(an - fd) - fd_err) / gnorm)
        assert abs(an - fd) <= CHAIN_TOL * gnorm + fd_err, (an, fd, fd_err, gnorm)
    print(f"chain {n}: max |g.v - FD| / |g| = {max(worst, 0.0):.2e} (bound {CHAIN_TOL})")


def test_full_parameter_gradient_16cube(T):
    """Every one of the 150 fitted parameters, 16^3 grid, 200 bins: the GPU
    chain gradient against the FP64 oracle chain's central differences
    (Richardson-extrapolated), component by component."""
    n = (16, 16, 16)
    model, p64, idx, grad, e64, target = chain_setup(T, n, 200)
    fd = np.zeros(idx.size)
    fd_err = np.zeros(idx.size)
    for j, i in enumerate(idx):
        e = np.zeros_like(p64)
        e[i] = 1.0
        fd[j], fd_err[j] = richardson(lambda h: chain_loss_oracle(p64 + h * e, model, n, e64, target), 2e-4)
    scale = np.max(np.abs(fd))
    err = np.abs(grad[idx] - fd)
    print(f"16^3 full gradient, 150 parameters: max |g - FD| / max|FD| = {np.max(err) / scale:.2e}, "
          f"max FD error estimate / max|FD| = {np.max(fd_err) / scale:.2e}")
    assert np.all(err <= CHAIN_TOL * scale + fd_err), np.max(err) / scale
