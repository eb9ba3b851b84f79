"""GPU batched Hermitian eigensolver (tetra_eig) against LAPACK (FP64 numpy.eigh)."""
import numpy as np
import pytest

import oracle
import tbgen
from helpers import model_arrays, rounded_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import paper_1710_10789_gb300 as T
    T.build()
    return T


def gpu_eig(T, model, n, wdtype="f32"):
    n1, n2, n3 = n
    no = model["onsite"].shape[0]
    plan = T.Plan(n1, n2, n3, no, no, 16, weight_dtype=wdtype)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    torch.cuda.synchronize()
    return plan, eps.cpu().float().numpy(), w.cpu().float().numpy()


@pytest.mark.parametrize("n_orb", [1, 2, 3, 5, 8])
def test_eigenvalues_and_weights_match_lapack(T, n_orb):
    n = (7, 6, 5)
    model = tbgen.tb_model(10 + n_orb, n_orb=n_orb)
    plan, E, W = gpu_eig(T, model, n)
    e_ref, w_ref = oracle.eig(rounded_model(model), *n)
    nb = n_orb
    e = E[:n[2], :n[1], :n[0], :nb].reshape(-1, nb)
    w = W[:n[2], :n[1], :n[0], :nb * n_orb].reshape(-1, nb, n_orb)
    scale = max(1.0, np.abs(e_ref).max())
    assert np.max(np.abs(e - e_ref)) < 3e-6 * scale * max(1, n_orb)
    # weights are unique where the band is separated from its neighbours
    gap = np.full(e_ref.shape, np.inf)
    if nb > 1:
        d = np.diff(e_ref, axis=1)
        gap[:, :-1] = np.minimum(gap[:, :-1], d)
        gap[:, 1:] = np.minimum(gap[:, 1:], d)
    ok = gap > 1e-2
    err = np.abs(w - w_ref).max(axis=2)
    assert np.all(err[ok] < 2e-4), err[ok].max()
    np.testing.assert_allclose(w.sum(axis=2), 1.0, atol=2e-5)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=2e-5)


def test_halo_points_duplicate_the_periodic_images(T):
    n = (5, 4, 3)
    model = tbgen.tb_model(3, n_orb=8)
    plan, E, W = gpu_eig(T, model, n)
    np.testing.assert_array_equal(E[:, :, n[0]], E[:, :, 0])
    np.testing.assert_array_equal(E[:, n[1], :], E[:, 0, :])
    np.testing.assert_array_equal(E[n[2], :, :], E[0, :, :])
    np.testing.assert_array_equal(W[n[2], n[1], n[0]], W[0, 0, 0])


def test_simple_cubic_band(T):
    plan, E, W = gpu_eig(T, tbgen.sc_model(), (16, 16, 16))
    e_ref, _ = oracle.eig(tbgen.sc_model(), 16, 16, 16)
    np.testing.assert_allclose(E[:16, :16, :16, 0].ravel(), e_ref[:, 0], atol=2e-6)


@pytest.mark.parametrize("wdtype", ["f16", "bf16"])
def test_low_precision_weight_storage(T, wdtype):
    n = (6, 6, 6)
    model = tbgen.tb_model(4)
    _, E32, W32 = gpu_eig(T, model, n, "f32")
    _, E16, W16 = gpu_eig(T, model, n, wdtype)
    np.testing.assert_array_equal(E32, E16)
    tol = 1e-3 if wdtype == "f16" else 8e-3
    assert np.max(np.abs(W16[..., :64] - W32[..., :64])) < tol


def test_64cube_sampled_points(T):
    n = (64, 64, 64)
    model = tbgen.tb_model(0)
    plan, E, W = gpu_eig(T, model, n)
    m = rounded_model(model)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 64, size=(300, 3))
    H = oracle.hamiltonian(m, 64, 64, 64).reshape(64, 64, 64, 8, 8)
    Hs = H[pts[:, 2], pts[:, 1], pts[:, 0]]
    ev = np.linalg.eigvalsh(Hs)
    e = E[pts[:, 2], pts[:, 1], pts[:, 0], :8]
    assert np.max(np.abs(e - ev)) < 5e-5


def test_slab_plan_writes_only_its_planes(T):
    """A slab plan (cube planes [2, 5)) computes the point planes 2..5, bit for
    bit as the whole-grid plan does, and leaves every other plane untouched."""
    n = (6, 5, 7)
    model = tbgen.tb_model(33, n_orb=8)
    _, E, W = gpu_eig(T, model, n)
    plan = T.Plan(*n, 8, 8, 16, z_range=(2, 5))
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    eps, w = plan.empty_inputs()
    eps.fill_(float("nan"))
    w.fill_(float("nan"))
    plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev), eps, w)
    torch.cuda.synchronize()
    Es, Ws = eps.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(Es[2:6], E[2:6])
    assert np.array_equal(Ws[2:6, ..., :64], W[2:6, ..., :64])   # w_stride 68: 4 padding entries
    assert np.isnan(Es[:2]).all() and np.isnan(Es[6:]).all()
    assert np.isnan(Ws[:2]).all() and np.isnan(Ws[6:]).all()


def test_orbital_subset_weights(T):
    """A plan with fewer orbitals than the model stores the weights of the
    model's first orbitals, bit for bit as the full projection does."""
    n = (5, 6, 4)
    model = tbgen.tb_model(12, n_orb=8)
    _, E8, W8 = gpu_eig(T, model, n)
    plan = T.Plan(*n, 8, 5, 16)
    p, R = model_arrays(model)
    dev = torch.device("cuda")
    eps, w = plan.eig(torch.from_numpy(p).to(dev), torch.from_numpy(R).to(dev))
    torch.cuda.synchronize()
    E5, W5 = eps.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(E5, E8)
    w8 = W8[..., :64].reshape(W8.shape[:3] + (8, 8))
    w5 = W5[..., :40].reshape(W5.shape[:3] + (8, 5))
    assert np.array_equal(w5, w8[..., :5])
