"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: the corner weights are checked
against geometric integrals over the clipped tetrahedron and its iso-energy
cross-section, Bloechl's closed-form tetrahedron DOS, finite differences,
symmetries of the grid, the analytic simple-cubic DOS, Monte-Carlo sampling
of the linear interpolant, and LAPACK.
"""
import itertools

import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle
import tbgen

RNG = np.random.default_rng(12345)
# Table I of the paper (corner labels), kept here independently of the oracle.
TABLE_I = [(1, 2, 3, 6), (2, 3, 4, 6), (1, 3, 5, 6), (3, 4, 6, 8), (3, 5, 6, 7), (3, 6, 7, 8)]


def corner_offset(c):
    c -= 1
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float)


# ---------------------------------------------------------------- geometry helpers
STD = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0, 0, 0]])  # simplex vertices


def lam_of(P):
    """Barycentric coordinates of points P (…,3) of the standard simplex."""
    return np.concatenate([P, 1.0 - P.sum(-1, keepdims=True)], -1)


def clipped_linear_integrals(e, E):
    """Integral of lam_l over {eps < E} within the standard simplex (exact)."""
    eps_v = np.asarray(e, float)
    pts = [STD[i] for i in range(4) if eps_v[i] < E]
    for i, j in itertools.combinations(range(4), 2):
        a, b = eps_v[i], eps_v[j]
        if (a - E) * (b - E) < 0:
            t = (E - a) / (b - a)
            pts.append(STD[i] + t * (STD[j] - STD[i]))
    if len(pts) < 4:
        return np.zeros(4)
    P = np.array(pts)
    try:
        hull = ConvexHull(P)
    except Exception:
        return np.zeros(4)
    c0 = P.mean(0)
    tot = np.zeros(4)
    for simp in hull.simplices:
        A, B, C = P[simp]
        vol = abs(np.dot(A - c0, np.cross(B - c0, C - c0))) / 6.0
        cen = (A + B + C + c0) / 4.0
        tot += vol * lam_of(cen)
    return tot


def cross_section_linear_integrals(e, E):
    """Integral of lam_l delta(E - eps) over the standard simplex (exact)."""
    eps_v = np.asarray(e, float)
    pts = []
    for i, j in itertools.combinations(range(4), 2):
        a, b = eps_v[i], eps_v[j]
        if (a - E) * (b - E) < 0:
            t = (E - a) / (b - a)
            pts.append(STD[i] + t * (STD[j] - STD[i]))
    if len(pts) < 3:
        return np.zeros(4)
    P = np.array(pts)
    c0 = P.mean(0)
    grad = eps_v[:3] - eps_v[3]
    nrm = grad / np.linalg.norm(grad)
    ref = P[0] - c0
    ref /= np.linalg.norm(ref)
    other = np.cross(nrm, ref)
    ang = np.arctan2((P - c0) @ other, (P - c0) @ ref)
    P = P[np.argsort(ang)]
    tot = np.zeros(4)
    for q in range(len(P)):
        A, B = P[q], P[(q + 1) % len(P)]
        area = 0.5 * np.linalg.norm(np.cross(A - c0, B - c0))
        tot += area * lam_of((A + B + c0) / 3.0)
    return tot / np.linalg.norm(grad)


def random_sorted_energies(rng, degenerate=None):
    e = np.sort(rng.normal(0, 1, 4))
    if degenerate == "12":
        e[1] = e[0]
    elif degenerate == "23":
        e[2] = e[1]
    elif degenerate == "34":
        e[3] = e[2]
    return e


F = 1.0 / 24.0  # V_T/(4 V_G) for a 1x1x1 grid; any positive value works


# ---------------------------------------------------------------- single tetrahedron
@pytest.mark.parametrize("trial", range(12))
def test_weights_equal_clipped_volume_integrals(trial):
    rng = np.random.default_rng(100 + trial)
    e = random_sorted_energies(rng)
    for E in np.linspace(e[0] - 0.1, e[3] + 0.1, 23):
        w, _ = oracle.corner_weights(e, E, F)
        ref = 24.0 * F * clipped_linear_integrals(e, E)
        np.testing.assert_allclose(w, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("trial", range(12))
def test_weight_derivatives_equal_cross_section_integrals(trial):
    rng = np.random.default_rng(200 + trial)
    e = random_sorted_energies(rng)
    for E in np.linspace(e[0] + 1e-3, e[3] - 1e-3, 31):
        if np.min(np.abs(E - e)) < 1e-6:
            continue
        _, dw = oracle.corner_weights(e, E, F)
        ref = 24.0 * F * cross_section_linear_integrals(e, E)
        np.testing.assert_allclose(dw, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("trial", range(8))
def test_weight_derivative_matches_finite_difference(trial):
    rng = np.random.default_rng(300 + trial)
    e = random_sorted_energies(rng)
    h = 1e-6
    for E in np.linspace(e[0] + 0.01, e[3] - 0.01, 40):
        if np.min(np.abs(E - e)) < 10 * h:
            continue
        wp, _ = oracle.corner_weights(e, E + h, F)
        wm, _ = oracle.corner_weights(e, E - h, F)
        _, dw = oracle.corner_weights(e, E, F)
        np.testing.assert_allclose(dw, (wp - wm) / (2 * h), rtol=1e-6, atol=1e-9)


def bloechl_total_dos(e, E, vt_vg):
    """Closed-form DOS of one tetrahedron (Bloechl et al., PRB 49, 16223)."""
    E1, E2, E3, E4 = e
    if E <= E1 or E >= E4:
        return 0.0
    if E <= E2:
        return vt_vg * 3 * (E - E1) ** 2 / ((E2 - E1) * (E3 - E1) * (E4 - E1))
    if E <= E3:
        E21, E31, E41, E32, E42 = E2 - E1, E3 - E1, E4 - E1, E3 - E2, E4 - E2
        return vt_vg / (E31 * E41) * (3 * E21 + 6 * (E - E2) - 3 * (E31 + E42) * (E - E2) ** 2 / (E32 * E42))
    return vt_vg * 3 * (E4 - E) ** 2 / ((E4 - E1) * (E4 - E2) * (E4 - E3))


@pytest.mark.parametrize("trial", range(10))
def test_sum_of_corner_derivatives_is_bloechl_total_dos(trial):
    rng = np.random.default_rng(400 + trial)
    e = random_sorted_energies(rng)
    for E in np.linspace(e[0] - 0.05, e[3] + 0.05, 57):
        _, dw = oracle.corner_weights(e, E, F)
        assert abs(dw.sum() - bloechl_total_dos(e, E, 4 * F)) < 1e-12 * max(1.0, abs(dw.sum()))


@pytest.mark.parametrize("deg", [None, "12", "23", "34"])
def test_continuity_and_limits(deg):
    rng = np.random.default_rng(7)
    for _ in range(10):
        e = random_sorted_energies(rng, deg)
        for Eb in e:
            wl, dl = oracle.corner_weights(e, Eb - 1e-10, F)
            wr, dr = oracle.corner_weights(e, Eb + 1e-10, F)
            assert np.all(np.isfinite(wl)) and np.all(np.isfinite(dl))
            np.testing.assert_allclose(wl, wr, atol=1e-8)
        w0, d0 = oracle.corner_weights(e, e[0], F)
        assert np.all(w0 == 0) and np.all(d0 == 0)
        w4, d4 = oracle.corner_weights(e, e[3], F)
        assert np.all(w4 == F) and np.all(d4 == 0)
        # derivative continuity where both sides are in the interior
        for Eb in (e[1], e[2]):
            if e[0] < Eb < e[3] and len(set(e)) == 4:
                _, dl = oracle.corner_weights(e, Eb - 1e-9, F)
                _, dr = oracle.corner_weights(e, Eb + 1e-9, F)
                np.testing.assert_allclose(dl, dr, rtol=1e-6, atol=1e-8)


def test_all_degenerate_tetrahedron_is_a_step():
    e = np.array([0.3, 0.3, 0.3, 0.3])
    w, dw = oracle.corner_weights(e, 0.2, F)
    assert np.all(w == 0)
    w, dw = oracle.corner_weights(e, 0.4, F)
    assert np.all(w == F) and np.all(dw == 0)


@pytest.mark.parametrize("trial", range(6))
def test_subdivision_invariance_linear_data(trial):
    """Splitting a tetrahedron into 8 sub-tetrahedra with linearly interpolated
    energies and orbital weights leaves the weighted DOS unchanged (the method
    is exact for linear data)."""
    rng = np.random.default_rng(500 + trial)
    e = rng.normal(0, 1, 4)
    b = rng.uniform(0, 1, 4)
    V = np.eye(4)  # corners in barycentric coordinates
    mid = {}
    for i, j in itertools.combinations(range(4), 2):
        mid[(i, j)] = 0.5 * (V[i] + V[j])
    m = lambda i, j: mid[(min(i, j), max(i, j))]
    subs = [
        [V[0], m(0, 1), m(0, 2), m(0, 3)], [V[1], m(0, 1), m(1, 2), m(1, 3)],
        [V[2], m(0, 2), m(1, 2), m(2, 3)], [V[3], m(0, 3), m(1, 3), m(2, 3)],
        [m(0, 1), m(0, 2), m(0, 3), m(1, 3)], [m(0, 1), m(0, 2), m(1, 2), m(1, 3)],
        [m(0, 2), m(0, 3), m(1, 3), m(2, 3)], [m(0, 2), m(1, 2), m(1, 3), m(2, 3)],
    ]

    def contrib(ev, bv, f, E):
        order = np.argsort(ev, kind="stable")
        _, dw = oracle.corner_weights(ev[order], E, f)
        return float(np.dot(bv[order], dw)), np.array([
            oracle.corner_weights(ev[order], E, f)[0]]).ravel(), order

    for E in np.linspace(e.min() + 0.01, e.max() - 0.01, 17):
        whole = contrib(e, b, F, E)[0]
        parts = 0.0
        for S in subs:
            S = np.array(S)
            parts += contrib(S @ e, S @ b, F / 8.0, E)[0]
        assert abs(whole - parts) < 1e-11 * max(1.0, abs(whole))


@pytest.mark.parametrize("trial", range(6))
def test_weight_moments_match_finite_difference(trial):
    rng = np.random.default_rng(600 + trial)
    e = random_sorted_energies(rng)
    h = 1e-6
    for E in np.linspace(e[0] + 0.02, e[3] - 0.02, 15):
        if np.min(np.abs(E - e)) < 1e-3:
            continue
        M = oracle.weight_moments(e, E, F)
        for i in range(4):
            ep = e.copy(); ep[i] += h
            em = e.copy(); em[i] -= h
            wp, _ = oracle.corner_weights(np.sort(ep), E, F)
            wm, _ = oracle.corner_weights(np.sort(em), E, F)
            np.testing.assert_allclose(-M[:, i], (wp - wm) / (2 * h), rtol=1e-5, atol=1e-9)
        # shift invariance: sum_i dw_l/de_i = -dw_l/dE
        _, dw = oracle.corner_weights(e, E, F)
        np.testing.assert_allclose(M.sum(1), dw, rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------- whole grids
def test_table_one_partitions_the_cube():
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, (4000, 3))
    count = np.zeros(len(pts), int)
    for tet in TABLE_I:
        P = np.array([corner_offset(c) for c in tet])
        T = (P[:3] - P[3]).T
        lam = np.linalg.solve(T, (pts - P[3]).T).T
        lam = np.concatenate([lam, 1 - lam.sum(1, keepdims=True)], 1)
        count += np.all(lam >= -1e-12, axis=1)
    assert np.all(count == 1)


def small_problem(seed=3, n=(3, 2, 4), nb=2, norb=3):
    n1, n2, n3 = n
    rng = np.random.default_rng(seed)
    nk = n1 * n2 * n3
    eps = np.sort(rng.normal(0, 1, (nk, nb)), axis=1)
    w = rng.uniform(0.05, 1, (nk, nb, norb))
    w /= w.sum(2, keepdims=True)
    return n1, n2, n3, eps, w


def test_translation_invariance_of_grid_origin():
    n1, n2, n3, eps, w = small_problem()
    E = np.linspace(-2.5, 2.5, 41)
    d0 = oracle.dos(eps, w, n1, n2, n3, E)
    sh = lambda a: np.roll(a.reshape(n3, n2, n1, *a.shape[1:]), (1, -1, 2), axis=(0, 1, 2)).reshape(a.shape)
    d1 = oracle.dos(sh(eps), sh(w), n1, n2, n3, E)
    np.testing.assert_allclose(d0, d1, rtol=1e-12, atol=1e-14)


def test_bin_mode_sum_rule_and_total():
    model = tbgen.tb_model(5, n_orb=4)
    n1 = n2 = n3 = 4
    eps, w = oracle.eig(model, n1, n2, n3)
    edges = np.linspace(eps.min() - 0.1, eps.max() + 0.1, 61)
    d = oracle.dos(eps, w, n1, n2, n3, edges, mode="bin")
    widths = np.diff(edges)
    np.testing.assert_allclose((d * widths).sum(1), 1.0, rtol=0, atol=1e-12)
    dtot = oracle.dos(eps, np.ones((eps.shape[0], eps.shape[1], 1)), n1, n2, n3, edges, mode="bin")
    np.testing.assert_allclose(d.sum(0), dtot[0], rtol=1e-12, atol=1e-12)


def test_point_mode_total_is_sum_over_orbitals():
    model = tbgen.tb_model(6, n_orb=3)
    eps, w = oracle.eig(model, 3, 3, 3)
    E = np.linspace(eps.min(), eps.max(), 37)
    d = oracle.dos(eps, w, 3, 3, 3, E)
    dtot = oracle.dos(eps, np.ones((eps.shape[0], eps.shape[1], 1)), 3, 3, 3, E)
    np.testing.assert_allclose(d.sum(0), dtot[0], rtol=1e-11, atol=1e-12)


def test_thread_count_does_not_change_result_beyond_rounding():
    n1, n2, n3, eps, w = small_problem(n=(4, 4, 6))
    E = np.linspace(-2, 2, 33)
    d1 = oracle.dos(eps, w, n1, n2, n3, E, nthreads=1)
    d3 = oracle.dos(eps, w, n1, n2, n3, E, nthreads=3)
    np.testing.assert_allclose(d1, d3, rtol=1e-12, atol=1e-15)


def test_z_range_partition_adds_up():
    n1, n2, n3, eps, w = small_problem(n=(3, 3, 5))
    E = np.linspace(-2, 2, 21)
    full = oracle.dos(eps, w, n1, n2, n3, E)
    parts = sum(oracle.dos(eps, w, n1, n2, n3, E, z_range=(a, b)) for a, b in [(0, 2), (2, 3), (3, 5)])
    np.testing.assert_allclose(full, parts, rtol=1e-12, atol=1e-15)


def test_monte_carlo_histogram_of_linear_interpolant():
    """Bin DOS equals the histogram of the piecewise-linear interpolant sampled
    uniformly over each cube (tetrahedron located from Table I)."""
    n1, n2, n3, eps, w = small_problem(seed=11, n=(2, 2, 2), nb=1, norb=2)
    rng = np.random.default_rng(99)
    edges = np.linspace(eps.min() - 0.05, eps.max() + 0.05, 13)
    hist = np.zeros((2, len(edges) - 1))
    tets = [np.array([corner_offset(c) for c in tet]) for tet in TABLE_I]
    inv = [np.linalg.inv((P[:3] - P[3]).T) for P in tets]
    ns = 400_000
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                pts = rng.uniform(0, 1, (ns, 3))
                for P, Ti, tet in zip(tets, inv, TABLE_I):
                    lam = (Ti @ (pts - P[3]).T).T
                    lam = np.concatenate([lam, 1 - lam.sum(1, keepdims=True)], 1)
                    inside = np.all(lam >= 0, axis=1)
                    L = lam[inside]
                    ks = []
                    for c in tet:
                        o = corner_offset(c).astype(int)
                        ks.append(((x + o[0]) % n1) + n1 * (((y + o[1]) % n2) + n2 * ((z + o[2]) % n3)))
                    ev = L @ eps[ks, 0]
                    for s in range(2):
                        bv = L @ w[ks, 0, s]
                        h, _ = np.histogram(ev, bins=edges, weights=bv)
                        hist[s] += h
    hist /= (ns * n1 * n2 * n3) * np.diff(edges)
    d = oracle.dos(eps, w, n1, n2, n3, edges, mode="bin")
    assert np.max(np.abs(hist - d)) < 0.02 * np.max(d)


def sc_exact_dos(E, t=1.0):
    """Exact DOS of eps = -2t(cos kx + cos ky + cos kz), from the square-lattice
    DOS (complete elliptic integral) averaged over k_z."""
    from scipy.integrate import quad
    from scipy.special import ellipk

    def rho2(e):
        if abs(e) >= 4 * t:
            return 0.0
        m = 1.0 - (e / (4 * t)) ** 2
        return ellipk(m) / (2 * np.pi ** 2 * t)

    val, _ = quad(lambda kz: rho2(E + 2 * t * np.cos(kz)), 0, np.pi, limit=200)
    return val / np.pi


def sc_eps(n):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    return (-2 * (np.cos(k * x) + np.cos(k * y) + np.cos(k * z))).reshape(-1, 1)


def test_simple_cubic_particle_hole_symmetry():
    n = 8
    eps = sc_eps(n)
    w = np.ones((n ** 3, 1, 1))
    E = np.linspace(-6.5, 6.5, 131)
    d = oracle.dos(eps, w, n, n, n, E)
    np.testing.assert_allclose(d[0], d[0][::-1], rtol=1e-10, atol=1e-12)


def test_simple_cubic_converges_to_analytic_dos():
    E = np.array([-5.0, -3.0, -1.0, 1.0, 3.0, 5.0])
    exact = np.array([sc_exact_dos(x) for x in E])
    errs = []
    for n in (12, 24):
        eps = sc_eps(n)
        d = oracle.dos(eps, np.ones((n ** 3, 1, 1)), n, n, n, E)[0]
        errs.append(np.max(np.abs(d - exact)))
    assert errs[1] < 0.01 * exact.max()
    assert errs[0] / errs[1] > 2.5  # second order in the grid spacing


def test_eig_matches_simple_cubic_dispersion_and_is_orthonormal():
    eps, w, V = oracle.eig(tbgen.sc_model(), 5, 5, 5, return_vectors=True)
    np.testing.assert_allclose(eps, sc_eps(5), atol=1e-13)
    model = tbgen.tb_model(2)
    H = oracle.hamiltonian(model, 3, 2, 2)
    ev, w, V = oracle.eig(model, 3, 2, 2, return_vectors=True)
    np.testing.assert_allclose(H @ V, V * ev[:, None, :], atol=1e-12)
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-12)   # sum over bands
    np.testing.assert_allclose(w.sum(2), 1.0, atol=1e-12)   # sum over orbitals
    np.testing.assert_allclose(H, np.conj(np.transpose(H, (0, 2, 1))), atol=0)


def test_bin_gradient_matches_finite_difference():
    n1, n2, n3, eps, w = small_problem(seed=21, n=(2, 2, 3), nb=2, norb=2)
    edges = np.linspace(eps.min() - 0.2, eps.max() + 0.2, 9)
    g = np.random.default_rng(4).normal(0, 1, (2, 8))
    geps, gw = oracle.dos_bin_grad(eps, w, n1, n2, n3, edges, g)
    L = lambda e_, w_: float((g * oracle.dos(e_, w_, n1, n2, n3, edges, mode="bin")).sum())
    h = 1e-6
    for idx in [(0, 0), (3, 1), (7, 0), (11, 1)]:
        ep = eps.copy(); ep[idx] += h
        em = eps.copy(); em[idx] -= h
        fd = (L(ep, w) - L(em, w)) / (2 * h)
        assert abs(fd - geps[idx]) < 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (5, 1, 1), (9, 0, 1)]:
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        fd = (L(eps, wp) - L(eps, wm)) / (2 * h)
        assert abs(fd - gw[idx]) < 1e-7 * max(1.0, abs(fd))


def test_eig_backward_matches_finite_difference_of_fp64_chain():
    model = tbgen.tb_model(8, n_orb=4)
    n1, n2, n3 = 3, 3, 2
    eps, w = oracle.eig(model, n1, n2, n3)
    edges = np.linspace(eps.min() - 0.3, eps.max() + 0.3, 11)
    g = np.random.default_rng(5).normal(0, 1, (4, 10))

    def loss(p):
        m = oracle.params_to_model(p, model)
        e_, w_ = oracle.eig(m, n1, n2, n3)
        return float((g * oracle.dos(e_, w_, n1, n2, n3, edges, mode="bin")).sum())

    geps, gw = oracle.dos_bin_grad(eps, w, n1, n2, n3, edges, g)
    grad = oracle.eig_backward(model, n1, n2, n3, geps, gw)
    p0 = oracle.model_to_params(model)
    assert grad.shape == p0.shape
    h = 1e-6
    for i in [0, 3, 5, 20, 41, 77, 130, 200, 227]:
        pp = p0.copy(); pp[i] += h
        pm = p0.copy(); pm[i] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - grad[i]) < 2e-5 * max(1.0, abs(fd)), (i, fd, grad[i])


# ---------------------------------------------------------------- integrated occupation n_s(E)
def test_integrated_occupation_limits():
    """Below every band n_s(E) = 0; above every band each k-point is a corner
    of 24 tetrahedra of weight V_T/(4 V_G) = 1/(24 N_k), so n_s is the plain
    k-average of sum_n b_sn (computed here directly from the weights)."""
    n1, n2, n3, eps, w = small_problem(seed=5, n=(3, 4, 2), nb=3, norb=2)
    E = np.array([eps.min() - 1.0, eps.max() + 1.0])
    n = oracle.dos(eps, w, n1, n2, n3, E, mode="integrated")
    np.testing.assert_array_equal(n[:, 0], 0.0)
    np.testing.assert_allclose(n[:, 1], w.sum(axis=1).mean(axis=0), rtol=1e-12)


def test_integrated_occupation_monte_carlo_of_linear_interpolant():
    """n_s(E) equals the integral of the linearly interpolated weight b_s over
    the region where the linearly interpolated band lies below E (uniform
    samples in every cube, tetrahedron located from Table I)."""
    n1, n2, n3, eps, w = small_problem(seed=12, n=(2, 2, 2), nb=1, norb=2)
    rng = np.random.default_rng(7)
    E = np.linspace(eps.min() + 0.1, eps.max() - 0.1, 7)
    acc = np.zeros((2, len(E)))
    tets = [np.array([corner_offset(c) for c in tet]) for tet in TABLE_I]
    inv = [np.linalg.inv((P[:3] - P[3]).T) for P in tets]
    ns = 300_000
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                pts = rng.uniform(0, 1, (ns, 3))
                for P, Ti, tet in zip(tets, inv, TABLE_I):
                    lam = (Ti @ (pts - P[3]).T).T
                    lam = np.concatenate([lam, 1 - lam.sum(1, keepdims=True)], 1)
                    L = lam[np.all(lam >= 0, axis=1)]
                    ks = []
                    for c in tet:
                        o = corner_offset(c).astype(int)
                        ks.append(((x + o[0]) % n1) + n1 * (((y + o[1]) % n2) + n2 * ((z + o[2]) % n3)))
                    ev = L @ eps[ks, 0]
                    for s in range(2):
                        bv = L @ w[ks, 0, s]
                        acc[s] += [(bv * (ev < e)).sum() for e in E]
    acc /= ns * n1 * n2 * n3
    n = oracle.dos(eps, w, n1, n2, n3, E, mode="integrated")
    assert np.max(np.abs(acc - n)) < 0.01 * np.max(n)


def test_simple_cubic_half_filling():
    """eps(k + (pi,pi,pi)) = -eps(k) on an even grid maps the states below E
    onto those above -E, so N(0) = 1/2 exactly and the Fermi level of half
    filling is 0."""
    n = 8
    eps = sc_eps(n)
    N = oracle.dos(eps, np.ones((n ** 3, 1, 1)), n, n, n, np.array([0.0]), mode="integrated")
    assert abs(N[0, 0] - 0.5) < 1e-12
    assert abs(oracle.fermi_level(eps, n, n, n, 0.5)) < 1e-9


def test_fermi_level_is_the_root_of_the_count():
    n1, n2, n3, eps, w = small_problem(seed=8, n=(4, 3, 3), nb=3, norb=2)
    for ne in (0.4, 1.0, 2.3):
        ef = oracle.fermi_level(eps, n1, n2, n3, ne)
        N = oracle.dos(eps, np.ones(w.shape[:2] + (1,)), n1, n2, n3, np.array([ef - 1e-6, ef, ef + 1e-6]),
                       mode="integrated")[0]
        assert N[0] <= ne + 1e-9 and N[2] >= ne - 1e-9
        assert abs(N[1] - ne) < 1e-6


# ---------------------------------------------------------------- spectral Lindhard function
def test_pair_bands_spectral_function_is_odd_at_q0():
    """At q = 0 the pairs (n, m) and (m, n) have opposite energies and
    opposite weights, so S(-w) = -S(w) point by point."""
    n1, n2, n3, eps, _ = small_problem(seed=4, n=(4, 3, 3), nb=3, norb=1)
    d, w = oracle.pair_bands(eps, n1, n2, n3, (0, 0, 0), kT=0.2, mu=0.1)
    E = np.linspace(-3, 3, 61)
    s = oracle.dos(d, w, n1, n2, n3, E)[0]
    np.testing.assert_allclose(s, -s[::-1], atol=1e-12 * np.abs(s).max())


@pytest.mark.parametrize("q", [(0, 0, 0), (1, 0, 0), (2, 1, 1)])
def test_pair_bands_spectral_weight_integrates_to_zero(q):
    """The integral of S over all energies is the grid average of
    sum_{n,m} [f_n(k) - f_m(k+q)] = nb (<f>_k - <f>_{k+q}) = 0 on a periodic
    grid (bin mode integrates exactly); the positive part is checked against a
    direct sum of the occupation differences."""
    n1, n2, n3, eps, _ = small_problem(seed=6, n=(4, 4, 3), nb=2, norb=1)
    d, w = oracle.pair_bands(eps, n1, n2, n3, q, kT=0.3, mu=0.0)
    edges = np.linspace(d.min() - 0.1, d.max() + 0.1, 41)
    s = oracle.dos(d, w, n1, n2, n3, edges, mode="bin")[0]
    total = (s * np.diff(edges)).sum()
    assert abs(total) < 1e-12
    # the definition, term by term, for one k-point and pair
    f = oracle.fermi_dirac
    k = 5
    z, rem = divmod(k, n1 * n2)
    y, x = divmod(rem, n1)
    kq = ((x + q[0]) % n1) + n1 * (((y + q[1]) % n2) + n2 * ((z + q[2]) % n3))
    assert d[k, 0 * 2 + 1] == eps[kq, 1] - eps[k, 0]
    assert abs(w[k, 0 * 2 + 1, 0] - (f(eps[k, 0], 0.3, 0.0) - f(eps[kq, 1], 0.3, 0.0))) < 1e-15


# ---------------------------------------------------------------- Fermi-Dirac occupation (pair bands)
def test_fermi_dirac_identities():
    """f(mu) = 1/2, f(mu + x) + f(mu - x) = 1, f(mu + kT) = 1/(1 + e), limits
    0 and 1, and f decreasing: the properties that fix the function."""
    f = oracle.fermi_dirac
    kT, mu = 0.07, 0.3
    assert f(mu, kT, mu) == 0.5
    x = np.linspace(-2, 2, 81)
    np.testing.assert_allclose(f(mu + x, kT, mu) + f(mu - x, kT, mu), 1.0, atol=1e-15)
    assert abs(f(mu + kT, kT, mu) - 1.0 / (1.0 + np.e)) < 1e-15
    assert f(mu + 50, kT, mu) < 1e-300 and f(mu - 50, kT, mu) == 1.0
    assert np.all(np.diff(f(mu + x, kT, mu)) < 0)


def twisted_model(model, q, n):
    """The model whose H at grid point k is H(k + 2 pi q / n): every hopping
    t(R) picks up the phase e^{2 pi i q.R / n}, so diagonalising it on the
    grid gives the bands at k + q without shifting any index."""
    qf = np.asarray(q, np.float64) / np.asarray(n, np.float64)
    ph = np.exp(2j * np.pi * (model["R"].astype(np.float64) @ qf))
    return {"onsite": model["onsite"], "R": model["R"], "t": model["t"] * ph[:, None, None]}


def test_pair_bands_shift_k_plus_q_and_sign():
    """pair_bands at momentum q: the energy is e_m(k + q) - e_n(k) and the
    weight f(e_n(k)) - f(e_m(k + q)), with the bands at k + q from a separate
    diagonalisation of H(k + q) (twisted hoppings); the model has no
    time-reversal symmetry, so k - q would give other values. For w above the
    largest spread of the transition energy inside any tetrahedron every
    tetrahedron that contributes has positive transition energy at all
    corners, hence non-negative weight: S(q, w) >= 0 there (and S <= 0 below
    minus that spread)."""
    n = (5, 4, 3)
    q = (2, 1, 1)
    model = tbgen.tb_model(7, n_orb=3)
    eps, _ = oracle.eig(model, *n)
    epq, _ = oracle.eig(twisted_model(model, q, n), *n)
    kT, mu = 0.2, float(np.median(eps))
    d, w = oracle.pair_bands(eps, *n, q, kT, mu)
    nb = eps.shape[1]
    for nn in range(nb):
        for m in range(nb):
            np.testing.assert_allclose(d[:, nn * nb + m], epq[:, m] - eps[:, nn], atol=1e-11)
            ref = 0.5 * (np.tanh(0.5 * (epq[:, m] - mu) / kT) - np.tanh(0.5 * (eps[:, nn] - mu) / kT))
            np.testing.assert_allclose(w[:, nn * nb + m, 0], ref, atol=1e-12)
    dm, _ = oracle.pair_bands(eps, *n, tuple(-v for v in q), kT, mu)
    assert np.max(np.abs(dm - d)) > 1e-3   # k - q is distinguishable
    # sign: spread of the transition energy over each tetrahedron's corners
    spread = 0.0
    n1, n2, n3 = n
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                for t in oracle.table_i() - 1:
                    ks = [((x + (c & 1)) % n1) + n1 * (((y + ((c >> 1) & 1)) % n2) + n2 * ((z + (c >> 2)) % n3))
                          for c in t]
                    spread = max(spread, float(np.max(np.ptp(d[ks], axis=0))))
    E = np.linspace(spread + 1e-6, d.max() + 0.1, 40)
    s = oracle.dos(d, w, *n, E)[0]
    assert np.all(s >= -1e-14) and s.max() > 0
    s_neg = oracle.dos(d, w, *n, -E)[0]
    assert np.all(s_neg <= 1e-14)


# ---------------------------------------------------------------- spectral function at T = 0
def mc_t0_histogram(a, c, edges, n_samples, seed):
    """Monte-Carlo estimate of the bin-averaged T = 0 contribution of one
    tetrahedron (units of V_T/V_G): uniform points (Dirichlet(1,1,1,1)
    barycentric coordinates), fields a, c interpolated linearly, occupation
    difference +1 on {a < 0 < c}, -1 on {c < 0 < a}, histogram of c - a."""
    rng = np.random.default_rng(seed)
    lam = rng.dirichlet(np.ones(4), size=n_samples)
    A = lam @ a
    C = lam @ c
    wgt = ((A < 0) & (C > 0)).astype(float) - ((A > 0) & (C < 0)).astype(float)
    h, _ = np.histogram(C - A, bins=edges, weights=wgt)
    h2, _ = np.histogram(C - A, bins=edges, weights=wgt * wgt)
    width = np.diff(edges)
    return h / n_samples / width, np.sqrt(h2) / n_samples / width


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_t0_tetra_against_monte_carlo(seed):
    """Clipping by both step functions, for random corner values of mixed
    sign: bin averages against a Monte-Carlo histogram (5 sigma)."""
    rng = np.random.default_rng(100 + seed)
    a = rng.normal(0, 1, 4)
    c = rng.normal(0.2, 1, 4)
    d = c - a
    edges = np.linspace(d.min() - 0.05, d.max() + 0.05, 17)
    s = oracle.spectral_t0_tetra(a, c, edges, mode="bin")
    mc, sig = mc_t0_histogram(a, c, edges, 2_000_000, seed)
    assert np.all(np.abs(s - mc) <= 5 * sig + 1e-3), (s, mc, sig)


def test_t0_tetra_unclipped_is_the_tetrahedron_density():
    """All corners occupied in band n and empty in band m: no clipping, the
    distribution of the transition energy over the whole tetrahedron, i.e.
    the total of the Sec. II.C corner weight derivatives (oracle.corner_weights,
    pinned above) divided by V_T/V_G."""
    a = np.array([-1.0, -0.4, -0.7, -0.2])
    c = np.array([0.3, 0.9, 0.35, 1.4])
    d = np.sort(c - a)
    E = np.linspace(d[0] - 0.1, d[3] + 0.1, 57)
    s = oracle.spectral_t0_tetra(a, c, E)
    f = 0.25
    ref = np.array([oracle.corner_weights(d, x, f)[1].sum() for x in E])
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-12)
    # and band n empty everywhere: nothing
    assert np.all(oracle.spectral_t0_tetra(-a, c, E) == 0.0)


@pytest.mark.parametrize("inside", [1, 3])
def test_t0_tetra_clipped_volume_closed_form(inside):
    """Band m empty at every corner, band n occupied at `inside` corners: the
    total weight (bin mode over every transition energy) is the volume of the
    occupied part of the tetrahedron, a corner tetrahedron with edge ratios
    -a_i / (a_j - a_i) (one corner occupied) or the complement of one (three)."""
    a = np.array([-0.6, 0.5, 0.8, 1.1]) if inside == 1 else np.array([-0.6, -0.5, -0.8, 1.1])
    c = np.array([0.4, 0.9, 1.3, 2.0])
    edges = np.linspace(-1, 4, 6)
    total = (oracle.spectral_t0_tetra(a, c, edges, mode="bin") * np.diff(edges)).sum()
    if inside == 1:
        ref = np.prod([-a[0] / (a[j] - a[0]) for j in (1, 2, 3)])
    else:
        ref = 1.0 - np.prod([a[3] / (a[3] - a[j]) for j in (0, 1, 2)])
    assert abs(total - ref) < 1e-13


def test_t0_spectral_sign_sum_rule_and_symmetry():
    """On a periodic grid with a model without time-reversal symmetry:
    S(q, w) >= 0 for w > 0 and <= 0 for w < 0 (the occupation difference is
    +1 only where the transition energy is positive); the total weight is
    zero (the occupied volume of band n and of the shifted band m are equal);
    S(-q, -w) = -S(q, w) (pairs (n, m) at k and (m, n) at k + q); and the
    bands at k + q taken from the twisted model give the same S."""
    n = (4, 3, 3)
    q = (1, 2, 1)
    model = tbgen.tb_model(9, n_orb=3)
    eps, _ = oracle.eig(model, *n)
    mu = float(np.median(eps))
    edges = np.linspace(-12, 12, 97)
    s = oracle.spectral_t0(eps, *n, q, mu, edges, mode="bin")
    mid = 0.5 * (edges[1:] + edges[:-1])
    assert np.all(s[mid > 0.13] >= -1e-14) and np.all(s[mid < -0.13] <= 1e-14)
    assert abs((s * np.diff(edges)).sum()) < 1e-12
    sm = oracle.spectral_t0(eps, *n, tuple(-v for v in q), mu, -edges[::-1], mode="bin")
    np.testing.assert_allclose(sm[::-1], -s, atol=1e-13)
    epq, _ = oracle.eig(twisted_model(model, q, n), *n)
    st = oracle.spectral_t0(eps, *n, (0, 0, 0), mu, edges, mode="bin", eps_kq=epq)
    np.testing.assert_allclose(st, s, atol=1e-11)
    sneg = oracle.spectral_t0(eps, *n, tuple(-v for v in q), mu, edges, mode="bin")
    assert np.max(np.abs(sneg - s)) > 1e-4 * np.max(np.abs(s))


def test_t0_spectral_grid_against_monte_carlo():
    """Whole-grid bin averages against a Monte-Carlo histogram over all
    tetrahedra and band pairs (a tiny grid, 2 bands)."""
    n = (3, 2, 2)
    n1, n2, n3 = n
    rng = np.random.default_rng(21)
    eps = np.sort(rng.normal(0, 1, (n1 * n2 * n3, 2)), axis=1)
    q, mu = (1, 1, 0), 0.1
    edges = np.linspace(-5, 5, 21)
    s = oracle.spectral_t0(eps, *n, q, mu, edges, mode="bin")
    acc = np.zeros(len(edges) - 1)
    var = np.zeros(len(edges) - 1)
    ntet = 6 * n1 * n2 * n3
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                for t in oracle.table_i() - 1:
                    kk, kq = [], []
                    for c in t:
                        xx, yy, zz = (x + (c & 1)) % n1, (y + ((c >> 1) & 1)) % n2, (z + (c >> 2)) % n3
                        kk.append(xx + n1 * (yy + n2 * zz))
                        kq.append((xx + q[0]) % n1 + n1 * (((yy + q[1]) % n2) + n2 * ((zz + q[2]) % n3)))
                    for nn in range(2):
                        for m in range(2):
                            h, sg = mc_t0_histogram(eps[kk, nn] - mu, eps[kq, m] - mu, edges, 40_000,
                                                    len(kk) + 7 * nn + 3 * m + 31 * x + 17 * y + 5 * z)
                            acc += h / ntet
                            var += (sg / ntet) ** 2
    assert np.all(np.abs(s - acc) <= 5 * np.sqrt(var) + 1e-4), np.max(np.abs(s - acc))


# ---- real part of the T = 0 susceptibility --------------------------------

def linear_density(d, x):
    """Normalised density of a linear function with corner values d over a
    tetrahedron, read from the oracle's T = 0 tetrahedron in a configuration
    where the +1 region is the whole tetrahedron (a < 0 < c at every corner;
    that density is pinned above by Monte-Carlo histograms)."""
    a = -10.0 * np.ones(4)
    c = np.asarray(d, float) + 100.0
    return float(oracle.spectral_t0_tetra(a, c, np.atleast_1d(x) + 110.0)[0])


def principal_value_by_quadrature(d, w):
    """P int g(x) / (w - x) dx by adaptive quadrature (QUADPACK), split at the
    corner values; the piece holding w with the Cauchy weight."""
    from scipy import integrate
    knots = sorted(set(float(v) for v in d))
    tot = 0.0
    for lo, hi in zip(knots[:-1], knots[1:]):
        if lo < w < hi:
            v, _ = integrate.quad(lambda x: linear_density(d, x), lo, hi, weight="cauchy", wvar=w,
                                  limit=500, epsabs=1e-14, epsrel=1e-12)
            tot -= v
        else:
            v, _ = integrate.quad(lambda x: linear_density(d, x) / (w - x), lo, hi, limit=500,
                                  epsabs=1e-14, epsrel=1e-12)
            tot += v
    return tot


@pytest.mark.parametrize("trial", range(12))
def test_t0_inverse_average_against_quadrature(trial):
    """P<1/(w - D)> over a tetrahedron (closed-form pieces near w, moment
    series far from it) against adaptive quadrature of the density, for
    energies inside each piece, near the knots, beside and far outside the
    support, with nearly coincident and coincident corner values."""
    rng = np.random.default_rng(100 + trial)
    d = np.sort(rng.normal(0, 1, 4))
    if trial % 4 == 1:
        d[1] = d[0] + 1e-7
    if trial % 4 == 2:
        d[2] = d[1]
    if trial % 4 == 3:
        d[3] = d[2] + 1e-9
    ws = list(rng.uniform(d[0] - 1, d[3] + 1, 3)) + [0.5 * (d[0] + d[3]), d[1] + 1e-3, d[2] - 1e-3,
                                                       d[3] + 5.0, d[0] - 30.0]
    for w in ws:
        r = oracle.t0_inverse_average(d, w)
        ref = principal_value_by_quadrature(d, w)
        assert abs(r - ref) <= 1e-8 * abs(ref) + 1e-12, (d, w, r, ref)


@pytest.mark.parametrize("w", [3.5, 6.0, -4.0])
def test_t0_inverse_average_far_field_monte_carlo(w):
    """Outside the range of D the integrand is smooth: the plain Monte-Carlo
    mean of 1/(w - D) over uniform points of the tetrahedron."""
    rng = np.random.default_rng(7)
    d = rng.normal(0, 1, 4)
    lam = rng.dirichlet(np.ones(4), 1_000_000)
    vals = 1.0 / (w - lam @ d)
    mc, se = vals.mean(), vals.std() / np.sqrt(len(vals))
    assert abs(oracle.t0_inverse_average(d, w) - mc) < 5 * se


def test_t0_inverse_average_flat_knots_and_continuity():
    """A flat D gives 1/(w - d); at a corner value the result is finite and
    equals the limit from both sides (the logarithms of the two pieces that
    meet there cancel); corner order does not matter."""
    assert oracle.t0_inverse_average([0.3] * 4, 1.3) == pytest.approx(1.0)
    d = np.array([-0.7, 0.1, 0.35, 1.2])
    for k in d:
        r = oracle.t0_inverse_average(d, k)
        side = 0.5 * (oracle.t0_inverse_average(d, k + 1e-9) + oracle.t0_inverse_average(d, k - 1e-9))
        assert np.isfinite(r) and abs(r - side) < 1e-7
    assert oracle.t0_inverse_average(d[::-1].copy(), 0.2) == pytest.approx(oracle.t0_inverse_average(d, 0.2),
                                                                          rel=1e-14)


def test_chi0_real_is_the_hilbert_transform_of_s():
    """Kramers-Kronig on the grid: Re chi0(q, w) = P int S(q, w') / (w - w') dw',
    with S from the oracle's exact bin averages on 6000 bins (the transform of
    a piecewise-constant S is a sum of logarithms); agreement to the binning
    error. Also Re chi0(-q, -w) = Re chi0(q, w) (S is odd under that map),
    and Re chi0 -> M1 / w^2 for large w, M1 = int w' S(w') dw' (S has zero
    total weight)."""
    n = (5, 4, 4)
    model = tbgen.tb_model(9, n_orb=3)
    eps, _ = oracle.eig(model, *n)
    mu = float(np.median(eps))
    q = (2, 1, 0)
    span = float(eps.max() - eps.min()) + 0.5
    edges = np.linspace(-span, span, 6001)
    s = oracle.spectral_t0(eps, *n, q, mu, edges, mode="bin")
    w = np.array([-2.3, -0.6, 0.05, 0.9, 2.2, 4.5])
    r = oracle.chi0_real_t0(eps, *n, q, mu, w)
    lo, hi = edges[:-1], edges[1:]
    kk = np.array([np.sum(s * np.log(np.abs((x - lo) / (x - hi)))) for x in w])
    assert np.max(np.abs(r - kk)) < 2e-3 * np.max(np.abs(r)), (r, kk)
    rm = oracle.chi0_real_t0(eps, *n, tuple(-v for v in q), mu, -w)
    np.testing.assert_allclose(rm, r, rtol=0, atol=1e-12 * np.max(np.abs(r)))
    big = np.array([400.0, 800.0])
    m1 = float(np.sum(s * 0.5 * (lo + hi) * (hi - lo)))
    rb = oracle.chi0_real_t0(eps, *n, q, mu, big)
    np.testing.assert_allclose(rb * big ** 2, m1, rtol=2e-2)


# ---- corner-permutation invariance ------------------------------------------

def grid_map(a, n, how):
    """Relabel the k-grid of per-point data a (nk, ...) in x-fastest order:
    "swap_xz" k' = (z, y, x) (needs n1 == n3), "invert" k' = -k (periodic)."""
    n1, n2, n3 = n
    A = a.reshape((n3, n2, n1) + a.shape[1:])          # [z][y][x]
    if how == "swap_xz":
        B = np.swapaxes(A, 0, 2)
    else:
        B = np.roll(np.flip(A, axis=(0, 1, 2)), 1, axis=(0, 1, 2))
    return np.ascontiguousarray(B).reshape(a.shape)


@pytest.mark.parametrize("how", ["swap_xz", "invert"])
@pytest.mark.parametrize("mode", ["point", "bin"])
def test_dos_invariant_under_maps_of_the_triangulation(how, mode):
    """Table I's six tetrahedra share the cube diagonal from corner (0,1,0) to
    (1,0,1); swapping the x and z axes, or inverting k, maps that
    triangulation onto itself with every tetrahedron's corners in another
    order. The DOS must not change: the corner sort and the weight-to-corner
    bookkeeping are order independent (corner-permutation invariance)."""
    n = (4, 3, 4)
    rng = np.random.default_rng(77)
    nk = n[0] * n[1] * n[2]
    eps = np.sort(rng.normal(0, 1, (nk, 3)), axis=1)
    w = rng.uniform(0.05, 1, (nk, 3, 2))
    edges = np.linspace(eps.min() - 0.2, eps.max() + 0.2, 41)
    om = edges if mode == "bin" else 0.5 * (edges[1:] + edges[:-1])
    d0 = oracle.dos(eps, w, *n, om, mode=mode)
    d1 = oracle.dos(grid_map(eps, n, how), grid_map(w, n, how), *n, om, mode=mode)
    np.testing.assert_allclose(d1, d0, rtol=0, atol=1e-12 * np.max(np.abs(d0)))
    # a relabelling that moves the diagonal (swapping x and y) does change
    # the DOS at this resolution, so the check has teeth
    m = (4, 4, 4)
    e4 = np.sort(rng.normal(0, 1, (64, 3)), axis=1)
    w4 = rng.uniform(0.05, 1, (64, 3, 2))
    A = e4.reshape(4, 4, 4, 3)
    Wa = w4.reshape(4, 4, 4, 3, 2)
    exy = np.ascontiguousarray(np.swapaxes(A, 1, 2)).reshape(64, 3)
    wxy = np.ascontiguousarray(np.swapaxes(Wa, 1, 2)).reshape(64, 3, 2)
    f0 = oracle.dos(e4, w4, *m, om, mode=mode)
    f1 = oracle.dos(exy, wxy, *m, om, mode=mode)
    assert np.max(np.abs(f1 - f0)) > 1e-6 * np.max(np.abs(f0))
