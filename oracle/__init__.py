"""FP64 CPU oracle for the linear tetrahedron orbital-resolved DOS.

TEST INFRASTRUCTURE ONLY: this package is the slow, plain reference that the
CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with ``paper_1710_10789_gb300`` and neither imports the other.

Pieces and the passages they follow (arXiv:1710.10789):
  * ``hamiltonian`` / ``eig``: H(k) from the hopping form of Eq. (1) and its
    dense diagonalisation (Sec. II.A); orbital weights b = |a|^2, Eq. (3).
  * ``corner_weights``: the five energy cases of Sec. II.C (C code).
  * ``dos``: Eqs. (8)-(9), point values dw/dE or bin averages of w (C code).
  * ``weight_moments`` / ``dos_bin_grad``: derivative of the bin-averaged DOS
    with respect to corner energies and orbital weights, from the integral
    definition of the corner weights (C code).
  * ``eig_backward``: first-order perturbation theory of the Hermitian
    eigenproblem, chained to the hopping parameters of Eq. (1).
  * ``pair_bands`` / ``spectral_t0``: the spectral part of the bare
    susceptibility, the extension the paper names (abstract, Conclusions):
    with Fermi-Dirac occupations interpolated linearly (pair bands fed to
    ``dos``), and at T = 0 with step occupations clipped exactly inside each
    tetrahedron (C code).
  * ``chi0_real_t0`` / ``t0_inverse_average``: the real part at T = 0 on the
    same clipped sub-tetrahedra, the principal-value average of 1/(w - D)
    over each (C code).

Every numerical convention (grid, corner labels, region boundaries, the
corrected dw3/dE term) is listed in the header of ``tetra_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "tetra_oracle.c")
_lock = threading.Lock()
_lib = None

#: Regularisation of 1/(e_n - e_m) in the eigenvector derivative:
#: F = d / (d^2 + ETA^2) with d in eV (reading of degenerate pairs).
ETA = 1e-8


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_lib/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIBPATH)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            lib.oracle_corner_weights.argtypes = [d, ctypes.c_double, ctypes.c_double, d, d]
            lib.oracle_corner_weights.restype = None
            lib.oracle_weight_moments.argtypes = [d, ctypes.c_double, ctypes.c_double, d]
            lib.oracle_weight_moments.restype = None
            lib.oracle_dos_range.argtypes = [i, i, i, i, i, d, d, i, i, d, d, i, i, d, i]
            lib.oracle_dos_range.restype = i
            lib.oracle_dos_bin_grad.argtypes = [i, i, i, i, i, d, d, i, d, d, d, d, d]
            lib.oracle_dos_bin_grad.restype = i
            lib.oracle_table_i.argtypes = [ctypes.POINTER(ctypes.c_int)]
            lib.oracle_table_i.restype = None
            lib.oracle_t0_tetra.argtypes = [d, d, i, i, d, d, d]
            lib.oracle_t0_tetra.restype = None
            lib.oracle_t0_spectral.argtypes = [i, i, i, i, d, d, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                               i, i, d, d, i, i, d, i]
            lib.oracle_t0_spectral.restype = i
            lib.oracle_t0_inverse_average.argtypes = [d, ctypes.c_double]
            lib.oracle_t0_inverse_average.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- per tetrahedron
def table_i() -> np.ndarray:
    """The oracle's tetrahedron table (Table I): (6, 4) corner labels 1..8."""
    lib = _load()
    out = np.zeros(24, dtype=np.int32)
    lib.oracle_table_i(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out.reshape(6, 4)


def corner_weights(e_sorted, E: float, f: float):
    """(w[4], dw/dE[4]) of one tetrahedron with sorted corner energies."""
    lib = _load()
    e = _c64(e_sorted)
    w = np.zeros(4)
    dw = np.zeros(4)
    lib.oracle_corner_weights(_p(e), float(E), float(f), _p(w), _p(dw))
    return w, dw


def weight_moments(e_sorted, E: float, f: float) -> np.ndarray:
    """M[l, i] with d w_l / d e_i = -M[l, i] (sorted indices)."""
    lib = _load()
    e = _c64(e_sorted)
    M = np.zeros((4, 4))
    lib.oracle_weight_moments(_p(e), float(E), float(f), _p(M))
    return M


# ---------------------------------------------------------------- model + eig
def hamiltonian(model: dict, n1: int, n2: int, n3: int) -> np.ndarray:
    """H(k) on the Gamma-centred periodic grid k = 2 pi (x/n1, y/n2, z/n3),
    flat order k = x + n1*(y + n2*z). Returns (nk, n_orb, n_orb) complex128."""
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    kf = np.stack([x.ravel() / n1, y.ravel() / n2, z.ravel() / n3], axis=1)
    n_orb = model["onsite"].shape[0]
    H = np.zeros((kf.shape[0], n_orb, n_orb), np.complex128)
    H[:, np.arange(n_orb), np.arange(n_orb)] = model["onsite"][None, :]
    for R, t in zip(model["R"], model["t"]):
        ph = np.exp(2j * np.pi * (kf @ R.astype(np.float64)))
        H += ph[:, None, None] * t[None] + np.conj(ph)[:, None, None] * t.conj().T[None]
    return H


def eig(model: dict, n1: int, n2: int, n3: int, return_vectors: bool = False):
    """FP64 dense diagonalisation at every grid point (LAPACK via numpy).
    Returns eps (nk, nb) ascending and w (nk, nb, n_orb) with
    w[k, n, s] = |V[k, s, n]|^2."""
    H = hamiltonian(model, n1, n2, n3)
    ev, V = np.linalg.eigh(H)
    w = np.abs(np.transpose(V, (0, 2, 1))) ** 2
    if return_vectors:
        return ev, w, V
    return ev, w


# ---------------------------------------------------------------- DOS
def dos(eps, w, n1, n2, n3, energies, mode="point", edges_hi=None, z_range=None,
        nthreads: int = 1) -> np.ndarray:
    """Orbital-resolved DOS, Eqs. (8)-(9).

    eps (nk, nb), w (nk, nb, norb) in the natural layout. Point mode:
    ``energies`` is any list of E values. Integrated mode: the orbital
    occupation n_s(E) = sum_{tetra,n} sum_l b_{n,l,s} w_l(E) (Eq. (2) with the
    step function as occupation) at each E of ``energies``. Bin mode: either ``energies`` holds
    nbins+1 ascending edges, or ``energies``/``edges_hi`` hold the lower and
    upper edge of each bin. Returns (norb, npts).
    """
    lib = _load()
    eps = _c64(eps)
    w = _c64(w)
    nk = n1 * n2 * n3
    nb = eps.shape[1]
    norb = w.shape[2]
    assert eps.shape == (nk, nb) and w.shape == (nk, nb, norb)
    if mode == "point":
        ea = _c64(energies)
        eb = ea
        m = 0
    elif mode == "integrated":
        ea = _c64(energies)
        eb = ea
        m = 2
    elif mode == "bin":
        if edges_hi is None:
            e = _c64(energies)
            ea = np.ascontiguousarray(e[:-1])
            eb = np.ascontiguousarray(e[1:])
        else:
            ea = _c64(energies)
            eb = _c64(edges_hi)
        m = 1
    else:
        raise ValueError(mode)
    npts = ea.shape[0]
    out = np.zeros((norb, npts))
    z0, z1 = (0, n3) if z_range is None else z_range
    rc = lib.oracle_dos_range(n1, n2, n3, nb, norb, _p(eps), _p(w), m, npts, _p(ea), _p(eb),
                              int(z0), int(z1), _p(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_dos_range failed ({rc})")
    return out


def dos_bin_grad(eps, w, n1, n2, n3, edges, g):
    """Gradient of L = sum g * DOS_bin w.r.t. eps (nk, nb) and w (nk, nb, norb)."""
    lib = _load()
    eps = _c64(eps)
    w = _c64(w)
    e = _c64(edges)
    ea = np.ascontiguousarray(e[:-1])
    eb = np.ascontiguousarray(e[1:])
    nk = n1 * n2 * n3
    nb = eps.shape[1]
    norb = w.shape[2]
    g = _c64(g)
    assert g.shape == (norb, ea.shape[0])
    geps = np.zeros((nk, nb))
    gw = np.zeros((nk, nb, norb))
    rc = lib.oracle_dos_bin_grad(n1, n2, n3, nb, norb, _p(eps), _p(w), ea.shape[0], _p(ea),
                                 _p(eb), _p(g), _p(geps), _p(gw))
    if rc != 0:
        raise RuntimeError(f"oracle_dos_bin_grad failed ({rc})")
    return geps, gw


# ---------------------------------------------------------------- eig backward
def n_params(model: dict) -> int:
    n_orb = model["onsite"].shape[0]
    return n_orb + 2 * model["t"].shape[0] * n_orb * n_orb


def model_to_params(model: dict) -> np.ndarray:
    """Real parameter vector [onsite, Re t(R), Im t(R)]."""
    return np.concatenate([model["onsite"], model["t"].real.ravel(), model["t"].imag.ravel()])


def params_to_model(p: np.ndarray, like: dict) -> dict:
    n_orb = like["onsite"].shape[0]
    nR = like["t"].shape[0]
    m = n_orb * n_orb * nR
    t = (p[n_orb:n_orb + m] + 1j * p[n_orb + m:n_orb + 2 * m]).reshape(nR, n_orb, n_orb)
    return {"onsite": p[:n_orb].copy(), "R": like["R"], "t": t}


def eig_backward(model: dict, n1: int, n2: int, n3: int, geps, gw) -> np.ndarray:
    """dL/dparams given dL/deps (nk, nb) and dL/dw (nk, nb, norb).

    Per k: d eps_n = <n|dH|n> (Hellmann-Feynman) and
    d c_n = sum_{m != n} c_m <m|dH|n> F_nm with F_nm = 1/(eps_n - eps_m),
    regularised as d/(d^2 + ETA^2). With b_ns = |c_sn|^2 this gives
    dL = Re sum_ij dH_ij Q_ij, Q = conj(V) (diag(geps) + 2 B) V^T,
    B_mn = F_nm sum_s gw_ns conj(V_sn) V_sm. H(k) = D + sum_R t_R e^{ik.R} + h.c.
    then gives dL/dRe t_R = Re sum_k Z, dL/dIm t_R = -Im sum_k Z,
    Z = e^{ik.R} (Q + Q^H), and dL/dD_i = Re sum_k Q_ii.
    """
    H = hamiltonian(model, n1, n2, n3)
    ev, V = np.linalg.eigh(H)
    geps = _c64(geps)
    gw = _c64(gw)
    d = ev[:, :, None] - ev[:, None, :]          # d[k, n, m] = e_n - e_m
    F = d / (d * d + ETA * ETA)
    F[:, np.arange(d.shape[1]), np.arange(d.shape[1])] = 0.0
    # A[k, n, m] = sum_s gw[k, n, s] conj(V[k, s, n]) V[k, s, m]
    A = np.einsum("kns,ksn,ksm->knm", gw, np.conj(V), V)
    B = np.transpose(A * F, (0, 2, 1))            # B[k, m, n] = A[k, n, m] F[k, n, m]
    inner = 2.0 * B
    idx = np.arange(d.shape[1])
    inner[:, idx, idx] += geps
    Q = np.einsum("kim,kmn,kjn->kij", np.conj(V), inner, V)
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    kf = np.stack([x.ravel() / n1, y.ravel() / n2, z.ravel() / n3], axis=1)
    QQ = Q + np.conj(np.transpose(Q, (0, 2, 1)))
    g_on = np.real(np.einsum("kii->i", Q))
    g_re = []
    g_im = []
    for R in model["R"]:
        ph = np.exp(2j * np.pi * (kf @ R.astype(np.float64)))
        Zs = np.einsum("k,kij->ij", ph, QQ)
        g_re.append(np.real(Zs))
        g_im.append(-np.imag(Zs))
    return np.concatenate([g_on, np.array(g_re).ravel(), np.array(g_im).ravel()])


# ---------------------------------------------------------------- Fermi level
def fermi_level(eps, n1, n2, n3, n_electrons, tol=1e-12, nthreads: int = 1):
    """Energy E_F at which the integrated count of states per spin,
    N(E) = sum_{tetra,n} sum_l w_l(E) (Eq. (2), Sec. II.C weights, every
    orbital weight 1), equals n_electrons; plain bisection in FP64 on
    [min eps, max eps]. N is continuous and non-decreasing, so bisection
    converges to the lowest such energy within tol."""
    eps = _c64(eps)
    nk, nb = eps.shape
    ones = np.ones((nk, nb, 1))
    lo, hi = float(eps.min()), float(eps.max())
    if not (0.0 <= n_electrons <= nb):
        raise ValueError("n_electrons must lie in [0, n_bands]")

    def count(E):
        return float(dos(eps, ones, n1, n2, n3, np.array([E]), mode="integrated",
                         nthreads=nthreads)[0, 0])

    while hi - lo > tol * max(1.0, abs(lo), abs(hi)):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------- pair bands (spectral Lindhard function)
def fermi_dirac(eps, kT, mu):
    """Occupation 1 / (1 + exp((eps - mu) / kT)) in FP64 (kT > 0)."""
    x = (np.asarray(eps, np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def pair_bands(eps, n1, n2, n3, q, kT, mu):
    """Transition "bands" of the bare susceptibility at momentum q (integer
    grid vector): for every k and band pair (n, m), with j = n * nb + m,
      energy  Delta_j(k) = eps_m(k + q) - eps_n(k),
      weight  f(eps_n(k)) - f(eps_m(k + q))     (f: Fermi-Dirac at kT, mu).
    Their tetrahedron DOS S(q, w) = sum_{n,m} int [f_n - f_m'] delta(w - Delta)
    is the spectral part of the bare Lindhard function, Im chi0(q, w) = -pi S
    (the paper names susceptibilities as the method's extension; the energy
    difference and the occupation difference are linear inside each
    tetrahedron by the method's own interpolation). Returns (Delta (nk, nb^2),
    weight (nk, nb^2, 1))."""
    eps = _c64(eps)
    nk, nb = eps.shape
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    kq = ((x + q[0]) % n1) + n1 * (((y + q[1]) % n2) + n2 * ((z + q[2]) % n3))
    e_k = eps
    e_kq = eps[kq.ravel()]
    f_k = fermi_dirac(e_k, kT, mu)
    f_kq = fermi_dirac(e_kq, kT, mu)
    delta = (e_kq[:, None, :] - e_k[:, :, None]).reshape(nk, nb * nb)
    weight = (f_k[:, :, None] - f_kq[:, None, :]).reshape(nk, nb * nb, 1)
    return delta, weight


# ---------------------------------------------------------------- spectral function at T = 0
def _edges_pair(energies, mode, edges_hi):
    if mode in ("point", "real"):
        ea = _c64(energies)
        return ea, ea, 0 if mode == "point" else 2
    if edges_hi is None:
        e = _c64(energies)
        return np.ascontiguousarray(e[:-1]), np.ascontiguousarray(e[1:]), 1
    return _c64(energies), _c64(edges_hi), 1


def spectral_t0_tetra(a, c, energies, mode="point", edges_hi=None) -> np.ndarray:
    """One tetrahedron's T = 0 spectral contribution in units of V_T/V_G:
    a[4] = e_n - mu and c[4] = e_m(k+q) - mu at its corners; the transition
    energy c - a over {a < 0, c > 0} counts +1, over {a > 0, c < 0} -1
    (point density at ``energies``, or bin averages as in ``dos``; mode
    "real": the principal-value average of 1/(w - D) instead, the real part
    of chi0)."""
    lib = _load()
    ea, eb, m = _edges_pair(energies, mode, edges_hi)
    out = np.zeros(ea.shape[0])
    lib.oracle_t0_tetra(_p(_c64(a)), _p(_c64(c)), m, ea.shape[0], _p(ea), _p(eb), _p(out))
    return out


def t0_inverse_average(d, w) -> float:
    """Principal-value average of 1/(w - D) over a tetrahedron on whose
    corners the linear function D takes the values d[4] (C code: the
    density's three quadratic pieces integrated against 1/(w - x) in closed
    form near w and by their moment series far from it)."""
    lib = _load()
    return float(lib.oracle_t0_inverse_average(_p(_c64(d)), float(w)))


def chi0_real_t0(eps, n1, n2, n3, q, mu, energies, eps_kq=None, z_range=None, nthreads: int = 1) -> np.ndarray:
    """Real part of the T = 0 bare susceptibility at the points ``energies``,
    Re chi0(q, w) = sum_{n,m} (1/V_G) P int [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
                    / (w - e_m(k+q) + e_n(k)) dk,
    the Hilbert transform of ``spectral_t0``: the same exact clipping, each
    sub-tetrahedron adding sign * nu * P<1/(w - D)> (``t0_inverse_average``).
    Arguments as ``spectral_t0``. Returns (npts,)."""
    return spectral_t0(eps, n1, n2, n3, q, mu, energies, mode="real", eps_kq=eps_kq, z_range=z_range,
                       nthreads=nthreads)


def spectral_t0(eps, n1, n2, n3, q, mu, energies, mode="point", edges_hi=None, eps_kq=None,
                z_range=None, nthreads: int = 1) -> np.ndarray:
    """T = 0 spectral function of the bare susceptibility,
    S(q, w) = sum_{n,m} (1/V_G) int [Theta(mu - e_n(k)) - Theta(mu - e_m(k+q))]
              delta(w - e_m(k+q) + e_n(k)) dk,   Im chi0(q, w + i0) = -pi S,
    with every band linear inside each tetrahedron and the step occupations
    clipped exactly (C code, ``oracle_t0_spectral``). eps (nk, nb) natural
    layout; eps_kq, if given, holds the bands at k + q on the same flat index
    (otherwise eps shifted by the integer grid vector q). nthreads > 1 splits
    the cube planes into contiguous blocks and adds the per-thread results in
    thread order. Returns (npts,)."""
    lib = _load()
    eps = _c64(eps)
    nk, nb = eps.shape
    assert nk == n1 * n2 * n3
    epq = None if eps_kq is None else _c64(eps_kq)
    ea, eb, m = _edges_pair(energies, mode, edges_hi)
    out = np.zeros(ea.shape[0])
    qa = (ctypes.c_int * 3)(*[int(v) for v in q])
    z0, z1 = (0, n3) if z_range is None else z_range
    rc = lib.oracle_t0_spectral(n1, n2, n3, nb, _p(eps), _p(epq) if epq is not None else None, qa,
                                float(mu), m, ea.shape[0], _p(ea), _p(eb), int(z0), int(z1), _p(out),
                                int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_t0_spectral failed ({rc})")
    return out
