"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and fixes problem definitions (model
parameters, grid sizes, energy grids). It holds none of the tetrahedron
method's arithmetic: it does not build H(k), diagonalise, sort corners or
compute weights. Both the FP64 oracle (``oracle/``) and the CUDA path
(``paper_1710_10789_gb300``) receive what it returns as plain arrays.

Models
------
The paper's benchmark uses an eight-orbital tight-binding model of FeSe
(Sec. II.A, Eq. 1) whose hopping parameters are not given in the paper. The
stand-in is a seeded eight-orbital tetragonal model with the same size and
structure: real on-site energies U[-2, 2] eV and complex hopping matrices
t(R) with i.i.d. N(0, 0.3^2) real and imaginary parts to the in-plane first,
second and third neighbours and to the +z neighbour. ``t(-R) = t(R)^dagger``
is implied, so H(k) = diag(onsite) + sum_R [t(R) e^{ik.R} + h.c.] is Hermitian.
"""
from __future__ import annotations

import numpy as np

#: Independent lattice vectors R of the synthetic tetragonal model (in units
#: of the lattice constants): in-plane 1st (100, 010), 2nd (110, 1-10),
#: 3rd (200, 020) neighbours and the +z nearest neighbour.
TETRAGONAL_R = np.array(
    [[1, 0, 0], [0, 1, 0], [1, 1, 0], [1, -1, 0], [2, 0, 0], [0, 2, 0], [0, 0, 1]],
    dtype=np.int64,
)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def tb_model(seed: int, n_orb: int = 8, onsite_range: float = 2.0,
             hop_sigma: float = 0.3) -> dict:
    """Seeded synthetic tight-binding model.

    Returns a dict with ``onsite`` (n_orb,) float64, ``R`` (nR, 3) int64 and
    ``t`` (nR, n_orb, n_orb) complex128.
    """
    rng = _rng(seed)
    onsite = rng.uniform(-onsite_range, onsite_range, n_orb)
    nR = TETRAGONAL_R.shape[0]
    re = rng.normal(0.0, hop_sigma, (nR, n_orb, n_orb))
    im = rng.normal(0.0, hop_sigma, (nR, n_orb, n_orb))
    return {"onsite": onsite, "R": TETRAGONAL_R.copy(), "t": re + 1j * im}


def sc_model(t: float = 1.0) -> dict:
    """Single-band simple-cubic nearest-neighbour model, eps(k) = -2t sum cos k_i.

    Written in the same hopping form: on-site 0 and t(R) = -t for the three
    independent R = (100), (010), (001).
    """
    R = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int64)
    tt = np.full((3, 1, 1), -t, dtype=np.complex128)
    return {"onsite": np.zeros(1), "R": R, "t": tt}


def uniform_grid(lo: float, hi: float, n: int) -> np.ndarray:
    """n equidistant energies including both end points (FP32, as the kernels read them)."""
    return np.linspace(lo, hi, n, dtype=np.float64).astype(np.float32)


def bin_edges(lo: float, hi: float, nbins: int) -> np.ndarray:
    """nbins + 1 equidistant bin edges (FP32)."""
    return np.linspace(lo, hi, nbins + 1, dtype=np.float64).astype(np.float32)


def synthetic_bands(seed: int, n1: int, n2: int, n3: int, nb: int, n_orb: int,
                    n_terms: int = 3):
    """Cheap seeded band-like fields on a periodic grid, for parity checks at
    sizes where an FP64 eigensolve of every k-point would take too long.

    Energies are smooth periodic functions (sums of a few cosines per band,
    offset per band), sorted ascending at each k; orbital weights are smooth,
    positive and normalised over orbitals for each band. Natural layout:
    eps[k, n], w[k, n, s] with k = x + n1 * (y + n2 * z).
    """
    rng = _rng(seed)
    x = np.arange(n1) / n1
    y = np.arange(n2) / n2
    z = np.arange(n3) / n3
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ph = 2.0 * np.pi
    eps = np.empty((n3, n2, n1, nb), np.float64)
    for n in range(nb):
        acc = np.full(X.shape, -8.0 + 16.0 * (n + 0.5) / nb)
        for _ in range(n_terms):
            m = rng.integers(-2, 3, size=3)
            if not m.any():
                m[0] = 1
            a = rng.normal(0.0, 1.2)
            p = rng.uniform(0, ph)
            acc += a * np.cos(ph * (m[0] * X + m[1] * Y + m[2] * Z) + p)
        eps[..., n] = acc
    eps.sort(axis=-1)
    w = np.empty((n3, n2, n1, nb, n_orb), np.float64)
    for n in range(nb):
        for s in range(n_orb):
            m = rng.integers(-1, 2, size=3)
            p = rng.uniform(0, ph)
            amp = rng.uniform(0.2, 0.9)
            w[..., n, s] = 1.0 + amp * np.cos(ph * (m[0] * X + m[1] * Y + m[2] * Z) + p)
    w /= w.sum(axis=-1, keepdims=True)
    return eps.reshape(-1, nb), w.reshape(-1, nb, n_orb)


def batched_problems(n_models: int = 64, seed0: int = 1000, n_lo: int = 16,
                     n_hi: int = 96, w_lo: int = 500, w_hi: int = 3000) -> list:
    """Batched workload definition: per model a seed, a cubic grid size
    N ~ U{n_lo..n_hi} and an energy-point count ~ U{w_lo..w_hi}."""
    out = []
    for i in range(n_models):
        rng = _rng(seed0 + i)
        out.append({"seed": seed0 + i,
                    "n": int(rng.integers(n_lo, n_hi + 1)),
                    "n_omega": int(rng.integers(w_lo, w_hi + 1))})
    return out


def fit_parameter_subset(seed: int, n_params: int, n_total: int) -> np.ndarray:
    """Seeded choice of which real model parameters are fitted (the rest frozen)."""
    rng = _rng(seed + 1)
    return np.sort(rng.choice(n_total, size=n_params, replace=False))
