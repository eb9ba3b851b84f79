"""Test-side helpers: problem construction and layout conversion.

These convert natural-layout arrays (eps[k, n], w[k, n, s], k = x + n1*(y +
n2*z)) into the library's padded point-major layout. They belong to the tests;
neither the oracle nor the library imports them.
"""
import numpy as np

import oracle
import tbgen


def to_layout(eps, w, n1, n2, n3, eps_stride, w_stride, w_dtype=np.float32):
    nb = eps.shape[1]
    no = w.shape[2]
    e = eps.reshape(n3, n2, n1, nb)
    e = np.pad(e, ((0, 1), (0, 1), (0, 1), (0, 0)), mode="wrap")
    E = np.zeros(e.shape[:3] + (eps_stride,), np.float32)
    E[..., :nb] = e
    ww = w.reshape(n3, n2, n1, nb * no)
    ww = np.pad(ww, ((0, 1), (0, 1), (0, 1), (0, 0)), mode="wrap")
    W = np.zeros(ww.shape[:3] + (w_stride,), w_dtype)
    W[..., :nb * no] = ww
    return E, W


def from_layout(E, W, n1, n2, n3, nb, no):
    eps = np.asarray(E)[:n3, :n2, :n1, :nb].reshape(-1, nb)
    w = np.asarray(W)[:n3, :n2, :n1, :nb * no].reshape(-1, nb, no)
    return eps, w


def tb_problem(seed, n, n_orb=8):
    """FP64 eigen-data of the synthetic model, rounded to FP32 (the GPU input)."""
    n1, n2, n3 = n
    model = tbgen.tb_model(seed, n_orb=n_orb)
    eps, w = oracle.eig(model, n1, n2, n3)
    return model, eps.astype(np.float32), w.astype(np.float32)


def sc_problem(n):
    model = tbgen.sc_model()
    eps, w = oracle.eig(model, n, n, n)
    return model, eps.astype(np.float32), w.astype(np.float32)


def energy_window(eps, n_omega, pad=0.1):
    return tbgen.uniform_grid(float(eps.min()) - pad, float(eps.max()) + pad, n_omega)


def model_arrays(model):
    """(params float32, R int32) packed as in tetra_model_t."""
    params = np.concatenate([model["onsite"], model["t"].real.ravel(), model["t"].imag.ravel()])
    return params.astype(np.float32), model["R"].astype(np.int32)


def rounded_model(model):
    """The model with parameters rounded to FP32 (what the GPU sees), in FP64."""
    p, _ = model_arrays(model)
    return oracle.params_to_model(p.astype(np.float64), model)
