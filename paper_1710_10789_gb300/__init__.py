"""Python binding of libtetra (GB300 / sm_103a linear tetrahedron DOS).

The functions named ``tetra_*`` mirror the C ABI in ``include/tetra.h``
one-to-one (argument marshalling through ctypes; pointers are integers). The
``Plan`` class and the autograd functions in ``autograd`` add PyTorch tensor
convenience on top: PyTorch provides device memory and streams only, every
step of the method runs in the library's CUDA kernels.

The library must be built first (``paper_1710_10789_gb300.build()`` or
``python -c "import __graft_entry__ as g; g.build()"``); without it every call
raises ``TetraError`` — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "TETRA_OK", "TETRA_POINT", "TETRA_BIN", "TETRA_INTEGRATED", "TETRA_F32", "TETRA_F16", "TETRA_BF16",
    "TetraError", "TetraDesc", "TetraLayout", "TetraModel", "build", "lib", "lib_path",
    "tetra_plan", "tetra_plan_destroy", "tetra_layout", "tetra_workspace_bytes", "tetra_dos",
    "tetra_dos_backward", "tetra_eig", "tetra_eig_backward", "tetra_eig_workspace_bytes",
    "tetra_workspace_status", "tetra_strerror", "tetra_version", "tetra_dos_noalloc",
    "tetra_noalloc_status", "Plan",
    "EXPORTED_SYMBOLS", "TetraTune", "tetra_plan_batched", "tetra_batch_plan_destroy",
    "tetra_batch_layout", "tetra_batch_workspace_bytes", "tetra_batch_info", "tetra_dos_batched",
    "BatchPlan", "TETRA_MAX_BATCH", "tetra_fermi_workspace_bytes", "tetra_fermi_level", "tetra_pair_bands",
    "tetra_spectral_t0_workspace_bytes", "tetra_spectral_t0", "tetra_chi0_real_t0_workspace_bytes",
    "tetra_chi0_real_t0",
]

TETRA_OK, TETRA_EINVAL, TETRA_EUNSUPPORTED, TETRA_ECUDA, TETRA_ENOMEM, TETRA_ETIMEOUT, TETRA_ERANGE = range(7)
TETRA_POINT, TETRA_BIN, TETRA_INTEGRATED = 0, 1, 2
TETRA_F32, TETRA_F16, TETRA_BF16 = 0, 1, 2
_DTYPES = {"f32": TETRA_F32, "f16": TETRA_F16, "bf16": TETRA_BF16}
_MODES = {"point": TETRA_POINT, "bin": TETRA_BIN, "integrated": TETRA_INTEGRATED}

#: Every extern "C" symbol declared in include/tetra.h.
EXPORTED_SYMBOLS = (
    "tetra_plan", "tetra_plan_destroy", "tetra_layout", "tetra_workspace_bytes", "tetra_dos",
    "tetra_dos_backward", "tetra_eig", "tetra_eig_backward", "tetra_eig_workspace_bytes",
    "tetra_workspace_status", "tetra_strerror", "tetra_version", "tetra_dos_noalloc",
    "tetra_noalloc_status", "tetra_plan_batched", "tetra_batch_plan_destroy", "tetra_batch_layout",
    "tetra_batch_workspace_bytes", "tetra_batch_info", "tetra_dos_batched",
    "tetra_fermi_workspace_bytes", "tetra_fermi_level", "tetra_pair_bands",
    "tetra_spectral_t0_workspace_bytes", "tetra_spectral_t0", "tetra_chi0_real_t0_workspace_bytes",
    "tetra_chi0_real_t0",
)
TETRA_MAX_BATCH = 64


class TetraError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = tetra_strerror(status) if _LIB is not None else f"status {status}"
        super().__init__(f"{what}: {msg}" if what else msg)


class TetraDesc(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("n_bands", ctypes.c_int), ("n_orb", ctypes.c_int), ("n_omega", ctypes.c_int),
                ("mode", ctypes.c_int), ("weight_dtype", ctypes.c_int),
                ("z_begin", ctypes.c_int), ("z_end", ctypes.c_int)]


class TetraLayout(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("eps_stride", ctypes.c_int), ("w_stride", ctypes.c_int),
                ("eps_elems", ctypes.c_size_t), ("w_elems", ctypes.c_size_t)]


class TetraTune(ctypes.Structure):
    _fields_ = [("box_x", ctypes.c_int), ("box_y", ctypes.c_int), ("box_z", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int)]


class TetraModel(ctypes.Structure):
    _fields_ = [("n_orb", ctypes.c_int), ("n_R", ctypes.c_int),
                ("params", ctypes.c_void_p), ("R", ctypes.c_void_p)]


_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libtetra.so in-tree for sm_103a."""
    return _build.build(force=force)


def lib_path() -> str:
    return _build.LIBPATH


def lib():
    """The loaded libtetra (raises if it was not built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(_build.LIBPATH):
                raise TetraError(TETRA_ECUDA, f"libtetra.so missing at {_build.LIBPATH}; "
                                 "build it with paper_1710_10789_gb300.build()")
            L = ctypes.CDLL(_build.LIBPATH)
            vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            L.tetra_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(TetraDesc), i]
            L.tetra_plan_destroy.argtypes = [vp]
            L.tetra_layout.argtypes = [vp, ctypes.POINTER(TetraLayout)]
            L.tetra_workspace_bytes.argtypes = [vp]
            L.tetra_workspace_bytes.restype = sz
            L.tetra_dos.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
            L.tetra_dos_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
            L.tetra_noalloc_status.argtypes = [i, vp]
            L.tetra_dos_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
            L.tetra_eig.argtypes = [vp, ctypes.POINTER(TetraModel), vp, vp, vp]
            L.tetra_eig_backward.argtypes = [vp, ctypes.POINTER(TetraModel), vp, vp, vp, vp, sz, vp]
            L.tetra_eig_workspace_bytes.argtypes = [vp, i]
            L.tetra_eig_workspace_bytes.restype = sz
            L.tetra_workspace_status.argtypes = [vp, vp]
            L.tetra_plan_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(TetraDesc), i,
                                             ctypes.POINTER(TetraTune), i]
            L.tetra_batch_plan_destroy.argtypes = [vp]
            L.tetra_batch_layout.argtypes = [vp, i, ctypes.POINTER(TetraLayout)]
            L.tetra_batch_workspace_bytes.argtypes = [vp]
            L.tetra_batch_workspace_bytes.restype = sz
            L.tetra_batch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
            L.tetra_dos_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(vp), ctypes.POINTER(vp), vp, sz, vp]
            L.tetra_fermi_workspace_bytes.argtypes = [vp]
            L.tetra_fermi_workspace_bytes.restype = sz
            L.tetra_fermi_level.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_float),
                                            vp, sz, vp]
            L.tetra_pair_bands.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_float,
                                           ctypes.c_float, vp, vp, vp, vp]
            L.tetra_spectral_t0_workspace_bytes.argtypes = [vp, i]
            L.tetra_spectral_t0_workspace_bytes.restype = sz
            L.tetra_spectral_t0.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_float, i, i, vp, vp,
                                            vp, sz, vp]
            L.tetra_chi0_real_t0_workspace_bytes.argtypes = [vp, i]
            L.tetra_chi0_real_t0_workspace_bytes.restype = sz
            L.tetra_chi0_real_t0.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_float, i, vp, vp,
                                             vp, sz, vp]
            L.tetra_strerror.argtypes = [i]
            L.tetra_strerror.restype = ctypes.c_char_p
            L.tetra_version.restype = ctypes.c_char_p
            for name in ("tetra_plan", "tetra_plan_destroy", "tetra_layout", "tetra_dos",
                         "tetra_dos_noalloc", "tetra_noalloc_status",
                         "tetra_dos_backward", "tetra_eig", "tetra_eig_backward",
                         "tetra_workspace_status", "tetra_plan_batched",
                         "tetra_batch_plan_destroy", "tetra_batch_layout", "tetra_batch_info",
                         "tetra_dos_batched", "tetra_fermi_level", "tetra_pair_bands",
                         "tetra_spectral_t0", "tetra_chi0_real_t0"):
                getattr(L, name).restype = i
            _LIB = L
    return _LIB


def _check(st: int, what: str):
    if st != TETRA_OK:
        raise TetraError(st, what)


# ------------------------------------------------------------------ C ABI mirror
def tetra_plan(desc: TetraDesc, device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().tetra_plan(ctypes.byref(h), ctypes.byref(desc), int(device)), "tetra_plan")
    return h.value


def tetra_plan_destroy(plan: int) -> int:
    return lib().tetra_plan_destroy(plan)


def tetra_layout(plan: int) -> TetraLayout:
    L = TetraLayout()
    _check(lib().tetra_layout(plan, ctypes.byref(L)), "tetra_layout")
    return L


def tetra_workspace_bytes(plan: int) -> int:
    return int(lib().tetra_workspace_bytes(plan))


def tetra_dos(plan, eps, w, omega, dos, ws, ws_bytes, stream) -> int:
    return lib().tetra_dos(plan, eps, w, omega, dos, ws, ws_bytes, stream)


def tetra_fermi_workspace_bytes(plan) -> int:
    return lib().tetra_fermi_workspace_bytes(plan)


def tetra_fermi_level(plan, eps, w, n_electrons, ef, ws, ws_bytes, stream) -> int:
    return lib().tetra_fermi_level(plan, eps, w, float(n_electrons), ef, ws, ws_bytes, stream)


def tetra_pair_bands(plan, eps, q, kT, mu, pair_plan, eps_pairs, w_pairs, stream) -> int:
    qa = (ctypes.c_int * 3)(*[int(v) for v in q])
    return lib().tetra_pair_bands(plan, eps, qa, float(kT), float(mu), pair_plan, eps_pairs, w_pairs, stream)


def tetra_dos_noalloc(plan, eps, w, omega, dos, stream) -> int:
    """tetra_dos with the library's fixed scratch instead of a workspace (see tetra.h)."""
    return lib().tetra_dos_noalloc(plan, eps, w, omega, dos, stream)


def tetra_spectral_t0_workspace_bytes(plan, n_omega) -> int:
    return int(lib().tetra_spectral_t0_workspace_bytes(plan, int(n_omega)))


def tetra_spectral_t0(plan, eps, q, mu, mode, n_omega, omega, S, ws, ws_bytes, stream) -> int:
    qa = (ctypes.c_int * 3)(*[int(v) for v in q])
    return lib().tetra_spectral_t0(plan, eps, qa, float(mu), int(mode), int(n_omega), omega, S, ws, ws_bytes,
                                   stream)


def tetra_chi0_real_t0_workspace_bytes(plan, n_omega) -> int:
    return int(lib().tetra_chi0_real_t0_workspace_bytes(plan, int(n_omega)))


def tetra_chi0_real_t0(plan, eps, q, mu, n_omega, omega, R, ws, ws_bytes, stream) -> int:
    qa = (ctypes.c_int * 3)(*[int(v) for v in q])
    return lib().tetra_chi0_real_t0(plan, eps, qa, float(mu), int(n_omega), omega, R, ws, ws_bytes, stream)


def tetra_noalloc_status(device, stream) -> int:
    """Device-side status of the last tetra_dos_noalloc call on `device`."""
    return lib().tetra_noalloc_status(int(device), stream)


def tetra_dos_backward(plan, eps, w, omega, grad_dos, grad_eps, grad_w, ws, ws_bytes, stream) -> int:
    return lib().tetra_dos_backward(plan, eps, w, omega, grad_dos, grad_eps, grad_w, ws, ws_bytes,
                                    stream)


def tetra_eig(plan, model: TetraModel, eps, w, stream) -> int:
    return lib().tetra_eig(plan, ctypes.byref(model), eps, w, stream)


def tetra_eig_backward(plan, model: TetraModel, grad_eps, grad_w, grad_params, ws, ws_bytes,
                       stream) -> int:
    return lib().tetra_eig_backward(plan, ctypes.byref(model), grad_eps, grad_w, grad_params, ws,
                                    ws_bytes, stream)


def tetra_eig_workspace_bytes(plan, n_R: int) -> int:
    return int(lib().tetra_eig_workspace_bytes(plan, int(n_R)))


def tetra_workspace_status(ws, stream) -> int:
    return lib().tetra_workspace_status(ws, stream)


def tetra_plan_batched(descs, tune: "TetraTune | None" = None, device: int = 0) -> int:
    arr = (TetraDesc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().tetra_plan_batched(ctypes.byref(h), arr, len(descs),
                                    ctypes.byref(tune) if tune is not None else None, int(device)),
           "tetra_plan_batched")
    return h.value


def tetra_batch_plan_destroy(plan: int) -> int:
    return lib().tetra_batch_plan_destroy(plan)


def tetra_batch_layout(plan: int, model: int) -> TetraLayout:
    L = TetraLayout()
    _check(lib().tetra_batch_layout(plan, int(model), ctypes.byref(L)), "tetra_batch_layout")
    return L


def tetra_batch_workspace_bytes(plan: int) -> int:
    return int(lib().tetra_batch_workspace_bytes(plan))


def tetra_batch_info(plan: int):
    """(box (bx, by, bz), persistent CTAs, partial slots) chosen by the plan."""
    box = (ctypes.c_int * 3)()
    grid, slots = ctypes.c_int(), ctypes.c_int()
    _check(lib().tetra_batch_info(plan, box, ctypes.byref(grid), ctypes.byref(slots)),
           "tetra_batch_info")
    return tuple(box), grid.value, slots.value


def tetra_dos_batched(plan, eps, w, omega, dos, ws, ws_bytes, stream) -> int:
    """eps, w, omega, dos: sequences of device pointers (one per model)."""
    n = len(eps)
    arrs = [(ctypes.c_void_p * n)(*[int(x) for x in a]) for a in (eps, w, omega, dos)]
    return lib().tetra_dos_batched(plan, *arrs, ws, ws_bytes, stream)


def tetra_strerror(status: int) -> str:
    return lib().tetra_strerror(int(status)).decode()


def tetra_version() -> str:
    return lib().tetra_version().decode()


# ------------------------------------------------------------------ tensor convenience
def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr())


class Plan:
    """A tetra plan plus tensor-level calls (PyTorch for memory and streams)."""

    def __init__(self, n1, n2, n3, n_bands, n_orb, n_omega, mode="point", weight_dtype="f32",
                 z_range=None, device=None):
        torch = _torch()
        dev = torch.cuda.current_device() if device is None else int(device)
        z0, z1 = (0, 0) if z_range is None else z_range
        self.desc = TetraDesc(n1, n2, n3, n_bands, n_orb, n_omega, _MODES[mode],
                              _DTYPES[weight_dtype], z0, z1)
        self.mode = mode
        self.weight_dtype = weight_dtype
        self.device = dev
        with torch.cuda.device(dev):
            self.handle = tetra_plan(self.desc, dev)
        self.layout = tetra_layout(self.handle)
        self.workspace_bytes = tetra_workspace_bytes(self.handle)
        self._ws = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.tetra_plan_destroy(h)
            self.handle = None

    # memory helpers -----------------------------------------------------
    @property
    def torch_weight_dtype(self):
        torch = _torch()
        return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.weight_dtype]

    def empty_inputs(self):
        """(eps, w) device tensors shaped (nz, ny, nx, stride) in the tetra layout."""
        torch = _torch()
        L = self.layout
        dev = torch.device("cuda", self.device)
        eps = torch.zeros((L.nz, L.ny, L.nx, L.eps_stride), dtype=torch.float32, device=dev)
        w = torch.zeros((L.nz, L.ny, L.nx, L.w_stride), dtype=self.torch_weight_dtype, device=dev)
        return eps, w

    def workspace(self):
        torch = _torch()
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                   device=torch.device("cuda", self.device))
        return self._ws

    # calls ----------------------------------------------------------------
    def dos(self, eps, w, omega, out=None, stream=None):
        torch = _torch()
        no, nw = self.desc.n_orb, self.desc.n_omega
        if out is None:
            out = torch.empty((no, nw), dtype=torch.float32, device=eps.device)
        ws = self.workspace()
        _check(tetra_dos(self.handle, _ptr(eps), _ptr(w), _ptr(omega), _ptr(out), _ptr(ws),
                         ws.numel(), _stream_handle(stream)), "tetra_dos")
        return out

    def dos_backward(self, eps, w, omega, grad_dos, grad_eps=None, grad_w=None, stream=None):
        torch = _torch()
        if grad_eps is None:
            grad_eps = torch.empty(eps.shape, dtype=torch.float32, device=eps.device)
        if grad_w is None:
            grad_w = torch.empty(w.shape, dtype=torch.float32, device=w.device)
        ws = self.workspace()
        _check(tetra_dos_backward(self.handle, _ptr(eps), _ptr(w), _ptr(omega),
                                  _ptr(grad_dos.contiguous()), _ptr(grad_eps), _ptr(grad_w),
                                  _ptr(ws), ws.numel(), _stream_handle(stream)), "tetra_dos_backward")
        return grad_eps, grad_w

    def fermi_level(self, eps, w, n_electrons, stream=None) -> float:
        """E_F with sum over the plan's orbitals of n_s(E_F) = n_electrons per spin
        (tetra_fermi_level)."""
        torch = _torch()
        nbytes = tetra_fermi_workspace_bytes(self.handle)
        if nbytes == 0:
            raise TetraError(TETRA_EUNSUPPORTED, "tetra_fermi_workspace_bytes")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=eps.device)
        ef = ctypes.c_float(0.0)
        _check(tetra_fermi_level(self.handle, _ptr(eps), _ptr(w), n_electrons, ctypes.byref(ef), _ptr(ws),
                                 ws.numel(), _stream_handle(stream)), "tetra_fermi_level")
        return float(ef.value)

    def pair_bands(self, eps, q, kT, mu, pair_plan, stream=None):
        """Transition bands of the bare susceptibility at grid vector q
        (tetra_pair_bands) in pair_plan's layout: (eps_pairs, w_pairs)."""
        eps_p, w_p = pair_plan.empty_inputs()
        _check(tetra_pair_bands(self.handle, _ptr(eps), q, kT, mu, pair_plan.handle, _ptr(eps_p), _ptr(w_p),
                                _stream_handle(stream)), "tetra_pair_bands")
        return eps_p, w_p

    def spectral_t0(self, eps, q, mu, omega, mode="point", out=None, stream=None):
        """T = 0 spectral function of the bare susceptibility at grid vector q
        (tetra_spectral_t0): S at the energies ``omega`` (point mode) or the
        bin averages between consecutive edges (bin mode). Returns S; its
        device status is ``spectral_status()``."""
        torch = _torch()
        m = _MODES[mode]
        n_om = omega.numel() - 1 if m == TETRA_BIN else omega.numel()
        if out is None:
            out = torch.empty((n_om,), dtype=torch.float32, device=eps.device)
        nbytes = tetra_spectral_t0_workspace_bytes(self.handle, n_om)
        if getattr(self, "_spec_ws", None) is None or self._spec_ws.numel() < nbytes:
            self._spec_ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=eps.device)
        ws = self._spec_ws
        _check(tetra_spectral_t0(self.handle, _ptr(eps), q, mu, m, n_om, _ptr(omega), _ptr(out), _ptr(ws),
                                 ws.numel(), _stream_handle(stream)), "tetra_spectral_t0")
        return out

    def chi0_real_t0(self, eps, q, mu, omega, out=None, stream=None):
        """Real part of the T = 0 bare susceptibility at grid vector q
        (tetra_chi0_real_t0) at the energies ``omega``. Returns Re chi0; its
        device status is ``spectral_status()``."""
        torch = _torch()
        n_om = omega.numel()
        if out is None:
            out = torch.empty((n_om,), dtype=torch.float32, device=eps.device)
        nbytes = tetra_chi0_real_t0_workspace_bytes(self.handle, n_om)
        if getattr(self, "_spec_ws", None) is None or self._spec_ws.numel() < nbytes:
            self._spec_ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=eps.device)
        ws = self._spec_ws
        _check(tetra_chi0_real_t0(self.handle, _ptr(eps), q, mu, n_om, _ptr(omega), _ptr(out), _ptr(ws),
                                  ws.numel(), _stream_handle(stream)), "tetra_chi0_real_t0")
        return out

    def spectral_status(self, stream=None) -> int:
        return tetra_workspace_status(_ptr(self._spec_ws), _stream_handle(stream))

    def _model(self, params, R):
        n_orb = self.desc.n_bands
        return TetraModel(n_orb, int(R.shape[0]), _ptr(params), _ptr(R))

    def eig(self, params, R, eps=None, w=None, stream=None):
        """params: float32 device [n_orb + 2 n_R n_orb^2]; R: int32 device [n_R, 3]."""
        if eps is None or w is None:
            eps, w = self.empty_inputs()
        m = self._model(params, R)
        _check(tetra_eig(self.handle, m, _ptr(eps), _ptr(w), _stream_handle(stream)), "tetra_eig")
        return eps, w

    def eig_backward(self, params, R, grad_eps, grad_w, stream=None):
        torch = _torch()
        m = self._model(params, R)
        nbytes = tetra_eig_workspace_bytes(self.handle, m.n_R)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=params.device)
        g = torch.empty_like(params)
        _check(tetra_eig_backward(self.handle, m, _ptr(grad_eps), _ptr(grad_w), _ptr(g), _ptr(ws),
                                  ws.numel(), _stream_handle(stream)), "tetra_eig_backward")
        return g

    def status(self, stream=None) -> int:
        ws = self.workspace()
        return tetra_workspace_status(_ptr(ws), _stream_handle(stream))


class BatchPlan:
    """Many independent DOS problems (same n_bands, n_orb, mode, weight dtype) in
    one launch; ``graph()`` captures that launch in a CUDA graph."""

    def __init__(self, grids, n_omegas, n_bands, n_orb, mode="point", weight_dtype="f32",
                 tune=None, device=None):
        torch = _torch()
        if len(grids) != len(n_omegas):
            raise ValueError("one energy count per grid")
        dev = torch.cuda.current_device() if device is None else int(device)
        self.descs = [TetraDesc(int(g[0]), int(g[1]), int(g[2]), n_bands, n_orb, int(nw), _MODES[mode],
                                _DTYPES[weight_dtype], 0, 0) for g, nw in zip(grids, n_omegas)]
        self.mode = mode
        self.weight_dtype = weight_dtype
        self.device = dev
        self.tune = tune
        t = None
        if tune is not None:
            t = TetraTune(*[int(x) for x in tune.get("box", (0, 0, 0))], int(tune.get("ctas_per_sm", 0)))
        with torch.cuda.device(dev):
            self.handle = tetra_plan_batched(self.descs, t, dev)
        self.layouts = [tetra_batch_layout(self.handle, m) for m in range(len(self.descs))]
        self.workspace_bytes = tetra_batch_workspace_bytes(self.handle)
        self.box, self.grid, self.n_slots = tetra_batch_info(self.handle)
        self._ws = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.tetra_batch_plan_destroy(h)
            self.handle = None

    def __len__(self):
        return len(self.descs)

    @property
    def torch_weight_dtype(self):
        torch = _torch()
        return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.weight_dtype]

    def empty_inputs(self, m):
        torch = _torch()
        L = self.layouts[m]
        dev = torch.device("cuda", self.device)
        eps = torch.zeros((L.nz, L.ny, L.nx, L.eps_stride), dtype=torch.float32, device=dev)
        w = torch.zeros((L.nz, L.ny, L.nx, L.w_stride), dtype=self.torch_weight_dtype, device=dev)
        return eps, w

    def workspace(self):
        torch = _torch()
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                   device=torch.device("cuda", self.device))
        return self._ws

    def empty_outputs(self):
        torch = _torch()
        dev = torch.device("cuda", self.device)
        return [torch.empty((d.n_orb, d.n_omega), dtype=torch.float32, device=dev) for d in self.descs]

    def dos(self, eps, w, omega, out=None, stream=None):
        if out is None:
            out = self.empty_outputs()
        ws = self.workspace()
        _check(tetra_dos_batched(self.handle, [_ptr(x) for x in eps], [_ptr(x) for x in w],
                                 [_ptr(x) for x in omega], [_ptr(x) for x in out], _ptr(ws),
                                 ws.numel(), _stream_handle(stream)), "tetra_dos_batched")
        return out

    def graph(self, eps, w, omega, out=None):
        """Captures one batched DOS launch (memset, forward kernel, reduce) over
        these tensors in a CUDA graph. Returns (graph, out): ``graph.replay()``
        recomputes ``out`` from the current contents of the inputs."""
        torch = _torch()
        if out is None:
            out = self.empty_outputs()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.dos(eps, w, omega, out)   # loads the kernels before capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.dos(eps, w, omega, out)
        return g, out

    def status(self, stream=None) -> int:
        ws = self.workspace()
        return tetra_workspace_status(_ptr(ws), _stream_handle(stream))
