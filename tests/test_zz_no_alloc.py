"""The allocation-free entry point tetra_dos_noalloc, called through the C ABI.

It is for callers that cannot allocate device memory where they need a DOS
(a host framework that owns all allocations, a fixed memory budget, a loop
that must not call cudaMalloc): the kernel's scratch lives in a fixed array
inside the library. Its output must agree with tetra_dos (caller workspace)
within the tolerance of the parity tests, on two calls in a row (the second
call reuses the array the first one left behind). This file sorts last so a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import tbgen
from helpers import energy_window, tb_problem, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5


def test_noalloc_matches_workspace_entry_point():
    import paper_1710_10789_gb300 as T

    T.build()
    n = (10, 9, 11)
    _, eps, w = tb_problem(0, n)
    omega = energy_window(eps, 301)
    plan = T.Plan(*n, 8, 8, len(omega))
    L = plan.layout
    E, W = to_layout(eps, w, *n, L.eps_stride, L.w_stride)
    dev = torch.device("cuda")
    Et = torch.from_numpy(E).to(dev)
    Wt = torch.from_numpy(W).to(dev)
    om = torch.from_numpy(omega).to(dev)
    ref = torch.empty((8, len(omega)), dtype=torch.float32, device=dev)
    ws = plan.workspace()
    stream = torch.cuda.current_stream().cuda_stream
    st = T.tetra_dos(plan.handle, Et.data_ptr(), Wt.data_ptr(), om.data_ptr(), ref.data_ptr(),
                     ws.data_ptr(), ws.numel(), stream)
    assert st == T.TETRA_OK
    torch.cuda.synchronize()
    r = ref.cpu().numpy().astype(np.float64)
    for call in range(2):
        out = torch.full((8, len(omega)), float("nan"), dtype=torch.float32, device=dev)
        st = T.tetra_dos_noalloc(plan.handle, Et.data_ptr(), Wt.data_ptr(), om.data_ptr(),
                                 out.data_ptr(), stream)
        assert st == T.TETRA_OK, T.tetra_strerror(st)
        torch.cuda.synchronize()
        g = out.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(g - r))
        assert err <= TOL * np.max(np.abs(r)), (call, err)
        assert T.tetra_noalloc_status(torch.cuda.current_device(), stream) == T.TETRA_OK


SCRATCH = 32 << 20


@pytest.mark.parametrize("mode,n_omega", [("point", 4000), ("bin", 3800), ("integrated", 2000)])
def test_noalloc_with_fewer_ctas_is_bitwise_equal(mode, n_omega):
    """Problems whose per-CTA partial sums exceed the 32 MiB scratch with one
    CTA per SM run on fewer CTAs; the exact integer accumulation makes the
    result bit-identical to tetra_dos with a full workspace."""
    import paper_1710_10789_gb300 as T

    T.build()
    n = 24   # 6^3 = 216 boxes of 4^3 cubes: one CTA per SM with the default plan
    eps, w = tbgen.synthetic_bands(3, n, n, n, 8, 8)
    lo, hi = float(eps.min()) - 0.1, float(eps.max()) + 0.1
    omega = tbgen.bin_edges(lo, hi, n_omega) if mode == "bin" else tbgen.uniform_grid(lo, hi, n_omega)
    plan = T.Plan(n, n, n, 8, 8, n_omega, mode=mode)
    L = plan.layout
    E, W = to_layout(eps.astype(np.float32), w.astype(np.float32), n, n, n, L.eps_stride, L.w_stride)
    dev = torch.device("cuda")
    Et, Wt, om = (torch.from_numpy(a).to(dev) for a in (E, W, omega))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    parts = 256 + (2 if mode == "integrated" else 1) * 8 * 8 * min(216, sms) * n_omega
    assert parts > SCRATCH, "the case must not fit the scratch with the default CTA count"
    ref = plan.dos(Et, Wt, om)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        st = T.tetra_dos_noalloc(plan.handle, Et.data_ptr(), Wt.data_ptr(), om.data_ptr(), out.data_ptr(),
                                 stream)
        assert st == T.TETRA_OK, T.tetra_strerror(st)
        torch.cuda.synchronize()
        assert T.tetra_noalloc_status(torch.cuda.current_device(), stream) == T.TETRA_OK
        assert torch.equal(out, ref), (mode, call)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_1710_10789_gb300 as T

    T.build()
    # 16 orbitals x 300000 energies x 8 bytes of partial sums exceed 32 MiB
    plan = T.Plan(4, 4, 4, 1, 16, 300000)
    dev = torch.device("cuda")
    eps, w = plan.empty_inputs()
    om = torch.linspace(-1, 1, 300000, device=dev)
    out = torch.empty((16, 300000), device=dev)
    st = T.tetra_dos_noalloc(plan.handle, eps.data_ptr(), w.data_ptr(), om.data_ptr(),
                             out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == T.TETRA_ENOMEM
