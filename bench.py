"""Benchmark of the linear tetrahedron orbital-resolved DOS on GB300.

One step = the whole hot path on one synthetic tight-binding model: H(k) and
the batched Hermitian eigensolve on the GPU (tetra_eig), then the orbital-resolved
DOS by the linear tetrahedron method (tetra_dos). Default workload: seeded
8-orbital tetragonal model, 256^3 k-grid (100.7M tetrahedra), 8 bands,
8 orbitals, 4000 energies on [eps_min - 0.1, eps_max + 0.1], FP32 weights,
point mode. Inputs (4.9 GB of eigen-data) are larger than L2.

Metric: tetrahedron x band x energy updates per second, counting every
(tetrahedron, band, energy) triple the method defines (the dense count the
paper's thread-per-energy kernel evaluates); the in-window count is reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank integrates its own seeded model (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tetrahedron*band*omega updates/sec"
UNIT = "updates/s"
# FP32 lanes per SM on GB300 (4 partitions x 32) and the SM count
FP32_LANES_PER_SM = 128
# algorithmic FP32 FMA-pipe instructions: per in-window (tetra, band, energy)
# triple with n_orb = 8, and per (tetra, band) item (sort, window, reciprocals)
OPS_PER_TRIPLE = 44
OPS_PER_ITEM = 40
# DRAM bytes (read + write) of one tetra_dos_fwd_kernel launch from an ncu
# capture of the 128^3, 4000-energy, FP32, point-mode launch, scaled by the
# number of boxes to other cubic grids (the traffic is per box: halo reads of
# the TMA boxes). Valid only for the kernel source it was taken from: first 16
# hex digits of the SHA-256 of csrc/dos.cu up to the reduce kernels (the
# forward kernel and every device function it calls); otherwise the bench
# reports null.
DOS_TRAFFIC_CAPTURE = {"dos_fwd_sha256": "3ddeea97f2fb5a4a", "grid": 128, "n_omega": 4000,
                       "bytes": 691929856 + 4707840}
DOS_FWD_END = b"// Single model: dos[s][w0+j] = u * sum over CTAs of the int64 partials (exact)."


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--n-omega", type=int, default=4000)
    ap.add_argument("--weight-dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--mode", default="point", choices=["point", "bin"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip e2e and extra measurements")
    ap.add_argument("--variant", default=None,
                    choices=["differentiation", "paper_shape", "lindhard", "spectral_t0", "chi0_real_t0",
                             "near_balance", "integrated"],
                    help="run one extra workload alone and print its JSON (for profiling)")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def model_arrays(model):
    p = np.concatenate([model["onsite"], model["t"].real.ravel(), model["t"].imag.ravel()])
    return p.astype(np.float32), model["R"].astype(np.int32)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def in_window_count(torch, eps, n, nb, omega, mode, zc=16):
    """Exact number of (tetra, band, energy) triples with the energy strictly
    inside (E1, E4) (point mode) or the bin overlapping it (bin mode), for an
    n^3 grid in the tetra layout (zc cube planes at a time)."""
    table = [(0, 1, 2, 5), (1, 2, 3, 5), (0, 2, 4, 5), (2, 3, 5, 7), (2, 4, 5, 6), (2, 5, 6, 7)]
    om = omega.double()
    total = 0
    for z0 in range(0, n, zc):
        nz = min(zc, n - z0)
        planes = eps[z0:z0 + nz + 1, :, :, :nb].double()  # (nz+1, n+1, n+1, nb)
        for t in table:
            cs = []
            for c in t:
                dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
                cs.append(planes[dz:dz + nz, dy:dy + n, dx:dx + n, :])
            st = torch.stack(cs, 0)
            e1 = st.min(0).values.reshape(-1)
            e4 = st.max(0).values.reshape(-1)
            if mode == "point":
                lo = torch.searchsorted(om, e1, right=True)
                hi = torch.searchsorted(om, e4, right=False)
            else:
                lo = torch.searchsorted(om, e1, right=True) - 1
                hi = torch.searchsorted(om, e4, right=False)
                lo = lo.clamp(min=0)
                hi = hi.clamp(max=om.numel() - 1)
            total += int((hi - lo).clamp(min=0).sum().item())
    return total


def dos_traffic(n, n_omega, mode, weight_dtype):
    """Captured DRAM bytes per forward launch scaled to an n^3 grid, or None
    when the capture does not describe this kernel source or configuration."""
    import hashlib
    c = DOS_TRAFFIC_CAPTURE
    src = os.path.join(ROOT, "paper_1710_10789_gb300", "csrc", "dos.cu")
    text = open(src, "rb").read()
    end = text.find(DOS_FWD_END)
    sha = hashlib.sha256(text[:end]).hexdigest()[:16] if end > 0 else None
    if sha != c["dos_fwd_sha256"] or n_omega != c["n_omega"] or mode != "point" or weight_dtype != "f32":
        return None
    return c["bytes"] * (n / c["grid"]) ** 3


def alu_roofline(torch, dev, triples, items, ms):
    """Algorithmic FP32-pipe throughput of the forward kernel against the FP32
    peak of the GPU (SMs x 128 lanes x 2 flop x max SM clock)."""
    mp = {}
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_max = float(mp.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops = 2.0 * (OPS_PER_TRIPLE * triples + OPS_PER_ITEM * items)
    ach = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "tetra_dos_fwd_kernel", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                           "(sm_max_mhz of measured MEASURED_PEAKS.json)",
            "algorithmic": f"{OPS_PER_TRIPLE} FMA-pipe ops x {triples} in-window triples + "
                           f"{OPS_PER_ITEM} x {items} tetra-bands"}


def eig_ops_per_point(n_orb=8, n_R=7):
    """Algorithmic FP32 FMA-pipe operations per k-point of the eigensolver
    (textbook counts for an n x n complex Hermitian matrix, n = n_orb):
    H(k) from n_R hopping matrices (4 FMA per upper-triangle entry and R),
    Householder reduction to tridiagonal form (16/3 n^3 real flops), implicit
    QR on the real tridiagonal with the rotations accumulated (6 n^3 flops),
    back-transformation of the eigenvectors by the reflectors (n^3 complex
    multiply-adds) and the squared moduli (2 n^2)."""
    n = n_orb
    h_build = n_R * (n * (n + 1) // 2) * 4
    tridiag = 16 * n ** 3 // 6
    qr = 3 * n ** 3
    back = 4 * n ** 3
    return h_build + tridiag + qr + back + 2 * n * n


def eig_bwd_ops_per_point(n_orb=8, n_R=7):
    """Algorithmic FP32 FMA-pipe operations per k-point of the eigensolver
    adjoint: the forward's eigensolver with its eigenvectors (recomputed;
    eig_ops_per_point without the squared moduli), the pair sums of S
    (n(n-1)/2 pairs x n orbitals: a weight difference, two complex products,
    two accumulations), Y = S V^T (n^2 complex dot products of length n),
    the Hermitian half of Z = conj(V) Y, and the phase sums (4 per complex
    output (R, i, j), plus the diagonal)."""
    n = n_orb
    return (eig_ops_per_point(n, n_R) - 2 * n * n + 6 * n * n * (n - 1) // 2 + 4 * n ** 3 + 2 * n * n * (n + 1)
            + 4 * n_R * n * n + n)


def eig_roofline(torch, dev, points, ms):
    """The eigensolver's algorithmic FP32 throughput against the same FP32 peak."""
    mp = {}
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_max = float(mp.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ops = eig_ops_per_point()
    ach = 2.0 * ops * points / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "tetra_eig_kernel", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak,
            "algorithmic": f"{ops} FMA-pipe ops per k-point x {points} padded k-points (H(k), Householder, "
                           "tridiagonal QR with rotations, back-transformation, |V|^2)"}


def time_dos(torch, plan, eps, w, omega, out, steps, warmup):
    """Mean ms of the DOS call alone (events on the launching stream)."""
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.dos(eps, w, omega, out=out)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(steps):
        plan.dos(eps, w, omega, out=out)
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def sec_iv_protocol(times_ms, runs=7, keep=5):
    """The paper's timing protocol (Sec. IV): of `runs` timed repetitions, the
    mean of the `keep` fastest, with the largest deviation of any repetition
    from that mean. Fewer repetitions than `runs`: all of them, the fastest
    len - 2 kept."""
    r = list(times_ms[:runs])
    k = keep if len(r) >= runs else max(1, len(r) - 2)
    m = statistics.mean(sorted(r)[:k])
    return {"runs": len(r), "kept_fastest": k, "mean_ms": m, "min_ms": min(r), "max_ms": max(r),
            "max_dev_pct": 100.0 * max(abs(x - m) for x in r) / m}


def near_balance_workload(torch, T, n, params, R, steps, warmup, local, nbins=200):
    """The configuration with the fewest energies per tetrahedron, closest to
    the HBM roofline: n^3 grid, 8 bands x 8 orbitals, 200 bins (bin mode), the
    orbital weights stored in FP32 / FP16 / BF16. Per weight type: DOS time,
    the algorithmic input bytes of one launch (eps + weights of every padded
    point, read once) and their rate against the measured HBM copy bandwidth,
    and the deviation from the FP32-weight DOS."""
    import tbgen
    mp = {}
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(mp.get("hbm_gbs", 6800.0))
    out = {"workload": f"{n}^3 grid, 8 bands, 8 orbitals, {nbins} bins (bin mode), FP32 arithmetic",
           "hbm_peak_gbs": hbm, "hbm_peak_source": "hbm_gbs of MEASURED_PEAKS.json" if mp else "fallback"}
    edges = d32 = None
    for wd in ("f32", "f16", "bf16"):
        plan = T.Plan(n, n, n, 8, 8, nbins, mode="bin", weight_dtype=wd, device=local)
        eps, w = plan.empty_inputs()
        plan.eig(params, R, eps, w)
        torch.cuda.synchronize()
        if edges is None:
            lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
            edges = torch.from_numpy(tbgen.bin_edges(lo, hi, nbins)).to(eps.device)
        d = torch.empty((8, nbins), dtype=torch.float32, device=eps.device)
        ms = time_dos(torch, plan, eps, w, edges, d, steps, warmup)
        assert plan.status() == T.TETRA_OK
        nbytes = (n + 1) ** 3 * 8 * (4 + 8 * (4 if wd == "f32" else 2))
        gbs = nbytes / (ms * 1e-3) / 1e9
        if d32 is None:
            d32 = d.clone()
        out[wd] = {"dos_ms": ms, "algorithmic_input_bytes": nbytes, "input_gbs": gbs,
                   "frac_of_hbm": gbs / hbm,
                   "max_rel_dev_vs_f32_weights": float((d - d32).abs().max() / d32.abs().max())}
        del eps, w, plan
        torch.cuda.empty_cache()
    return out


def precision_variants(torch, T, n, nw, mode, params, R, omega, dos32, steps, warmup, local):
    """Same workload with the orbital weights stored in FP16 / BF16 (FP32
    arithmetic): DOS time, roofline and the largest deviation from the FP32-weight
    DOS relative to its maximum."""
    out = {}
    for wd in ("f16", "bf16"):
        plan = T.Plan(n, n, n, 8, 8, nw, mode=mode, weight_dtype=wd, device=local)
        eps, w = plan.empty_inputs()
        plan.eig(params, R, eps, w)
        d = torch.empty_like(dos32)
        ms = time_dos(torch, plan, eps, w, omega, d, steps, warmup)
        assert plan.status() == T.TETRA_OK
        dev_ = float((d - dos32).abs().max() / dos32.abs().max())
        out[wd] = {"dos_ms": ms, "dense_updates_per_s": 6 * n ** 3 * 8 * nw / (ms * 1e-3),
                   "weight_bytes": int(w.numel() * w.element_size()),
                   "max_rel_dev_vs_f32_weights": dev_}
        del eps, w, plan
        torch.cuda.empty_cache()
    return out


def differentiation_workload(torch, T, steps, warmup, local):
    """Loss = sum (bin DOS - target)^2 on the 8-orbital model, 64^3 grid, 200
    bins; one step = forward (eig + bin DOS) and backward through both
    adjoints to the model parameters. Target from a second seeded model."""
    import tbgen
    from paper_1710_10789_gb300.autograd import model_dos
    dev = torch.device("cuda", local)
    n, nbins = 64, 200
    plan = T.Plan(n, n, n, 8, 8, nbins, mode="bin", device=local)
    pt, Rt = (torch.from_numpy(a).to(dev) for a in model_arrays(tbgen.tb_model(1, n_orb=8)))
    et, wt = plan.eig(pt, Rt)
    lo, hi = float(et[..., :8].min()) - 0.1, float(et[..., :8].max()) + 0.1
    edges = torch.from_numpy(tbgen.bin_edges(lo, hi, nbins)).to(dev)
    target = plan.dos(et, wt, edges).clone()
    p0, R0 = (torch.from_numpy(a).to(dev) for a in model_arrays(tbgen.tb_model(0, n_orb=8)))
    params = p0.clone().requires_grad_(True)

    def step():
        params.grad = None
        loss = ((model_dos(params, R0, edges, plan) - target) ** 2).sum()
        loss.backward()
        return loss

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        step()
    b.record(s_)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # the two adjoints alone, on the step's eigen-data and seeded gradients
    eps, w = plan.eig(params.detach(), R0)
    gen = torch.Generator(device=dev).manual_seed(5)
    gd = torch.randn((8, nbins), device=dev, generator=gen)
    ge = torch.randn(eps.shape, device=dev, generator=gen)
    gw = torch.randn(w.shape, device=dev, generator=gen)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        a.record(s_)
        for _ in range(steps):
            fn()
        b.record(s_)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    dos_bwd_ms = timed(lambda: plan.dos_backward(eps, w, edges, gd))
    eig_bwd_ms = timed(lambda: plan.eig_backward(params.detach(), R0, ge, gw))
    roof = eig_roofline(torch, dev, n ** 3, eig_bwd_ms)
    ops = eig_bwd_ops_per_point()
    roof.update({"kernel": "tetra_eig_bwd_kernel", "achieved": 2.0 * ops * n ** 3 / (eig_bwd_ms * 1e-3) / 1e12,
                 "algorithmic": f"{ops} FMA-pipe ops per k-point x {n ** 3} k-points (eigensolver with "
                                "eigenvectors recomputed, pair sums of S, S V^T, Hermitian half of conj(V) S V^T, "
                                "phase sums)"})
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"workload": "8-orbital model, 64^3 grid, 200 bins, loss = sum (bin DOS - target)^2, "
                        "forward + backward to 904 model parameters (eig, bin DOS, both adjoints)",
            "ms_per_step": ms, "grad_norm": float(params.grad.norm()),
            "dos_backward_ms": dos_bwd_ms, "eig_backward_ms": eig_bwd_ms, "eig_backward_roofline": roof}


def batched_workload(torch, T, mode, steps, warmup, local, count_window=True):
    """64 seeded 8-orbital models, cubic grids N ~ U{16..96}, 500-3000 energies
    over each model's own band window; eigen-data by tetra_eig; box shape from
    the autotuner (timed on these inputs, cached); all DOS in one
    graph-captured launch. Returns timing and counts."""
    import tbgen
    from paper_1710_10789_gb300 import autotune
    dev = torch.device("cuda", local)
    specs = tbgen.batched_problems(64)
    grids = [(s["n"],) * 3 for s in specs]
    nws = [s["n_omega"] for s in specs]
    E, W, OM = [], [], []
    for m, s in enumerate(specs):
        model = tbgen.tb_model(s["seed"], n_orb=8)
        p_np, R_np = model_arrays(model)
        plan = T.Plan(*grids[m], 8, 8, s["n_omega"], mode=mode, device=local)
        eps, w = plan.eig(torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev))
        torch.cuda.synchronize()
        lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
        om = tbgen.uniform_grid(lo, hi, s["n_omega"]) if mode == "point" else \
            tbgen.bin_edges(lo, hi, s["n_omega"])
        E.append(eps)
        W.append(w)
        OM.append(torch.from_numpy(om).to(dev))
    t0 = time.perf_counter()
    tune = autotune.tune_batched(grids, nws, 8, 8, E, W, OM, mode=mode)
    tune_s = time.perf_counter() - t0
    bplan = T.BatchPlan(grids, nws, 8, 8, mode=mode, tune=tune, device=local)
    g, out = bplan.graph(E, W, OM)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        g.replay()
    b.record(s_)
    torch.cuda.synchronize()
    assert bplan.status() == T.TETRA_OK
    ms = a.elapsed_time(b) / steps
    # the same 64 DOS as 64 single-model launches, for comparison
    plans = [T.Plan(*grids[m], 8, 8, nws[m], mode=mode, device=local) for m in range(64)]
    outs = [torch.empty_like(o) for o in out]
    for m in range(64):
        plans[m].dos(E[m], W[m], OM[m], out=outs[m])
    torch.cuda.synchronize()
    a.record(s_)
    for m in range(64):
        plans[m].dos(E[m], W[m], OM[m], out=outs[m])
    b.record(s_)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    same = all(torch.equal(x, y) for x, y in zip(out, outs))
    dense = sum(6 * s["n"] ** 3 * 8 * s["n_omega"] for s in specs)
    items = sum(6 * s["n"] ** 3 * 8 for s in specs)
    triples = None
    if count_window:
        triples = sum(in_window_count(torch, E[m], specs[m]["n"], 8, OM[m], mode) for m in range(64))
    return {"ms": ms, "dense": dense, "items": items, "triples": triples, "box": list(bplan.box),
            "ctas": bplan.grid, "tune": tune, "tune_seconds": tune_s, "sequential_ms": seq_ms,
            "bitwise_equal_to_single": same, "specs": specs, "E": E, "W": W, "OM": OM}


def paper_shape_workload(torch, T, steps, warmup, local):
    """The paper's benchmark shape (Sec. IV, Table II largest case): 60 x 60 x 10
    k-grid (n_k = 36000), 8 bands, DOS projected on 5 orbitals, 1024 energies,
    FP32; synthetic 8-orbital model (the paper's FeSe hoppings are not given).
    Eigensolve and DOS timed separately (the paper's timings exclude the
    diagonalisation)."""
    import tbgen
    dev = torch.device("cuda", local)
    n = (60, 60, 10)
    p_np, R_np = model_arrays(tbgen.tb_model(21, n_orb=8))
    params, R = torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev)
    plan = T.Plan(*n, 8, 5, 1024, device=local)
    eps, w = plan.empty_inputs()
    plan.eig(params, R, eps, w)
    torch.cuda.synchronize()
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    omega = torch.from_numpy(tbgen.uniform_grid(lo, hi, 1024)).to(dev)
    dos = torch.empty((5, 1024), dtype=torch.float32, device=dev)
    s_ = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.eig(params, R, eps, w)
        plan.dos(eps, w, omega, out=dos)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(s_)
        plan.eig(params, R, eps, w)
        ev[i][1].record(s_)
        plan.dos(eps, w, omega, out=dos)
        ev[i][2].record(s_)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    eig_ms = statistics.mean(a.elapsed_time(b) for a, b, c in ev)
    dos_ms = statistics.mean(b.elapsed_time(c) for a, b, c in ev)
    dense = 6 * 36000 * 8 * 1024
    return {"workload": "60x60x10 k-grid (n_k = 36000), 8 bands, 5 projected orbitals, 1024 energies, "
                        "FP32, synthetic 8-orbital model",
            "eig_ms": eig_ms, "dos_ms": dos_ms, "dense_updates_per_s_dos_only": dense / (dos_ms * 1e-3),
            "paper_context": "paper Table II, n_k = 36000, 1024 energies, 64 per block: GeForce GTX 970 "
                             "kernels only 732.0 ms, Intel i7-4790K single core 121515 ms "
                             "(FeSe model, 5 Fe-d orbitals plus the total DOS)"}


def integrated_workload(torch, T, n, eps, w, steps, warmup, local):
    """The orbital occupation n_s(E) (TETRA_INTEGRATED mode) at 1000 energies
    over the band window (one energy chunk) and at 6000 (three chunks), and
    the Fermi level of half filling (4 of 8 bands; one untimed call first),
    on the benchmark's own eigen-data."""
    dev = torch.device("cuda", local)
    nw = 1000
    plan = T.Plan(n, n, n, 8, 8, nw, mode="integrated", device=local)
    lo, hi = float(eps[..., :8].min()) - 0.1, float(eps[..., :8].max()) + 0.1
    import tbgen
    omega = torch.from_numpy(tbgen.uniform_grid(lo, hi, nw)).to(dev)
    out = torch.empty((8, nw), dtype=torch.float32, device=dev)
    for _ in range(warmup):
        plan.dos(eps, w, omega, out=out)
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        plan.dos(eps, w, omega, out=out)
    b.record(s_)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    ms = a.elapsed_time(b) / steps
    top = float(out[:, -1].sum())
    nw6 = 6000
    plan6 = T.Plan(n, n, n, 8, 8, nw6, mode="integrated", device=local)
    omega6 = torch.from_numpy(tbgen.uniform_grid(lo, hi, nw6)).to(dev)
    out6 = torch.empty((8, nw6), dtype=torch.float32, device=dev)
    plan6.dos(eps, w, omega6, out=out6)
    torch.cuda.synchronize()
    a.record(s_)
    for _ in range(steps):
        plan6.dos(eps, w, omega6, out=out6)
    b.record(s_)
    torch.cuda.synchronize()
    assert plan6.status() == T.TETRA_OK
    ms6 = a.elapsed_time(b) / steps
    plan.fermi_level(eps, w, 4.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ef = plan.fermi_level(eps, w, 4.0)
    fermi_s = time.perf_counter() - t0
    return {"workload": f"occupation n_s(E) at {nw} and at {nw6} energies and the Fermi level of 4 electrons "
                        f"per spin, {n}^3 grid, 8 bands, 8 orbitals, FP32",
            "integrated_ms": ms, "integrated_6000_ms": ms6, "fermi_level_eV": ef, "fermi_level_seconds": fermi_s,
            "total_occupation_top": top}


def lindhard_workload(torch, T, steps, warmup, local):
    """Spectral function of the bare susceptibility S(q, w) (tetra_pair_bands +
    tetra_dos on the 64 transition bands) on the 8-orbital model, 64^3 grid,
    q = (16, 0, 0), kT = 0.025 eV, chemical potential at 4 electrons per spin,
    400 energies on [0, 4] eV."""
    import tbgen
    dev = torch.device("cuda", local)
    n = 64
    p_np, R_np = model_arrays(tbgen.tb_model(0, n_orb=8))
    plan = T.Plan(n, n, n, 8, 8, 16, device=local)
    eps, w = plan.eig(torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    pplan = T.Plan(n, n, n, 64, 1, 400, device=local)
    ep, wp = pplan.empty_inputs()
    omega = torch.from_numpy(tbgen.uniform_grid(0.0, 4.0, 400)).to(dev)
    out = torch.empty((1, 400), dtype=torch.float32, device=dev)
    from paper_1710_10789_gb300 import tetra_pair_bands, _ptr, _stream_handle

    def step():
        st = tetra_pair_bands(plan.handle, _ptr(eps), (16, 0, 0), 0.025, mu, pplan.handle, _ptr(ep), _ptr(wp),
                              _stream_handle(None))
        assert st == T.TETRA_OK
        pplan.dos(ep, wp, omega, out=out)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        step()
    b.record(s_)
    torch.cuda.synchronize()
    assert pplan.status() == T.TETRA_OK
    return {"workload": "bare-susceptibility spectral function S(q, w), 8-orbital model, 64^3 grid, "
                        "q = (16, 0, 0), kT = 0.025 eV, 64 transition bands, 400 energies on [0, 4] eV",
            "ms_per_evaluation": a.elapsed_time(b) / steps, "chemical_potential_eV": mu}


def oracle_sample_eigendata(n, planes, seed=0):
    """FP64 eigen-data (LAPACK) of the seeded 8-orbital model on point planes
    z = 0 .. planes of the n^3 grid, natural layout: a grid of planes + 1
    planes whose first `planes` cube planes are cube planes 0 .. planes - 1 of
    the full grid."""
    import tbgen
    model = tbgen.tb_model(seed)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    H = []
    for z in range(planes + 1):
        kf = np.stack([x.ravel() / n, y.ravel() / n, np.full(x.size, z / n)], 1)
        Hz = np.zeros((kf.shape[0], 8, 8), np.complex128)
        Hz[:, np.arange(8), np.arange(8)] = model["onsite"]
        for R, t in zip(model["R"], model["t"]):
            ph = np.exp(2j * np.pi * (kf @ R.astype(float)))
            Hz += ph[:, None, None] * t[None] + np.conj(ph)[:, None, None] * t.conj().T[None]
        H.append(Hz)
    ev, V = np.linalg.eigh(np.concatenate(H))
    w = np.abs(np.transpose(V, (0, 2, 1))) ** 2
    return ev, w


def spectral_t0_workload(torch, T, steps, warmup, local):
    """Spectral function of the bare susceptibility at T = 0 by exact
    double-band clipping of every tetrahedron (tetra_spectral_t0) on the
    8-orbital model, 64^3 grid, q = (16, 0, 0), chemical potential at 4
    electrons per spin, 400 energies on [0, 4] eV (point mode)."""
    import tbgen
    dev = torch.device("cuda", local)
    n = 64
    p_np, R_np = model_arrays(tbgen.tb_model(0, n_orb=8))
    plan = T.Plan(n, n, n, 8, 8, 16, device=local)
    eps, w = plan.eig(torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    omega = torch.from_numpy(tbgen.uniform_grid(0.0, 4.0, 400)).to(dev)
    out = torch.empty((400,), dtype=torch.float32, device=dev)
    for _ in range(warmup):
        plan.spectral_t0(eps, (16, 0, 0), mu, omega, out=out)
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        plan.spectral_t0(eps, (16, 0, 0), mu, omega, out=out)
    b.record(s_)
    torch.cuda.synchronize()
    assert plan.spectral_status() == T.TETRA_OK
    return {"workload": "bare-susceptibility spectral function S(q, w) at T = 0 (exact double-band clipping), "
                        "8-orbital model, 64^3 grid, q = (16, 0, 0), 64 band pairs, 400 energies on [0, 4] eV",
            "ms_per_evaluation": a.elapsed_time(b) / steps, "chemical_potential_eV": mu,
            "spectral_weight_0_to_4eV": float(out.sum()) * 4.0 / 399}


def chi0_real_t0_workload(torch, T, steps, warmup, local):
    """Real part of the T = 0 bare susceptibility (tetra_chi0_real_t0) on the
    8-orbital model, 64^3 grid, q = (16, 0, 0), chemical potential at 4
    electrons per spin, 400 energies on [0, 4] eV."""
    import tbgen
    dev = torch.device("cuda", local)
    n = 64
    p_np, R_np = model_arrays(tbgen.tb_model(0, n_orb=8))
    plan = T.Plan(n, n, n, 8, 8, 16, device=local)
    eps, w = plan.eig(torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev))
    mu = plan.fermi_level(eps, w, 4.0)
    omega = torch.from_numpy(tbgen.uniform_grid(0.0, 4.0, 400)).to(dev)
    out = torch.empty((400,), dtype=torch.float32, device=dev)
    for _ in range(warmup):
        plan.chi0_real_t0(eps, (16, 0, 0), mu, omega, out=out)
    torch.cuda.synchronize()
    s_ = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s_)
    for _ in range(steps):
        plan.chi0_real_t0(eps, (16, 0, 0), mu, omega, out=out)
    b.record(s_)
    torch.cuda.synchronize()
    assert plan.spectral_status() == T.TETRA_OK
    return {"workload": "real part of the bare susceptibility Re chi0(q, w) at T = 0 (exact double-band "
                        "clipping, principal-value averages), 8-orbital model, 64^3 grid, q = (16, 0, 0), "
                        "64 band pairs, 400 energies on [0, 4] eV",
            "ms_per_evaluation": a.elapsed_time(b) / steps, "chemical_potential_eV": mu,
            "re_chi0_at_0_eV": float(out[0]), "re_chi0_at_4_eV": float(out[-1])}


def cpu_baseline(n, n_omega, seed=0, planes=None, threads=None, stride=1, omega=None, keep=False):
    """The FP64 oracle on the host cores over a bounded sample of the same
    workload: `planes` cube planes (n x n x planes cubes) of the n^3 grid, all
    bands, every `stride`-th energy of the grid (the oracle is dense over
    energies, so its cost per update does not depend on which energies),
    eigen-data from LAPACK. `omega` is the benchmark's energy grid (else one
    over the sample's own band window). The oracle gives each thread a block
    of whole cube planes, so the sample has one plane per thread unless
    `planes` says otherwise. keep=True also returns the sample's eigen-data,
    energies and oracle DOS (for the accuracy figures)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    planes = planes or threads
    threads = min(threads, planes)
    ev, w = oracle_sample_eigendata(n, planes, seed)
    if omega is None:
        e_lo, e_hi = ev.min() - 0.1, ev.max() + 0.1
        omega = np.linspace(e_lo, e_hi, n_omega).astype(np.float32)
    omega = np.ascontiguousarray(np.asarray(omega, np.float64)[::stride])
    n3 = planes + 1
    t0 = time.perf_counter()
    d = oracle.dos(ev, w, n, n, n3, omega, z_range=(0, planes), nthreads=threads)
    dt = time.perf_counter() - t0
    updates = n * n * planes * 6 * 8 * omega.size
    every = f"1 in {stride} of {n_omega}" if stride > 1 else f"all {n_omega}"
    out = {"value": updates / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{planes} cube plane(s) of the {n}^3 grid ({n * n * planes * 6} tetrahedra) "
                     f"x 8 bands x {omega.size} energies ({every}), FP64, dense over energies",
           "seconds": dt}
    if keep:
        # the oracle's DOS of the slab, scaled to the full grid's volume factor
        out["_sample"] = {"ev": ev, "w": w, "planes": planes, "omega": omega, "stride": stride,
                          "dos": d * (n3 / n)}
    return out


def sample_accuracy(torch, T, n, omega_dev, params, R, local, smp, threads, sub=8):
    """Accuracy of the GPU path on the cpu_baseline sample (cube planes
    0 .. planes - 1 of the benchmark grid, every `stride`-th energy), against
    the FP64 oracle:
      * parity: tetra_eig + tetra_dos on a slab plan of those planes against
        the oracle on the same eigen-data (the FP32 values the kernel reads,
        widened), FP32 weights and FP16 / BF16 weights (the oracle fed the
        same rounded weights);
      * storage: the FP16 / BF16-weight DOS against the oracle on the
        unrounded FP32 weights;
      * end to end: GPU eigensolver + DOS against LAPACK + the oracle.
    Errors are max |difference| / max |oracle DOS| over the sampled energies
    (every `sub`-th energy of the cpu_baseline sample)."""
    import oracle
    planes, stride = smp["planes"], smp["stride"] * sub
    nw = omega_dev.numel()
    idx = np.arange(0, nw, smp["stride"])[::sub]
    om_s = np.ascontiguousarray(smp["omega"][::sub])
    d64 = smp["dos"][:, ::sub]
    out = {"sample": f"cube planes 0..{planes - 1} of the {n}^3 grid, {idx.size} energies (1 in {stride})",
           "reference": "FP64 oracle (oracle/), same sample as cpu_baseline"}
    ref32 = None
    for wd in ("f32", "f16", "bf16"):
        plan = T.Plan(n, n, n, 8, 8, nw, weight_dtype=wd, z_range=(0, planes), device=local)
        eps, w = plan.empty_inputs()
        plan.eig(params, R, eps, w)
        g = plan.dos(eps, w, omega_dev)
        torch.cuda.synchronize()
        assert plan.status() == T.TETRA_OK
        g = g.cpu().numpy().astype(np.float64)[:, idx]
        E = eps[:planes + 1, :n, :n, :8].cpu().numpy().astype(np.float64).reshape(-1, 8)
        W = w[:planes + 1, :n, :n, :64].to(torch.float32).cpu().numpy().astype(np.float64).reshape(-1, 8, 8)
        del eps, w, plan
        torch.cuda.empty_cache()
        r = oracle.dos(E, W, n, n, planes + 1, om_s, z_range=(0, planes), nthreads=threads)
        r *= (planes + 1) / n
        scale = np.max(np.abs(r))
        rec = {"parity_max_rel_err": float(np.max(np.abs(g - r)) / scale),
               "end_to_end_max_rel_err": float(np.max(np.abs(g - d64)) / np.max(np.abs(d64)))}
        if wd == "f32":
            ref32 = r
        else:
            rec["vs_oracle_on_unrounded_weights_max_rel_err"] = float(np.max(np.abs(g - ref32)) /
                                                                      np.max(np.abs(ref32)))
        out[wd] = rec
    return out


def config_of(args, world):
    """The workload both arms report: the model, grid, energies and layout."""
    n, nw = args.grid, args.n_omega
    esize = 4 if args.weight_dtype == "f32" else 2
    eig_bytes = (n + 1) ** 3 * 8 * (4 + 8 * esize)   # eps + weights, halo points included
    return {"workload": f"tb8_{n}cube_{nw}w_{args.mode}_{args.weight_dtype}",
            "model": "seeded 8-orbital tetragonal tight binding", "grid": [n, n, n],
            "tetrahedra": 6 * n ** 3, "n_bands": 8, "n_orb": 8, "n_omega": nw,
            "mode": args.mode, "weight_dtype": args.weight_dtype,
            "l2": "inputs larger than L2 (eigen-data %.1f GB)" % (eig_bytes / 1e9),
            "parallelism": f"{world} independent model(s), one per GPU"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    # bounded sample per step (one cube plane per host thread, 1 in 32
    # energies: a few seconds), so that K + W steps end within minutes
    import oracle  # noqa: F401
    res = []
    for i in range(warm + steps):
        r = cpu_baseline(args.grid, args.n_omega, stride=32)
        if i >= warm:
            res.append(r)
    v = statistics.mean(r["value"] for r in res)
    cb = dict(res[0])
    cb["value"] = v
    cb.pop("seconds", None)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": statistics.mean(r["seconds"] for r in res) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config_of(args, world),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import paper_1710_10789_gb300 as T
    import tbgen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T.build()
    if args.variant is not None:
        if args.variant == "near_balance":
            p_np, R_np = model_arrays(tbgen.tb_model(rank, n_orb=8))
            r = near_balance_workload(torch, T, args.grid, torch.from_numpy(p_np).to(dev),
                                      torch.from_numpy(R_np).to(dev), args.steps, args.warmup, local)
        elif args.variant == "integrated":
            p_np, R_np = model_arrays(tbgen.tb_model(rank, n_orb=8))
            n = args.grid
            plan = T.Plan(n, n, n, 8, 8, args.n_omega, device=local)
            eps, w = plan.eig(torch.from_numpy(p_np).to(dev), torch.from_numpy(R_np).to(dev))
            r = integrated_workload(torch, T, n, eps, w, args.steps, args.warmup, local)
        else:
            fn = {"differentiation": differentiation_workload, "paper_shape": paper_shape_workload,
                  "lindhard": lindhard_workload, "spectral_t0": spectral_t0_workload,
                  "chi0_real_t0": chi0_real_t0_workload}[args.variant]
            r = fn(torch, T, args.steps, args.warmup, local)
        if rank == 0:
            print(json.dumps(r), flush=True)
        return
    n, nw = args.grid, args.n_omega
    model = tbgen.tb_model(rank, n_orb=8)
    p_np, R_np = model_arrays(model)
    params = torch.from_numpy(p_np).to(dev)
    R = torch.from_numpy(R_np).to(dev)
    plan = T.Plan(n, n, n, 8, 8, nw, mode=args.mode, weight_dtype=args.weight_dtype, device=local)
    eps, w = plan.empty_inputs()
    ws = plan.workspace()
    stream = torch.cuda.current_stream()
    # energy window from the eigenvalues the DOS kernel consumes (fixed before timing)
    plan.eig(params, R, eps, w)
    torch.cuda.synchronize()
    emin = float(eps[..., :8].min())
    emax = float(eps[..., :8].max())
    if args.mode == "point":
        omega = torch.from_numpy(tbgen.uniform_grid(emin - 0.1, emax + 0.1, nw)).to(dev)
    else:
        omega = torch.from_numpy(tbgen.bin_edges(emin - 0.1, emax + 0.1, nw)).to(dev)
    dos = torch.empty((8, nw), dtype=torch.float32, device=dev)

    def step():
        plan.eig(params, R, eps, w)
        plan.dos(eps, w, omega, out=dos)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    # timed region: K steps, per-kernel events on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.eig(params, R, eps, w)
            ev[i][1].record(stream)
            plan.dos(eps, w, omega, out=dos)
            ev[i][2].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    eig_ms = statistics.mean(a.elapsed_time(b) for a, b, c in ev)
    dos_ms = statistics.mean(b.elapsed_time(c) for a, b, c in ev)
    protocol = {"step": sec_iv_protocol([a.elapsed_time(c) for a, b, c in ev]),
                "dos": sec_iv_protocol([b.elapsed_time(c) for a, b, c in ev]),
                "eig": sec_iv_protocol([a.elapsed_time(b) for a, b, c in ev])}
    ms_step = total_ms / args.steps
    n_tet = 6 * n ** 3
    dense = n_tet * 8 * nw
    value = dense * world / (ms_step * 1e-3)
    if rank != 0:
        return
    triples = in_window_count(torch, eps, n, 8, omega, args.mode)
    clocks = clk.summary()
    roof = alu_roofline(torch, dev, triples, n_tet * 8, dos_ms)
    eig_roof = eig_roofline(torch, dev, (n + 1) ** 3, eig_ms)
    roof["traffic"] = dos_traffic(n, nw, args.mode, args.weight_dtype)
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 128^3 launch "
                              "scaled by boxes (see profiles/)")
    # end to end through the public API: host model in, host DOS out
    e2e = None
    if not args.quick:
        p_host = torch.from_numpy(p_np).pin_memory()
        R_host = torch.from_numpy(R_np).pin_memory()
        d_host = torch.empty((8, nw), dtype=torch.float32).pin_memory()
        p_dev = torch.empty_like(params)
        R_dev = torch.empty_like(R)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            p_dev.copy_(p_host, non_blocking=True)
            R_dev.copy_(R_host, non_blocking=True)
            plan.eig(p_dev, R_dev, eps, w)
            plan.dos(eps, w, omega, out=dos)
            d_host.copy_(dos, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        e2e = {"value": dense / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(p_host.numel() * 4 + R_host.numel() * 4),
               "d2h_bytes_per_step": int(d_host.numel() * 4), "ms_per_step": e2e_ms}
    variants = None
    if not args.quick:
        variants = {"precision": precision_variants(torch, T, n, nw, args.mode, params, R, omega, dos,
                                                    args.steps, args.warmup, local)}
        bt = batched_workload(torch, T, args.mode, args.steps, args.warmup, local)
        variants["batched"] = {
            "workload": "64 seeded 8-orbital models, N^3 grids N ~ U{16..96}, 500-3000 energies each, "
                        "FP32, one graph-captured launch (memset + forward + per-model scale)",
            "ms_per_launch": bt["ms"], "dense_updates_per_s": bt["dense"] / (bt["ms"] * 1e-3),
            "in_window_updates_per_s": bt["triples"] / (bt["ms"] * 1e-3),
            "in_window_triples": bt["triples"], "tetra_bands": bt["items"],
            "box": bt["box"], "ctas": bt["ctas"], "autotune_seconds": bt["tune_seconds"],
            "autotune_timed": bt["tune"].get("timed"),
            "sequential_single_launches_ms": bt["sequential_ms"],
            "bitwise_equal_to_single_launches": bt["bitwise_equal_to_single"],
            "roofline": alu_roofline(torch, dev, bt["triples"], bt["items"], bt["ms"])}
        del bt
        torch.cuda.empty_cache()
        variants["differentiation"] = differentiation_workload(torch, T, args.steps, args.warmup, local)
        variants["paper_shape"] = paper_shape_workload(torch, T, args.steps, args.warmup, local)
        if args.mode == "point" and args.weight_dtype == "f32":
            variants["integrated"] = integrated_workload(torch, T, n, eps, w, args.steps, args.warmup, local)
        variants["lindhard"] = lindhard_workload(torch, T, args.steps, args.warmup, local)
        variants["spectral_t0"] = spectral_t0_workload(torch, T, args.steps, args.warmup, local)
        variants["chi0_real_t0"] = chi0_real_t0_workload(torch, T, args.steps, args.warmup, local)
        variants["near_balance"] = near_balance_workload(torch, T, n, params, R, args.steps, args.warmup, local)
    cb = None
    if not args.no_cpu_baseline:
        om_np = omega.cpu().numpy()
        cb = cpu_baseline(n, nw, seed=0, stride=4, omega=om_np, keep=True)
        cb.pop("seconds", None)
        smp = cb.pop("_sample")
        cb["accuracy"] = sample_accuracy(torch, T, n, omega, params, R, local, smp, cb["cores"])
        del smp
        # the paper's protocol times its CPU code on one core
        one = cpu_baseline(n, nw, seed=0, planes=1, threads=1, stride=8, omega=om_np)
        cb["single_core"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(args, world),
        "step": {"eig_ms": eig_ms, "dos_ms": dos_ms},
        "sec_iv_protocol": protocol,
        "in_window_updates_per_s": triples / (dos_ms * 1e-3),
        "dense_updates_per_s_dos_only": dense / (dos_ms * 1e-3),
        "in_window_triples": triples,
        "roofline": roof, "eig_roofline": eig_roof, "cpu_baseline": cb, "e2e": e2e, "clocks": clocks, "variants": variants,
        "gpu_launches": 3 * args.steps,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
