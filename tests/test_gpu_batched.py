"""Batched DOS (tetra_dos_batched): many models with their own grids and energy
grids in one launch of the forward kernel. Checked against the single-model
path bit for bit (both sum exact integers, so any schedule gives the same
bits), against the FP64 oracle within 2e-5 * max, and through CUDA-graph
capture and replay."""
import os

import numpy as np
import pytest

import oracle
import tbgen
from helpers import tb_problem, to_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def T():
    import paper_1710_10789_gb300 as T
    T.build()
    assert torch.cuda.is_available()
    return T


def upload(T, layout, eps, w, n, wdtype):
    npw = {"f32": np.float32, "f16": np.float16, "bf16": np.float32}[wdtype]
    E, W = to_layout(eps, w, *n, layout.eps_stride, layout.w_stride, npw)
    dev = torch.device("cuda")
    Et, Wt = torch.from_numpy(E).to(dev), torch.from_numpy(W).to(dev)
    if wdtype == "bf16":
        Wt = Wt.to(torch.bfloat16)
    return Et, Wt


def rounded_weights(w, wdtype):
    if wdtype == "f16":
        return w.astype(np.float16).astype(np.float64)
    if wdtype == "bf16":
        return torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    return w.astype(np.float64)


def window(eps, n_omega, mode, frac=(0.0, 1.0), pad=0.1):
    """Energy grid over a fraction of the band range of one model."""
    lo, hi = float(eps.min()) - pad, float(eps.max()) + pad
    a, b = lo + frac[0] * (hi - lo), lo + frac[1] * (hi - lo)
    if mode == "point":
        return tbgen.uniform_grid(a, b, n_omega)
    return tbgen.bin_edges(a, b, n_omega)


def single_dos(T, n, nb, no, nw, mode, wdtype, Et, Wt, om):
    plan = T.Plan(*n, nb, no, nw, mode=mode, weight_dtype=wdtype)
    out = plan.dos(Et, Wt, om)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    return out.cpu().numpy()


# Ragged grids (not multiples of the box), own windows: full band range, a
# middle slice, a window entirely above the bands, and a single energy.
SMALL = [((9, 7, 6), 120, (0.0, 1.0)), ((16, 16, 16), 401, (0.0, 1.0)),
         ((12, 10, 8), 57, (0.3, 0.7)), ((5, 6, 7), 300, (0.0, 1.0)),
         ((20, 18, 16), 1000, (0.0, 1.0)), ((8, 8, 8), 64, (1.2, 1.5)),
         ((11, 13, 9), 1, (0.5, 0.5))]


@pytest.mark.parametrize("wdtype", ["f32", "bf16"])
@pytest.mark.parametrize("mode", ["point", "bin"])
def test_small_batch_matches_single_and_oracle(T, mode, wdtype):
    # (in bin mode the single-model launch spreads its tile adds over several
    # copies of the tile and the batch uses one: equal bits also check the
    # copies' add counts and flushes)
    specs = [s for s in SMALL if not (mode == "bin" and s[1] == 1)]
    probs = [tb_problem(40 + i, n) for i, (n, _, _) in enumerate(specs)]
    plan = T.BatchPlan([s[0] for s in specs], [s[1] for s in specs], 8, 8, mode=mode,
                       weight_dtype=wdtype)
    dev = torch.device("cuda")
    E, W, OM = [], [], []
    for m, ((n, nw, frac), (_, eps, w)) in enumerate(zip(specs, probs)):
        Et, Wt = upload(T, plan.layouts[m], eps, w, n, wdtype)
        E.append(Et)
        W.append(Wt)
        OM.append(torch.from_numpy(window(eps, nw, mode, frac)).to(dev))
    out = plan.dos(E, W, OM)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK
    for m, ((n, nw, frac), (_, eps, w)) in enumerate(zip(specs, probs)):
        g = out[m].cpu().numpy()
        s = single_dos(T, n, 8, 8, nw, mode, wdtype, E[m], W[m], OM[m])
        assert np.array_equal(g, s), m
        om = OM[m].cpu().numpy().astype(np.float64)
        r = oracle.dos(eps, rounded_weights(w, wdtype), *n, om, mode=mode, nthreads=NTHREADS)
        scale = np.max(np.abs(r))
        if scale == 0.0:
            assert np.all(g == 0.0), m
        else:
            assert np.max(np.abs(g - r)) <= TOL * scale, m


def test_batch_tuning_options_give_the_same_bits(T):
    """Box shape and CTAs per SM change only the launch shape, never the
    result."""
    specs = SMALL[:5]
    probs = [tb_problem(60 + i, n) for i, (n, _, _) in enumerate(specs)]
    dev = torch.device("cuda")
    ref = None
    for tune in (None, {"box": (2, 2, 2)}, {"box": (4, 2, 1)},
                 {"box": (1, 4, 4), "ctas_per_sm": 2}):
        plan = T.BatchPlan([s[0] for s in specs], [s[1] for s in specs], 8, 8, tune=tune)
        E, W, OM = [], [], []
        for m, ((n, nw, frac), (_, eps, w)) in enumerate(zip(specs, probs)):
            Et, Wt = upload(T, plan.layouts[m], eps, w, n, "f32")
            E.append(Et)
            W.append(Wt)
            OM.append(torch.from_numpy(window(eps, nw, "point", frac)).to(dev))
        out = [o.cpu().numpy() for o in plan.dos(E, W, OM)]
        assert plan.status() == T.TETRA_OK
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b), tune


def test_graph_capture_and_replay(T):
    """One captured launch recomputes every model's DOS from the current input
    contents; the result equals a direct call on the same data."""
    specs = SMALL[:4]
    plan = T.BatchPlan([s[0] for s in specs], [s[1] for s in specs], 8, 8)
    dev = torch.device("cuda")
    data = []
    for seed in (70, 80):
        probs = [tb_problem(seed + i, n) for i, (n, _, _) in enumerate(specs)]
        d = []
        for m, ((n, nw, frac), (_, eps, w)) in enumerate(zip(specs, probs)):
            Et, Wt = upload(T, plan.layouts[m], eps, w, n, "f32")
            d.append((Et, Wt, torch.from_numpy(window(eps, nw, "point", frac)).to(dev)))
        data.append(d)
    E = [x[0].clone() for x in data[0]]
    W = [x[1].clone() for x in data[0]]
    OM = [x[2].clone() for x in data[0]]
    g, out = plan.graph(E, W, OM)
    g.replay()
    torch.cuda.synchronize()
    first = [o.cpu().numpy() for o in out]
    # new contents, same buffers
    for m in range(len(specs)):
        E[m].copy_(data[1][m][0])
        W[m].copy_(data[1][m][1])
        OM[m].copy_(data[1][m][2])
    g.replay()
    torch.cuda.synchronize()
    second = [o.cpu().numpy() for o in out]
    assert plan.status() == T.TETRA_OK
    for k, res in ((0, first), (1, second)):
        direct = plan.dos([x[0] for x in data[k]], [x[1] for x in data[k]], [x[2] for x in data[k]])
        torch.cuda.synchronize()
        for a, b in zip(res, direct):
            assert np.array_equal(a, b.cpu().numpy())
    assert not all(np.array_equal(a, b) for a, b in zip(first, second))


def test_batched_64_models_full_size(T):
    """The batched workload at full size: 64 seeded models, cubic grids N ~
    U{16..96}, 500-3000 energies each over its own band window, 8 bands x 8
    orbitals, FP32, one launch. Every model equals its single-model result bit
    for bit; the oracle agrees at sampled energies of four models (two
    smallest, two largest); a bin-mode batch over the same data meets the
    per-orbital sum rule of every model."""
    specs = tbgen.batched_problems(64)
    grids = [(s["n"],) * 3 for s in specs]
    nws = [s["n_omega"] for s in specs]
    plan = T.BatchPlan(grids, nws, 8, 8)
    bplan = T.BatchPlan(grids, nws, 8, 8, mode="bin")
    dev = torch.device("cuda")
    E, W, OM, ED, expect = [], [], [], [], []
    host = {}
    order = np.argsort([s["n"] for s in specs])
    check = set(order[:2].tolist() + order[-2:].tolist())
    for m, s in enumerate(specs):
        n = grids[m]
        eps, w = tbgen.synthetic_bands(s["seed"], *n, 8, 8)
        eps, w = eps.astype(np.float32), w.astype(np.float32)
        Et, Wt = upload(T, plan.layouts[m], eps, w, n, "f32")
        E.append(Et)
        W.append(Wt)
        om = window(eps, s["n_omega"], "point")
        OM.append(torch.from_numpy(om).to(dev))
        ED.append(torch.from_numpy(tbgen.bin_edges(float(om[0]), float(om[-1]), s["n_omega"])).to(dev))
        expect.append(w.astype(np.float64).sum(1).mean(0))
        if m in check:
            host[m] = (eps, w)
    out = plan.dos(E, W, OM)
    outb = bplan.dos(E, W, ED)
    torch.cuda.synchronize()
    assert plan.status() == T.TETRA_OK and bplan.status() == T.TETRA_OK
    for m, s in enumerate(specs):
        n = grids[m]
        g = out[m].cpu().numpy()
        single = single_dos(T, n, 8, 8, s["n_omega"], "point", "f32", E[m], W[m], OM[m])
        assert np.array_equal(g, single), m
        # integral of DOS_s over a window holding every band = k-average of
        # sum_n w[k, n, s]; exact in bin mode
        ed = ED[m].cpu().numpy().astype(np.float64)
        integral = (outb[m].cpu().numpy().astype(np.float64) * np.diff(ed)[None, :]).sum(1)
        np.testing.assert_allclose(integral, expect[m], rtol=1e-4, err_msg=str(m))
        if m in check:
            om = OM[m].cpu().numpy().astype(np.float64)
            idx = np.linspace(0, s["n_omega"] - 1, 6).astype(int)[1:-1]
            eps, w = host[m]
            r = oracle.dos(eps, w, *n, om[idx], nthreads=NTHREADS)
            assert np.max(np.abs(g[:, idx] - r)) <= TOL * np.max(np.abs(g)), m


def test_autotuner_on_a_small_batch(T, tmp_path):
    """The tuner times candidate shapes through graph replays and returns one
    whose plan gives the same bits as the default plan."""
    from paper_1710_10789_gb300 import autotune

    specs = SMALL[:5]
    grids, nws = [s[0] for s in specs], [s[1] for s in specs]
    probs = [tb_problem(90 + i, n) for i, (n, _, _) in enumerate(specs)]
    base = T.BatchPlan(grids, nws, 8, 8)
    dev = torch.device("cuda")
    E, W, OM = [], [], []
    for m, ((n, nw, frac), (_, eps, w)) in enumerate(zip(specs, probs)):
        Et, Wt = upload(T, base.layouts[m], eps, w, n, "f32")
        E.append(Et)
        W.append(Wt)
        OM.append(torch.from_numpy(window(eps, nw, "point", frac)).to(dev))
    ref = [o.cpu().numpy() for o in base.dos(E, W, OM)]
    best = autotune.tune_batched(grids, nws, 8, 8, E, W, OM, path=str(tmp_path / "tune.json"),
                                 cands=list(autotune.candidates(((4, 4, 2), (2, 2, 2), (4, 2, 1)))))
    assert best["seconds"] > 0 and len(best["timed"]) >= 2
    tuned = T.BatchPlan(grids, nws, 8, 8, tune=best)
    for a, b in zip(tuned.dos(E, W, OM), ref):
        assert np.array_equal(a.cpu().numpy(), b)
