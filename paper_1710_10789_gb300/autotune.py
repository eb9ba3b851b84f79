"""Launch-shape autotuner for batched DOS launches (tetra_dos_batched).

The paper varies the number of energies and cubes handled per thread block
by hand and keeps the fastest (Sec. IV.B); here the same search runs
automatically. For one batch signature (the models' grids and energy counts,
bands, orbitals, mode, weight type) and one GPU it times each candidate box
shape of the forward kernel on the caller's own inputs, each as a replayed
CUDA graph, and keeps the fastest. Results are cached as JSON, keyed by the signature and the GPU,
so a later process with the same batch skips the search.

The launch shape never changes the result: the DOS is summed in exact
integers, so every candidate returns the same bits.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

from . import BatchPlan, TetraError, tetra_version

# Box shapes (cubes per side); the plan clips them to the smallest grid, and
# shapes that clip to one already timed are skipped.
BOX_CANDIDATES = ((4, 4, 2), (4, 4, 1), (4, 2, 2), (2, 4, 2), (2, 2, 4), (8, 4, 1), (8, 2, 2),
                  (4, 4, 4), (2, 2, 2))


def cache_path() -> str:
    """JSON cache file: $TETRA_TUNE_CACHE, else ~/.cache/paper_1710_10789_gb300/tune.json."""
    p = os.environ.get("TETRA_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1710_10789_gb300", "tune.json")


def gpu_identity(device: int = 0) -> dict:
    import torch
    props = torch.cuda.get_device_properties(device)
    return {"name": props.name, "sms": int(props.multi_processor_count),
            "cc": f"{props.major}.{props.minor}"}


def signature(grids, n_omegas, n_bands, n_orb, mode, weight_dtype, gpu: dict,
              version: str) -> tuple[str, dict]:
    """(hash, key) of a batch on a GPU. Model order is part of the key: the
    static schedule walks the models in the given order."""
    key = {"models": [[int(g[0]), int(g[1]), int(g[2]), int(nw)] for g, nw in zip(grids, n_omegas)],
           "n_bands": int(n_bands), "n_orb": int(n_orb), "mode": mode,
           "weight_dtype": weight_dtype, "gpu": gpu, "lib": version}
    h = hashlib.sha1(json.dumps(key, sort_keys=True).encode()).hexdigest()
    return h, key


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    """Writes the cache atomically (temporary file + rename)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def candidates(boxes=BOX_CANDIDATES):
    for b in boxes:
        yield {"box": [int(x) for x in b]}


def graph_time(plan: BatchPlan, eps, w, omega, reps: int = 3) -> float:
    """Median seconds of `reps` replays of a captured launch (after one replay
    that is not timed)."""
    import torch
    g, _ = plan.graph(eps, w, omega)
    g.replay()
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        g.replay()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
    times.sort()
    return times[len(times) // 2]


def tune_batched(grids, n_omegas, n_bands, n_orb, eps=None, w=None, omega=None, mode="point",
                 weight_dtype="f32", cands=None, reps: int = 3, use_cache: bool = True,
                 path: str | None = None, measure=None, gpu: dict | None = None,
                 version: str | None = None) -> dict:
    """Best launch shape for a batch: {"box": [bx, by, bz], "seconds": t,
    "timed": [...]} (from the cache when present).

    `measure(tune) -> seconds or None` times one candidate; by default it
    builds a BatchPlan with that tune and replays a captured launch over
    (eps, w, omega), lists of device tensors in the plan's layouts."""
    path = path or cache_path()
    gpu = gpu if gpu is not None else gpu_identity()
    version = version if version is not None else tetra_version()
    h, key = signature(grids, n_omegas, n_bands, n_orb, mode, weight_dtype, gpu, version)
    cache = load_cache(path) if use_cache else {}
    if h in cache and "tune" in cache[h]:
        return cache[h]["tune"]

    seen = set()

    def default_measure(tune):
        try:
            plan = BatchPlan(grids, n_omegas, n_bands, n_orb, mode=mode, weight_dtype=weight_dtype,
                             tune=tune)
        except TetraError:
            return None   # this shape does not fit the device
        eff = tuple(plan.box)
        if eff in seen:
            return None
        seen.add(eff)
        return graph_time(plan, eps, w, omega, reps)

    measure = measure or default_measure
    timed = []
    for tune in (cands if cands is not None else candidates()):
        t = measure(tune)
        if t is not None:
            timed.append({"box": list(tune["box"]), "seconds": t})
    if not timed:
        raise RuntimeError("no candidate launch shape could be timed")
    best = min(timed, key=lambda r: r["seconds"])
    result = {"box": best["box"], "seconds": best["seconds"], "timed": timed}
    if use_cache:
        cache = load_cache(path)
        cache[h] = {"key": key, "tune": result}
        save_cache(path, cache)
    return result
