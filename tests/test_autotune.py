"""CPU checks of the batched-launch autotuner's host logic: signature, JSON
cache and selection (timings injected; no GPU)."""
import json

import pytest

pytest.importorskip("torch")
from paper_1710_10789_gb300 import autotune  # noqa: E402

GPU = {"name": "test-gpu", "sms": 152, "cc": "10.3"}
GRIDS = [(16, 16, 16), (40, 40, 40), (96, 96, 96)]
NW = [500, 1200, 3000]


def test_signature_depends_on_every_part_of_the_key():
    h0, key = autotune.signature(GRIDS, NW, 8, 8, "point", "f32", GPU, "0.1.0")
    assert key["models"][2] == [96, 96, 96, 3000]
    variants = [
        autotune.signature(GRIDS[::-1], NW[::-1], 8, 8, "point", "f32", GPU, "0.1.0"),
        autotune.signature(GRIDS, [500, 1200, 2999], 8, 8, "point", "f32", GPU, "0.1.0"),
        autotune.signature(GRIDS, NW, 8, 4, "point", "f32", GPU, "0.1.0"),
        autotune.signature(GRIDS, NW, 8, 8, "bin", "f32", GPU, "0.1.0"),
        autotune.signature(GRIDS, NW, 8, 8, "point", "bf16", GPU, "0.1.0"),
        autotune.signature(GRIDS, NW, 8, 8, "point", "f32", dict(GPU, sms=148), "0.1.0"),
        autotune.signature(GRIDS, NW, 8, 8, "point", "f32", GPU, "0.2.0"),
    ]
    hashes = {h0} | {v[0] for v in variants}
    assert len(hashes) == 1 + len(variants)
    assert autotune.signature(GRIDS, NW, 8, 8, "point", "f32", GPU, "0.1.0")[0] == h0


def test_tuner_picks_the_fastest_and_caches_it(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    calls = []

    def measure(tune):
        calls.append(tuple(tune["box"]))
        if tune["box"] == [8, 4, 1]:
            return None                       # does not fit: skipped
        return {(4, 4, 2): 3.0, (2, 2, 4): 1.5}.get(tuple(tune["box"]), 2.0)

    r = autotune.tune_batched(GRIDS, NW, 8, 8, path=path, measure=measure, gpu=GPU, version="0.1.0")
    assert r["box"] == [2, 2, 4] and r["seconds"] == 1.5
    assert len(r["timed"]) == len(autotune.BOX_CANDIDATES) - 1
    assert len(calls) == len(autotune.BOX_CANDIDATES)
    stored = json.load(open(path))
    h, _ = autotune.signature(GRIDS, NW, 8, 8, "point", "f32", GPU, "0.1.0")
    assert stored[h]["tune"]["box"] == [2, 2, 4]
    # a second call with the same signature reads the cache and times nothing
    calls.clear()
    r2 = autotune.tune_batched(GRIDS, NW, 8, 8, path=path, measure=measure, gpu=GPU, version="0.1.0")
    assert r2 == r and not calls
    # another batch adds its own entry and keeps the first
    autotune.tune_batched(GRIDS[:2], NW[:2], 8, 8, path=path, measure=measure, gpu=GPU,
                          version="0.1.0")
    assert len(json.load(open(path))) == 2


def test_tuner_without_any_fitting_shape_raises(tmp_path):
    with pytest.raises(RuntimeError):
        autotune.tune_batched(GRIDS, NW, 8, 8, path=str(tmp_path / "t.json"),
                              measure=lambda t: None, gpu=GPU, version="0.1.0")


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}
    r = autotune.tune_batched(GRIDS, NW, 8, 8, path=str(path), measure=lambda t: 1.0, gpu=GPU,
                              version="0.1.0")
    assert r["box"] == list(autotune.BOX_CANDIDATES[0])
