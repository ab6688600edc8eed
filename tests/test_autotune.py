"""Host logic of the launch-shape autotuner (size classes, the choice among gated
candidates, the JSON cache) and, on the GPU, one tuning run on a small batch."""
import numpy as np
import pytest

from paper_1401_4950_gb300 import autotune


def test_size_class_buckets():
    assert autotune.size_class([8192, 8192, 8192]) == "nmat4_nmax8192_rows32768"
    assert autotune.size_class([1000]) == "nmat1_nmax1024_rows1024"
    assert autotune.size_class([32, 1024, 500]) == "nmat4_nmax1024_rows2048"
    assert autotune.size_class([]) == "empty"
    # the class depends on the orders only, not on their order in the batch
    assert autotune.size_class([5, 700, 9]) == autotune.size_class([700, 9, 5])
    # tree options that change the work are part of the class; unset ones are not
    assert autotune.size_class([1000], {"abs_split": -1, "erep": 0}) == \
        "nmat1_nmax1024_rows1024_abs_split-1"
    assert autotune.size_class([1000], {"abs_split": 0}) == autotune.size_class([1000])


def test_choose_skips_candidates_that_failed_the_gates():
    timings = {"0,0": 5.0, "2,48": 3.0, "8,24": 4.0}
    assert autotune.choose(timings, {"0,0": True, "2,48": False, "8,24": True}) == "8,24"
    assert autotune.choose(timings, {"0,0": True, "2,48": True, "8,24": True}) == "2,48"
    assert autotune.choose(timings, {}) is None


def test_cache_round_trip(tmp_path, monkeypatch):
    import paper_1401_4950_gb300 as mr3
    path = str(tmp_path / "tune.json")
    monkeypatch.setattr(autotune, "_device_key", lambda: "fake-gpu|0123")
    sizes = [300, 400]
    assert autotune.lookup(sizes, path) is None
    o = autotune.tuned_opts(sizes, path)
    assert (o.rqi_team, o.bisect_warps) == (0, 0)
    autotune._store("fake-gpu|0123", autotune.size_class(sizes),
                    {"rqi_team": 8, "bisect_warps": 24}, path)
    # a second class in the same file leaves the first in place
    autotune._store("fake-gpu|0123", "nmat1_nmax1_rows1", {"rqi_team": 2, "bisect_warps": 64}, path)
    assert autotune.lookup(sizes, path)["rqi_team"] == 8
    o = autotune.tuned_opts(sizes, path, prec=mr3.FP64)
    assert (o.rqi_team, o.bisect_warps, o.prec) == (8, 24, mr3.FP64)
    # an explicit argument wins over the cache
    assert autotune.tuned_opts(sizes, path, rqi_team=2).rqi_team == 2
    # another device (or library build) does not see the entry
    monkeypatch.setattr(autotune, "_device_key", lambda: "other-gpu|0123")
    assert autotune.lookup(sizes, path) is None


def test_cache_ignores_a_damaged_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    monkeypatch.setattr(autotune, "_device_key", lambda: "fake-gpu|0123")
    assert autotune.lookup([10], str(path)) is None
    autotune._store("fake-gpu|0123", "c", {"rqi_team": 2}, str(path))
    assert autotune._load(str(path)) == {"fake-gpu|0123": {"c": {"rqi_team": 2}}}


@pytest.mark.gpu
def test_tune_small_batch(cuda, tmp_path):
    import torch
    import paper_1401_4950_gb300 as mr3
    import testmats as tm
    sizes = [64, 200, 512, 97]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.concatenate([tm.uniform(500 + b, n) for b, n in enumerate(sizes)])
    e = np.concatenate([np.r_[tm.uniform(600 + b, n - 1), 0.0] for b, n in enumerate(sizes)])
    dt, et = torch.tensor(d, device=cuda), torch.tensor(e, device=cuda)
    path = str(tmp_path / "tune.json")
    rec = autotune.tune(n_off, dt, et, reps=1, warmup=0, path=path)
    assert set(rec["timings"]) == {"%d,%d" % c for c in autotune.CANDIDATES}
    # every launch shape meets the gates on these matrices
    assert all(r <= autotune.GATE and q <= autotune.GATE and st in (0, 1)
               for r, q, st in rec["gates"].values()), rec
    assert rec["ms"] is not None, rec
    assert autotune.lookup(sizes, path)["rqi_team"] == rec["rqi_team"]
    o = autotune.tuned_opts(sizes, path)
    assert (o.rqi_team, o.bisect_warps) == (rec["rqi_team"], rec["bisect_warps"])
    # the tuned shape gives the same eigenvalues as the library's defaults (to rounding)
    _, w0, _, _, _ = mr3.stemr_batched(n_off, dt, et)
    _, w1, _, _, _ = mr3.stemr_batched(n_off, dt, et, opts=o)
    tn = float(w0.abs().max())
    assert float((w0 - w1).abs().max()) <= 4 * max(sizes) * 2.0 ** -53 * tn
