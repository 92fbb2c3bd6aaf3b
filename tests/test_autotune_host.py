"""Host-side logic of the autotuner (no GPU): the stratified batch sample,
the choice of the fastest converged candidate, and the per-(GPU, build, key)
cache.  The timed solve is replaced by a table of fixed times."""
import json

import pytest

from paper_1907_01995_gb300 import autotune


def test_batch_sample_spans_the_work_quantiles():
    work = [5, 1, 9, 3, 7, 2, 8, 4, 6, 10, 0, 11]
    idx = autotune.batch_sample(work, 4)
    assert idx == sorted(idx) and len(set(idx)) == 4
    got = sorted(work[i] for i in idx)
    assert got[0] == min(work) and got[-1] == max(work)   # both ends of the mix
    assert autotune.batch_sample(work, 20) == sorted(range(len(work)), key=lambda i: (work[i], i))
    # ties broken by index: the same sample every time
    assert autotune.batch_sample([1] * 10, 3) == autotune.batch_sample([1] * 10, 3)


def _fake_times(table):
    calls = []

    def fake(A, b, common, storage, form, grid, reps=2):
        calls.append((storage, form, grid))
        return table.get((storage, form, grid))
    return fake, calls


def test_choose_takes_the_fastest_converged_candidate(monkeypatch, tmp_path):
    monkeypatch.setenv("RAC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda device: "testgpu")
    times = {("fp32", "gram", 0): 3e-3, ("fp32", "gram", 16): 2.5e-3,
             ("bf16", "gram", 16): 1.9e-3, ("bf16", "gram", 32): None,   # did not converge
             ("bf16", "residual", 64): 2.2e-3}
    fake, calls = _fake_times(times)
    monkeypatch.setattr(autotune, "_time_solve", fake)
    res = autotune.choose(None, None, {}, key="w1")
    assert (res["storage"], res["form"], res["grid"]) == ("bf16", "gram", 16)
    assert res["seconds"] == 1.9e-3
    n_grid = sum(len(autotune.DEFAULT_GRIDS[f]) for _, f in autotune.DEFAULT_CANDIDATES)
    assert len(calls) == n_grid == len(res["table"])
    # cached per (GPU, build, key): the second call times nothing
    calls.clear()
    again = autotune.choose(None, None, {}, key="w1")
    assert calls == [] and again["grid"] == 16
    cache = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("testgpu|") and k.endswith("|w1") for k in cache)
    # another key is tuned afresh
    autotune.choose(None, None, {}, key="w2")
    assert len(calls) == n_grid


def test_choose_fails_loudly_when_nothing_converges(monkeypatch, tmp_path):
    monkeypatch.setenv("RAC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    fake, _ = _fake_times({})
    monkeypatch.setattr(autotune, "_time_solve", fake)
    with pytest.raises(RuntimeError):
        autotune.choose(None, None, {}, key="none", use_cache=False)
