"""Host-side logic that runs without a GPU: the Section 3 time-step rule, the
seeded ensemble and request generators of the batched and served workloads,
and the autotuner's cache and selection (its timing step is replaced by a
fake, so no kernel runs)."""
import json

import numpy as np
import pytest

from paper_1610_09146_gb300 import autotune, workloads


# ------------------------------------------------------------ Section 3 dt rule


@pytest.mark.parametrize("n,dt", [(64, 3.385e-3), (128, 1.6925e-3), (256, 8.4625e-4), (384, 5.641666666666667e-4),
                                  (512, 4.23125e-4)])
def test_time_step_halves_per_grid_doubling(n, dt):
    assert workloads.dt_for_grid(n) == pytest.approx(dt, rel=1e-15)


@pytest.mark.parametrize("n", [32, 48])
def test_grids_below_64_keep_the_64_cube_step(n):
    assert workloads.dt_for_grid(n) == workloads.dt_for_grid(64)


# ------------------------------------------------------------ batched ensemble


def test_ensemble_is_seeded_and_within_its_distributions():
    a = workloads.ensemble()
    b = workloads.ensemble()
    assert a == b
    assert len(a) == 64
    grids = [s["n"] for s in a]
    assert set(grids) == set(workloads.ENSEMBLE_GRIDS)  # 64 draws hit all five sizes
    for s in a:
        assert 400 <= s["Re"] <= 3200 and 0.1 <= s["Mach"] <= 0.4
        assert s["Pr"] == 0.71 and s["gamma"] == 1.4 and s["steps"] == 100
        assert s["dt"] == workloads.dt_for_grid(s["n"])
    assert workloads.ensemble(seed=1) != a


def test_ensemble_grid_draws_are_roughly_uniform():
    grids = np.array([s["n"] for s in workloads.ensemble(count=5000, seed=7)])
    counts = np.array([(grids == g).sum() for g in workloads.ENSEMBLE_GRIDS])
    assert np.all(np.abs(counts - 1000) < 5 * np.sqrt(1000))


# ------------------------------------------------------------ request stream


def test_requests_are_a_seeded_poisson_stream():
    r = workloads.requests()
    assert r == workloads.requests()
    assert len(r) == 400
    t = np.array([q["t"] for q in r])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # mean inter-arrival 1/20 s; 400 exponential gaps: standard error 5 %
    assert abs(gaps.mean() * 20.0 - 1.0) < 0.2
    # exponential gaps: coefficient of variation 1
    assert 0.8 < gaps.std() / gaps.mean() < 1.2


def test_request_parameters_within_their_ranges():
    r = workloads.requests()
    allowed = set(range(48, 193, 16))
    for q in r:
        assert q["n"] in allowed
        assert 50 <= q["steps"] <= 500
        assert 400 <= q["Re"] <= 3200 and 0.1 <= q["Mach"] <= 0.4
        assert q["dtype"] in ("f32", "f64")
        assert q["dt"] == workloads.dt_for_grid(q["n"])
    assert [q["id"] for q in r] == list(range(len(r)))
    frac32 = np.mean([q["dtype"] == "f32" for q in r])
    assert 0.4 < frac32 < 0.6


def test_request_options():
    r = workloads.requests(count=50, rate=0.9, grids=[64], steps_range=(7, 7))
    assert len(r) == 50 and {q["n"] for q in r} == {64} and {q["steps"] for q in r} == {7}
    assert r[-1]["t"] > 50 / 0.9 / 3  # a 0.9 req/s stream spans tens of seconds


# ------------------------------------------------------------ autotuner


def test_copies_fill_about_eight_million_points():
    assert autotune.copies_for(32) == (8 << 20) // 32**3
    assert autotune.copies_for(128) == 4
    assert autotune.copies_for(512) == 4
    for n in (32, 48, 64, 96, 128, 192):
        assert autotune.copies_for(n) * n**3 >= min(8 << 20, 4 * n**3) - n**3


def test_cache_round_trip_and_corrupt_file(tmp_path):
    p = tmp_path / "sub" / "cache.json"
    assert autotune._load(str(p)) == {}
    autotune._save(str(p), {"a": 1})
    assert json.loads(p.read_text()) == {"a": 1}
    p.write_text("{not json")
    assert autotune._load(str(p)) == {}


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    """The autotuner with a fake device name and a fake timer: recompute-all is
    faster for grids up to 64, store-some above; tile 1024 is best."""
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "FakeGPU")
    calls = []

    def timer(n, dtype, family, tile, steps=4, warmup=2):
        calls.append((n, dtype, family, tile))
        base = 1.0 if (family == "recompute_all") == (n <= 64) else 2.0
        return base * autotune.copies_for(n) * (1.0 + abs(tile - 1024) / 1e4)

    monkeypatch.setattr(autotune, "time_candidate", timer)
    return str(tmp_path / "tune.json"), calls


def test_tune_times_every_candidate_once_then_uses_the_cache(fake_gpu):
    path, calls = fake_gpu
    fam, tile, ms = autotune.tune(48, "f32", path=path)
    assert (fam, tile) == ("recompute_all", 1024) and ms == pytest.approx(1.0)
    assert len(calls) == len(autotune.FAMILIES) * len(autotune.TILES)
    entry = json.load(open(path))[autotune.key("FakeGPU", "f32", 48)]
    assert len(entry["candidates"]) == len(calls)
    assert autotune.tune(48, "f32", path=path) == (fam, tile, ms)
    assert len(calls) == len(autotune.FAMILIES) * len(autotune.TILES)  # cache hit: nothing timed
    autotune.tune(48, "f32", path=path, refresh=True)
    assert len(calls) == 2 * len(autotune.FAMILIES) * len(autotune.TILES)


def test_choose_assigns_each_grid_its_tuned_family(fake_gpu):
    path, calls = fake_gpu
    specs = [dict(n=32), dict(n=128), dict(n=(96, 96, 128)), dict(n=32, Re=900.0)]
    out, best = autotune.choose(specs, "f64", path=path)
    assert sorted(best) == [32, 128]
    assert [s["algorithm"] for s in out] == ["recompute_all", "store_some", "store_some", "recompute_all"]
    assert all(s["tile_points"] == 1024 for s in out)
    assert out[3]["Re"] == 900.0 and "algorithm" not in specs[0]
    assert {c[0] for c in calls} == {32, 128}
