"""Host-side logic on the CPU: the seeded input generator both sides consume, the pixel
sample of the parity tests and the benchmark, and the autotuner's candidate sets, proxy
workloads, signatures and cache (its timing runs on the GPU)."""
import json

import numpy as np

from paper_2005_05386_gb300 import autotune, scenes


def test_splitmix64_matches_the_published_sequence():
    """SplitMix64 (Steele, Lea and Flood 2014) from state 0: the first outputs of the reference
    generator."""
    g = scenes.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_form_equals_the_stream():
    """The vectorised hash of state k * golden is the k-th output of the sequential stream."""
    g = scenes.SplitMix64(12345)
    seq = [g.next_u64() for _ in range(8)]
    states = np.array([(12345 + k * 0x9E3779B97F4A7C15) & scenes.MASK64 for k in range(8)], np.uint64)
    assert [int(v) for v in scenes.splitmix64_hash(states)] == seq
    u = scenes.SplitMix64(7)
    draws = [u.uniform(-4.0, 4.0) for _ in range(1000)]
    assert min(draws) >= -4.0 and max(draws) < 4.0 and abs(np.mean(draws)) < 0.3


def test_pixel_sample_is_seeded_and_of_the_asked_size():
    n = 1920 * 1080
    a = scenes.pixel_sample(n, 1, 0.01)
    b = scenes.pixel_sample(n, 1, 0.01)
    c = scenes.pixel_sample(n, 2, 0.01)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(np.diff(a) > 0) and a[0] >= 0 and a[-1] < n
    sd = np.sqrt(n * 0.01 * 0.99)
    assert abs(len(a) - 0.01 * n) < 4 * sd
    assert len(scenes.pixel_sample(n, 1, 0.0)) == 0 and len(scenes.pixel_sample(100, 1, 1.0)) == 100


def test_autotuner_candidates_follow_the_metric():
    w = scenes.config_1080p_64()
    c = autotune.candidates(w)
    assert all(set(x) == set(autotune.KNOBS) for x in c)
    assert len({tuple(sorted(x.items())) for x in c}) == len(c)          # no duplicates
    assert {x["cull_grid"] for x in c} == set(autotune.CANDIDATE_GRIDS)
    assert {x["ctas_per_sm"] for x in c} == set(autotune.CANDIDATE_CTAS)
    assert {x["tile_shape"] for x in c} == set(autotune.CANDIDATE_TILES)
    assert {x["sum_lists"] for x in c} == {0, 1}
    assert {x["refill"] for x in c} == {0, 1} and all(x["ctas_per_sm"] == 0 for x in c if x["refill"] == 1)
    assert all(x["sum_lists"] == 0 for x in c if x["cull_grid"] == -1)  # dense sums take no lists
    assert all(x["cull_grid"] == -1 for x in c if x["rays_per_thread"] == 2)
    assert {x["batch_order"] for x in c} == {0} and {x["batch_order"] for x in autotune.candidates(w, True)} == {0, 1}
    for other in (scenes.config_1080p_twist(), scenes.config_local_lattice(K=8)):
        oc = autotune.candidates(other)
        assert {x["cull_grid"] for x in oc} == {-1} and {x["rays_per_thread"] for x in oc} == {1}
        assert {x["tile_shape"] for x in oc} == set(autotune.CANDIDATE_TILES)
        assert {x["refill"] for x in oc} == {0, 1} and all(x["ctas_per_sm"] == 0 for x in oc if x["refill"] == 1)
    aniso = scenes.config_1080p_64()
    aniso.metric.sigma = aniso.metric.sigma * np.array([1.0, 1.2, 0.9], np.float32)
    assert {x["cull_grid"] for x in autotune.candidates(aniso)} == {-1}
    untruncated = scenes.config_1080p_64()
    untruncated.metric.cutoff = 0.0
    assert {x["cull_grid"] for x in autotune.candidates(untruncated)} == {-1}


def test_autotuner_proxy_and_signature():
    w = scenes.config_1080p_64()
    p = autotune.proxy(w)
    assert 0.9 * 2 ** 20 <= p.width * p.height <= 2 ** 20
    assert abs(p.width / p.height - 16 / 9) < 0.02
    assert p.metric is w.metric and p.h == w.h and p.max_steps == w.max_steps
    small = scenes.config_parity_64()
    assert autotune.proxy(small) is small and autotune.proxy(scenes.config_1080p_64(width=960, height=540)).width == 960
    s = autotune.signature(w)
    assert s == autotune.signature(scenes.scaled(w, 1900, 1080))  # same power-of-two size bucket
    assert s != autotune.signature(scenes.scaled(w, 960, 540))
    assert s != autotune.signature(scenes.config_4k_1024())


def test_autotuner_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuning.json"
    monkeypatch.setenv("RGEO_TUNING_CACHE", str(path))
    assert autotune._load() == {}
    db = {"GB300|k0-K64": {"cull_grid": 128, "rays_per_thread": 1, "ms": 12.5}}
    autotune._store(db)
    assert autotune._load() == db
    assert json.load(open(path)) == db
