"""Host logic of the launch-shape autotuner (no GPU): candidate choice,
tie-breaking, JSON cache round trip and reuse."""

from paper_1107_5719_gb300 import autotune as A


def test_pick_fastest_and_tie_breaks_to_fewer_groups():
    assert A.pick({1: 5.0, 2: 3.0, 4: 3.5, 8: 9.0}) == 2
    assert A.pick({1: 3.0, 2: 3.0, 4: 3.0}) == 1


def test_tune_caches_and_reuses(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def timer(g):
        calls.append(g)
        return {1: 10.0, 2: 7.0, 4: 6.0, 8: 6.5}[g]

    key = A.cache_key(65, 65, 65, 1024, 0, 152)
    best, t = A.tune(key, timer, cache_path=path)
    assert best == 4 and calls == [1, 2, 4, 8]
    calls.clear()
    best2, t2 = A.tune(key, timer, cache_path=path)
    assert best2 == 4 and calls == [] and t2 == t
    best3, _ = A.tune(key, lambda g: {1: 1.0, 2: 2.0, 4: 3.0, 8: 4.0}[g], cache_path=path,
                      refresh=True)
    assert best3 == 1
    assert A.load_cache(path)[key]["groups"] == 1


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text("{not json")
    assert A.load_cache(str(path)) == {}
    best, _ = A.tune("k", lambda g: float(g), cache_path=str(path))
    assert best == 1


def test_key_distinguishes_shape_precision_and_device():
    keys = {A.cache_key(65, 65, 65, 1024, 0, 152), A.cache_key(65, 65, 65, 1024, 1, 152),
            A.cache_key(65, 65, 65, 1024, 0, 148), A.cache_key(129, 129, 129, 1024, 0, 152)}
    assert len(keys) == 4


def test_pairs_of_groups_and_threads_round_trip_through_the_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    ms = {(g, t): 10.0 - g * 0.5 + (t == 128) * 0.1 for (g, t) in A.CANDIDATES_FP32}
    best, _ = A.tune("k32", lambda c: ms[c], A.CANDIDATES_FP32, cache_path=path)
    assert best == (8, 64)
    calls = []
    best2, t2 = A.tune("k32", lambda c: calls.append(c) or 0.0, A.CANDIDATES_FP32, cache_path=path)
    assert best2 == (8, 64) and not calls and set(t2) == set(A.CANDIDATES_FP32)


def test_fp32_candidates_cover_every_block_size_and_group_count():
    assert {t for _, t in A.CANDIDATES_FP32} == {64, 128, 256}
    assert {g for g, _ in A.CANDIDATES_FP32} == set(A.CANDIDATES)
