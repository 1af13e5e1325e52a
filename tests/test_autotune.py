"""Host logic of the launch-shape autotuner (no GPU): candidate choice,
tie-breaking, JSON cache round trip and reuse."""

import pytest

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


def test_fp32_launch_shapes_round_trip_through_the_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    ms = {(g, t, o): 10.0 - g * 0.5 + (t == 128) * 0.1 - (o == 2) * 0.05
          for (g, t, o) in A.CANDIDATES_FP32}
    best, _ = A.tune("k32", lambda c: ms[c], A.CANDIDATES_FP32, cache_path=path)
    assert best == (8, 64, 2)
    calls = []
    best2, t2 = A.tune("k32", lambda c: calls.append(c) or 0.0, A.CANDIDATES_FP32, cache_path=path)
    assert best2 == (8, 64, 2) and not calls and set(t2) == set(A.CANDIDATES_FP32)


def test_fp32_candidates_cover_every_block_size_group_count_and_order():
    assert {t for _, t, _ in A.CANDIDATES_FP32} == {64, 128, 256}
    assert {g for g, _, _ in A.CANDIDATES_FP32} == set(A.CANDIDATES)
    assert {o for _, _, o in A.CANDIDATES_FP32} == {1, 2}
    assert len(set(A.CANDIDATES_FP32)) == 24


@pytest.mark.gpu
def test_autotune_solver_and_batch_on_gpu(tmp_path):
    """The tuner times every candidate on the GPU, caches the winner and
    applies it; J is unchanged by the tuned launch shape."""
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_5719_gb300 import build as B
    B.build()
    from paper_1107_5719_gb300 import rt3d as R, workloads as W
    R.load()
    path = str(tmp_path / "tune.json")
    p = W.random_slab(21, 17, 9, n_theta=6, n_phi=4, seed=3)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J0, _ = s.formal_solution(want_lstar=False)
        best = A.autotune_solver(s, cache_path=path, repeats=1)
        J1, _ = s.formal_solution(want_lstar=False)
    assert best in A.CANDIDATES_FP32
    assert np.array_equal(J0, J1)
    assert len(A.load_cache(path)) == 1
    probs = W.batch_65(n_lambda=3, n=9, n_theta=4, n_phi=4)
    b = R.rt_batch_create(probs, precision=R.RT_FP32_SWEEP)
    try:
        bb = A.autotune_batch(b, probs, cache_path=path)
        assert bb in A.CANDIDATES_FP32
        r = R.rt_batch_solve(b, len(probs), tol=1e-6, max_iter=500)
        assert r["converged"]
    finally:
        R.rt_batch_destroy(b)
    assert len(A.load_cache(path)) == 2
