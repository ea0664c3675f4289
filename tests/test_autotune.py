"""Host logic of the batched path's autotuner (no GPU): candidate set,
selection, timing loop and the on-disk choice cache."""
import pytest

from paper_2403_16438_gb300 import autotune as at


def test_candidates_respect_workspace():
    assert at.candidates(512) == [(c, g) for c in (64, 128, 256, 512) for g in (False, True)]
    assert at.candidates(200) == [(64, False), (64, True), (128, False), (128, True)]
    assert at.candidates(32) == []


def test_pick_fastest_then_smaller_chunk_then_direct():
    t = {(256, True): 1.0, (128, False): 1.0, (128, True): 1.0, (512, False): 2.0}
    assert at.pick(t) == (128, False)
    assert at.pick({(64, True): 0.5, (64, False): 0.7}) == (64, True)


def test_tune_takes_best_of_reps():
    calls = []
    noisy = {(64, False): [3.0, 1.0], (128, False): [2.0, 2.5]}

    def run(c):
        calls.append(c)
        return noisy[c][sum(1 for x in calls if x == c) - 1]

    best, table = at.tune([(64, False), (128, False)], run, reps=2)
    assert best == (64, False)
    assert table == {(64, False): 1.0, (128, False): 2.0}
    assert len(calls) == 4


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "tune.json")
    k1 = at.key_of("GB300", [(256, 256, 20000), (1024, 1024, 5000)])
    k2 = at.key_of("GB300", [(512, 512, 12000)])
    assert at.load(p, k1) is None
    at.store(p, k1, (256, True), {(256, True): 1.5, (64, False): 2.0})
    at.store(p, k2, (128, False))
    assert at.load(p, k1) == (256, True)
    assert at.load(p, k2) == (128, False)
    assert at.load(p, "other") is None


def test_pick_group_fastest_then_larger():
    assert at.pick_group({11: 2.0, 10: 1.5, 8: 1.7, 7: 1.5}) == 10
    assert at.pick_group({11: 1.0, 7: 1.0}) == 11
    with pytest.raises(ValueError):
        at.pick_group({})


def test_group_candidates_are_the_library_sizes():
    # the sizes the C ABI accepts for vimg_params.corr_group (besides 0 = 11)
    assert set(at.GROUPS) == {11, 10, 8, 7}
