"""Host logic of the autotuner: size classes and the winner/separation rule."""
import types

from paper_1612_09447_gb300 import autotune


def test_size_classes_partition_by_N():
    probs = [types.SimpleNamespace(N=n) for n in (16, 40, 25, 26, 37, 38, 48, 20)]
    cls = autotune.size_classes(probs, bounds=(26, 38))
    assert sorted(i for c in cls for i in c) == list(range(len(probs)))
    assert cls == [[0, 2, 7], [3, 4], [1, 5, 6]]
    assert autotune.size_classes([types.SimpleNamespace(N=30)], bounds=(26, 38)) == [[0]]


def test_summary_picks_the_median_winner_and_judges_separation():
    stats, best, sep = autotune._summary({"a": [10.0, 10.2, 9.9], "b": [12.0, 12.5, 11.8]})
    assert best == "a" and sep
    assert stats["a"][0] == 10.0 and abs(stats["a"][1] - 0.3) < 1e-12
    _, best, sep = autotune._summary({"a": [10.0, 11.5, 9.0], "b": [10.5, 10.4, 10.6]})
    assert best == "a" and not sep  # 0.5 apart, spread 2.5: within the noise
    _, best, sep = autotune._summary({"only": [3.0]})
    assert best == "only" and sep
