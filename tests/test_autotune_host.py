"""The batched launch's autotuner, host logic on CPU with a fake batch and
fake timings: among the candidates within the slack of the fastest the first
in preference order wins, the choice is applied to the batch, cached under
its key, and a cached choice is applied without timing."""
import json

import pytest

from paper_2001_01158_gb300 import autotune


class FakeBatch:
    def __init__(self, sizes):
        self.sizes = sizes
        self.nsys = len(sizes)
        self.cells = sum(sizes)
        self.tuning = {}

    def set_tuning(self, key, value):
        self.tuning[key] = value


@pytest.fixture
def fake(monkeypatch, tmp_path):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("LC_AUTOTUNE_CACHE", str(cache))
    monkeypatch.setattr(autotune, "_key", lambda batch: "GPU|batched-v2|" + autotune.size_class(batch))
    timed = []
    # the third candidate is fastest; the first is within 3 % of it, the second is not
    ms = {autotune.CANDIDATES[0]: 10.2, autotune.CANDIDATES[1]: 10.6, autotune.CANDIDATES[2]: 10.0}

    def time_config(batch, b, x0, params, cand, reps=5):
        timed.append(cand)
        return ms.get(cand, 20.0)

    monkeypatch.setattr(autotune, "time_config", time_config)
    return cache, timed


def test_first_candidate_within_slack_wins_and_is_cached(fake):
    cache, timed = fake
    batch = FakeBatch([64 * 64, 128 * 128, 500 * 500])
    cfg = autotune.tune_batch(batch, None, None, None)
    assert len(timed) == len(autotune.CANDIDATES)
    assert tuple(cfg[k] for k in autotune.KEYS) == autotune.CANDIDATES[0]
    assert cfg["best_ms"] == 10.0 and cfg["ms"] == 10.2
    assert batch.tuning == dict(zip(autotune.KEYS, autotune.CANDIDATES[0]))
    stored = json.load(open(cache))
    assert list(stored) == ["GPU|batched-v2|" + autotune.size_class(batch)]
    # a second batch of the same size class takes the cached choice without timing
    timed.clear()
    other = FakeBatch([64 * 64, 128 * 128, 500 * 500])
    assert autotune.tune_batch(other, None, None, None)["ms"] == 10.2 and not timed
    assert other.tuning == batch.tuning


def test_zero_slack_takes_the_fastest(fake):
    _, timed = fake
    cfg = autotune.tune_batch(FakeBatch([100, 200]), None, None, None, use_cache=False, slack=0.0)
    assert tuple(cfg[k] for k in autotune.KEYS) == autotune.CANDIDATES[2]


def test_size_class():
    assert autotune.size_class(FakeBatch([64, 64])) == "n2-mean2^6-max2^6"
    assert autotune.size_class(FakeBatch([1, 1023])) == "n2-mean2^9-max2^10"
