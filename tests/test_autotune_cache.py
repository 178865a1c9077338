"""Autotuner bookkeeping on the host (no GPU): keys, cache round trip, subset choice."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _S:
    def __init__(self, n):
        self.n_src = n


def test_subset_spreads_over_sizes_and_respects_the_budget():
    from paper_1805_06106_gb300 import autotune

    surfs = [_S(n) for n in (5000, 200000, 12000, 48000, 7000, 90000, 30000, 15000, 60000, 9000)]
    dens = list(range(len(surfs)))
    sub, d = autotune._subset(surfs, dens, 100_000)
    assert 1 <= len(sub) <= len(surfs)
    assert sum(s.n_src for s in sub) <= 100_000 or len(sub) == 1
    assert [dens[surfs.index(s)] for s in sub] == d
    sizes = [s.n_src for s in sub]
    assert sizes == sorted(sizes)  # picked in size order, smallest first


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_1805_06106_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    assert autotune._load() == {}
    autotune._store({"k": {"n_max": 48, "tiles": [16, 48]}})
    assert json.load(open(tmp_path / "autotune.json"))["k"]["n_max"] == 48
    assert autotune._load()["k"]["tiles"] == [16, 48]
