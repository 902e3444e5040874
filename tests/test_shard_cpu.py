"""Batched scenes across ranks (section "Conclusion" names multi-GPU runs
as the way past one device): the host logic of the scene split, on CPU."""
import numpy as np
import pytest

from paper_2311_15088_gb300 import scenes, shard


def test_greedy_bin_pack_by_hand():
    """Longest first, each scene to the least-loaded rank (ties: lower rank):
    5 -> r0, 4 -> r1, 3 -> r1 (4 < 5), 3 -> r0 (5 < 7), 2 -> r1 (7 < 8)."""
    parts = shard.assign([5, 4, 3, 3, 2], 2)
    assert parts == [[0, 3], [1, 2, 4]]
    assert shard.imbalance([5, 4, 3, 3, 2], parts) == pytest.approx(9 / 8.5 - 1)
    assert shard.assign([7], 3) == [[0], [], []]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batched_tanks_split_every_scene_once_and_balanced(world):
    """The 256 tanks of the batched workload: every scene on exactly one
    rank, and no rank's particles more than 5 % above the mean."""
    w = [shard.scene_weight(sc) for sc in scenes.batched_tanks()]
    parts = shard.assign(w, world)
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(w)))
    assert shard.imbalance(w, parts) <= 0.05


def test_gather_rejects_missing_and_doubled_scenes():
    out, owner = shard.gather({1: "b", 0: "a"}, 2, 1)
    assert out == ["a", "b"] and owner == [0, 0]
    with pytest.raises(RuntimeError):
        shard.gather({0: "a"}, 2, 1)
