"""LargeGraphGPU scheduler invariants (host only, no GPU): the inside-out order
(Sec. 5.1), every part pair once per round, never more parts resident than
bins, both parts of a kernel resident when it runs, and loads only when a part
is missing."""
import pytest


@pytest.fixture(scope="module")
def g():
    from paper_2110_10049_gb300 import build, gosh
    build.build()
    return gosh


def test_inside_out_order(g):
    pairs, _ = g.gosh_large_plan(1000, 4, 3, 1)
    assert [tuple(p) for p in pairs] == [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2),
                                        (3, 0), (3, 1), (3, 2), (3, 3)]


@pytest.mark.parametrize("K,bins,rounds", [(1, 2, 3), (2, 2, 2), (5, 3, 3), (8, 2, 2), (9, 4, 3), (16, 3, 2)])
def test_schedule_invariants(g, K, bins, rounds):
    pairs, loads = g.gosh_large_plan(10 ** 6, K, bins, rounds)
    per_round = K * (K + 1) // 2
    assert len(pairs) == rounds * per_round
    for r in range(rounds):
        seen = {tuple(p) for p in pairs[r * per_round:(r + 1) * per_round]}
        assert seen == {(a, b) for a in range(K) for b in range(a + 1)}
    resident = {}
    for (a, b), (l0, l1) in zip(pairs, loads):
        for ld in (l0, l1):
            if ld >= 0:
                part, bin_ = divmod(int(ld), 1000)
                assert part not in resident.values()   # loaded only when missing
                assert 0 <= bin_ < bins
                resident[bin_] = part
        assert a in resident.values() and b in resident.values()
        assert len(resident) <= bins


@pytest.mark.parametrize("K,bins,rounds", [(0, 3, 1), (4, 1, 1), (4, 0, 1), (3, 1000, 1), (3, 3, -1)])
def test_invalid_arguments_rejected(g, K, bins, rounds):
    # one bin cannot hold both parts of a pair: rejected, not simulated
    with pytest.raises(g.GoshError):
        g.gosh_large_plan(1000, K, bins, rounds)
    cnt = g.lib().gosh_large_plan(1000, K, bins, rounds, None, None, 0)
    assert cnt == -2


def test_capacity_checked_before_writing(g):
    import numpy as np
    pairs = np.full((3, 2), -7, dtype=np.int32)
    loads = np.full((3, 2), -7, dtype=np.int32)
    assert g.lib().gosh_large_plan(1000, 3, 2, 1, pairs.ctypes.data, loads.ctypes.data, 3) == -1
    assert (pairs == -7).all() and (loads == -7).all()
