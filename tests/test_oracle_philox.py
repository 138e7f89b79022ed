"""Pins for the oracle's Philox4x64-10 and its sample draws (Alg. 3, Sec. 3.1).

Philox is pinned to numpy's independent implementation (numpy.random.Philox
is Philox4x64-10; it increments its counter before each block, so its first
block is f_key(counter + 1)).  The draws are pinned by their distributions.
"""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((1, 2), (0, 0, 0, 0)),
    ((0xDEADBEEFCAFEF00D, 0x0123456789ABCDEF), (7, 0, (3 << 32) | 11, 0)),
    ((2**64 - 1, 2**64 - 1), (2**64 - 2, 2**64 - 1, 2**64 - 1, 2**64 - 1)),
])
def test_philox_matches_numpy(orc, key, ctr):
    g = np.random.Philox(key=np.array(key, dtype=np.uint64),
                         counter=np.array(ctr, dtype=np.uint64))
    ref = g.random_raw(8)
    c = np.array(ctr, dtype=np.uint64)
    blocks = []
    for _ in range(2):
        # numpy adds one (with carry) before computing a block
        c = c.copy()
        for i in range(4):
            c[i] = np.uint64((int(c[i]) + 1) % 2**64)
            if c[i] != 0:
                break
        blocks.append(orc.philox4x64(c, key))
    np.testing.assert_array_equal(np.concatenate(blocks), ref)


def test_positive_uniform_over_neighbours(orc):
    # star-ish vertex 0 with 5 neighbours; chi-square over 5000 epochs
    n = 8
    src = np.array([0, 0, 0, 0, 0, 1, 2])
    dst = np.array([1, 2, 3, 4, 5, 6, 7])
    g = synth.csr_from_edges(n, src, dst, compact=False)
    counts = {}
    for ep in range(5000):
        u = orc.draw_samples(g.rowptr, g.col, 3, 0, ep, 99, 0, 0)
        assert u[0] in (1, 2, 3, 4, 5)
        counts[u[0]] = counts.get(u[0], 0) + 1
    obs = np.array([counts.get(i, 0) for i in (1, 2, 3, 4, 5)], dtype=float)
    chi2 = ((obs - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 20.5  # chi2(4) 0.9996 quantile


def test_negatives_uniform_and_self_skipped(orc):
    n = 10
    g = synth.csr_from_edges(n, np.arange(9), np.arange(1, 10), compact=False)
    counts = np.zeros(n)
    skipped = 0
    for ep in range(2000):
        u = orc.draw_samples(g.rowptr, g.col, 5, 2, ep, 5, 0, 3)
        for t in range(1, 6):
            if u[t] < 0:
                skipped += 1
            else:
                assert u[t] != 3
                counts[u[t]] += 1
    # the draw lands on the source itself 1/n of the time and is skipped
    total = 2000 * 5
    assert abs(skipped - total / n) < 5 * np.sqrt(total / n)
    others = np.delete(counts, 3)
    exp = total / n
    chi2 = ((others - exp) ** 2 / exp).sum()
    assert chi2 < 33.7  # chi2(8) 0.99995 quantile


def test_isolated_source_has_no_positive(orc):
    g = synth.csr_from_edges(4, np.array([0]), np.array([1]), compact=False)
    u = orc.draw_samples(g.rowptr, g.col, 3, 0, 0, 1, 0, 3)
    assert u[0] == -1


def test_draws_depend_on_every_counter_field(orc):
    g = synth.rmat_graph(8, 8, 1)
    base = orc.draw_samples(g.rowptr, g.col, 7, 1, 2, 3, 4, 5)
    for args in [(7, 0, 2, 3, 4, 5), (7, 1, 3, 3, 4, 5), (7, 1, 2, 4, 4, 5),
                 (7, 1, 2, 3, 5, 5), (7, 1, 2, 3, 4, 6)]:
        assert not np.array_equal(base, orc.draw_samples(g.rowptr, g.col, *args))
