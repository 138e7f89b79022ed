"""The LargeGraphGPU edge blocks (Sec. 5: the edges of a part pair, streamed
to the device for its kernel) as the library builds them on host threads,
on the CPU: for every part pair (a, b) of K contiguous parts, block (a, b)
lists for every u in V^a exactly its neighbours in V^b, ascending, as ids
local to V^b (and the same for V^b against V^a), for graphs with isolated
vertices, hubs, parts of one vertex and rows longer than one build chunk;
and the host sample pools (large_pools = 1) against the oracle's draws."""
import numpy as np
import pytest

import synth
from paper_2110_10049_gb300 import build, gosh as g


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


def expected_side(gr, K, a, b):
    n = gr.n
    a0, a1 = n * a // K, n * (a + 1) // K
    b0, b1 = n * b // K, n * (b + 1) // K
    rp, cols = [0], []
    for u in range(a0, a1):
        row = gr.col[gr.rowptr[u]:gr.rowptr[u + 1]]
        sel = row[(row >= b0) & (row < b1)] - b0
        cols.extend(sel.tolist())
        rp.append(len(cols))
    return np.array(rp, np.int64), np.array(cols, np.int32)


def graphs():
    return [synth.rmat_graph(10, 8, 3), synth.random_graph(30, 0.2, 4),
            synth.csr_from_edges(9, np.array([0, 0, 0, 0, 5]), np.array([1, 2, 3, 8, 6]), compact=False)]


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_blocks_equal_definition(K):
    for gr in graphs():
        total = 0
        for a in range(K):
            for b in range(a + 1):
                rp_ab, col_ab, rp_ba, col_ba = g.gosh_large_block(gr.rowptr, gr.col, K, a, b)
                erp, ecol = expected_side(gr, K, a, b)
                np.testing.assert_array_equal(rp_ab, erp)
                np.testing.assert_array_equal(col_ab, ecol)
                total += len(col_ab)
                if a != b:
                    erp, ecol = expected_side(gr, K, b, a)
                    np.testing.assert_array_equal(rp_ba, erp)
                    np.testing.assert_array_equal(col_ba, ecol)
                    total += len(col_ba)
                else:
                    assert rp_ba is None
        assert total == gr.nnz  # every CSR entry lands in exactly one block side


def test_rows_spanning_build_chunks():
    # more rows per part than one build chunk (32768), so a side is written
    # by several items whose offsets come from the count pass
    for scale, K, pairs in ((17, 1, ((0, 0),)), (18, 2, ((1, 0),))):
        gr = synth.rmat_graph(scale, 4, 9)
        assert gr.n // K > 32768
        for a, b in pairs:
            rp_ab, col_ab, rp_ba, col_ba = g.gosh_large_block(gr.rowptr, gr.col, K, a, b)
            for got_rp, got_col, (x, y) in ((rp_ab, col_ab, (a, b)), (rp_ba, col_ba, (b, a))):
                if got_rp is None:
                    continue
                erp, ecol = expected_side(gr, K, x, y)
                np.testing.assert_array_equal(got_rp, erp)
                np.testing.assert_array_equal(got_col, ecol)


def test_invalid_pairs_rejected():
    gr = synth.random_graph(20, 0.2, 1)
    for K, a, b in ((3, 1, 2), (3, 3, 0), (0, 0, 0), (21, 0, 0)):
        with pytest.raises(g.GoshError):
            g.gosh_large_block(gr.rowptr, gr.col, K, a, b)


@pytest.mark.parametrize("K,B,seed", [(1, 1, 3), (3, 5, 4), (4, 2, 5)])
def test_sample_pools_equal_oracle_draws(K, B, seed):
    """Host sample pools (Sec. 5: positives drawn on the host, sent as pools)
    equal, entry for entry, the oracle's draws of the same pairs and rounds;
    every entry is a neighbour in the opposite part (local id), and -1
    exactly where the source has no neighbour there."""
    import oracle
    gr = synth.rmat_graph(9, 8, seed)
    n = gr.n
    st = [n * i // K for i in range(K + 1)]
    for a in range(K):
        for b in range(a + 1):
            for r in (0, 2):
                got = g.gosh_large_pool(gr.rowptr, gr.col, K, a, b, r, B, 1, 77 + seed, 5)
                want = oracle.large_pool(gr.rowptr, gr.col, K, a, b, r, B, 1, 77 + seed, 5)
                np.testing.assert_array_equal(got, want)
                srcs = list(range(st[a], st[a + 1])) + (list(range(st[b], st[b + 1])) if a != b else [])
                for s, u in enumerate(srcs):
                    own_a = s < st[a + 1] - st[a]
                    o0, o1 = (st[b], st[b + 1]) if own_a else (st[a], st[a + 1])
                    nb = gr.col[gr.rowptr[u]:gr.rowptr[u + 1]]
                    inside = nb[(nb >= o0) & (nb < o1)]
                    if len(inside) == 0:
                        assert (got[s] == -1).all()
                    else:
                        assert np.isin(got[s] + o0, inside).all()
