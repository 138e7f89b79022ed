"""Oracle of LargeGraphGPU (Sec. 5), run sequentially, pinned to what the
method fixes independently of the code:

- one part with one positive per round is exactly Alg. 3: the same updates,
  bit for bit, as the sequential oracle (graphs without isolated vertices);
- on a complete graph every vertex has neighbours in every part, so it is a
  source in K pairs per round and the positives claimed are exactly
  min(e*|V|, rounds*K*|V|*B); every applied slot is a positive or a negative
  of one, so the update count lies between the positives and (k+1) times
  them, and is (k+1) times them when no negative can hit its own source;
- the library's host schedule (gosh_large_plan) visits the same
  lower-triangle pair order as the oracle's reading of Sec. 5.1;
- the global positive budget on stars cut into one-vertex parts, where every
  draw is forced, equals the hand count of tests/golden/large_budget_hand.txt
  (positives and updates, including the negatives of sources without a
  positive while the budget lasts).
"""
import os

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("k,seed", [(0, 1), (3, 2), (5, 3)])
def test_one_part_one_positive_is_alg3(k, seed):
    gr = synth.rmat_graph(8, 8, seed)
    assert (np.diff(gr.rowptr) > 0).all()
    M0 = oracle.init_uniform(gr.n, 32, 0, seed) * 20
    A, B = M0.copy(), M0.copy()
    nu, npos = oracle.train_large(gr.rowptr, gr.col, A, k, 2, 7, 0.05, 1e-4, seed, 1, 1)
    _, nb = oracle.train_sequential(gr.rowptr, gr.col, B, k, 2, 7, 0.05, 1e-4, seed)
    assert nu == nb and npos == 7 * gr.n
    np.testing.assert_array_equal(A, B)


def complete_graph(n):
    s, t = np.triu_indices(n, 1)
    return synth.csr_from_edges(n, s, t, compact=False)


@pytest.mark.parametrize("K,B,e", [(2, 1, 4), (3, 2, 5), (4, 5, 3), (3, 5, 20)])
def test_positive_budget_on_a_complete_graph(K, B, e):
    n, k = 24, 3
    gr = complete_graph(n)
    M = oracle.init_uniform(n, 32, 0, 1)
    nu, npos = oracle.train_large(gr.rowptr, gr.col, M, k, 0, e, 0.05, 1e-4, 9, K, B)
    rounds = -(-e // B)
    assert npos == min(e * n, rounds * K * n * B)
    assert npos <= nu <= (k + 1) * npos
    M1 = oracle.init_uniform(n, 32, 0, 1)
    nu1, npos1 = oracle.train_large(gr.rowptr, gr.col, M1, 0, 0, e, 0.05, 1e-4, 9, K, B)
    assert nu1 == npos1 == npos


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_pair_order_matches_library_schedule(K):
    from paper_2110_10049_gb300 import build, gosh as g
    build.build()
    pairs, _ = g.gosh_large_plan(100, K, max(2, K), 1)
    expect = [(a, b) for a in range(K) for b in range(a + 1)]
    assert [tuple(p) for p in pairs.tolist()] == expect


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_budget_hand.txt")


def star(n):
    return synth.csr_from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), compact=False)


def budget_cases():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, K, B, k, e, npos, nup = line.split()
        out.append((int(name[4:]), int(K), int(B), int(k), int(e), int(npos), int(nup)))
    return out


@pytest.mark.parametrize("n,K,B,k,e,npos,nup", budget_cases())
def test_budget_hand_count(n, K, B, k, e, npos, nup):
    gr = star(n)
    M = oracle.init_uniform(n, 16, 0, 3)
    got_u, got_p = oracle.train_large(gr.rowptr, gr.col, M, k, 0, e, 0.05, 1e-4, 7, K, B)
    assert (got_p, got_u) == (npos, nup)
