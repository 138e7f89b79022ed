"""Oracle of random-walk sampling (Sec. 3.2), pinned to properties the
definition fixes independently of the code:

- consecutive walk vertices are graph edges, and every pair lies within graph
  distance g (breadth-first search on the graph, not the walk);
- a walk's first step is uniform over the start's neighbours (chi-square);
- the number of pair positions per walk is the closed form
  g*(l-1-g) + g*(g+1)/2 (l > g), and holes appear exactly where the walk
  stopped or returned to the same vertex;
- the shuffle is a bijection of [0, P) for every P tried and far from the
  identity;
- training with k = 0 on the two-vertex graph is Alg. 1 applied in the
  permuted order (UPDATEEMBED itself is pinned in test_oracle_update.py);
- training lowers the loss and fits the edges.
"""
from collections import deque

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle
import synth


def bfs_dist(rowptr, col, s, cap):
    dist = {s: 0}
    q = deque([s])
    while q:
        x = q.popleft()
        if dist[x] == cap:
            continue
        for y in col[rowptr[x]:rowptr[x + 1]]:
            if y not in dist:
                dist[int(y)] = dist[x] + 1
                q.append(int(y))
    return dist


@pytest.mark.parametrize("l,g", [(2, 1), (4, 2), (8, 3), (5, 7)])
def test_positions_per_walk_closed_form(l, g):
    gg = min(g, l - 1)
    assert oracle.walk_pairs_per_walk(l, g) == gg * (l - 1 - gg) + gg * (gg + 1) // 2


def test_pairs_are_walk_steps_within_distance_g():
    gr = synth.rmat_graph(9, 4, 3)
    l, g = 8, 3
    W = oracle.walk_pairs_per_walk(l, g)
    pr = oracle.walk_pairs(gr.rowptr, gr.col, l, g, 0, 2, 11)
    edges = set()
    for v in range(gr.n):
        for u in gr.col[gr.rowptr[v]:gr.rowptr[v + 1]]:
            edges.add((v, int(u)))
    rng = np.random.default_rng(0)
    for v in rng.choice(gr.n, 60, replace=False):
        block = pr[v * W:(v + 1) * W]
        r = 0
        for i in range(l - 1):
            for j in range(i + 1, min(i + g, l - 1) + 1):
                s, t = block[r]
                if s >= 0:
                    if j == i + 1:
                        assert (int(s), int(t)) in edges
                    if i == 0:
                        assert s == v
                    d = bfs_dist(gr.rowptr, gr.col, int(s), g)
                    assert int(t) in d and d[int(t)] <= j - i
                r += 1


def test_first_step_uniform_over_neighbours():
    gr = synth.rmat_graph(8, 8, 5)
    deg = np.diff(gr.rowptr)
    v = int(np.argmax(deg))
    nb = gr.col[gr.rowptr[v]:gr.rowptr[v + 1]]
    W = oracle.walk_pairs_per_walk(3, 1)
    counts = np.zeros(len(nb))
    idx = {int(u): i for i, u in enumerate(nb)}
    for e in range(3000):
        pr = oracle.walk_pairs(gr.rowptr, gr.col, 3, 1, 0, e, 21)
        counts[idx[int(pr[v * W][1])]] += 1
    assert chisquare(counts).pvalue > 1e-4


def test_holes_where_walks_stop_or_return():
    # a star: every walk alternates centre and leaves, so pairs at distance
    # two join a vertex to itself (centre) or two leaves
    s = np.zeros(5, np.int64)
    t = np.arange(1, 6)
    gr = synth.csr_from_edges(6, s, t, compact=False)
    l, g = 5, 2
    W = oracle.walk_pairs_per_walk(l, g)
    pr = oracle.walk_pairs(gr.rowptr, gr.col, l, g, 0, 0, 3)
    blk = pr[0:W]  # walk from the centre: 0, leaf, 0, leaf, 0
    r = 0
    for i in range(l - 1):
        for j in range(i + 1, min(i + g, l - 1) + 1):
            if (j - i) % 2 == 0 and i % 2 == 0:
                assert blk[r][0] == -1  # centre to centre: a hole
            r += 1
    # an isolated vertex ends its walk at once: all its positions are holes
    gr2 = synth.csr_from_edges(4, np.array([0]), np.array([1]), compact=False)
    W2 = oracle.walk_pairs_per_walk(4, 2)
    pr2 = oracle.walk_pairs(gr2.rowptr, gr2.col, 4, 2, 0, 0, 3)
    assert (pr2[2 * W2:4 * W2, 0] == -1).all()


@pytest.mark.parametrize("P", [1, 2, 3, 5, 17, 100, 1000, 4097, 65537])
def test_shuffle_is_a_bijection(P):
    perm = oracle.walk_perm(P, 9, 4, 1, 3)
    assert np.array_equal(np.sort(perm), np.arange(P))
    if P >= 100:
        assert (perm == np.arange(P)).mean() < 0.05
        # different epochs give different orders
        assert not np.array_equal(perm, oracle.walk_perm(P, 9, 4, 1, 4))


def test_two_vertex_training_is_alg1_in_permuted_order():
    gr = synth.csr_from_edges(2, np.array([0]), np.array([1]), compact=False)
    M0 = oracle.init_uniform(2, 8, 0, 4) * 50
    M = M0.copy()
    oracle.train_walks(gr.rowptr, gr.col, M, 0, 0, 3, 0.3, 1e-4, 4, 2, 1)
    R = M0.copy()
    for e in range(3):
        lr = oracle.epoch_lr(0.3, 1e-4, e, 3)
        pr = oracle.walk_pairs(gr.rowptr, gr.col, 2, 1, 0, e, 4)
        for q in oracle.walk_perm(len(pr), 4, 0, 0, e):
            s, t = pr[q]
            a, b, _ = oracle.update_embed(R[s], R[t], 1, lr)
            R[s], R[t] = a, b
    np.testing.assert_allclose(M, R, rtol=0, atol=0)


def test_walk_training_lowers_loss_and_fits_edges():
    sp = synth.workload("rmat12")
    gr = sp.train
    M = oracle.init_uniform(gr.n, 32, 0, 8)
    loss, nup = oracle.train_walks(gr.rowptr, gr.col, M, 3, 0, 20, 0.1, 1e-4, 8, 6, 2)
    assert nup > 0
    assert loss[-1] < loss[0] * 0.93
    src = np.repeat(np.arange(gr.n), np.diff(gr.rowptr))
    rng = np.random.default_rng(1)
    rnd = np.stack([rng.integers(0, gr.n, 20000), rng.integers(0, gr.n, 20000)], 1)
    assert oracle.link_auc(M, np.stack([src, gr.col], 1), rnd) > 0.8
