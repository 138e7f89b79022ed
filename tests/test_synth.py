"""The seeded input generator (synth/) on the CPU: the C CSR builder equals
the independent numpy construction on the same R-MAT draws (symmetrised,
self-loops dropped, deduplicated, isolated vertices dropped, rows sorted);
graphs are reproducible from their seed and skewed like R-MAT; the link
split holds out about 20% of the undirected edges, keeps a valid training
CSR without isolated vertices, and draws as many negatives as positives,
none of them a training edge, a test edge or a self-pair."""
import numpy as np
import pytest

import synth


def check_csr(gr, compact=True):
    rp, col = gr.rowptr, gr.col
    assert rp[0] == 0 and (np.diff(rp) >= 0).all() and rp[-1] == len(col)
    src = np.repeat(np.arange(gr.n), np.diff(rp))
    assert (col >= 0).all() and (col < gr.n).all() and (src != col).all()
    for v in range(gr.n):
        assert (np.diff(col[rp[v]:rp[v + 1]]) > 0).all()
    fwd = set(zip(src.tolist(), col.tolist()))
    assert all((b, a) in fwd for a, b in fwd)
    if compact:
        assert (np.diff(rp) > 0).all()
    return fwd


@pytest.mark.parametrize("scale,ef,seed", [(8, 4, 1), (10, 8, 7), (11, 16, 20211020)])
def test_c_builder_equals_numpy_construction(scale, ef, seed):
    src, dst = synth.rmat_edges(scale, ef, seed)
    a = synth.rmat_graph(scale, ef, seed)
    b = synth.csr_from_edges(1 << scale, src.astype(np.int64), dst.astype(np.int64), compact=True)
    np.testing.assert_array_equal(a.rowptr, b.rowptr)
    np.testing.assert_array_equal(a.col, b.col)
    check_csr(a)


def test_reproducible_and_skewed():
    a = synth.rmat_graph(12, 8, 5)
    b = synth.rmat_graph(12, 8, 5)
    c = synth.rmat_graph(12, 8, 6)
    np.testing.assert_array_equal(a.col, b.col)
    assert a.nnz != c.nnz or not np.array_equal(a.col, c.col)
    deg = np.diff(a.rowptr)
    assert deg.max() > 20 * deg.mean()  # power-law hubs
    assert np.median(deg) < deg.mean()


@pytest.mark.parametrize("seed", [1, 2])
def test_link_split(seed):
    g = synth.rmat_graph(11, 8, 3)
    sp = synth.link_split(g, seed)
    train = check_csr(sp.train)
    m_full = g.nnz // 2
    m_train = sp.train.nnz // 2
    m_test = len(sp.test_pos)
    assert m_train + m_test <= m_full
    assert abs(m_test - 0.2 * m_full) <= 0.02 * m_full  # test edges lost with dropped vertices are few
    assert m_train >= 0.78 * m_full
    pos = {tuple(x) for x in sp.test_pos.tolist()}
    for u, v in pos:
        assert (u, v) not in train and u != v
        assert 0 <= u < sp.train.n and 0 <= v < sp.train.n
    assert len(sp.test_neg) == m_test
    for u, v in sp.test_neg.tolist():
        assert u != v and (u, v) not in train and (u, v) not in pos and (v, u) not in pos


def test_planted_partition_graph():
    """Degree-corrected planted partition (synth/sbm.py): reproducible from
    its seed, a valid symmetric CSR, skewed degrees, and about mu + (1 - mu)
    * sum_c share_c^2 of the draws inside a community (share_c: community c's
    fraction of the degree propensity)."""
    n, C, ef, mu, seed = 4096, 32, 8, 0.8, 11
    s1, d1, comm = synth.sbm_edges(n, C, ef, mu, seed)
    s2, d2, _ = synth.sbm_edges(n, C, ef, mu, seed)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(d1, d2)
    s3, _, _ = synth.sbm_edges(n, C, ef, mu, seed + 1)
    assert not np.array_equal(s1, s3)
    inside = (comm[s1] == comm[d1]).mean()
    rng = np.random.Generator(np.random.PCG64(seed))
    rng.integers(0, C, n)
    theta = 1.0 / np.sqrt(1.0 - rng.random(n))
    share = np.bincount(comm, weights=theta, minlength=C) / theta.sum()
    expect = mu + (1 - mu) * float((share ** 2).sum())
    assert abs(inside - expect) < 0.01, (inside, expect)
    g = synth.sbm_graph(n, C, ef, mu, seed)
    check_csr(g)
    deg = np.diff(g.rowptr)
    assert deg.max() > 8 * deg.mean()
    lk = synth.workload("sbm12")
    assert 0.15 < len(lk.test_pos) / (lk.train.nnz / 2 + len(lk.test_pos)) < 0.25


@pytest.mark.parametrize("scale,ef,seed", [(8, 4, 1), (11, 16, 20211020), (13, 8, 5)])
def test_large_builder_equals_small_builder(scale, ef, seed):
    """The many-threaded, lower-memory CSR builder for very large graphs gives
    exactly the CSR of the default builder."""
    a = synth.rmat_graph(scale, ef, seed)
    b = synth.rmat_graph_large(scale, ef, seed)
    np.testing.assert_array_equal(a.rowptr, b.rowptr)
    np.testing.assert_array_equal(a.col, b.col)
