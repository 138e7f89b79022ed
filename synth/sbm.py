"""Degree-corrected planted partition (input preparation only).

R-MAT graphs have little transitivity: their held-out edges are predictable
mostly from degree, which a dot-product embedding captures poorly, so a
held-out AUC measured on them sits near 1/2 whatever the training.  This
graph keeps R-MAT's skewed degrees but plants communities that a dot product
can recover (the degree-corrected stochastic block model of Karrer and
Newman, 2011), so that held-out link prediction measures what training
learned.

Recipe (seeded, numpy PCG64, identical on every host):
  1. every vertex draws a community uniformly from C and a degree propensity
     theta = 1/sqrt(1 - U), U uniform on [0, 1) (a Pareto tail of index 2,
     heavy like R-MAT's degrees; sqrt is correctly rounded everywhere);
  2. ef * n directed draws: the source with probability proportional to
     theta over all vertices; with probability mu the target is drawn
     proportional to theta inside the source's community, otherwise over
     all vertices;
  3. symmetrise, drop self-loops, deduplicate, drop isolated vertices and
     compact ids (the R-MAT recipe's steps 3-5).
Vertex ids carry no community information (communities are drawn per id).
"""
from __future__ import annotations

import numpy as np

from .rmat import Graph, _csr_c


def sbm_edges(n: int, communities: int, edge_factor: int, mu: float, seed: int):
    """Directed draws of steps 1-2: (src, dst, community of every vertex)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    comm = rng.integers(0, communities, n)
    theta = 1.0 / np.sqrt(1.0 - rng.random(n))
    order = np.argsort(comm, kind="stable")
    cum = np.cumsum(theta[order])
    lo = np.searchsorted(comm[order], np.arange(communities), side="left")
    hi = np.searchsorted(comm[order], np.arange(communities), side="right")
    base = np.where(lo > 0, cum[np.maximum(lo - 1, 0)], 0.0)
    width = np.where(hi > lo, cum[np.maximum(hi - 1, 0)] - base, 0.0)
    m = edge_factor * n
    total = cum[-1]
    src_pos = np.minimum(np.searchsorted(cum, rng.random(m) * total, side="right"), n - 1)
    src = order[src_pos]
    inside = rng.random(m) < mu
    r = rng.random(m)
    c = comm[src]
    pos_in = np.searchsorted(cum, base[c] + r * width[c], side="right")
    pos_in = np.clip(pos_in, lo[c], hi[c] - 1)
    pos_out = np.minimum(np.searchsorted(cum, r * total, side="right"), n - 1)
    dst = order[np.where(inside, pos_in, pos_out)]
    return src.astype(np.uint32), dst.astype(np.uint32), comm.astype(np.int32)


def sbm_graph(n: int, communities: int, edge_factor: int, mu: float, seed: int) -> Graph:
    """Steps 1-3: the CSR (int64 row pointer, int32 ascending columns)."""
    s, d, _ = sbm_edges(n, communities, edge_factor, mu, seed)
    return _csr_c(n, s, d, compact=True)
