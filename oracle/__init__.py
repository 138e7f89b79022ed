"""CPU oracle for the GOSH embedding step (arxiv 2110.10049).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; nothing in the product package
imports it.  The arithmetic lives in ``gosh_oracle.c`` (plain C, FP64,
single-threaded) and ``mlp.py`` (numpy FP64); this module marshals numpy
arrays into the C functions and holds the host-side driver logic of Alg. 2 and
Alg. 4 (level loop, stop condition, epoch split), each written out from the
paper.

Parity pins for every function are in ``tests/test_oracle_*.py``.

Parity unpinned (what the GPU path is judged by instead): lock-free training
beyond the single-warp case, whose update order is not reproducible
(link-prediction AUC against ``train_sequential``); LargeGraphGPU on the
device with its default schedule, whose part-pair kernels may overlap on two
streams (AUC against the resident step; with the kernels on one stream,
graphs whose part pairs fit one tile are compared with ``train_large``, the
sequential schedule, to 1e-5); the learned projection's training trajectory
(the gradients are pinned; the trained network is judged by its AUC gain).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gosh_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TAG_SAMPLE = 0
TAG_INIT = 1


def build(force: bool = False) -> str:
    """Compile gosh_oracle.c with gcc into oracle/liboracle.so (host ISA only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        i64, i32, u64, f64, vp = C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_void_p
        sig = {
            "orc_philox4x64": (None, [vp, vp, vp]),
            "orc_draw_samples": (None, [i64, vp, vp, i32, i32, i32, u64, u64, i64, vp]),
            "orc_sample_loss": (f64, [f64, i32]),
            "orc_update_embed": (f64, [vp, vp, i32, i32, f64]),
            "orc_epoch_lr": (f64, [f64, f64, i32, i32]),
            "orc_train_sequential": (None, [i64, vp, vp, vp, i32, i32, i32, i32, f64, f64,
                                            u64, u64, vp, vp]),
            "orc_train_deterministic": (None, [i64, vp, vp, vp, i32, i32, i32, i32, f64, f64,
                                               u64, u64, i64, vp, vp]),
            "orc_det_batch": (None, [vp, i32, i64, i64, i32, vp, f64, vp, vp]),
            "orc_init_uniform": (None, [i64, i32, i32, u64, u64, vp]),
            "orc_degree_order": (None, [i64, vp, vp]),
            "orc_mec_map": (i64, [i64, vp, vp, vp]),
            "orc_coarsen": (i64, [i64, vp, vp, vp, i64, vp, vp]),
            "orc_project_copy": (None, [i64, vp, vp, vp, i32]),
            "orc_pair_scores": (None, [vp, i32, i64, vp, vp]),
            "orc_auc": (f64, [i64, vp, i64, vp]),
            "orc_walk_pairs_per_walk": (i64, [i32, i32]),
            "orc_walk_pairs": (None, [i64, vp, vp, i32, i32, i32, i32, u64, u64, vp]),
            "orc_walk_perm_key": (C.c_uint32, [u64, u64, i32, i32]),
            "orc_walk_perm": (u64, [u64, u64, C.c_uint32]),
            "orc_train_walks": (None, [i64, vp, vp, vp, i32, i32, i32, i32, f64, f64, u64, u64, i32, i32,
                                       vp, vp]),
            "orc_train_large": (None, [i64, vp, vp, vp, i32, i32, i32, i32, f64, f64, u64, u64, i32, i32,
                                       vp, vp]),
            "orc_large_pool": (None, [i64, vp, vp, i32, i32, i32, i32, i32, i32, u64, u64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(rowptr, col):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rowptr, col


# --------------------------------------------------------------------------
# Philox4x64-10 and sampling
# --------------------------------------------------------------------------
def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def draw_samples(rowptr, col, k, level, epoch, seed, graph, v) -> np.ndarray:
    """The k+1 sample ids of source v (index 0 positive); -1 marks a skipped sample."""
    rowptr, col = _csr(rowptr, col)
    u = np.zeros(k + 1, dtype=np.int32)
    lib().orc_draw_samples(len(rowptr) - 1, _p(rowptr), _p(col), k, level, epoch,
                           seed, graph, v, _p(u))
    return u


# --------------------------------------------------------------------------
# Alg. 1 and the loss
# --------------------------------------------------------------------------
def sample_loss(x: float, b: int) -> float:
    return lib().orc_sample_loss(float(x), int(b))


def update_embed(mv, mu, b, lr):
    """One UPDATEEMBED on copies; returns (mv', mu', x)."""
    mv = np.array(mv, dtype=np.float64)
    mu = np.array(mu, dtype=np.float64)
    x = lib().orc_update_embed(_p(mv), _p(mu), mv.size, int(b), float(lr))
    return mv, mu, x


def epoch_lr(lr, lr_floor, j, e_i) -> float:
    return lib().orc_epoch_lr(lr, lr_floor, j, e_i)


# --------------------------------------------------------------------------
# Alg. 3 (sequential) and the deterministic batched mode
# --------------------------------------------------------------------------
def train_sequential(rowptr, col, M, k, level, epochs, lr, lr_floor, seed, graph=0):
    """Runs Alg. 3 on M (|V| x d float64, updated in place). Returns (loss[epochs], n_updates)."""
    rowptr, col = _csr(rowptr, col)
    assert M.dtype == np.float64 and M.flags.c_contiguous
    loss = np.zeros(max(epochs, 1), dtype=np.float64)
    nup = np.zeros(1, dtype=np.int64)
    lib().orc_train_sequential(len(rowptr) - 1, _p(rowptr), _p(col), _p(M), M.shape[1], k,
                               level, epochs, lr, lr_floor, seed, graph, _p(loss), _p(nup))
    return loss[:epochs], int(nup[0])


def walk_pairs_per_walk(l: int, g: int) -> int:
    """Pairs (w_i, w_j), 0 < j - i <= g, of a walk of l vertices (Sec. 3.2)."""
    return int(lib().orc_walk_pairs_per_walk(l, g))


def walk_pairs(rowptr, col, l, g, level, epoch, seed, graph=0) -> np.ndarray:
    """The epoch's walk positions (Sec. 3.2): int32 [n * W, 2] of (source,
    positive), -1 for holes; the walk from v fills rows v*W .. v*W+W-1."""
    rowptr, col = _csr(rowptr, col)
    n = len(rowptr) - 1
    out = np.zeros((n * walk_pairs_per_walk(l, g), 2), dtype=np.int32)
    lib().orc_walk_pairs(n, _p(rowptr), _p(col), l, g, level, epoch, seed, graph, _p(out))
    return out


def walk_perm(P: int, seed, graph, level, epoch) -> np.ndarray:
    """Visiting order of an epoch's P walk positions (the shuffle)."""
    key = lib().orc_walk_perm_key(seed, graph, level, epoch)
    return np.array([lib().orc_walk_perm(i, P, key) for i in range(P)], dtype=np.int64)


def train_walks(rowptr, col, M, k, level, epochs, lr, lr_floor, seed, l, g, graph=0):
    """Sequential epochs of walk-based positives (Sec. 3.2) on M (float64, in
    place). Returns (loss[epochs], n_updates)."""
    rowptr, col = _csr(rowptr, col)
    assert M.dtype == np.float64 and M.flags.c_contiguous
    loss = np.zeros(max(epochs, 1), dtype=np.float64)
    nup = np.zeros(1, dtype=np.int64)
    lib().orc_train_walks(len(rowptr) - 1, _p(rowptr), _p(col), _p(M), M.shape[1], k, level, epochs, lr,
                          lr_floor, seed, graph, l, g, _p(loss), _p(nup))
    return loss[:epochs], int(nup[0])


def train_large(rowptr, col, M, k, level, epochs, lr, lr_floor, seed, K, B, graph=0):
    """LargeGraphGPU (Sec. 5) run sequentially on M (float64, in place):
    rounds of part pairs, B positives per source per pair from the opposite
    part, tiles of 32 sources claiming a global positive budget of e*|V|.
    Returns (n_updates, n_positives)."""
    rowptr, col = _csr(rowptr, col)
    assert M.dtype == np.float64 and M.flags.c_contiguous
    nup = np.zeros(1, dtype=np.int64)
    npos = np.zeros(1, dtype=np.int64)
    lib().orc_train_large(len(rowptr) - 1, _p(rowptr), _p(col), _p(M), M.shape[1], k, level, epochs, lr, lr_floor,
                          seed, graph, K, B, _p(nup), _p(npos))
    return int(nup[0]), int(npos[0])


def large_pool(rowptr, col, K, a, b, r, B, level, seed, graph=0) -> np.ndarray:
    """Positives of pair (a, b) in round r for each of its sources (Sec. 5's
    host sample pool): int32 [sources, B] of local ids, -1 = no neighbour."""
    rowptr, col = _csr(rowptr, col)
    n = len(rowptr) - 1
    st = [n * i // K for i in range(K + 1)]
    ns = (st[a + 1] - st[a]) + ((st[b + 1] - st[b]) if a != b else 0)
    out = np.zeros((max(ns, 1), B), dtype=np.int32)
    lib().orc_large_pool(n, _p(rowptr), _p(col), K, a, b, r, B, level, seed, graph, _p(out))
    return out[:ns]


def train_deterministic(rowptr, col, M, k, level, epochs, lr, lr_floor, seed, m, graph=0):
    rowptr, col = _csr(rowptr, col)
    assert M.dtype == np.float64 and M.flags.c_contiguous
    loss = np.zeros(max(epochs, 1), dtype=np.float64)
    nup = np.zeros(1, dtype=np.int64)
    lib().orc_train_deterministic(len(rowptr) - 1, _p(rowptr), _p(col), _p(M), M.shape[1], k,
                                  level, epochs, lr, lr_floor, seed, graph, int(m),
                                  _p(loss), _p(nup))
    return loss[:epochs], int(nup[0])


def det_batch(M, b0, b1, samples, lr):
    """One snapshot batch of the deterministic mode on M (float64, in place)
    with given samples: int32 [(b1-b0), k+1], column 0 the positive, -1 =
    skipped.  Returns (summed loss, applied updates)."""
    assert M.dtype == np.float64 and M.flags.c_contiguous
    smp = np.ascontiguousarray(samples, dtype=np.int32)
    nap = np.zeros(1, dtype=np.int64)
    loss = np.zeros(1, dtype=np.float64)
    lib().orc_det_batch(_p(M), M.shape[1], int(b0), int(b1), smp.shape[1] - 1, _p(smp), float(lr), _p(loss), _p(nap))
    return float(loss[0]), int(nap[0])


def init_uniform(n, d, level, seed, graph=0) -> np.ndarray:
    M = np.zeros((n, d), dtype=np.float64)
    lib().orc_init_uniform(n, d, level, seed, graph, _p(M))
    return M


# --------------------------------------------------------------------------
# Alg. 4 MULTIEDGECOLLAPSE
# --------------------------------------------------------------------------
def degree_order(rowptr) -> np.ndarray:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    n = len(rowptr) - 1
    order = np.zeros(max(n, 1), dtype=np.int32)
    lib().orc_degree_order(n, _p(rowptr), _p(order))
    return order[:n]


def mec_map(rowptr, col):
    """One level of Alg. 4's mapping loop. Returns (map int32[n], n_coarse)."""
    rowptr, col = _csr(rowptr, col)
    n = len(rowptr) - 1
    mp = np.zeros(max(n, 1), dtype=np.int32)
    nc = lib().orc_mec_map(n, _p(rowptr), _p(col), _p(mp))
    return mp[:n], int(nc)


def coarsen(rowptr, col, mp, nc):
    """COARSEN(G_i, map_i): CSR of G_{i+1}."""
    rowptr, col = _csr(rowptr, col)
    mp = np.ascontiguousarray(mp, dtype=np.int32)
    n = len(rowptr) - 1
    rp = np.zeros(nc + 1, dtype=np.int64)
    co = np.zeros(max(int(rowptr[-1]), 1), dtype=np.int32)
    nnz = lib().orc_coarsen(n, _p(rowptr), _p(col), _p(mp), nc, _p(rp), _p(co))
    return rp, co[:nnz].copy()


def continue_coarsening(n_new: int, n_old: int, threshold: int, shrink: float) -> bool:
    """Loop condition of Alg. 4: keep going while |V_i| > threshold and
    |V_i| <= shrink * |V_{i-1}| (shrink = 0.8 in the paper)."""
    return n_new > threshold and n_new <= math.floor(shrink * n_old)


def mec_hierarchy(rowptr, col, threshold=100, shrink=0.8, max_levels=64):
    """Alg. 4: returns (graphs [(rowptr, col)], maps [map_i]) with graphs[0] = G_0.
    The do-while body always runs once; the last graph produced is kept."""
    graphs = [(np.asarray(rowptr, np.int64), np.asarray(col, np.int32))]
    maps = []
    while True:
        rp, co = graphs[-1]
        mp, nc = mec_map(rp, co)
        graphs.append(coarsen(rp, co, mp, nc))
        maps.append(mp)
        n_new, n_old = len(graphs[-1][0]) - 1, len(rp) - 1
        if len(graphs) >= max_levels or not continue_coarsening(n_new, n_old, threshold, shrink):
            break
    return graphs, maps


# --------------------------------------------------------------------------
# Epoch split (Sec. 3) and EXPANDEMBEDDING
# --------------------------------------------------------------------------
def epoch_split(e: int, p: float, D: int) -> list[int]:
    """CALCULATEEPOCHS: a fraction p of e spread uniformly over the D levels and
    the remaining (1-p) spread geometrically, each level getting twice its finer
    neighbour's share: e_i = p*e/D + (1-p)*e*2^i/(2^D - 1).  Reading: levels
    i >= 1 take the floor and level 0 takes the remainder, so the sum is e."""
    if D == 1:
        return [e]
    real = [p * e / D + (1.0 - p) * e * (2.0 ** i) / (2.0 ** D - 1.0) for i in range(D)]
    out = [0] * D
    for i in range(1, D):
        out[i] = int(math.floor(real[i]))
    out[0] = e - sum(out[1:])
    return out


def epoch_passes(e: int, n0: int, nnz0: int) -> int:
    """Alg. 3 passes for e epochs of |E| updates (Sec. 6's setup defines one
    epoch as |E| updates and adjusts the epoch count accordingly; one Alg. 3
    pass makes |V| positive draws).  Reading: the conversion applies to the
    total e of Alg. 2, by the input graph's |E|/|V|; |E| counts CSR entries
    (both directions, the count in Alg. 4's density delta = |E_i|/|V_i|);
    the quotient is rounded half up, and any e >= 1 keeps at least one
    pass."""
    if e == 0:
        return 0
    from fractions import Fraction
    q = Fraction(e * nnz0, n0)
    return max(1, math.floor(q + Fraction(1, 2)))


def level_epochs(e: int, p: float, sizes, nnzs, epoch_unit: str = "V") -> list[int]:
    """Passes per level: for the |E| unit the total converted by
    epoch_passes on G_0, then the Sec. 3 split over the levels."""
    if epoch_unit == "E":
        e = epoch_passes(e, sizes[0], nnzs[0])
    else:
        assert epoch_unit == "V"
    return epoch_split(e, p, len(sizes))


def project_copy(mp, Mc) -> np.ndarray:
    mp = np.ascontiguousarray(mp, dtype=np.int32)
    Mc = np.ascontiguousarray(Mc, dtype=np.float64)
    Mf = np.zeros((len(mp), Mc.shape[1]), dtype=np.float64)
    lib().orc_project_copy(len(mp), _p(mp), _p(Mc), _p(Mf), Mc.shape[1])
    return Mf


# --------------------------------------------------------------------------
# Link-prediction scores and AUC (Sec. 6.1)
# --------------------------------------------------------------------------
def pair_scores(M, pairs) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(max(len(pairs), 1), dtype=np.float64)
    lib().orc_pair_scores(_p(M), M.shape[1], len(pairs), _p(pairs), _p(out))
    return out[:len(pairs)]


def auc(pos_scores, neg_scores) -> float:
    pos = np.ascontiguousarray(pos_scores, dtype=np.float64)
    neg = np.ascontiguousarray(neg_scores, dtype=np.float64)
    return lib().orc_auc(len(pos), _p(pos), len(neg), _p(neg))


def link_auc(M, pos_pairs, neg_pairs) -> float:
    return auc(pair_scores(M, pos_pairs), pair_scores(M, neg_pairs))


# --------------------------------------------------------------------------
# Alg. 2 GOSH end to end (copy projection)
# --------------------------------------------------------------------------
def embed(rowptr, col, d, k, lr, e, p, seed, threshold=100, shrink=0.8, lr_floor=1e-4,
          mode="sequential", det_batch=1, storage=np.float32, graph=0, coarsening=True, epoch_unit="V"):
    """GOSH (Alg. 2) with every level D-1..0 trained (level 0 included: the
    algorithm returns M_0, and the single-level configuration must train).
    M_{D-1} starts from the init rounded to the storage precision; training
    runs in FP64.  epoch_unit "V": an epoch is one Alg. 3 pass over V_i; "E":
    an epoch is |E| updates (Sec. 6), see epoch_passes.  Returns (M_0, info)."""
    if coarsening:
        graphs, maps = mec_hierarchy(rowptr, col, threshold, shrink)
    else:
        graphs, maps = [(np.asarray(rowptr, np.int64), np.asarray(col, np.int32))], []
    D = len(graphs)
    ep = level_epochs(e, p, [len(g[0]) - 1 for g in graphs], [int(g[0][-1]) for g in graphs], epoch_unit)
    n_top = len(graphs[-1][0]) - 1
    M = init_uniform(n_top, d, D - 1, seed, graph).astype(storage).astype(np.float64)
    losses, updates = [], 0
    for i in range(D - 1, -1, -1):
        rp, co = graphs[i]
        if mode == "sequential":
            loss, nu = train_sequential(rp, co, M, k, i, ep[i], lr, lr_floor, seed, graph)
        else:
            loss, nu = train_deterministic(rp, co, M, k, i, ep[i], lr, lr_floor, seed,
                                           det_batch, graph)
        losses.append(loss)
        updates += nu
        if i > 0:
            M = project_copy(maps[i - 1], M)
    return M, {"levels": D, "epochs": ep, "loss": losses, "updates": updates,
               "sizes": [len(g[0]) - 1 for g in graphs]}
