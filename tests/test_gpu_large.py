"""LargeGraphGPU (Sec. 5) on the GPU.

- K = 1, B = 1 draws exactly the samples of the resident step (same Philox
  counters, one part pair per round = one epoch); on a graph that fits one
  warp with one source per round both are sequential, so they agree to the
  deterministic-mode tolerance 1e-5;
- with K = 2 or 3 parts and B = 1..3 positives per round, kernels in stream
  order (large_serial) and every part pair within one tile of 32 sources,
  the device run is the oracle's sequential LargeGraphGPU (same positives
  claimed, same updates, embeddings within 1e-5);
- the global budget as counted by hand on stars cut into one-vertex parts
  (tests/golden/large_budget_hand.txt), with the oracle's embeddings;
- with K = 4 parts and 3 bins the default schedule (kernels of part pairs
  overlapping on two streams, which reorders updates) reaches the held-out
  AUC of the sequential oracle within 0.005 on the planted partition,
  launches rounds * K(K+1)/2 kernels, and the global counter caps positives
  at e * |V|;
- BF16 tables run through the same path;
- every case above also runs with host sample pools (large_pools = 1: the
  positives drawn on host threads and streamed, Sec. 5's scheme), which
  draw the same samples as the edge blocks.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_single_part_equals_resident_step():
    g = gosh()
    gr = synth.random_graph(30, 0.2, 17)
    M0 = (oracle.init_uniform(gr.n, 128, 0, 3) * 60).astype(np.float32)
    p = g.default_params(d=128, k=3, lr=0.05, seed=8, B=1, large_parts=1, p_gpu=2, s_gpu=1)
    Mh = M0.copy()
    st = g.gosh_train_level_large(gr.rowptr, gr.col, Mh, 0, 12, p)
    assert st["parts"] == 1 and st["rounds"] == 12 and st["kernels"] == 12
    csr = g.to_device_csr(gr.rowptr, gr.col)
    Md = torch.from_numpy(M0.copy()).cuda()
    nup = torch.zeros(1, dtype=torch.int64, device="cuda")
    # register kernel, 32 lanes: one warp takes the sources strictly in order
    g.gosh_train_level(csr, Md, 0, 12, g.default_params(d=128, k=3, lr=0.05, seed=8, lanes_per_row=32,
                                                        samples_per_pass=2, vertices_per_warp=32), n_updates=nup)
    assert st["updates"] == int(nup.item())
    assert rel_fro(Mh, Md.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("pools", [0, 1])
@pytest.mark.parametrize("K,B,seed", [(2, 2, 3), (3, 1, 5), (2, 3, 9)])
def test_serial_parts_equal_sequential_oracle(K, B, seed, pools):
    # every part pair has at most 32 sources: one tile, one warp, one source
    # at a time; with the kernels in stream order the device run is the
    # oracle's sequential LargeGraphGPU
    g = gosh()
    gr = synth.random_graph(30, 0.25, seed)
    e = 10
    M0 = (oracle.init_uniform(gr.n, 128, 0, seed) * 60).astype(np.float32).astype(np.float64)
    Mo = M0.copy()
    nup_o, npos_o = oracle.train_large(gr.rowptr, gr.col, Mo, 3, 0, e, 0.05, 1e-4, seed, K, B)
    Mh = M0.astype(np.float32)
    p = g.default_params(d=128, k=3, lr=0.05, seed=seed, B=B, large_parts=K, p_gpu=2, s_gpu=1, large_serial=1,
                         large_pools=pools)
    st = g.gosh_train_level_large(gr.rowptr, gr.col, Mh, 0, e, p)
    assert st["positives"] == npos_o
    assert st["updates"] == nup_o
    assert rel_fro(Mh.astype(np.float64), Mo) <= 1e-5


def golden_budget_cases():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_budget_hand.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, K, B, k, e, npos, nup = line.split()
        out.append((int(name[4:]), int(K), int(B), int(k), int(e), int(npos), int(nup)))
    return out


@pytest.mark.parametrize("pools", [0, 1])
@pytest.mark.parametrize("n,K,B,k,e,npos,nup", golden_budget_cases())
def test_budget_hand_count_on_device(n, K, B, k, e, npos, nup, pools):
    """The global positive budget as counted by hand (stars cut into
    one-vertex parts: every draw is forced), run on the device in stream
    order; the embeddings equal the sequential oracle's."""
    g = gosh()
    gr = synth.csr_from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), compact=False)
    M0 = (oracle.init_uniform(n, 128, 0, 5) * 60).astype(np.float32).astype(np.float64)
    Mo = M0.copy()
    nup_o, npos_o = oracle.train_large(gr.rowptr, gr.col, Mo, k, 0, e, 0.05, 1e-4, 7, K, B)
    assert (npos_o, nup_o) == (npos, nup)
    Mh = M0.astype(np.float32)
    p = g.default_params(d=128, k=k, lr=0.05, seed=7, B=B, large_parts=K, p_gpu=2, s_gpu=1, large_serial=1,
                         large_pools=pools)
    st = g.gosh_train_level_large(gr.rowptr, gr.col, Mh, 0, e, p)
    assert (st["positives"], st["updates"]) == (npos, nup)
    assert rel_fro(Mh.astype(np.float64), Mo) <= 1e-5


_oracle_held = {}


@pytest.mark.parametrize("pools", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_parts_reach_oracle_quality(dtype, pools):
    """The default (overlapping) schedule on the planted partition of the
    small workload, K = 4 parts, 3 bins, B = 5, e = 300 from the random init:
    held-out AUC within 0.005 of the sequential LargeGraphGPU oracle's (means
    over 3 seeds; the oracle reaches >= 0.8), rounds * K(K+1)/2 kernels, and
    the global counter stops positives at e * |V|."""
    g = gosh()
    s = synth.workload("sbm12")
    gr = s.train
    e, K, B = 300, 4, 5
    got, ref = [], []
    for seed in (1, 2, 3):
        M0 = oracle.init_uniform(gr.n, 32, 0, seed).astype(np.float32)
        if seed not in _oracle_held:
            Mo = M0.astype(np.float64)
            oracle.train_large(gr.rowptr, gr.col, Mo, 3, 0, e, 0.045, 1e-4, seed, K, B)
            _oracle_held[seed] = oracle.link_auc(Mo, s.test_pos, s.test_neg)
        ref.append(_oracle_held[seed])
        Mh = torch.from_numpy(M0).to(dtype).contiguous()
        p = g.default_params(d=32, k=3, lr=0.045, seed=seed, dtype=dtype, B=B, large_parts=K, p_gpu=3, s_gpu=2,
                             large_pools=pools)
        st = g.gosh_train_level_large(gr.rowptr, gr.col, Mh, 0, e, p)
        assert st["parts"] == K and st["rounds"] == e // B and st["kernels"] == (e // B) * K * (K + 1) // 2
        assert st["positives"] == e * gr.n
        got.append(oracle.link_auc(Mh.double().numpy(), s.test_pos, s.test_neg))
    assert np.mean(ref) >= 0.8, ref
    assert abs(np.mean(got) - np.mean(ref)) <= 0.005, (np.round(got, 4), np.round(ref, 4))
