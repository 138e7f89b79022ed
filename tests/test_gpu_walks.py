"""Random-walk positives (Sec. 3.2) through the C ABI against the oracle.

- Graphs whose epochs have at most 32 pair positions, trained with 32 lanes
  per source (FP32, d = 128), run in one warp one pair at a time in the
  permuted order: the epochs are the oracle's sequential ones (walks drawn on
  host threads, permutation and negatives on the device), to 1e-5, with the
  same number of updates; a device CSR gives the same result as a host one.
- On the planted partition of the small workload the held-out AUC of
  lock-free walk training (FP32 and BF16 tables) is within 0.005 of the
  sequential oracle's (means over 3 seeds).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def small_graphs():
    gs = [synth.random_graph(5, 0.5, 3), synth.random_graph(6, 0.4, 4),
          synth.csr_from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]), compact=False),
          synth.csr_from_edges(6, np.array([0, 0, 0]), np.array([1, 2, 3]), compact=False)]
    return gs


@pytest.mark.parametrize("k", [0, 3])
def test_walks_single_warp_is_sequential(k):
    g = gosh()
    l, w = 4, 2
    for gi, gr in enumerate(small_graphs()):
        assert gr.n * oracle.walk_pairs_per_walk(l, w) <= 32
        M0 = oracle.init_uniform(gr.n, 128, 0, 3 + gi).astype(np.float32).astype(np.float64) * 60
        Mo = M0.copy()
        _, no = oracle.train_walks(gr.rowptr, gr.col, Mo, k, 1, 6, 0.05, 1e-4, 11 + gi, l, w)
        p = g.default_params(d=128, k=k, lr=0.05, seed=11 + gi, lanes_per_row=32, walk_length=l, walk_window=w)
        for on_device in (False, True):
            M = torch.tensor(M0, dtype=torch.float32, device="cuda")
            nup = torch.zeros(1, dtype=torch.int64, device="cuda")
            if on_device:
                csr = g.to_device_csr(gr.rowptr, gr.col)
                cg = csr.c()
                g._check("gosh_train_level_walks", g.lib().gosh_train_level_walks(
                    g.C.byref(cg), g._ptr(M), 1, 6, g.C.byref(p), None, g._ptr(nup), None))
            else:
                g.gosh_train_level_walks(gr.rowptr, gr.col, M, 1, 6, p, n_updates=nup)
            torch.cuda.synchronize()
            assert int(nup.item()) == no
            assert rel_fro(M.double().cpu().numpy(), Mo) <= 1e-5


_oracle_held = {}


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_walks_auc_matches_oracle(dtype):
    """Lock-free walk training (walks of 6, window 2, k = 3, 20 epochs, lr
    0.1) on the planted partition of the small workload: held-out AUC within
    0.005 of the sequential oracle's (means over 3 seeds; the oracle reaches
    >= 0.8)."""
    g = gosh()
    s = synth.workload("sbm12")
    gr = s.train
    got, ref = [], []
    for seed in (1, 2, 3):
        M0 = oracle.init_uniform(gr.n, 32, 0, seed)
        if seed not in _oracle_held:
            Mo = M0.copy()
            oracle.train_walks(gr.rowptr, gr.col, Mo, 3, 0, 20, 0.1, 1e-4, seed, 6, 2)
            _oracle_held[seed] = oracle.link_auc(Mo, s.test_pos, s.test_neg)
        ref.append(_oracle_held[seed])
        p = g.default_params(d=32, k=3, lr=0.1, seed=seed, dtype=dtype, walk_length=6, walk_window=2)
        M = torch.tensor(M0, dtype=torch.float32).to(dtype).cuda()
        st = g.gosh_train_level_walks(gr.rowptr, gr.col, M, 0, 20, p)
        assert st["positions"] == gr.n * oracle.walk_pairs_per_walk(6, 2)
        got.append(oracle.link_auc(M.double().cpu().numpy(), s.test_pos, s.test_neg))
    assert np.mean(ref) >= 0.8, ref
    assert abs(np.mean(got) - np.mean(ref)) <= 0.005, (np.round(got, 4), np.round(ref, 4))
