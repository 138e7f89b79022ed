"""TMA-staged lock-free training kernel (cp.async.bulk row gathers into a
shared-memory ring) against the oracle.

- one warp with one source per round (FP32, d = 128, 32 lanes) prefetches the
  next round's rows while updating the current round, so rows of a later
  source may be staged before an earlier source updated them; when
  consecutive sources touch disjoint rows (edges (i, i+16), negatives
  excluded by k = 0) the result is still the sequential epoch: within 1e-5
  of the oracle;
- on the planted partition of the small workload (300 level-0 epochs,
  d = 128) the staged kernel reaches the oracle's held-out AUC within 0.005
  (means over 3 seeds; FP32 and BF16, both with atomic row changes), and
  draws exactly the oracle's update count.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_staged_single_warp_matches_sequential():
    g = gosh()
    n = 32
    # edges (i, i+16): consecutive sources q and q+1 touch disjoint rows
    gr = synth.csr_from_edges(n, np.arange(0, 16), np.arange(16, 32), compact=False)
    M0 = oracle.init_uniform(n, 128, 0, 3).astype(np.float32).astype(np.float64) * 60
    Mo = M0.copy()
    lo, no = oracle.train_sequential(gr.rowptr, gr.col, Mo, 0, 0, 10, 0.05, 1e-4, 8)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = torch.from_numpy(M0.astype(np.float32)).cuda()
    nup = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = g.default_params(d=128, k=0, lr=0.05, seed=8, lanes_per_row=32, samples_per_pass=-4, vertices_per_warp=32)
    g.gosh_train_level(csr, M, 0, 10, p, n_updates=nup)
    torch.cuda.synchronize()
    assert int(nup.item()) == no
    assert rel_fro(M.double().cpu().numpy(), Mo) <= 1e-5


_oracle_held = {}


def oracle_held(s, k, seed):
    """Held-out AUC of the sequential oracle: 300 epochs of level-0 training
    on the planted partition of the small workload (d = 128, lr 0.045) from
    the init; returns (AUC, update count)."""
    if (k, seed) not in _oracle_held:
        Mo = oracle.init_uniform(s.train.n, 128, 0, seed).astype(np.float32).astype(np.float64)
        _, no = oracle.train_sequential(s.train.rowptr, s.train.col, Mo, k, 0, 300, 0.045, 1e-4, seed)
        _oracle_held[(k, seed)] = (oracle.link_auc(Mo, s.test_pos, s.test_neg), no)
    return _oracle_held[(k, seed)]


@pytest.mark.parametrize("dtype,lanes,ks", [(torch.float32, 32, 4), (torch.float32, 16, 6),
                                            (torch.bfloat16, 8, 4), (torch.bfloat16, 4, 6)])
def test_staged_kernel_quality_and_counts(dtype, lanes, ks):
    g = gosh()
    s = synth.workload("sbm12")
    gr = s.train
    k = ks - 1
    csr = g.to_device_csr(gr.rowptr, gr.col)
    got, ref = [], []
    for seed in (1, 2, 3):
        a_o, no = oracle_held(s, k, seed)
        M0 = oracle.init_uniform(gr.n, 128, 0, seed).astype(np.float32)
        M = torch.from_numpy(M0).to(dtype).cuda()
        nup = torch.zeros(1, dtype=torch.int64, device="cuda")
        p = g.default_params(d=128, k=k, lr=0.045, seed=seed, dtype=dtype, lanes_per_row=lanes, samples_per_pass=-ks)
        g.gosh_train_level(csr, M, 0, 300, p, n_updates=nup)
        assert g.lib().gosh_device_check(None) == 0
        assert int(nup.item()) == no
        got.append(oracle.link_auc(M.double().cpu().numpy(), s.test_pos, s.test_neg))
        ref.append(a_o)
    # FP32 and 16-bit rows both change by atomic additions at L2 (16-bit: the
    # stochastically rounded change), so rows staged a round ahead are read
    # stale but no update is overwritten
    assert np.mean(ref) >= 0.8, ref
    assert abs(np.mean(got) - np.mean(ref)) <= 0.005, (np.round(got, 4), np.round(ref, 4))
