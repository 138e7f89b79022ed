"""TMA-staged lock-free training kernel (cp.async.bulk row gathers into a
shared-memory ring) against the oracle.

- one warp with one source per round (FP32, d = 128, 32 lanes) prefetches the
  next round's rows while updating the current round, so rows of a later
  source may be staged before an earlier source updated them; when
  consecutive sources touch disjoint rows (edges (i, i+16), negatives
  excluded by k = 0) the result is still the sequential epoch: within 1e-5
  of the oracle;
- on R-MAT scale 12 the staged kernel reaches the oracle's training-edge AUC
  within 0.01 (FP32 and BF16, both with atomic row changes), and draws
  exactly the oracle's update count.
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


def fit_auc(M, gr, seed=0):
    src = np.repeat(np.arange(gr.n), np.diff(gr.rowptr))
    rng = np.random.default_rng(seed)
    rnd = np.stack([rng.integers(0, gr.n, 20000), rng.integers(0, gr.n, 20000)], 1)
    return oracle.link_auc(M, np.stack([src, gr.col], 1), rnd)


@pytest.mark.parametrize("dtype,lanes,ks", [(torch.float32, 32, 4), (torch.float32, 16, 6),
                                            (torch.bfloat16, 8, 4), (torch.bfloat16, 4, 6)])
def test_staged_kernel_quality_and_counts(dtype, lanes, ks):
    g = gosh()
    gr = synth.rmat_graph(12, 8, 41)
    k = ks - 1
    M0 = oracle.init_uniform(gr.n, 128, 0, 4).astype(np.float32) * 20
    Mo = M0.astype(np.float64)
    _, no = oracle.train_sequential(gr.rowptr, gr.col, Mo, k, 0, 60, 0.045, 1e-4, 6)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = torch.from_numpy(M0).to(dtype).cuda()
    nup = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = g.default_params(d=128, k=k, lr=0.045, seed=6, dtype=dtype, lanes_per_row=lanes, samples_per_pass=-ks)
    g.gosh_train_level(csr, M, 0, 60, p, n_updates=nup)
    assert g.lib().gosh_device_check(None) == 0
    assert int(nup.item()) == no
    a_o, a_g = fit_auc(Mo, gr), fit_auc(M.double().cpu().numpy(), gr)
    # FP32 and 16-bit rows both change by atomic additions at L2 (16-bit: the
    # stochastically rounded change), so rows staged a round ahead are read
    # stale but no update is overwritten
    assert abs(a_o - a_g) <= 0.01, (a_o, a_g)
