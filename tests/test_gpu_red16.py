"""16-bit tables in the lock-free atomic mode (the default): each row change
is the stochastically rounded new row minus the row read, added at L2.

- without a concurrent writer the stored row becomes exactly the rounded new
  row whenever the change fits the 16-bit significand (always for changes
  below 256 ulps of the stored value, the regime where stochastic rounding
  matters); with every value in [0.25, 0.5) in magnitude and small steps, a
  single warp whose simultaneous sources touch disjoint rows (edges
  (i, i+16), k = 0, one L-lane group per source) therefore leaves tables
  bit-identical to the plain stochastic-rounding stores of the paper's
  scheme (same rounding bits), for BF16 and FP16 and both lane widths;
- with many warps racing on the rows of the planted partition, the atomic
  mode reaches the sequential oracle's held-out AUC within 0.005 (means over
  3 seeds; plain stores lose updates on hub rows).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("lanes,spp", [(16, 2), (8, 2), (8, 4)])
def test_uncontended_atomic_equals_rounded_store(dtype, lanes, spp):
    g = gosh()
    n = 32
    gr = synth.csr_from_edges(n, np.arange(0, 16), np.arange(16, 32), compact=False)
    rng = np.random.default_rng(3)
    mag = rng.uniform(0.27, 0.47, (n, 128)) * np.where(rng.random((n, 128)) < 0.5, -1.0, 1.0)
    M0 = torch.from_numpy(mag.astype(np.float32)).to(dtype).cuda()
    csr = g.to_device_csr(gr.rowptr, gr.col)
    out = []
    for plain in (1, 0):
        M = M0.clone()
        p = g.default_params(d=128, k=0, lr=0.01, seed=8, dtype=dtype, lanes_per_row=lanes, samples_per_pass=spp,
                             vertices_per_warp=32, plain_stores=plain)
        g.gosh_train_level(csr, M, 0, 10, p)
        torch.cuda.synchronize()
        out.append(M.cpu())
    assert not torch.equal(out[1], M0.cpu())
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_atomic_16bit_reaches_oracle_auc(dtype):
    """300 level-0 epochs on the planted partition of the small workload
    (d = 128, k = 3, lr 0.045, default kernels): held-out AUC within 0.005 of
    the sequential FP64 oracle's (means over 3 seeds; the oracle reaches
    >= 0.8)."""
    g = gosh()
    s = synth.workload("sbm12")
    gr = s.train
    csr = g.to_device_csr(gr.rowptr, gr.col)
    got, ref = [], []
    for seed in (1, 2, 3):
        M0 = oracle.init_uniform(gr.n, 128, 0, seed).astype(np.float32)
        Mo = M0.astype(np.float64)
        oracle.train_sequential(gr.rowptr, gr.col, Mo, 3, 0, 300, 0.045, 1e-4, seed)
        ref.append(oracle.link_auc(Mo, s.test_pos, s.test_neg))
        M = torch.from_numpy(M0).to(dtype).cuda()
        g.gosh_train_level(csr, M, 0, 300, g.default_params(d=128, k=3, lr=0.045, seed=seed, dtype=dtype))
        got.append(oracle.link_auc(M.double().cpu().numpy(), s.test_pos, s.test_neg))
    assert np.mean(ref) >= 0.8, ref
    assert abs(np.mean(got) - np.mean(ref)) <= 0.005, (np.round(got, 4), np.round(ref, 4))
