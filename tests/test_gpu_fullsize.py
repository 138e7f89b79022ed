"""Parity at the benchmark's full size: R-MAT scale 20, edge factor 16, 80%
training split (614,524 vertices, 25.1 M CSR entries), d = 128, k = 3.

- coarsening: every level's map and CSR bit-exact against the oracle;
- one deterministic epoch of level 0 (FP32, snapshot batches of 4096) within
  the deterministic-mode bar, 1e-5 relative, against the FP64 oracle;
- the lock-free step as bench.py runs it (e = 200 over the hierarchy): the
  FP32 held-out and training-edge AUC within 0.005 of the sequential oracle's
  and sane update counts for the BF16 tables.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c2():
    return synth.workload("rmat20")


def test_fullsize_coarsening_bit_exact(c2):
    g = gosh()
    gr = c2.train
    graphs, maps = oracle.mec_hierarchy(gr.rowptr, gr.col)
    h = g.gosh_coarsen(g.to_device_csr(gr.rowptr, gr.col))
    assert len(h) == len(graphs)
    for i in range(len(graphs)):
        rp, co, mp = h.level_arrays(i)
        np.testing.assert_array_equal(rp, graphs[i][0])
        np.testing.assert_array_equal(co, graphs[i][1])
        if i < len(maps):
            np.testing.assert_array_equal(mp, maps[i])


def test_fullsize_deterministic_epoch(c2):
    g = gosh()
    gr = c2.train
    M0 = oracle.init_uniform(gr.n, 128, 0, 7).astype(np.float32).astype(np.float64) * 30
    Mo = M0.copy()
    lo, no = oracle.train_deterministic(gr.rowptr, gr.col, Mo, 3, 0, 1, 0.045, 1e-4, 21, 4096)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = torch.from_numpy(M0.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    nup = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = g.default_params(d=128, k=3, lr=0.045, seed=21, mode="deterministic", det_batch=4096)
    g.gosh_train_level(csr, M, 0, 1, p, loss=loss, n_updates=nup)
    assert int(nup.item()) == no
    assert rel_fro(M.double().cpu().numpy(), Mo) <= 1e-5
    assert abs(float(loss.item()) - lo[0]) <= 1e-5 * lo[0]


def fit_auc(M, gr, seed=0):
    src = np.repeat(np.arange(gr.n), np.diff(gr.rowptr))
    rng = np.random.default_rng(seed)
    rnd = np.stack([rng.integers(0, gr.n, 200000), rng.integers(0, gr.n, 200000)], 1)
    pick = rng.integers(0, len(src), 200000)
    return oracle.link_auc(M, np.stack([src[pick], gr.col[pick]], 1), rnd)


def test_fullsize_lockfree_matches_oracle_auc(c2):
    g = gosh()
    gr = c2.train
    Mo, info = oracle.embed(gr.rowptr, gr.col, 128, 3, 0.045, 200, 0.3, seed=11)
    rp, co = torch.from_numpy(gr.rowptr).cuda(), torch.from_numpy(gr.col).cuda()
    p = g.default_params(d=128, k=3, lr=0.045, epochs=200, p=0.3, seed=11)
    Mg, st = g.gosh_embed(rp, co, p)
    s = g.stats_dict(st)
    assert s["epochs"] == info["epochs"]
    Mgn = Mg.double().cpu().numpy()
    ho = oracle.link_auc(Mo, c2.test_pos, c2.test_neg)
    hg = oracle.link_auc(Mgn, c2.test_pos, c2.test_neg)
    fo, fg = fit_auc(Mo, gr), fit_auc(Mgn, gr)
    assert abs(ho - hg) <= 0.005, (ho, hg)
    assert abs(fo - fg) <= 0.005, (fo, fg)
    # BF16 tables as bench.py times them: finite, and the applied-update count
    # within the draws' skip rate (a source without neighbours skips its
    # positive; a negative equal to the source is skipped)
    pb = g.default_params(d=128, k=3, lr=0.045, epochs=200, p=0.3, seed=11, dtype=torch.bfloat16)
    Mb, stb = g.gosh_embed(rp, co, pb)
    sb = g.stats_dict(stb)
    assert torch.isfinite(Mb.float()).all()
    full = sum(e * n * 4 for e, n in zip(sb["epochs"], sb["n"]))
    assert 0.99 * full <= sb["updates"] <= full
