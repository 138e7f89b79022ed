"""The OpenMP FP32 lock-free CPU baseline (cpu_hogwild/) that bench.py times
against the GPU: it builds, uses the host's threads, applies the expected
number of updates (k+1 per source and epoch, less sources without neighbours
and negatives equal to the source), and trains: on the planted-partition
graph of the small workload it predicts held-out edges."""
import numpy as np

import cpu_hogwild
import oracle
import synth


def test_hogwild_baseline_counts_and_learns():
    sp = synth.workload("sbm12")
    gr = sp.train
    assert cpu_hogwild.threads() >= 1
    M = (oracle.init_uniform(gr.n, 32, 0, 1)).astype(np.float32)
    e, k = 300, 3
    nup = cpu_hogwild.train_level(gr.rowptr, gr.col, M, k, e, 0.045, seed=3)
    full = e * gr.n * (k + 1)
    # negatives equal to the source: about e*n*k/n = e*k of them
    assert full - 10 * e * k <= nup <= full
    assert np.isfinite(M).all()
    assert oracle.link_auc(M.astype(np.float64), sp.test_pos, sp.test_neg) > 0.75
