"""Epoch concurrency on large levels (the future work of the paper's
epoch-synchronisation experiment, Sec. 6.3; gosh_params.epoch_overlap = c):
with up to c = 2 or 4 consecutive epochs of a level running at once (here on
every level of at least 1024 vertices, so that the small workload's level 0
overlaps), the embed keeps the sequential oracle's quality: R-MAT
training-edge AUC and planted-partition held-out AUC within 0.005 of the
oracle's (means over 3 seeds), as for the serialised epochs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

C1 = dict(k=3, lr=0.045, p=0.3)
_ref = {}


def fit_auc(M, gr):
    pos, neg = synth.fit_pairs(gr)
    return oracle.link_auc(M, pos, neg)


@pytest.mark.parametrize("c", [2, 4])
def test_overlapping_epochs_keep_oracle_quality(c):
    g = gosh()
    r, s = synth.workload("rmat12"), synth.workload("sbm12")
    got, ref = [], []
    for seed in (1, 2, 3):
        if seed not in _ref:
            Mr, _ = oracle.embed(r.train.rowptr, r.train.col, 32, e=200, seed=seed, epoch_unit="E", **C1)
            Ms, _ = oracle.embed(s.train.rowptr, s.train.col, 32, e=200, seed=seed, epoch_unit="E", **C1)
            _ref[seed] = (fit_auc(Mr, r.train), oracle.link_auc(Ms, s.test_pos, s.test_neg))
        ref.append(_ref[seed])
        row = []
        for sp in (r, s):
            p = g.default_params(d=32, epochs=200, seed=seed, epoch_unit=1, epoch_overlap=c,
                                 overlap_min_vertices=1024, **C1)
            M, _ = g.gosh_embed(torch.from_numpy(sp.train.rowptr).cuda(), torch.from_numpy(sp.train.col).cuda(), p)
            row.append(M.double().cpu().numpy())
        got.append((fit_auc(row[0], r.train), oracle.link_auc(row[1], s.test_pos, s.test_neg)))
    got, ref = np.array(got), np.array(ref)
    assert (np.abs(got.mean(0) - ref.mean(0)) <= 0.005).all(), (np.round(got, 4), np.round(ref, 4))
