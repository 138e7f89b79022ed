"""Learned projection on the GPU (tcgen05 GEMMs) against the FP64 oracle.

Tolerances: the GPU multiplies BF16 operands (weights, features, hidden
activations and back-propagated gradients are rounded to BF16, relative step
2^-8) with FP32 accumulation; the oracle runs FP64 on the same BF16-rounded
weights and features.  A chain of three roundings bounds the relative error
of a gradient by a few times 2^-8, so the tests take 3e-2 (norm-wise).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp
from gpu_common import bf16_round_np, gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 3e-2


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("d,hidden,n", [(32, 64, 300), (128, 256, 1000), (64, 256, 4096)])
def test_grads_match_oracle(d, hidden, n):
    g = gosh()
    m = g.Mlp(d, hidden, seed=1)
    rng = np.random.default_rng(d + n)
    din = 2 * d + 1
    W1 = bf16_round_np(rng.normal(size=(hidden, din)) * 0.2)
    b1 = rng.normal(size=hidden).astype(np.float32) * 0.1
    W2 = bf16_round_np(rng.normal(size=(d, hidden)) * 0.2)
    b2 = rng.normal(size=d).astype(np.float32) * 0.1
    m.set_weights(W1, b1, W2, b2)
    X = bf16_round_np(rng.normal(size=(n, din)))
    R = rng.normal(size=(n, d)).astype(np.float32)
    Xd = torch.zeros((n, m.stride), dtype=torch.bfloat16)
    Xd[:, :din] = torch.from_numpy(X).to(torch.bfloat16)
    L, (dW1, db1, dW2, db2) = m.grads(Xd.cuda(), torch.from_numpy(R).cuda())
    Lo, oW1, ob1, oW2, ob2 = omlp.loss_and_grads(W1, b1.astype(np.float64), W2, b2.astype(np.float64), X, R)
    assert abs(L - Lo) / Lo < TOL
    for got, ref in ((dW1, oW1), (db1, ob1), (dW2, oW2), (db2, ob2)):
        assert rel(got, ref) < TOL, rel(got, ref)


def test_features_match_oracle():
    g = gosh()
    gr = synth.rmat_graph(10, 8, 5)
    rng = np.random.default_rng(0)
    nc, d = 200, 64
    mp = rng.integers(0, nc, gr.n).astype(np.int32)
    Mc = bf16_round_np(rng.normal(size=(nc, d)))
    m = g.Mlp(d, 64)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    X = m.features(csr, torch.from_numpy(mp).cuda(), torch.from_numpy(Mc).to(torch.bfloat16).cuda())
    ref = omlp.features(gr.rowptr, gr.col, mp, Mc)
    got = X.float().cpu().numpy()[:, :2 * d + 1]
    # each entry is one BF16 rounding of an FP32 value: relative 2^-8
    np.testing.assert_allclose(got, ref, rtol=2 ** -7, atol=1e-6)
    assert np.all(X.float().cpu().numpy()[:, 2 * d + 1:] == 0)


def test_untrained_network_is_copy_projection():
    g = gosh()
    gr = synth.rmat_graph(10, 8, 6)
    rng = np.random.default_rng(1)
    nc, d = 150, 32
    mp = rng.integers(0, nc, gr.n).astype(np.int32)
    Mc = torch.from_numpy(rng.normal(size=(nc, d)).astype(np.float32)).cuda()
    csr = g.to_device_csr(gr.rowptr, gr.col)
    m = g.Mlp(d, 256, seed=3)
    Mf = torch.empty((gr.n, d), device="cuda")
    m.project(Mc, torch.from_numpy(mp).cuda(), csr, Mf)
    np.testing.assert_array_equal(Mf.cpu().numpy(), Mc.cpu().numpy()[mp])


def test_training_fits_a_teacher_network():
    """Targets produced by a random teacher MLP on real features: Adam on the
    GPU must cut the residual error by an order of magnitude."""
    g = gosh()
    gr = synth.rmat_graph(12, 8, 7)
    rng = np.random.default_rng(2)
    nc, d = 400, 32
    mp = rng.integers(0, nc, gr.n).astype(np.int32)
    Mc = rng.normal(size=(nc, d)).astype(np.float32) * 0.3
    X = omlp.features(gr.rowptr, gr.col, mp, Mc)
    tW1 = rng.normal(size=(64, 2 * d + 1)) * 0.2
    tW2 = rng.normal(size=(d, 64)) * 0.2
    Y, _ = omlp.forward(tW1, np.zeros(64), tW2, np.zeros(d), X)
    Mf = (Mc[mp] + Y).astype(np.float32)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    m = g.Mlp(d, 256, seed=4)
    mpd = torch.from_numpy(mp).cuda()
    first = m.train(csr, mpd, torch.from_numpy(Mc).cuda(), torch.from_numpy(Mf).cuda(), epochs=1, lr=1e-3, batch=512)
    last = m.train(csr, mpd, torch.from_numpy(Mc).cuda(), torch.from_numpy(Mf).cuda(), epochs=60, lr=1e-3, batch=512)
    base = float((Y ** 2).sum(1).mean())   # error of the copy projection
    assert first < base
    assert last < 0.1 * base, (first, last, base)


def test_learned_projection_gains_over_copy():
    """What the trained network adds: on R-MAT scale 12 (d=32, k=3, lr 0.045,
    100 epochs of |E| updates over the hierarchy, BF16 tables) the learned
    projection between levels fits the training edges better than the copy
    projection at the same epochs: training-edge AUC higher by more than
    0.01 (means over 3 seeds; measured about +0.03)."""
    g = gosh()
    sp = synth.workload("rmat12")
    gr = sp.train
    rp, co = torch.from_numpy(gr.rowptr).cuda(), torch.from_numpy(gr.col).cuda()
    src = np.repeat(np.arange(gr.n), np.diff(gr.rowptr))
    keep = src < gr.col
    pos = np.stack([src[keep], gr.col[keep]], 1)
    rng = np.random.default_rng(5)
    neg = rng.integers(0, gr.n, size=(len(pos), 2))
    neg = neg[neg[:, 0] != neg[:, 1]]
    pos_d, neg_d = torch.from_numpy(pos.astype(np.int32)).cuda(), torch.from_numpy(neg.astype(np.int32)).cuda()
    auc = {0: [], 1: []}
    for seed in (1, 2, 3):
        for proj in (0, 1):
            p = g.default_params(d=32, k=3, lr=0.045, epochs=100, p=0.3, seed=seed, dtype=torch.bfloat16,
                                 projection=proj, epoch_unit=1)
            M, _ = g.gosh_embed(rp, co, p)
            auc[proj].append(g.gosh_link_auc(M, pos_d, neg_d))
    assert np.mean(auc[1]) > np.mean(auc[0]) + 0.01, auc


def test_features_hubs_and_isolated_vertices():
    """Rows longer than one gather span (a 5000-leaf star and a 2500-entry
    hub) are summed from span partials; vertices without neighbours get a zero
    mean; both against the oracle's definition."""
    g = gosh()
    rng = np.random.default_rng(5)
    n = 9000
    s = np.concatenate([np.zeros(5000, np.int64), np.full(2500, 6000), rng.integers(7000, 8000, 3000)])
    t = np.concatenate([np.arange(1, 5001), rng.choice(np.arange(6001, 9000), 2500, replace=False),
                        rng.integers(7000, 8000, 3000)])
    keep = s != t
    gr = synth.csr_from_edges(n, s[keep], t[keep], compact=False)
    assert np.diff(gr.rowptr).max() >= 5000 and (np.diff(gr.rowptr) == 0).any()
    nc, d = 300, 128
    mp = rng.integers(0, nc, n).astype(np.int32)
    Mc = bf16_round_np(rng.normal(size=(nc, d)))
    m = g.Mlp(d, 64)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    X = m.features(csr, torch.from_numpy(mp).cuda(), torch.from_numpy(Mc).to(torch.bfloat16).cuda())
    ref = omlp.features(gr.rowptr, gr.col, mp, Mc)
    np.testing.assert_allclose(X.float().cpu().numpy()[:, :2 * d + 1], ref, rtol=2 ** -7, atol=1e-6)


@pytest.mark.parametrize("d,hidden", [(32, 64), (128, 256), (64, 512)])
def test_projection_matches_oracle_forward(d, hidden):
    """gosh_project_learned with random weights: Mf - copy equals the oracle's
    forward pass on the BF16-rounded weights and features (the GPU also rounds
    the hidden layer to BF16: tolerance 3e-2 norm-wise)."""
    g = gosh()
    gr = synth.rmat_graph(11, 8, 9)
    rng = np.random.default_rng(d + hidden)
    nc = 500
    din = 2 * d + 1
    mp = rng.integers(0, nc, gr.n).astype(np.int32)
    Mc = bf16_round_np(rng.normal(size=(nc, d)) * 0.5)
    W1 = bf16_round_np(rng.normal(size=(hidden, din)) * 0.2)
    b1 = rng.normal(size=hidden).astype(np.float32) * 0.1
    W2 = bf16_round_np(rng.normal(size=(d, hidden)) * 0.2)
    b2 = rng.normal(size=d).astype(np.float32) * 0.1
    m = g.Mlp(d, hidden, seed=1)
    m.set_weights(W1, b1, W2, b2)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    Mf = torch.empty((gr.n, d), device="cuda")
    m.project(torch.from_numpy(Mc.astype(np.float32)).cuda(), torch.from_numpy(mp).cuda(), csr, Mf)
    X = bf16_round_np(omlp.features(gr.rowptr, gr.col, mp, Mc)).astype(np.float64)
    Y, _ = omlp.forward(W1, b1.astype(np.float64), W2, b2.astype(np.float64), X)
    got = Mf.double().cpu().numpy() - Mc[mp]
    assert rel(got, Y) < TOL, rel(got, Y)


def _bf16_forward_ref(W1, b1, W2, b2, X):
    """The forward pass with the GPU's roundings: BF16 features and weights
    (given), FP64 sums, the hidden layer rounded to BF16."""
    H = bf16_round_np(np.maximum(X @ W1.T + b1, 0.0))
    return H @ W2.T + b2


@pytest.mark.parametrize("d,hidden,dt,scale", [(128, 256, "f32", 16), (128, 256, "bf16", 15), (64, 256, "f16", 15),
                                                (32, 64, "bf16", 15), (64, 128, "f32", 15)])
def test_projection_tiles_tables_ragged(d, hidden, dt, scale):
    """gosh_project_learned over more 128-row tiles than SMs (so each CTA of
    the fused persistent kernel walks several tiles, its stage ring and
    barrier phases wrapping), a ragged last tile, and every table type: Mf -
    copy against the oracle's forward pass with the GPU's BF16 roundings
    (features, weights, hidden layer), norm-wise and row by row (a row from
    the wrong tile or a mis-swizzled hidden block is off by O(1)).  Hidden
    width 64 takes the two-GEMM form (the fused kernel takes 128 and 256)."""
    g = gosh()
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dt]
    gr = synth.rmat_graph(scale, 8, 9)
    assert gr.n > 152 * 128 and gr.n % 128 != 0
    rng = np.random.default_rng(d + hidden + scale)
    nc = 3000
    din = 2 * d + 1
    mp = rng.integers(0, nc, gr.n).astype(np.int32)
    Mc_t = torch.from_numpy((rng.normal(size=(nc, d)) * 0.5).astype(np.float32)).to(tdt)
    Mc = Mc_t.double().numpy()
    W1 = bf16_round_np(rng.normal(size=(hidden, din)) * 0.1)
    b1 = rng.normal(size=hidden).astype(np.float32) * 0.1
    W2 = bf16_round_np(rng.normal(size=(d, hidden)) * 0.1)
    b2 = rng.normal(size=d).astype(np.float32) * 0.1
    m = g.Mlp(d, hidden, seed=1)
    m.set_weights(W1, b1, W2, b2)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    Mf = torch.empty((gr.n, d), device="cuda", dtype=tdt)
    m.project(Mc_t.cuda(), torch.from_numpy(mp).cuda(), csr, Mf)
    X = bf16_round_np(omlp.features(gr.rowptr, gr.col, mp, Mc)).astype(np.float64)
    Y = _bf16_forward_ref(W1, b1.astype(np.float64), W2, b2.astype(np.float64), X)
    got = Mf.double().cpu().numpy() - Mc[mp]
    # FP32 tables: FP32 accumulation and hidden-layer rounding flips only;
    # 16-bit tables add the rounding of Mf itself (2^-9 / 2^-12 of |Mf|)
    tol = {"f32": 4e-3, "f16": 6e-3, "bf16": 2.5e-2}[dt]
    assert rel(got, Y) < tol, rel(got, Y)
    row_err = np.linalg.norm(got - Y, axis=1) / np.maximum(np.linalg.norm(Y, axis=1), 1e-3)
    assert row_err.max() < 8 * tol, (int(row_err.argmax()), float(row_err.max()))
