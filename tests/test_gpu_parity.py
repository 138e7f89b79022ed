"""GPU path (through the C ABI) against the CPU oracle, element by element.

Bars (see the tolerance derivation next to each test):
  - integer work (coarsening maps, coarse CSRs), initialisation and copy
    projection: bit-exact;
  - deterministic-mode training (FP32 tables) vs the FP64 oracle running the
    same snapshot batches: relative Frobenius error <= 1e-5;
  - Hogwild on a graph small enough to occupy one warp with one source per
    round is sequential, so it meets the same 1e-5 bar against the sequential
    oracle; larger graphs are judged by link-prediction AUC within 0.005 of
    the oracle's (means over 3 seeds) at a schedule where the oracle learns.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import bf16_round_np, gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

DET_TOL = 1e-5  # relative Frobenius, deterministic FP32 vs FP64 oracle


@pytest.fixture(scope="module")
def g():
    return gosh()


@pytest.fixture(scope="module")
def c1():
    return synth.workload("rmat12")


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ----------------------------------------------------------------- init
@pytest.mark.parametrize("d", [32, 64, 128])
@pytest.mark.parametrize("n", [1, 33, 1000])
def test_init_bit_exact(g, d, n):
    M = torch.empty((n, d), dtype=torch.float32, device="cuda")
    g.gosh_init_embedding(M, level=5, seed=123, graph_id=7)
    ref = oracle.init_uniform(n, d, 5, 123, 7).astype(np.float32)
    np.testing.assert_array_equal(M.cpu().numpy(), ref)
    Mb = torch.empty((n, d), dtype=torch.bfloat16, device="cuda")
    g.gosh_init_embedding(Mb, level=5, seed=123, graph_id=7)
    np.testing.assert_array_equal(Mb.float().cpu().numpy(), bf16_round_np(ref))


# ----------------------------------------------------------------- coarsening
def check_hierarchy(g, rowptr, col, threshold=100, shrink=0.8):
    graphs, maps = oracle.mec_hierarchy(rowptr, col, threshold, shrink)
    csr = g.to_device_csr(rowptr, col)
    h = g.gosh_coarsen(csr, threshold, shrink)
    assert len(h) == len(graphs)
    for i in range(len(graphs)):
        rp, co, mp = h.level_arrays(i)
        np.testing.assert_array_equal(rp, graphs[i][0])
        np.testing.assert_array_equal(co, graphs[i][1])
        if i < len(maps):
            np.testing.assert_array_equal(mp, maps[i])
    h.close()
    return len(graphs)


def test_coarsen_rmat12_bit_exact(g, c1):
    D = check_hierarchy(g, c1.train.rowptr, c1.train.col)
    assert D >= 3


@pytest.mark.parametrize("scale,ef,seed", [(14, 4, 1), (15, 16, 2), (10, 32, 3)])
def test_coarsen_rmat_bit_exact(g, scale, ef, seed):
    gr = synth.rmat_graph(scale, ef, seed)
    check_hierarchy(g, gr.rowptr, gr.col)


@pytest.mark.parametrize("bitmap_max", ["0", "2000"])
def test_coarsen_sorted_path_bit_exact(g, monkeypatch, bitmap_max):
    # coarse graphs with more vertices than the bitmap limit are built by a
    # radix sort of packed edge keys; lowering the limit runs that path on
    # every level ("0") or on the wide first levels only ("2000")
    monkeypatch.setenv("GOSH_COARSEN_BITMAP_MAX", bitmap_max)
    gr = synth.rmat_graph(14, 8, 5)
    assert check_hierarchy(g, gr.rowptr, gr.col) >= 3


def test_coarsen_multi_chunk_rows(g):
    # two hubs with 6000 leaves each plus leaf-leaf edges across them: each
    # hub's cluster row spans several 4096-entry chunks (global bitmap path)
    rng = np.random.default_rng(9)
    leaves = 6000
    a = np.arange(2, 2 + leaves)
    b = np.arange(2 + leaves, 2 + 2 * leaves)
    s = np.concatenate([np.zeros(leaves, np.int64), np.ones(leaves, np.int64), rng.choice(a, 3000)])
    t = np.concatenate([a, b, rng.choice(b, 3000)])
    gr = synth.csr_from_edges(2 + 2 * leaves, s, t, compact=False)
    check_hierarchy(g, gr.rowptr, gr.col, threshold=1)


def test_coarsen_edge_cases(g):
    # no edges at all: every vertex is its own cluster, one level added
    check_hierarchy(g, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32))
    # single vertex
    check_hierarchy(g, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32))
    # isolated vertices mixed with a star and a path; threshold 1 forces depth
    s = np.array([0, 0, 0, 0, 5, 6, 7])
    t = np.array([1, 2, 3, 4, 6, 7, 8])
    gr = synth.csr_from_edges(12, s, t, compact=False)
    check_hierarchy(g, gr.rowptr, gr.col, threshold=1)
    # random small graphs of every density
    rng = np.random.default_rng(0)
    for trial in range(40):
        n = int(rng.integers(2, 200))
        gr = synth.random_graph(n, float(rng.uniform(0.0, 0.5)), int(rng.integers(1 << 30)))
        check_hierarchy(g, gr.rowptr, gr.col, threshold=int(rng.integers(1, 20)))


# ----------------------------------------------------------------- projection
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_project_copy_exact(g, dtype):
    rng = np.random.default_rng(1)
    nc, nf, d = 300, 5000, 64
    mp = rng.integers(0, nc, nf).astype(np.int32)
    Mc = torch.randn(nc, d, generator=torch.Generator().manual_seed(0)).to(dtype)
    ref = oracle.project_copy(mp, Mc.double().numpy())
    Mf = torch.empty((nf, d), dtype=dtype, device="cuda")
    g.gosh_project(Mc.cuda(), dev(mp), Mf)
    np.testing.assert_array_equal(Mf.double().cpu().numpy(), ref)


# ----------------------------------------------------------------- training
def train_gpu(g, gr, M0, k, level, epochs, lr, seed, mode, m=1, dtype=torch.float32, d=None, lanes=0, pas=0):
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = dev(M0, dtype)
    p = g.default_params(d=M0.shape[1], k=k, lr=lr, dtype=dtype, mode=mode, det_batch=m, seed=seed,
                         lanes_per_row=lanes, samples_per_pass=pas, vertices_per_warp=32 if lanes == 32 else 0)
    loss = torch.zeros(max(epochs, 1), dtype=torch.float64, device="cuda")
    nup = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.gosh_train_level(csr, M, level, epochs, p, loss=loss, n_updates=nup)
    torch.cuda.synchronize()
    return M.double().cpu().numpy(), loss.cpu().numpy()[:epochs], int(nup.item())


@pytest.mark.parametrize("d", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("k,m", [(3, 64), (3, 1), (5, 257), (1, 10 ** 6)])
def test_deterministic_matches_oracle(g, c1, d, k, m):
    gr = c1.train
    epochs = 3 if m == 1 else 8
    M0 = oracle.init_uniform(gr.n, d, 2, 99).astype(np.float32).astype(np.float64) * 30
    Mo = M0.copy()
    lo, no = oracle.train_deterministic(gr.rowptr, gr.col, Mo, k, 2, epochs, 0.045, 1e-4, 4242, m)
    Mg, lg, ng = train_gpu(g, gr, M0, k, 2, epochs, 0.045, 4242, "deterministic", m=m)
    assert ng == no
    assert rel_fro(Mg, Mo) <= DET_TOL
    np.testing.assert_allclose(lg, lo, rtol=1e-5)


def test_deterministic_is_run_to_run_identical(g, c1):
    gr = c1.train
    M0 = oracle.init_uniform(gr.n, 64, 0, 5).astype(np.float32).astype(np.float64) * 30
    a = train_gpu(g, gr, M0, 3, 0, 4, 0.045, 1, "deterministic", m=500)[0]
    b = train_gpu(g, gr, M0, 3, 0, 4, 0.045, 1, "deterministic", m=500)[0]
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_hogwild_single_warp_is_sequential(g, k):
    # n <= 32 and 32 lanes per source (FP32, d=128): one warp, one source per
    # round, so the lock-free epoch runs the sources in id order.
    gr = synth.random_graph(30, 0.2, 17)
    M0 = oracle.init_uniform(gr.n, 128, 0, 3).astype(np.float32).astype(np.float64) * 60
    Mo = M0.copy()
    lo, no = oracle.train_sequential(gr.rowptr, gr.col, Mo, k, 0, 20, 0.05, 1e-4, 8)
    for pas in (2, 4):
        Mg, lg, ng = train_gpu(g, gr, M0, k, 0, 20, 0.05, 8, "hogwild", lanes=32, pas=pas)
        assert ng == no
        assert rel_fro(Mg, Mo) <= DET_TOL
        np.testing.assert_allclose(lg, lo, rtol=1e-5)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_hogwild_single_warp_all_epochs_in_one_launch(g, k):
    # With cooperative_epochs and no loss request a small level runs every
    # epoch in one cooperative launch, each epoch's samples drawn before the
    # barrier that closes the previous one: the single-warp epochs must still
    # be the sequential ones.
    gr = synth.random_graph(30, 0.2, 17)
    M0 = oracle.init_uniform(gr.n, 128, 0, 3).astype(np.float32).astype(np.float64) * 60
    Mo = M0.copy()
    _, no = oracle.train_sequential(gr.rowptr, gr.col, Mo, k, 0, 20, 0.05, 1e-4, 8)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    for coop in (1, 0):
        for pas in (2, 4):
            M = dev(M0, torch.float32)
            p = g.default_params(d=128, k=k, lr=0.05, seed=8, lanes_per_row=32, samples_per_pass=pas,
                                 vertices_per_warp=32, cooperative_epochs=coop)
            nup = torch.zeros(1, dtype=torch.int64, device="cuda")
            g.gosh_train_level(csr, M, 0, 20, p, n_updates=nup)
            torch.cuda.synchronize()
            assert int(nup.item()) == no
            assert rel_fro(M.double().cpu().numpy(), Mo) <= DET_TOL


# Quality bars of the lock-free path (held-out and training-edge AUC) are
# applied where the oracle learns: the small workload's schedule (d = 32, k = 3,
# lr 0.045, e = 200 epochs of |E| updates, p = 0.3) fits the R-MAT scale-12
# training edges (oracle AUC >= 0.9) and predicts held-out edges of the
# planted partition of the same size (oracle AUC >= 0.8); each bar is a mean
# over seeds 1-3, and the seed spread is reported with it.
SEEDS = (1, 2, 3)
C1 = dict(k=3, lr=0.045, p=0.3)
E1 = 200


@pytest.fixture(scope="module")
def s1():
    return synth.workload("sbm12")


def fit_auc(M, gr, seed=5):
    """Training-edge AUC: every training edge (u < v) against as many uniform
    vertex pairs."""
    src = np.repeat(np.arange(gr.n), np.diff(gr.rowptr))
    keep = src < gr.col
    pos = np.stack([src[keep], gr.col[keep]], 1)
    rng = np.random.default_rng(seed)
    neg = rng.integers(0, gr.n, size=(len(pos), 2))
    return oracle.link_auc(M, pos, neg[neg[:, 0] != neg[:, 1]])


_oracle_cache = {}


def oracle_quality(r, s, d):
    """Oracle (FP64, sequential) AUCs per seed: (R-MAT fit, planted held-out, planted fit)."""
    key = d
    if key not in _oracle_cache:
        out = []
        for seed in SEEDS:
            Mr, _ = oracle.embed(r.train.rowptr, r.train.col, d, e=E1, seed=seed, epoch_unit="E", **C1)
            Ms, _ = oracle.embed(s.train.rowptr, s.train.col, d, e=E1, seed=seed, epoch_unit="E", **C1)
            out.append((fit_auc(Mr, r.train), oracle.link_auc(Ms, s.test_pos, s.test_neg), fit_auc(Ms, s.train)))
        _oracle_cache[key] = np.array(out)
    return _oracle_cache[key]


def gpu_quality(g, r, s, d, dtype=torch.float32, **kw):
    out = []
    for seed in SEEDS:
        row = []
        for sp in (r, s):
            p = g.default_params(d=d, epochs=E1, seed=seed, dtype=dtype, epoch_unit=1, **C1, **kw)
            M, _ = g.gosh_embed(dev(sp.train.rowptr), dev(sp.train.col), p)
            row.append(M.double().cpu().numpy())
        out.append((fit_auc(row[0], r.train), oracle.link_auc(row[1], s.test_pos, s.test_neg),
                    fit_auc(row[1], s.train)))
    return np.array(out)


def check_quality(got, ref, bar=0.005, floors=(0.9, 0.8, 0.9)):
    names = ("R-MAT training-edge", "planted held-out", "planted training-edge")
    for j, name in enumerate(names):
        msg = "%s AUC: GPU %s (spread %.4f) vs oracle %s (spread %.4f)" % (
            name, np.round(got[:, j], 4), np.ptp(got[:, j]), np.round(ref[:, j], 4), np.ptp(ref[:, j]))
        assert ref[:, j].mean() >= floors[j], msg
        assert abs(got[:, j].mean() - ref[:, j].mean()) <= bar, msg


def test_hogwild_auc_matches_oracle(g, c1, s1):
    """FP32 lock-free embed over the full hierarchy against the sequential FP64
    oracle: R-MAT training-edge AUC and planted-partition held-out and
    training-edge AUC within 0.005 (means over 3 seeds), where the oracle
    learns."""
    check_quality(gpu_quality(g, c1, s1, 32), oracle_quality(c1, s1, 32))


@pytest.mark.parametrize("d,floor", [(16, 0.85), (8, 0.75)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_small_d_embed_auc_matches_oracle(g, c1, s1, dtype, d, floor):
    """Small d (Sec. 3.1.1): at d = 16 a warp updates 8 (FP32) or 16 (16-bit)
    sources at once, at d = 8 16 or 32; the small levels fall back from the
    staged kernel to registers.  The same 0.005 bars as d = 32; the oracle's
    R-MAT training-edge AUC is lower at these widths (0.889 at d = 16, 0.789
    at d = 8, over the three seeds), so its floor is 0.85 / 0.75."""
    check_quality(gpu_quality(g, c1, s1, d, dtype), oracle_quality(c1, s1, d), floors=(floor, 0.8, 0.9))


def test_bf16_tables_reach_fp32_auc(g, c1, s1):
    """BF16 tables (FP32 arithmetic, stochastic rounding) reach the FP32
    tables' AUCs within 0.005 (means over 3 seeds), and the oracle's."""
    f32 = gpu_quality(g, c1, s1, 32, torch.float32)
    b16 = gpu_quality(g, c1, s1, 32, torch.bfloat16)
    assert (b16.mean(0) >= f32.mean(0) - 0.005).all(), (b16, f32)
    check_quality(b16, oracle_quality(c1, s1, 32))


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_16bit_tables_error_vs_oracle(g, c1, dtype):
    """Deterministic mode with 16-bit tables against the FP64 oracle: the
    error is that of storage rounding (BF16: 8-bit significand, about 2^-9
    relative per rounding; FP16: 2^-12), not of the arithmetic."""
    gr = c1.train
    M0 = bf16_round_np(oracle.init_uniform(gr.n, 64, 0, 5).astype(np.float32)) * 32  # exact in both formats
    Mo = M0.copy()
    oracle.train_deterministic(gr.rowptr, gr.col, Mo, 3, 0, 4, 0.045, 1e-4, 9, 256)
    Mg = train_gpu(g, gr, M0, 3, 0, 4, 0.045, 9, "deterministic", m=256, dtype=dtype)[0]
    err = rel_fro(Mg, Mo)
    bound = 2e-2 if dtype == torch.bfloat16 else 3e-3
    assert err <= bound, err


def test_embed_deterministic_matches_oracle(g, c1):
    sp = c1
    m = 128
    Mo, info = oracle.embed(sp.train.rowptr, sp.train.col, 64, 3, 0.045, 60, 0.3, seed=11,
                            mode="deterministic", det_batch=m)
    p = g.default_params(d=64, k=3, lr=0.045, epochs=60, p=0.3, seed=11, mode="deterministic", det_batch=m)
    Mg, st = g.gosh_embed(dev(sp.train.rowptr), dev(sp.train.col), p)
    s = g.stats_dict(st)
    assert s["levels"] == info["levels"] and s["epochs"] == info["epochs"]
    assert s["updates"] == info["updates"]
    assert rel_fro(Mg.double().cpu().numpy(), Mo) <= DET_TOL


def test_embed_host_buffers_equal_device_buffers(g, c1):
    sp = c1
    p = g.default_params(d=32, k=3, lr=0.045, epochs=30, p=0.3, seed=3, mode="deterministic", det_batch=256)
    Md, _ = g.gosh_embed(dev(sp.train.rowptr), dev(sp.train.col), p)
    Mh, _ = g.gosh_embed(sp.train.rowptr, sp.train.col, p)
    assert not Mh.is_cuda
    np.testing.assert_array_equal(Md.cpu().numpy(), Mh.numpy())


# ----------------------------------------------------------------- AUC
def test_auc_matches_oracle(g, c1):
    sp = c1
    rng = np.random.default_rng(5)
    M = rng.normal(size=(sp.train.n, 32)).astype(np.float32)
    Md = dev(M)
    pos, neg = dev(sp.test_pos), dev(sp.test_neg)
    sc_pos = g.gosh_pair_scores(Md, pos).cpu().numpy().astype(np.float64)
    sc_neg = g.gosh_pair_scores(Md, neg).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(sc_pos, oracle.pair_scores(M, sp.test_pos), rtol=1e-5, atol=1e-5)
    a = g.gosh_link_auc(Md, pos, neg)
    # same float32 scores on both sides: the AUC must agree to rounding
    assert abs(a - oracle.auc(sc_pos, sc_neg)) < 1e-12
    # ties: all-equal scores give exactly 1/2
    z = torch.zeros((sp.train.n, 32), device="cuda")
    assert g.gosh_link_auc(z, pos, neg) == 0.5


# ----------------------------------------------------------------- errors
def test_invalid_arguments_rejected_before_launch(g, c1):
    gr = c1.train
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = torch.zeros((gr.n, 48), device="cuda")
    p = g.default_params(d=48)
    with pytest.raises(g.GoshError) as e:
        g.gosh_train_level(csr, M, 0, 1, p)
    assert e.value.status == 1
    # unsorted row / self loop / asymmetric CSR caught by validation
    bad_col = gr.col.copy()
    r0, r1 = gr.rowptr[5], gr.rowptr[6]
    assert r1 - r0 >= 2
    bad_col[r0], bad_col[r0 + 1] = bad_col[r0 + 1], bad_col[r0]
    with pytest.raises(g.GoshError, match="ascending"):
        g.gosh_validate_csr(g.to_device_csr(gr.rowptr, bad_col))
    asym = synth.Graph(np.array([0, 1, 1], dtype=np.int64), np.array([1], dtype=np.int32))
    with pytest.raises(g.GoshError, match="symmetric"):
        g.gosh_validate_csr(g.to_device_csr(asym.rowptr, asym.col))
    g.gosh_validate_csr(csr)
    # deterministic mode needs all samples in one pass
    p = g.default_params(d=32, k=9, mode="deterministic")
    with pytest.raises(g.GoshError):
        g.gosh_train_level(csr, torch.zeros((gr.n, 32), device="cuda"), 0, 1, p)
