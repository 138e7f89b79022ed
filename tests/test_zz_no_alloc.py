"""gosh_train_level_noalloc, the entry point for callers that cannot allocate
device memory (a framework arena owns it all, or the library must never
call cudaMalloc/cudaFree), against gosh_train_level.

Collected last on purpose (file name): a failure here leaves every other
test already run.  It also passes alone in a fresh process.

The graph has 30 vertices and FP32 d = 128 tables (32 lanes per source), so
one warp processes the sources strictly in id order: both entry points then
compute the same sequence of updates, and the test can hold them to the
deterministic-mode tolerance of the other GPU tests (relative Frobenius error
1e-5; update counts exact) on two calls in a row.
"""
import numpy as np
import pytest

import synth
from gpu_common import gosh, needs_gpu, rel_fro, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = 1e-5


def test_noalloc_matches_train_level_on_two_calls():
    g = gosh()
    gr = synth.random_graph(30, 0.2, 17)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    rng = np.random.default_rng(4)
    M0 = torch.from_numpy(rng.uniform(-0.3, 0.3, (gr.n, 128)).astype(np.float32)).cuda()
    p = g.default_params(d=128, k=5, lr=0.05, seed=8, lanes_per_row=32, vertices_per_warp=32)
    Ma, Mb = M0.clone(), M0.clone()
    for call in range(2):
        epochs = 7 + call
        la = torch.zeros(epochs, dtype=torch.float64, device="cuda")
        lb = torch.zeros(epochs, dtype=torch.float64, device="cuda")
        na = torch.zeros(1, dtype=torch.int64, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        g.gosh_train_level(csr, Ma, call, epochs, p, loss=la, n_updates=na)
        g.gosh_train_level_noalloc(csr, Mb, call, epochs, p, loss=lb, n_updates=nb)
        torch.cuda.synchronize()
        assert int(na.item()) == int(nb.item()) > 0
        assert rel_fro(Mb.double().cpu().numpy(), Ma.double().cpu().numpy()) <= TOL
        np.testing.assert_allclose(lb.cpu().numpy(), la.cpu().numpy(), rtol=TOL)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_noalloc_default_kernels_match_train_level(dtype):
    """Automatic lanes and samples per pass on a level under 2^14 rows pick
    the staged (TMA) kernels for both table types; with every source in one
    warp's tile the warp's order is fixed, so both entry points give the
    same tables, update counts and losses.  The second call passes no loss
    buffer (the partial sums are then not written at all)."""
    g = gosh()
    gr = synth.random_graph(30, 0.2, 19)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    rng = np.random.default_rng(6)
    M0 = torch.from_numpy(rng.uniform(-0.3, 0.3, (gr.n, 128)).astype(np.float32)).to(dtype).cuda()
    p = g.default_params(d=128, k=3, lr=0.05, seed=12, dtype=dtype, vertices_per_warp=32)
    Ma, Mb = M0.clone(), M0.clone()
    for call in range(2):
        epochs = 5 + call
        la = torch.zeros(epochs, dtype=torch.float64, device="cuda") if call == 0 else None
        lb = torch.zeros(epochs, dtype=torch.float64, device="cuda") if call == 0 else None
        na = torch.zeros(1, dtype=torch.int64, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        g.gosh_train_level(csr, Ma, call, epochs, p, loss=la, n_updates=na)
        g.gosh_train_level_noalloc(csr, Mb, call, epochs, p, loss=lb, n_updates=nb)
        torch.cuda.synchronize()
        assert int(na.item()) == int(nb.item()) > 0
        assert rel_fro(Mb.double().cpu().numpy(), Ma.double().cpu().numpy()) <= TOL
        if la is not None:
            np.testing.assert_allclose(lb.cpu().numpy(), la.cpu().numpy(), rtol=TOL)
    g.gosh_device_check()


def test_noalloc_rejects_deterministic_mode():
    g = gosh()
    gr = synth.random_graph(30, 0.2, 17)
    csr = g.to_device_csr(gr.rowptr, gr.col)
    M = torch.zeros((gr.n, 32), device="cuda")
    p = g.default_params(d=32, mode="deterministic")
    with pytest.raises(g.GoshError) as e:
        g.gosh_train_level_noalloc(csr, M, 0, 1, p)
    assert e.value.status == 6
