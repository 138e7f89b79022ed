"""The caller's device allocator (gosh_set_allocator): with PyTorch's caching
allocator installed, every working buffer of an end-to-end embed and of an
out-of-core LargeGraphGPU call comes from it and goes back to it (each block
with the size it was lent with), and the results are bit-identical to those
with the library's own stream-ordered pool; an allocator that refuses makes
the call fail with GOSH_ERR_OOM and leaves the library usable."""
import numpy as np
import pytest

import synth
from gpu_common import gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


class Counting:
    def __init__(self, refuse=False):
        self.live, self.allocs, self.frees, self.refuse = {}, 0, 0, refuse
        self.dev = torch.cuda.current_device()

    def alloc(self, n, stream):
        self.allocs += 1
        if self.refuse:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(n, self.dev, stream)
        self.live[ptr] = n
        return ptr

    def free(self, ptr, n, stream):
        assert self.live.pop(ptr) == n
        self.frees += 1
        torch.cuda.caching_allocator_delete(ptr)


def test_torch_allocator_serves_every_buffer():
    g = gosh()
    gr = synth.workload("rmat12").train
    rp, co = torch.from_numpy(gr.rowptr).cuda(), torch.from_numpy(gr.col).cuda()
    p = g.default_params(d=32, k=3, lr=0.045, epochs=30, p=0.3, seed=3, mode="deterministic", det_batch=256)
    # LargeGraphGPU is reproducible where its order is (kernels in stream order,
    # every part pair within one tile, one source at a time: FP32, d = 128)
    small = synth.random_graph(30, 0.25, 3)
    q = g.default_params(d=128, k=3, lr=0.05, seed=4, B=2, large_parts=2, p_gpu=2, s_gpu=1, large_serial=1)
    M0 = (np.random.default_rng(1).uniform(-0.3, 0.3, (small.n, 128))).astype(np.float32)
    ref, _ = g.gosh_embed(rp, co, p)
    Lref = M0.copy()
    g.gosh_train_level_large(small.rowptr, small.col, Lref, 0, 6, q)
    a = Counting()
    g.gosh_set_allocator(a.alloc, a.free)
    try:
        got, _ = g.gosh_embed(rp, co, p)
        L = M0.copy()
        g.gosh_train_level_large(small.rowptr, small.col, L, 0, 6, q)
        torch.cuda.synchronize()
    finally:
        g.gosh_set_allocator(None, None)
    assert a.allocs > 10 and a.frees == a.allocs and not a.live, (a.allocs, a.frees, a.live)
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    np.testing.assert_array_equal(L, Lref)


def test_refusing_allocator_fails_cleanly():
    g = gosh()
    gr = synth.workload("rmat12").train
    rp, co = torch.from_numpy(gr.rowptr).cuda(), torch.from_numpy(gr.col).cuda()
    p = g.default_params(d=32, k=3, lr=0.045, epochs=10, p=0.3, seed=3)
    a = Counting(refuse=True)
    g.gosh_set_allocator(a.alloc, a.free)
    try:
        with pytest.raises(g.GoshError) as e:
            g.gosh_embed(rp, co, p)
        assert e.value.status == 2 and a.allocs >= 1
    finally:
        g.gosh_set_allocator(None, None)
    M, _ = g.gosh_embed(rp, co, p)  # the library's own pool again
    assert torch.isfinite(M).all()
