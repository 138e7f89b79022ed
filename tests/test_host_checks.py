"""Host-side argument checks of the entry points that take a HOST CSR, run on
the CPU (each call returns before any device work): gosh_walk_pairs always
checks the CSR's content, gosh_train_level_large and gosh_train_level_walks
when params.validate is set; every kind of bad CSR is rejected with
GOSH_ERR_INVALID_ARG and a message naming the fault."""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_2110_10049_gb300 import build, gosh as g


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


def bad_csrs():
    gr = synth.random_graph(12, 0.4, 3)
    rp, col = gr.rowptr.copy(), gr.col.copy()
    v = int(np.argmax(np.diff(rp)))  # a row with at least two entries
    assert rp[v + 1] - rp[v] >= 2
    out = []
    r = rp.copy(); r[0] = 1; out.append(("rowptr[0]", r, col))
    r = rp.copy(); r[v + 1] = r[v] - 1; out.append(("decreases", r, col))
    c = col.copy(); c[rp[v]] = 12; out.append(("out of range", rp, c))
    c = col.copy(); c[rp[v]] = -3; out.append(("out of range", rp, c))
    c = col.copy(); c[rp[v]] = v; c[rp[v]:rp[v + 1]].sort(); out.append(("self-loop", rp, c))
    c = col.copy(); c[rp[v]], c[rp[v] + 1] = c[rp[v] + 1], c[rp[v]]; out.append(("ascending", rp, c))
    c = col.copy(); c[rp[v] + 1] = c[rp[v]]; out.append(("ascending", rp, c))
    return gr, out


def test_walk_pairs_rejects_bad_csrs():
    gr, cases = bad_csrs()
    g.gosh_walk_pairs(gr.rowptr, gr.col, 4, 2, 0, 0, 1)  # the good graph passes
    for what, rp, col in cases:
        with pytest.raises(g.GoshError) as e:
            g.gosh_walk_pairs(rp, col, 4, 2, 0, 0, 1)
        assert e.value.status == 1 and what in str(e.value), (what, str(e.value))


def _csr(rp, col):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return g.gosh_csr(len(rp) - 1, rp.ctypes.data, col.ctypes.data, 0), (rp, col)


@pytest.mark.parametrize("entry", ["large", "walks"])
def test_validate_rejects_bad_host_csrs_before_device_work(entry):
    gr, cases = bad_csrs()
    L = g.lib()
    M = np.zeros((gr.n, 32), dtype=np.float32)
    p = g.default_params(d=32, k=3, validate=1, large_parts=2, p_gpu=2, s_gpu=1, B=1)
    for what, rp, col in cases:
        cg, keep = _csr(rp, col)
        if entry == "large":
            st = g.gosh_large_stats()
            rc = L.gosh_train_level_large(C.byref(cg), C.c_void_p(M.ctypes.data), 0, 3, C.byref(p), None,
                                          C.byref(st))
        else:
            st = g.gosh_walk_stats()
            rc = L.gosh_train_level_walks(C.byref(cg), C.c_void_p(M.ctypes.data), 0, 3, C.byref(p), None, None,
                                          C.byref(st))
        assert rc == 1, (what, rc)
        assert what in L.gosh_last_error().decode(), (what, L.gosh_last_error())


def test_release_host_buffers_without_any_held():
    # nothing pinned in this process: nothing to free, no device involved
    assert g.gosh_release_host_buffers() == 0
    assert g.gosh_release_host_buffers() == 0


@pytest.mark.parametrize("entry", ["large", "walks"])
@pytest.mark.parametrize("bad", [dict(lr=0.0), dict(lr=float("nan")), dict(d=48), dict(k=-1), dict(lr_floor=2.0),
                                 dict(dtype=7)])
def test_bad_params_rejected_before_device_work(entry, bad):
    gr = synth.random_graph(12, 0.4, 3)
    L = g.lib()
    M = np.zeros((gr.n, 32), dtype=np.float32)
    p = g.default_params(d=32, k=3, large_parts=2, p_gpu=2, s_gpu=1, B=1)
    for key, val in bad.items():
        setattr(p, key, val)
    cg, keep = _csr(gr.rowptr, gr.col)
    if entry == "large":
        rc = L.gosh_train_level_large(C.byref(cg), C.c_void_p(M.ctypes.data), 0, 3, C.byref(p), None,
                                      C.byref(g.gosh_large_stats()))
    else:
        rc = L.gosh_train_level_walks(C.byref(cg), C.c_void_p(M.ctypes.data), 0, 3, C.byref(p), None, None,
                                      C.byref(g.gosh_walk_stats()))
    assert rc == 1, (bad, rc, L.gosh_last_error())


@pytest.mark.parametrize("bad", [dict(epoch_overlap=9), dict(epoch_overlap=-1), dict(overlap_min_vertices=-5)])
def test_epoch_overlap_limits_checked_first(bad):
    # the parameter check precedes any device work, so placeholder device
    # pointers are never touched
    L = g.lib()
    p = g.default_params(d=32)
    assert p.epoch_overlap == 1 and p.overlap_min_vertices == 65536
    for key, val in bad.items():
        setattr(p, key, val)
    cg = g.gosh_csr(10, 256, 512, 1)
    rc = L.gosh_train_level(C.byref(cg), C.c_void_p(1024), 0, 3, C.byref(p), None, None, None)
    assert rc == 1 and "overlap" in L.gosh_last_error().decode()


@pytest.mark.parametrize("bad", [dict(cooperative_epochs=2), dict(cooperative_epochs=-1), dict(epoch_unit=2)])
def test_launch_and_unit_flags_checked_first(bad):
    # both flags take 0 or 1; checked before any device work (placeholder
    # device pointers are never touched); the defaults are 0
    L = g.lib()
    p = g.default_params(d=32)
    assert p.cooperative_epochs == 0 and p.epoch_unit == 0
    for key, val in bad.items():
        setattr(p, key, val)
    cg = g.gosh_csr(10, 256, 512, 1)
    rc = L.gosh_train_level(C.byref(cg), C.c_void_p(1024), 0, 3, C.byref(p), None, None, None)
    name = next(iter(bad))
    assert rc == 1 and name in L.gosh_last_error().decode()


def test_allocator_needs_both_functions():
    """gosh_set_allocator takes both callbacks or neither (no device use)."""
    L = g.lib()
    noop_alloc = g.ALLOC_FN(lambda n, s, c: None)
    with pytest.raises(g.GoshError) as e:
        g._check("gosh_set_allocator", L.gosh_set_allocator(C.cast(noop_alloc, C.c_void_p), None, None))
    assert e.value.status == 1
    g.gosh_set_allocator(None, None)
