"""Thin ctypes binding of libgosh (include/gosh.h).

Argument marshalling only: every function forwards torch tensors' device
pointers and the current CUDA stream to the C entry point of the same name and
raises GoshError on a non-zero status.  There is no fallback: if libgosh.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgosh.so")

GOSH_F32, GOSH_BF16, GOSH_F16 = 0, 1, 2
GOSH_HOGWILD, GOSH_DETERMINISTIC = 0, 1
MAX_LEVELS = 64

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "BUDGET", 4: "CUDA", 5: "TIMEOUT", 6: "UNSUPPORTED"}


class GoshError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__("%s -> GOSH_ERR_%s: %s" % (fn, _STATUS.get(status, status), msg))
        self.status = status


class gosh_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("on_device", C.c_int)]


class gosh_params(C.Structure):
    _fields_ = [("d", C.c_int), ("k", C.c_int), ("lr", C.c_double), ("lr_floor", C.c_double),
                ("epochs", C.c_int), ("p", C.c_double), ("threshold", C.c_int), ("shrink", C.c_double),
                ("max_levels", C.c_int), ("dtype", C.c_int), ("mode", C.c_int), ("det_batch", C.c_int64),
                ("seed", C.c_uint64), ("graph_id", C.c_uint64), ("lanes_per_row", C.c_int),
                ("samples_per_pass", C.c_int), ("device_budget_bytes", C.c_int64), ("validate", C.c_int),
                ("plain_stores", C.c_int), ("projection", C.c_int), ("mlp_hidden", C.c_int),
                ("mlp_epochs", C.c_int), ("mlp_lr", C.c_double), ("mlp_batch", C.c_int),
                ("mlp_max_rows", C.c_int64), ("p_gpu", C.c_int), ("s_gpu", C.c_int), ("B", C.c_int), ("large_parts", C.c_int),
                ("persistent_small_levels", C.c_int), ("vertices_per_warp", C.c_int),
                ("walk_length", C.c_int), ("walk_window", C.c_int), ("large_serial", C.c_int),
                ("large_evict", C.c_int), ("overlap_min_vertices", C.c_int64), ("epoch_overlap", C.c_int),
                ("large_pools", C.c_int), ("epoch_unit", C.c_int),
                ("cooperative_epochs", C.c_int)]


class gosh_walk_stats(C.Structure):
    _fields_ = [("positions", C.c_int64), ("epochs", C.c_int), ("host_ms", C.c_double), ("total_ms", C.c_double),
                ("h2d_bytes", C.c_int64)]


class gosh_large_stats(C.Structure):
    _fields_ = [("parts", C.c_int), ("rounds", C.c_int), ("kernels", C.c_int64), ("swaps", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("positives", C.c_ulonglong),
                ("updates", C.c_ulonglong), ("device_bytes", C.c_int64), ("total_ms", C.c_double),
                ("setup_ms", C.c_double)]


class gosh_stats(C.Structure):
    _fields_ = [("levels", C.c_int), ("n", C.c_int64 * MAX_LEVELS), ("nnz", C.c_int64 * MAX_LEVELS),
                ("epochs", C.c_int * MAX_LEVELS), ("train_ms", C.c_double * MAX_LEVELS),
                ("coarsen_ms", C.c_double), ("project_ms", C.c_double), ("total_ms", C.c_double),
                ("updates", C.c_ulonglong)]


class gosh_batch_stats(C.Structure):
    _fields_ = [("graphs", C.c_int), ("phases", C.c_int64), ("level0_vertices", C.c_int64),
                ("lanes_per_row", C.c_int), ("samples_per_pass", C.c_int), ("sources_per_item", C.c_int),
                ("autotuned", C.c_int), ("coarsen_ms", C.c_double), ("train_ms", C.c_double),
                ("total_ms", C.c_double), ("updates", C.c_ulonglong)]


_lib = None


def lib() -> C.CDLL:
    """Loads libgosh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgosh.so is not built: run __graft_entry__.build() "
                               "(or python -m paper_2110_10049_gb300.build)")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, u64, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_uint64, C.c_double
        P = C.POINTER
        sig = {
            "gosh_params_default": [P(gosh_params)],
            "gosh_validate_csr": [P(gosh_csr), vp],
            "gosh_coarsen": [P(gosh_csr), i32, f64, i32, vp, P(vp)],
            "gosh_coarsen_batch": [vp, i32, i32, f64, i32, vp, vp],
            "gosh_hierarchy_level": [vp, i32, P(gosh_csr), P(vp)],
            "gosh_hierarchy_sizes": [vp, i32, P(C.c_int64), P(C.c_int64)],
            "gosh_hierarchy_copy_level": [vp, i32, vp, vp, vp, vp],
            "gosh_init_embedding": [vp, i64, i32, i32, i32, u64, u64, vp],
            "gosh_train_level": [P(gosh_csr), vp, i32, i32, P(gosh_params), vp, vp, vp],
            "gosh_train_level_noalloc": [P(gosh_csr), vp, i32, i32, P(gosh_params), vp, vp, vp],
            "gosh_project": [vp, i64, vp, vp, i64, i32, i32, vp],
            "gosh_embed": [P(gosh_csr), P(gosh_params), vp, vp, P(gosh_stats)],
            "gosh_pair_scores": [vp, i32, i32, vp, i64, vp, vp],
            "gosh_link_auc": [vp, i32, i32, vp, i64, vp, i64, vp, P(C.c_double)],
            "gosh_tc_gemm_bf16": [vp, i64, vp, i64, vp, i64, i32, i32, i32, i32, vp],
            "gosh_embed_batch": [i32, vp, P(gosh_params), vp, vp, P(gosh_batch_stats)],
            "gosh_device_check": [vp],
            "gosh_train_level_large": [P(gosh_csr), vp, i32, i32, P(gosh_params), vp, P(gosh_large_stats)],
            "gosh_train_level_walks": [P(gosh_csr), vp, i32, i32, P(gosh_params), vp, vp, P(gosh_walk_stats)],
            "gosh_walk_pairs": [P(gosh_csr), i32, i32, i32, i32, u64, u64, vp],
            "gosh_walk_order": [i64, i32, i32, u64, u64, vp],
            "gosh_large_plan": [i64, i32, i32, i32, i32, vp, vp, i32],
            "gosh_large_block": [P(gosh_csr), i32, i32, i32, vp, vp, vp, vp, vp, vp],
            "gosh_mlp_create": [i32, i32, u64, P(vp)],
            "gosh_mlp_get_weights": [vp, vp, vp, vp, vp],
            "gosh_mlp_set_weights": [vp, vp, vp, vp, vp],
            "gosh_mlp_features": [P(gosh_csr), vp, vp, i32, i32, vp, vp],
            "gosh_mlp_grads": [vp, vp, vp, i64, vp, vp, vp, vp, P(C.c_double), vp],
            "gosh_mlp_train": [vp, P(gosh_csr), vp, vp, vp, i32, i32, i32, f64, i32, i64, vp, P(C.c_double)],
            "gosh_project_learned": [vp, vp, vp, P(gosh_csr), vp, i32, i32, vp],
            "gosh_round_stochastic": [vp, vp, i64, i32, u64, vp],
            "gosh_level_epochs": [i32, f64, i32, i32, vp, vp, vp],
            "gosh_large_pool": [P(gosh_csr), i32, i32, i32, i32, i32, i32, u64, u64, vp],
        }
        L.gosh_mlp_free.restype = None
        L.gosh_mlp_free.argtypes = [vp]
        L.gosh_mlp_feature_stride.restype = C.c_int
        L.gosh_mlp_feature_stride.argtypes = [C.c_int]
        L.gosh_kernel_launches.restype = C.c_ulonglong
        L.gosh_kernel_launches.argtypes = []
        L.gosh_release_host_buffers.restype = C.c_ulonglong
        L.gosh_release_host_buffers.argtypes = []
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.gosh_last_error.restype = C.c_char_p
        L.gosh_last_error.argtypes = []
        L.gosh_hierarchy_levels.restype = C.c_int
        L.gosh_hierarchy_levels.argtypes = [vp]
        L.gosh_hierarchy_free.restype = None
        L.gosh_hierarchy_free.argtypes = [vp]
        L.gosh_set_allocator.restype = C.c_int
        L.gosh_set_allocator.argtypes = [vp, vp, vp]
        _lib = L
    return _lib


def _check(fn: str, status: int):
    if status != 0:
        raise GoshError(fn, status, lib().gosh_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


_DT = {"f32": GOSH_F32, "bf16": GOSH_BF16, "f16": GOSH_F16}


def dtype_code(t) -> int:
    import torch
    if isinstance(t, int):
        return t
    if isinstance(t, str):
        return _DT[t]
    return {torch.float32: GOSH_F32, torch.bfloat16: GOSH_BF16, torch.float16: GOSH_F16}[t]


def torch_dtype(code: int):
    import torch
    return {GOSH_F32: torch.float32, GOSH_BF16: torch.bfloat16, GOSH_F16: torch.float16}[code]


def default_params(**kw) -> gosh_params:
    p = gosh_params()
    _check("gosh_params_default", lib().gosh_params_default(C.byref(p)))
    for k, v in kw.items():
        if k == "dtype":
            v = dtype_code(v)
        if k == "mode" and isinstance(v, str):
            v = {"hogwild": GOSH_HOGWILD, "deterministic": GOSH_DETERMINISTIC}[v]
        setattr(p, k, v)
    return p


@dataclass
class Csr:
    """Device CSR kept alive alongside its ctypes view."""
    rowptr: object  # torch.int64 [n+1]
    col: object     # torch.int32 [nnz]

    @property
    def n(self) -> int:
        return self.rowptr.numel() - 1

    def c(self) -> gosh_csr:
        return gosh_csr(self.n, self.rowptr.data_ptr(), self.col.data_ptr(), 1)


def to_device_csr(rowptr, col, device="cuda") -> Csr:
    import torch
    rp = torch.as_tensor(np.ascontiguousarray(rowptr, dtype=np.int64)).to(device)
    co = torch.as_tensor(np.ascontiguousarray(col, dtype=np.int32))
    if co.numel() == 0:
        co = torch.zeros(1, dtype=torch.int32)
    return Csr(rp, co.to(device))


def gosh_validate_csr(g: Csr, stream=None):
    cg = g.c()
    _check("gosh_validate_csr", lib().gosh_validate_csr(C.byref(cg), _stream(stream)))


class Hierarchy:
    """Owns a gosh_hierarchy handle (level 0 aliases the input CSR)."""

    def __init__(self, handle, g0: Csr):
        self.handle = handle
        self._g0 = g0

    def __len__(self):
        return lib().gosh_hierarchy_levels(self.handle)

    def level(self, i: int):
        """(n, rowptr ptr, col ptr, map ptr or None) of level i (device pointers)."""
        cg = gosh_csr()
        mp = C.c_void_p()
        _check("gosh_hierarchy_level", lib().gosh_hierarchy_level(self.handle, i, C.byref(cg), C.byref(mp)))
        return cg, mp.value

    def sizes(self, i: int):
        n, nnz = C.c_int64(), C.c_int64()
        _check("gosh_hierarchy_sizes", lib().gosh_hierarchy_sizes(self.handle, i, C.byref(n), C.byref(nnz)))
        return n.value, nnz.value

    def level_arrays(self, i: int, stream=None):
        """Copies level i's CSR and map (None for the last level) to host numpy arrays."""
        n, nnz = self.sizes(i)
        rp = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        m = np.zeros(max(n, 1), dtype=np.int32)
        last = i == len(self) - 1
        _check("gosh_hierarchy_copy_level", lib().gosh_hierarchy_copy_level(
            self.handle, i, rp.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
            None if last else m.ctypes.data_as(C.c_void_p), _stream(stream)))
        return rp, col[:nnz], (None if last else m[:n])

    def close(self):
        if self.handle:
            lib().gosh_hierarchy_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gosh_coarsen(g: Csr, threshold=100, shrink=0.8, max_levels=MAX_LEVELS, stream=None) -> Hierarchy:
    cg = g.c()
    h = C.c_void_p()
    _check("gosh_coarsen", lib().gosh_coarsen(C.byref(cg), threshold, shrink, max_levels, _stream(stream),
                                              C.byref(h)))
    return Hierarchy(h.value, g)


def gosh_coarsen_batch(graphs, threshold=100, shrink=0.8, max_levels=MAX_LEVELS, stream=None):
    """Coarsens a list of device CSRs (Csr) together; one Hierarchy per graph."""
    G = len(graphs)
    arr = (gosh_csr * G)(*[g.c() for g in graphs])
    hs = (C.c_void_p * G)()
    _check("gosh_coarsen_batch", lib().gosh_coarsen_batch(C.cast(arr, C.c_void_p), G, threshold, shrink, max_levels,
                                                          _stream(stream), C.cast(hs, C.c_void_p)))
    return [Hierarchy(hs[i], graphs[i]) for i in range(G)]


def gosh_init_embedding(M, level=0, seed=0, graph_id=0, stream=None):
    n, d = M.shape
    _check("gosh_init_embedding", lib().gosh_init_embedding(_ptr(M), n, d, dtype_code(M.dtype), level, seed,
                                                            graph_id, _stream(stream)))


def gosh_train_level(g, M, level, epochs, params: gosh_params, loss=None, n_updates=None, stream=None):
    """g: Csr or gosh_csr (device).  loss: torch.float64[epochs] (device) or None.
    n_updates: torch.int64[1] (device) or None (incremented)."""
    cg = g.c() if isinstance(g, Csr) else g
    _check("gosh_train_level", lib().gosh_train_level(C.byref(cg), _ptr(M), level, epochs, C.byref(params),
                                                      _stream(stream), _ptr(loss), _ptr(n_updates)))


def gosh_train_level_noalloc(g, M, level, epochs, params: gosh_params, loss=None, n_updates=None, stream=None):
    """gosh_train_level without any device allocation by the library (lock-free
    mode only; see include/gosh.h for the limits)."""
    cg = g.c() if isinstance(g, Csr) else g
    _check("gosh_train_level_noalloc", lib().gosh_train_level_noalloc(
        C.byref(cg), _ptr(M), level, epochs, C.byref(params), _stream(stream), _ptr(loss), _ptr(n_updates)))


def gosh_device_check(stream=None):
    """Synchronises the stream and raises GoshError (GOSH_ERR_TIMEOUT) if a
    bounded device-side wait gave up since the last check."""
    _check("gosh_device_check", lib().gosh_device_check(_stream(stream)))


def gosh_round_stochastic(x, dtype, seed=0, stream=None):
    """x: torch.float32 device tensor; dtype: torch.bfloat16 / torch.float16 or
    a GOSH_* code.  Returns the stochastically rounded tensor."""
    import torch
    code = dtype if isinstance(dtype, int) else dtype_code(dtype)
    out = torch.empty(x.shape, dtype=torch_dtype(code), device=x.device)
    _check("gosh_round_stochastic", lib().gosh_round_stochastic(_ptr(x), _ptr(out), x.numel(), code, seed,
                                                                _stream(stream)))
    return out


def gosh_project(Mc, map_ptr, Mf, stream=None):
    """map_ptr: a torch.int32 tensor or a raw device pointer."""
    mp = C.c_void_p(map_ptr.data_ptr()) if hasattr(map_ptr, "data_ptr") else C.c_void_p(map_ptr)
    _check("gosh_project", lib().gosh_project(_ptr(Mc), Mc.shape[0], mp, _ptr(Mf), Mf.shape[0], Mc.shape[1],
                                              dtype_code(Mc.dtype), _stream(stream)))


def gosh_embed(rowptr, col, params: gosh_params, out=None, stream=None):
    """Alg. 2 end to end.  rowptr/col: torch device tensors (device path) or
    numpy arrays (host path; out must then be a host tensor or None).
    Returns (M0, stats)."""
    import torch
    on_dev = hasattr(rowptr, "is_cuda") and rowptr.is_cuda
    if on_dev:
        cg = gosh_csr(rowptr.numel() - 1, rowptr.data_ptr(), col.data_ptr(), 1)
        n = rowptr.numel() - 1
    else:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        cg = gosh_csr(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, 0)
        n = len(rowptr) - 1
    if out is None:
        out = torch.empty((n, params.d), dtype=torch_dtype(params.dtype),
                          device="cuda" if on_dev else "cpu")
    st = gosh_stats()
    _check("gosh_embed", lib().gosh_embed(C.byref(cg), C.byref(params), _ptr(out), _stream(stream),
                                          C.byref(st)))
    return out, st


def gosh_embed_batch(graphs, params: gosh_params, outs=None, stream=None):
    """Embeds a list of device CSRs (Csr) in one persistent launch.
    Returns (list of M tensors, stats dict)."""
    import torch
    G = len(graphs)
    arr = (gosh_csr * G)(*[g.c() for g in graphs])
    if outs is None:
        outs = [torch.empty((g.n, params.d), dtype=torch_dtype(params.dtype), device="cuda") for g in graphs]
    ptrs = (C.c_void_p * G)(*[o.data_ptr() for o in outs])
    st = gosh_batch_stats()
    _check("gosh_embed_batch", lib().gosh_embed_batch(G, C.cast(arr, C.c_void_p), C.byref(params),
                                                      C.cast(ptrs, C.c_void_p), _stream(stream), C.byref(st)))
    stats = {f: getattr(st, f) for f, _ in gosh_batch_stats._fields_}
    return outs, stats


def gosh_train_level_large(rowptr, col, M, level, epochs, params: gosh_params, stream=None):
    """LargeGraphGPU on a host CSR (numpy) and host M (numpy or CPU tensor,
    updated in place).  Returns the stats dict."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    cg = gosh_csr(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, 0)
    ptr = M.ctypes.data if isinstance(M, np.ndarray) else M.data_ptr()
    st = gosh_large_stats()
    _check("gosh_train_level_large", lib().gosh_train_level_large(C.byref(cg), C.c_void_p(ptr), level, epochs,
                                                                  C.byref(params), _stream(stream), C.byref(st)))
    return {f: getattr(st, f) for f, _ in gosh_large_stats._fields_}


def gosh_train_level_walks(rowptr, col, M, level, epochs, params: gosh_params, n_updates=None, stream=None):
    """Random-walk positives (Sec. 3.2) on a host CSR (numpy) and a device M
    (torch, updated in place).  Returns the stats dict."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    cg = gosh_csr(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, 0)
    st = gosh_walk_stats()
    _check("gosh_train_level_walks", lib().gosh_train_level_walks(C.byref(cg), _ptr(M), level, epochs,
                                                                  C.byref(params), _stream(stream),
                                                                  _ptr(n_updates), C.byref(st)))
    return {f: getattr(st, f) for f, _ in gosh_walk_stats._fields_}


def gosh_large_block(rowptr, col, K, a, b):
    """The LargeGraphGPU edge block of part pair (a, b) as the library builds
    it (host only): (rp_ab, col_ab, rp_ba, col_ba), the ba side None when
    a == b."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    n = len(rowptr) - 1
    cg = gosh_csr(n, rowptr.ctypes.data, col.ctypes.data, 0)
    m_ab, m_ba = C.c_int64(0), C.c_int64(0)
    _check("gosh_large_block", lib().gosh_large_block(C.byref(cg), K, a, b, C.byref(m_ab), C.byref(m_ba),
                                                      None, None, None, None))
    na = n * (a + 1) // K - n * a // K
    nb = n * (b + 1) // K - n * b // K
    rp_ab = np.zeros(na + 1, np.int64)
    col_ab = np.zeros(max(m_ab.value, 1), np.int32)
    rp_ba = np.zeros(nb + 1, np.int64)
    col_ba = np.zeros(max(m_ba.value, 1), np.int32)
    _check("gosh_large_block", lib().gosh_large_block(C.byref(cg), K, a, b, C.byref(m_ab), C.byref(m_ba),
                                                      rp_ab.ctypes.data, col_ab.ctypes.data, rp_ba.ctypes.data,
                                                      col_ba.ctypes.data))
    if a == b:
        return rp_ab, col_ab[:m_ab.value], None, None
    return rp_ab, col_ab[:m_ab.value], rp_ba, col_ba[:m_ba.value]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_allocator_refs = None  # keeps the installed callbacks alive


def gosh_set_allocator(alloc=None, free=None):
    """Installs Python callables as the library's device allocator:
    alloc(bytes, stream) -> int device pointer (0 on failure) and
    free(ptr, bytes, stream); both None restores the stream-ordered pool."""
    global _allocator_refs
    if alloc is None and free is None:
        _check("gosh_set_allocator", lib().gosh_set_allocator(None, None, None))
        _allocator_refs = None
        return
    a = ALLOC_FN(lambda nbytes, stream, ctx: alloc(int(nbytes), stream or 0) or None)
    f = FREE_FN(lambda ptr, nbytes, stream, ctx: free(int(ptr), int(nbytes), stream or 0))
    _check("gosh_set_allocator", lib().gosh_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None))
    _allocator_refs = (a, f)


def use_torch_allocator(device=None):
    """Serves the library's device memory from PyTorch's caching allocator
    (the memory then shows in torch.cuda.memory_allocated)."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    gosh_set_allocator(lambda n, stream: torch.cuda.caching_allocator_alloc(n, dev, stream),
                       lambda ptr, n, stream: torch.cuda.caching_allocator_delete(ptr))


def gosh_large_pool(rowptr, col, K, a, b, rnd, B, level, seed, graph_id=0) -> np.ndarray:
    """The host sample pool of pair (a, b) in round rnd (no GPU use): int32
    [sources, B] of local ids in the opposite part, -1 = no neighbour there."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    co = np.ascontiguousarray(col, dtype=np.int32)
    if co.size == 0:
        co = np.zeros(1, dtype=np.int32)
    n = len(rp) - 1
    start = [n * i // K for i in range(K + 1)]
    ns = (start[a + 1] - start[a]) + ((start[b + 1] - start[b]) if a != b else 0)
    out = np.empty((max(ns, 1), B), dtype=np.int32)
    cg = gosh_csr(n, rp.ctypes.data, co.ctypes.data, 0)
    _check("gosh_large_pool", lib().gosh_large_pool(C.byref(cg), K, a, b, rnd, B, level, seed, graph_id,
                                                    out.ctypes.data))
    return out[:ns]


def gosh_release_host_buffers() -> int:
    """Free the pinned host buffers kept across LargeGraphGPU and walk calls
    (those no running call holds); returns the bytes freed."""
    return int(lib().gosh_release_host_buffers())


def gosh_walk_pairs(rowptr, col, walk_length, walk_window, level, epoch, seed, graph_id=0):
    """An epoch's walk pair table (host only): int32 [n * W, 2], -1 for holes."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    n = len(rowptr) - 1
    W = sum(min(walk_window, walk_length - 1 - i) for i in range(walk_length - 1))
    out = np.zeros((n * W, 2), dtype=np.int32)
    cg = gosh_csr(n, rowptr.ctypes.data, col.ctypes.data, 0)
    _check("gosh_walk_pairs", lib().gosh_walk_pairs(C.byref(cg), walk_length, walk_window, level, epoch, seed,
                                                    graph_id, out.ctypes.data))
    return out


def gosh_walk_order(positions, level, epoch, seed, graph_id=0):
    """The order of an epoch's walk positions on the device (host only)."""
    out = np.zeros(positions, dtype=np.int64)
    _check("gosh_walk_order", lib().gosh_walk_order(positions, level, epoch, seed, graph_id, out.ctypes.data))
    return out


def gosh_level_epochs(epochs, p, D, epoch_unit=0, n=None, nnz=None) -> list:
    """Per-level passes of gosh_embed's schedule (host only)."""
    out = np.zeros(max(D, 1), dtype=np.int32)
    nv = None if n is None else np.ascontiguousarray(n, dtype=np.int64)
    ne = None if nnz is None else np.ascontiguousarray(nnz, dtype=np.int64)
    _check("gosh_level_epochs", lib().gosh_level_epochs(
        int(epochs), float(p), int(D), int(epoch_unit), None if nv is None else nv.ctypes.data,
        None if ne is None else ne.ctypes.data, out.ctypes.data))
    return [int(x) for x in out[:D]]


def gosh_large_plan(n, K, p_gpu, rounds, evict=0):
    """Host-only schedule simulation: (pairs [kernels x 2], loads [kernels x 2])."""
    cap = max(rounds * K * (K + 1) // 2, 0)
    pairs = np.zeros((max(cap, 1), 2), dtype=np.int32)
    loads = np.zeros((max(cap, 1), 2), dtype=np.int32)
    cnt = lib().gosh_large_plan(n, K, p_gpu, rounds, evict, pairs.ctypes.data, loads.ctypes.data, cap)
    if cnt == -2:
        raise GoshError("gosh_large_plan", 1, "need K >= 1, 2 <= p_gpu <= 999, rounds >= 0, evict 0 or 1")
    if cnt < 0:
        raise GoshError("gosh_large_plan", 1, "capacity")
    return pairs[:cnt], loads[:cnt]


class Mlp:
    """Owns a gosh_mlp handle (learned projection network)."""

    def __init__(self, d, hidden=256, seed=0):
        h = C.c_void_p()
        _check("gosh_mlp_create", lib().gosh_mlp_create(d, hidden, seed, C.byref(h)))
        self.handle, self.d, self.hidden = h.value, d, hidden

    @property
    def stride(self) -> int:
        return lib().gosh_mlp_feature_stride(self.d)

    def get_weights(self):
        din = 2 * self.d + 1
        W1 = np.zeros((self.hidden, din), np.float32)
        b1 = np.zeros(self.hidden, np.float32)
        W2 = np.zeros((self.d, self.hidden), np.float32)
        b2 = np.zeros(self.d, np.float32)
        _check("gosh_mlp_get_weights", lib().gosh_mlp_get_weights(
            self.handle, W1.ctypes.data, b1.ctypes.data, W2.ctypes.data, b2.ctypes.data))
        return W1, b1, W2, b2

    def set_weights(self, W1, b1, W2, b2):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2)]
        _check("gosh_mlp_set_weights", lib().gosh_mlp_set_weights(self.handle, *[a.ctypes.data for a in arrs]))

    def features(self, g, map_ptr, Mc, stream=None):
        """Device BF16 feature matrix (n_fine x stride) of g's vertices."""
        import torch
        cg = g.c() if isinstance(g, Csr) else g
        X = torch.empty((cg.n, self.stride), dtype=torch.bfloat16, device="cuda")
        mp = map_ptr.data_ptr() if hasattr(map_ptr, "data_ptr") else map_ptr
        _check("gosh_mlp_features", lib().gosh_mlp_features(C.byref(cg), C.c_void_p(mp), _ptr(Mc), self.d,
                                                            dtype_code(Mc.dtype), _ptr(X), _stream(stream)))
        return X

    def grads(self, X, R, stream=None):
        din = 2 * self.d + 1
        out = [np.zeros((self.hidden, din), np.float32), np.zeros(self.hidden, np.float32),
               np.zeros((self.d, self.hidden), np.float32), np.zeros(self.d, np.float32)]
        loss = C.c_double()
        _check("gosh_mlp_grads", lib().gosh_mlp_grads(self.handle, _ptr(X), _ptr(R), X.shape[0],
                                                      *[a.ctypes.data for a in out], C.byref(loss), _stream(stream)))
        return loss.value, out

    def train(self, g, map_ptr, Mc, Mf, epochs=4, lr=1e-3, batch=4096, max_rows=0, stream=None):
        cg = g.c() if isinstance(g, Csr) else g
        mp = map_ptr.data_ptr() if hasattr(map_ptr, "data_ptr") else map_ptr
        loss = C.c_double()
        _check("gosh_mlp_train", lib().gosh_mlp_train(self.handle, C.byref(cg), C.c_void_p(mp), _ptr(Mc), _ptr(Mf),
                                                      self.d, dtype_code(Mc.dtype), epochs, lr, batch, max_rows,
                                                      _stream(stream), C.byref(loss)))
        return loss.value

    def project(self, Mc, map_ptr, g, Mf, stream=None):
        cg = g.c() if isinstance(g, Csr) else g
        mp = map_ptr.data_ptr() if hasattr(map_ptr, "data_ptr") else map_ptr
        _check("gosh_project_learned", lib().gosh_project_learned(self.handle, _ptr(Mc), C.c_void_p(mp),
                                                                  C.byref(cg), _ptr(Mf), self.d,
                                                                  dtype_code(Mc.dtype), _stream(stream)))

    def close(self):
        if self.handle:
            lib().gosh_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gosh_pair_scores(M, pairs, out=None, stream=None):
    import torch
    npairs = pairs.shape[0]
    if out is None:
        out = torch.empty(npairs, dtype=torch.float32, device=M.device)
    _check("gosh_pair_scores", lib().gosh_pair_scores(_ptr(M), M.shape[1], dtype_code(M.dtype), _ptr(pairs),
                                                      npairs, _ptr(out), _stream(stream)))
    return out


def gosh_link_auc(M, pos, neg, stream=None) -> float:
    a = C.c_double()
    _check("gosh_link_auc", lib().gosh_link_auc(_ptr(M), M.shape[1], dtype_code(M.dtype), _ptr(pos),
                                                pos.shape[0], _ptr(neg), neg.shape[0], _stream(stream),
                                                C.byref(a)))
    return a.value


def stats_dict(st: gosh_stats) -> dict:
    D = st.levels
    return {"levels": D, "n": list(st.n[:D]), "nnz": list(st.nnz[:D]), "epochs": list(st.epochs[:D]),
            "train_ms": list(st.train_ms[:D]), "coarsen_ms": st.coarsen_ms, "project_ms": st.project_ms,
            "total_ms": st.total_ms, "updates": int(st.updates)}
