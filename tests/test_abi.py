"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gosh.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(gosh_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gosh_coarsen", "gosh_train_level", "gosh_project", "gosh_embed"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2110_10049_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2110_10049_gb300 import gosh
    monkeypatch.setattr(gosh, "_lib", None)
    monkeypatch.setattr(gosh, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        gosh.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("binding loaded a missing library")


def test_params_default_on_host():
    from paper_2110_10049_gb300 import build, gosh
    build.build()
    p = gosh.default_params()
    assert (p.d, p.k, p.threshold) == (128, 3, 100)
    assert abs(p.shrink - 0.8) < 1e-12 and abs(p.lr_floor - 1e-4) < 1e-18
    # the paper's LargeGraphGPU settings and the defaults that keep its
    # serialised epochs and overlapping part-pair kernels
    assert (p.p_gpu, p.s_gpu, p.B) == (3, 2, 5)
    assert (p.large_serial, p.large_evict, p.epoch_overlap, p.overlap_min_vertices) == (0, 0, 1, 65536)
    assert (p.walk_length, p.walk_window) == (8, 3)


def test_struct_layouts_match_binding(tmp_path):
    """sizeof/offsetof of every ABI struct as gcc sees include/gosh.h equals
    the ctypes mirror in the binding."""
    import subprocess
    from paper_2110_10049_gb300 import gosh
    structs = {"gosh_params": gosh.gosh_params, "gosh_stats": gosh.gosh_stats, "gosh_csr": gosh.gosh_csr,
               "gosh_batch_stats": gosh.gosh_batch_stats, "gosh_large_stats": gosh.gosh_large_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gosh.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[name + "." + f]) == getattr(cls, f).offset, (name, f)
