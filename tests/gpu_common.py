"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def gosh():
    from paper_2110_10049_gb300 import build, gosh as g
    build.build()
    return g


def bf16_round_np(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest even) -> float64, on the host via torch CPU."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def rel_fro(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
