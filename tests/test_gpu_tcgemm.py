"""The tcgen05 BF16 GEMM (tensor memory accumulators) against an FP64 host
product of the same BF16 operands.

Tolerance: each output sums K products of BF16 values exactly representable in
FP32, accumulated in FP32, so |error| <= K * 2^-24 * sum_k |a_k b_k| (plus the
order of accumulation); the test uses 1e-5 * (sum_k |a_k b_k|) + 1e-6.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_common import gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def run(M, N, K, splits=1, seed=0):
    g = gosh()
    gen = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K, generator=gen).to(torch.bfloat16)
    B = torch.randn(N, K, generator=gen).to(torch.bfloat16)
    Cd = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    Ad, Bd = A.cuda(), B.cuda()
    lib = g.lib()
    fn = lib.gosh_tc_gemm_bf16
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                   C.c_int, C.c_void_p]
    fn.restype = C.c_int
    st = fn(Ad.data_ptr(), K, Bd.data_ptr(), K, Cd.data_ptr(), N, M, N, K, splits,
            torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.gosh_last_error()
    ref = A.double() @ B.double().T
    bound = (A.double().abs() @ B.double().abs().T) * 1e-5 + 1e-6
    err = (Cd.double().cpu() - ref).abs()
    assert bool((err <= bound).all()), float((err - bound).max())


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (128, 16, 16), (300, 200, 272), (1000, 48, 32),
                                   (129, 144, 1040), (256, 300, 128)])
def test_tc_gemm_shapes(M, N, K):
    run(M, N, K)


@pytest.mark.parametrize("splits", [2, 8])
def test_tc_gemm_split_k(splits):
    run(128, 128, 4096, splits=splits, seed=3)
    run(256, 272, 2048, splits=splits, seed=4)
