"""Stochastic rounding of 16-bit tables (gosh_round_stochastic applies the
rounding every 16-bit table write uses) against its definition:

- every result is one of the two 16-bit values that bracket x (the one toward
  zero and the next one away from zero); representable values, infinities and
  NaN pass unchanged;
- unbiased: for x a fraction f of the way between its neighbours the result
  is the upper one with probability f, so over 2^22 draws the mean is x and
  the fraction rounded up is f, within 6 standard errors (plus the 2^-16
  resolution of the random bits); BF16 and FP16;
- different seeds give different roundings.
"""
import numpy as np
import pytest

from gpu_common import gosh, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def round16(x, dtype, seed=1):
    g = gosh()
    out = g.gosh_round_stochastic(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(), dtype, seed)
    torch.cuda.synchronize()
    return out.cpu().float().numpy().astype(np.float64)


def bf16_neighbours(x):
    b = np.asarray(x, np.float32).view(np.uint32)
    lo = (b & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((b & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    return lo, hi


def f16_neighbours(x):
    x = np.asarray(x, np.float32)
    r = x.astype(np.float16)
    away = np.abs(r.astype(np.float64)) > np.abs(x.astype(np.float64))
    toward0 = np.where(away, np.nextafter(r, np.float16(0)), r)
    up = np.nextafter(toward0, np.where(x < 0, np.float16(-np.inf), np.float16(np.inf)).astype(np.float16))
    return toward0.astype(np.float64), up.astype(np.float64)


@pytest.mark.parametrize("dtype,lo_mag,hi_mag", [(torch.bfloat16, 1e-30, 1e30), (torch.float16, 1e-4, 6e4)])
def test_result_is_a_bracketing_neighbour(dtype, lo_mag, hi_mag):
    rng = np.random.default_rng(0)
    x = (np.exp(rng.uniform(np.log(lo_mag), np.log(hi_mag), 200000)) *
         np.where(rng.random(200000) < 0.5, -1, 1)).astype(np.float32)
    y = round16(x, dtype)
    lo, hi = bf16_neighbours(x) if dtype == torch.bfloat16 else f16_neighbours(x)
    ok = (y == lo) | (y == hi)
    assert ok.all(), (x[~ok][:5], y[~ok][:5], lo[~ok][:5], hi[~ok][:5])
    assert (y != lo).any() and (y != hi).any()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_representable_and_special_values_unchanged(dtype):
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.normal(size=4096).astype(np.float32)).to(dtype).float().numpy()
    x = np.concatenate([x, np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -2.0], np.float32)])
    y = round16(x, dtype)
    np.testing.assert_array_equal(y, x.astype(np.float64))
    z = round16(np.array([np.nan] * 8, np.float32), dtype)
    assert np.isnan(z).all()


@pytest.mark.parametrize("dtype,base,gap", [(torch.bfloat16, 1.0, 2.0 ** -7), (torch.float16, 1.0, 2.0 ** -10),
                                            (torch.bfloat16, -3.0, 2.0 ** -6)])
@pytest.mark.parametrize("f", [0.1, 0.5, 0.9, 0.125])
def test_unbiased(dtype, base, gap, f):
    n = 1 << 22
    x0 = base + (f * gap if base > 0 else -f * gap)
    x = np.full(n, x0, np.float32)
    y = round16(x, dtype, seed=7)
    up = np.abs(y) > abs(base)
    se = np.sqrt(f * (1 - f) / n)
    assert abs(up.mean() - f) < 6 * se + 2.0 ** -16, (up.mean(), f)
    assert abs(y.mean() - float(np.float32(x0))) < gap * (6 * se + 2.0 ** -16)


def test_seeds_differ():
    x = np.full(4096, 1.0 + 0.5 * 2.0 ** -7, np.float32)
    a, b = round16(x, torch.bfloat16, seed=1), round16(x, torch.bfloat16, seed=2)
    assert (a != b).any() and abs(a.mean() - b.mean()) < 0.05 * 2.0 ** -7 * 8
