"""The solvers' inner products on the GPU (mh3d_dot: exact FP32 products
summed in float pairs through fixed warp, block and grid trees, one FP64
total) against the exact sum.

Products of two float32 values are exact in float64 (24 + 24 significand
bits), so math.fsum of the float64 products is the correctly rounded exact
value.  The bar is relative to sum |a_i b_i|, the scale that bounds the
rounding error of any summation (FP64 recursive summation of 2^20 terms
guarantees only ~1e-10 of it, pairwise summation ~2e-15): inputs with
alternating signs, a dynamic range of 1e12 and exact cancellation make the
value itself far smaller than that scale.
"""
import math

import numpy as np
import pytest

import workloads as W
from tests._cases import gpu_plan, params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(kind, n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-6.0, 6.0, n)
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    a = (mag * sign).astype(np.float32)
    b = rng.uniform(0.5, 1.5, n).astype(np.float32)
    if kind == "positive":
        a = np.abs(a)
    elif kind == "exact_cancel":
        # neighbours cancel exactly; the value is one small leftover term
        a = np.repeat(a[0::2], 2)[:n]
        a[1::2] *= -1.0
        b = np.ones(n, dtype=np.float32)
        a[-1] = np.float32(1.5)
    return a, b


@pytest.mark.parametrize("kind", ["alternating", "positive", "exact_cancel"])
@pytest.mark.parametrize("n", [1 << 20, 1_000_003])
def test_pair_dot_matches_exact_sum(kind, n):
    from paper_2503_13802_gb300 import mh3d_dot

    plan = gpu_plan(params((16, 8, 8), kmin=2, kmax=3))
    a, b = _case(kind, n, 7 + n % 5)
    prods = a.astype(np.float64) * b.astype(np.float64)
    exact = math.fsum(prods)
    scale = float(np.sum(np.abs(prods)))
    got = mh3d_dot(plan, torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"))
    np64 = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    print(f"{kind} n={n}: exact {exact:.17g}, GPU error {abs(got - exact) / scale:.2e}, "
          f"numpy FP64 error {abs(np64 - exact) / scale:.2e} (relative to sum |a b|)")
    assert abs(got - exact) <= 1e-13 * scale, (got, exact, scale)
    if kind == "positive":   # no cancellation: relative to the value itself
        assert abs(got - exact) <= 1e-13 * abs(exact)


def test_pair_dot_is_deterministic_and_handles_edge_lengths():
    """Fixed trees: the same inputs give the same bits; n = 0 gives 0 and
    n = 1 the exact product."""
    from paper_2503_13802_gb300 import mh3d_dot

    plan = gpu_plan(params((16, 8, 8), kmin=2, kmax=3))
    a = torch.as_tensor(W.random_volume((64, 64, 64), 3).astype(np.float32), device="cuda").reshape(-1)
    b = torch.as_tensor(W.random_volume((64, 64, 64), 4).astype(np.float32), device="cuda").reshape(-1)
    v = [mh3d_dot(plan, a, b) for _ in range(3)]
    assert v[0] == v[1] == v[2]
    assert mh3d_dot(plan, a[:0], b[:0]) == 0.0
    assert mh3d_dot(plan, a[:1], b[:1]) == float(a[0].double() * b[0].double())
