"""The flop model bench.py reports against its closed form.  The metric counts,
for e eliminated pivots of an n x p supernode (m = n - p rows below),
  factor+solve = sum_{k=1..e} [(n-k) + 2((n-p)(p-k) + (p-k)(p-k+1)/2)],
  form         = (n-p)(n-p+1) e,
and the closed form below sums those series with the power-sum formulas, so an
off-by-one in the benchmark's loop would fail."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _s1(x):
    return x * (x + 1) // 2 if x >= 0 else 0


def _s2(x):
    return x * (x + 1) * (2 * x + 1) // 6 if x >= 0 else 0


def _closed_form(n, p, e):
    m = n - p
    pivots = e * n - e * (e + 1) // 2                     # sum (n - k)
    a21 = 2 * m * (e * p - e * (e + 1) // 2)              # sum 2 m (p - k)
    a11 = (_s2(p - 1) - _s2(p - e - 1)) + (_s1(p - 1) - _s1(p - e - 1))  # sum (p-k)(p-k+1), t = p-k
    return pivots + a21 + a11, m * (m + 1) * e


@pytest.mark.parametrize("n,p,e", [(1, 1, 1), (2000, 64, 13), (200000, 256, 256), (200000, 256, 12),
                                   (40, 40, 40), (300, 17, 0)])
def test_flop_model_closed_form(n, p, e):
    assert bench.flops_model(n, p, e) == _closed_form(n, p, e)


def test_flop_model_random():
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = int(rng.integers(1, 300))
        n = p + int(rng.integers(0, 5000))
        e = int(rng.integers(0, p + 1))
        assert bench.flops_model(n, p, e) == _closed_form(n, p, e)


def test_flop_model_all_eliminated():
    """With every pivot eliminated (e = p) the factor+solve count is
    m p^2 + p^3/3 + p^2/2 - 5p/6, i.e. about n p^2 - 2p^3/3."""
    for n, p in ((200000, 256), (2000, 64), (10, 10)):
        m = n - p
        fs, _ = bench.flops_model(n, p, p)
        assert 6 * fs == 6 * m * p * p + 2 * p ** 3 + 3 * p * p - 5 * p
