"""The scorer's constant tables, read from the CUDA source and checked on the CPU.

A cell group of G queries (1 <= G <= 32) gives each query k = floor(32 / G)
lanes; lane l serves query floor(l / k), computed as (l * m_k) >> 10 with
m_k = ceil(1024 / k).  A wrong entry in either table would hand a lane the
wrong query (or none) and change nearest neighbours, so both are checked
against the arithmetic they replace for every G and every lane.
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_00326_gb300", "csrc",
                   "perch_kernels.cu")


def _table(name):
    text = open(SRC).read()
    m = re.search(name + r"\[33\]\s*=\s*\{([^}]*)\}", text)
    assert m, name
    return [int(x) for x in m.group(1).replace("\n", " ").split(",") if x.strip()]


def test_lanes_per_query_table():
    k = _table("c_lanes_per_query")
    assert len(k) == 33
    for g in range(1, 33):
        assert k[g] == 32 // g, g


def test_lane_to_query_division_is_exact():
    k_of = _table("c_lanes_per_query")
    m_of = _table("c_lane_div")
    assert len(m_of) == 33
    for g in range(1, 33):
        k = k_of[g]
        m = m_of[k]
        lanes = np.arange(32)
        assert np.array_equal((lanes * m) >> 10, lanes // k), (g, k, m)
        # every query gets its k lanes, and only the first g * k lanes are used
        q = (lanes[: g * k] * m) >> 10
        assert np.array_equal(np.bincount(q, minlength=g), np.full(g, k)), g


def test_small_division_by_reciprocal_is_exact():
    """The scorer's integer division without a divide instruction: for
    0 <= n < 2^24 and 1 <= d < 2^24, trunc(fl(fl(n) fl(1/d))) is within one of
    floor(n / d) (both operands exact in binary32, two roundings of 2^-24 each,
    quotient below 2^23 unless d = 1, where the product is exact), so one
    correction step by the exact remainder gives the quotient.  Checked in
    binary32 arithmetic on random and extreme operands."""
    rng = np.random.default_rng(0)
    n = np.concatenate([rng.integers(0, 1 << 24, 200000), np.array([0, 1, (1 << 24) - 1] * 3)])
    d = np.concatenate([rng.integers(1, 1 << 24, 100000), rng.integers(1, 64, 100000),
                        np.array([1, 1, 1, 2, 3, (1 << 24) - 1, (1 << 23) + 1, 7, 65535])])
    r = np.float32(1.0) / d.astype(np.float32)                 # correctly rounded reciprocal
    q = np.trunc(n.astype(np.float32) * r).astype(np.int64)    # one more rounding, then toward zero
    rem = n - q * d
    assert np.all(np.abs(n // d - q) <= 1)
    q = q + (rem >= d) - (rem < 0)
    assert np.array_equal(q, n // d)


def test_edge_coefficients_are_exact_in_32_bits():
    """A staged triangle's edge i at the sample (16 u, 16 v) is evaluated as
    a u + b v + c in wrapping 32-bit arithmetic, a = -16 dy, b = 16 dx,
    c = dy x_p - dx y_p (p, q the edge's vertices, dx = x_q - x_p, ...): the
    partial products may wrap, but the value is the edge function itself
    whenever that lies in int32, which the guard band guarantees for samples
    of the image (|x| < 32 W, |y| < 32 H in 1/16 px).  Checked against int64
    edge functions for vertices anywhere in the guard band of a 1023 x 1023
    image and samples anywhere in it."""
    rng = np.random.default_rng(1)
    W = H = 1023
    m = 400000
    xp, xq = rng.integers(-16 * W, 32 * W, m), rng.integers(-16 * W, 32 * W, m)
    yp, yq = rng.integers(-16 * H, 32 * H, m), rng.integers(-16 * H, 32 * H, m)
    u, v = rng.integers(0, W, m), rng.integers(0, H, m)
    dx, dy = xq - xp, yq - yp
    exact = dx * (16 * v - yp) - dy * (16 * u - xp)               # int64
    mask = (1 << 32) - 1
    a, b, c = (-16 * dy) & mask, (16 * dx) & mask, (dy * xp - dx * yp) & mask
    w = (a * u + b * v + c) & mask                                 # wrapping 32-bit sum
    w = np.where(w >= (1 << 31), w - (1 << 32), w)
    inside = np.abs(exact) < (1 << 31)
    assert inside.mean() > 0.99
    assert np.array_equal(w[inside], exact[inside])
