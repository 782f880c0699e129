"""The exactness claims behind the block-floating-point split pass, checked in IEEE FP32 on the host.

The pass rounds the leading part h of every component of r_n to a multiple of a quantum q (a power of
two) with |h| <= 2^21 q, and stores s A r with integer neighbour weights.  Its stencil then relies on:

1. fl(h + Cq) - Cq, with Cq = 1.5 * 2^23 * q, is h rounded to the nearest multiple of q, and h - hq is
   exact (the remainder joins the trailing part);
2. the six-neighbour sum ((n0 + n1) + (n2 + n3)) + (n4 + n5) of such leading parts is exact in FP32;
3. 16 * S1 is exact, and TwoSum(16 S1, -S2) returns the exact value of 16 S1 - S2 as a pair.

These are properties of FP32 arithmetic, checked here with numpy float32 against exact FP64 values
(every quantity involved has at most 24 + 28 significant bits, so FP64 holds them exactly).
"""

import numpy as np

f32 = np.float32


def _quantised(rng, n, q, bits=21):
    """n random multiples of q with |value| <= 2^bits q, as float32."""
    m = rng.integers(-(2 ** bits), 2 ** bits + 1, size=n)
    return (m.astype(np.float64) * q).astype(f32)


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def test_requantisation_rounds_to_the_grid_and_keeps_the_remainder_exact():
    rng = np.random.default_rng(11)
    for q_exp in (-40, -20, -3, 0, 7):
        q = 2.0 ** q_exp
        cq = f32(1.5 * 2.0 ** 23 * q)
        # leading parts of a normalised double-float value up to the bound
        h = (rng.uniform(-1.0, 1.0, 20000) * 2.0 ** 21 * q).astype(f32)
        hq = f32(f32(h + cq) - cq)
        k = hq.astype(np.float64) / q
        assert np.array_equal(k, np.round(k)), "hq is not a multiple of q"
        assert np.all(np.abs(hq.astype(np.float64) - h.astype(np.float64)) <= 0.5 * q)
        d = f32(h - hq)
        assert np.array_equal(d.astype(np.float64), h.astype(np.float64) - hq.astype(np.float64))


def test_six_neighbour_sums_of_leading_parts_are_exact():
    rng = np.random.default_rng(12)
    for q_exp in (-60, -17, 0, 3):
        q = 2.0 ** q_exp
        n = [_quantised(rng, 50000, q) for _ in range(6)]
        s = f32(f32(f32(n[0] + n[1]) + f32(n[2] + n[3])) + f32(n[4] + n[5]))
        exact = sum(x.astype(np.float64) for x in n)
        assert np.array_equal(s.astype(np.float64), exact)
        # the worst case: every neighbour at the bound
        top = f32(2.0 ** 21 * q)
        t = f32(f32(f32(top + top) + f32(top + top)) + f32(top + top))
        assert float(t) == 6 * 2.0 ** 21 * q


def test_weighted_fourth_order_sum_is_exact_as_a_pair():
    rng = np.random.default_rng(13)
    q = 2.0 ** -30
    n1 = [_quantised(rng, 50000, q) for _ in range(6)]
    n2 = [_quantised(rng, 50000, q) for _ in range(6)]
    s1 = f32(f32(f32(n1[0] + n1[1]) + f32(n1[2] + n1[3])) + f32(n1[4] + n1[5]))
    s2 = f32(f32(f32(n2[0] + n2[1]) + f32(n2[2] + n2[3])) + f32(n2[4] + n2[5]))
    a = f32(f32(16.0) * s1)
    assert np.array_equal(a.astype(np.float64), 16.0 * s1.astype(np.float64))
    lh, le = _two_sum(a, f32(-s2))
    exact = 16.0 * s1.astype(np.float64) - s2.astype(np.float64)
    assert np.array_equal(lh.astype(np.float64) + le.astype(np.float64), exact)


def test_a_plain_fp32_sum_of_unquantised_values_is_not_exact():
    """The point of the grid: the same sums without it lose low-order bits."""
    rng = np.random.default_rng(14)
    n = [rng.uniform(-1.0, 1.0, 50000).astype(f32) for _ in range(6)]
    s = f32(f32(f32(n[0] + n[1]) + f32(n[2] + n[3])) + f32(n[4] + n[5]))
    exact = sum(x.astype(np.float64) for x in n)
    assert not np.array_equal(s.astype(np.float64), exact)
