"""The fetch's canonical angles (gather_angles_kernel) are computed without an
FP64 arctangent: a rough FP32 angle picks the nearest of 256 equally spaced
angles t_j, (c, s) is rotated back by t_j, and theta = t_j + arcsin x with
x = s cos t_j - c sin t_j, the arcsine summed as its Maclaurin series to x^9.
This test restates that method in numpy (the FP32 estimate from the doubles'
high words, the table in extended precision, the same fused operations) and
checks it against numpy's arctan2 within one unit in the last place of pi,
over random angles and the edge cases (+-pi, +-0, +-pi/2, near +-pi).  The
kernel itself is held to the oracle's angles within 2e-15 rad by the GPU
parity tests."""
import math

import mpmath
import numpy as np

STEPS = 256
T = STEPS + 1


def _table():
    tab = np.zeros(3 * T)
    two_pi = 2 * mpmath.pi
    for j in range(T):
        t = float(mpmath.mpf(j - STEPS // 2) * two_pi / STEPS)
        tab[j] = t
        tab[T + j] = float(mpmath.cos(mpmath.mpf(t)))
        tab[2 * T + j] = float(mpmath.sin(mpmath.mpf(t)))
    return tab


def _rough_float(v):
    hi = (np.asarray(v, np.float64).view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    mag = hi & np.uint32(0x7fffffff)
    bits = np.where(mag < np.uint32(897 << 20), np.uint32(0), (mag - np.uint32(896 << 20)) << np.uint32(3))
    return (bits | (hi & np.uint32(0x80000000))).view(np.float32)


def _fma(a, b, c):
    # a fused multiply-add, emulated: product and sum in extended precision (64-bit
    # significand on x86), then one rounding to double
    return (np.longdouble(a) * np.longdouble(b) + np.longdouble(c)).astype(np.float64)


def _angle(c, s, tab):
    est = np.arctan2(_rough_float(s), _rough_float(c)).astype(np.float32)
    j = np.clip(np.rint(est * np.float32(STEPS / (2 * math.pi))).astype(np.int64), -STEPS // 2, STEPS // 2)
    j += STEPS // 2
    tj, cj, sj = tab[j], tab[T + j], tab[2 * T + j]
    r = _fma(s, cj, -(c * sj))
    r2 = r * r
    q = _fma(r2, 35.0 / 1152.0, 5.0 / 112.0)
    q = _fma(r2, q, 3.0 / 40.0)
    q = _fma(r2, q, 1.0 / 6.0)
    return tj + _fma(r * r2, q, r)


def test_table_reduction_and_arcsine_series_match_arctan2():
    tab = _table()
    rng = np.random.default_rng(7)
    th = rng.uniform(-math.pi, math.pi, 200_000)
    c, s = np.cos(th), np.sin(th)
    edge = np.array([[1.0, 0.0], [-1.0, 0.0], [-1.0, -0.0], [0.0, 1.0], [0.0, -1.0], [-1.0, 1e-300],
                     [-1.0, -1e-300], [math.cos(math.pi - 1e-9), math.sin(math.pi - 1e-9)],
                     [math.cos(-math.pi + 1e-9), math.sin(-math.pi + 1e-9)],
                     [math.cos(math.pi / 256), math.sin(math.pi / 256)]])
    c = np.concatenate([c, edge[:, 0]])
    s = np.concatenate([s, edge[:, 1]])
    got, ref = _angle(c, s, tab), np.arctan2(s, c)
    assert np.max(np.abs(got - ref)) <= np.spacing(math.pi)
    assert np.all(np.abs(got) <= math.pi)
    # a norm off 1 by rounding moves the angle by far less than an ulp
    k = 1 + 3e-16
    assert np.max(np.abs(_angle(c * k, s * k, tab) - ref)) <= np.spacing(math.pi)


def test_series_truncation_bound():
    # the first omitted term, 63 x^11 / 2816, over the widest reduced angle
    x = math.pi / STEPS + 2e-6
    assert 63 * x ** 11 / 2816 < 1e-22
