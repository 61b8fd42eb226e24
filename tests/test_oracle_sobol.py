"""Pins of the Sobol initialisation reference (App. A-A), on the CPU:
  * dimension 1 is the base-2 van der Corput sequence of the Gray code of the
    index (closed form: bit reversal of n ^ (n >> 1));
  * every 1-D projection of the first 2^m points puts exactly one point in
    each interval [j / 2^m, (j + 1) / 2^m) (the defining stratification);
  * dimensions 1 and 2 of the first 2^m points form a (0, m, 2)-net: each
    elementary box of area 2^-m holds exactly one point;
  * point 0 is the box's lower corner; skipping s points gives rows s.. of the
    unskipped sequence; the scaled points stay in the box.
A scrambled sequence, another ordering or a wrong scaling fails one of them.
"""
import numpy as np

from oracle import sobol_oracle as so


def _radical_inverse_gray(n, bits=32):
    g = n ^ (n >> 1)
    r = 0
    for j in range(bits):
        if (g >> j) & 1:
            r |= 1 << (bits - 1 - j)
    return r / 2.0 ** bits


def test_first_dimension_is_van_der_corput_of_gray_code():
    x = so.sobol_unit(1000, 3)
    ref = np.array([_radical_inverse_gray(n) for n in range(1000)])
    assert np.array_equal(x[:, 0], ref)


def test_one_dimensional_stratification():
    for m in (1, 4, 8, 11):
        x = so.sobol_unit(2 ** m, 16)
        cells = np.floor(x * 2 ** m).astype(np.int64)
        for k in range(16):
            assert np.array_equal(np.sort(cells[:, k]), np.arange(2 ** m)), (m, k)


def test_first_two_dimensions_form_a_0m2_net():
    m = 10
    x = so.sobol_unit(2 ** m, 2)
    for p in range(m + 1):
        q = m - p
        a = np.floor(x[:, 0] * 2 ** p).astype(np.int64)
        b = np.floor(x[:, 1] * 2 ** q).astype(np.int64)
        counts = np.bincount(a * 2 ** q + b, minlength=2 ** m)
        assert np.all(counts == 1), p


def test_box_scaling_and_skip():
    lo, hi = np.array([0.5, -2.0, 10.0]), np.array([1.5, 2.0, 11.0])
    th = so.sobol_box(300, lo, hi)
    assert np.array_equal(th[0], lo)
    assert np.all(th >= lo) and np.all(th < hi)
    assert np.allclose(th[1], lo + 0.5 * (hi - lo), rtol=0, atol=0)
    tail = so.sobol_box(100, lo, hi, skip=200)
    assert np.array_equal(tail, th[200:])
