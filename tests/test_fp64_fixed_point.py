"""CPU: the FP64 backprojection's detector coordinate in 64-bit fixed point.

The plan keeps u = (X2 cos/tau + Y2 sin/tau) / 2 + (n_det - 1)/2 as an integer
in units of 2^-S, with X2 = 2c - (n-1), Y2 = 2r - (n-1) and cos/tau, sin/tau
per angle in units of 2^-(S-1); S is the largest number of fraction bits (at
most 48) that keeps |u| 2^S, for every pixel and the partial block of pixels
beyond the image, below 2^62.  This test applies that rule, forms the
coordinate with exact integer arithmetic for sampled angles and pixels, and
checks it against the FP64 formula and the 64-bit range."""
import math

import numpy as np
import pytest


def _fraction_bits(n, D, c, s):
    half = 0.5 * (n - 1) + 16.0
    bound = half * (np.abs(c).max() + np.abs(s).max()) + 0.5 * (D - 1) + 1.0
    b = 0
    while 2.0 ** b <= bound:
        b += 1
    return min(48, 62 - b)


@pytest.mark.parametrize("n,A,D,tau", [(512, 720, 725, 1.0), (3, 2, 5, 1.0), (64, 9, 1500, 1.0),
                                       (96, 90, 137, 0.5), (2048, 64, 2899, 1.0),
                                       (16384, 8, 23171, 1.0)])
def test_fixed_point_coordinate(n, A, D, tau):
    th = np.arange(A) * math.pi / A
    c, s = np.cos(th) / tau, np.sin(th) / tau
    S = _fraction_bits(n, D, c, s)
    assert 24 <= S <= 48
    unit = 2.0 ** (S - 1)
    cx = [round(v * unit) for v in c]
    sy = [round(v * unit) for v in s]
    hd = round(0.5 * (D - 1) * 2.0 ** S)
    assert hd == 0.5 * (D - 1) * 2.0 ** S  # the detector offset is exact
    rng = np.random.default_rng(n + A)
    last = ((n + 15) // 16) * 16 - 1  # threads of a partial block go this far
    cols = [0, last] + list(rng.integers(0, n, 6))
    rows = [0, last] + list(rng.integers(0, n, 6))
    worst = 0.0
    for i in range(0, A, max(1, A // 16)):
        for col in cols:
            for row in rows:
                X2, Y2 = 2 * int(col) - (n - 1), 2 * int(row) - (n - 1)
                u_fx = X2 * cx[i] + Y2 * sy[i] + hd          # Python ints: exact
                assert abs(u_fx) < 2 ** 62 and abs(X2 * cx[i]) < 2 ** 62
                if col < n and row < n:
                    u = (col - 0.5 * (n - 1)) * c[i] + (row - 0.5 * (n - 1)) * s[i] + 0.5 * (D - 1)
                    worst = max(worst, abs(u_fx / 2.0 ** S - u))
    # the rounding of cos/tau and sin/tau to 2^-(S-1), times |X2|, |Y2| <= n
    assert worst <= n * 2.0 ** -S + 64 * np.finfo(float).eps * (n + D), worst
