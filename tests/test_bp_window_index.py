"""CPU: every (mid, slope) pair the backprojection kernel reads lies inside the
detector window its producer warp staged for that tile and angle.

The producer computes, in FP64, the window's first pair from the tile's
smallest detector coordinate (aligned down to 16 bytes) and the tile-local
offset of the coordinate; the consumers form each pixel's local coordinate in
FP32 (two FMAs), round it with the 1.5 * 2^23 shift and read the pair at the
rounded value with no clamp.  The window has one bin of margin below and at
least half a bin above the coordinates the tile can reach, far beyond the FP32
error of a local coordinate, so the index stays in [0, wp - 1].  This test
rebuilds the window width as the plan does and forms every pixel's index as
the kernel does, for the shapes and geometries of the GPU tests and a sample
of the bench's."""
import math

import numpy as np
import pytest

import synthetic

M = np.float32(12582912.0)  # 1.5 * 2^23


def _window_pairs(c, s, tx, ty, align):
    ext = max((tx - 1) * abs(ci) + (ty - 1) * abs(si) for ci, si in zip(c, s))
    wp = math.ceil(ext + 1e-6) + align + 2
    return ((wp + align - 1) // align) * align


def _index_range(n, A, D, tau=1.0, theta=None, tile=(32, 32), align=2, angle_step=1):
    th = np.arange(A) * math.pi / A if theta is None else np.asarray(theta)
    c, s = np.cos(th) / tau, np.sin(th) / tau
    TX, TY = tile
    wp = _window_pairs(c, s, TX, TY, align)
    hn, hd = 0.5 * (n - 1), 0.5 * (D - 1)
    LX, LY = np.meshgrid(np.arange(TX, dtype=np.float32), np.arange(TY, dtype=np.float32))
    lo, hi = 1 << 30, -(1 << 30)
    for by in range(-(-n // TY)):
        for bx in range(-(-n // TX)):
            x0, y0 = bx * TX - hn, by * TY - hn
            for i in range(0, len(th), angle_step):
                u0 = x0 * c[i] + y0 * s[i] + hd
                umin = u0 + min(0.0, (TX - 1) * c[i]) + min(0.0, (TY - 1) * s[i])
                pb = math.floor(umin) & ~(align - 1)
                off = np.float32(u0 - (pb - 1) - 0.5)
                c32, s32 = np.float32(c[i]), np.float32(s[i])
                # fma rounding: the FP32 product is exact in FP64, one rounding after the add
                xc = (LX.astype(np.float64) * c32 + off).astype(np.float32)
                v = (LY.astype(np.float64) * s32 + xc).astype(np.float32)
                k = ((v + M).astype(np.float32).view(np.int32) - 0x4B400000)
                lo, hi = min(lo, int(k.min())), max(hi, int(k.max()))
    return lo, hi, wp


@pytest.mark.parametrize("geom", [
    dict(n=100, A=37, D=143),
    dict(n=33, A=50, D=60, tau=0.8),
    dict(n=70, A=21, D=70, tau=1.6),
    dict(n=5, A=3, D=9),
    dict(n=96, A=90, D=137, tile=(8, 32)),
    dict(n=96, A=90, D=137, tile=(32, 64)),
    dict(n=48, A=29, D=synthetic.det_for(48),
         theta=np.sort(np.random.default_rng(99).uniform(-3.0, 7.0, 29))),
    dict(n=200, A=150, D=284, align=4),  # FP16 pairs: 16-byte alignment is 4 pairs
    dict(n=512, A=720, D=725, angle_step=23),
    dict(n=2048, A=2048, D=2899, tile=(32, 64), angle_step=257),
])
def test_pair_index_stays_in_window(geom):
    lo, hi, wp = _index_range(**geom)
    assert 0 <= lo and hi <= wp - 1, (lo, hi, wp)


def _pair_index_range(n, A, D, tau=1.0, theta=None, tile=(32, 32), align=2, angle_step=1):
    """Point-symmetric tile pairs: the partner pixel of a thread reads pair
    K - j of the partner tile's window, K = n_det - pb_A - pb_B, j the thread's
    own index (formed as in _index_range).  Returns the range of K - j."""
    th = np.arange(A) * math.pi / A if theta is None else np.asarray(theta)
    c, s = np.cos(th) / tau, np.sin(th) / tau
    TX, TY = tile
    assert n % TX == 0 and n % TY == 0
    gx, gy = n // TX, n // TY
    assert not (gx % 2 and gy % 2)
    wp = _window_pairs(c, s, TX, TY, align)
    hn, hd = 0.5 * (n - 1), 0.5 * (D - 1)
    LX, LY = np.meshgrid(np.arange(TX, dtype=np.float32), np.arange(TY, dtype=np.float32))
    lo, hi = 1 << 30, -(1 << 30)
    tiles = gx * gy
    for a in range(tiles // 2):
        b = tiles - 1 - a
        x0, y0 = (a % gx) * TX - hn, (a // gx) * TY - hn
        x0b, y0b = (b % gx) * TX - hn, (b // gx) * TY - hn
        for i in range(0, len(th), angle_step):
            ex = min(0.0, (TX - 1) * c[i]) + min(0.0, (TY - 1) * s[i])
            u0 = x0 * c[i] + y0 * s[i] + hd
            pb = math.floor(u0 + ex) & ~(align - 1)
            pbb = math.floor(x0b * c[i] + y0b * s[i] + hd + ex) & ~(align - 1)
            K = D - pb - pbb
            off = np.float32(u0 - (pb - 1) - 0.5)
            c32, s32 = np.float32(c[i]), np.float32(s[i])
            xc = (LX.astype(np.float64) * c32 + off).astype(np.float32)
            v = (LY.astype(np.float64) * s32 + xc).astype(np.float32)
            j = ((v + M).astype(np.float32).view(np.int32) - 0x4B400000)
            jb = K - j
            lo, hi = min(lo, int(jb.min())), max(hi, int(jb.max()))
    return lo, hi, wp


@pytest.mark.parametrize("geom", [
    dict(n=128, A=90, D=183),
    dict(n=128, A=45, D=120, tau=1.6),
    dict(n=64, A=50, D=120, tau=0.8),
    dict(n=256, A=180, D=363, tile=(8, 32)),
    dict(n=256, A=97, D=363, tile=(32, 64),
         theta=np.sort(np.random.default_rng(98).uniform(-3.0, 7.0, 97))),
    dict(n=192, A=120, D=273, align=4),  # FP16 pairs
    dict(n=512, A=720, D=725, tile=(32, 64), angle_step=23),
    dict(n=2048, A=2048, D=2899, tile=(32, 64), angle_step=257),
])
def test_point_pair_partner_index_stays_in_window(geom):
    lo, hi, wp = _pair_index_range(**geom)
    assert 0 <= lo and hi <= wp - 1, (lo, hi, wp)
