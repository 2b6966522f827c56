"""CPU: the FDK backprojection reads detector rows r and r + 1 of each angle's
shared-memory window without clamping r, because the window spans the rows of
the tile's eight corners (where the perspective image of a box takes its
extremes) with one row of margin on each side.  This test rebuilds the windows
as the plan does (FP64 corner projections) and forms every voxel's row index
as the kernel does (FP32, the 1.5 * 2^23 rounding shift), for the geometries
of the GPU tests and a sample of the bench's 256^3 reconstruction, and checks
that r stays within [0, wv - 2] with the margin intact."""
import math

import numpy as np
import pytest

KT = 16  # voxel tile edge


def _fma32(a, b, c):
    # a * b is exact in FP64 for FP32 operands; one rounding to FP32 after the add
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) +
            np.asarray(c, np.float64)).astype(np.float32)


def _row_range(A, nv, R, nx, ny, nz, dv=1.0, beta=None, angle_step=1, col_step=1):
    f32 = np.float32
    beta = np.arange(A) * 2 * math.pi / A if beta is None else beta
    h = 0.5 * (KT - 1)

    def kv_of(x, y, z, cb, sb):
        return R * z / (R - (x * cb + y * sb)) / dv + 0.5 * (nv - 1)

    prm, wv = [], 2
    for tz in range(-(-nz // KT)):
        for ty in range(-(-ny // KT)):
            for tx in range(-(-nx // KT)):
                xc = tx * KT + h - 0.5 * (nx - 1)
                yc = ty * KT + h - 0.5 * (ny - 1)
                zc = tz * KT + h - 0.5 * (nz - 1)
                for a in range(0, A, angle_step):
                    cb, sb = math.cos(beta[a]), math.sin(beta[a])
                    vs = [kv_of(xc + (h if k & 1 else -h), yc + (h if k & 2 else -h),
                                zc + (h if k & 4 else -h), cb, sb) for k in range(8)]
                    r0 = math.floor(min(vs)) - 1
                    wv = max(wv, math.floor(max(vs)) + 2 - r0 + 1)
                    uc = R - (xc * cb + yc * sb)
                    prm.append((f32(zc), f32(cb), f32(sb), f32(uc),
                                f32(kv_of(xc, yc, zc, cb, sb) - r0)))
    d = (np.arange(KT) - 0.5 * (KT - 1)).astype(np.float32)
    DX, DY = np.meshgrid(d[::col_step], d[::col_step])
    DX, DY = DX.ravel(), DY.ravel()
    Rv, M = f32(R / dv), f32(12582912.0)
    lo, hi = 1 << 30, -(1 << 30)
    for zc, c, s, uc, kvo in prm:
        ds = _fma32(DX, c, (DY * s).astype(np.float32))
        inv = (f32(1.0) / ((uc - ds).astype(np.float32) * uc).astype(np.float32)).astype(np.float32)
        bz = ((Rv * uc).astype(np.float32) * inv).astype(np.float32)
        v0 = (_fma32(((Rv * zc).astype(np.float32) * ds).astype(np.float32), inv, kvo)
              - f32(0.5)).astype(np.float32)
        t = (_fma32(d[None, :], bz[:, None], v0[:, None]) + M).astype(np.float32)
        r = t.view(np.int32) - 0x4B400000
        lo, hi = min(lo, int(r.min())), max(hi, int(r.max()))
    return lo, hi, wv


@pytest.mark.parametrize("geom", [
    dict(A=60, nv=20, R=60.0, nx=32, ny=32, nz=16),
    dict(A=180, nv=96, R=150.0, nx=64, ny=64, nz=64),
    dict(A=73, nv=41, R=90.0, nx=37, ny=29, nz=21, dv=1.2,
         beta=np.sort(np.random.default_rng(23).uniform(0, 2 * np.pi, 73))),
    dict(A=40, nv=16, R=50.0, nx=24, ny=24, nz=16),
    dict(A=360, nv=320, R=1024.0, nx=256, ny=256, nz=256, angle_step=45, col_step=5),
])
def test_rows_stay_in_window(geom):
    lo, hi, wv = _row_range(**geom)
    assert lo >= 1 and hi + 1 <= wv - 2, (lo, hi, wv)
