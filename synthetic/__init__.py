"""Seeded synthetic inputs for parallel-beam FBP: ellipse phantoms and their sinograms.

This module is the ONLY code shared by the FP64 oracle tests and the GPU path's
tests and benchmark.  It holds none of the reconstruction arithmetic (no filter,
no interpolation, no backprojection): it makes inputs.

The paper measures on Visible Human CT data (section "Benchmark"), which is not
available here; seeded random-ellipse phantoms with analytic line integrals
stand in for it.

Recipe (every draw comes from one SplitMix64 stream per seed):
  * SplitMix64 (Steele, Lea, Flood 2014), U[0,1) = (z >> 11) * 2**-53.
  * ellipse: centre uniform in the unit disk by rejection (cx = 2u-1, cy = 2u-1
    until cx^2 + cy^2 < 1), semi-axes a, b ~ U[0.05, 0.6], density
    rho ~ U[-0.2, 1.0], rotation alpha ~ U[0, pi); drawn in that order.
  * phantom coordinates: the n x n image spans [-1, 1]^2, so a pixel is 2/n
    phantom units and detector coordinate t (pixel units) is s = 2 t / n.
  * analytic projection of one ellipse (Kak & Slaney, ch. 3):
      p(theta, s) = 2 rho a b sqrt(a2 - s'^2) / a2  for s'^2 <= a2, else 0,
      a2 = a^2 cos^2(theta-alpha) + b^2 sin^2(theta-alpha),
      s' = s - (cx cos theta + cy sin theta),
    sampled at the bin centres t_k = (k - (n_det-1)/2) tau.
  * noise (Lambert-Beer, Eq. 1): counts ~ Poisson(I0 exp(-p)) with a numpy PCG64
    generator seeded by ``noise_seed``, then p~ = -ln(max(counts, 1) / I0).
  * the sinogram handed to FBP is the line integral in pixel-length units,
    (n/2) * p, so that the reconstruction approximates rho.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator (64-bit state, one output per call)."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """U[0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def choice(self, seq):
        return seq[min(int(self.uniform() * len(seq)), len(seq) - 1)]


@dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    rho: float
    alpha: float


def random_ellipses(count: int, seed: int) -> list[Ellipse]:
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        while True:
            cx = 2.0 * rng.uniform() - 1.0
            cy = 2.0 * rng.uniform() - 1.0
            if cx * cx + cy * cy < 1.0:
                break
        a = rng.uniform_range(0.05, 0.6)
        b = rng.uniform_range(0.05, 0.6)
        rho = rng.uniform_range(-0.2, 1.0)
        alpha = rng.uniform_range(0.0, math.pi)
        out.append(Ellipse(cx, cy, a, b, rho, alpha))
    return out


def default_angles(n_angles: int) -> np.ndarray:
    """theta_i = i*pi/n_angles (uniform on [0, pi))."""
    return np.arange(n_angles, dtype=np.float64) * (math.pi / n_angles)


def det_for(n_pix: int) -> int:
    """Detector count that covers the image diagonal: ceil(n*sqrt(2)) + 1."""
    return int(math.ceil(n_pix * math.sqrt(2.0))) + 1


def analytic_projection(ellipses, theta: np.ndarray, n_det: int, n_pix: int,
                        tau: float = 1.0) -> np.ndarray:
    """Line integrals in PHANTOM units, [n_angles][n_det], float64."""
    theta = np.asarray(theta, dtype=np.float64)
    t = (np.arange(n_det, dtype=np.float64) - 0.5 * (n_det - 1)) * tau
    s = t * (2.0 / n_pix)
    p = np.zeros((theta.shape[0], n_det), dtype=np.float64)
    ct = np.cos(theta)[:, None]
    st = np.sin(theta)[:, None]
    for e in ellipses:
        a2 = (e.a * np.cos(theta - e.alpha)) ** 2 + (e.b * np.sin(theta - e.alpha)) ** 2
        a2 = a2[:, None]
        sp = s[None, :] - (e.cx * ct + e.cy * st)
        inside = sp * sp <= a2
        val = np.where(inside, 2.0 * e.rho * e.a * e.b * np.sqrt(np.maximum(a2 - sp * sp, 0.0)) / a2, 0.0)
        p += val
    return p


def poisson_counts(p_phantom: np.ndarray, i0: float, noise_seed: int) -> np.ndarray:
    """Lambert-Beer (Eq. 1) measurement: photon counts ~ Poisson(i0 e^-p), float64."""
    rng = np.random.Generator(np.random.PCG64(noise_seed))
    return rng.poisson(i0 * np.exp(-p_phantom)).astype(np.float64)


def poisson_log(p_phantom: np.ndarray, i0: float, noise_seed: int) -> np.ndarray:
    """Lambert-Beer (Eq. 1) measurement and its log transform, float64."""
    counts = poisson_counts(p_phantom, i0, noise_seed)
    return -np.log(np.maximum(counts, 1.0) / i0)


def phantom_image(ellipses, n_pix: int, supersample: int = 4) -> np.ndarray:
    """Pixel-averaged density on the n x n grid (supersample^2 points per pixel)."""
    ss = int(supersample)
    off = (np.arange(ss, dtype=np.float64) + 0.5) / ss - 0.5
    idx = np.arange(n_pix, dtype=np.float64) - 0.5 * (n_pix - 1)
    xs = ((idx[:, None] + off[None, :]).reshape(-1)) * (2.0 / n_pix)
    X, Y = np.meshgrid(xs, xs)  # X varies along columns, Y along rows
    img = np.zeros_like(X)
    for e in ellipses:
        dx = X - e.cx
        dy = Y - e.cy
        ca, sa = math.cos(e.alpha), math.sin(e.alpha)
        u = dx * ca + dy * sa
        v = -dx * sa + dy * ca
        img += np.where((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0, e.rho, 0.0)
    return img.reshape(n_pix, ss, n_pix, ss).mean(axis=(1, 3))


@dataclass
class SliceSpec:
    n_pix: int
    n_angles: int
    n_det: int
    n_ellipses: int
    seed: int
    tau: float = 1.0
    filter: int = 0  # 0 Ram-Lak, 1 Shepp-Logan, 2 none
    i0: float | None = None  # None = noise-free
    noise_seed: int | None = None

    @property
    def updates(self) -> int:
        return self.n_pix * self.n_pix * self.n_angles


def sinogram(spec: SliceSpec, theta: np.ndarray | None = None) -> np.ndarray:
    """Sinogram in pixel-length units, float64 [n_angles][n_det]."""
    if theta is None:
        theta = default_angles(spec.n_angles)
    ell = random_ellipses(spec.n_ellipses, spec.seed)
    p = analytic_projection(ell, theta, spec.n_det, spec.n_pix, spec.tau)
    if spec.i0 is not None:
        p = poisson_log(p, spec.i0, spec.noise_seed if spec.noise_seed is not None else spec.seed)
    return p * (0.5 * spec.n_pix)


@dataclass
class Ellipsoid:
    """Ellipsoid in voxel units: centre, semi-axes, rotation about z, density."""
    cx: float
    cy: float
    cz: float
    a: float
    b: float
    c: float
    alpha: float
    rho: float


def random_ellipsoids(count: int, seed: int, n: int) -> list[Ellipsoid]:
    """Seeded ellipsoids inside an n^3 volume: centres uniform in the ball of
    radius 0.45 n, semi-axes U[0.05, 0.3] n, rotation U[0, pi), density
    U[-0.2, 1.0]."""
    rng = SplitMix64(seed)
    out = []
    while len(out) < count:
        x, y, z = (2.0 * rng.uniform() - 1.0 for _ in range(3))
        if x * x + y * y + z * z > 1.0:
            continue
        r = 0.45 * n
        out.append(Ellipsoid(x * r, y * r, z * r * 0.6, (0.05 + 0.25 * rng.uniform()) * n,
                             (0.05 + 0.25 * rng.uniform()) * n, (0.05 + 0.25 * rng.uniform()) * n,
                             math.pi * rng.uniform(), -0.2 + 1.2 * rng.uniform()))
    return out


def cone_beta(n_angles: int) -> np.ndarray:
    """Full-turn projection angles b_a = 2 pi a / A."""
    return np.arange(n_angles, dtype=np.float64) * (2.0 * np.pi / n_angles)


def cone_projection(ellipsoids, beta: np.ndarray, R: float, nu: int, nv: int, du: float = 1.0,
                    dv: float = 1.0) -> np.ndarray:
    """Exact cone-beam line integrals [A][nv][nu] of ellipsoids: the source at
    (R cos b, R sin b, 0), a virtual flat detector through the z axis with u
    along (-sin b, cos b, 0) and v along z, bin centres u_j = (j - (nu-1)/2) du,
    v_i = (i - (nv-1)/2) dv.  Each ray's chord through an ellipsoid comes from
    the quadratic |M (S + l d - c)|^2 = 1 (M: rotation then axis scaling)."""
    beta = np.asarray(beta, dtype=np.float64)
    u = (np.arange(nu) - 0.5 * (nu - 1)) * du
    v = (np.arange(nv) - 0.5 * (nv - 1)) * dv
    cb, sb = np.cos(beta)[:, None, None], np.sin(beta)[:, None, None]
    U, V = u[None, None, :], v[None, :, None]
    S = (R * cb, R * sb, np.zeros_like(cb))
    D = (-U * sb - R * cb, U * cb - R * sb, V + 0.0 * cb)  # detector point minus source
    dlen = np.sqrt(D[0] ** 2 + D[1] ** 2 + D[2] ** 2)
    out = np.zeros((beta.size, nv, nu))
    for e in ellipsoids:
        ca, sa = math.cos(e.alpha), math.sin(e.alpha)
        ex, ey, ez = S[0] - e.cx, S[1] - e.cy, S[2] - e.cz

        def frame(x, y, z):
            return ((x * ca + y * sa) / e.a, (-x * sa + y * ca) / e.b, z / e.c)
        e1 = frame(ex, ey, ez)
        g1 = frame(*D)
        qa = g1[0] ** 2 + g1[1] ** 2 + g1[2] ** 2
        qb = e1[0] * g1[0] + e1[1] * g1[1] + e1[2] * g1[2]
        qc = e1[0] ** 2 + e1[1] ** 2 + e1[2] ** 2 - 1.0
        disc = np.maximum(qb * qb - qa * qc, 0.0)
        out += e.rho * 2.0 * np.sqrt(disc) / qa * dlen
    return out


def photon_counts(spec: SliceSpec, theta: np.ndarray | None = None) -> np.ndarray:
    """The raw measurement behind a noisy slice: photon counts [n_angles][n_det]
    (float64) for the analytic projections in phantom units, the same draw
    sinogram() log-transforms.  Requires spec.i0."""
    if spec.i0 is None:
        raise ValueError("photon_counts needs a noisy spec (i0 set)")
    if theta is None:
        theta = default_angles(spec.n_angles)
    ell = random_ellipses(spec.n_ellipses, spec.seed)
    p = analytic_projection(ell, theta, spec.n_det, spec.n_pix, spec.tau)
    return poisson_counts(p, spec.i0, spec.noise_seed if spec.noise_seed is not None else spec.seed)


# Workloads: the five configurations of the benchmark plan, as synthetic recipes.
def cfg_plain() -> SliceSpec:
    """256x256, 180 angles, 363 bins, Ram-Lak (FFT length 1024), 10 ellipses, seed 1."""
    return SliceSpec(256, 180, 363, 10, seed=1, filter=0)


def cfg_float_double() -> SliceSpec:
    """512x512, 720 angles, 725 bins, Shepp-Logan, 20 ellipses, seed 2, Poisson I0=1e5."""
    return SliceSpec(512, 720, 725, 20, seed=2, filter=1, i0=1e5, noise_seed=102)


def cfg_float_double_slice(i: int) -> SliceSpec:
    """Slice i of a batch of float-vs-double slices: the same geometry and
    recipe, phantom seed 2 + 1000 i and noise seed 102 + 1000 i (i = 0 is
    cfg_float_double itself)."""
    base = cfg_float_double()
    return SliceSpec(base.n_pix, base.n_angles, base.n_det, base.n_ellipses,
                     seed=base.seed + 1000 * i, filter=base.filter, i0=base.i0,
                     noise_seed=base.noise_seed + 1000 * i)


def cfg_large() -> SliceSpec:
    """2048x2048, 2048 angles, 2899 bins, Ram-Lak, 40 ellipses, seed 4."""
    return SliceSpec(2048, 2048, 2899, 40, seed=4, filter=0)


def cfg_batch(count: int = 64, seed: int = 3) -> list[SliceSpec]:
    """Uneven slices: n from {256,384,512,768}, A from {180,360,720,1440}."""
    rng = SplitMix64(seed)
    out = []
    for s in range(count):
        n = rng.choice((256, 384, 512, 768))
        a = rng.choice((180, 360, 720, 1440))
        out.append(SliceSpec(n, a, det_for(n), 10, seed=1000 + s, filter=0))
    return out


def serving_stream(count: int, seed: int = 5, rate: float = 2000.0):
    """(arrival_time_s, SliceSpec) pairs: exponential gaps of mean 1/rate."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = rng.choice((256, 512, 768, 1024))
        a = rng.choice((360, 720, 1440))
        out.append((t, SliceSpec(n, a, det_for(n), 10, seed=50000 + r, filter=0,
                                 i0=1e5, noise_seed=150000 + r)))
    return out
