"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each checks it against an
independent route (a closed form, a library routine, an invariant, or brute
force on a tiny case), chosen so that a dropped term, a wrong sign or index, or
a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- filter taps
def _dtft(h, n_det, f):
    m = np.arange(-(n_det - 1), n_det, dtype=np.float64)
    return float(np.sum(h * np.cos(2.0 * np.pi * f * m)))


@pytest.mark.parametrize("n_det", [64, 363])
def test_ramlak_frequency_response_is_ramp(n_det):
    """Ram-Lak taps: tau * DTFT -> |f| on |f| <= 1/2 (Kak & Slaney eq. 3.61)."""
    h = oracle.taps(oracle.RAM_LAK, n_det, 1.0)
    tail = 1.05 / (math.pi ** 2 * (n_det - 1))  # sum of the dropped |h(m)|, |m| >= n_det
    for f in (0.0, 0.05, 0.125, 0.25, 0.37, 0.5):
        assert abs(_dtft(h, n_det, f) - abs(f)) <= tail


@pytest.mark.parametrize("n_det", [64, 725])
def test_shepp_logan_frequency_response(n_det):
    """Shepp-Logan taps: DTFT -> |f| sinc(f) = sin(pi |f|)/pi on |f| <= 1/2."""
    h = oracle.taps(oracle.SHEPP_LOGAN, n_det, 1.0)
    tail = 1.05 / (math.pi ** 2 * (n_det - 1))
    for f in (0.0, 0.05, 0.2, 0.3, 0.5):
        assert abs(_dtft(h, n_det, f) - math.sin(math.pi * abs(f)) / math.pi) <= tail


def test_ramlak_truncated_sum_closed_form():
    """sum_{|m|<=M} h(m) = (2/pi^2) sum_{odd m>M} 1/m^2 (the infinite sum is 0)."""
    M = 362
    h = oracle.taps(oracle.RAM_LAK, M + 1, 1.0)
    odd = np.arange(M + 1 if (M + 1) % 2 else M + 2, 4_000_001, 2, dtype=np.float64)
    expect = 2.0 / math.pi ** 2 * (np.sum(1.0 / odd ** 2) + 1.0 / (2.0 * 4_000_001))
    assert abs(float(h.sum()) - expect) < 1e-12
    assert abs(expect - 1.0 / (math.pi ** 2 * M)) < 1e-6


def test_taps_scale_with_spacing():
    """h_tau(m) = h_1(m) / tau^2 for both kernels; 'none' is a delta of height 1/tau."""
    for kind in (oracle.RAM_LAK, oracle.SHEPP_LOGAN):
        h1 = oracle.taps(kind, 40, 1.0)
        h2 = oracle.taps(kind, 40, 0.5)
        np.testing.assert_allclose(h2, h1 / 0.25, rtol=1e-15)
    h = oracle.taps(oracle.NONE, 10, 0.5)
    assert h[9] == 2.0 and np.count_nonzero(h) == 1


# --------------------------------------------------------------- row filter
@pytest.mark.parametrize("kind", [oracle.RAM_LAK, oracle.SHEPP_LOGAN])
def test_filter_equals_library_convolution(kind):
    """Direct sum == numpy linear convolution == FFT product with N >= 2D-1."""
    rng = np.random.default_rng(11)
    A, D, tau = 7, 45, 0.8
    P = rng.standard_normal((A, D))
    Q = oracle.filter_rows(P, kind, tau)
    h = oracle.taps(kind, D, tau)
    for i in range(A):
        full = np.convolve(P[i], h)  # length 3D-2; output k sits at index k + D - 1
        np.testing.assert_allclose(Q[i], tau * full[D - 1:2 * D - 1], rtol=0, atol=1e-13)
    N = 128  # >= 2D - 1 = 89: circular convolution equals the linear one on [0, D)
    hc = np.zeros(N)
    hc[:D] = h[D - 1:]
    hc[N - D + 1:] = h[:D - 1]
    Qf = tau * np.fft.irfft(np.fft.rfft(P, N, axis=1) * np.fft.rfft(hc), N, axis=1)[:, :D]
    np.testing.assert_allclose(Q, Qf, rtol=0, atol=1e-12 * np.abs(Q).max())


def test_filter_brute_force_toeplitz():
    """Q = P T^T with the explicit D x D matrix T[k][j] = tau h(k-j), D <= 32."""
    rng = np.random.default_rng(12)
    A, D, tau = 5, 32, 1.0
    P = rng.standard_normal((A, D))
    h = oracle.taps(oracle.RAM_LAK, D, tau)
    T = np.array([[tau * h[k - j + D - 1] for j in range(D)] for k in range(D)])
    np.testing.assert_allclose(oracle.filter_rows(P, oracle.RAM_LAK, tau), P @ T.T,
                               rtol=0, atol=1e-14)


def test_filter_kills_constant_in_the_middle():
    """The ramp has no DC: a constant row filters to ~0 away from the ends."""
    D = 301
    Q = oracle.filter_rows(np.ones((1, D)), oracle.RAM_LAK, 1.0)[0]
    mid = Q[D // 2]
    # far from both ends the residual is the truncated-tail sum ~ 2/(pi^2 * 150)
    assert abs(mid) < 2.0 / (math.pi ** 2 * 140)
    assert Q[0] > 0.1  # the edge keeps its value (zero outside the detector)


# ----------------------------------------------------------- backprojection
def _geom(n, A):
    return synthetic.det_for(n), oracle.default_angles(A)


def test_backprojection_of_constant_rows_is_pi_c():
    """Weights sum to 1 inside the detector, so f = (pi/A) * A * c = pi c."""
    n, A = 16, 12
    D, th = _geom(n, A)
    f = oracle.backproject(np.full((A, D), 2.5), th, 1.0, n)
    np.testing.assert_allclose(f, math.pi * 2.5, rtol=1e-14)


@pytest.mark.parametrize("A", [180, 7])
def test_backprojection_of_linear_rows_closed_form(A):
    """Q_i[k] = t_k is reproduced exactly by linear interpolation, so
    f(x,y) = (pi/A)(x sum cos th_i + y sum sin th_i), with sum cos = 1 and
    sum sin = cot(pi/(2A)) for th_i = i pi / A."""
    n, tau = 20, 1.0
    D, th = _geom(n, A)
    t = (np.arange(D) - 0.5 * (D - 1)) * tau
    f = oracle.backproject(np.tile(t, (A, 1)), th, tau, n)
    xy = np.arange(n) - 0.5 * (n - 1)
    X, Y = np.meshgrid(xy, xy)
    expect = (math.pi / A) * (X * 1.0 + Y / math.tan(math.pi / (2 * A)))
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-11 * np.abs(expect).max())
    if A == 180:
        assert abs(expect.max() / (math.pi / A) - (9.5 + 9.5 * 114.58865012931011)) < 1e-6


def test_quarter_turn_symmetry():
    """Rows shifted by A/2 (flipped on wrap, p(th+pi, t) = p(th, -t)) rotate f by 90 degrees."""
    n, A = 24, 16
    D, th = _geom(n, A)
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((A, D))
    Q2 = np.concatenate([Q[A // 2:], Q[:A // 2, ::-1]], axis=0)
    f = oracle.backproject(Q, th, 1.0, n)
    f2 = oracle.backproject(Q2, th, 1.0, n)
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    np.testing.assert_allclose(f2, f[c, n - 1 - r], rtol=0, atol=1e-12)


def test_adjoint_dot_product():
    """<R x, y> = (A/pi) <x, B y> for the splat R and the backprojection B."""
    n, A = 24, 30
    D, th = _geom(n, A)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((n, n))
    y = rng.standard_normal((A, D))
    lhs = float(np.sum(oracle.forward(x, th, D) * y))
    rhs = (A / math.pi) * float(np.sum(x * oracle.backproject(y, th, 1.0, n)))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


def test_forward_conserves_mass():
    """Interpolation weights sum to 1: every projection carries the image's total."""
    n, A = 20, 9
    D, th = _geom(n, A)
    f = np.random.default_rng(5).random((n, n))
    P = oracle.forward(f, th, D)
    np.testing.assert_allclose(P.sum(axis=1), f.sum(), rtol=1e-13)


def test_forward_converges_to_analytic_line_integrals():
    """Splat of a rasterised phantom -> analytic ellipse projections as n grows.

    A pixel-driven splat aliases bin by bin (its per-bin pattern does not vanish
    with refinement), so the projections are compared summed over blocks of a
    fixed phantom-space width (1/8 unit = n/16 bins); those converge at O(1/n)."""
    ell = synthetic.random_ellipses(3, seed=21)
    errs = []
    for n in (32, 64, 128):
        D, th = _geom(n, 12)
        img = synthetic.phantom_image(ell, n, supersample=8)
        P = oracle.forward(img, th, D)
        ref = synthetic.analytic_projection(ell, th, D, n) * (0.5 * n)
        B = n // 16
        m = (D // B) * B
        Pb = P[:, :m].reshape(len(th), -1, B).sum(axis=2)
        Rb = ref[:, :m].reshape(len(th), -1, B).sum(axis=2)
        errs.append(np.linalg.norm(Pb - Rb) / np.linalg.norm(Rb))
    assert errs[0] > 1.6 * errs[1] and errs[1] > 1.6 * errs[2]
    assert errs[2] < 0.006


def test_brute_force_system_matrix_8x8():
    """FBP = (pi/A) M^T (I (x) T) p with M built entry by entry from the hat
    function max(0, 1 - |u - k|) (no floor), for an 8x8 image."""
    n, A, tau = 8, 10, 1.0
    D, th = _geom(n, A)
    rng = np.random.default_rng(6)
    p = rng.standard_normal((A, D))
    M = np.zeros((A * D, n * n))
    for i in range(A):
        for r in range(n):
            for c in range(n):
                x, y = c - 0.5 * (n - 1), r - 0.5 * (n - 1)
                u = (x * math.cos(th[i]) + y * math.sin(th[i])) / tau + 0.5 * (D - 1)
                for k in range(D):
                    M[i * D + k, r * n + c] = max(0.0, 1.0 - abs(u - k))
    h = oracle.taps(oracle.SHEPP_LOGAN, D, tau)
    T = np.array([[tau * h[k - j + D - 1] for j in range(D)] for k in range(D)])
    q = (p @ T.T).reshape(-1)
    brute = (math.pi / A) * (M.T @ q)
    f = oracle.fbp(p, th, tau, oracle.SHEPP_LOGAN, n)
    np.testing.assert_allclose(f.reshape(-1), brute, rtol=0, atol=1e-13 * np.abs(brute).max())
    # and the splat is M itself
    img = rng.standard_normal((n, n))
    np.testing.assert_allclose(oracle.forward(img, th, D).reshape(-1), M @ img.reshape(-1),
                               rtol=0, atol=1e-13)


def test_pixel_subset_matches_full_image():
    n, A = 17, 11
    D, th = _geom(n, A)
    Q = np.random.default_rng(7).standard_normal((A, D))
    f = oracle.backproject(Q, th, 1.0, n, nthreads=3)
    rows = np.array([0, 16, 8, 3])
    cols = np.array([0, 16, 5, 12])
    np.testing.assert_array_equal(oracle.backproject_pixels(Q, th, 1.0, n, rows, cols), f[rows, cols])
    np.testing.assert_array_equal(oracle.backproject(Q, th, 1.0, n, nthreads=1), f)


# ----------------------------------------------------------------- whole FBP
@pytest.mark.parametrize("kind", [oracle.RAM_LAK, oracle.SHEPP_LOGAN])
def test_fbp_of_disk_recovers_density(kind):
    """Analytic projections of a centred disk (rho = 1, radius 0.5) reconstruct
    rho = 1 inside it (mean over the inner 80% of the radius within 1%) and 0
    well outside it: pins the tau and pi/A normalisation of the whole chain."""
    n, A = 128, 180
    D, th = _geom(n, A)
    disk = [synthetic.Ellipse(0.0, 0.0, 0.5, 0.5, 1.0, 0.0)]
    p = synthetic.analytic_projection(disk, th, D, n) * (0.5 * n)
    f = oracle.fbp(p, th, 1.0, kind, n, nthreads=4)
    xy = (np.arange(n) - 0.5 * (n - 1)) * (2.0 / n)
    X, Y = np.meshgrid(xy, xy)
    R = np.hypot(X, Y)
    assert abs(f[R < 0.4].mean() - 1.0) < 0.01
    assert abs(f[(R > 0.65) & (R < 0.9)].mean()) < 0.01


def test_fbp_with_detector_spacing():
    """Same disk sampled with tau = 0.5 (twice the bins) reconstructs the same density."""
    n, A, tau = 96, 120, 0.5
    D = 2 * synthetic.det_for(n)
    th = oracle.default_angles(A)
    disk = [synthetic.Ellipse(0.0, 0.0, 0.5, 0.5, 1.0, 0.0)]
    p = synthetic.analytic_projection(disk, th, D, n, tau) * (0.5 * n)
    f = oracle.fbp(p, th, tau, oracle.RAM_LAK, n, nthreads=4)
    xy = (np.arange(n) - 0.5 * (n - 1)) * (2.0 / n)
    X, Y = np.meshgrid(xy, xy)
    assert abs(f[np.hypot(X, Y) < 0.4].mean() - 1.0) < 0.01


def test_threaded_filter_and_fbp_match_single_thread():
    rng = np.random.default_rng(8)
    P = rng.standard_normal((13, 40))
    np.testing.assert_array_equal(oracle.filter_rows(P, oracle.RAM_LAK, 1.0, nthreads=4),
                                  oracle.filter_rows(P, oracle.RAM_LAK, 1.0, nthreads=1))
    th = oracle.default_angles(13)
    np.testing.assert_array_equal(oracle.fbp(P, th, 1.0, oracle.SHEPP_LOGAN, 21, nthreads=5),
                                  oracle.fbp(P, th, 1.0, oracle.SHEPP_LOGAN, 21, nthreads=1))


def test_lambert_beer_round_trip_and_floor():
    """Eq. 1: intensities made as I = i0 e^-p give back p (to rounding); counts
    at or below one photon give the floor ln(i0); scaling I and i0 together
    leaves p unchanged (above the floor)."""
    p = np.linspace(0.0, 9.0, 37)
    i0 = 1e5
    got = oracle.lambert_beer(i0 * np.exp(-p), i0)
    assert np.allclose(got, p, rtol=0, atol=1e-12)
    floor = oracle.lambert_beer(np.array([0.0, 0.5, 1.0, -3.0]), i0)
    assert np.allclose(floor, math.log(i0), rtol=0, atol=1e-12)
    counts = np.array([[2.0, 17.0, 4096.0], [99999.0, 3.0, 1.5]])
    assert np.allclose(oracle.lambert_beer(8.0 * counts, 8.0 * i0),
                       oracle.lambert_beer(counts, i0), rtol=0, atol=1e-12)
    assert oracle.lambert_beer(counts, i0).shape == counts.shape


# ------------------------------------------------ quality metrics (Eqs. 3, 4)
def test_psnr_closed_forms():
    """Eq. 3: identical images give +inf; an image off by a constant c from the
    reference y has MSE = c^2, so PSNR = 20 log10(max|y| / |c|); scaling both
    images leaves PSNR unchanged."""
    y = np.random.default_rng(7).normal(size=(30, 41))
    assert oracle.psnr(y, y)[0] == math.inf
    db, mse, mx = oracle.psnr(y + 0.125, y)
    assert mse == pytest.approx(0.125 ** 2, rel=1e-12)
    assert mx == np.abs(y).max()
    assert db == pytest.approx(20 * math.log10(np.abs(y).max() / 0.125), rel=1e-12)
    x = y + np.random.default_rng(8).normal(scale=0.01, size=y.shape)
    assert oracle.psnr(3.0 * x, 3.0 * y)[0] == pytest.approx(oracle.psnr(x, y)[0], rel=1e-12)


def test_ssim_identity_symmetry_and_constant_images():
    """Eq. 4: SSIM(x, x) = 1; SSIM is symmetric for a fixed L; two constant
    images a and b have zero variances, so every window gives
    (2ab + C1)/(a^2 + b^2 + C1) with C1 = (0.01 L)^2."""
    rng = np.random.default_rng(9)
    x = rng.random((37, 29))
    y = x + rng.normal(scale=0.05, size=x.shape)
    assert oracle.ssim(x, x, 1.0) == pytest.approx(1.0, abs=1e-14)
    assert oracle.ssim(x, y, 1.0) == pytest.approx(oracle.ssim(y, x, 1.0), abs=1e-14)
    a, b, L = 0.7, 0.4, 2.0
    c1 = (0.01 * L) ** 2
    got = oracle.ssim(np.full((20, 16), a), np.full((20, 16), b), L)
    assert got == pytest.approx((2 * a * b + c1) / (a * a + b * b + c1), rel=1e-12)


def test_ssim_dynamic_range_defaults_to_reference_span():
    rng = np.random.default_rng(10)
    y = rng.random((24, 24)) * 3.0 - 1.0
    x = y + rng.normal(scale=0.1, size=y.shape)
    assert oracle.ssim(x, y) == pytest.approx(oracle.ssim(x, y, y.max() - y.min()), rel=1e-14)


def test_ssim_window_from_an_impulse():
    """The window (Wang et al. 2004: 11 x 11 Gaussian, sigma 1.5, normalised),
    probed with an impulse: x is zero but for a 1 at the centre of a 31 x 31
    image, y is zero.  Windows that miss the impulse compare two zero patches
    (SSIM 1); a window holding it at offset (a, b) has mu_x = w_ab,
    sigma_x^2 = w_ab (1 - w_ab), mu_y = sigma_y = sigma_xy = 0, so its SSIM is
    C1 C2 / ((w_ab^2 + C1)(w_ab (1 - w_ab) + C2)); 121 of the 441 windows hold it."""
    n, L = 31, 1.0
    x = np.zeros((n, n))
    x[15, 15] = 1.0
    y = np.zeros((n, n))
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    d = np.arange(11) - 5
    g = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * 1.5 ** 2))
    w = g / g.sum()
    s = c1 * c2 / ((w ** 2 + c1) * (w * (1 - w) + c2))
    want = (441 - 121 + s.sum()) / 441
    assert oracle.ssim(x, y, L) == pytest.approx(want, rel=1e-12)
    assert math.isnan(oracle.ssim(np.zeros((10, 30)), np.zeros((10, 30)), 1.0))


# ------------------------------------------------ volume from a slice stack
def test_volume_is_exact_on_fields_linear_in_z():
    """Linear interpolation reproduces any field linear in z, on uneven slice
    spacing too: slices A + z_k B give planes A + z B at every z."""
    rng = np.random.default_rng(11)
    n = 6
    A, B = rng.normal(size=(n, n)), rng.normal(size=(n, n))
    z = np.array([0.0, 0.7, 1.1, 2.5, 4.0])
    zo = np.array([0.0, 0.35, 1.1, 1.9, 3.99, 4.0])
    vol = oracle.volume(A + z[:, None, None] * B, z, zo)
    assert np.allclose(vol, A + zo[:, None, None] * B, rtol=0, atol=1e-13)


def test_volume_hits_slices_and_midpoints_and_rejects_outside():
    rng = np.random.default_rng(12)
    S = rng.normal(size=(4, 5, 5))
    z = np.array([1.0, 2.0, 3.0, 5.0])
    vol = oracle.volume(S, z, np.array([2.0, 5.0, 1.5, 4.0]))
    assert np.array_equal(vol[0], S[1]) and np.array_equal(vol[1], S[3])
    assert np.allclose(vol[2], 0.5 * (S[0] + S[1]), atol=1e-15)
    assert np.allclose(vol[3], 0.5 * (S[2] + S[3]), atol=1e-15)
    with pytest.raises(ValueError):
        oracle.volume(S, z, np.array([0.5]))
    with pytest.raises(ValueError):
        oracle.volume(S, np.array([1.0, 2.0, 2.0, 3.0]), np.array([1.5]))


# ------------------------------------------------ FDK cone-beam (future work)
@pytest.mark.parametrize("du", [1.0, 0.8])
def test_fdk_tends_to_parallel_fbp_of_each_row(du):
    """As the source radius grows the cone turns parallel: every FDK weight
    tends to 1, u -> t and v -> z, and the reconstruction of any projections
    tends to the (pinned) parallel-beam FBP of each detector row at angles
    b + pi/2 (the full turn giving every line twice, which the 1/2 of FDK
    cancels against Eq. 2's pi/A over 2A... here A angles over 2 pi)."""
    rng = np.random.default_rng(13)
    A, nv, nu, n = 40, 6, 23, 16
    P = rng.normal(size=(A, nv, nu))
    beta = synthetic.cone_beta(A)
    f = oracle.fdk(P, beta, 1e10, du, 1.0, 0, n, n, nv)
    for iz in range(nv):
        g = oracle.fbp(P[:, iz, :], beta + np.pi / 2, du, 0, n)
        assert np.abs(f[iz] - g).max() <= 1e-7 * np.abs(g).max(), iz


def _ball_volume(fbp_kind, R, n, nz, A, nu, nv, ball):
    beta = synthetic.cone_beta(A)
    P = synthetic.cone_projection([ball], beta, R, nu, nv)
    return oracle.fdk(P, beta, R, 1.0, 1.0, fbp_kind, n, n, nz, nthreads=16)


def test_fdk_reconstructs_a_centred_ball():
    """A ball of density 1 (radius 20) at the centre, source radius 200: the
    mid-plane is fan-beam FBP (exact up to sampling): inside the ball the
    density is 1, outside 0, within 2%."""
    n, nz = 64, 5
    f = _ball_volume(1, 200.0, n, nz, 360, 112, 24, synthetic.Ellipsoid(0, 0, 0, 20, 20, 20, 0, 1.0))
    mid = f[nz // 2]
    c = np.arange(n) - 0.5 * (n - 1)
    r = np.hypot(c[None, :], c[:, None])
    assert abs(mid[r < 16].mean() - 1.0) < 0.02
    assert abs(mid[(r > 24) & (r < 30)].mean()) < 0.02


def test_fdk_weights_off_axis_in_the_mid_plane():
    """A small ball far off the axis (at x = 30, source radius 100, so the
    magnification along each ray varies by a factor of two over the turn):
    the fan-beam weights (R/U)^2 and the magnification u = R t / U must put it
    at the right place with density 1."""
    n, nz = 96, 9
    f = _ball_volume(1, 100.0, n, nz, 360, 432, 32, synthetic.Ellipsoid(30, 0, 0, 8, 8, 8, 0, 1.0))
    mid = f[nz // 2]
    c = np.arange(n) - 0.5 * (n - 1)
    X, Y = c[None, :], c[:, None]
    inside = np.hypot(X - 30, Y) < 5
    assert abs(mid[inside].mean() - 1.0) < 0.03
    w = np.clip(mid, 0, None) * (np.hypot(X - 30, Y) < 12)
    assert abs((w * X).sum() / w.sum() - 30.0) < 0.2 and abs((w * Y).sum() / w.sum()) < 0.2


def test_fdk_places_an_off_plane_ball():
    """A ball above the mid-plane and off the axis under a wide cone (source
    radius 60, ball at (20, 0, 10), so R / U runs from 0.75 to 1.5 over the
    turn): the cone magnification v = R z / U must put it at its height (FDK
    is approximate off the mid-plane; its own shift here is 0.06 voxel) with
    density near 1."""
    n, nz, R = 56, 32, 60.0
    beta = synthetic.cone_beta(360)
    P = synthetic.cone_projection([synthetic.Ellipsoid(20, 0, 10, 5, 5, 5, 0, 1.0)], beta, R,
                                  240, 100)
    f = oracle.fdk(P, beta, R, 1.0, 1.0, 1, n, n, nz, nthreads=16)
    z = np.arange(nz) - 0.5 * (nz - 1)
    c = np.arange(n) - 0.5 * (n - 1)
    Z, Y, X = np.meshgrid(z, c, c, indexing="ij")
    d = np.sqrt((X - 20) ** 2 + Y ** 2 + (Z - 10) ** 2)
    w = np.clip(f, 0, None) * (d < 9)
    for coord, want in ((X, 20.0), (Y, 0.0), (Z, 10.0)):
        assert abs((w * coord).sum() / w.sum() - want) < 0.2
    assert abs(f[d < 3].mean() - 1.0) < 0.03


def test_fdk_wide_fan_is_exact_in_the_mid_plane():
    """In the mid-plane FDK is fan-beam FBP, exact up to sampling.  With the
    source only 60 voxels from the axis and a ball 25 voxels off it, the rays
    through the ball reach u = 64 (cosine weight 0.68) and the distance weight
    (R/U)^2 swings from 0.4 to 3: the density must still be 1 within 0.5% and
    the ball where it is."""
    n, nz, R = 64, 3, 60.0
    beta = synthetic.cone_beta(720)
    P = synthetic.cone_projection([synthetic.Ellipsoid(25, 0, 0, 6, 6, 6, 0, 1.0)], beta, R,
                                  400, 8)
    mid = oracle.fdk(P, beta, R, 1.0, 1.0, 1, n, n, nz, nthreads=16)[1]
    c = np.arange(n) - 0.5 * (n - 1)
    X, Y = c[None, :], c[:, None]
    assert abs(mid[np.hypot(X - 25, Y) < 3.5].mean() - 1.0) < 0.005
    w = np.clip(mid, 0, None) * (np.hypot(X - 25, Y) < 10)
    assert abs((w * X).sum() / w.sum() - 25.0) < 0.05
