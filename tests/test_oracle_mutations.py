"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/fbp_oracle.c (on the CPU),
builds it, and runs the pin suite against it in a subprocess: the suite must
fail.  The unmodified source must pass the same way (the control)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fbp_oracle.c")

MUTATIONS = [
    ("filter without the tau factor", "q[k] = tau * s;", "q[k] = s;"),
    ("Shepp-Logan denominator sign",
     "(1.0 - 4.0 * (double)m * (double)m)", "(4.0 * (double)m * (double)m - 1.0)"),
    ("Ram-Lak odd taps positive", "v = -1.0 / (M_PI * M_PI", "v = 1.0 / (M_PI * M_PI"),
    ("interpolation weights swapped", "return (1.0 - w) * q0 + w * q1;",
     "return w * q0 + (1.0 - w) * q1;"),
    ("x and y transposed in Eq. 2",
     "double t = x * cos(theta[i]) + y * sin(theta[i]);\n        double u = t / tau",
     "double t = y * cos(theta[i]) + x * sin(theta[i]);\n        double u = t / tau"),
    ("angular weight pi/A dropped", "return s * (M_PI / (double)n_angles);", "return s;"),
    ("detector centre off by half a bin",
     "double u = t / tau + 0.5 * (double)(n_det - 1);\n        s += interp",
     "double u = t / tau + 0.5 * (double)n_det;\n        s += interp"),
    ("splat weights swapped", "if (k >= 0 && k < n_det) p[k] += (1.0 - w) * v;",
     "if (k >= 0 && k < n_det) p[k] += w * v;"),
    ("Lambert-Beer without the one-count floor", "const double v = I[k] > 1.0 ? I[k] : 1.0;",
     "const double v = I[k];"),
    ("Lambert-Beer sign", "p[k] = -log(v / i0);", "p[k] = log(v / i0);"),
    ("PSNR with 10 log10", "out[0] = mse > 0.0 ? 20.0 * log10(", "out[0] = mse > 0.0 ? 10.0 * log10("),
    ("PSNR peak taken from the image", "if (fabs(y[k]) > mx) mx = fabs(y[k]);",
     "if (fabs(x[k]) > mx) mx = fabs(x[k]);"),
    ("SSIM window sigma 1", "w[a][b] = exp(-d2 / (2.0 * 1.5 * 1.5));",
     "w[a][b] = exp(-d2 / (2.0 * 1.0 * 1.0));"),
    ("SSIM C2 from K1", "c2 = (0.03 * L) * (0.03 * L);", "c2 = (0.01 * L) * (0.01 * L);"),
    ("SSIM covariance without its factor 2", "((2.0 * mx * my + c1) * (2.0 * cxy + c2))",
     "((2.0 * mx * my + c1) * (cxy + c2))"),
    ("volume weights swapped", "out[(long)m * np + p] = (1.0 - t) * slices[(long)k * np + p] +",
     "out[(long)m * np + p] = t * slices[(long)k * np + p] +"),
    ("volume picks the wrong interval", "while (k + 1 < K - 1 && zo[m] > z[k + 1]) ++k;",
     "while (k + 1 < K - 1 && zo[m] >= z[k]) ++k;"),
    ("FDK distance weight (R/U) instead of (R/U)^2", "sum += (J->R / U) * (J->R / U) * q;",
     "sum += (J->R / U) * q;"),
    ("FDK cosine weight dropped", "Pw[k] = P[k] * R / sqrt(R * R + u * u + v * v);",
     "Pw[k] = P[k];"),
    ("FDK without the v magnification", "const double u = J->R * t / U, v = J->R * z / U;",
     "const double u = J->R * t / U, v = z;"),
    ("FDK without the u magnification", "const double u = J->R * t / U, v = J->R * z / U;",
     "const double u = t, v = J->R * z / U;"),
    ("FDK detector axis mirrored", "t = -x * sb + y * cb;", "t = x * sb - y * cb;"),
    ("FDK scale for a half turn", "sum * (M_PI / (double)J->A)", "sum * (2.0 * M_PI / (double)J->A)"),
]


def _run_pins(lib_path):
    env = dict(os.environ, FBP_ORACLE_LIB=lib_path)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def _build(src_text, tmp_path, name):
    import oracle
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(so), str(c), "-lm", "-lpthread"])
    return str(so)


def test_unmodified_oracle_passes_its_pins(tmp_path):
    src = open(SRC).read()
    assert _run_pins(_build(src, tmp_path, "control")) == 0


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    broken = src.replace(old, new, 1)
    assert _run_pins(_build(broken, tmp_path, "mutant")) != 0, f"pins missed: {name}"
