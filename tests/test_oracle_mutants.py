"""The oracle's pins reject a wrong oracle.

Each case below plants one plausible mistake in a copy of the oracle's C
source (a flipped sign, a dropped term, a transposed operand, a wrong index
or offset), compiles the copy, and runs the oracle pin suites
(test_oracle_qr.py, test_oracle_siddon.py) against it in a child process.
The suites must fail for every mutant, and must pass for an unmodified copy
built the same way.  The mistakes are planted in the CPU oracle only; no
GPU code is involved.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ctqr_oracle.c")
PIN_SUITES = [os.path.join(ROOT, "tests", "test_oracle_qr.py"),
              os.path.join(ROOT, "tests", "test_oracle_siddon.py")]

# (name, original text, planted text, which occurrence of the original)
MUTANTS = [
    # Householder reflectors (Sec. 2 Eq. 2, LAPACK's larfg convention)
    ("beta_sign", "double beta = (alpha >= 0.0) ? -norm : norm;",
     "double beta = (alpha >= 0.0) ? norm : -norm;", 0),
    ("tau_sign", "tau[j] = (beta - alpha) / beta;", "tau[j] = (alpha - beta) / beta;", 0),
    ("v_scale_sign", "double scale = 1.0 / (alpha - beta);", "double scale = 1.0 / (beta - alpha);", 0),
    ("update_drops_unit_head", "double dot = a[0];", "double dot = 0.0;", 0),
    ("update_drops_tau", "double wk = tj * dot;", "double wk = dot;", 0),
    # Q^T B and Q B (Sec. 2 Eq. 3)
    ("qt_wrong_rows", "dot += v[i] * b[j + i];", "dot += v[i] * b[i];", 0),
    ("q_reflectors_in_wrong_order", "for (int64_t j = ((n < M) ? n : M) - 1; j >= 0; --j) {",
     "for (int64_t j = 0; j < ((n < M) ? n : M); ++j) {", 0),
    # triangular solves (Sec. 2 Eq. 3, Sec. 2.1)
    ("backsolve_transposed_r", "b[i] -= A[i + j * lda] * xj;", "b[i] -= A[j + i * lda] * xj;", 0),
    ("backsolve_drops_diagonal", "b[j] /= A[j + j * lda];", "b[j] /= 1.0;", 0),
    ("rt_solve_transposed_r", "acc -= A[i + j * lda] * b[i];", "acc -= A[j + i * lda] * b[i];", 0),
    # Siddon lengths (Sec. 2 Eq. 1) and the parallel-beam geometry
    ("pixel_from_segment_start", "double sm = (work[q] + work[q + 1]) * 0.5;", "double sm = work[q];", 0),
    ("pixel_centre_offset", "int ix = (int)floor((xm + h) / w);", "int ix = (int)floor((xm + h) / w + 0.5);", 0),
    ("ray_direction_sign", "double ym = y0 + sm * c;", "double ym = y0 - sm * c;", 0),
    ("pixel_index_transposed", "pix[nseg] = iy * n_side + ix;", "pix[nseg] = ix * n_side + iy;", 0),
    ("view_endpoint_included", "((double)v * arc_deg / (double)n_views) * (M_PI / 180.0);",
     "((double)v * arc_deg / (double)(n_views - 1)) * (M_PI / 180.0);", 0),
    ("bin_centre_offset", "return ((double)d - 0.5 * (double)(n_bins - 1)) * bin_width;",
     "return ((double)d - 0.5 * (double)n_bins) * bin_width;", 0),
    # fan-beam rays (Sec. 3.1 / 3.2 scanner tables)
    ("fan_offset_sign", "out[3 * i + 2] = -(sid * sin(gamma));", "out[3 * i + 2] = sid * sin(gamma);", 0),
    ("fan_angle_sign", "const double theta = (beta + gamma) + 0.5 * M_PI;",
     "const double theta = (beta - gamma) + 0.5 * M_PI;", 0),
    # Joseph's projector (Sec. 3.1)
    ("joseph_weights_swapped", "val[n] = (1.0 - f) * L;", "val[n] = f * L;", 0),
    ("joseph_length_inverted", "const double L = w / (rows ? fabs(c) : fabs(s));",
     "const double L = w * (rows ? fabs(c) : fabs(s));", 0),
    ("joseph_wrong_sampling_axis", "const int rows = fabs(c) >= fabs(s);", "const int rows = fabs(c) < fabs(s);", 0),
    # regularisation rows, forward projection, brute force and certificate
    ("lambda_rows_squared", "A[(m + j) + j * lda] = sqrt_lambda;",
     "A[(m + j) + j * lda] = sqrt_lambda * sqrt_lambda;", 0),
    ("forward_ignores_slice", "acc += val[q] * x[col_idx[q] + s * ldx];", "acc += val[q] * x[col_idx[q]];", 0),
    ("normal_eq_lambda_not_squared", "const long double lam = (long double)sqrt_lambda * (long double)sqrt_lambda;",
     "const long double lam = (long double)sqrt_lambda;", 0),
    ("residual_sign", "acc -= (long double)val[q] * (long double)x[col_idx[q] + s * ldx];",
     "acc += (long double)val[q] * (long double)x[col_idx[q] + s * ldx];", 0),
    ("certificate_drops_lambda_rows", "gs[j] += (long double)sqrt_lambda * rj;", "gs[j] += 0.0L * rj;", 0),
    # more: clipping, norms, spacing, brute force
    ("ray_exit_from_near_side", "s_out = fmin(s_out, fmax(sa, sb));", "s_out = fmin(s_out, fmin(sa, sb));", 1),
    ("norm_drops_head", "double norm = sqrt(alpha * alpha + ss);", "double norm = sqrt(ss);", 0),
    ("rt_solve_drops_diagonal", "b[j] = acc / A[j + j * lda];", "b[j] = acc;", 0),
    ("joseph_fraction_sign", "const double f = fp - fl;", "const double f = fl - fp;", 0),
    ("fan_detector_spacing", "(fan_deg / (double)(n_det - 1))", "(fan_deg / (double)n_det)", 0),
    ("cholesky_drops_square", "d -= G[j + p * n] * G[j + p * n];", "d -= G[j + p * n];", 0),
    ("normal_eq_rhs_slice_zero", "(long double)b[i + s * ldb];", "(long double)b[i];", 0),
]


# Mistakes planted in the oracle's Python layer (oracle/__init__.py): the
# package is copied, patched, and loaded by the pin suites in place of the
# original (the compiled C part is the unmodified one).
PY_MUTANTS = [
    ("certificate_lambda_not_squared", "lam = g.sqrt_lambda ** 2\n    xn", "lam = g.sqrt_lambda\n    xn", 0),
    ("certificate_without_lambda", "np.linalg.norm(gg, axis=0) / lam / np.maximum(xn, 1e-300)",
     "np.linalg.norm(gg, axis=0) / np.maximum(xn, 1e-300)", 0),
    ("rhs_zero_rows_on_top", "Bt[: g.m] = B", "Bt[g.rows - g.m:] = B", 0),
    ("lapack_route_transposed_solve", "lower=0, trans=0", "lower=0, trans=1", 0),
    ("joseph_bin_offset", "t = (d - 0.5 * (g.n_bins - 1)) * g.bin_width",
     "t = (d - 0.5 * g.n_bins) * g.bin_width", 0),
    ("psnr_amplitude_form", "10.0 * math.log10(max_val ** 2 / mse)", "20.0 * math.log10(max_val ** 2 / mse)", 0),
    ("snr_inverted", "10.0 * math.log10(sig / err)", "10.0 * math.log10(err / sig)", 0),
    ("gradient_rt_solve_untransposed", "lower=0, trans=1)", "lower=0, trans=0)", 0),
    ("gradient_q_transposed", 'ormqr("N", full)', 'ormqr("T", full)', 0),
    ("gradient_drops_factor_two", "gx = 2.0 * (X - ", "gx = 1.0 * (X - ", 0),
]


def _plant(text, old, new, occurrence):
    at = -1
    for _ in range(occurrence + 1):
        at = text.find(old, at + 1)
        assert at >= 0, f"mutation site not found: {old!r}"
    return text[:at] + new + text[at + len(old):]


def _build(tmp_path, name, text):
    sys.path.insert(0, ROOT)
    from oracle import build as ob
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return ob.compile_source(str(src), str(tmp_path / f"lib{name}.so"))


def _run_pins(lib, pkg=None):
    env = dict(os.environ, CTQR_ORACLE_LIB=lib)
    if pkg:
        env["CTQR_ORACLE_PKG"] = pkg
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_SUITES],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_pins(tmp_path):
    res = _run_pins(_build(tmp_path, "control", open(SRC).read()))
    assert res.returncode == 0, res.stdout[-2000:]


@pytest.mark.parametrize("name,old,new,occurrence", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new, occurrence):
    text = _plant(open(SRC).read(), old, new, occurrence)
    res = _run_pins(_build(tmp_path, name, text))
    # 1: some pin failed (not a collection or usage error, which would be 2-4)
    assert res.returncode == 1, f"{name} survived the pins:\n{res.stdout[-2000:]}"


@pytest.mark.parametrize("name,old,new,occurrence", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_reject_python_mutant(tmp_path, name, old, new, occurrence):
    sys.path.insert(0, ROOT)
    from oracle import build as ob
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    (pkg / "__init__.py").write_text(_plant(src, old, new, occurrence))
    (pkg / "build.py").write_text(open(os.path.join(ROOT, "oracle", "build.py")).read())
    res = _run_pins(ob.build(), str(pkg))
    assert res.returncode == 1, f"{name} survived the pins:\n{res.stdout[-2000:]}"


def test_unmodified_python_copy_passes_the_pins(tmp_path):
    sys.path.insert(0, ROOT)
    from oracle import build as ob
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    for f in ("__init__.py", "build.py"):
        (pkg / f).write_text(open(os.path.join(ROOT, "oracle", f)).read())
    res = _run_pins(ob.build(), str(pkg))
    assert res.returncode == 0, res.stdout[-2000:]
