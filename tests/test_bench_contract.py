"""bench.py's host-side contract, on the CPU: the reference arm (the oracle
timed on the host cores, one bounded sample of the 256x256 workload per
step) prints one JSON line with the keys the benchmark contract asks for,
on the same metric, unit and workload as the GPU arm; ranks other than 0
print nothing; the flop counts follow their closed forms."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(*args, env=None):
    e = dict(os.environ, **(env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    res = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "TFLOP/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.workload_desc("c3")
    assert {k: d["config"][k] for k in ("n_side", "views", "bins", "rows", "unknowns", "slices")} == \
        {"n_side": 256, "views": 360, "bins": 364, "rows": 196576, "unknowns": 65536, "slices": 512}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    res = _run("--impl", "reference", "--steps", "1", "--warmup", "0",
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip() == ""


def test_oracle_threads_follow_omp_num_threads(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.oracle_threads() == 3
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.oracle_threads() >= 1


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_flop_counts(name):
    ns, nv, nb, sl, k, _, _ = bench.WORKLOADS[name]
    n, m = ns * ns, nv * nb
    M, n2, qr_d, solve_d = bench.flops_of(ns, nv, nb, sl, k, dense=True)
    assert (M, n2) == (m + (n if sl > 0 else 0), n)
    assert qr_d == pytest.approx(2.0 * M * n * n - 2.0 / 3.0 * n ** 3, rel=1e-12)
    assert solve_d == pytest.approx(k * (4.0 * M * n - n * n), rel=1e-12)
    _, _, qr_s, solve_s = bench.flops_of(ns, nv, nb, sl, k)
    if sl > 0:
        # column j's reflector spans the m - j ray rows below the diagonal and
        # the j + 1 regularisation rows filled so far: 4 (m + 1) flops per
        # remaining column, summed over j
        assert qr_s == pytest.approx(sum(4.0 * (m + 1) * (n - j - 1) for j in range(n)), rel=1e-12)
        assert qr_s < qr_d
    else:
        assert (qr_s, solve_s) == (qr_d, solve_d)


def test_oracle_certificate_bounds_the_error(monkeypatch):
    """The bench's error-vs-oracle figure on a small geometry: it is tiny for
    the oracle's own least-squares solution, and it bounds the true error of
    a perturbed solution."""
    import numpy as np
    import oracle as O
    monkeypatch.setitem(bench.WORKLOADS, "t12", (12, 20, 18, 0.05, 3, None, 4))
    g = bench.oracle_geometry_of(O, "t12")
    csr = O.siddon_csr(g)
    rng = np.random.default_rng(3)
    B = rng.random((g.m, 3))
    Xs, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    assert bench.oracle_certificate("t12", B.T, Xs) <= 1e-10
    # the bound is ||A~^T A~ e|| / (lambda ||x||): at least the error, at most
    # sigma_max^2 / lambda times it, and linear in the perturbation e
    E = rng.standard_normal(Xs.shape)
    Xp = Xs + 1e-3 * E
    err = np.linalg.norm(Xp - Xs, axis=0) / np.linalg.norm(Xp, axis=0)
    bound = bench.oracle_certificate("t12", B.T, Xp)
    assert err.max() <= bound
    Xq = Xs + 1e-5 * E
    assert bench.oracle_certificate("t12", B.T, Xq) == pytest.approx(bound / 100, rel=2e-2)


def test_paper_context_rates():
    """The paper's printed seconds (Sec. 3.1, 512^2, 2048 slices) turned into
    rates: 2.46e16 QR flops in 3439.7 s (FP64) and 2444.9 s (FP32); 2048
    slices in 148.1 s and 76.1 s."""
    pc = bench.paper_context()
    assert pc["fp64"]["qr_tflops_derived"] == pytest.approx(7.157, rel=1e-3)
    assert pc["fp32"]["qr_tflops_derived"] == pytest.approx(10.069, rel=1e-3)
    assert pc["fp64"]["slices_per_s_derived"] == pytest.approx(13.83, rel=1e-3)
    assert pc["fp32"]["slices_per_s_derived"] == pytest.approx(26.91, rel=1e-3)
    assert pc["fp32"]["solve_tflops_derived"] == pytest.approx(5.67, rel=2e-3)


def _prof(**cls):
    import paper_2412_07631_b300 as ct
    out = {c: {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "count": 0} for c in ct.STAT_CLASSES}
    for c, (ms, fl, n) in cls.items():
        out[c] = {"ms": ms, "flops": fl, "bytes": 0.0, "count": n}
    return out


def test_roofline_arithmetic():
    """achieved = class flops / class time, frac = achieved / peak; the class
    and the peak follow the precision (BF16 sustained for the BF16 paths,
    BF16 sustained x 1.1/2.25 for TF32, CUDA-core peaks for FP32/FP64)."""
    peaks = {"bf16_tflops_sustained": 1357.3}
    prof = _prof(tc_gemm_bf16=(1000.0, 1.2e15, 4000), tc_gemm=(500.0, 2.0e14, 900),
                 simt_gemm=(100.0, 5.0e12, 50))
    r = bench.roofline_of(prof, "bf16", peaks, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["launches_per_step"] == 4000
    assert r["achieved"] == pytest.approx(1200.0) and r["peak"] == 1357.3
    assert r["frac"] == pytest.approx(1200.0 / 1357.3)
    assert r["tf32_class"]["achieved"] == pytest.approx(400.0)
    assert r["tf32_class"]["peak"] == pytest.approx(1357.3 * 1.1 / 2.25)
    r = bench.roofline_of(prof, "tf32", peaks, "measured")
    assert r["achieved"] == pytest.approx(400.0) and "tf32_class" not in r
    r = bench.roofline_of(prof, "fp32", peaks, "measured")
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(50.0)
    assert r["peak"] == pytest.approx(148 * 128 * 2 * 2.032e9 / 1e12)
    assert bench.roofline_of(prof, "fp64", peaks, "measured")["peak"] == 1.25


def test_roofline_uses_measured_tf32_peak():
    peaks = {"bf16_tflops_sustained": 1357.3, "tf32_tflops_sustained": 740.0, "tf32_how": "test"}
    prof = _prof(tc_gemm=(500.0, 2.0e14, 900))
    r = bench.roofline_of(prof, "tf32", peaks, "measured")
    assert r["peak"] == 740.0 and r["frac"] == pytest.approx(400.0 / 740.0)
    assert "measured tf32" in r["peak_source"]


def test_accuracy_figures_against_the_oracle(oracle_mod):
    """The line's accuracy figures on a small case: the residual
    ||A X - B||_F / ||B||_F equals the one formed with the oracle's dense A
    (ray rows), and the per-slice SNR, RMSE and PSNR equal the oracle's
    quality() (Sec. 3.1.3 equations) averaged over the slices."""
    import numpy as np
    from paper_2412_07631_b300 import synth
    O = oracle_mod
    g = O.Geometry(10, 16, 15, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    Xt = synth.phantom_batch(10, 3, 8)
    B = synth.poisson_sinogram(O.forward(csr, Xt), 10, 1e4, seed=5)
    X, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    A = O.dense_system(g, csr)[: g.m]
    want = np.linalg.norm(A @ X - B) / np.linalg.norm(B)
    got = bench.residual_rel(O.forward(csr, X).T, B.T)
    assert got == pytest.approx(want, rel=1e-12)
    q = bench.quality_of(Xt, X)
    per = [O.quality(Xt[:, s], X[:, s]) for s in range(3)]
    assert q["snr_mean"] == pytest.approx(np.mean([p["snr"] for p in per]), rel=1e-12)
    assert q["rmse_mean"] == pytest.approx(np.mean([p["rmse"] for p in per]), rel=1e-12)
    assert q["psnr_mean"] == pytest.approx(np.mean([p["psnr"] for p in per]), rel=1e-12)
    # consistent data: the residual of the exact least-squares image of
    # noiseless sinograms is the lambda bias alone, far below the noisy one
    P = O.forward(csr, Xt)
    X0, _, _ = O.qr_solve(g, O.dense_system(g, csr), P)
    assert bench.residual_rel(O.forward(csr, X0).T, P.T) < 0.1 * got


def test_solve_roofline_arithmetic():
    """floor = max(direct-solve flops / tensor peak, factor bytes / HBM
    peak); frac = measured slices/s over k / floor."""
    peaks = {"bf16_tflops_sustained": 1357.3, "tf32_tflops_sustained": 700.0, "hbm_gbs": 6500.0}
    prof = _prof(tc_gemm=(300.0, 1.5e14, 100), spmm_fp64=(250.0, 3.0e11, 10))
    ns, nv, nb, sl, k, _, _ = bench.WORKLOADS["c3"]
    M, n, _, solve_fl = bench.flops_of(ns, nv, nb, sl, k)
    r = bench.solve_roofline_of(prof, 900.0, k, M, n, solve_fl, "bf16", peaks)
    floor = max(solve_fl / 700e12, M * n * 4 / 6500e9)
    assert r["bound"] == "tensor" and r["floor_ms"] == pytest.approx(floor * 1e3)
    assert r["frac"] == pytest.approx((k / 0.9) / (k / floor))
    assert r["classes"]["tc_gemm"]["achieved_tflops"] == pytest.approx(500.0)
    assert r["classes"]["spmm_fp64"]["frac"] == pytest.approx(1.2 / 1.25)
    r = bench.solve_roofline_of(prof, 900.0, k, M, n, solve_fl, "fp64", peaks)
    assert r["bound"] == "alu" and r["floor_ms"] == pytest.approx(solve_fl / 1.25e12 * 1e3)


def test_host_link_arithmetic():
    """Out-of-core copy evidence: GB/s per copy class, overlap = 1 - stall /
    streaming time, link floor = bytes over the measured copy rates."""
    prof = _prof(h2d_v=(400.0, 0.0, 20), h2d_cols=(100.0, 0.0, 2), d2h_cols=(120.0, 0.0, 2),
                 copy_wait=(40.0, 0.0, 20))
    prof["h2d_v"]["bytes"], prof["h2d_cols"]["bytes"], prof["d2h_cols"]["bytes"] = 20e9, 5e9, 5e9
    link = {"h2d_gbs": 50.0, "d2h_gbs": 25.0}
    r = bench.host_link_of(prof, 2000.0, link)
    assert r["h2d_v"]["gbs"] == pytest.approx(50.0) and r["d2h_cols"]["gbs"] == pytest.approx(5e9 / 0.12 / 1e9)
    assert r["overlap"] == pytest.approx(0.9)
    assert r["link_floor_ms"] == pytest.approx((25e9 / 50e9 + 5e9 / 25e9) * 1e3)
    assert r["link_floor_frac_of_qr"] == pytest.approx(700.0 / 2000.0)
    assert bench.host_link_of(_prof(), 1.0, link) is None


def test_traffic_of_the_bf16_class():
    """roofline.traffic = the captured DRAM/algorithmic ratio times the class's
    mean algorithmic bytes per launch."""
    peaks = {"bf16_tflops_sustained": 1401.4}
    prof = _prof(tc_gemm_bf16=(800.0, 1.1e15, 4000))
    prof["tc_gemm_bf16"]["bytes"] = 4000 * 2.0e9
    r = bench.roofline_of(prof, "bf16", peaks, "measured")
    ratio = bench.traffic_ratio()
    assert 1.0 < ratio < 4.0
    assert r["traffic"] == pytest.approx(ratio * 2.0e9)
    assert bench.roofline_of(prof, "tf32", peaks, "measured")["traffic"] is None
