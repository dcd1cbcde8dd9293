#!/usr/bin/env python
"""Benchmark of the direct CT reconstruction hot path (arxiv 2412.07631) on B300.

One step = the whole hot path for one batch: build the Siddon system matrix
A~ = [A; sqrt(lambda) I] on the GPU, factor it by blocked Householder QR with
BF16 (default) or TF32 tensor-core trailing updates (FP32 storage), and solve
k noisy sinograms x = R^-1 Q^T b~ with FP64 refinement on the low-precision
factors.

Workload (default): 256 x 256 image (n = 65,536), 360 views x 364 bins
(m = 131,040) + 65,536 regularisation rows (sqrt(lambda) = 0.05), 512
sinograms of seeded 10-ellipse phantoms with Poisson noise at I0 = 5e3.

Reported value: algorithmic TFLOP/s of the step's QR + direct solve over the
device-timed step (build + QR + solve + refinement; refinement flops are not
counted).  The flops are those the method must perform on A~ = [A;
sqrt(lambda) I], whose identity block is untouched below the current column
(see flops_of); the dense-matrix equivalent is reported alongside.  The
line also carries the QR-phase TFLOP/s, the slices/s of the solve phase, the
refinement steps, a certified error bound against the exact least-squares
solution on sampled slices, the roofline of the dominant (tensor-core GEMM)
kernel class, the oracle timed on the host cores, and an end-to-end arm that
passes the sinograms and images through pinned host memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QR TFLOP/s + slices/s at 256², mixed-prec+refine vs FP64, err vs FP64 oracle"
WORKLOADS = {
    # name: (n_side, views, bins, sqrt_lambda, k, I0, ellipses)
    "c3": (256, 360, 364, 0.05, 512, 5e3, 10),
    "c2": (128, 180, 182, 0.05, 64, 1e4, 10),
    "c1": (32, 60, 46, 0.0, 1, None, 8),
    # fan beam, the paper's scanner scaled to 256^2: 360 source positions over
    # 360 degrees, 512 detectors over a 30-degree fan, source at 720 pixels
    # (the fan covers the image's half-diagonal of 181 pixels)
    "fan256": (256, 360, 512, 0.05, 512, 5e3, 10),
    # the 256^2 scan (360 views x 364 bins) over a 64^2 image: panels as tall
    # as the 256^2 workload's (131,072 rows) in a 2.2 GB matrix, for kernel
    # profiles on a small case
    "tall64": (64, 360, 364, 0.05, 64, 5e3, 10),
    # the differentiation workload: the 128^2 geometry, 256 sinograms through
    # the autograd solve layer (bench.py --diff)
    "c4": (128, 180, 182, 0.05, 256, 1e4, 10),
}
FAN = {"fan256": (720.0, 30.0)}  # name: (source_dist, fan_deg)


def geometry_of(ct, name):
    ns, nv, nb, sl = WORKLOADS[name][:4]
    if name in FAN:
        sid, fan = FAN[name]
        return ct.make_geometry(ns, nv, nb, sl, kind="fan", source_dist=sid, fan_deg=fan)
    return ct.make_geometry(ns, nv, nb, sl)


def oracle_geometry_of(O, name):
    ns, nv, nb, sl = WORKLOADS[name][:4]
    if name in FAN:
        sid, fan = FAN[name]
        return O.Geometry(ns, nv, nb, arc_deg=360.0, sqrt_lambda=sl, kind="fan", source_dist=sid, fan_deg=fan)
    return O.Geometry(ns, nv, nb, sqrt_lambda=sl)
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate (fallback only)

# DRAM traffic of the BF16 SM-pair GEMM (gemm_pair_kernel<1>), one ncu launch
# each (dram__bytes_read.sum + dram__bytes_write.sum, 1 pass) on the two
# products of a 256^2 outer-block update at full size, beside the
# algorithmic bytes of the same launch (BF16 operands once, FP32 C read and
# written); profiles/gemm_pair_kernel_bf16_traffic_256x256.md.
BF16_PAIR_TRAFFIC = {
    "TN 2048x16384x131040": {"dram_bytes": 16870233856 + 131341824,
                             "algorithmic_bytes": 2 * (2048 * 131040 + 131040 * 16384) + 2 * 4 * 2048 * 16384},
    "NN 131040x32768x2048": {"dram_bytes": 36604698112 + 17159480320,
                             "algorithmic_bytes": 2 * (131040 * 2048 + 2048 * 32768) + 2 * 4 * 131040 * 32768},
}


def traffic_ratio():
    """DRAM bytes over algorithmic bytes of the captured BF16 update products
    (one TN and one NN product per outer block, summed)."""
    d = sum(v["dram_bytes"] for v in BF16_PAIR_TRAFFIC.values())
    a = sum(v["algorithmic_bytes"] for v in BF16_PAIR_TRAFFIC.values())
    return d / a


def measure_tf32_peaks(torch, n=8192, seconds=4.0):
    """TF32 tensor-core peaks of this GPU, measured the way the BF16 peaks
    beside them were: cuBLAS (torch.matmul with TF32 allowed) on n^3 FP32
    operands, 2 n^3 flops per product; burst = best of 10 single products
    (CUDA events), sustained = products back to back for `seconds`."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        g = torch.Generator(device="cuda").manual_seed(1)
        a = torch.randn((n, n), device="cuda", generator=g)
        b = torch.randn((n, n), device="cuda", generator=g)
        c = torch.empty((n, n), device="cuda")
        for _ in range(3):
            torch.matmul(a, b, out=c)
        best = float("inf")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(10):
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        fl = 2.0 * n ** 3
        reps = max(1, int(seconds * 1e3 / best))
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        sus = fl * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b, c
        return {"tf32_tflops": fl / (best * 1e-3) / 1e12, "tf32_tflops_sustained": sus,
                "how": f"torch.matmul TF32 {n}^3 (2*N^3): best of 10 (burst) and {reps} back to back "
                       f"(sustained), CUDA events, in this run"}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev

# The paper's own timings (Sec. 3.1, the table of residuals and times for
# 2048 simultaneous slices; the machine from the opening of Sec. 3).  Another
# machine, another workload (fan beam, Joseph's projector, no regularisation
# rows, factored out of core): context beside the line, never a target and
# never a ratio.  The rates are derived: QR flops 2 m n^2 - 2/3 n^3 and solve
# flops (4 m n - n^2) per slice over the printed seconds.
PAPER_M, PAPER_N, PAPER_SLICES = 260 * 1025, 512 * 512, 2048
PAPER_TIMES_S = {"fp64": {"qr": 3439.7, "solve": 148.1}, "fp32": {"qr": 2444.9, "solve": 76.1}}


def paper_context():
    m, n, k = PAPER_M, PAPER_N, PAPER_SLICES
    qr_fl = 2.0 * m * n * n - 2.0 / 3.0 * n ** 3
    solve_fl = k * (4.0 * m * n - n * n)
    return {
        "hardware": "1x NVIDIA A100 40 GiB, 2x AMD EPYC 7282 (32 cores), 768 GiB RAM; "
                    "libflame + cuSOLVER + cuBLAS, QR out of core",
        "workload": "512x512 image, fan beam (360 deg, 30 deg fan), 260 views x 1025 detectors, "
                    "Joseph projector: A 266,500 x 262,144, no regularisation rows, 2048 slices",
        "source": "Sec. 3.1, table of residuals and times",
        **{prec: {"qr_s": t["qr"], "solve_s": t["solve"],
                  "qr_tflops_derived": qr_fl / t["qr"] / 1e12,
                  "slices_per_s_derived": k / t["solve"],
                  "solve_tflops_derived": solve_fl / t["solve"] / 1e12}
           for prec, t in PAPER_TIMES_S.items()},
    }


def workload_desc(name):
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[name]
    noise = f"Poisson I0={i0:g}" if i0 else "noiseless"
    if name in FAN:
        sid, fan = FAN[name]
        return (f"{ns}x{ns} fan-beam Siddon, {nv} sources x {nb} detectors over {fan:g} deg, source at "
                f"{sid:g} px" + (f" + sqrt(lambda)={sl} I rows" if sl > 0 else "")
                + f", {k} sinograms of {ne}-ellipse phantoms, {noise}")
    return (f"{ns}x{ns} parallel-beam Siddon, {nv} views x {nb} bins"
            + (f" + sqrt(lambda)={sl} I rows" if sl > 0 else "")
            + f", {k} sinograms of {ne}-ellipse phantoms, {noise}")


def flops_of(ns, nv, nb, sl, k, dense=False):
    """Algorithmic flops of the QR and of k solves.

    With sqrt(lambda) I rows below A, the reflector of column j touches only
    the m - j ray rows below the diagonal and the j + 1 regularisation rows
    m..m+j (the rest of the identity block is untouched until its column is
    reached), so column j costs 4 (m + 1) flops per remaining column and the
    QR costs sum_j 4 (m + 1)(n - j - 1) ~ 2 (m + 1) n^2; a solve costs
    4 (m + 1) n (Q^T) + n^2 (R^-1).  dense=True returns the dense-QR counts
    2 M' n^2 - 2/3 n^3 and 4 M' n - n^2 of an unstructured M' x n matrix."""
    n = ns * ns
    m = nv * nb
    M = m + (n if sl > 0 else 0)
    if dense or sl <= 0:
        qr = 2.0 * M * n * n - 2.0 / 3.0 * n ** 3
        solve = k * (4.0 * M * n - n * n)
    else:
        qr = 4.0 * (m + 1) * (n - 1) * n / 2.0
        solve = k * (4.0 * (m + 1) * n + n * n)
    return M, n, qr, solve


# ---------------------------------------------------------------------------
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
def make_inputs(ct, torch, name, rank=0):
    """Seeded phantoms, GPU forward projection (the library's own FP64 sparse
    product), Poisson noise from the seeded generator.  Untimed."""
    from paper_2412_07631_b300 import synth
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[name]
    from paper_2412_07631_b300 import replicas
    _, first = replicas.rank_slices(rank, int(os.environ.get("WORLD_SIZE", "1")), k, synth.BASE_SEED)
    X = synth.phantom_batch(ns, k, ne, first)
    sysg = ct.System(geometry_of(ct, name), "fp32")
    P = sysg.forward(torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T
    sysg.free()
    del sysg
    B = synth.poisson_sinogram(P, ns, i0, seed=first) if i0 else P
    return X, np.ascontiguousarray(np.asarray(B).T)  # (n x k) phantoms, (k x m) sinograms


NB_OUTER = 0  # 0: the library's default outer block width
SOLVE_PLAN = (0, 0)  # (superblock rows, least split-K depth) of the solve; (0, 0): library defaults
OOC_BUDGET = 0  # > 0: out-of-core path with this device budget (bytes)
DISK_PATH = ""  # out of core with A~ in this file (disk tier) instead of pinned host memory
HOST_CACHE = 0  # pinned block cache of the disk tier (bytes)


def run_step(ct, torch, geom, precision, B, max_iter, tol, host=False, prof=None, out=None):
    """One pass of the hot path.  Returns (X, info, per-phase ms).  With a
    dict `prof`, the library's per-kernel-class accounting is read after the
    factorisation (prof["qr"], build included) and after the solve
    (prof["solve"])."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    if prof is not None:
        ct.stats_reset(True)
    ev[0].record()
    storage = "fp64" if precision == "fp64" else "fp32"
    if OOC_BUDGET > 0 and DISK_PATH:  # out of core, disk tier: A~ in a file + block cache
        sysg = ct.System(geom, storage, disk_path=DISK_PATH, host_cache=HOST_CACHE,
                         block_cols=NB_OUTER)
        ev[1].record()
        F = sysg.factor_ooc(precision, device_budget=OOC_BUDGET)
    elif OOC_BUDGET > 0:  # out of core: host-resident A~, bounded device working set
        sysg = ct.System(geom, storage, host_budget=OOC_BUDGET)
        ev[1].record()
        F = sysg.factor_ooc(precision, device_budget=OOC_BUDGET, nb_outer=NB_OUTER)
    else:
        sysg = ct.System(geom, storage)
        ev[1].record()
        F = sysg.factor(precision, nb_outer=NB_OUTER)
    ev[2].record()
    if prof is not None:
        prof["qr"] = ct.stats_read()
        ct.stats_reset(True)
    F.solve_plan = SOLVE_PLAN
    if host:
        X = F.solve_host(B, out=out, max_iter=max_iter, tol=tol)
    else:
        X = F.solve(B, max_iter=max_iter, tol=tol, allow_noconv=True)
    ev[3].record()
    if prof is not None:
        prof["solve"] = ct.stats_read()
        ct.stats_reset(False)
    info = dict(F.last_info or {})
    F.free()
    sysg.free()
    torch.cuda.synchronize()
    ph = {"build": ev[0].elapsed_time(ev[1]), "qr": ev[1].elapsed_time(ev[2]),
          "solve": ev[2].elapsed_time(ev[3])}
    return X, info, ph


def run_step_kept(ct, torch, geom, precision, B, max_iter, tol):
    """run_step that returns the system and factor as well (untimed uses:
    accuracy figures need the forward projector and further solves)."""
    storage = "fp64" if precision == "fp64" else "fp32"
    if OOC_BUDGET > 0 and DISK_PATH:
        sysg = ct.System(geom, storage, disk_path=DISK_PATH, host_cache=HOST_CACHE, block_cols=NB_OUTER)
        F = sysg.factor_ooc(precision, device_budget=OOC_BUDGET)
    elif OOC_BUDGET > 0:
        sysg = ct.System(geom, storage, host_budget=OOC_BUDGET)
        F = sysg.factor_ooc(precision, device_budget=OOC_BUDGET, nb_outer=NB_OUTER)
    else:
        sysg = ct.System(geom, storage)
        F = sysg.factor(precision, nb_outer=NB_OUTER)
    F.solve_plan = SOLVE_PLAN
    X = F.solve(B, max_iter=max_iter, tol=tol, allow_noconv=True)
    return X, sysg, F


# ---------------------------------------------------------------------------
def cpu_oracle_sample(name, cols=None):
    """The oracle as it stands on a bounded sample of the workload: the plain
    Householder QR of the first `cols` columns of A~ (all M' rows), with the
    reflectors applied to one sinogram and the back-substitution.  Returns
    (TFLOP/s, seconds, description, cores)."""
    import oracle as O
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[name]
    g = oracle_geometry_of(O, name)
    n = g.n
    w = cols or min(n, 512)
    csr = O.siddon_csr(g)
    S = csr.to_scipy()
    A = np.zeros((g.rows, w), order="F")
    A[: g.m] = S[:, :w].toarray()
    if sl > 0:
        A[g.m + np.arange(w), np.arange(w)] = sl
    b = np.zeros((g.rows, 1), order="F")
    b[: g.m, 0] = np.asarray(S[:, :w] @ np.ones(w)).ravel()
    t0 = time.perf_counter()
    VR, tau = O.householder_qr(A)
    C_ = O.apply_qt(VR, tau, b)
    O.backsolve(VR, C_)
    dt = time.perf_counter() - t0
    M = g.rows
    fl = 2.0 * M * w * w - 2.0 / 3.0 * w ** 3 + 4.0 * M * w - w * w
    desc = (f"oracle plain Householder QR of the first {w} of {n} columns of A~ "
            f"({M} x {w}), Q^T applied to one sinogram, back-substitution")
    return fl / dt / 1e12, dt, desc, oracle_threads()


def oracle_certificate(name, Bk, Xk):
    """Largest certified bound ||x - x*|| / ||x*|| over the given slices
    (sinograms Bk, k x m; images Xk, n x k), x* the exact least-squares
    solution of [A; sqrt(lambda) I] x = [b; 0], evaluated by the oracle in
    long double from its own Siddon matrix."""
    import oracle as O
    g = oracle_geometry_of(O, name)
    csr = O.siddon_csr(g)
    cert = O.certificate(g, csr, np.asfortranarray(Bk.T), np.asfortranarray(Xk))
    return float(cert.max())


def oracle_threads():
    """Threads the oracle's OpenMP loops use: OMP_NUM_THREADS if set, else the
    CPUs this process may run on."""
    env = os.environ.get("OMP_NUM_THREADS", "").split(",")[0].strip()
    if env.isdigit() and int(env) > 0:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def workload_config(name):
    """The `config` keys both arms report for a workload."""
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[name]
    M, n, _, _ = flops_of(ns, nv, nb, sl, k)
    return {"workload": workload_desc(name), "n_side": ns, "views": nv, "bins": nb, "rows": M,
            "unknowns": n, "slices": k}


# ---------------------------------------------------------------------------
def gemm_only(args):
    """The GEMM engine on one shape (the trailing-update products in
    isolation): C += op(A) op(B) with random operands, `warmup` untimed and
    `steps` timed calls (CUDA events), one JSON line."""
    import torch
    import paper_2412_07631_b300 as ct
    kind, tr, shape = args.gemm.split(":")
    ta, tb = tr[0], tr[1]
    M, N, K = (int(v) for v in shape.split(","))
    ra, ca = (K, M) if ta == "T" else (M, K)
    rb, cb = (N, K) if tb == "T" else (K, N)
    lda, ldb = -(-ra // 32) * 32, -(-rb // 32) * 32
    dt = torch.float64 if kind == "fp64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.rand((ca, lda), device="cuda", dtype=dt, generator=g)
    B = torch.rand((cb, ldb), device="cuda", dtype=dt, generator=g)
    Cm = torch.rand((N, M), device="cuda", dtype=dt, generator=g)
    for _ in range(args.warmup):
        ct.gemm(kind, ta, tb, M, N, K, -1.0, A, lda, B, ldb, 1.0, Cm, M)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ct.gemm(kind, ta, tb, M, N, K, -1.0, A, lda, B, ldb, 1.0, Cm, M)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    es = 8 if kind == "fp64" else 4
    print(json.dumps({"kernel": "gemm engine", "kind": kind, "trans": tr, "M": M, "N": N, "K": K,
                      "ms": ms, "tflops": 2.0 * M * N * K / ms / 1e9,
                      "algorithmic_bytes": es * (M * K + K * N + 2 * M * N),
                      "steps": args.steps, "warmup": args.warmup}))


# CUDA-core peaks of the FP32 and FP64 paths, whose GEMMs run on the CUDA
# cores: FP32 = 148 SMs x 128 FMA lanes x 2 flops x 2.032 GHz (the maximum SM
# clock); FP64 = the part's nominal dense FP64 rate.
ALU_PEAKS = {"fp32": 148 * 128 * 2 * 2.032e9 / 1e12, "fp64": 1.25}


def roofline_of(prof, precision, peaks, peak_src):
    """The roofline object of a step's dominant kernel class, from the
    per-class CUDA-event timing of a profiled step (`prof` =
    stats_read() after stats_reset(True) and one step): achieved =
    algorithmic flops of all the class's launches / their summed duration.
    The class is the trailing-update GEMMs: BF16-operand tcgen05 GEMMs for
    the BF16 paths (the TF32-operand class beside it as `tf32_class`),
    TF32-operand tcgen05 GEMMs for the TF32 paths, CUDA-core GEMMs for the
    plain FP32 and FP64 paths."""
    def roof(cls, bound, peak, src, kernel):
        t = prof[cls]
        ach = t["flops"] / (t["ms"] * 1e-3) / 1e12 if t["ms"] > 0 else 0.0
        return {"bound": bound, "kernel": f"{kernel} ({cls}, all launches of a step)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak if peak else None,
                "traffic": None, "peak_source": src, "launches_per_step": t["count"], "ms_per_step": t["ms"]}
    if "tf32_tflops_sustained" in peaks:
        tf32_peak = peaks["tf32_tflops_sustained"]
        tf32_src = "measured tf32 sustained (" + peaks.get("tf32_how", "cuBLAS") + ")"
    else:
        tf32_peak = peaks["bf16_tflops_sustained"] * TF32_OVER_BF16
        tf32_src = f"{peak_src} bf16 sustained x nominal TF32/BF16 ratio {TF32_OVER_BF16:.3f}"
    if precision in ("bf16", "bf16x3"):
        r = roof("tc_gemm_bf16", "tensor", peaks["bf16_tflops_sustained"], f"{peak_src} bf16 sustained",
                 "tcgen05 GEMMs")
        t = prof["tc_gemm_bf16"]
        if precision == "bf16" and t["count"]:
            ratio = traffic_ratio()
            r["traffic"] = ratio * t["bytes"] / t["count"]
            r["traffic_basis"] = {"per_launch_algorithmic_bytes": t["bytes"] / t["count"],
                                  "dram_over_algorithmic": ratio, "captures": BF16_PAIR_TRAFFIC,
                                  "how": "ncu DRAM bytes of the two full-size update products, scaled to the "
                                         "class's mean algorithmic bytes per launch"}
        if prof["tc_gemm"]["count"]:
            r["tf32_class"] = roof("tc_gemm", "tensor", tf32_peak, tf32_src, "tcgen05 GEMMs")
        return r
    if precision in ("tf32", "tf32x3"):
        return roof("tc_gemm", "tensor", tf32_peak, tf32_src, "tcgen05 GEMMs")
    src = ("148 SMs x 128 FP32 lanes x 2 flops x 2.032 GHz" if precision == "fp32"
           else "nominal dense FP64 rate of the part")
    return roof("simt_gemm", "alu", ALU_PEAKS[precision], src, "CUDA-core GEMMs")


def quality_of(Xtrue, X):
    """Image quality of reconstructions X against the phantoms Xtrue (both
    n x k), with the equations of Sec. 3.1.3 per slice: MSE over the pixels,
    RMSE, PSNR = 10 log10(MAX^2 / MSE) with MAX = 1 (the phantoms' range) and
    SNR = 10 log10(sum x_true^2 / sum (x_true - x)^2); means over the slices."""
    Xtrue = np.asarray(Xtrue, np.float64)
    X = np.asarray(X, np.float64)
    err = np.sum((X - Xtrue) ** 2, axis=0)
    sig = np.sum(Xtrue ** 2, axis=0)
    mse = err / Xtrue.shape[0]
    with np.errstate(divide="ignore"):
        psnr = 10.0 * np.log10(1.0 / mse)
        snr = 10.0 * np.log10(sig / err)
    return {"rmse_mean": float(np.sqrt(mse).mean()), "psnr_mean": float(psnr.mean()),
            "snr_mean": float(snr.mean())}


def residual_rel(AX, B):
    """The paper's accuracy figure ||A X - B||_F / ||B||_F over the batch
    (Sec. 3.1.2, table of residuals and times): A the ray rows, AX the
    forward projection of the reconstructed images and B the sinograms, both
    k x m."""
    AX = np.asarray(AX, np.float64)
    B = np.asarray(B, np.float64)
    return float(np.linalg.norm(AX - B) / np.linalg.norm(B))


def solve_roofline_of(prof_solve, solve_ms, k, M, n, solve_fl, precision, peaks):
    """Roofline of the solve phase (k slices).  The direct solve
    x = R^-1 Q^T b~ of a batch costs solve_fl flops and must read the factors
    (V and R: M' n elements) once, so its floor is max(flops / tensor peak,
    bytes / HBM peak) (CUDA-core FP64 peak for the FP64 path, FP32 for FP32);
    slices/s at that floor is the roofline the measured slices/s (refinement
    included) is set against.  The solve's own kernel classes beside it:
    its tensor-core GEMMs (Q^T sweep, TRSM, inner correction solves) against
    the TF32 peak, its FP64 and FP32 sparse products against the FP64 and
    FP32 CUDA-core rates."""
    es = 8 if precision == "fp64" else 4
    if precision in ("fp64", "fp32"):
        peak, src = ALU_PEAKS[precision], "CUDA-core peak"
    else:
        peak, src = peaks.get("tf32_tflops_sustained", peaks["bf16_tflops_sustained"] * TF32_OVER_BF16), \
            "tf32 sustained"
    t_flops = solve_fl / (peak * 1e12)
    t_bytes = M * n * es / (peaks["hbm_gbs"] * 1e9)
    floor_s = max(t_flops, t_bytes)
    sps = k / (solve_ms * 1e-3)
    out = {"bound": "tensor" if t_flops >= t_bytes and precision not in ("fp64", "fp32")
           else ("alu" if t_flops >= t_bytes else "hbm"),
           "direct_flops_per_batch": solve_fl, "factor_bytes_per_batch": M * n * es,
           "floor_ms": floor_s * 1e3, "floor_peak": f"{peak:.1f} TFLOP/s ({src}), "
           f"{peaks['hbm_gbs']:.0f} GB/s HBM", "slices_per_s": sps,
           "slices_per_s_roofline": k / floor_s, "frac": sps * floor_s / k,
           "note": "measured time includes the FP64 refinement; the roofline counts the direct solve only"}

    def cls(name, pk):
        t = prof_solve[name]
        if not t["count"] or t["ms"] <= 0:
            return None
        ach = t["flops"] / (t["ms"] * 1e-3) / 1e12
        return {"achieved_tflops": ach, "peak": pk, "frac": ach / pk, "ms": t["ms"],
                "launches": t["count"]}

    tc_peak = peaks.get("tf32_tflops_sustained", peaks["bf16_tflops_sustained"] * TF32_OVER_BF16)
    out["classes"] = {"tc_gemm": cls("tc_gemm", tc_peak),
                      "spmm_fp64": cls("spmm_fp64", ALU_PEAKS["fp64"]),
                      "spmm_fp32": cls("spmm_fp32", ALU_PEAKS["fp32"]),
                      "simt_gemm": cls("simt_gemm", ALU_PEAKS["fp64" if precision == "fp64" else "fp32"])}
    out["classes"] = {c: v for c, v in out["classes"].items() if v}
    return out


def measure_host_link(torch, nbytes=1 << 30):
    """Pinned host <-> device copy rates of this machine (GB/s): best of 5
    copies of nbytes each way, CUDA events."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = float("inf")
        for _ in range(5):
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = nbytes / (best * 1e-3) / 1e9
    out["how"] = f"pinned <-> device copies of {nbytes >> 20} MiB, best of 5, CUDA events"
    return out


def host_link_of(prof_qr, qr_ms, link):
    """Host-link evidence of the out-of-core factorisation, from the copy
    classes of one profiled QR: bytes and achieved GB/s of the V blocks
    streamed on the copy stream, of the superpanel columns loaded and of the
    factored columns written back (both on the compute stream); the compute
    stream's stalls on streamed V blocks, and the overlap = the share of the
    V-streaming time hidden behind compute (1 - stall / streaming time); the
    link floor = all host bytes over the measured pinned copy rates, against
    the QR time."""
    v, c_in, c_out, wait = (prof_qr[c] for c in ("h2d_v", "h2d_cols", "d2h_cols", "copy_wait"))
    if not (v["count"] or c_in["count"]):
        return None

    def one(t):
        return {"gb": t["bytes"] / 1e9, "ms": t["ms"], "copies": t["count"],
                "gbs": t["bytes"] / (t["ms"] * 1e-3) / 1e9 if t["ms"] > 0 else None}

    h2d = v["bytes"] + c_in["bytes"]
    floor_ms = (h2d / (link["h2d_gbs"] * 1e9) + c_out["bytes"] / (link["d2h_gbs"] * 1e9)) * 1e3
    return {"h2d_v": one(v), "h2d_cols": one(c_in), "d2h_cols": one(c_out),
            "copy_wait_ms": wait["ms"],
            "overlap": 1.0 - wait["ms"] / v["ms"] if v["ms"] > 0 else None,
            "link_peak": link, "link_floor_ms": floor_ms, "qr_ms": qr_ms,
            "link_floor_frac_of_qr": floor_ms / qr_ms if qr_ms > 0 else None}


def merge_prof(a, b):
    """Sum of two per-class accounting reads (stats_read())."""
    out = {"launches": a["launches"] + b["launches"]}
    for c, v in a.items():
        if c != "launches":
            out[c] = {f: v[f] + b[c][f] for f in ("ms", "flops", "bytes", "count")}
    return out


def diff_only(args):
    """The differentiation workload: the 128x128 geometry (180 views x 182
    bins + sqrt(lambda) = 0.05 I rows), a batch of 256 noisy sinograms through
    the autograd solve layer (CTSolve): forward X = R^-1 Q^T b~ refined in
    FP64, loss = mean squared error to the phantoms, backward grad_b =
    [Q R^-T grad_x]_{0:m} refined in FP64.  The factorisation is made once,
    untimed (the layer reuses it for every batch of the geometry); `warmup`
    untimed and `steps` timed forward + backward passes, CUDA events on the
    launching stream.  After timing, <grad_b, d> is checked against a
    central difference of the loss along one random unit direction (h =
    1e-3; the loss is quadratic in b).  One JSON line."""
    import torch
    import paper_2412_07631_b300 as ct
    name = "c4"
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[name]
    M, n, _, solve_fl = flops_of(ns, nv, nb, sl, k)
    precision = args.precision
    Xtrue, Bh = make_inputs(ct, torch, name)
    io_dt = torch.float32 if precision == "fp32" else torch.float64
    B = torch.from_numpy(Bh).to(io_dt).cuda()
    Xt = torch.from_numpy(np.ascontiguousarray(Xtrue.T)).to(io_dt).cuda()
    sysg = ct.System(geometry_of(ct, name), "fp64" if precision == "fp64" else "fp32")
    F = sysg.factor(precision, nb_outer=args.nb_outer)
    it, tol = args.max_iter, args.tol

    def step():
        Bv = B.detach().requires_grad_(True)
        Xr = ct.CTSolve.apply(Bv, F, it, tol)
        fwd = dict(F.last_info or {})
        loss = ((Xr - Xt) ** 2).mean()
        loss.backward()
        return loss, Bv.grad, fwd, dict(F.last_info or {})

    for _ in range(args.warmup):
        step()
    ct.stats_reset(False)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = []
    for _ in range(args.steps):
        loss, grad, fwd, bwd = step()
        infos.append((fwd, bwd))
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ct.stats_read()["launches"]
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    with torch.no_grad():
        rng = np.random.default_rng(11)
        d = torch.from_numpy(rng.standard_normal(tuple(B.shape))).to(io_dt).cuda()
        d /= d.norm()
        h = 1e-3
        lp = ((F.solve((B + h * d).contiguous(), max_iter=it, tol=tol) - Xt) ** 2).mean().item()
        lm = ((F.solve((B - h * d).contiguous(), max_iter=it, tol=tol) - Xt) ** 2).mean().item()
        fd = (lp - lm) / (2 * h)
        an = float((grad * d).sum())
    F.free()
    sysg.free()
    print(json.dumps({
        "mode": "differentiation (autograd solve layer, forward + backward)",
        "workload": workload_desc(name), "precision": precision,
        "slices_per_s": k / (ms * 1e-3), "ms_per_step": ms,
        "tflops_direct": 2 * solve_fl / (ms * 1e-3) / 1e12,
        "tflops_note": "algorithmic flops of one direct solve and one direct adjoint per slice "
                       "(refinement not counted)",
        "refine_iters": [[f.get("iterations"), b.get("iterations")] for f, b in infos],
        "refine_inner_iters": [[f.get("inner_iterations"), b.get("inner_iterations")] for f, b in infos],
        "backward_stop_measure": infos[-1][1].get("stop_measure") if infos else None,
        "loss": float(loss.detach()), "fd_check": {"analytic": an, "central_difference": fd,
                                          "rel": abs(fd - an) / max(abs(an), 1e-300)},
        "gpu_launches": launches, "clocks": clk, "steps": args.steps, "warmup": args.warmup}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=list(WORKLOADS))
    ap.add_argument("--precision", default=None,
                    choices=["tf32", "bf16", "tf32x3", "bf16x3", "fp32", "fp64"],
                    help="default: bf16 for the full step, tf32 for --diff")
    ap.add_argument("--max-iter", type=int, default=40)
    ap.add_argument("--tol", type=float, default=5e-7)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cert", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the library's default outer block width and solve plan instead of the ones "
                         "autotune.outer_block and autotune.solve_plan measure on this workload before the "
                         "warm-up (untimed)")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the profiled step, the TF32 peak measurement and the accuracy run "
                         "(for the long FP64 runs at 256^2)")
    ap.add_argument("--nb-outer", type=int, default=0, help="outer WY block width (0: default)")
    ap.add_argument("--ooc-budget-gb", type=float, default=0.0,
                    help="run the out-of-core path: A~ in pinned host memory, this many GB of device working set")
    ap.add_argument("--disk", type=str, default="",
                    help="with --ooc-budget-gb: keep A~ in a file in this directory (disk tier)")
    ap.add_argument("--host-cache-gb", type=float, default=8.0,
                    help="pinned block cache of the disk tier")
    ap.add_argument("--gemm", type=str, default="",
                    help="time only the GEMM engine on one shape, 'KIND:TA TB:M,N,K' (e.g. "
                         "'tf32:TN:768,16384,32768'), beta = 1; for kernel profiling")
    ap.add_argument("--diff", action="store_true",
                    help="time the autograd solve layer (forward + backward) on the 128x128 "
                         "differentiation workload instead of the full step")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "tf32" if args.diff else "bf16"
    if args.gemm:
        return gemm_only(args)
    if args.diff:
        return diff_only(args)
    global NB_OUTER, OOC_BUDGET, DISK_PATH, HOST_CACHE, SOLVE_PLAN
    NB_OUTER = args.nb_outer
    OOC_BUDGET = int(args.ooc_budget_gb * (1 << 30))
    HOST_CACHE = int(args.host_cache_gb * (1 << 30))
    if args.disk:
        if not OOC_BUDGET:
            ap.error("--disk needs --ooc-budget-gb")
        os.makedirs(args.disk, exist_ok=True)
        DISK_PATH = os.path.join(args.disk, "ctqr_rank%s.ctqrd" % os.environ.get("RANK", "0"))

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ns, nv, nb, sl, k, i0, ne = WORKLOADS[args.workload]
    M, n, qr_fl, solve_fl = flops_of(ns, nv, nb, sl, k)

    if args.impl == "reference":
        if rank != 0:
            return
        # The reference arm is the oracle on the host cores, one bounded sample per step.
        for _ in range(args.warmup):
            cpu_oracle_sample(args.workload)
        vals, secs = [], []
        for _ in range(args.steps):
            v, dt, desc, cores = cpu_oracle_sample(args.workload)
            vals.append(v)
            secs.append(dt)
        val = float(np.median(vals))
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload_config(args.workload), precision="fp64 (oracle)",
                               parallelism="host cores"),
                "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2412_07631_b300 as ct
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    peaks, peak_src = load_peaks()

    geom = geometry_of(ct, args.workload)
    Xtrue, Bh = make_inputs(ct, torch, args.workload, rank)
    io_dt = torch.float32 if args.precision == "fp32" else torch.float64
    B = torch.from_numpy(Bh).to(io_dt).cuda()
    Bpin = torch.from_numpy(Bh).to(io_dt).pin_memory()
    # the end-to-end arm's images land in pinned host memory, as its sinograms come from it
    Xpin = torch.empty((Bh.shape[0], n), dtype=io_dt).pin_memory()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # ---- solve plan: autotune.solve_plan on this workload's factor and batch
    #      (untimed; in-core tensor-core factors only) ----
    tune = tune_nb = None
    if not args.no_tune and OOC_BUDGET == 0 and args.precision not in ("fp32", "fp64"):
        from paper_2412_07631_b300 import autotune
        if NB_OUTER == 0:  # the outer block width too, unless given
            NB_OUTER = autotune.outer_block(geom, args.precision, candidates=(2048, 2560, 3072), retune=True)
            tune_nb = dict(autotune.load_cache().get(
                autotune._key(geom, args.precision, torch.cuda.get_device_name()), {}))
        Xt_, sys_t, F_t = run_step_kept(ct, torch, geom, args.precision, B, args.max_iter, args.tol)
        del Xt_
        SOLVE_PLAN = autotune.solve_plan(F_t, B, max_iter=args.max_iter, tol=args.tol, retune=True)
        tune = dict(autotune.load_cache().get(
            autotune._key(geom, args.precision, torch.cuda.get_device_name()) + f"|k{k}|solve", {}))
        F_t.free()
        sys_t.free()

    for _ in range(args.warmup):
        run_step(ct, torch, geom, args.precision, B, args.max_iter, args.tol)

    # ---- timed region (device-resident inputs) ----
    clocks = ClockSampler(local)
    ct.stats_reset(False)
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ct.disk_stats(reset=True)
    e0.record()
    torch.cuda.nvtx.range_push("timed_step")  # lets ncu select the timed launches
    phases, infos = [], []
    for _ in range(args.steps):
        X, info, ph = run_step(ct, torch, geom, args.precision, B, args.max_iter, args.tol)
        phases.append(ph)
        infos.append(info)
    torch.cuda.nvtx.range_pop()
    e1.record()
    barrier()
    clk = clocks.stop()
    launches = ct.stats_read()["launches"]
    disk_io = None
    if DISK_PATH:
        io = ct.disk_stats()
        disk_io = {k: v / args.steps for k, v in io.items()}
        disk_io["read_gbs"] = io["bytes_read"] / io["read_s"] / 1e9 if io["read_s"] else None
        disk_io["write_gbs"] = io["bytes_written"] / io["write_s"] / 1e9 if io["write_s"] else None
        disk_io["note"] = "per timed step; read_s and write_s sum the busy time of the I/O threads"
    ms = e0.elapsed_time(e1) / args.steps
    from paper_2412_07631_b300 import replicas
    ms = replicas.max_over_ranks(ms, dist, device="cuda")
    step_fl = (qr_fl + solve_fl) * world
    value = step_fl / (ms * 1e-3) / 1e12
    qr_ms = float(np.median([p["qr"] for p in phases]))
    solve_ms = float(np.median([p["solve"] for p in phases]))
    build_ms = float(np.median([p["build"] for p in phases]))

    # ---- profiled step (per-kernel-class CUDA events, not part of the timing),
    #      then the TF32 tensor peaks of this GPU (cuBLAS, as the BF16 peaks) ----
    roofline = breakdown = solve_roof = host_link = None
    if not args.no_profile:
        pr = {}
        _, _, pph = run_step(ct, torch, geom, args.precision, B, args.max_iter, args.tol, prof=pr)
        if OOC_BUDGET > 0:
            host_link = host_link_of(pr["qr"], pph["qr"], measure_host_link(torch))
        prof = merge_prof(pr["qr"], pr["solve"])
        tf = measure_tf32_peaks(torch)
        peaks = dict(peaks, tf32_tflops=tf["tf32_tflops"], tf32_tflops_sustained=tf["tf32_tflops_sustained"],
                     tf32_how=tf["how"])
        roofline = roofline_of(prof, args.precision, peaks, peak_src)
        roofline["tf32_peaks_measured"] = tf
        breakdown = {c: {"ms": round(prof[c]["ms"], 3), "count": prof[c]["count"]}
                     for c in ct.STAT_CLASSES if prof[c]["count"]}
        solve_roof = solve_roofline_of(pr["solve"], solve_ms, k, M, n, solve_fl, args.precision, peaks)

    # ---- end-to-end arm: pinned host sinograms in, host images out ----
    e2e = None
    if not args.no_e2e:
        for _ in range(1):
            run_step(ct, torch, geom, args.precision, Bpin, args.max_iter, args.tol, host=True, out=Xpin)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Xh, _, _ = run_step(ct, torch, geom, args.precision, Bpin, args.max_iter, args.tol,
                                host=True, out=Xpin)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        es = 4 if args.precision == "fp32" else 8
        e2e = {"value": step_fl / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(k * (M - (n if sl > 0 else 0)) * es),
               "d2h_bytes_per_step": int(k * n * es), "ms_per_step": e2e_ms,
               "api": "ct_build_system + ct_qr_factor + ct_solve_host"}

    # ---- accuracy (untimed): quality vs phantom (Sec. 3.1.3), the paper's
    #      residual ||AX - B|| / ||B|| (Sec. 3.1.2), for the noisy sinograms of
    #      the step and for noiseless sinograms of the same phantoms (the
    #      setting of the paper's quality tables); the error vs the oracle is
    #      part of the oracle leg below ----
    Xn = X.double().cpu().numpy().T
    q = quality_of(Xtrue, Xn)
    acc = {"rmse_vs_phantom_mean": q["rmse_mean"], "psnr_vs_phantom_mean": q["psnr_mean"],
           "snr_mean": q["snr_mean"]}
    if not args.no_profile:
        Xa, sysa, Fa = run_step_kept(ct, torch, geom, args.precision, B, args.max_iter, args.tol)
        acc["residual_rel"] = residual_rel(sysa.forward(Xa.double()).cpu().numpy(), Bh)
        Xt_dev = torch.from_numpy(np.ascontiguousarray(Xtrue.T)).cuda()
        P0 = sysa.forward(Xt_dev)
        X0 = Fa.solve(P0.to(io_dt).contiguous(), max_iter=args.max_iter, tol=args.tol, allow_noconv=True)
        q0 = quality_of(Xtrue, X0.double().cpu().numpy().T)
        acc["noiseless"] = {**q0, "residual_rel": residual_rel(sysa.forward(X0.double()).cpu().numpy(),
                                                               P0.cpu().numpy()),
                            "note": "the same phantoms, sinograms A x_true without noise"}
        acc["residual_note"] = ("noisy data: the residual holds the noise, which no image removes; "
                                "A is the ray rows only (the regularisation rows excluded)")
        Fa.free()
        sysa.free()
        del Xa, X0, P0, Xt_dev

    # ---- FP64 GPU path vs mixed path, measured on the 128x128 geometry and
    #      extrapolated to this workload by the flop ratio (FP64 at 256^2 takes
    #      about half an hour at the FP64 rate of this part: bench.py
    #      --precision fp64 --steps 1 --warmup 0 --no-profile measures it) ----
    cmp = None
    if rank == 0 and not args.no_fp64_compare and args.workload == "c3":
        cns, cnv, cnb, csl, ck, ci0, cne = WORKLOADS["c2"]
        cM, cn, cqr, csolve = flops_of(cns, cnv, cnb, csl, ck)
        cg = ct.make_geometry(cns, cnv, cnb, csl)
        _, cB = make_inputs(ct, torch, "c2")
        cmp = {"workload": workload_desc("c2")}
        mixed = args.precision if args.precision not in ("fp64", "fp32") else "tf32"
        # the tuned blocking belongs to the main workload
        plan_c3, SOLVE_PLAN = SOLVE_PLAN, (0, 0)
        nb_c3, NB_OUTER = NB_OUTER, args.nb_outer
        for prec in ("fp64", mixed):
            Bd = torch.from_numpy(cB).double().cuda()
            run_step(ct, torch, cg, prec, Bd, args.max_iter, args.tol) if prec == mixed else None
            _, inf, ph = run_step(ct, torch, cg, prec, Bd, args.max_iter, args.tol)
            cmp[prec] = {"qr_tflops": cqr / (ph["qr"] * 1e-3) / 1e12,
                         "slices_per_s": ck / (ph["solve"] * 1e-3),
                         "refine_iters": inf.get("iterations", 0),
                         "inner_iters": inf.get("inner_iterations", 0)}
        SOLVE_PLAN, NB_OUTER = plan_c3, nb_c3
        # the FP64 path at this workload: its 128^2 QR rate over this
        # workload's QR flops, its 128^2 per-slice solve time scaled by the
        # per-slice flop ratio
        per_slice = solve_fl / k
        c_per_slice = csolve / ck
        f64 = cmp["fp64"]
        cmp["this_workload"] = {
            "workload": workload_desc(args.workload),
            "fp64": {"qr_tflops": f64["qr_tflops"], "qr_s": qr_fl / (f64["qr_tflops"] * 1e12),
                     "slices_per_s": f64["slices_per_s"] * c_per_slice / per_slice,
                     "extrapolated": True,
                     "how": "128x128 FP64 rates measured above, scaled by the QR and per-slice solve flop ratios"},
            args.precision: {"qr_tflops": qr_fl / (qr_ms * 1e-3) / 1e12, "qr_s": qr_ms * 1e-3,
                             "slices_per_s": k / (solve_ms * 1e-3), "extrapolated": False}}

    # ---- the oracle leg (rank 0, after every GPU measurement): the oracle
    #      timed on the host cores, and the certified error bound of sampled
    #      GPU slices against the exact least-squares solution, evaluated by
    #      the oracle from its own FP64 Siddon matrix ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, desc, cores = cpu_oracle_sample(args.workload)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": dt}
        if not args.no_cert and sl > 0:
            pick = np.linspace(0, k - 1, min(k, 4)).astype(int)
            acc["cert_bound_max"] = oracle_certificate(args.workload, Bh[pick], Xn[:, pick])
            acc["cert_slices"] = [int(p) for p in pick]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32": "tf32 (FP32 storage) + f64 refinement",
                      "bf16": "bf16 trailing updates (FP32 storage, tf32 solve) + f64 refinement",
                      "tf32x3": "tf32x3 split trailing updates (FP32 storage, tf32 solve) + f64 refinement",
                      "bf16x3": "bf16x3 split trailing updates (FP32 storage, tf32 solve) + f64 refinement",
                      "fp32": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {**workload_config(args.workload),
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "out_of_core": ({"device_budget_gb": args.ooc_budget_gb,
                                        "host_matrix": (("file on local disk + %.0f GB pinned block cache"
                                                         % args.host_cache_gb) if DISK_PATH
                                                        else "pinned host memory")}
                                       if OOC_BUDGET else None),
                       "l2": "inputs larger than L2 (dense A~ of %.1f GB rebuilt every step)"
                             % (M * n * 4 / 1e9),
                       "solve_plan": {"solve_block": SOLVE_PLAN[0], "solve_split": SOLVE_PLAN[1],
                                      "tuned": tune},
                       "nb_outer": {"value": NB_OUTER or "library default", "tuned": tune_nb}},
            "qr_tflops": qr_fl / (qr_ms * 1e-3) / 1e12,
            "qr_tflops_dense_equivalent": flops_of(ns, nv, nb, sl, k, dense=True)[2] / (qr_ms * 1e-3) / 1e12,
            "slices_per_s": k / (solve_ms * 1e-3),
            "phases_ms": {"build": build_ms, "qr": qr_ms, "solve_refine": solve_ms},
            "refine_iters": [i.get("iterations") for i in infos],
            "refine_inner_iters": [i.get("inner_iterations") for i in infos],
            "accuracy": acc,
            "roofline": roofline,
            "solve_roofline": solve_roof,
            "kernel_breakdown_ms": breakdown,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "fp64_vs_mixed": cmp,
            "paper_context": paper_context(),
            "disk_io": disk_io,
            "host_link": host_link,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
