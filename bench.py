#!/usr/bin/env python3
"""Benchmark of ADMM-TV laminography on B300: seconds per ADMM-TV iteration
(FP32, 4 CG steps per iteration, L-hat / L-hat^H in the Algorithm 2 form) and
the L-hat + L-hat^H bandwidth against the HBM roofline, at 1024^3.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (``large``): volume 1024 x 1024 x 1024 FP32, 1024 angles uniform on
[0, 2 pi), detector 1024 x 1024, tilt phi = 30 deg, seeded ellipsoid +
thin-layer circuit phantom, data = L u + 1 % Gaussian noise, alpha = 1e-3,
rho = 0.5 (adaptive), oversampling 2, Gaussian half-width 4.  A step is one
outer ADMM-TV iteration (LSP with 4 CG steps, RSP, multiplier and penalty
updates) replayed as a CUDA graph.  All inputs are synthetic; working sets are
tens of GB, far larger than L2, so no explicit L2 flush is needed.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one kv plane of the 2D stage, four x-slabs of the z stage) and
scales it to seconds per iteration.  Under torchrun (N > 1) every rank runs an
independent replica (weak scaling, no data-path collective); only the timing
is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALPHA, RHO, N_INNER, PHI_DEG = 1e-3, 0.5, 4, 30.0
EXACT_CENTRE_JOBS = 3  # the library's FP32 default (LAM_OPT_EXACT_CENTRE_JOBS)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=1024, help="n = nz = h = w = n_theta")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--iters", type=int, default=32, help="--op precision: ADMM-TV iterations compared")
    ap.add_argument("--spread", default=None, help="adjoint spread variant of the FP32 plans (library default if unset)")
    ap.add_argument("--taus", default="0.86,0.90,0.92,0.94,0.96", help="--op memo: thresholds")
    ap.add_argument("--op", choices=["admm", "lhat_pair", "batch", "ablation", "precision", "fbp", "memo"],
                    default="admm",
                    help="lhat_pair: time only L-hat + L-hat^H on the workload (no ADMM state); "
                         "a small footprint for profiling.  batch: the batching workload (16 "
                         "reconstructions of uneven sizes, batched operators, graph-captured ADMM).  "
                         "ablation: the plain LSP form (Algorithm 1) against the cancelled and fused "
                         "form (Algorithm 2) on the workload.  precision: FP32 (graph) against the plain FP64 "
                         "GPU path over --iters ADMM-TV iterations on the workload (relative L2 of u at "
                         "iterations 1, 2, 4, ..., s/iter of both).  fbp: the FBP-style single pass "
                         "(L^H of ramp-filtered data) on the workload: seconds per pass, voxels/s.  memo: "
                         "ADMM-TV with F*_u2D memoized per plane job at each of --taus against the run "
                         "without (accuracy error E of Section 6.1, reused jobs, s/iter)")
    return ap.parse_args()


def workload_name(n):
    return (f"large: ADMM-TV {n}^3 FP32, {n} angles on [0,2pi), detector {n}x{n}, phi=30deg, "
            f"ellipsoid+circuit phantom, 1% noise, alpha=1e-3, rho=0.5 adaptive, 4 CG steps/iter")


# ---------------------------------------------------------------------------
# algorithmic traffic (stage-boundary tensors; f32 volume, c64 spectra)
# ---------------------------------------------------------------------------

def lhat_bytes(n, nz, h, w, T):
    """L-hat: read u (4 B/voxel), write + read u1 (8 B per (x, kv, y) point
    each) for the h/2 + 1 kv planes a real volume needs (the others are the
    conjugate mirrors), write d_hat (8 B per T h w point).  L-hat^H moves the
    same bytes."""
    return 4 * n * n * nz + 16 * n * n * (h // 2 + 1) + 8 * T * h * w


# ---------------------------------------------------------------------------
# multi-rank timing (replicas: no data-path collective; only the clock is reduced)
# ---------------------------------------------------------------------------

def _strip_comments(src: str) -> str:
    """C/C++ source without // and /* */ comments (string literals in these
    files hold no comment markers), whitespace runs collapsed to one space."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return re.sub(r"\s+", " ", src).strip()


def full_source_hash():
    """SHA-256 of the code (comments stripped) of every CUDA source of the
    library (csrc/*.cu, *.cuh, *.h, sorted): ties a stored FP32-vs-FP64
    trajectory record to the code it was measured on."""
    import hashlib
    d = os.path.join(ROOT, "paper_2511_01893_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(d, f), encoding="utf-8") as fh:
                h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()


def source_hash():
    """SHA-256 of the code (comments stripped) of the sources the L-hat /
    L-hat^H stage kernels are built from (csrc/common.cuh, fft.cuh,
    kernels.h, usfft1d.cu, usfft2d.cu, in that order): ties a stored
    DRAM-traffic figure of those kernels to the code it was measured on."""
    import hashlib
    d = os.path.join(ROOT, "paper_2511_01893_b300", "csrc")
    h = hashlib.sha256()
    for f in ("common.cuh", "fft.cuh", "kernels.h", "usfft1d.cu", "usfft2d.cu"):
        h.update(f.encode())
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()


def admm_iteration_bytes(n, nz, h, w, T, n_inner=N_INNER):
    """Algorithmic HBM bytes of one ADMM-TV outer iteration (Algorithm 2 form):
    per CG step one L-hat^H and one L-hat (lhat_bytes each), the LSP gradient
    (reads L-hat^H r, e, lambda, writes G: 32 B/voxel; from the second step
    also du, p, G_prev: +12), the direction update (12 B/voxel), ||grad p||^2
    (4), u / du update (8, +4 from the second step, +8 on the last step for u),
    ||L-hat p||^2 (8 B per data point) and r += gamma L-hat p (24 B per data
    point); then the RSP (reads u, du, e, lambda, writes e, lambda, dpsi: 68
    B/voxel) and ||div dpsi||^2 (12).  Stencil neighbours count once."""
    K, D = n * n * nz, T * h * w
    vox = 0
    for k in range(n_inner):
        later = 12 if k > 0 else 0
        vox += 32 + later + 12 + 4 + 8 + (4 if k > 0 else 0) + (8 if k == n_inner - 1 else 0)
    vox += 68 + 12
    return n_inner * 2 * lhat_bytes(n, nz, h, w, T) + K * vox + D * n_inner * (8 + 24)


# the kernel each adjoint spread variant launches for the non-centre plane jobs
SPREAD_KERNELS = {"tiles": "k_spread2d_tiles", "sweep": "k_spread2d_sweep", "tiles2": "k_spread2d_tiles2",
                  "tiles_exact": "k_spread2d_tiles_exact", "halo": "k_spread2d_halo", "atomic": "k_scatter2d_atomic",
                  "exact": "k_scatter2d_atomic"}


def spread_point_flops(m=4):
    """Algorithmic FP32 flops the adjoint spread spends per slice point: its
    (2m)^2 cells, each a complex accumulation of a real weight times the value
    (4 flops), and the 4m Gaussian weight exponentials (counted as 1 each)."""
    return (2 * m) ** 2 * 4 + 4 * m


def lhat_flops(n, nz, h, w, T, m=4):
    """Algorithmic FP32 flops of one L-hat (5 N log2 N per complex FFT of
    length N): the z stage's n^2 FFTs of length 2 nz; per kv plane n row FFTs
    and 2n column FFTs of length 2n (zero rows pruned); the 2D gather's
    (2m)^2 taps x 4 flops + 4m weight exponentials per slice point; the 1D
    gather's 2m taps x 4 flops per (x, kv, y).  L-hat^H has the same count."""
    M0, M = 2 * nz, 2 * n
    z = n * n * 5 * M0 * np.log2(M0)
    planes = h * (n + M) * 5 * M * np.log2(M)
    g2 = T * h * w * ((2 * m) ** 2 * 4 + 4 * m)
    g1 = n * n * h * 2 * m * 4
    return float(z + planes + g2 + g1)


def plane_fft_comparator(plan, glam, dev, stream, reps=3):
    """The forward's plane FFTs (ours: deapodise, pad, pruned row FFTs, column
    FFTs) against torch.fft.fft2 (cuFFT) on the same number of zero-padded
    2n x 2n planes; cuFFT is a comparator only, never on the path."""
    import torch
    n = plan.n
    nb = min(32, plan.info()["planes_per_batch"], plan.h)
    u1 = torch.randn((nb, n, n), dtype=torch.complex64, device=dev)
    P = torch.empty((nb, 2 * n, 2 * n), dtype=torch.complex64, device=dev)
    Pin = torch.zeros((nb, 2 * n, 2 * n), dtype=torch.complex64, device=dev)
    Pin[:, n // 2:n // 2 + n, n // 2:n // 2 + n] = u1
    times = {"ours": [], "cufft": []}
    with torch.cuda.stream(stream):
        for r in range(reps + 1):
            for kind in ("ours", "cufft"):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if kind == "ours":
                    plan.plane_ffts(u1, P)
                else:
                    torch.fft.fft2(Pin)
                e1.record(stream)
                stream.synchronize()
                if r:
                    times[kind].append(e0.elapsed_time(e1) / 1e3 / nb)
    return {"planes": nb, "ours_s_per_plane": statistics.median(times["ours"]),
            "cufft_fft2_s_per_plane": statistics.median(times["cufft"]),
            "note": "ours prunes the n zero rows and folds deapodisation; cuFFT does the full padded 2D FFT"}


def job_seconds_per_iter(t_local, steps, world, device=None):
    """Seconds per ADMM iteration of a job of `world` independent replicas,
    each running `steps` iterations of its own problem: the slowest rank's
    time over `steps` (a replica's iteration does not get shorter because
    other GPUs run theirs).  Returns (s/iter, slowest time, aggregate
    iterations per second over all replicas = world * steps / slowest time)."""
    import torch
    import torch.distributed as dist
    t = float(t_local)
    if world > 1:
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = tt.item()
    return t / steps, t, world * steps / t


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clock, power and clock-event reasons every 200 ms through
    NVML (read-only queries) while the timed region runs."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, gpu_index, period=0.2):
        self.gpu, self.period = gpu_index, period
        self.samples = []
        self.errors = []
        self._stop = None

    def _run(self):
        import pynvml
        h = pynvml.nvmlDeviceGetHandleByIndex(self.gpu)
        mx = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)
        while not self._stop.is_set():
            try:
                sm = pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)
                try:
                    rs = pynvml.nvmlDeviceGetCurrentClocksEventReasons(h)
                except AttributeError:
                    rs = pynvml.nvmlDeviceGetCurrentClocksThrottleReasons(h)
                pw = pynvml.nvmlDeviceGetPowerUsage(h) / 1000.0
                self.samples.append((sm, mx, rs, pw))
            except Exception as ex:
                self.errors.append(repr(ex))
            self._stop.wait(self.period)

    def __enter__(self):
        import threading
        self._smi = None
        try:
            import pynvml
            pynvml.nvmlInit()
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            if vis and vis.split(",")[0].strip().isdigit():
                self.gpu = int(vis.split(",")[self.gpu].strip())
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        except Exception:
            # no NVML bindings: nvidia-smi writes samples to a file
            import subprocess
            import tempfile
            self._stop = None
            self._file = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False).name
            q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap")
            try:
                self._smi = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                              "--format=csv,noheader,nounits", "-lms", str(int(self.period * 1000)),
                                              "-f", self._file], stdout=subprocess.DEVNULL,
                                             stderr=subprocess.DEVNULL)
            except OSError as ex:
                self.errors.append(repr(ex))
        return self

    def __exit__(self, *exc):
        if self._stop is not None:
            self._stop.set()
            self._t.join(timeout=2)
        if self._smi is not None:
            self._smi.terminate()
            try:
                self._smi.wait(timeout=5)
            except Exception:
                self._smi.kill()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            bits = [self.REASONS[k] for k in names]
            try:
                for line in open(self._file):
                    f = [x.strip() for x in line.split(",")]
                    if len(f) < 7:
                        continue
                    try:
                        sm, mx, pw = float(f[0]), float(f[1]), float(f[2])
                    except ValueError:
                        continue
                    rs = sum(b for b, v in zip(bits, f[3:7]) if v.lower() == "active")
                    self.samples.append((sm, mx, rs, pw))
                os.unlink(self._file)
            except OSError as ex:
                self.errors.append(repr(ex))

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "errors": self.errors[:3]}
        reasons = sorted({k for s in self.samples for k, bit in self.REASONS.items() if s[2] & bit})
        return {"sm_mhz": statistics.median(s[0] for s in self.samples), "sm_max_mhz": max(s[1] for s in self.samples),
                "power_w_max": max(s[3] for s in self.samples), "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
#
# The FP64 oracle runs as it stands, one NumPy thread per worker process and
# one worker per host core (a spawn pool: no fork after CUDA).  The work of one
# ADMM-TV iteration at n^3 splits into independent units (kv planes of the 2D
# stage, x-slabs of the z stage, x-slabs of the elementwise TV steps), so a
# sample of units timed on all cores at once, scaled by the units one
# iteration needs, is that iteration's time on those cores.

def _oracle_geom(n):
    from oracle import lamino as olam
    from paper_2511_01893_b300 import inputs
    return olam.Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=inputs.angles(n), phi=np.deg2rad(PHI_DEG))


_ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_unit(kind, n, idx):
    """One unit of an n^3 ADMM-TV iteration's oracle work, timed in a worker
    process; returns (kind, seconds of the forward part, seconds of the
    transpose / rest).  kind: "plane" (F_u2D of one kv plane and its
    transpose), "slab" (F_u1D of one x-slab and its transpose), "tv" (the
    elementwise steps of one outer iteration, 4 CG steps + RSP, on one
    x-slab)."""
    from oracle import lamino as olam
    from oracle import tv as otv
    from oracle import usfft
    g = _oracle_geom(n)
    rng = np.random.default_rng(1000 + idx)
    if kind == "plane":
        kv = (n // 2 + 7 * idx) % n
        t, ku = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        xi_x, xi_y, _ = olam.slice_frequency_points(g, t.ravel(), np.full(t.size, kv), ku.ravel())
        xi_x, xi_y = xi_x.reshape(n, n), xi_y.reshape(n, n)
        plane = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        vals = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        t0 = time.perf_counter()
        usfft.usfft2d_type2(plane, xi_x, xi_y)
        t1 = time.perf_counter()
        usfft.usfft2d_type1(vals, xi_x, xi_y, n, n)
        return kind, t1 - t0, time.perf_counter() - t1
    if kind == "slab":
        _, _, xi_z = olam.slice_frequencies(olam.Geometry(n1=1, n0=n, n2=1, h=n, w=1, theta=np.zeros(1),
                                                          phi=g.phi))
        slab = rng.standard_normal((1, n, n))
        t0 = time.perf_counter()
        u1 = usfft.usfft1d_type2(slab, xi_z, axis=1)
        t1 = time.perf_counter()
        usfft.usfft1d_type1(u1, xi_z, n, axis=1)
        return kind, t1 - t0, time.perf_counter() - t1
    # elementwise TV / CG / RSP steps of one outer iteration on one x-slab,
    # the oracle's primitives in admm.lsp / admm.admm order
    u = rng.standard_normal((1, n, n))
    psi = rng.standard_normal((3, 1, n, n))
    lam = rng.standard_normal((3, 1, n, n))
    rho = 0.5
    t0 = time.perf_counter()
    gg = psi - lam / rho
    p = Gp = None
    for i in range(N_INNER):
        G = rng.standard_normal(u.shape) - rho * otv.div(otv.grad(u) - gg)  # data term stands in for L^H r
        p = -G if i == 0 else -G + (np.vdot(G, G).real / np.vdot(p, G - Gp).real) * p
        gp = otv.grad(p)
        gamma = -np.vdot(G, p).real / (1.0 + rho * np.vdot(gp, gp).real)
        u = u + gamma * p
        Gp = G
    gu = otv.grad(u)
    psi_new = otv.shrink_iso(gu + lam / rho, 1e-3 / rho)
    lam = lam + rho * (gu - psi_new)
    np.linalg.norm((gu - psi_new).ravel())
    np.linalg.norm(otv.div(psi_new - psi).ravel())
    otv.tv(u)
    return kind, time.perf_counter() - t0, 0.0


def oracle_pool(workers=None):
    """A spawn pool of one process per host core.  The workers inherit the
    environment at spawn time: one BLAS / OpenMP thread each, set before they
    import NumPy (no initializer: a pool whose initializer fails respawns its
    workers without end)."""
    import multiprocessing as mp
    w = workers or len(os.sched_getaffinity(0))
    saved = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update(_ONE_THREAD)
    try:
        pool = mp.get_context("spawn").Pool(w)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, w


def oracle_iteration_sample(pool, workers, n):
    """Time one sample of an n^3 ADMM-TV iteration's oracle work on `workers`
    processes: `workers` kv planes, `workers` x-slabs of the z stage and
    `workers` x-slabs of the elementwise steps, each wave run concurrently.
    One iteration = 4 CG steps x (2 L-hat + 1 L-hat^H) over h planes and n
    x-slabs, plus the elementwise steps over n x-slabs; the sample's per-unit
    times scale to it (units / workers concurrent).  Returns (s/iter on these
    cores, wall seconds the sample took, description)."""
    t_start = time.perf_counter()
    res = {}
    for kind in ("plane", "slab", "tv"):
        # bounded wait: a worker that dies raises here instead of waiting forever
        out = pool.starmap_async(_oracle_unit, [(kind, n, i) for i in range(workers)]).get(timeout=900)
        res[kind] = (float(np.mean([o[1] for o in out])), float(np.mean([o[2] for o in out])))
    waves = n / workers
    pf, pa = res["plane"]
    sf, sa = res["slab"]
    s_iter = N_INNER * waves * ((2 * pf + pa) + (2 * sf + sa)) + waves * res["tv"][0]
    wall = time.perf_counter() - t_start
    desc = (f"FP64 oracle as it stands on {workers} host cores (one process, one thread each): per sample "
            f"{workers} kv planes (F_u2D + transpose), {workers} x-slabs (F_u1D + transpose) and {workers} "
            f"x-slabs of the elementwise TV/CG/RSP steps of the {n}^3 workload, timed concurrently and "
            f"scaled to one ADMM-TV iteration (4 CG steps x (2 L-hat + 1 L-hat^H) over {n} planes and "
            f"{n} x-slabs + the elementwise steps over {n} x-slabs): {workers}/{n} of the work")
    return s_iter, wall, desc


def oracle_full_runs(pool, workers, n=None, s_iter=None):
    """Oracle runs done in full (not sampled), on the same cores: the plain
    workload (64^3, 64 angles, 8 x 4 ADMM-TV iterations, one process: its
    steps are too small to split) and one L-hat + L-hat^H at 512^3 (planes
    and x-slabs spread over the workers)."""
    out = {}
    t0 = time.perf_counter()
    r = pool.apply_async(_oracle_plain_admm)
    nf = 512  # the size run in full (n is the workload's)
    planes = pool.starmap_async(_oracle_unit, [("plane", nf, i) for i in range(nf)]).get(timeout=1800)
    slabs = pool.starmap_async(_oracle_unit, [("slab", nf, i) for i in range(nf)]).get(timeout=1800)
    out["lhat_pair_512_s"] = time.perf_counter() - t0
    out["lhat_pair_512_note"] = (f"one L-hat + L-hat^H at 512^3 (512 kv planes and 512 x-slabs over "
                                 f"{workers} processes), wall time; run in full")
    out["plain_admm_64_s"] = r.get(timeout=1800)
    out["plain_admm_64_note"] = "plain workload 64^3, 8 outer x 4 CG ADMM-TV, one process, run in full"
    if n and s_iter:
        # one iteration = 4 x (2 L-hat + 1 L-hat^H) + elementwise: a pair is
        # at most a quarter of it
        out[f"lhat_pair_{n}"] = (f"not run in full ({n}^3): the sampled units put one iteration at "
                                 f"{s_iter:.0f} s on these cores (a pair is under a quarter of it)")
    del planes, slabs
    return out


def _oracle_plain_admm():
    from oracle import admm as oadmm
    from oracle import lamino as olam
    from paper_2511_01893_b300 import inputs
    n = 64
    g = _oracle_geom(n)
    u = inputs.ellipsoid_phantom(n, n, 12, seed=1234).numpy()
    clean = olam.lam_forward(u, g)
    d = clean + 0.01 * np.abs(clean.real).max() * inputs.noise((n, n, n), seed=99).numpy()
    t0 = time.perf_counter()
    oadmm.admm(d, g, ALPHA, RHO, 8, N_INNER, adapt_rho=True)
    return time.perf_counter() - t0


def run_reference(args):
    """The oracle arm: each step is one sample of the workload's ADMM-TV
    iteration on all host cores (oracle_iteration_sample), scaled to s/iter;
    ms_per_step is the wall time a step (a sample) took.  After the timed
    steps, the plain workload and a 512^3 L-hat + L-hat^H run in full."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.size
    pool, workers = oracle_pool()
    try:
        vals, walls = [], []
        for i in range(args.warmup + args.steps):
            v, wall, desc = oracle_iteration_sample(pool, workers, n)
            if i >= args.warmup:
                vals.append(v)
                walls.append(wall)
        full = oracle_full_runs(pool, workers, n, statistics.median(vals))
    finally:
        pool.close()
        pool.join()
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "ADMM-TV seconds per iteration", "value": value, "unit": "s/iter",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(walls) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(n), "precision": "FP64 CPU oracle"},
        "step": f"one sample ({workers}/{n} of an iteration's work) per step; value = the sample scaled to s/iter",
        "cpu_baseline": {"value": value, "unit": "s/iter", "cores": workers, "kind": "oracle", "sample": desc,
                         "host_cores": os.cpu_count()},
        "full_runs": full,
        "e2e": {"value": value, "unit": "s/iter", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_op_pair(args):
    """Time L-hat + L-hat^H (steps pairs after warmup pairs) on the workload's
    geometry with a random volume; prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    n = args.size
    dev = torch.device("cuda", 0)
    plan = glam.Plan(n, n, n, n, inputs.angles(n), np.deg2rad(PHI_DEG), prec="f32", device=dev, workspace="hat",
                     spread=args.spread)
    u = torch.rand((n, n, n), device=dev, dtype=torch.float32)
    d = torch.empty(plan.data_shape, dtype=plan.cdtype, device=dev)
    v = torch.empty_like(u)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))  # u was drawn on the current stream
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            plan.forward_hat(u, out=d)
            plan.adjoint_hat(d, out=v)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = ta = 0.0
        for _ in range(args.steps):
            e[0].record(s)
            plan.forward_hat(u, out=d)
            e[1].record(s)
            plan.adjoint_hat(d, out=v)
            e[2].record(s)
            s.synchronize()
            tf += e[0].elapsed_time(e[1]) / 1e3
            ta += e[1].elapsed_time(e[2]) / 1e3
    tf /= max(args.steps, 1)
    ta /= max(args.steps, 1)
    byt = 2 * lhat_bytes(n, n, n, n, n)
    # adjoint identity <L_hat u, r> = <u, Re L_hat^H r> on random data r (a
    # property that holds at any size; FP64 dot products of the FP32
    # results).  r is drawn per angle from fixed seeds, first against L_hat u,
    # then again into the same buffer for L_hat^H: no second data-sized array.
    def r_chunk(k):
        gen = torch.Generator(device=dev).manual_seed(1000 + k)
        return torch.randn(plan.data_shape[1:], dtype=plan.cdtype, device=dev, generator=gen)
    with torch.cuda.stream(s):
        plan.forward_hat(u, out=d)
        lhs = dn2 = drn2 = 0.0
        for k in range(d.shape[0]):
            rk = r_chunk(k)
            lhs += torch.vdot(d[k].flatten(), rk.flatten()).real.double().item()
            dn2 += torch.vdot(d[k].flatten(), d[k].flatten()).real.double().item()
            drn2 += torch.vdot(rk.flatten(), rk.flatten()).real.double().item()
        for k in range(d.shape[0]):
            d[k].copy_(r_chunk(k))
        plan.adjoint_hat(d, out=v)
        rhs = sum(torch.dot(u[k].double().flatten(), v[k].double().flatten()).item() for k in range(u.shape[0]))
    s.synchronize()
    dn, drn = dn2 ** 0.5, drn2 ** 0.5
    adj = abs(lhs - rhs) / (dn * drn)
    print(json.dumps({"op": "lhat_pair", "size": n, "t_lhat_s": tf, "t_lhat_adj_s": ta,
                      "gbs": byt / (tf + ta) / 1e9, "adjoint_identity_rel": adj, "plan": plan.info()}), flush=True)
    return 0


def run_ablation(args):
    """Algorithm 1 (each CG step: r = L u - d with the full L, the full L^H, and
    L of the direction: two L and one L^H, F*_2D / F_2D each time) against
    Algorithm 2 (F*_2D / F_2D cancelled, subtraction fused, residual carried
    by linearity: one L_hat and one L_hat^H) on the workload, FP32, graph
    replay.  Prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    n = args.size
    dev = torch.device("cuda", 0)
    theta = inputs.angles(n)
    plan = glam.Plan(n, n, n, n, theta, np.deg2rad(PHI_DEG), prec="f32", device=dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        u_true = inputs.ellipsoid_circuit_phantom(n, n, seed=1238, device=dev, dtype=torch.float32)
        d = plan.forward(u_true)
        del u_true
        gen = torch.Generator(device=dev).manual_seed(99)
        d.real.add_(torch.randn(d.shape, generator=gen, device=dev, dtype=torch.float32),
                    alpha=0.01 * d.real.abs().max().item())
    s.synchronize()
    res, us = {}, {}
    for form in (1, 2):
        a = glam.Admm(plan)
        with torch.cuda.stream(s):
            a.init(d, ALPHA, RHO, N_INNER, form=form)
            a.run(args.warmup, graph=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            a.run(args.steps, graph=True)
            e1.record(s)
        s.synchronize()
        res[form] = e0.elapsed_time(e1) / 1e3 / max(args.steps, 1)
        us[form] = a.u.clone()
        res[f"status{form}"] = a.status()
        del a
        torch.cuda.empty_cache()
    diff = (us[1].double() - us[2].double()).norm().item() / us[2].double().norm().item()
    print(json.dumps({"op": "ablation", "size": n, "steps": args.steps, "warmup": args.warmup,
                      "alg1_s_per_iter": res[1], "alg2_s_per_iter": res[2], "speedup_alg2": res[1] / res[2],
                      "rel_l2_u_alg1_vs_alg2": diff, "status": max(res["status1"], res["status2"]),
                      "note": "FP32; both forms from the same data, same number of outer iterations"}),
          flush=True)
    return 0


def precision_data(glam, inputs, n, dev, stream):
    """The workload's data at n^3: the ellipsoid + circuit phantom through the
    FP64 GPU forward operator, 1 % Gaussian noise (seed 99), rounded to complex64
    (FP32-representable, so both precisions start from the same data)."""
    import torch
    theta = inputs.angles(n)
    phi = np.deg2rad(PHI_DEG)
    p64 = glam.Plan(n, n, n, n, theta, phi, prec="f64", device=dev, workspace="hat")
    with torch.cuda.stream(stream):
        u = inputs.ellipsoid_circuit_phantom(n, n, seed=1238, device=dev, dtype=torch.float64)
        d = p64.forward(u)
        del u
        sigma = 0.01 * d.real.abs().max().item()
        gen = torch.Generator(device=dev).manual_seed(99)
        for k in range(d.shape[0]):  # per angle: no second data-sized FP64 array
            d[k].real.add_(torch.randn(d.shape[1:], generator=gen, device=dev, dtype=torch.float64), alpha=sigma)
        d32 = d.to(torch.complex64)
    stream.synchronize()
    del d, p64
    torch.cuda.empty_cache()
    return theta, phi, d32


PRECISION_SNAPS = (1, 2, 4, 8, 16, 32, 64, 128)


def run_precision(args):
    """FP32 ADMM-TV (the library's FP32 defaults, graph replay) against the
    plain FP64 GPU path (eager, no graph) on the workload at --size, --iters
    outer iterations each, from the same FP32-representable data: relative L2
    of u at iterations 1, 2, 4, ... and s/iter of both.  Prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    n, iters = args.size, args.iters
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = torch.cuda.Stream(device=dev)
    theta, phi, d32 = precision_data(glam, inputs, n, dev, s)
    snaps = [k for k in PRECISION_SNAPS if k <= iters]
    res = {}
    for prec in ("f64", "f32"):
        plan = glam.Plan(n, n, n, n, theta, phi, prec=prec, device=dev)
        a = glam.Admm(plan)
        with torch.cuda.stream(s):
            a.init(d32, ALPHA, RHO, N_INNER, adapt_rho=True)
        s.synchronize()
        t, done, timed, us = 0.0, 0, 0, {}
        for k in snaps:
            with torch.cuda.stream(s):
                if prec == "f32" and done == 0:
                    a.run(1, graph=True)  # the capture stays outside the timed region
                    done = 1
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                a.run(k - done, graph=(prec == "f32"))
                e1.record(s)
            s.synchronize()
            t += e0.elapsed_time(e1) / 1e3
            timed += k - done
            done = k
            # the FP64 snapshots wait in host memory while the FP32 run has the device
            us[k] = a.u.to(torch.float64).cpu() if prec == "f64" else a.u.clone()
        res[prec] = {"s_per_iter": t / max(timed, 1), "u": us, "rho": a.history(iters)[:, 1].tolist(),
                     "status": a.status(), "objective": a.history(iters)[:, 0].tolist()}
        del a, plan
        torch.cuda.empty_cache()
    rel = {}
    for k in snaps:
        ref = res["f64"]["u"][k].to(dev)
        rel[k] = (torch.linalg.vector_norm(res["f32"]["u"][k].double() - ref) / torch.linalg.vector_norm(ref)).item()
    obj = np.array(res["f32"]["objective"]) / np.array(res["f64"]["objective"]) - 1
    print(json.dumps({
        "op": "precision", "size": n, "iters": iters,
        "workload": workload_name(n).replace("FP32, ", ""),
        "f32_graph_s_per_iter": res["f32"]["s_per_iter"], "f64_plain_s_per_iter": res["f64"]["s_per_iter"],
        "speedup": res["f64"]["s_per_iter"] / res["f32"]["s_per_iter"],
        "rel_l2_u_f32_vs_f64": {str(k): v for k, v in rel.items()},
        "max_rel_objective_diff": float(np.abs(obj).max()),
        "rho_same": res["f32"]["rho"] == res["f64"]["rho"],
        "status": max(res["f32"]["status"], res["f64"]["status"]),
        "source_sha256": full_source_hash(),
        "note": "FP32: exact spreads for the 3 centre plane jobs, compensated residual carry, graph replay; "
                "FP64: plain eager path",
    }), flush=True)
    return 0


def run_fbp(args):
    """FBP-style single pass (lam_fbp: F_2D, ramp, L-hat^H) on the workload's
    data at --size: seconds per pass over --steps passes after --warmup, and
    the relative L2 distance of the result from the phantom (the missing cone
    and the 1 % noise bound it; ADMM-TV is the method, FBP the one-pass
    baseline).  Prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    n = args.size
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    plan = glam.Plan(n, n, n, n, inputs.angles(n), np.deg2rad(PHI_DEG), prec="f32", device=dev)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        u_true = inputs.ellipsoid_circuit_phantom(n, n, seed=1238, device=dev, dtype=torch.float32)
        d = plan.forward(u_true)
        gen = torch.Generator(device=dev).manual_seed(99)
        d.real.add_(torch.randn(d.shape, generator=gen, device=dev, dtype=torch.float32),
                    alpha=0.01 * d.real.abs().max().item())
        out = torch.empty_like(u_true)
        for _ in range(args.warmup):
            plan.fbp(d, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            plan.fbp(d, out=out)
        e1.record(s)
    s.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / max(args.steps, 1)
    err = (torch.linalg.vector_norm(out - u_true) / torch.linalg.vector_norm(u_true)).item()
    print(json.dumps({"op": "fbp", "size": n, "s_per_pass": t, "voxels_per_s": n ** 3 / t,
                      "rel_l2_vs_phantom": err, "steps": args.steps, "warmup": args.warmup,
                      "note": "F_2D + ramp + L-hat^H, FP32; the phantom has content in the missing cone"}),
          flush=True)
    return 0


def run_memo(args):
    """Memoization of F*_u2D per plane job (LAM_OPT_MEMO_TAU) on the workload:
    --steps ADMM-TV iterations (FP32, graph replay) without memoization, the
    reference R_comp, then with each tau of --taus: the accuracy error
    E = ||R_comp - R|| / ||R_comp|| (Section 6.1, Eq. 4), the fraction of
    plane jobs served from the cache, s/iter.  Prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    n = args.size
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = torch.cuda.Stream(device=dev)
    theta, phi = inputs.angles(n), np.deg2rad(PHI_DEG)
    plan = glam.Plan(n, n, n, n, theta, phi, prec="f32", device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        u_true = inputs.ellipsoid_circuit_phantom(n, n, seed=1238, device=dev, dtype=torch.float32)
        d = plan.forward(u_true)
        gen = torch.Generator(device=dev).manual_seed(99)
        d.real.add_(torch.randn(d.shape, generator=gen, device=dev, dtype=torch.float32),
                    alpha=0.01 * d.real.abs().max().item())
    s.synchronize()
    res, ref = [], None
    for tau in [0.0] + [float(t) for t in args.taus.split(",")]:
        plan.set_memo(tau)
        a = glam.Admm(plan)
        with torch.cuda.stream(s):
            a.init(d, ALPHA, RHO, N_INNER)
            a.run(1, graph=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            a.run(args.steps - 1, graph=True)
            e1.record(s)
        s.synchronize()
        sc = a.scalars()
        u = a.u.clone()
        if ref is None:
            ref = u
        err = (torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref)).item()
        res.append({"tau": tau, "s_per_iter": e0.elapsed_time(e1) / 1e3 / max(args.steps - 1, 1), "E": err,
                    "one_minus_E": 1 - err, "reused_fraction": sc["memo_hits"] / max(sc["memo_lookups"], 1),
                    "objective": sc["objective"], "status": a.status()})
        del a
        torch.cuda.empty_cache()
    print(json.dumps({"op": "memo", "size": n, "iters": args.steps, "runs": res,
                      "note": "tau = 0: no memoization (R_comp); E of each run against it (Section 6.1, Eq. 4)"}),
          flush=True)
    return 0


BATCH_SIZES = [96, 128, 160, 192]


BATCH_STREAMS = (2, 4, 16)  # other side-stream counts tried by the concurrent batch mode
DEFAULT_BATCH_STREAMS = 8  # the library's default for 16 problems


def run_batch(args):
    """Batching workload: 16 FP32 reconstructions, n in {96, 128, 160, 192}
    (four each), nz = n / 2, n angles, detector n x n, tilt 20 + 20 i / 15 deg,
    ellipsoid phantoms + 1 % noise, launch shapes from the autotuner.  A step
    is one ADMM-TV outer iteration (4 CG steps) of all 16 problems in the
    library's default batch mode: every problem's own iteration on side
    stream i mod 8, forked and joined inside one CUDA graph.  Also timed: the
    persistent mode (every operator stage one launch over the batch), the same
    16 problems one after another (one graph per problem) and other stream
    counts.  Prints one JSON line."""
    import torch

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    plans, datas = [], []
    tune = 0.0
    for i in range(16):
        n = BATCH_SIZES[i % 4]
        phi = np.deg2rad(20.0 + 20.0 * i / 15)
        p = glam.Plan(n, n // 2, n, n, inputs.angles(n), phi, prec="f32", device=dev)
        t0 = time.perf_counter()
        p.autotune(reps=2)
        tune += time.perf_counter() - t0
        u = inputs.ellipsoid_phantom(n, n // 2, 12, seed=1234 + 3 * 100 + i, device=dev)
        d = p.forward(u)
        gen = torch.Generator(device=dev).manual_seed(4000 + i)
        d.real.add_(torch.randn(d.shape, generator=gen, device=dev), alpha=0.01 * d.real.abs().max().item())
        plans.append(p)
        datas.append(d)
    batch = glam.Batch(plans)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))  # the data were made on the current stream
    res = {}
    # "batched": the library's default (concurrent, 8 side streams); then the
    # persistent batched stages, the problems one after another, other stream counts
    modes = ["batched", "persistent", "sequential"] + [f"concurrent{k}" for k in BATCH_STREAMS]
    with torch.cuda.stream(s):
        for mode in modes:
            admms = [glam.Admm(p).init(d, ALPHA, RHO, N_INNER) for p, d in zip(plans, datas)]
            if mode.startswith("concurrent"):
                batch.set_streams(int(mode[len("concurrent"):]))
            elif mode == "persistent":
                batch.set_streams(0)

            def step(k):
                if mode == "sequential":
                    for a in admms:
                        a.run(k, graph=True)
                else:
                    batch.admm_run(admms, k, graph=True)
            step(args.warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.synchronize()
            e0.record(s)
            step(args.steps)
            e1.record(s)
            s.synchronize()
            res[mode] = e0.elapsed_time(e1) / 1e3 / max(args.steps, 1)
            res[mode + "_u"] = [a.u.clone() for a in admms]
            res[mode + "_status"] = max(a.status() for a in admms)
            if mode == "persistent":
                info = batch.info()  # persistent-mode stage grids and graph kernels
    same = all(all(torch.equal(a, b) for a, b in zip(res[m + "_u"], res["sequential_u"])) for m in modes)
    conc = {k: res[f"concurrent{k}"] for k in BATCH_STREAMS}
    conc[DEFAULT_BATCH_STREAMS] = res["batched"]
    best_k = min(conc, key=conc.get)
    vox = sum(p.n * p.nz * p.n for p in plans)
    line = {
        "metric": "batched ADMM-TV seconds per iteration (16 problems)", "value": res["batched"], "unit": "s/iter",
        "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batching: 16 reconstructions n in {96,128,160,192} x4, nz=n/2, n angles, "
                               "detector n x n, phi 20-40 deg, FP32, 4 CG steps/iter, graph-captured",
                   "sizes": [p.n for p in plans]},
        "sequential_s_per_iter": res["sequential"], "speedup_vs_sequential": res["sequential"] / res["batched"],
        "mode": f"concurrent: each problem's outer iteration on side stream i mod {DEFAULT_BATCH_STREAMS}, one graph",
        "persistent_s_per_iter": res["persistent"],
        "persistent_speedup_vs_sequential": res["sequential"] / res["persistent"],
        "concurrent_s_per_iter": dict(sorted(conc.items())), "concurrent_best": {"streams": best_k, "s_per_iter": conc[best_k],
                                                           "speedup_vs_sequential": res["sequential"] / conc[best_k]},
        "voxel_updates_per_s": vox / res["batched"], "batched_equals_sequential_bitwise": same,
        "status": max(res[m + "_status"] for m in modes), "autotune_s": tune,
        "launches_per_iter": info["graph_kernels"],
        "stage_grids": {k: v for k, v in info.items() if k != "graph_kernels"},
        "plans": [p.info() for p in plans[:4]],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2511_01893_b300 import inputs
    from paper_2511_01893_b300 import lamino as glam

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.size
    nz = h = w = T = n
    phi = np.deg2rad(PHI_DEG)
    theta = inputs.angles(T)

    # ---- inputs (synthetic, resident in HBM) --------------------------------
    u_true = inputs.ellipsoid_circuit_phantom(n, nz, seed=1238, device=dev, dtype=torch.float32)
    plan = glam.Plan(n, nz, h, w, theta, phi, prec="f32", device=dev, spread=args.spread)
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))  # u_true was made on the current stream
    with torch.cuda.stream(stream):
        d = plan.forward(u_true)
        sigma = 0.01 * d.real.abs().max().item()
        gen = torch.Generator(device=dev).manual_seed(99 + rank)
        d.real.add_(torch.randn(d.shape, generator=gen, device=dev, dtype=torch.float32), alpha=sigma)
    stream.synchronize()
    del u_true
    torch.cuda.empty_cache()

    admm = glam.Admm(plan)
    with torch.cuda.stream(stream):
        admm.init(d, ALPHA, RHO, N_INNER, adapt_rho=True)
        admm.run(args.warmup, graph=True)
    stream.synchronize()
    launches_per_step = admm.graph_kernels()

    # ---- timed ADMM iterations ------------------------------------------------
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            admm.run(args.steps, graph=True)
            ev1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    s_per_iter, t_admm, agg_iters = job_seconds_per_iter(ev0.elapsed_time(ev1) / 1e3, args.steps, world, dev)
    status = admm.status()
    sc = admm.scalars()

    # ---- L-hat + L-hat^H operator pair (bandwidth vs HBM roofline) ----------
    reps = 3
    p = admm.u.clone()
    out_c = torch.empty(plan.data_shape, dtype=plan.cdtype, device=dev)
    out_r = torch.empty(plan.vol_shape, dtype=plan.rdtype, device=dev)
    with torch.cuda.stream(stream):
        plan.forward_hat(p, out=out_c)
        plan.adjoint_hat(out_c, out=out_r)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps + 1)]
        evs[0].record(stream)
        for r in range(reps):
            plan.forward_hat(p, out=out_c)
            evs[2 * r + 1].record(stream)
            plan.adjoint_hat(out_c, out=out_r)
            evs[2 * r + 2].record(stream)
    stream.synchronize()
    t_fwd = statistics.median([evs[2 * r].elapsed_time(evs[2 * r + 1]) / 1e3 for r in range(reps)])
    t_adj = statistics.median([evs[2 * r + 1].elapsed_time(evs[2 * r + 2]) / 1e3 for r in range(reps)])
    op_bytes = 2 * lhat_bytes(n, nz, h, w, T)
    achieved = op_bytes / (t_fwd + t_adj) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak, peak_src = json.load(open(peaks_path))["hbm_gbs"], "measured"
    else:
        peak, peak_src = 6400.0, "fallback"
    # ---- the dominant kernel alone: the adjoint spread, one operator batch per
    # launch, CUDA events on its stream.  The launch covers the operator's plane
    # jobs per batch, starting after the centre jobs that take the exact spread
    # (LAM_OPT_EXACT_CENTRE_JOBS), so that it is the tile kernel alone ----------
    kreps = 5
    j0s = EXACT_CENTRE_JOBS
    with torch.cuda.stream(stream):
        nbj = plan.spread(out_c, j0s)
        kev = [torch.cuda.Event(enable_timing=True) for _ in range(kreps + 1)]
        kev[0].record(stream)
        for r in range(kreps):
            plan.spread(out_c, j0s, nbj)
            kev[r + 1].record(stream)
    stream.synchronize()
    t_spread = statistics.median([kev[r].elapsed_time(kev[r + 1]) / 1e3 for r in range(kreps)])
    spread_kernel = SPREAD_KERNELS[plan.info()["spread"]]
    planes = plan.job_planes(j0s, nbj)
    M = 2 * n
    # reads the batch's slice values (8 B per (theta, ku) of each data plane),
    # writes one padded plane (8 B per cell) per job
    spread_bytes = planes * T * w * 8 + nbj * M * M * 8
    spread_flops = planes * T * w * spread_point_flops()
    traffic = pair_traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        tj = json.load(open(prof))
        # only while the kernels are the ones the counters were taken on.  The
        # counters come from a small capture (capture_size^3, a few GB on the
        # device) and scale to this size by the units processed: a spread job's
        # traffic (its two planes' slice values and its padded plane) grows as
        # n^2 for T = w = h = n, the operator pair's as n^3
        if tj.get("source_sha256") == source_hash() and tj.get("capture_size"):
            f = n / tj["capture_size"]
            if tj.get("spread_bytes_per_job"):
                traffic = tj["spread_bytes_per_job"] * f ** 2 * nbj
            if tj.get("lhat_pair_dram_bytes"):
                pair_traffic = tj["lhat_pair_dram_bytes"] * f ** 3
    del p, out_c, out_r
    fma = glam.fma_peak(dev)
    op_flops = 2 * lhat_flops(n, nz, h, w, T)
    alu_achieved = op_flops / (t_fwd + t_adj)
    it_bytes = admm_iteration_bytes(n, nz, h, w, T)
    comparator = plane_fft_comparator(plan, glam, dev, stream) if rank == 0 else None

    line = {
        "metric": "ADMM-TV seconds per iteration", "value": s_per_iter, "unit": "s/iter", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_admm / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(n), "n": n, "nz": nz, "det_h": h, "det_w": w, "n_theta": T,
                   "phi_deg": PHI_DEG, "n_inner": N_INNER, "graph": True, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state ~80 GB)"},
        "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": spread_bytes / t_spread / 1e9, "peak": peak,
                     "frac": spread_bytes / t_spread / 1e9 / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": f"{spread_kernel} (adjoint spread; one launch = plane jobs {j0s}..{j0s + nbj - 1}, "
                               f"{planes} kv planes)",
                     "traffic_note": "dram bytes per job from a 512^3 capture, scaled by (n/512)^2 per job",
                     "algorithmic_bytes": spread_bytes, "t_launch_s": t_spread,
                     "note": "bound by the L1/shared pipe (ncu: 74 % of its peak) and instruction issue, not by HBM"},
        "roofline_alu": {"bound": "alu", "unit": "TFLOP/s", "achieved": spread_flops / t_spread / 1e12,
                         "peak": fma / 1e12, "frac": spread_flops / t_spread / fma,
                         "peak_source": "measured FMA probe", "kernel": spread_kernel,
                         "algorithmic_flops": spread_flops},
        "iteration_hbm": {"bound": "hbm", "unit": "GB/s", "achieved": it_bytes / s_per_iter / 1e9, "peak": peak,
                          "frac": it_bytes / s_per_iter / 1e9 / peak, "algorithmic_bytes": it_bytes,
                          "note": "one whole outer iteration: 8 operator applications, CG elementwise passes, RSP"},
        "operator_pair": {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak,
                          "frac": achieved / peak, "traffic": pair_traffic, "algorithmic_bytes": op_bytes,
                          "t_lhat_s": t_fwd, "t_lhat_adj_s": t_adj,
                          "alu_tflops": alu_achieved / 1e12, "alu_frac": alu_achieved / fma,
                          "algorithmic_flops": op_flops},
        "plane_fft_comparator": comparator,
        "aggregate": {"value": agg_iters, "unit": "iterations/s", "replicas": world,
                      "note": "every replica's iterations over the slowest replica's time"},
        "gpu_launches": launches_per_step * args.steps,
        "admm": {"status": status, "objective": sc["objective"], "rho": sc["rho"], "iters_done": sc["iter"]},
    }

    # ---- end to end through the one-call API (host data in, host volume out) -
    del admm, plan
    torch.cuda.empty_cache()
    if args.no_e2e:
        del d
    else:
        d_host = torch.empty(d.shape, dtype=torch.float32, pin_memory=True)
        d_host.copy_(d.real)
        del d
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        u_host = glam.reconstruct(d_host.numpy(), theta, phi, n, nz, args.steps, ALPHA, RHO)
        e2e_value, _, _ = job_seconds_per_iter(time.perf_counter() - t0, args.steps, world, dev)
        line["e2e"] = {"value": e2e_value, "unit": "s/iter",
                       "h2d_bytes_per_step": int(d_host.numel() * 4 // args.steps),
                       "d2h_bytes_per_step": int(u_host.size * 4 // args.steps),
                       "api": "reconstruct() one call, K iterations, host data/volume, includes plan + allocation"}
    line["clocks"] = clk.summary()

    # ---- the chosen FP32 form against the plain FP64 GPU path at this size --
    if not args.no_f64 and rank == 0:
        torch.cuda.empty_cache()
        line["f64_comparison"] = f64_comparison(glam, inputs, dev, stream, n)

    # ---- oracle on the host cores (rank 0, N = 1) ----------------------------
    if not args.no_cpu and rank == 0 and world == 1:
        pool, workers = oracle_pool()
        try:
            v, spent, sample = oracle_iteration_sample(pool, workers, n)
            line["cpu_baseline"] = {"value": v, "unit": "s/iter", "cores": workers, "kind": "oracle",
                                    "sample": sample, "host_cores": os.cpu_count(), "sample_seconds": spent}
        except Exception as ex:  # the GPU line stands without it
            line["cpu_baseline"] = {"value": None, "error": repr(ex)[:300]}
        finally:
            pool.terminate()
            pool.join()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0 if status == 0 else 1


def f64_comparison(glam, inputs, dev, stream, n, iters=2):
    """The chosen form (FP32, graph replay, the library's FP32 defaults) against
    the plain FP64 GPU path (eager) on the workload at n^3 from the same
    FP32-representable data (precision_data): s/iter of both and the relative
    L2 of u after `iters` iterations, measured here; the 32-iteration
    comparison comes from the record bench.py --op precision wrote
    (profiles/precision_<n>.json), attached only while its source hash matches
    the current CUDA sources."""
    import torch
    theta, phi, d32 = precision_data(glam, inputs, n, dev, stream)
    out = {"workload": f"{workload_name(n).replace('FP32, ', '')} (precision_data: FP64 forward, noise per angle)",
           "iters": iters}
    res = {}
    for prec in ("f64", "f32"):
        plan = glam.Plan(n, n, n, n, theta, phi, prec=prec, device=dev)
        a = glam.Admm(plan)
        with torch.cuda.stream(stream):
            a.init(d32, ALPHA, RHO, N_INNER)
            pre = 0
            if prec == "f32":
                a.run(1, graph=True)  # the capture stays outside the timed region
                pre = 1
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            a.run(iters - pre, graph=(prec == "f32"))
            e1.record(stream)
        stream.synchronize()
        res[prec] = (e0.elapsed_time(e1) / 1e3 / max(iters - pre, 1), a.u.double().cpu(), a.status())
        del a, plan
        torch.cuda.empty_cache()
    err = (torch.linalg.vector_norm(res["f32"][1] - res["f64"][1]) / torch.linalg.vector_norm(res["f64"][1])).item()
    out.update({"f32_graph_s_per_iter": res["f32"][0], "f64_plain_s_per_iter": res["f64"][0],
                "speedup": res["f64"][0] / res["f32"][0], f"rel_l2_f32_vs_f64_after_{iters}": err,
                "status": max(res["f32"][2], res["f64"][2])})
    rec = os.path.join(ROOT, "profiles", f"precision_{n}.json")
    if os.path.exists(rec):
        r = json.load(open(rec))
        if r.get("source_sha256") == full_source_hash():
            out["record_32_iterations"] = {k: r[k] for k in ("iters", "rel_l2_u_f32_vs_f64", "f32_graph_s_per_iter",
                                                              "f64_plain_s_per_iter", "speedup", "rho_same")
                                           if k in r}
        else:
            out["record_32_iterations"] = "stale (sources changed since the record was taken)"
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.op == "lhat_pair":
        return run_op_pair(args)
    if args.op == "batch":
        return run_batch(args)
    if args.op == "ablation":
        return run_ablation(args)
    if args.op == "precision":
        return run_precision(args)
    if args.op == "fbp":
        return run_fbp(args)
    if args.op == "memo":
        return run_memo(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
