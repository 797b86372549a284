"""Benchmark: BEM operator-apply Ginteractions/s on the synthetic rib / fat /
liver scene (~41k triangles, 0.5 MHz), FP32 matrix-free PMCHWT apply.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one application of the multiple-domain PMCHWT Galerkin operator
A_hat to a vector (trial gather -> far-field interactions -> projection with
the Sauter-Schwab near-field correction -> vertex reduction), inputs resident
in HBM.  An interaction is one Green's-function evaluation at one
(target point, source point) pair at one wavenumber.  Prints one JSON line.
Under torchrun each rank runs an independent replica (weak scaling, no
data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BEM operator-apply Ginteractions/s"
UNIT = "Ginteractions/s"
# Algorithmic FP32 work per (target point, source point) pair: the direct
# evaluation of the interaction formulas (G, F = G (ik - 1/r)/r, the four
# accumulations; FFMA = 2 flops, FADD/FMUL = 1, MUFU excluded), counted once
# and kept fixed as the unit of work, so that a kernel which reaches the same
# result with fewer operations shows a higher achieved rate: shared geometry
# 21 flops + per-triangle shared terms 11/6; per wavenumber 52 flops (54 when
# Im k != 0: the exp(-Im k r) factor) + per-triangle 32/6.
FL_SHARED = 21.0 + 11.0 / 6.0
FL_SLOT_LOSSLESS = 52.0 + 32.0 / 6.0
FL_SLOT_LOSSY = 54.0 + 32.0 / 6.0
# Of a slot's flops, the part that does not depend on the densities: the phase,
# G, the gradient factor F and the sum of G w (14 + 4 flops; +2 for Im k != 0).
# With R right-hand sides sharing a pair's G and F (far32m_kernel) the work of
# R interactions is R x the one-vector count minus (R - 1) x this part and the
# shared geometry.
FL_SLOT_SHARED_LOSSLESS = 18.0
FL_SLOT_SHARED_LOSSY = 20.0
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12


def measured_fp32_peak(stream=None):
    """Packed-FFMA rate measured on this GPU now (bem_peak_probe), TFLOP/s."""
    from paper_1910_01011_gb300 import api
    return max(api.peak_probe(0, 20000, stream) for _ in range(2)) / 1e12


def _measured_bf16():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1900.0  # fallback figure of the profiling recipe


BF16_PEAK_TFLOPS = _measured_bf16()


def workload(name):
    from synth import scenes
    if name == "rib":
        s = scenes.rib_scene()
        desc = "rib/fat/liver scene, 0.5 MHz, ~41k triangles (5 capsule ribs as one bone domain, fat slab, liver)"
    elif name == "rib_small":
        s = scenes.rib_scene(h=6e-3)
        desc = "rib/fat/liver scene at 6 mm element size (~8k triangles; profiling case)"
    elif name == "rib_small_resolved":
        s = scenes.rib_scene(h=6e-3, freq=0.1e6 * 2.65 / 6.0)
        desc = "rib/fat/liver scene at 6 mm element size and the frequency it resolves (k h ~ 1; ~8k triangles)"
    elif name == "rib_resolved":
        s = scenes.rib_scene_resolved()
        desc = "rib/fat/liver scene, 0.1 MHz (k h ~ 1), ~41k triangles (the solve-time workload)"
    elif name == "kidney":
        s = scenes.kidney_scene()
        desc = "kidney + perinephric fat shell, 1 MHz, ~62k triangles"
    elif name == "sphere":
        s = scenes.sphere_scene(3)
        desc = "unit sphere, icosphere level 3, k0=5, k1=5.25, rho ratio 1.1"
    else:
        raise SystemExit(f"unknown workload {name}")
    return s, desc


def algorithmic_flops_multi(s, R):
    """FP32 flops of one far-field launch on scene s for R right-hand sides
    that share each pair's geometry, G and F (see the constants above)."""
    slot0 = (FL_SLOT_SHARED_LOSSY if complex(s.k0).imag != 0 else FL_SLOT_SHARED_LOSSLESS)
    P = [6 * d.tris.shape[0] for d in s.domains]
    tot = sum(P)
    shared = 0.0
    for d, p in zip(s.domains, P):
        slot1 = FL_SLOT_SHARED_LOSSY if complex(d.k).imag != 0 else FL_SLOT_SHARED_LOSSLESS
        shared += p * (tot - p) * (FL_SHARED + slot0) + p * p * (FL_SHARED + slot0 + slot1)
    return R * algorithmic_flops(s) - (R - 1) * shared


def pair_counts(s):
    P = [6 * d.tris.shape[0] for d in s.domains]
    tot = sum(P)
    fused = sum(p * p for p in P)
    single = tot * tot - fused
    return single, fused, single + 2 * fused


def algorithmic_flops(s):
    """FP32 flops of one far32 launch on scene s (see the constants above)."""
    slot0 = FL_SLOT_LOSSY if complex(s.k0).imag != 0 else FL_SLOT_LOSSLESS
    P = [6 * d.tris.shape[0] for d in s.domains]
    tot = sum(P)
    fl = 0.0
    for d, p in zip(s.domains, P):
        slot1 = FL_SLOT_LOSSY if complex(d.k).imag != 0 else FL_SLOT_LOSSLESS
        fl += p * (tot - p) * (FL_SHARED + slot0) + p * p * (FL_SHARED + slot0 + slot1)
    return fl


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 200 ms) during the
    timed region; kept in `path` when one is given, else in a temporary file
    that is removed after the summary."""

    def __init__(self, index, path=None):
        import tempfile
        self.index = index
        self.p = None
        self.keep = path is not None
        if path is None:
            fd, path = tempfile.mkstemp(prefix="bench_clocks_", suffix=".csv")
            os.close(fd)
        self.path = path

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not self.keep:
            os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(s, n_rows_per_domain, seed=11):
    """Time the FP64 oracle's matrix-free apply on sampled output rows of
    the same scene; returns (interactions, seconds, description)."""
    import numpy as np

    from oracle import galerkin, pmchwt
    from synth import scenes
    galerkin.build()
    rng = np.random.default_rng(seed)
    rows = [rng.choice(d.verts.shape[0], size=n_rows_per_domain, replace=False) for d in s.domains]
    x = scenes.random_complex(2 * s.n_vertices, seed)
    n_int = 0
    for j, dj in enumerate(s.domains):
        for i, di in enumerate(s.domains):
            e = galerkin.regular_evals(dj.tris, di.tris.shape[0], rows[j], dj.verts.shape[0])
            n_int += e * (2 if i == j else 1)
    t0 = time.perf_counter()
    pmchwt.apply_rows(s, x, rows)
    dt = time.perf_counter() - t0
    return n_int, dt, f"{n_rows_per_domain} output vertices per domain (both rows), all sources"


def traffic_from_profile():
    """dram bytes per far-field launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "far32_kernel_rib_scene.md")
    src = os.path.join(ROOT, "paper_1910_01011_gb300", "csrc", "k_apply.cu")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != h.group(1)[:16]:
        return None
    return float(m.group(1))


def kidney_apply_metrics(local, steps=3, n_rhs=16, peak=FP32_PEAK_TFLOPS):
    """The same operator application on the kidney + perinephric fat scene
    (61,996 triangles, 1 MHz), autotuned launch shape, L2 flushed between
    steps; then the kidney workload of 16 right-hand sides in ONE matrix-free
    FP32 far-field launch (far32m_kernel, the pair's G and F shared by groups
    of four vectors), as interaction-RHS per second."""
    import torch

    from paper_1910_01011_gb300.api import Context
    s, desc = workload("kidney")
    stream = torch.cuda.current_stream()
    c = Context.from_scene(s, device=local, stream=stream.cuda_stream)
    N = c.n_dofs
    g = torch.Generator(device="cuda").manual_seed(99)
    x = torch.complex(torch.randn(N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(N, dtype=torch.float64, device="cuda", generator=g))
    y = torch.empty_like(x)
    c.apply(x, precision=1, out=y)
    tuned = c.autotune(1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        c.apply(x, precision=1, out=y)
    c.profile(True)
    c.profile_read(reset=True)
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.apply(x, precision=1, out=y)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    prof = c.profile_read(reset=True)
    far_ms = prof["far_ms"] / max(1, prof["far_launches"])
    achieved = algorithmic_flops(s) / (far_ms / 1e3) / 1e12
    n_int = pair_counts(s)[2]
    single = {"workload": desc, "value": n_int * steps / (ms / 1e3) / 1e9, "unit": UNIT,
              "far_field_chunk_tiles": tuned["chunk_tiles"],
              "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "kernel_ms": far_ms}}
    # 16 right-hand sides in one launch
    X = torch.complex(torch.randn(n_rhs, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(n_rhs, N, dtype=torch.float64, device="cuda", generator=g))
    Y = torch.empty_like(X)
    c.apply(X, precision=1, out=Y)
    c.profile_read(reset=True)
    ms_m = []
    for _ in range(2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.apply(X, precision=1, out=Y)
        b.record(stream)
        torch.cuda.synchronize()
        ms_m.append(a.elapsed_time(b))
    prof = c.profile_read(reset=True)
    c.close()
    far_m = prof["far_ms"] / max(1, prof["far_launches"])
    ach_m = algorithmic_flops_multi(s, n_rhs) / (far_m / 1e3) / 1e12
    ms_med = sorted(ms_m)[len(ms_m) // 2]
    single["multi_rhs"] = {
        "workload": f"kidney scene, {n_rhs} right-hand sides in one FP32 far-field launch (far32m_kernel)",
        "value": n_int * n_rhs / (ms_med / 1e3) / 1e9, "unit": "Ginteraction-RHS/s", "ms_per_apply": ms_med,
        "speedup_vs_single_rhs_applies": (ms * n_rhs / steps) / ms_med,
        "roofline": {"bound": "alu", "achieved": ach_m, "peak": peak, "unit": "TFLOP/s", "frac": ach_m / peak,
                     "kernel": "far32m_kernel", "kernel_ms": far_m,
                     "work": "R x the one-vector flops minus (R-1) x the density-independent geometry, G and F"}}
    return single


def sphere_solve_metrics(local, reps=12):
    """Config-1 sphere (icosphere level 3, k0 = 5, k1 = 5.25, density ratio
    1.1, plane wave): seconds per solve of the mixed path (FP32 operator
    inside a flexible GMRES, FP64 residual refinement) against the plain FP64
    GPU path, both to an FP64 relative residual of 1e-9, and the p50 / p99 of
    repeated mixed solves; then the off-surface field of the solution on the
    200 x 200 grid over +-3 R (the paper's sphere check) through bem_field."""
    import numpy as np

    from paper_1910_01011_gb300.api import Context
    from synth import scenes
    s = scenes.sphere_scene(3)
    c = Context.from_scene(s, device=local, n_pade=4, r_eps=0.2)
    c.set_plane_wave((0, 0, 1))
    c.solve(precision=1, tol=1e-9)  # set-up (near field, preconditioner) outside timing
    t64 = []
    for _ in range(3):
        t0 = time.perf_counter()
        r64 = c.solve(precision=0, tol=1e-9)
        t64.append(time.perf_counter() - t0)
    u64 = c.solution(0)
    t32 = []
    for _ in range(reps):
        t0 = time.perf_counter()
        r32 = c.solve(precision=1, tol=1e-9)
        t32.append(time.perf_counter() - t0)
    u32 = c.solution(0)
    # off-surface field on a 200 x 200 grid over +-3 R in the xz-plane, through
    # the public call with host arrays (copies and synchronisation included)
    g1 = np.linspace(-3.0, 3.0, 200)
    X, Z = np.meshgrid(g1, g1, indexing="ij")
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], axis=1)
    dom = np.where(np.linalg.norm(pts, axis=1) < 1.0, 0, -1).astype(np.int32)
    c.field(pts, dom)  # warm-up
    tf = []
    for _ in range(reps):
        t0 = time.perf_counter()
        c.field(pts, dom)
        tf.append(time.perf_counter() - t0)
    n_src = 6 * s.domains[0].tris.shape[0]
    c.close()
    field = {"grid": "200 x 200 over +-3 R, xz-plane", "points": int(pts.shape[0]),
             "ms_per_grid": 1e3 * float(np.median(tf)),
             "ginteractions_per_s": pts.shape[0] * n_src / float(np.median(tf)) / 1e9}
    return {"workload": "unit sphere, icosphere level 3 (1280 triangles), k0=5, k1=5.25, rho ratio 1.1, plane wave",
            "tol_fp64_residual": 1e-9, "fp64_s_per_rhs": float(np.median(t64)), "mixed_s_per_rhs": float(np.median(t32)),
            "mixed_p50_s": float(np.percentile(t32, 50)), "mixed_p99_s": float(np.percentile(t32, 99)),
            "speedup_vs_fp64": float(np.median(t64) / np.median(t32)),
            "trace_rel_diff_mixed_vs_fp64": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
            "iterations": {"fp64": r64["iterations"], "mixed": r32["iterations"], "refinements": r32["refinements"]},
            "ms_per_iteration": {"fp64": 1e3 * float(np.median(t64)) / max(1, r64["iterations"]),
                                 "mixed": 1e3 * float(np.median(t32)) / max(1, r32["iterations"])},
            "field": field}


def rib_solve_metrics(local, n_rhs=16, tol=1e-8, reps=3):
    """The rib / fat / liver scene at the frequency its mesh resolves (0.1 MHz,
    41k triangles, k h ~ 1), random-phase piston excitations of the 256-piston
    bowl, every path to an FP64 relative residual of tol, operators assembled
    once (set-up reported separately, kept on the device for later requests):
      * mixed batched: n_rhs excitations in lockstep, split-BF16 tensor-core
        GEMM inside a flexible GMRES, OSRC with loose sparse solves, FP64
        residual refinement; run `reps` times (p50 / p99 per excitation);
      * FP64 batched: the same n_rhs excitations in lockstep, FP64-accurate
        assembled operator inside the same GMRES (the baseline at the same
        batching);
      * one excitation alone, mixed and FP64;
      * block GMRES (one Krylov space per block of the n_rhs excitations,
        grown by n_rhs vectors per step), mixed (`reps` runs) and FP64.
    The traces of the mixed and FP64 paths agree to the reported difference."""
    import numpy as np
    import torch

    from paper_1910_01011_gb300.api import BF16X3, FP64_ASSEMBLED, Context
    from synth import scenes
    s = scenes.rib_scene_resolved()
    tr = s.transducer
    # R_eps: the paper's rib value (1e-4 m at 1 MHz) at the same k R_eps for this 0.1 MHz scene
    r_eps = 1e-4 * 1e6 / s.freq
    c = Context.from_scene(s, device=local, n_pade=8, r_eps=r_eps)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2 * np.pi * s.freq * s.rho0)
    W = np.exp(2j * np.pi * np.random.default_rng(3).random((n_rhs, tr["radii"].size)))
    N = c.n_dofs
    x = torch.zeros(N, dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    c.apply(x, precision=FP64_ASSEMBLED)
    c.apply(x, precision=BF16X3)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0

    def timed(**kw):
        t = time.perf_counter()
        rep = c.solve(operator_mode=1, tol=tol, max_iter=20000, **kw)
        return time.perf_counter() - t, rep

    c.set_excitations(W[:1])
    t64_1, r64_1 = timed(precision=0)
    u64 = c.solution(0)
    t32_1, r32_1 = timed(precision=1)
    c.set_excitations(W)
    tb64, rb64 = timed(precision=0, batch_rhs=n_rhs)
    ub64 = c.solution(0)
    tbs, rbs = [], None
    for _ in range(reps):
        t, rbs = timed(precision=1, batch_rhs=n_rhs)
        tbs.append(t)
    ub = c.solution(0)
    tks, rks = [], None
    for _ in range(reps):
        t, rks = timed(precision=1, batch_rhs=n_rhs, block_gmres=1)
        tks.append(t)
    ubk = c.solution(0)
    tk64, rk64 = timed(precision=0, batch_rhs=n_rhs, block_gmres=1)
    ubk64 = c.solution(0)
    c.close()
    per = np.array(tbs) / n_rhs
    perk = np.array(tks) / n_rhs
    return {"workload": f"rib/fat/liver scene, 0.1 MHz, {s.n_triangles} triangles (N={N}), {n_rhs} random-phase "
                        f"excitations of the 256-piston bowl, n_pade 8, R_eps {r_eps * 1e3:.1f} mm, OSRC blocks at "
                        f"each domain's k_j",
            "tol_fp64_residual": tol, "setup_s": setup,
            "mixed_batched_s_per_rhs": float(np.median(per)),
            "mixed_batched_p50_s_per_rhs": float(np.percentile(per, 50)),
            "mixed_batched_p99_s_per_rhs": float(np.percentile(per, 99)),
            "mixed_batched_runs": len(tbs),
            "fp64_batched_s_per_rhs": tb64 / n_rhs,
            "mixed_block_s_per_rhs": float(np.median(perk)),
            "mixed_block_p50_s_per_rhs": float(np.percentile(perk, 50)),
            "mixed_block_p99_s_per_rhs": float(np.percentile(perk, 99)),
            "fp64_block_s_per_rhs": tk64 / n_rhs,
            "speedup_block_mixed_vs_block_fp64": (tk64 / n_rhs) / float(np.median(perk)),
            "speedup_block_mixed_vs_batched_fp64": (tb64 / n_rhs) / float(np.median(perk)),
            "trace_rel_diff_block_mixed_vs_fp64": float(np.linalg.norm(ubk - ub64) / np.linalg.norm(ub64)),
            "trace_rel_diff_block_fp64_vs_fp64": float(np.linalg.norm(ubk64 - ub64) / np.linalg.norm(ub64)),
            "mixed_single_s_per_rhs": t32_1, "fp64_single_s_per_rhs": t64_1,
            "speedup_batched_mixed_vs_batched_fp64": (tb64 / n_rhs) / float(np.median(per)),
            "speedup_single_mixed_vs_single_fp64": t64_1 / t32_1,
            "speedup_batched_mixed_vs_single_fp64": t64_1 / float(np.median(per)),
            "trace_rel_diff_mixed_vs_fp64": float(np.linalg.norm(ub - ub64) / np.linalg.norm(ub64)),
            "trace_rel_diff_single_fp64_vs_batched_fp64": float(np.linalg.norm(ub64 - u64) / np.linalg.norm(u64)),
            "iterations_per_rhs": {"fp64_single": r64_1["iterations"], "mixed_single": r32_1["iterations"],
                                   "fp64_batched": rb64["iterations"] / n_rhs,
                                   "mixed_batched": rbs["iterations"] / n_rhs,
                                   "mixed_block_steps": rks["iterations"] / n_rhs,
                                   "fp64_block_steps": rk64["iterations"] / n_rhs},
            "residual": {"fp64_batched": rb64["residual"], "mixed_batched": rbs["residual"],
                         "mixed_block": rks["residual"], "fp64_block": rk64["residual"]}}


def serving_metrics(local, n_req=12, max_exc=16, rate=20.0, budget=150 << 30, tol=1e-6, rank=0, world=1, slots=2,
                    pool=None):
    """Serving trace: Poisson arrivals (mean `rate`/s) of planning solves over
    a pool of scenes (spheres of 1k and 5k triangles, rib scenes of 10k and
    20k, kidney scenes of 20k and 40k, each at k h ~ 1), each request with
    1..max_exc random-phase piston excitations, through the request loop
    (device-resident scene cache, admission by the HBM budget; mixed
    precision with batched excitations solved by block GMRES, FP64
    refinement to tol, `slots` workers).  Baseline: the same trace, at the same arrival times, through a
    request loop that solves one excitation at a time in plain FP64 with one
    worker (sequential FP64 GPU solves).  Each loop's cache is warmed with one
    request per scene first (set-up not in the latencies)."""
    import numpy as np

    from paper_1910_01011_gb300.api import Server
    from synth import serving
    reqs, weights = serving.trace(n_req, rate=rate, max_exc=max_exc, pool=pool)
    # replicas: each rank serves its contiguous share of the trace
    b, e = shard(len(reqs), rank, world)
    if world > 1:
        t_b = reqs[b][0] if b < e else 0.0
        reqs = [(t - t_b, k, ne) for t, k, ne in reqs[b:e]]
        weights = (lambda w0, off: (lambda i, n_elem: w0(i + off, n_elem)))(weights, b)
        n_req = len(reqs)
    if not reqs:
        return {"requests": 0}
    keys = sorted({k for _, k, _ in reqs})
    built = {k: serving.POOL[k]() for k in keys}

    def run(**srv_kw):
        srv = Server(device=local, hbm_budget_bytes=budget, tol=tol, max_iter=20000, max_refine=20, **srv_kw)
        ids = {k: srv.add_scene(built[k], omega_rho0=built[k].meta["omega_rho0"], n_pade=8,
                                r_eps=built[k].meta["r_eps"]) for k in keys}
        tw = time.perf_counter()
        for k in keys:  # warm the cache (geometry, near field, assembled operators, preconditioner)
            h = srv.submit(ids[k], np.ones((1, srv.scenes[ids[k]][1])))
            srv.wait(h)
            srv.result(h, 1, ids[k])
        warm_s = time.perf_counter() - tw
        warm = srv.stats()
        t0 = time.perf_counter()
        hs = []
        for i, (ta, k, ne) in enumerate(reqs):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            hs.append((srv.submit(ids[k], weights(i, srv.scenes[ids[k]][1])), k, ne))
        lat, fails, its = [], [], {}
        for h, k, ne in hs:
            srv.wait(h)
            try:
                _, rep = srv.result(h, ne, ids[k])
                lat.append(rep["latency_ms"])
                its.setdefault(k, []).append(rep["iterations"] / max(1, rep["batch_exc"]))
            except Exception as ex:  # reported, not hidden
                fails.append(f"{k}: {ex}")
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return {"p50_ms": float(np.percentile(lat, 50)) if lat else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat else None,
                "wall_s": wall, "excitations_per_s": n_exc / wall, "requests_per_s": n_req / wall,
                "batches": st["batches"] - warm["batches"], "joined_requests": st["joined"] - warm["joined"],
                "peak_device_gib": st["peak_device_bytes"] / 2**30,
                "evictions": st["evictions"], "warm_up_s": warm_s,
                "iterations_per_excitation": {k: float(np.mean(v)) for k, v in its.items()},
                "failed_requests": fails}

    n_exc = sum(ne for _, _, ne in reqs)
    mixed = run(slots=slots, max_batch_rhs=64, precision=1, operator_mode=1)
    seq = run(slots=1, max_batch_rhs=1, precision=0, operator_mode=1, batch_rhs=1, block_gmres=0)
    out = {"workload": f"{n_req} requests, Poisson {rate}/s, 1..{max_exc} excitations each ({n_exc} total), "
                       f"scenes {keys}, tol {tol}, budget {budget / 2**30:.0f} GiB, {slots} workers",
           **mixed,
           "fp64_sequential": {"how": "the same trace and arrival times through a request loop with one worker, "
                                      "one excitation per plain FP64 solve", **seq},
           "speedup_vs_fp64_sequential": seq["wall_s"] / mixed["wall_s"]}
    return out


def assembled_metrics(ctx, s, n_int, local, n_rhs=256):
    """Config-3 form on the same scene: A_hat assembled once in complex64 and
    applied to n_rhs right-hand sides by the split-BF16 tensor-core GEMM."""
    import torch

    from paper_1910_01011_gb300.api import BF16X3
    N = ctx.n_dofs
    g = torch.Generator(device="cuda").manual_seed(7)
    X = torch.complex(torch.randn(n_rhs, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(n_rhs, N, dtype=torch.float64, device="cuda", generator=g))
    t0 = time.perf_counter()
    ctx.apply(X[:1].contiguous(), precision=BF16X3)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    Y = ctx.apply(X, precision=BF16X3)
    ts = []
    for _ in range(5):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.apply(X, precision=BF16X3, out=Y)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = sorted(ts)[len(ts) // 2]
    tflop = 48.0 * N * N * n_rhs / 1e12       # 12 split products x 2 flops x N x 2R x N
    return {"workload": f"same scene, {n_rhs} right-hand sides, assembled complex64 A_hat, split-BF16 (3 terms, 6 products) tcgen05 GEMM",
            "assembly_s": setup, "ms_per_apply": ms, "pair_rhs_per_s": n_int * n_rhs / (ms / 1e3),
            "roofline": {"bound": "tensor", "achieved": tflop / (ms / 1e3), "peak": BF16_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": tflop / (ms / 1e3) / BF16_PEAK_TFLOPS,
                         "peak_basis": "MEASURED_PEAKS.json bf16_tflops (burst)"}}


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over all ranks (timings: the job is as slow as its
    slowest replica); x itself on one process."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank in at most seconds_max (weak scaling)."""
    return world * units_per_rank / seconds_max


def shard(n: int, rank: int, world: int):
    """[begin, end) of rank's share of n independent items (excitations or
    requests), contiguous and balanced to within one item."""
    q, r = divmod(n, world)
    b = rank * q + min(rank, r)
    return b, b + q + (1 if rank < r else 0)


def prec_step(args, s, desc, local, world):
    """One OSRC preconditioner application to R right-hand sides per step
    (n_pade 8, sparse solves to a 10 % relative residual, as inside the
    flexible GMRES)."""
    import torch

    from paper_1910_01011_gb300.api import PREC, Context
    ctx = Context.from_scene(s, device=local, stream=torch.cuda.current_stream().cuda_stream, n_pade=8,
                             osrc_tol=0.1, osrc_solver=args.osrc_solver)
    N, R = ctx.n_dofs, args.prec_rhs
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.complex(torch.randn(R, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(R, N, dtype=torch.float64, device="cuda", generator=g))
    Y = torch.empty_like(X)
    for _ in range(max(3, args.warmup)):
        ctx.apply(X, op=PREC, out=Y)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.apply(X, op=PREC, out=Y)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    prof = ctx.profile_read(reset=True)
    ctx.close()
    print(json.dumps({"metric": "OSRC preconditioner applications (right-hand sides) per s", "value": R * args.steps / dt,
                      "unit": "RHS/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
                      "config": {"workload": desc, "n_rhs": R, "n_pade": 8, "osrc_tol": 0.1,
                                 "osrc_solver": ["automatic", "one CTA per system", "grid-wide", "cluster per system",
                                                 "cluster per group of shifts"][args.osrc_solver]},
                      "gpu_launches": prof["kernel_launches"]}))


def solve_step(args, s, desc, local, world):
    """Mixed batched solves (split-BF16 assembled operator, flexible GMRES,
    OSRC with loose FP32 sparse solves, FP64 refinement to 1e-8) of
    --prec-rhs random-phase piston excitations, --steps times after --warmup
    untimed solves; seconds per excitation."""
    import numpy as np

    from paper_1910_01011_gb300.api import Context
    tr = s.transducer
    ctx = Context.from_scene(s, device=local, n_pade=8, r_eps=1e-4 * 1e6 / s.freq, osrc_solver=args.osrc_solver)
    ctx.set_transducer(tr["centres"], tr["normals"], tr["radii"], 2 * np.pi * s.freq * s.rho0)
    R = args.prec_rhs
    ctx.set_excitations(np.exp(2j * np.pi * np.random.default_rng(3).random((R, tr["radii"].size))))
    kw = dict(precision=1, operator_mode=1, tol=1e-8, batch_rhs=R, max_iter=20000, block_gmres=1 if args.block else 0)
    for _ in range(max(1, args.warmup)):
        ctx.solve(**kw)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    t0 = time.perf_counter()
    rep = None
    for _ in range(args.steps):
        rep = ctx.solve(**kw)
    dt = time.perf_counter() - t0
    prof = ctx.profile_read(reset=True)
    ctx.close()
    print(json.dumps({"metric": "mixed batched solve, seconds per excitation", "value": dt / args.steps / R,
                      "unit": "s/RHS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": False,
                      "config": {"workload": desc, "n_rhs": R, "n_pade": 8, "tol": 1e-8,
                                 "gmres": "block" if args.block else "lockstep",
                                 "osrc_solver": ["automatic", "one CTA per system", "grid-wide", "cluster per system",
                                                 "cluster per group of shifts"][args.osrc_solver]},
                      "iterations_per_rhs": rep["iterations"] / R, "gpu_launches": prof["kernel_launches"]}))


def run_reference(args, rank, world):
    if rank != 0:
        return
    s, desc = workload(args.workload)
    cores = os.cpu_count()
    vals, times = [], []
    for _ in range(args.warmup):
        oracle_sample(s, 1)
    n_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        n, dt, sample = oracle_sample(s, args.ref_rows, seed=100 + k)
        n_tot += n
        t_tot += dt
    value = n_tot / t_tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n_triangles": s.n_triangles, "n_dofs": s.n_dofs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: {sample} (FP64 C oracle, OpenMP)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rib",
                    choices=["rib", "rib_small", "rib_small_resolved", "rib_resolved", "kidney", "sphere"])
    ap.add_argument("--ref-rows", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the solve and assembled-GEMM measurements")
    ap.add_argument("--quick", action="store_true", help="skip the rib-scene solve and the serving trace")
    ap.add_argument("--extra", action="append", default=None,
                    choices=["assembled", "solve_sphere", "apply_kidney", "solve", "serving"],
                    help="run only these extras (repeatable); default: all that the other flags allow")
    ap.add_argument("--step", default="apply", choices=["apply", "prec", "solve"],
                    help="apply: the operator application (the headline metric); prec: one OSRC preconditioner "
                         "application to --prec-rhs right-hand sides (for profiling the sparse solves); solve: one "
                         "mixed batched solve of --prec-rhs piston excitations with assembled operators (for "
                         "profiling the loose sparse solves inside the flexible GMRES)")
    ap.add_argument("--prec-rhs", type=int, default=8)
    ap.add_argument("--block", action="store_true", help="--step solve: block GMRES instead of lockstep GMRES")
    ap.add_argument("--rhs", type=int, default=1,
                    help="right-hand sides per apply step; > 1 applies them in one matrix-free far-field launch "
                         "(far32m_kernel) and reports interaction-RHS per second (profiling of the multi-RHS path)")
    ap.add_argument("--serving-max-exc", type=int, default=64,
                    help="serving trace: excitations per request drawn from 1..this (default: the stated 1..64)")
    ap.add_argument("--clocks-log", default=None, help="keep the raw nvidia-smi clock samples in this CSV file")
    ap.add_argument("--osrc-solver", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="sparse solver of the preconditioner step: 0 automatic, 1 one CTA per system, 2 grid-wide, "
                         "3 one thread-block cluster per system, 4 one cluster per group of Pade shifts")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in far-field launch shape instead of the autotuned one")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1910_01011_gb300.api import Context

    s, desc = workload(args.workload)
    stream = torch.cuda.current_stream()
    if args.step == "prec":
        return prec_step(args, s, desc, local, world)
    if args.step == "solve":
        return solve_step(args, s, desc, local, world)
    ctx = Context.from_scene(s, device=local, stream=stream.cuda_stream)
    N = ctx.n_dofs
    single, fused, n_int = pair_counts(s)
    assert n_int == ctx.interactions
    R = max(1, args.rhs)
    flops = algorithmic_flops(s) if R == 1 else algorithmic_flops_multi(s, R)

    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    shape = (N,) if R == 1 else (R, N)
    x = torch.complex(torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen),
                      torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen))
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ctx.apply(x, precision=1, out=y)          # set-up (geometry, near field) outside timing
    torch.cuda.synchronize()
    tuned = None if (args.no_autotune or R > 1) else ctx.autotune(1)   # launch shape picked by timing (bem_autotune)
    for _ in range(max(3, args.warmup)):
        ctx.apply(x, precision=1, out=y)
    torch.cuda.synchronize()

    ctx.profile(True)
    ctx.profile_read(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, args.clocks_log) as clk:
        for k in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps (outside the events)
            starts[k].record(stream)
            ctx.apply(x, precision=1, out=y)
            ends[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)), world)
    ms_per_step = ms / args.steps
    value = job_rate(n_int * R * args.steps, world, ms / 1e3) / 1e9
    # the FP32 FFMA rate measured on this GPU right after the timed region
    peak_meas = measured_fp32_peak(stream.cuda_stream)

    # e2e: the public call with host buffers (pinned), copies inside the timing
    xh = torch.empty(shape, dtype=torch.complex128).pin_memory()
    yh = torch.empty(shape, dtype=torch.complex128).pin_memory()
    xh.copy_(x.cpu())
    xa, ya = xh.numpy(), yh.numpy()
    ctx.apply(xa, precision=1, out=ya)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.apply(xa, precision=1, out=ya)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = job_rate(n_int * R * args.steps, world, e2e_s) / 1e9

    far_ms = prof["far_ms"] / max(1, prof["far_launches"])
    achieved = flops / (far_ms / 1e3) / 1e12
    traffic = traffic_from_profile()
    line = {"metric": METRIC if R == 1 else f"BEM operator-apply Ginteraction-RHS/s ({R} RHS in one launch)",
            "value": value, "unit": UNIT if R == 1 else "Ginteraction-RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n_triangles": s.n_triangles, "n_dofs": N,
                       "interactions_per_step": n_int * R, "rhs_per_step": R,
                       "precision": "FP32 far field, FP64 near field/output",
                       "l2": "flushed between timed steps (256 MB write)", "replicas": world,
                       "far_field_chunk_tiles": (tuned or {}).get("chunk_tiles", "built-in")},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_meas, "unit": "TFLOP/s",
                         "frac": achieved / peak_meas, "traffic": traffic if R == 1 else None,
                         "kernel": "far32_kernel" if R == 1 else "far32m_kernel", "kernel_ms": far_ms,
                         "peak_basis": "measured: packed FFMA2 chains on every SM (bem_peak_probe), in this run",
                         "peak_derived": FP32_PEAK_TFLOPS, "frac_of_derived": achieved / FP32_PEAK_TFLOPS,
                         "peak_derived_basis": "152 SMs x 128 FP32 lanes x 2 (FFMA) x 2070 MHz max clock"},
            "e2e": {"value": e2e_value, "unit": UNIT if R == 1 else "Ginteraction-RHS/s",
                    "h2d_bytes_per_step": 16 * N * R, "d2h_bytes_per_step": 16 * N * R},
            "gpu_launches": prof["kernel_launches"],
            "clocks": clk.summary()}
    if not args.no_extras:
        extra_s = line.setdefault("extra_seconds", {})

        def extra(name, fn, *a):
            if args.extra and name not in args.extra:
                return
            t_x = time.perf_counter()
            try:
                line[name] = fn(*a)
            except Exception as e:  # the line still prints; the failure is part of it
                line[name] = {"error": f"{type(e).__name__}: {e}"}
            extra_s[name] = round(time.perf_counter() - t_x, 1)
        extra("assembled", assembled_metrics, ctx, s, n_int, local)
        extra("solve_sphere", sphere_solve_metrics, local)
        if not args.quick and world == 1:
            extra("apply_kidney", kidney_apply_metrics, local, 3, 16, peak_meas)
            # the minutes-long solve and serving measurements run on one GPU; replicas
            # of them on more GPUs would only repeat the same numbers
            extra("solve", rib_solve_metrics, local)
            extra("serving", serving_metrics, local, 12, args.serving_max_exc, 20.0, 150 << 30, 1e-6, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, dt, sample = oracle_sample(s, args.ref_rows)
        line["cpu_baseline"] = {"value": n / dt / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample + f", {n:.3g} interactions in {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
