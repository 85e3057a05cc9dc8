#!/usr/bin/env python
"""Benchmark of the 6-D spectral transport step (one JSON line on rank 0).

Workload (default): the absorber problem on the 33 x 16^4 grid with 4 energy
groups in FP64 -- shell r in [0.2, 1], kappa = 1 + 0.5 sin(theta) cos(phi),
eta = kappa exp(-r^2), kappa_s = 0.5, seeded smooth initial data, static
inflow data, dt = 0.4 x the smallest radial node spacing, classical RK4.
One benchmark step = one RK4 step of every group (12 kernel launches).

Metric: phase-space point-updates per second (grid points x groups x steps /
device time), timed with CUDA events on the launching stream between a
barrier + synchronize on both sides, max over ranks. Under torchrun each rank
runs its own copy of the workload on its own GPU (weak scaling; no collective
on the data path).

Extra keys: roofline of the dominant kernel (per-launch device time from
ts_step_profile; FP64 ALU peak derived from the SM count, the FP64 lanes per SM
and the clock, with a measured DFMA-loop rate beside it), end-to-end rate
through ts_step_host (host buffers, copies inside the timed region), the
reduced-precision variants (FP32, FP32 + FP64 radial rows, tensor-core TF32x3
and BF16x3) and the adjoint step on the same workload, the same grid with
linearly anisotropic neutrino-nucleon scattering, with Thomson scattering and with
the paper's AB2 time marching, the Lambert-shell run of Sect. 5.3 on the hybrid
grid (upwind finite differences in r), the 64-problem batch,
the differentiation workload (33 x 16^4, 8 groups, 200 steps with sqrt(N)
checkpoints), the CPU oracle timed on a bounded sample on this host's cores,
and SM clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "phase-space point-updates/s per GB300 (fwd, adjoint) vs plain FP64 GPU form at stated err"
WORKLOADS = {
    # name: (R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups)
    "absorber_33x16^4_g4": (0.2, 1.0, 33, 16, 16, 16, 16, 4),
    "absorber_17x8^4_g1": (0.2, 1.0, 17, 8, 8, 8, 8, 1),
    "absorber_65x32^4_g1": (0.2, 1.0, 65, 32, 32, 32, 32, 1),
}
PRECISIONS = {"fp64": "TS_FP64", "fp32": "TS_FP32", "fp32_r64": "TS_FP32_R64",
              "tf32x3": "TS_TF32X3", "bf16x3": "TS_BF16X3"}
FP64_FMA_PER_SM_CLK = 2        # GB300: 2 FP64 FMA lanes per SM (1/64 of the 128 FP32 lanes)
FP32_FMA_PER_SM_CLK = 128
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


# ------------------------------------------------------------------ helpers
def max_over_ranks(ms, world, device):
    """The slowest rank's time: every rank runs its own replica of the workload
    (weak scaling), so the job takes as long as its slowest rank."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("ts_kernels.cuh", "ts_kernels_rb.cuh", "ts_launch.cuh", "ts_tc.cuh"):
        with open(os.path.join(ROOT, "paper_1104_5330_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload, precision):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    if the kernels changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("kernel_hash") != _kernel_hash():
        return None
    return t.get("per_launch_bytes", {}).get(f"{workload}/{precision}/{kernel}")


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"ts_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------- algorithmic work
def even_odd_passes(dims, es):
    """Which passes run in the register-blocked even/odd form (the library's rule)."""
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    rbA = 4 if es == 4 else 2
    return {"angular": NT % rbA == 0 and NP % 8 == 0,
            "plane": Nt % 2 == 0 and Np % 2 == 0 and NP % 8 == 0,
            "radial": Nr >= 9 and (Nr // 2) % 2 == 0 and (NT * NP) % 4 == 0}


def plane_square(dims):
    """The library's square-grid plane pass (16 nodes on every angular axis)."""
    return dims[3] == dims[4] == dims[5] == dims[6] == 16


def eo_kernel(name, dims):
    """Kernel of the register-blocked even/odd form of a pass: persistent
    k_angular_pp / k_plane_pp (k_plane_sq on square grids), one tile per CTA
    k_radial_eo."""
    if name == "radial":
        return "k_radial_eo"
    if name == "plane" and plane_square(dims):
        return "k_plane_sq"
    return f"k_{name}_pp"


def pass_work(dims, es):
    """Algorithmic flops and DRAM bytes per launch of each pass (one stage of
    all groups). Flops count the contractions the pass performs (2 per
    multiply-add; the even/odd forms need half the multiply-adds of a dense
    DFS or Chebyshev product) and the pointwise terms; bytes count each field
    the pass must read or write once."""
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    pts = Nr * Nt * Np * NT * NP * G
    eo = even_odd_passes(dims, es)
    flops = {
        # dTh and dPh on the DFS pair halves (even/odd) or dense, J, coefficients, collision
        # (even/odd: Theta folded twice -- DFS pair and Theta -> pi - Theta -- and Phi
        # on the pair halves: N_Theta/2 + N_Phi/2 multiply-adds per point)
        "angular": pts * ((NT + 3 + NP + 1 if eo["angular"] else 4 * NT + 2 * NP) + 2 + 11),
        # dth on the DFS pair, dph, coefficients
        # (square grids: theta folded twice, phi on the pair halves)
        "plane": pts * ((Nt + 3 + Np + 1) if eo["plane"] and plane_square(dims) else
                        ((2 * Nt + 1 if eo["plane"] else 4 * Nt) + 2 * Np)) + pts * 8,
        # dr (centro-antisymmetric halves), r term, Tau row, stage update
        "radial": pts * ((Nr + 1 if eo["radial"] else 2 * Nr) + 10),
    }
    byts = {
        "angular": pts * es * 2,        # read U, write K
        "plane": pts * es * 3,          # read U, read+write K
        "radial": pts * es * 5,         # read U, K, F, Acc; write U (or F) and Acc: 4-6 fields
    }
    # fused stages (float grids): the plane pass writes its terms (read U, write K),
    # the fused pass reads U, K and the stage update's fields: RK4 stages 1..4 move
    # 4, 6, 6, 5 fields (F and K / U, K, F, Acc and U, Acc / ... / U, K, F, Acc and F)
    flops["fused"] = flops["angular"] + flops["radial"]
    byts["plane_store"] = pts * es * 2
    byts["fused"] = pts * es * (4 + 6 + 6 + 5) / 4.0
    return pts, flops, byts


def pass_names(pn):
    """Names of the profiled pass buckets: (angular, plane, radial) for the
    three-pass form, (plane, fused) when the angular bucket is empty (the fused
    angular + radial pass runs in the radial bucket)."""
    if pn[0] == 0 and pn[2] > 0:
        return {1: "plane_store", 2: "fused"}
    return {0: "angular", 1: "plane", 2: "radial"}


KERNEL_OF = {"plane_store": None, "fused": "k_fused"}


def path_bytes_per_update(es):
    """Compulsory bytes per RK4 point-update (F, U, Acc: 17 field accesses)."""
    return 17 * es


# ------------------------------------------------------------- oracle side
def _oracle_task(args):
    """One group of the workload on the CPU oracle: `warm` untimed steps, then
    `nsteps` timed steps. Runs in a spawned process with one BLAS thread."""
    dims, g, warm, nsteps = args
    sys.path.insert(0, ROOT)
    from oracle.transport import Grid, Problem
    from paper_1104_5330_gb300 import inputs as I
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    og = Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=1)
    kap, eta, ks = I.absorber_fields(og.r, og.theta, og.phi, groups=1)
    F = I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, 1104 + g, R1, R2)[None]
    gR1, gR2 = I.inflow_from(F, NT)
    pr = Problem(og, kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(R1, R2, Nr)
    F = pr.run(F, dt, warm)
    t0 = time.perf_counter()
    F = pr.run(F, dt, nsteps)
    return time.perf_counter() - t0, og.points * nsteps


def oracle_rate(dims, warm, nsteps):
    """Point-updates/s of the oracle, one spawned process per group (up to the
    host's cores), all groups concurrently: the slowest process sets the time."""
    G = dims[-1]
    cores = min(G, os.cpu_count() or 1)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_task, [(dims, g, warm, nsteps) for g in range(G)])
    wall = max(r[0] for r in res)
    pts = sum(r[1] for r in res)
    oracle_rate.single = statistics.median(r[1] / r[0] for r in res)   # one process alone
    return pts / wall, wall, cores


# -------------------------------------------------------------------- runs
def run_reference(args, dims, wname):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    rate, wall, cores = oracle_rate(dims, args.warmup, args.steps)
    pts = dims[2] * dims[3] * dims[4] * dims[5] * dims[6] * dims[7]
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "point-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded smooth fields)",
        "config": {"workload": wname, "grid": list(dims[2:7]), "groups": dims[7],
                   "points_per_step": pts},
        "cpu_baseline": {"value": rate, "unit": "point-updates/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{args.steps} RK4 steps of every group of {wname} "
                                   f"(after {args.warmup} untimed), one process per group"},
        "e2e": {"value": rate, "unit": "point-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_differentiation(args, stream):
    """Differentiable stepping on the gradient workload (33 x 16^4, 8 groups,
    FP64, kappa in [0.5, 5]): n forward steps keeping ceil(sqrt(n)) checkpoints,
    then the objective's backward pass (segment recomputation + adjoint steps)
    for the gradients of the outgoing flux at R2 w.r.t. kappa, eta and F0."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    from paper_1104_5330_gb300.autograd import outgoing_flux, transport_steps
    R1, R2, Nr, Nt, Np, NT, NP, G = 0.2, 1.0, 33, 16, 16, 16, 16, 8
    n = args.diff_steps
    gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=ts.TS_FP64)
    r, th, ph, Th, Ph = gg.nodes()
    kap, eta, ks = I.gradient_fields(r, th, ph, G, 1104, R1, R2)
    F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, NT)
    dev = "cuda"
    tk = torch.tensor(kap, device=dev, requires_grad=True)
    te = torch.tensor(eta, device=dev, requires_grad=True)
    tks = torch.tensor(ks, device=dev)
    g1, g2 = torch.tensor(gR1, device=dev), torch.tensor(gR2, device=dev)
    F = torch.tensor(F0, device=dev, requires_grad=True)
    dt = I.dt_rule(R1, R2, Nr)
    # warm-up: one short differentiable run
    out = transport_steps(gg, F, tk, te, tks, dt, 2, g1, g2)
    outgoing_flux(gg, out).sum().backward()
    torch.cuda.synchronize()
    tk.grad = te.grad = F.grad = None
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    out = transport_steps(gg, F, tk, te, tks, dt, n, g1, g2)
    J = outgoing_flux(gg, out).sum()
    e[1].record(stream)
    J.backward()
    e[2].record(stream)
    torch.cuda.synchronize()
    ts.ts_sync_status(gg.handle)
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    pts = gg.points
    finite = bool(torch.isfinite(tk.grad).all() and torch.isfinite(te.grad).all())
    return {"workload": "gradient_33x16^4_g8", "steps": n,
            "checkpoint_segment": int(np.ceil(np.sqrt(n))),
            "value": pts * n / ((fwd_ms + bwd_ms) * 1e-3), "unit": "point-updates/s",
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "backward_point_updates_per_s": pts * n / (bwd_ms * 1e-3),
            "dtype": "f64", "objective": "outgoing flux at R2, all groups",
            "grad_norms": {"kappa": float(tk.grad.norm()), "eta": float(te.grad.norm())},
            "finite": finite}


def run_batch(args, stream):
    """The uneven batch: 64 seeded problems (N_r in {17,33,65}, angular N in
    {8,16,24} per axis, 1..24 groups, kappa scale U[0.1,100]); FP32 storage and
    angular contractions, FP64 radial rows near the ends, split scheme with the
    FP64 implicit collision step; problems below 2^22 points share one
    persistent launch per pass, the larger ones run their grid's own (compiled)
    passes; the step is graph-captured. Initial data: the Gaussian shell, zero
    inflow."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I

    specs = I.batch_problems(64, 1104)
    descs = [ts.GridDesc(s.R1, s.R2, s.Nr, s.Ntheta, s.Nphi, s.NTheta, s.NPhi, s.groups,
                         ts.TS_FP32_R64, ts.TS_RK4_SPLIT_IMPLICIT, ts.TS_BC_TAU_INFLOW, 0, 36.0, 16)
             for s in specs]
    t0 = time.perf_counter()
    b = ts.Batch(descs, autotune=True)
    t_setup = time.perf_counter() - t0
    Fs, dts = [], []
    for s, g in zip(specs, b.grids):
        r, th, ph, Th, Ph = g.nodes()
        kap, eta, ks = I.batch_fields(s, r, th, ph)
        g.set_coeffs(kap, eta, ks)
        rr = torch.as_tensor(r, device="cuda").view(1, -1, 1, 1, 1, 1)
        ct = torch.cos(torch.as_tensor(Th, device="cuda")).view(1, 1, 1, 1, -1, 1)
        F = (torch.exp(-((rr - 0.6) / 0.1) ** 2) * (1 + 0.5 * ct)).expand(g.shape)
        F = F.to(torch.float32).contiguous()
        g.apply_inflow(F)
        Fs.append(F)
        dts.append(I.dt_rule(s.R1, s.R2, s.Nr))
    pts = b.points
    b.step(Fs, dts, 3)              # graph capture + warm-up
    torch.cuda.synchronize()
    # check: the two smallest problems stepped alone on their own grids from the
    # same state must agree with the batch to FP32 rounding
    small = sorted(range(len(specs)), key=lambda q: b.grids[q].points)[:2]
    ref = {q: Fs[q].clone() for q in small}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(Fs, dts, args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    finite = all(bool(torch.isfinite(F).all()) for F in Fs)
    agree = {}
    for q in small:
        b.grids[q].step(ref[q], dts[q], args.batch_steps)
        torch.cuda.synchronize()
        agree[f"problem_{q}"] = float(torch.linalg.vector_norm((Fs[q] - ref[q]).double()) /
                                      torch.linalg.vector_norm(ref[q].double()))
    own = [g.points >= (1 << 22) for g in b.grids]
    launches = 13 * sum(own) + (13 if not all(own) else 0)   # 4 stages x 3 passes + collision
    out = {"value": pts * args.batch_steps / (ms * 1e-3), "unit": "point-updates/s",
           "ms_per_step": ms / args.batch_steps, "steps": args.batch_steps,
           "problems": len(specs), "points_per_step": pts, "dtype": "f32 (+f64 radial end rows, f64 collision)",
           "scheme": "RK4 streaming + implicit collision", "setup_s_incl_autotune": t_setup,
           "launches_per_step": launches, "problems_on_own_passes": int(sum(own)),
           "finite": finite,
           "rel_l2_vs_single_problem_steps": agree}
    del Fs
    b.close()
    # the same 64 problems under TS_AB2 (one stage derivative per step, explicit
    # collision, dt = 0.2 h_min): the batch keeps its history across calls
    descs = [ts.GridDesc(s.R1, s.R2, s.Nr, s.Ntheta, s.Nphi, s.NTheta, s.NPhi, s.groups,
                         ts.TS_FP32_R64, ts.TS_AB2, ts.TS_BC_TAU_INFLOW, 0, 36.0, 16)
             for s in specs]
    b = ts.Batch(descs, autotune=True)
    Fs, dts = [], []
    for s, g in zip(specs, b.grids):
        r, th, ph, Th, Ph = g.nodes()
        kap, eta, ks = I.batch_fields(s, r, th, ph)
        g.set_coeffs(kap, eta, ks)
        rr = torch.as_tensor(r, device="cuda").view(1, -1, 1, 1, 1, 1)
        ct = torch.cos(torch.as_tensor(Th, device="cuda")).view(1, 1, 1, 1, -1, 1)
        F = (torch.exp(-((rr - 0.6) / 0.1) ** 2) * (1 + 0.5 * ct)).expand(g.shape)
        F = F.to(torch.float32).contiguous()
        g.apply_inflow(F)
        Fs.append(F)
        dts.append(0.5 * I.dt_rule(s.R1, s.R2, s.Nr))
    b.step(Fs, dts, 3)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(Fs, dts, args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms2 = e0.elapsed_time(e1)
    out["ab2"] = {"value": pts * args.batch_steps / (ms2 * 1e-3), "unit": "point-updates/s",
                  "ms_per_step": ms2 / args.batch_steps, "steps": args.batch_steps,
                  "scheme": "AB2 (one stage derivative per step), dt = 0.2 h_min",
                  "finite": all(bool(torch.isfinite(F).all()) for F in Fs)}
    del Fs
    b.close()
    return out


def run_anisotropic(args, dims, stream):
    """The default grid with neutrino scattering on a neutron / proton mixture:
    kernel (kappa_s/4pi)(1 + b omega.omega'), kappa_s = 4 pi (A_n + A_p),
    b = -(A_n/3 + A_p/10)/(A_n + A_p) from seeded smooth amplitude fields, FP64,
    RK4 + Tau rows; and the same grid with Thomson scattering (3/16pi)(1 + mu^2)
    (c = 3/4) on the mixture's kappa_s. Reports the step rates and the angular
    pass's per-launch time beside that of the isotropic form on the same grid."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=ts.TS_FP64)
    r, th, ph, Th, Ph = gg.nodes()
    kap, eta, _ = I.absorber_fields(r, th, ph, groups=G)
    ks, b = ts.nucleon_scattering(*I.nucleon_densities(r, th, ph, G, 1104, R1, R2))
    F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, NT)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(R1, R2, Nr)
    F = torch.as_tensor(F0, dtype=torch.float64, device="cuda").contiguous()
    out = {}
    for name, bb, cc in (("isotropic", None, None), ("anisotropic", b, None),
                         ("thomson", None, 0.75)):
        gg.set_scattering_anisotropy(bb)
        gg.set_scattering_quadrupole(cc)
        gg.step(F, dt, args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gg.step(F, dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        pm, pn = ts.ts_step_profile(gg.handle, F, dt, max(2, min(args.steps, 10)))
        out[name] = (gg.points * args.steps / (ms * 1e-3), ms / args.steps, pm[0] / pn[0])
    ts.ts_sync_status(gg.handle)
    v, msps, ang = out["anisotropic"]
    return {"value": v, "unit": "point-updates/s", "ms_per_step": msps, "dtype": "f64",
            "workload": f"nucleon mixture on {Nr}x{Nt}x{Np}x{NT}x{NP}, {G} groups",
            "b_range": [float(b.min()), float(b.max())],
            "kappa_s_range": [float(ks.min()), float(ks.max())],
            "angular_ms_per_launch": ang,
            "isotropic_same_grid": {"value": out["isotropic"][0],
                                    "angular_ms_per_launch": out["isotropic"][2]},
            "thomson_same_grid": {"value": out["thomson"][0], "ms_per_step": out["thomson"][1],
                                  "angular_ms_per_launch": out["thomson"][2],
                                  "kernel": "(3/16pi)(1 + mu^2): b = 0, c = 3/4"}}


def run_ab2(args, dims, stream, rk4_ms_per_step):
    """The default workload with the paper's second-order Adams-Bashforth
    marching (one stage derivative per step) at dt = 0.2 x the smallest radial
    spacing (its stability limit on these grids; RK4 runs at 0.4). Reports the
    step rate and the simulated time advanced per second against RK4's."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=ts.TS_FP64, scheme=ts.TS_AB2)
    r, th, ph, Th, Ph = gg.nodes()
    kap, eta, ks = I.absorber_fields(r, th, ph, groups=G)
    F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, NT)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(R1, R2, Nr, 0.2)
    F = torch.as_tensor(F0, dtype=torch.float64, device="cuda").contiguous()
    gg.step(F, dt, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 4 * args.steps
    e0.record(stream)
    gg.step(F, dt, n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ts.ts_sync_status(gg.handle)
    dt_rk4 = I.dt_rule(R1, R2, Nr)
    return {"value": gg.points * n / (ms * 1e-3), "unit": "point-updates/s",
            "ms_per_step": ms / n, "steps": n, "dtype": "f64", "dt": dt,
            "launches_per_step": 3,
            "simulated_time_rate_vs_rk4": (dt / (ms / n)) / (dt_rk4 / rk4_ms_per_step)}


def run_hybrid(args, stream, zoned=False):
    """The 5-D shell run of Sect. 5.3 on the hybrid grid (first-order upwind
    differences in r on 129 uniform nodes, spectral angular axes 16 x 16 x 24 x 16,
    one group, FP64, RK4 at dt = 0.4 dr): empty shell 0.5 <= r <= 1, Lambert
    emission F0 cos(Theta) at R1, coherent scattering of optical depth 5 from a
    plasma vanishing at R2. Reports the step rate and the radial pass's time.
    zoned: the same shell on the three-zone grid of App. B (30 + 65 + 30 radial
    nodes, edge zones of width 0.1 (R2 - R1)), dt = 0.4 x the smallest spacing."""
    import numpy as np
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    R1, R2, Nr, Nt, Np, NT, NP = 0.5, 1.0, 123 if zoned else 129, 16, 16, 24, 16
    if zoned:
        gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=1, precision=ts.TS_FP64,
                     radial=ts.TS_RADIAL_ZONED, zone_nodes=30, zone_width=0.1)
    else:
        gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=1, precision=ts.TS_FP64,
                     radial=ts.TS_RADIAL_UPWIND_FD)
    r, th, ph, Th, Ph = gg.nodes()
    ks = I.shell_scattering(r, th, ph, R1, R2, 5.0)
    gR1, gR2 = I.lambert_inflow(Th, Nt, Np, NP)
    gg.set_coeffs(None, None, ks, gR1, gR2)
    dt = 0.4 * float(np.diff(r).min())
    F = gg.apply_inflow(torch.zeros(gg.shape, dtype=torch.float64, device="cuda"))
    gg.step(F, dt, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gg.step(F, dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pm, pn = ts.ts_step_profile(gg.handle, F, dt, max(2, min(args.steps, 10)))
    ts.ts_sync_status(gg.handle)
    return {"value": gg.points * args.steps / (ms * 1e-3), "unit": "point-updates/s",
            "ms_per_step": ms / args.steps, "dtype": "f64",
            "workload": f"Lambert shell, optical depth 5, {Nr}x{Nt}x{Np}x{NT}x{NP}, 1 group",
            "radial": ("30 + 65 + 30 nodes: upwind differences in edge zones of width "
                       "0.1 (R2 - R1), Chebyshev in the central zone" if zoned else
                       "first-order upwind differences on uniform nodes"),
            "dt": dt,
            "pass_ms_per_launch": {n: float(pm[a] / pn[a])
                                   for a, n in enumerate(("angular", "plane", "radial"))}}


def run_cons5d(args, dims, stream, adv_ms_per_step):
    """The conservative form of App. A (Eq. Cohercons) on the default grid: the
    absorber workload carried as Fhat = r^2 sin(th) sin(Th) F (inflow J g), FP64
    RK4 at dt = 0.4 h_min; the step rate, each pass's time and the rate against
    the advective form's. Then the number balance of both forms on the Lambert
    shell of Sect. 5.3 on the same grid (empty shell 0.2 <= r <= 1, emission
    F0 cos Th at R1, a spherically symmetric scattering plasma vanishing at R2,
    optical depths 0.5, 2, 5, 10 over the four groups), 100 RK4 steps each:
    |dN/dt + J_R2 - J_R1| of the operator relative to the fluxes."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=ts.TS_FP64,
                 form=ts.TS_FORM_CONSERVATIVE)
    r, th, ph, Th, Ph = gg.nodes()
    J = (r[:, None, None, None, None] ** 2 * np.sin(th)[None, :, None, None, None]
         * np.sin(Th)[None, None, None, :, None])
    kap, eta, ks = I.absorber_fields(r, th, ph, groups=G)
    F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, NT)
    h = NT // 2
    gg.set_coeffs(kap, eta, ks, gR1 * J[None, 0, :, :, :h], gR2 * J[None, -1, :, :, h:])
    dt = I.dt_rule(R1, R2, Nr)
    X = torch.as_tensor(J[None] * F0, dtype=torch.float64, device="cuda").contiguous()
    gg.step(X, dt, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gg.step(X, dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pm, pn = ts.ts_step_profile(gg.handle, X, dt, max(2, min(args.steps, 10)))
    ts.ts_sync_status(gg.handle)
    gg.close()
    # number balance of both forms on the Lambert shell
    prof = 9.0 / (R2 - R1) * (1.0 - (r - R1) / (R2 - R1)) ** 8
    taus = np.array([0.5, 2.0, 5.0, 10.0][:G] + [5.0] * max(0, G - 4))
    ksh = np.ascontiguousarray(np.broadcast_to(
        (taus[:, None] * prof[None, :])[:, :, None, None], (G, Nr, Nt, Np)))
    lR1, lR2 = I.lambert_inflow(Th, Nt, Np, NP, groups=G)
    res = {}
    for name, form in (("conservative", ts.TS_FORM_CONSERVATIVE),
                       ("advective", ts.TS_FORM_ADVECTIVE)):
        gs = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=ts.TS_FP64, form=form)
        w1, w2 = (J[None, 0, :, :, :h], J[None, -1, :, :, h:]) if name == "conservative" else (1, 1)
        gs.set_coeffs(None, None, ksh, lR1 * w1, lR2 * w2)
        Y = gs.apply_inflow(torch.zeros(gs.shape, dtype=torch.float64, device="cuda"))
        gs.step(Y, dt, 100)
        N, J1, J2, dN, S = gs.number_balance(Y).T
        res[name] = float(np.max(np.abs(dN + J2 - J1 - S) / (np.abs(J1) + np.abs(J2))))
        res[name + "_N"] = [float(v) for v in N]
        gs.close()
    return {"value": gg.points * args.steps / (ms * 1e-3), "unit": "point-updates/s",
            "ms_per_step": ms / args.steps, "steps": args.steps, "dtype": "f64", "dt": dt,
            "workload": "absorber, Fhat = r^2 sin th sin Th F, " + "x".join(map(str, dims[2:7]))
                        + f", {G} groups",
            "rate_vs_advective": adv_ms_per_step / (ms / args.steps),
            "pass_ms_per_launch": {n: float(pm[a] / pn[a])
                                   for a, n in enumerate(("angular", "plane", "radial"))},
            "balance": {"workload": "Lambert shell, optical depths 0.5, 2, 5, 10, 100 RK4 steps",
                        "residual_rel_max": {"conservative": res["conservative"],
                                             "advective": res["advective"]},
                        "N": {"conservative": res["conservative_N"],
                              "advective": res["advective_N"]}}}


def variant_line(ts, dims, wname, vname, vprec, pts, steps, ms, err, nv, pm, pn, peaks, sms,
                 smax):
    """Rate, error and per-pass roofline of one float variant: the dominant
    kernel's algorithmic bytes over its average launch time (CUDA events on the
    launching stream), and the path fraction 17 s x rate / HBM peak."""
    names = pass_names(pn)
    _, fl, by = pass_work(dims, 4)
    per = {n: pm[a] / pn[a] for a, n in names.items() if pn[a] > 0}
    tot = sum(pm[a] for a in names)
    dom = max(per, key=lambda n: pm[[a for a, m in names.items() if m == n][0]])
    avg = per[dom]
    hbm = by[dom] / (avg * 1e-3) / 1e9
    if dom == "fused":
        kn = "k_fused<float>"
    elif dom == "plane_store":
        kn = "plane pass (store form)"
    else:
        kf = eo_kernel(dom, dims) if even_odd_passes(dims, 4)[dom] else f"k_{dom}"
        kn = ("k_radial_tc" if dom == "radial" and vprec in (ts.TS_TF32X3, ts.TS_BF16X3)
              else kf) + "<float>"
    rate = pts * steps / (ms * 1e-3)
    return {"value": rate, "unit": "point-updates/s", "ms_per_step": ms / steps, "dtype": "f32",
            "rel_l2_vs_gpu_fp64": err, "after_steps": nv,
            "path_fraction_of_hbm": path_bytes_per_update(4) * rate / 1e9 / peaks["hbm_gbs"],
            "roofline": {"bound": "hbm", "kernel": kn, "achieved": hbm, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
                         "traffic": _traffic(dom, wname, vname),
                         "fp32_alu_tflops": fl.get(dom if dom != "plane_store" else "plane", 0) /
                         (avg * 1e-3) / 1e12,
                         "fp32_alu_peak_tflops": sms * 2 * FP32_FMA_PER_SM_CLK * smax * 1e6 / 1e12,
                         "pass_share": {n: float(pm[a] / tot) for a, n in names.items()},
                         "pass_ms_per_launch": {n: float(v) for n, v in per.items()},
                         "algorithmic_bytes_per_launch": by[dom]}}


def run_cons2d(args, stream, zoned=False):
    """The conservative 2-D variant of App. B (Fhat = r^2 sin Th F, Eq. speccons)
    on its shell problem: 0.5 <= r <= 1, empty at t = 0, Fhat(R1, Th) =
    cos Th sin Th on the outgoing directions, Thomson scattering (c = 3/4) from
    a plasma vanishing at R2, kappa_s = 9 tau/(R2 - R1) (1 - (r - R1)/(R2 - R1))^8;
    2048 independent problems with optical depths tau log-spaced over [0.1, 10],
    65 x 24 nodes each (the paper: 65 spectral radial points and 25 in Theta),
    RK4 at dt = 0.4 h_min, every step of a call in one launch. Reports the rate
    and the operator's discrete number balance |dN/dt + J_R2 - J_R1| relative to
    the fluxes after the run (zero to rounding: Eq. Cons). zoned: the paper's
    three-zone radial grid of App. B, 30 + 25 + 30 nodes (edge zones of width
    0.1 (R2 - R1); N_r = 83), dt = 0.4 x the smallest spacing; its balance holds
    up to the edge zones' first-order differences."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    P, Nr, NT, R1, R2 = 2048, (83 if zoned else 65), 24, 0.5, 1.0
    tau = np.logspace(-1, 1, P)
    zk = dict(radial=ts.TS_RADIAL_ZONED, zone_nodes=30, zone_width=0.1) if zoned else {}
    g = ts.Cons2D(R1, R2, Nr, NT, problems=P, scatter_c=0.75, **zk)
    r, th = g.nodes()
    ks = 9 * tau[:, None] / (R2 - R1) * (1 - (r[None, :] - R1) / (R2 - R1)) ** 8
    g1 = np.tile(np.cos(th[:NT // 2]) * np.sin(th[:NT // 2]), (P, 1))
    g.set_coeffs(ks, g1, None)
    X = g.apply_inflow(torch.zeros((P, Nr, NT), dtype=torch.float64, device="cuda"))
    dt = 0.4 * float(np.diff(r).min())   # the smallest spacing (Gauss-Lobatto or zoned)
    g.step(X, dt, args.warmup)
    torch.cuda.synchronize()
    n = 10 * args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(X, dt, n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    gb = ts.Cons2D(R1, R2, Nr, NT, problems=P, scatter_c=0.75, bc=ts.TS_BC_NONE, **zk)
    gb.set_coeffs(ks, g1, None)
    NJ, res = gb.balance(X)
    NJ, res = NJ.cpu().numpy(), res.cpu().numpy()
    scale = np.abs(NJ[:, 1:]).max(axis=1) + np.abs(NJ[:, 0]).max() * 1e-300
    pts = P * Nr * NT
    out = {"value": pts * n / (ms * 1e-3), "unit": "point-updates/s", "ms_per_step": ms / n,
           "steps": n, "dt": dt, "problems": P, "grid": [Nr, NT], "dtype": "f64",
           "launches_per_call": 1, "workload": "App. B shell: Lambert inflow at R1, Thomson scattering, tau in [0.1, 10]",
           "balance_residual_rel_max": float(np.max(np.abs(res) / scale)),
           "N_range": [float(NJ[:, 0].min()), float(NJ[:, 0].max())]}
    if zoned:
        out["radial"] = ("30 + 25 + 30 nodes: upwind differences in edge zones of width 0.1 "
                         "(R2 - R1), Chebyshev in the central zone")
    g.close()
    gb.close()
    return out


def run_workload_precisions(args, wname, stream, precisions, nv):
    """Rates of `precisions` on another workload of the same family (absorber,
    seeded smooth F0, static inflow, RK4 at dt = 0.4 h_min), and each float
    variant's relative L2 distance to the GPU FP64 result after nv steps.
    "fp64+filter": FP64 with the exponential filter on every axis after each
    step (alpha 36, order 16), its change against the unfiltered FP64 result and
    the filter's own time per launch."""
    import torch
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I
    dims = WORKLOADS[wname]
    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    dt = I.dt_rule(R1, R2, Nr)
    peaks, _ = _peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    smax = peaks.get("sm_max_mhz", 2070.0)
    out = {"workload": wname, "grid": [Nr, Nt, Np, NT, NP], "groups": G, "dt": dt,
           "steps": args.steps}
    ref = None
    for name in precisions:
        base, _, opt = name.partition("+")
        filt = opt == "filter"
        prec = getattr(ts, PRECISIONS[base])
        gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=prec, filter_on=filt)
        r, th, ph, Th, Ph = gg.nodes()
        kap, eta, ks = I.absorber_fields(r, th, ph, groups=G)
        F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
        gR1, gR2 = I.inflow_from(F0, NT)
        gg.set_coeffs(kap, eta, ks, gR1, gR2)
        F = torch.as_tensor(F0, dtype=gg.dtype, device="cuda").contiguous()
        gg.step(F, dt, nv)
        if prec == ts.TS_FP64 and not filt:
            ref = F.clone()
            err = None
        else:
            err = float(torch.linalg.vector_norm(F.double() - ref) / torch.linalg.vector_norm(ref))
        gg.step(F, dt, args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gg.step(F, dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ts.ts_sync_status(gg.handle)
        pm, pn = ts.ts_step_profile(gg.handle, F, dt, 2)
        if prec == ts.TS_FP64:
            out[name] = {"value": gg.points * args.steps / (ms * 1e-3), "unit": "point-updates/s",
                         "ms_per_step": ms / args.steps, "dtype": "f64",
                         "pass_ms_per_launch": {n: float(pm[a] / pn[a])
                                                for a, n in pass_names(pn).items()}}
            if filt:
                out[name]["filter"] = "exponential, alpha 36, order 16, every axis, after each step"
                out[name]["filter_ms_per_step"] = float(pm[3] / 2)   # two profiled steps
                out[name]["rel_l2_change_vs_unfiltered_fp64"] = err
        else:
            out[name] = variant_line(ts, dims, wname, name, prec, gg.points, args.steps, ms, err,
                                     nv, pm, pn, peaks, sms, smax)
        del gg, F
        torch.cuda.empty_cache()
    return out


def run_ours(args, dims, wname):
    import torch
    import torch.distributed as dist

    rank, local, world = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1104_5330_gb300 import build as b
    if rank == 0:
        b.build()
    if world > 1:
        dist.barrier()
    import paper_1104_5330_gb300.ts as ts
    from paper_1104_5330_gb300 import inputs as I

    R1, R2, Nr, Nt, Np, NT, NP, G = dims
    prec = getattr(ts, PRECISIONS[args.precision])
    tdt = torch.float64 if prec == ts.TS_FP64 else torch.float32
    es = 8 if prec == ts.TS_FP64 else 4

    def make(precision):
        gg = ts.Grid(R1, R2, Nr, Nt, Np, NT, NP, groups=G, precision=precision)
        r, th, ph, Th, Ph = gg.nodes()
        kap, eta, ks = I.absorber_fields(r, th, ph, groups=G)
        F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, 1104 + g, R1, R2) for g in range(G)])
        gR1, gR2 = I.inflow_from(F0, NT)
        gg.set_coeffs(kap, eta, ks, gR1, gR2)
        return gg, F0

    gg, F0 = make(prec)
    dt = I.dt_rule(R1, R2, Nr)
    pts = gg.points
    F = torch.as_tensor(F0, dtype=tdt, device="cuda").contiguous()
    stream = torch.cuda.current_stream()

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    gg.step(F, dt, args.warmup)
    sync_all()
    with ClockSampler(local) as clk:
        sync_all()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gg.step(F, dt, args.steps)
        e1.record(stream)
        sync_all()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    value = job_rate(pts * args.steps, world, ms)

    # per-pass device time (CUDA events on the launching stream)
    nprof = max(2, min(args.steps, 10))
    pass_ms, pass_n = ts.ts_step_profile(gg.handle, F, dt, nprof)
    bucket = pass_names(pass_n)
    names = [bucket[a] for a in sorted(bucket)]
    launches = int(sum(pass_n)) * args.steps // nprof   # every kernel of a step
    _, flops, byts = pass_work(dims, es)
    flops["plane_store"] = flops["plane"]
    tot = sum(pass_ms[a] for a in bucket)
    shares = [pass_ms[a] / tot for a in sorted(bucket)]
    dom = max(bucket, key=lambda a: pass_ms[a])
    dname = bucket[dom]
    avg_ms = pass_ms[dom] / pass_n[dom]
    peaks, peak_src = _peaks()
    if dname in KERNEL_OF:
        kfam = KERNEL_OF[dname] or "k_plane_sq"
    else:
        kfam = eo_kernel(dname, dims) if even_odd_passes(dims, es)[dname] else f"k_{dname}"
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    smax = peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = sms * 2 * FP64_FMA_PER_SM_CLK * smax * 1e6 / 1e12
    if prec == ts.TS_FP64:
        achieved = flops[dname] / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": f"{kfam}<double>", "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "peak_source": f"derived: {sms} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA/clk x 2 flop "
                               f"x {smax:.0f} MHz",
                "measured_dfma_loop_tflops": ts.ts_probe_fma_rate(ts.TS_FP64),
                "algorithmic_flops_per_launch": flops[dname],
                "traffic": _traffic(dname, wname, args.precision),
                "algorithmic_bytes_per_launch": byts[dname],
                "hbm_achieved_gbs": byts[dname] / (avg_ms * 1e-3) / 1e9}
    else:
        achieved = byts[dname] / (avg_ms * 1e-3) / 1e9
        if prec in (ts.TS_TF32X3, ts.TS_BF16X3) and dname == "radial":
            kfam = "k_radial_tc"
        roof = {"bound": "hbm", "kernel": f"{kfam}<float>", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{peak_src} hbm_gbs",
                "fp32_alu_tflops": flops[dname] / (avg_ms * 1e-3) / 1e12,
                "fp32_alu_peak_tflops": sms * 2 * FP32_FMA_PER_SM_CLK * smax * 1e6 / 1e12,
                "algorithmic_bytes_per_launch": byts[dname],
                "traffic": _traffic(dname, wname, args.precision)}
    roof["avg_launch_ms"] = avg_ms
    roof["pass_share"] = {n: float(s) for n, s in zip(names, shares)}

    line = {
        "metric": METRIC, "value": value, "unit": "point-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == ts.TS_FP64 else "f32",
        "data": "synthetic (seeded smooth fields; no dataset)",
        "config": {"workload": wname, "grid": [Nr, Nt, Np, NT, NP], "groups": G,
                   "R": [R1, R2], "dt": dt, "scheme": "RK4 + Tau inflow rows",
                   "points_per_step": pts,
                   "l2": f"inputs larger than L2: working set {4 * pts * es / 1e6:.0f} MB > 129 MB",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }

    # end to end through the host-buffer entry point (copies inside the timed region)
    if not args.skip_e2e:
        Fh = torch.as_tensor(F0, dtype=tdt).contiguous().pin_memory()
        ts.ts_step_host(gg.handle, Fh, dt, 1)
        ne = max(3, min(args.steps, 10))
        sync_all()
        t0 = time.perf_counter()
        for _ in range(ne):
            ts.ts_step_host(gg.handle, Fh, dt, 1)
        sync_all()
        te = time.perf_counter() - t0
        nbytes = pts * es
        line["e2e"] = {"value": pts * ne * world / te, "unit": "point-updates/s",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                       "steps": ne, "api": "ts_step_host (pinned host F, one step per call)"}

    # the FP32 variant and the adjoint, same workload (rank 0 reports them)
    if not args.skip_variants:
        ref = torch.as_tensor(F0, dtype=torch.float64, device="cuda").contiguous()
        nv = max(2, min(args.steps, 10))
        gg.step(ref, dt, nv)
        line["variants"] = {}
        kname = {"radial": "k_radial_tc"}
        for vname, vprec in (("fp32", ts.TS_FP32), ("fp32_r64", ts.TS_FP32_R64),
                             ("tf32x3_tensorcore_radial", ts.TS_TF32X3),
                             ("bf16x3_tensorcore_radial", ts.TS_BF16X3)):
            g32, _ = make(vprec)
            F32 = torch.as_tensor(F0, dtype=torch.float32, device="cuda").contiguous()
            g32.step(F32, dt, nv)
            err32 = float(torch.linalg.vector_norm(F32.double() - ref) / torch.linalg.vector_norm(ref))
            F32b = F32.clone()
            g32.step(F32b, dt, 2)
            torch.cuda.synchronize()
            e0.record(stream)
            g32.step(F32b, dt, args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.ts_sync_status(g32.handle)
            ms32 = e0.elapsed_time(e1)
            pm, pn = ts.ts_step_profile(g32.handle, F32b, dt, nv)
            line["variants"][vname] = variant_line(ts, dims, wname, vname, vprec, pts,
                                                   args.steps, ms32, err32, nv, pm, pn, peaks,
                                                   sms, smax)
            del g32, F32, F32b
        lam = torch.randn_like(F)
        gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
        ge = torch.zeros_like(gk)
        gg.adjoint_step(F, lam, gk, ge, dt)
        torch.cuda.synchronize()
        na = max(2, min(args.steps, 5))
        e0.record(stream)
        for _ in range(na):
            gg.adjoint_step(F, lam, gk, ge, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        msa = e0.elapsed_time(e1)
        line["adjoint"] = {"value": pts * na / (msa * 1e-3), "unit": "point-updates/s",
                           "ms_per_step": msa / na, "dtype": "f64",
                           "includes": "forward recomputation of the stage inputs"}

    if not args.skip_workloads:
        # the vacuum-free grid of the free-streaming check (17 x 8^4, 1 group) and the
        # precision grid (65 x 32^4, 1 group: 68M points) with every precision
        line["workload_17x8^4_g1"] = run_workload_precisions(
            args, "absorber_17x8^4_g1", stream, ["fp64", "fp32"], 10)
        line["precision_65x32^4_g1"] = run_workload_precisions(
            args, "absorber_65x32^4_g1", stream,
            ["fp64", "fp32", "fp32_r64", "tf32x3", "bf16x3", "fp64+filter"], 10)
    if not args.skip_workloads:
        line["conservative_2d"] = run_cons2d(args, stream)
        line["conservative_2d_zoned"] = run_cons2d(args, stream, zoned=True)
        line["conservative_5d"] = run_cons5d(args, dims, stream, ms / args.steps)
    if not args.skip_aniso:
        line["anisotropic_scattering"] = run_anisotropic(args, dims, stream)
        line["ab2"] = run_ab2(args, dims, stream, ms / args.steps)
        line["hybrid_radial_fd"] = run_hybrid(args, stream)
        line["zoned_radial"] = run_hybrid(args, stream, zoned=True)
    if not args.skip_batch:
        line["batch"] = run_batch(args, stream)
    if not args.skip_diff and args.diff_steps > 0:
        line["differentiation"] = run_differentiation(args, stream)

    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        rate, wall, cores = oracle_rate(dims, 0, 3)
        line["cpu_baseline"] = {"value": rate, "unit": "point-updates/s", "cores": cores,
                                "kind": "oracle",
                                "single_thread_value": oracle_rate.single,
                                "sample": f"3 RK4 steps of each of the {G} groups of {wname} "
                                          f"({wall:.1f} s wall, one process per group)"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="absorber_33x16^4_g4")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-aniso", action="store_true")
    ap.add_argument("--skip-workloads", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--skip-diff", action="store_true")
    ap.add_argument("--diff-steps", type=int, default=200)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)      # timing rule: at least 3 untimed steps
    dims = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, dims, args.workload)
    return run_ours(args, dims, args.workload)


if __name__ == "__main__":
    sys.exit(main())
