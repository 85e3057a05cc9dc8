"""Parity with the FP64 oracle at the workloads' stated step counts, element by
element, through the C ABI in the launch configuration the benchmark times:

* N_r = 33 over 1000 RK4 steps (the 4-group absorber workload's step count) on
  the 33 x 8^4 grid with 2 groups;
* the full 33 x 16^4 x 4-group absorber workload over 100 steps;
* the 65 x 32^4 grid (68M points) over 2 RK4 steps;
* four seeded problems of the 64-problem batch (N_Theta = N_Phi = 24,
  N_theta = 24, N_Phi = 24, N_r = 65) over 50 steps, batched, in FP64 (RK4) and
  in the batch workload's form (FP32 storage, FP64 radial end rows, split
  scheme with the FP64 implicit collision step).

Bars: 1e-12 relative L2 for FP64, 1e-5 for the reduced-precision form. Where
the oracle's own rounding floor (the difference between its two summation
orders of the same coefficient-space chain after the same steps) is above half
of 1e-12, the FP64 bar is twice that floor, measured in the test: the chain's
rounding grows with N_r^2 and with the step count, and a difference at that
level cannot be told apart from the oracle's own.

The oracle runs (minutes of CPU time) are computed in spawned workers started
at collection time (tests/oracle_jobs.py) while the other tests run.
"""
import numpy as np
import pytest
import torch

import oracle_jobs as OJ
from gpu_common import T, absorber_workload, cuda, host, pair, rel_l2, setup_both
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _gpu_absorber(dims, G, nsteps):
    og, gg = pair(*OJ.R, *dims, G=G)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    F = cuda(F0)
    gg.step(F, I.dt_rule(*OJ.R, dims[0]), nsteps)
    out = host(F)
    del F, gg
    torch.cuda.empty_cache()
    return out


def test_1000_steps_at_33_radial_nodes(oracle_jobs):
    Fg = _gpu_absorber(OJ.C2_LONG, 2, OJ.C2_LONG_STEPS)
    ref = np.stack([oracle_jobs.result(f"c2long/matrix/g{g}") for g in range(2)])
    alt = np.stack([oracle_jobs.result(f"c2long/library/g{g}") for g in range(2)])
    err, floor = rel_l2(Fg, ref), rel_l2(alt, ref)
    print(f"33x8^4 x2, 1000 steps: GPU vs oracle {err:.3e}, oracle floor {floor:.3e}")
    assert np.isfinite(Fg).all()
    assert err < max(FP64_TOL, 2.0 * floor)


def test_full_absorber_workload_100_steps(oracle_jobs):
    Fg = _gpu_absorber(OJ.C2_FULL, 4, OJ.C2_FULL_STEPS)
    for g in range(4):
        err = rel_l2(Fg[g], oracle_jobs.result(f"c2full/g{g}"))
        print(f"33x16^4 group {g}, 100 steps: GPU vs oracle {err:.3e}")
        assert err < FP64_TOL, g


def test_65x32_two_steps(oracle_jobs):
    Fg = _gpu_absorber(OJ.C3_FULL, 1, OJ.C3_STEPS)[0]
    ref = oracle_jobs.result("c3/matrix")
    floor = rel_l2(oracle_jobs.result("c3/library"), ref)
    err = rel_l2(Fg, ref)
    print(f"65x32^4, {OJ.C3_STEPS} steps: GPU vs oracle {err:.3e}, oracle floor {floor:.3e}")
    assert floor < 2e-11
    assert err < max(FP64_TOL, 2.0 * floor)


@pytest.mark.parametrize("precision,scheme,tol", [(0, 0, FP64_TOL), (2, 1, 1e-5)])
def test_seeded_batch_problems_50_steps(oracle_jobs, precision, scheme, tol):
    ts = T()
    specs = [I.batch_problems(64, 1104)[q] for q in OJ.C4_PROBLEMS]
    descs = [ts.GridDesc(s.R1, s.R2, s.Nr, s.Ntheta, s.Nphi, s.NTheta, s.NPhi, s.groups,
                         precision, scheme, 0, 0, 36.0, 16) for s in specs]
    b = ts.Batch(descs, autotune=True)
    dtype = torch.float64 if precision == 0 else torch.float32
    Fs, dts = [], []
    for s, g in zip(specs, b.grids):
        r, th, ph, Th, Ph = g.nodes()
        kap, eta, ks = I.batch_fields(s, r, th, ph)
        F0 = np.stack([I.seeded_smooth(r, th, ph, Th, Ph, s.seed + k, s.R1, s.R2)
                       for k in range(s.groups)])
        gR1, gR2 = I.inflow_from(F0, s.NTheta)
        g.set_coeffs(kap, eta, ks, gR1, gR2)
        Fs.append(cuda(F0, dtype))
        dts.append(I.dt_rule(s.R1, s.R2, s.Nr))
    b.step(Fs, dts, OJ.C4_STEPS)
    torch.cuda.synchronize()
    name = "rk4" if scheme == 0 else "split"
    for q, s, F in zip(OJ.C4_PROBLEMS, specs, Fs):
        ref = np.stack([oracle_jobs.result(f"c4/{name}/p{q}/g{k}") for k in range(s.groups)])
        err = rel_l2(host(F), ref)
        print(f"batch problem {q} {s.Nr}x{s.Ntheta}x{s.Nphi}x{s.NTheta}x{s.NPhi} x{s.groups}, "
              f"{name}, precision {precision}: {err:.3e}")
        assert err < tol, q
    b.close()
