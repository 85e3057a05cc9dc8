"""Batched steps of uneven problems (one persistent launch per pass over the
tiles of every problem below 2^22 points, the larger ones by their grid's own
passes; graph-captured) and the tile-shape autotuner.

Bars: the batched step performs the single-problem step's operations on each
problem's grid (the batched kernel runs the run-time-size form of each pass,
the single-problem kernels may run a form compiled for the grid's sizes), so
the two agree to rounding: relative L2 <= 2e-6 in FP32 (a few units of FP32
rounding, 6e-8, over three steps) and <= 1e-13 in FP64; FP64 batches match the
oracle to 1e-12 and FP32 split-scheme batches to 1e-5; replaying a batch's
graph and autotuned tile shapes change no result bit."""
import numpy as np
import pytest
import torch

from gpu_common import T, cuda, host, rel_l2
from oracle.transport import Grid as OGrid, Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


# uneven shapes drawn from the batch workload's ranges (N_r in {17,33,65},
# angular N in {8,16,24}), kept small enough for the oracle
SPECS = [
    (17, 8, 16, 8, 8, 2, 37.0),
    (33, 8, 8, 16, 8, 1, 0.4),
    (17, 16, 8, 8, 16, 3, 91.0),
    (17, 8, 8, 8, 8, 1, 5.0),
    (33, 8, 8, 8, 16, 2, 12.0),
]


def _descs(precision, scheme, specs=SPECS):
    ts = T()
    return [ts.GridDesc(0.2, 1.0, Nr, Nt, Np, NT, NP, G, precision, scheme, 0, 0, 36.0, 16)
            for (Nr, Nt, Np, NT, NP, G, s) in specs]


def _fields(og, spec, seed):
    Nr, Nt, Np, NT, NP, G, s = spec
    kap, eta, ks = I.absorber_fields(og.r, og.theta, og.phi, groups=G)
    F0 = np.stack([I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, seed + g, 0.2, 1.0)
                   for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, NT)
    return s * kap, s * eta, ks, F0, gR1, gR2


def _setup(batch, specs, dtype):
    ogs, data, Fs, dts = [], [], [], []
    for q, spec in enumerate(specs):
        og = OGrid(0.2, 1.0, *spec[:5], groups=spec[5])
        kap, eta, ks, F0, gR1, gR2 = _fields(og, spec, 1104 + 31 * q)
        batch.grids[q].set_coeffs(kap, eta, ks, gR1, gR2)
        ogs.append(og)
        data.append((kap, eta, ks, F0, gR1, gR2))
        Fs.append(cuda(F0, dtype))
        dts.append(I.dt_rule(0.2, 1.0, spec[0]))
    return ogs, data, Fs, dts


@pytest.mark.parametrize("precision,scheme", [(1, 1), (2, 1), (0, 0)])
def test_batch_matches_the_single_problem_step(precision, scheme):
    ts = T()
    b = ts.Batch(_descs(precision, scheme), autotune=True)
    dtype = torch.float64 if precision == 0 else torch.float32
    _, _, Fs, dts = _setup(b, SPECS, dtype)
    ref = [F.clone() for F in Fs]
    b.step(Fs, dts, 3)
    torch.cuda.synchronize()
    for q, g in enumerate(b.grids):
        g.step(ref[q], dts[q], 3)
    torch.cuda.synchronize()
    tol = 1e-13 if precision == 0 else 2e-6
    for q in range(len(SPECS)):
        assert rel_l2(host(Fs[q]), host(ref[q])) <= tol, q
    b.close()


def test_batch_fp64_matches_oracle():
    ts = T()
    b = ts.Batch(_descs(0, 0), autotune=False)
    ogs, data, Fs, dts = _setup(b, SPECS, torch.float64)
    b.step(Fs, dts, 4)
    torch.cuda.synchronize()
    for q, og in enumerate(ogs):
        kap, eta, ks, F0, gR1, gR2 = data[q]
        ref = OProblem(og, kap, eta, ks, gR1, gR2).run(F0, dts[q], 4)
        assert rel_l2(host(Fs[q]), ref) < 1e-12, q
    b.close()


def test_batch_fp32_r64_split_implicit_matches_oracle():
    """FP32 storage and angular contractions, FP64 radial rows near the ends,
    split scheme with the FP64 implicit collision step, kappa up to ~90."""
    ts = T()
    b = ts.Batch(_descs(2, 1), autotune=True)
    ogs, data, Fs, dts = _setup(b, SPECS, torch.float32)
    b.step(Fs, dts, 10)
    torch.cuda.synchronize()
    for q, og in enumerate(ogs):
        kap, eta, ks, F0, gR1, gR2 = data[q]
        ref = OProblem(og, kap, eta, ks, gR1, gR2, scheme="split").run(F0, dts[q], 10)
        assert rel_l2(host(Fs[q]), ref) < 1e-5, q
    b.close()


def test_batch_reuses_its_graph_with_new_fields_and_steps():
    ts = T()
    b = ts.Batch(_descs(1, 1, SPECS[:3]), autotune=False)
    _, _, Fs, dts = _setup(b, SPECS[:3], torch.float32)
    F2 = [F.clone() for F in Fs]
    ref = [F.clone() for F in Fs]
    b.step(Fs, dts, 2)
    b.step(Fs, dts, 3)          # same fields: graph and item table reused
    b.step(F2, dts, 5)          # new pointers: item table re-uploaded
    for q, g in enumerate(b.grids):
        g.step(ref[q], dts[q], 5)
    torch.cuda.synchronize()
    for q in range(3):
        assert torch.equal(Fs[q], F2[q])
        assert rel_l2(host(Fs[q]), host(ref[q])) <= 2e-6
    b.close()


# a problem of at least 2^22 points: the batch steps it with its grid's own passes
LARGE = (33, 16, 16, 16, 16, 2, 3.0)


@pytest.mark.parametrize("precision,scheme", [(0, 0), (2, 1)])
def test_batch_steps_large_problems_with_their_own_passes(precision, scheme):
    """A batch of small problems (work queue) and one of 4.3M points (its grid's
    own compiled passes, recorded into the batch's graph): the large problem is
    bit-identical to the single-problem step, the small ones agree to rounding,
    new fields and steps record the graph again, and in FP64 the large problem
    matches the oracle."""
    ts = T()
    specs = [SPECS[0], LARGE, SPECS[3]]
    b = ts.Batch(_descs(precision, scheme, specs), autotune=False)
    assert b.grids[1].points >= 1 << 22 and b.grids[0].points < 1 << 22
    dtype = torch.float64 if precision == 0 else torch.float32
    ogs, data, Fs, dts = _setup(b, specs, dtype)
    ref = [F.clone() for F in Fs]
    b.step(Fs, dts, 3)
    torch.cuda.synchronize()
    for q, g in enumerate(b.grids):
        g.step(ref[q], dts[q], 3)
    torch.cuda.synchronize()
    tol = 1e-13 if precision == 0 else 2e-6
    assert torch.equal(Fs[1], ref[1])
    for q in (0, 2):
        assert rel_l2(host(Fs[q]), host(ref[q])) <= tol, q
    if precision == 0:
        kap, eta, ks, F0, gR1, gR2 = data[1]
        oref = OProblem(ogs[1], kap, eta, ks, gR1, gR2).run(F0, dts[1], 3)
        assert rel_l2(host(Fs[1]), oref) < 1e-12
    # new field pointers and steps
    F2 = [cuda(d[3], dtype) for d in data]
    dt2 = [0.5 * d for d in dts]
    ref2 = [F.clone() for F in F2]
    b.step(F2, dt2, 2)
    torch.cuda.synchronize()
    for q, g in enumerate(b.grids):
        g.step(ref2[q], dt2[q], 2)
    torch.cuda.synchronize()
    assert torch.equal(F2[1], ref2[1])
    for q in (0, 2):
        assert rel_l2(host(F2[q]), host(ref2[q])) <= tol, q
    b.close()


def test_batch_of_large_problems_only():
    """Every problem on its grid's own passes (no work-queue launch): the batch
    equals the single-problem steps bit for bit."""
    ts = T()
    specs = [LARGE, LARGE]
    b = ts.Batch(_descs(1, 0, specs), autotune=False)
    _, _, Fs, dts = _setup(b, specs, torch.float32)
    ref = [F.clone() for F in Fs]
    b.step(Fs, dts, 2)
    torch.cuda.synchronize()
    for q, g in enumerate(b.grids):
        g.step(ref[q], dts[q], 2)
    torch.cuda.synchronize()
    for q in range(2):
        assert torch.equal(Fs[q], ref[q])
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ab2_batch_matches_single_problem_steps_and_the_oracle(precision):
    """TS_AB2 on every problem (small ones on the work queue, one of 4.3M points on
    its own passes): the batch keeps its history across calls (2 + 3 steps equal
    5 steps of separate grids: forward Euler, then Adams-Bashforth), the large
    problem bit for bit, the small ones to rounding, and in FP64 the small ones
    match the oracle's AB2 run."""
    ts = T()
    specs = [SPECS[0], LARGE, SPECS[4]]
    b = ts.Batch(_descs(precision, ts.TS_AB2, specs), autotune=False)
    dtype = torch.float64 if precision == 0 else torch.float32
    ogs, data, Fs, dts = _setup(b, specs, dtype)
    dts = [0.5 * d for d in dts]   # AB2's stability limit is below RK4's
    sep = []
    for q, spec in enumerate(specs):
        g = ts.Grid(0.2, 1.0, *spec[:5], groups=spec[5], precision=precision, scheme=ts.TS_AB2)
        kap, eta, ks, F0, gR1, gR2 = data[q]
        g.set_coeffs(kap, eta, ks, gR1, gR2)
        F = cuda(F0, dtype)
        g.step(F, dts[q], 5)
        sep.append(F)
    b.step(Fs, dts, 2)
    b.step(Fs, dts, 3)
    torch.cuda.synchronize()
    tol = 1e-13 if precision == 0 else 2e-6
    assert torch.equal(Fs[1], sep[1])
    for q in (0, 2):
        assert rel_l2(host(Fs[q]), host(sep[q])) <= tol, q
    if precision == 0:
        for q in (0, 2):
            kap, eta, ks, F0, gR1, gR2 = data[q]
            ref = OProblem(ogs[q], kap, eta, ks, gR1, gR2, scheme="ab2").run(F0, dts[q], 5)
            assert rel_l2(host(Fs[q]), ref) < 1e-12, q
    # a restart (new fields) begins with forward Euler again
    F2 = [cuda(d[3], dtype) for d in data]
    b.step(F2, dts, 5)
    torch.cuda.synchronize()
    assert torch.equal(F2[1], sep[1])
    b.close()


def test_autotune_changes_no_result_bits():
    ts = T()
    g = ts.Grid(0.2, 1.0, 17, 8, 16, 16, 8, groups=2, precision=1)
    og = OGrid(0.2, 1.0, 17, 8, 16, 16, 8, groups=2)
    kap, eta, ks, F0, gR1, gR2 = _fields(og, (17, 8, 16, 16, 8, 2, 1.0), 5)
    g.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(0.2, 1.0, 17)
    a = cuda(F0, torch.float32)
    g.step(a, dt, 3)
    before = ts.ts_tile_shape(g.handle)
    after = g.autotune()
    bb = cuda(F0, torch.float32)
    g.step(bb, dt, 3)
    assert all(x > 0 for x in before + after)
    assert torch.equal(a, bb)


def test_batch_errors():
    ts = T()
    with pytest.raises(ts.TSError):
        ts.Batch([ts.GridDesc(0.2, 1.0, 17, 8, 8, 8, 8, 1, 0, 0, 0, 0, 36.0, 16),
                  ts.GridDesc(0.2, 1.0, 17, 8, 8, 8, 8, 1, 1, 0, 0, 0, 36.0, 16)])
    b = ts.Batch(_descs(0, 0, SPECS[:2]), autotune=False)
    F = [torch.zeros(g.shape, dtype=torch.float64, device="cuda") for g in b.grids]
    with pytest.raises(ts.TSError) as e:
        b.step(F, [1e-3, 1e-3], 1)      # coefficients not set
    assert e.value.status == ts.TS_ERR_STATE
    b.close()
