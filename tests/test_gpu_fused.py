"""The fused angular + radial pass of float grids (one tile per (g, theta,
phi) position with every radial node and direction in shared memory, after a
plane pass that writes its theta / phi terms): parity with the FP64 oracle
(1e-5, the reduced-precision bar) for every stage mode, scattering kernel and
precision that takes it, and agreement with the three-pass form of the same
precision (the two differ by FP32 rounding only)."""
import os

import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, pair, rel_l2, setup_both
from oracle.transport import Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5

# compiled form (33 x 16^2 tiles, two staging buffers, one chunk), run-time forms
# with odd and even N_r, and a tile too large for two buffers (65 x 16^2: one
# buffer, the angular phase in two chunks)
GRIDS = [(0.2, 1.0, 33, 16, 16, 16, 16), (0.2, 1.0, 17, 6, 4, 8, 8), (0.3, 1.2, 16, 4, 6, 12, 16),
         (0.2, 1.0, 65, 4, 4, 16, 16), (0.2, 1.0, 13, 5, 6, 4, 8)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _grid(dims, G=2, precision=1, scheme=0, bc=0, fused=True):
    old = os.environ.get("TS_FUSED")
    os.environ["TS_FUSED"] = "1" if fused else "0"
    try:
        return pair(*dims, G=G, precision=precision, scheme=scheme, bc=bc)
    finally:
        if old is None:
            del os.environ["TS_FUSED"]
        else:
            os.environ["TS_FUSED"] = old


def _uses_fused(gg, F, dt):
    _, n = T().ts_step_profile(gg.handle, F.clone(), dt, 1)
    return n[0] == 0 and n[2] > 0      # no angular-pass launches: the fused pass ran


@pytest.mark.parametrize("dims", GRIDS)
def test_fused_rhs_and_steps_against_oracle(dims):
    og, gg = _grid(dims)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = setup_both(og, gg, kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    assert _uses_fused(gg, cuda(F0, torch.float32), dt)
    F = F0 + 0.1 * np.random.default_rng(3).standard_normal(og.shape)
    assert rel_l2(host(gg.rhs(cuda(F, torch.float32))), op.rhs(F)) < FP32_TOL
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 20)
    assert rel_l2(host(Fg), op.run(F0, dt, 20)) < FP32_TOL
    LF = host(gg.liouville(cuda(F, torch.float32)))
    assert rel_l2(LF, og.liouville(F)) < FP32_TOL


@pytest.mark.parametrize("dims", GRIDS[:2])
def test_fused_agrees_with_three_passes(dims):
    og, a = _grid(dims, G=3)
    _, b = _grid(dims, G=3, fused=False)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    for g in (a, b):
        g.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    assert _uses_fused(a, cuda(F0, torch.float32), dt)
    assert not _uses_fused(b, cuda(F0, torch.float32), dt)
    x, y = cuda(F0, torch.float32), cuda(F0, torch.float32)
    a.step(x, dt, 10)
    b.step(y, dt, 10)
    assert rel_l2(host(x), host(y)) < 2e-6


@pytest.mark.parametrize("scheme", [1, 2])
def test_fused_split_and_ab2_against_oracle(scheme):
    dims = GRIDS[1]
    og, gg = _grid(dims, scheme=scheme)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    name = {1: "split", 2: "ab2"}[scheme]
    k = 30.0 * kap if scheme == 1 else kap
    op = setup_both(og, gg, k, eta, ks, gR1, gR2, scheme=name)
    dt = I.dt_rule(dims[0], dims[1], dims[2], 0.2 if scheme == 2 else 0.4)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 15)
    assert rel_l2(host(Fg), op.run(F0, dt, 15)) < FP32_TOL


@pytest.mark.parametrize("form", ["linear", "thomson"])
def test_fused_anisotropic_kernels_against_oracle(form):
    dims = GRIDS[0] if form == "thomson" else GRIDS[2]
    og, gg = _grid(dims, G=1)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    b = I.signed_field(og.r, og.theta, og.phi, 1, 1104, og.R1, og.R2) if form == "linear" else None
    c = 0.75 if form == "thomson" else None
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    gg.set_scattering_anisotropy(b)
    gg.set_scattering_quadrupole(c)
    op = OProblem(og, kap, eta, ks, gR1, gR2, scatter_b=b, scatter_c=c)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 10)
    assert rel_l2(host(Fg), op.run(F0, dt, 10)) < FP32_TOL


@pytest.mark.parametrize("dims", [GRIDS[0], GRIDS[3]])
def test_fused_fp32_r64_against_oracle(dims):
    """FP32 storage with the radial rows nearest both ends in double (folded
    through the even/odd parts) and the FP64 implicit collision step."""
    og, gg = _grid(dims, G=1, precision=2, scheme=1)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = setup_both(og, gg, 20.0 * kap, eta, ks, gR1, gR2, scheme="split")
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    assert _uses_fused(gg, cuda(F0, torch.float32), dt)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 10)
    assert rel_l2(host(Fg), op.run(F0, dt, 10)) < FP32_TOL
