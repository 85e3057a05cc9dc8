"""The hybrid grid of Sect. 5.3 (first-order upwind differences in r on uniform
nodes, spectral angular axes) on the GPU against the FP64 oracle's GridUpwindR.

Bars as for the spectral grid: relative L2 <= 1e-12 in FP64, <= 1e-5 in FP32,
on ragged grids (run-time angular forms, several radial tiles), with the RK4,
split and AB2 schemes, the inflow nodes held or free, anisotropic kernels, the
moments (trapezoid rule in r), and the Lambert-shell workload of Sect. 5.3."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, rel_l2
from oracle.transport import GridUpwindR, Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5

RAGGED = (0.2, 1.0, 23, 7, 10, 6, 12)
SQUARE = (0.5, 1.5, 41, 16, 16, 16, 16)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _pair(dims, G=1, precision=0, scheme=0, bc=0):
    ts = T()
    og = GridUpwindR(*dims, groups=G)
    gg = ts.Grid(*dims, groups=G, precision=precision, scheme=scheme, bc=bc,
                 radial=ts.TS_RADIAL_UPWIND_FD)
    return og, gg


def _dt(og):
    return 0.4 * og.dr


def test_nodes_are_uniform():
    og, gg = _pair(RAGGED)
    assert np.abs(gg.nodes()[0] - og.r).max() < 1e-15


@pytest.mark.parametrize("dims", [RAGGED, SQUARE])
@pytest.mark.parametrize("bc", [0, 1])
def test_rhs_parity(dims, bc):
    og, gg = _pair(dims, G=2, bc=bc)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = OProblem(og, kap, eta, ks, gR1, gR2, bc="tau" if bc == 0 else "none")
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    F = F0 + 0.1 * np.random.default_rng(2).standard_normal(og.shape)
    assert rel_l2(host(gg.rhs(cuda(F))), op.rhs(F)) < FP64_TOL
    assert rel_l2(host(gg.liouville(cuda(F))), og.liouville(F)) < FP64_TOL


@pytest.mark.parametrize("scheme,name", [(0, "rk4"), (1, "split"), (2, "ab2")])
def test_steps_parity(scheme, name):
    og, gg = _pair(RAGGED, G=3, scheme=scheme)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    kap = kap * (40.0 if name == "split" else 1.0)
    op = OProblem(og, kap, eta, ks, gR1, gR2, scheme=name)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = _dt(og) * (0.5 if name == "ab2" else 1.0)
    Fg = cuda(F0)
    gg.step(Fg, dt, 20)
    assert rel_l2(host(Fg), op.run(F0, dt, 20)) < FP64_TOL


def test_anisotropic_kernel_on_the_hybrid_grid():
    og, gg = _pair(SQUARE, G=2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    b = I.signed_field(og.r, og.theta, og.phi, 2, 3, og.R1, og.R2)
    op = OProblem(og, kap, eta, 4 * ks, gR1, gR2, scatter_b=b, scatter_c=0.75)
    gg.set_coeffs(kap, eta, 4 * ks, gR1, gR2)
    gg.set_scattering_anisotropy(b)
    gg.set_scattering_quadrupole(0.75)
    Fg = cuda(F0)
    gg.step(Fg, _dt(og), 10)
    assert rel_l2(host(Fg), op.run(F0, _dt(og), 10)) < FP64_TOL


def test_fp32_variant():
    og, gg = _pair(SQUARE, G=2, precision=1)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = OProblem(og, kap, eta, ks, gR1, gR2)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, _dt(og), 20)
    assert rel_l2(host(Fg), op.run(F0, _dt(og), 20)) < FP32_TOL


def test_moments_use_the_trapezoid_rule():
    og, gg = _pair(RAGGED, G=2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    m = gg.moments(cuda(F0))
    ref = og.moments(F0)
    for a, b in zip(m, ref):
        assert rel_l2(host(a), b) < 1e-13


def test_lambert_shell_workload():
    """Sect. 5.3: empty shell, Lambert emission F0 cos(Theta) at R1, scattering
    plasma of optical depth 5 vanishing at R2, no emission or absorption."""
    dims = (0.5, 1.0, 65, 8, 8, 8, 8)
    og, gg = _pair(dims)
    ks = I.shell_scattering(og.r, og.theta, og.phi, 0.5, 1.0, 5.0)
    gR1, gR2 = I.lambert_inflow(og.Theta, og.Nt, og.Np, og.NP)
    op = OProblem(og, kappa_s=ks, g_R1=gR1, g_R2=gR2)
    gg.set_coeffs(None, None, ks, gR1, gR2)
    F0 = op.apply_inflow(np.zeros(og.shape))
    Fg = gg.apply_inflow(cuda(np.zeros(og.shape)))
    assert rel_l2(host(Fg), F0) == 0.0
    gg.step(Fg, _dt(og), 40)
    ref = op.run(F0, _dt(og), 40)
    assert rel_l2(host(Fg), ref) < FP64_TOL
    assert np.abs(host(Fg)).max() > 0.5      # the emitted front has entered the shell


def test_unsupported_combinations():
    ts = T()
    og, gg = _pair(RAGGED)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TSError):
        gg.adjoint_step(cuda(F0), cuda(F0), gk, torch.zeros_like(gk), _dt(og))
    d = ts.GridDesc(0.2, 1.0, 9, 4, 4, 4, 4, 1, 0, 0, 0, 0, 36.0, 16, ts.TS_RADIAL_UPWIND_FD)
    with pytest.raises(ts.TSError):
        ts.Batch([d], autotune=False)


def test_largest_radial_size_129_nodes():
    """N_r = 129 (the paper's hybrid run), ragged angular sizes, AB2 with held inflow."""
    ts = T()
    og, gg = _pair((0.5, 1.0, 129, 5, 6, 8, 10), G=2, scheme=ts.TS_AB2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = OProblem(og, kap, eta, ks, gR1, gR2, scheme="ab2")
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = 0.5 * _dt(og)
    Fg = cuda(F0)
    gg.step(Fg, dt, 12)
    assert rel_l2(host(Fg), op.run(F0, dt, 12)) < FP64_TOL
