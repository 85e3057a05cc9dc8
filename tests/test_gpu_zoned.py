"""The three-zone radial grid of App. B (first-order upwind differences in two
edge zones of width 0.1 (R2 - R1), Chebyshev in the central zone, the central
zone's inflow interface taken by the Tau method) on the GPU against the FP64
oracle's GridZonedR.

Bars as for the other radial grids: relative L2 <= 1e-12 in FP64, <= 1e-5 in
FP32, on ragged grids (run-time angular forms), with the RK4, split and AB2
schemes, the inflow nodes held or free, the moments (trapezoid + Clenshaw-Curtis
in r), and the paper's zone sizes (30 + 65 + 30 nodes with shared interfaces)."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, rel_l2
from oracle.transport import GridZonedR, Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5

# (R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi), zone_nodes
RAGGED = ((0.2, 1.0, 23, 7, 10, 6, 12), 6)
SQUARE = ((0.5, 1.5, 41, 8, 8, 12, 8), 9)
EVEN_CENTRAL = ((0.5, 1.0, 24, 4, 6, 8, 4), 5)     # 16 central nodes (odd degree)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _pair(case, G=1, precision=0, scheme=0, bc=0, width=0.1):
    ts = T()
    dims, nA = case
    og = GridZonedR(*dims, groups=G, zone_nodes=nA, zone_width=width)
    gg = ts.Grid(*dims, groups=G, precision=precision, scheme=scheme, bc=bc,
                 radial=ts.TS_RADIAL_ZONED, zone_nodes=nA, zone_width=width)
    return og, gg


def _dt(og):
    return 0.4 * np.diff(og.r).min()


@pytest.mark.parametrize("case", [RAGGED, SQUARE, EVEN_CENTRAL])
def test_nodes_match(case):
    og, gg = _pair(case)
    assert np.abs(gg.nodes()[0] - og.r).max() < 1e-15


@pytest.mark.parametrize("case", [RAGGED, SQUARE, EVEN_CENTRAL])
@pytest.mark.parametrize("bc", [0, 1])
def test_rhs_parity(case, bc):
    og, gg = _pair(case, G=2, bc=bc)
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


def test_wide_zones_and_anisotropic_kernel():
    og, gg = _pair(SQUARE, G=2, width=0.3)
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


def test_moments_use_the_zoned_rule():
    og, gg = _pair(RAGGED, G=2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    m = gg.moments(cuda(F0))
    ref = og.moments(F0)
    for a, b in zip(m, ref):
        assert rel_l2(host(a), b) < 1e-13


def test_paper_zone_sizes_lambert_shell():
    """30 + 65 + 30 radial nodes (the zones share their interface nodes: N_r =
    123), edge zones of width 0.1 (R2 - R1); the Lambert shell of Sect. 5.3 (empty
    shell, F(R1) = F0 cos(Theta), scattering plasma of optical depth 5)."""
    case = ((0.5, 1.0, 123, 4, 4, 8, 4), 30)
    og, gg = _pair(case)
    assert og.nB == 65
    ks = I.shell_scattering(og.r, og.theta, og.phi, 0.5, 1.0, 5.0)
    gR1, gR2 = I.lambert_inflow(og.Theta, og.Nt, og.Np, og.NP)
    op = OProblem(og, kappa_s=ks, g_R1=gR1, g_R2=gR2)
    gg.set_coeffs(None, None, ks, gR1, gR2)
    F0 = op.apply_inflow(np.zeros(og.shape))
    Fg = gg.apply_inflow(cuda(np.zeros(og.shape)))
    assert rel_l2(host(Fg), F0) == 0.0
    dt = _dt(og)
    gg.step(Fg, dt, 40)
    ref = op.run(F0, dt, 40)
    assert rel_l2(host(Fg), ref) < FP64_TOL
    assert np.abs(host(Fg)[:, 1:]).max() > 0.1   # the emitted front has left the inflow nodes


def test_unsupported_combinations():
    ts = T()
    og, gg = _pair(RAGGED)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TSError):
        gg.adjoint_step(cuda(F0), cuda(F0), gk, torch.zeros_like(gk), _dt(og))
    d = ts.GridDesc(0.2, 1.0, 23, 4, 4, 4, 4, 1, 0, 0, 0, 0, 36.0, 16, ts.TS_RADIAL_ZONED, 6, 0.1)
    with pytest.raises(ts.TSError):
        ts.Batch([d], autotune=False)
    for nA, w, prec in [(1, 0.1, 0), (12, 0.1, 0), (6, 0.0, 0), (6, 0.5, 0), (6, 0.1, 2)]:
        with pytest.raises(ts.TSError):
            ts.Grid(0.2, 1.0, 23, 4, 4, 4, 4, precision=prec, radial=ts.TS_RADIAL_ZONED,
                    zone_nodes=nA, zone_width=w)
