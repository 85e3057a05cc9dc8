"""The conservative 5-D form (App. A, Eq. Cohercons; TS_FORM_CONSERVATIVE) on the
GPU against the FP64 oracle's ConservativeProblem, and the number balance
(ts_number_balance) of both forms against the oracle's.

Bars: relative L2 <= 1e-12 for the stage derivative, the operator and RK4 / AB2
steps on ragged grids (run-time plane forms) and even ones (the register-blocked
plane pass, which the odd theta tables serve), with isotropic, linear and
quadratic scattering kernels; N, J_R1, J_R2, dN/dt and S to 1e-12 of their scale;
the balance residual of the conservative form to rounding on data without the
theta-coupled Fourier modes, where the advective form's is not; the full
33 x 16^4 x 4 grid."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, rel_l2
from oracle import conservative5d as C
from oracle.transport import Grid as OGrid, Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12
RAGGED = (0.2, 1.0, 11, 7, 10, 6, 12)
EVEN = (0.3, 1.2, 9, 8, 8, 8, 8)
WIDE = (0.5, 1.5, 13, 10, 6, 12, 16)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _pair(dims, G=2, scheme=0, bc=0):
    ts = T()
    og = OGrid(*dims, groups=G)
    gg = ts.Grid(*dims, groups=G, scheme=scheme, bc=bc, form=ts.TS_FORM_CONSERVATIVE)
    return og, gg


def _workload(og, seed=1104):
    """The absorber workload on Fhat = J F: inflow data J g."""
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og, seed)
    J = C.jacobian(og)
    h = og.NT // 2
    return kap, eta, ks, J * F0, gR1 * J[:, 0, :, :, :h], gR2 * J[:, -1, :, :, h:]


def _kernel(og, gg, form):
    """b, c fields for the scattering kernel form ('iso', 'linear', 'quadratic')."""
    b = c = None
    if form != "iso":
        b = I.signed_field(og.r, og.theta, og.phi, og.G, 5, og.R1, og.R2) * 0.5
        gg.set_scattering_anisotropy(b)
    if form == "quadratic":
        c = 0.75
        gg.set_scattering_quadrupole(c)
    return b, c


@pytest.mark.parametrize("dims", [RAGGED, EVEN, WIDE])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("form", ["iso", "linear", "quadratic"])
def test_rhs_and_operator_parity(dims, bc, form):
    og, gg = _pair(dims, bc=bc)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, g1, g2)
    b, c = _kernel(og, gg, form)
    op = C.ConservativeProblem(og, kap, eta, ks, g1, g2, bc="tau" if bc == 0 else "none",
                               scatter_b=b, scatter_c=c)
    X = X0 + 0.2 * np.random.default_rng(3).standard_normal(og.shape)
    assert rel_l2(host(gg.rhs(cuda(X))), op.rhs(X)) < TOL
    assert rel_l2(host(gg.liouville(cuda(X))), C.liouville_hat(og, X)) < TOL


@pytest.mark.parametrize("dims", [RAGGED, EVEN])
@pytest.mark.parametrize("scheme,name", [(0, "rk4"), (2, "ab2")])
def test_steps_parity(dims, scheme, name):
    og, gg = _pair(dims, G=2, scheme=scheme)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, g1, g2)
    b, c = _kernel(og, gg, "quadratic")
    op = C.ConservativeProblem(og, kap, eta, ks, g1, g2, scheme=name, scatter_b=b, scatter_c=c)
    dt = 0.4 * np.diff(og.r).min() * (0.5 if name == "ab2" else 1.0)
    Xg = cuda(X0)
    gg.step(Xg, dt, 20)
    assert rel_l2(host(Xg), op.run(X0, dt, 20)) < TOL


@pytest.mark.parametrize("dims", [RAGGED, EVEN])
def test_number_balance_parity_both_forms(dims):
    ts = T()
    og, gg = _pair(dims, G=2, bc=0)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, g1, g2)
    b, c = _kernel(og, gg, "quadratic")
    X = X0 + 0.1 * np.random.default_rng(4).standard_normal(og.shape)
    op = C.ConservativeProblem(og, kap, eta, ks, g1, g2, scatter_b=b, scatter_c=c)
    ref = np.stack(op.balance(X), axis=1)
    got = gg.number_balance(cuda(X))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the advective form of the same state F = Fhat / J, in FP64 and FP32
    F = X / C.jacobian(og)
    pp = OProblem(og, kap, eta, ks, scatter_b=b, scatter_c=c)
    refp = np.stack(C.plain_balance(pp, F), axis=1)
    for prec, tol, dt in ((ts.TS_FP64, 1e-12, torch.float64), (ts.TS_FP32, 1e-4, torch.float32)):
        gp = ts.Grid(*dims, groups=2, precision=prec)
        gp.set_coeffs(kap, eta, ks)
        _kernel(og, gp, "quadratic")
        got = gp.number_balance(cuda(F, dt))
        assert np.abs(got - refp).max() <= tol * np.abs(refp).max(), prec
        gp.close()


def test_conservative_balance_is_exact_and_the_advective_one_is_not():
    """Random Fhat without the (m = 0, M = +-1) Fourier modes, the only ones the
    theta flux brings into the phi and Phi trapezoid sums: every other flux
    integrates exactly, so the conservative residual is rounding; the advective
    form of the same state keeps a truncation-level residual."""
    ts = T()
    og, gg = _pair(EVEN, G=2, bc=1)
    X = np.random.default_rng(5).standard_normal(og.shape)
    c = np.fft.fft(np.fft.fft(X, axis=3), axis=5)
    c[:, :, :, 0, :, 1] = 0.0
    c[:, :, :, 0, :, -1] = 0.0
    X = np.real(np.fft.ifft(np.fft.ifft(c, axis=5), axis=3))
    ks = 0.3 + np.random.default_rng(6).random(gg.coef_shape)
    z = np.zeros(gg.coef_shape)
    gg.set_coeffs(z, z, ks)
    _kernel(og, gg, "quadratic")
    out = gg.number_balance(cuda(X))
    N, J1, J2, dN, S = out.T
    scale = np.abs(out[:, :3]).max()
    assert np.abs(dN + J2 - J1 - S).max() < 1e-12 * scale
    gp = ts.Grid(*EVEN, groups=2, bc=1)
    gp.set_coeffs(z, z, ks)
    _kernel(og, gp, "quadratic")
    Np_, J1p, J2p, dNp, Sp = gp.number_balance(cuda(X / C.jacobian(og))).T
    assert np.abs(dNp + J2p - J1p - Sp).max() > 1e-3 * scale
    assert np.abs(Np_ - N).max() < 1e-12 * scale     # the same number, both forms


@pytest.mark.parametrize("prec", ["fp32", "fp32_r64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("dims", [RAGGED, EVEN])
def test_float_precisions(prec, dims):
    """The float forms (angular pass in float, plane and radial passes of the
    precision: FP64 end rows, tcgen05 radial) against the FP64 oracle: stage
    derivative, 20 RK4 steps, AB2 steps and the number balance, <= 1e-5."""
    ts = T()
    P = {"fp32": ts.TS_FP32, "fp32_r64": ts.TS_FP32_R64, "tf32x3": ts.TS_TF32X3,
         "bf16x3": ts.TS_BF16X3}[prec]
    og = OGrid(*dims, groups=2)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    for scheme, name in ((ts.TS_RK4, "rk4"), (ts.TS_AB2, "ab2")):
        gg = ts.Grid(*dims, groups=2, precision=P, scheme=scheme, form=ts.TS_FORM_CONSERVATIVE)
        gg.set_coeffs(kap, eta, ks, g1, g2)
        b, c = _kernel(og, gg, "quadratic")
        op = C.ConservativeProblem(og, kap, eta, ks, g1, g2, scheme=name, scatter_b=b,
                                   scatter_c=c)
        if name == "rk4":
            assert rel_l2(host(gg.rhs(cuda(X0, torch.float32))), op.rhs(X0)) < 1e-5
            ref = np.stack(op.balance(X0), axis=1)
            got = gg.number_balance(cuda(X0, torch.float32))
            assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
        dt = 0.4 * np.diff(og.r).min() * (0.5 if name == "ab2" else 1.0)
        Xg = cuda(X0, torch.float32)
        gg.step(Xg, dt, 20)
        assert rel_l2(host(Xg), op.run(X0, dt, 20)) < 1e-5, name
        gg.close()


def test_full_size_grid():
    """33 x 16^4, 4 groups (the headline grid): stage derivative and two RK4 steps."""
    og, gg = _pair((0.2, 1.0, 33, 16, 16, 16, 16), G=4)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, g1, g2)
    op = C.ConservativeProblem(og, kap, eta, ks, g1, g2)
    assert rel_l2(host(gg.rhs(cuda(X0))), op.rhs(X0)) < TOL
    dt = 0.4 * np.diff(og.r).min()
    Xg = cuda(X0)
    gg.step(Xg, dt, 2)
    assert rel_l2(host(Xg), op.run(X0, dt, 2)) < TOL


def test_spherically_symmetric_shell_keeps_its_symmetry_and_balance():
    """The Lambert shell (empty shell, Fhat(R1) = J F0 cos Th on the outgoing
    directions, a spherically symmetric scattering plasma of optical depth 5):
    Fhat / (r^2 sin th sin Th) stays independent of theta, phi, Phi, and the
    operator's number balance at the final state holds to rounding (the theta
    flux of symmetric data integrates to zero over Phi)."""
    ts = T()
    dims = (0.5, 1.0, 17, 6, 4, 12, 8)
    og, gg = _pair(dims, G=1, bc=0)
    prof = 9.0 * 5.0 / 0.5 * (1.0 - (og.r - 0.5) / 0.5) ** 8     # optical depth 5
    ks = np.ascontiguousarray(np.broadcast_to(prof[None, :, None, None], (1, og.Nr, og.Nt, og.Np)))
    gR1, gR2 = I.lambert_inflow(og.Theta, og.Nt, og.Np, og.NP)
    J = C.jacobian(og)
    h = og.NT // 2
    g1, g2 = gR1 * J[:, 0, :, :, :h], gR2 * J[:, -1, :, :, h:]
    gg.set_coeffs(None, None, ks, g1, g2)
    op = C.ConservativeProblem(og, kappa_s=ks, g_R1=g1, g_R2=g2)
    Xg = gg.apply_inflow(cuda(np.zeros(og.shape)))
    X0 = op.apply_inflow(np.zeros(og.shape))
    assert rel_l2(host(Xg), X0) == 0.0
    dt = 0.4 * np.diff(og.r).min()
    gg.step(Xg, dt, 30)
    X = host(Xg)
    assert rel_l2(X, op.run(X0, dt, 30)) < TOL
    F = X / J
    assert np.abs(F - F[:, :, :1, :1, :, :1]).max() < 1e-12 * np.abs(F).max()
    N, J1, J2, dN, S = gg.number_balance(Xg)[0]
    assert abs(dN + J2 - J1 - S) < 1e-12 * (abs(J1) + abs(J2))


def test_unsupported_calls_on_the_conservative_form():
    ts = T()
    og, gg = _pair(RAGGED, G=1)
    kap, eta, ks, X0, g1, g2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, g1, g2)
    Xg = cuda(X0)
    with pytest.raises(ts.TSError):
        gg.moments(Xg)
    gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TSError):
        gg.adjoint_step(Xg, torch.zeros_like(Xg), gk, torch.zeros_like(gk), 1e-3)
    with pytest.raises(ts.TSError):
        gg.outgoing_flux(Xg)
    for kw in (dict(scheme=ts.TS_RK4_SPLIT_IMPLICIT), dict(filter_on=True),
               dict(radial=ts.TS_RADIAL_UPWIND_FD)):
        with pytest.raises(ts.TSError):
            ts.Grid(*RAGGED, form=ts.TS_FORM_CONSERVATIVE, **kw)
