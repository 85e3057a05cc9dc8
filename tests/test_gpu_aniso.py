"""Anisotropic scattering kernels (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)),
mu = omega.omega' (Eqs. sigmadif, crossnun, crossnup, sigmaTh) on the GPU
against the FP64 oracle.

Same bars as the isotropic parity tests: relative L2 <= 1e-12 for FP64, <= 1e-5
for the FP32 variants, on grids that run the run-time and the compiled forms of
the angular pass (warp-reduced and block-reduced moments), the split scheme's
implicit collision, the adjoint step and the batched step. Inputs: the neutron /
proton mixture of the neutrino workload (b between about -1/3 and -1/5), a
field covering b in [-1, 1], Thomson scattering (b = 0, c = 3/4) and fields
covering b in [-1, 1] with c in [-1.2, 1.2]."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, pair, rel_l2
from oracle.transport import Grid as OGrid, Problem as OProblem, nucleon_scattering
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5

RAGGED = (0.2, 1.0, 11, 7, 10, 6, 12)      # run-time angular form (N_Phi = 12)
WARP = (0.2, 1.0, 13, 6, 10, 8, 16)        # register-blocked run-time form, moments by warp shuffles
BLOCK = (0.3, 1.1, 9, 4, 6, 24, 24)        # compiled 24 x 24 form, moments per block
SQUARE = (0.2, 1.0, 17, 16, 16, 16, 16)    # compiled 16 x 16 form


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _fields(og, kind, seed=1104):
    """(kappa, eta, kappa_s, b, c, F0, inflow): c is None for the linear kernels."""
    kap, eta, _, F0, gR1, gR2 = absorber_workload(og, seed)
    c = None
    if kind == "mixture":
        ks, b = nucleon_scattering(*I.nucleon_densities(og.r, og.theta, og.phi, og.G, seed,
                                                        og.R1, og.R2))
    elif kind == "thomson":
        ks, b, c = np.full_like(kap, 0.8), None, np.full_like(kap, 0.75)
    else:
        ks = np.full_like(kap, 0.8)
        b = I.signed_field(og.r, og.theta, og.phi, og.G, seed, og.R1, og.R2)
        if kind == "general":
            c = 1.2 * I.signed_field(og.r, og.theta, og.phi, og.G, seed + 1, og.R1, og.R2)
    return kap, eta, ks, b, c, F0, gR1, gR2


def _both(dims, G, kind, precision=0, scheme=0, bc=0, kscale=1.0, kapscale=1.0):
    og, gg = pair(*dims, G=G, precision=precision, scheme=scheme, bc=bc)
    kap, eta, ks, b, c, F0, gR1, gR2 = _fields(og, kind)
    kap, ks = kap * kapscale, ks * kscale
    op = OProblem(og, kap, eta, ks, gR1, gR2, bc="tau" if bc == 0 else "none",
                  scheme="rk4" if scheme == 0 else "split", scatter_b=b, scatter_c=c)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    if b is not None:
        gg.set_scattering_anisotropy(b)
    if c is not None:
        gg.set_scattering_quadrupole(c)
    return og, gg, op, F0


@pytest.mark.parametrize("dims", [RAGGED, WARP, BLOCK, SQUARE])
@pytest.mark.parametrize("kind", ["mixture", "signed", "thomson", "general"])
def test_rhs_and_steps_parity(dims, kind):
    og, gg, op, F0 = _both(dims, 3, kind, kscale=6.0)
    F = F0 + 0.1 * np.random.default_rng(3).standard_normal(og.shape)
    assert rel_l2(host(gg.rhs(cuda(F))), op.rhs(F)) < FP64_TOL
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    Fg = cuda(F0)
    gg.step(Fg, dt, 8)
    assert rel_l2(host(Fg), op.run(F0, dt, 8)) < FP64_TOL


def test_anisotropy_changes_the_result_and_null_restores_isotropic():
    og, gg, op, F0 = _both(WARP, 2, "signed", kscale=6.0)
    dt = I.dt_rule(WARP[0], WARP[1], WARP[2])
    a = cuda(F0)
    gg.step(a, dt, 4)
    gg.set_scattering_anisotropy(None)
    b = cuda(F0)
    gg.step(b, dt, 4)
    _, fresh = pair(*WARP, G=2)
    kap, eta, ks, _, _, _, gR1, gR2 = _fields(og, "signed")
    fresh.set_coeffs(kap, eta, ks * 6.0, gR1, gR2)
    c = cuda(F0)
    fresh.step(c, dt, 4)
    assert torch.equal(b, c)
    assert rel_l2(host(a), host(c)) > 1e-4


@pytest.mark.parametrize("dims", [RAGGED, WARP])
@pytest.mark.parametrize("kind", ["signed", "general"])
def test_split_implicit_parity(dims, kind):
    """Backward-Euler collision with the first- and second-moment closed forms,
    kappa ~ 60."""
    og, gg, op, F0 = _both(dims, 2, kind, scheme=1, kscale=30.0, kapscale=60.0)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    Fg = cuda(F0)
    gg.step(Fg, dt, 6)
    assert rel_l2(host(Fg), op.run(F0, dt, 6)) < FP64_TOL


@pytest.mark.parametrize("dims", [RAGGED, (0.2, 1.0, 9, 16, 16, 16, 16)])
@pytest.mark.parametrize("kind", ["signed", "general"])
def test_adjoint_parity(dims, kind):
    og, gg, op, F0 = _both(dims, 2, kind, kscale=6.0)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    lam = np.random.default_rng(6).standard_normal(og.shape)
    lo, gko, geo = op.adjoint_step(F0, lam, dt)
    lg = cuda(lam)
    gk = torch.zeros(og.G, og.Nr, og.Nt, og.Np, dtype=torch.float64, device="cuda")
    ge = torch.zeros_like(gk)
    gg.adjoint_step(cuda(F0), lg, gk, ge, dt)
    assert rel_l2(host(lg), lo) < FP64_TOL
    assert rel_l2(host(gk), gko) < FP64_TOL
    assert rel_l2(host(ge), geo) < FP64_TOL


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("dims", [RAGGED, SQUARE])
@pytest.mark.parametrize("kind", ["mixture", "general"])
def test_fp32_variants(precision, dims, kind):
    og, gg, op, F0 = _both(dims, 2, kind, precision=precision, kscale=6.0)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 10)
    assert rel_l2(host(Fg), op.run(F0, dt, 10)) < FP32_TOL


@pytest.mark.parametrize("kind", ["mixture", "thomson"])
def test_full_size_33x16(kind):
    """The neutrino and photon workloads at full size: 33 x 16^4, 4 groups,
    every element after 2 steps, in the launch configuration the benchmark times."""
    dims = (0.2, 1.0, 33, 16, 16, 16, 16)
    og, gg, op, F0 = _both(dims, 4, kind)
    dt = I.dt_rule(0.2, 1.0, 33)
    Fg = cuda(F0)
    gg.step(Fg, dt, 2)
    assert rel_l2(host(Fg), op.run(F0, dt, 2)) < FP64_TOL


def test_library_mixture_helper_matches_the_oracle():
    An, Ap = I.nucleon_densities(np.linspace(0.2, 1, 5), np.linspace(0.1, 3, 4),
                                 np.linspace(0, 6, 6), 2, 7, 0.2, 1.0)
    ks1, b1 = T().nucleon_scattering(An, Ap)
    ks2, b2 = nucleon_scattering(An, Ap)
    assert np.allclose(ks1, ks2, rtol=1e-15) and np.allclose(b1, b2, rtol=1e-15)


def test_batch_with_anisotropic_and_isotropic_problems():
    """A batch whose problems mix the linear, quadratic and isotropic kernels
    agrees with the oracle (FP64) problem by problem."""
    ts = T()
    specs = [(17, 8, 16, 8, 8, 2), (17, 8, 8, 16, 16, 1), (9, 6, 10, 6, 12, 2)]
    descs = [ts.GridDesc(0.2, 1.0, *s, 0, 0, 0, 0, 36.0, 16) for s in specs]
    bt = ts.Batch(descs, autotune=False)
    Fs, refs, dts = [], [], []
    for q, s in enumerate(specs):
        og = OGrid(0.2, 1.0, *s[:5], groups=s[5])
        kap, eta, ks, b, c, F0, gR1, gR2 = _fields(og, "general", 1104 + 17 * q)
        aniso, quad = q != 1, q == 2
        bt.grids[q].set_coeffs(kap, eta, 6.0 * ks, gR1, gR2)
        if aniso:
            bt.grids[q].set_scattering_anisotropy(b)
        if quad:
            bt.grids[q].set_scattering_quadrupole(c)
        dt = I.dt_rule(0.2, 1.0, s[0])
        refs.append(OProblem(og, kap, eta, 6.0 * ks, gR1, gR2, scatter_b=b if aniso else None,
                             scatter_c=c if quad else None).run(F0, dt, 3))
        Fs.append(cuda(F0))
        dts.append(dt)
    bt.step(Fs, dts, 3)
    torch.cuda.synchronize()
    for q in range(len(specs)):
        assert rel_l2(host(Fs[q]), refs[q]) < FP64_TOL, q
    # switching problem 0 to isotropic between steps (same fields, same dt) is seen
    before = Fs[0].clone()
    bt.grids[0].set_scattering_anisotropy(None)
    ref_iso = before.clone()
    bt.step(Fs, dts, 1)
    torch.cuda.synchronize()
    bt.grids[0].step(ref_iso, dts[0], 1)
    assert rel_l2(host(Fs[0]), host(ref_iso)) < 1e-13
    bt.close()


def test_quadrupole_rejected_for_split_scheme_on_small_direction_grids():
    ts = T()
    og, gg = pair(0.2, 1.0, 9, 4, 4, 4, 8, G=1, scheme=1)
    with pytest.raises(ts.TSError):
        gg.set_scattering_quadrupole(0.75)
