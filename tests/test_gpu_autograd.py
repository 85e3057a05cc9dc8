"""Gradients of the outgoing flux through R2 (Eq. Flux) after n steps with
respect to the absorption kappa and the emissivity eta, via the library's
discrete adjoint behind torch.autograd with sqrt(N) checkpointing: against the
oracle's discrete adjoint (1e-12) and against central finite differences of the
GPU forward (1e-6)."""
import numpy as np
import pytest
import torch

from gpu_common import T, cuda, host, pair, rel_l2
from oracle.transport import Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _workload(og, seed=1104):
    G = og.G
    kap, eta, ks = I.gradient_fields(og.r, og.theta, og.phi, G, seed, og.R1, og.R2)
    F0 = np.stack([I.seeded_smooth(og.r, og.theta, og.phi, og.Theta, og.Phi, seed + g, og.R1, og.R2)
                   for g in range(G)])
    gR1, gR2 = I.inflow_from(F0, og.NT)
    return kap, eta, ks, F0, gR1, gR2


def _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, n, segment=None):
    from paper_1104_5330_gb300.autograd import outgoing_flux, transport_steps
    k = cuda(kap).requires_grad_()
    e = cuda(eta).requires_grad_()
    F = transport_steps(gg, cuda(F0), k, e, cuda(ks), dt, n, cuda(gR1), cuda(gR2), segment)
    J = outgoing_flux(gg, F).sum()
    J.backward()
    return float(J), k.grad, e.grad, F


def test_gradients_match_oracle_adjoint():
    og, gg = pair(0.2, 1.0, 11, 7, 10, 6, 12, G=2)
    kap, eta, ks, F0, gR1, gR2 = _workload(og)
    dt = I.dt_rule(0.2, 1.0, og.Nr)
    n = 7
    _, gk, ge, _ = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, n)
    op = OProblem(og, kap, eta, ks, gR1, gR2)
    Fs = [F0]
    for _ in range(n):
        Fs.append(op.rk4_step(Fs[-1], dt))
    lam = np.zeros(og.shape)
    lam[:, -1] = og.outgoing_flux_weights()
    GK, GE = np.zeros_like(kap), np.zeros_like(eta)
    for i in range(n - 1, -1, -1):
        lam, a, b = op.adjoint_step(Fs[i], lam, dt)
        GK += a
        GE += b
    assert rel_l2(host(gk), GK) < 1e-12
    assert rel_l2(host(ge), GE) < 1e-12


def test_checkpointing_does_not_change_gradients():
    og, gg = pair(0.2, 1.0, 11, 7, 10, 6, 12, G=1)
    kap, eta, ks, F0, gR1, gR2 = _workload(og)
    dt = I.dt_rule(0.2, 1.0, og.Nr)
    J1, k1, e1, F1 = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, 10, segment=10)
    J2, k2, e2, F2 = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, 10, segment=None)   # ceil(sqrt(10)) = 4
    J3, k3, e3, F3 = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, 10, segment=1)
    assert J1 == J2 == J3
    assert torch.equal(k1, k2) and torch.equal(k1, k3)
    assert torch.equal(e1, e2) and torch.equal(e1, e3)


@pytest.mark.parametrize("dims,G,n", [((0.2, 1.0, 11, 7, 10, 6, 12), 2, 20),
                                      ((0.2, 1.0, 33, 16, 16, 16, 16), 8, 200)])
def test_gradients_match_central_differences(dims, G, n):
    """The gradient workload: kappa in [0.5, 5] and eta from seeded smooth fields;
    the 33 x 16^4 x 8-group case is the full-size gradient workload (200 steps)."""
    og, gg = pair(*dims, G=G)
    kap, eta, ks, F0, gR1, gR2 = _workload(og)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    _, gk, ge, _ = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, n)
    gk, ge = host(gk), host(ge)
    from paper_1104_5330_gb300.autograd import outgoing_flux

    def J(k, e):
        gg.set_coeffs(k, e, ks, gR1, gR2)
        F = cuda(F0)
        gg.step(F, dt, n)
        return float(outgoing_flux(gg, F).sum())

    rng = np.random.default_rng(17)
    for which, grad in (("kappa", gk), ("eta", ge)):
        for _ in range(2):
            v = I.seeded_smooth(og.r, og.theta, og.phi, None, None, int(rng.integers(1 << 30)),
                                og.R1, og.R2, with_direction=False)
            v = np.broadcast_to(v, kap.shape)
            base = kap if which == "kappa" else eta
            eps = 1e-5 * np.linalg.norm(base) / np.linalg.norm(v)
            if which == "kappa":
                fd = (J(kap + eps * v, eta) - J(kap - eps * v, eta)) / (2 * eps)
            else:
                fd = (J(kap, eta + eps * v) - J(kap, eta - eps * v)) / (2 * eps)
            ad = float(np.sum(grad * v))
            assert abs(fd - ad) <= 1e-6 * abs(fd), (which, fd, ad)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-6)])
def test_outgoing_flux_matches_oracle_and_its_seed_is_the_weights(precision, tol):
    """ts_outgoing_flux against the oracle's J_R2 (Eq. Flux, App. A), and
    ts_outgoing_flux_adjoint against the oracle's weights at r = R2 scaled by a
    per-group cotangent, zero at every other radial node."""
    og, gg = pair(0.2, 1.0, 11, 7, 10, 6, 12, G=3, precision=precision)
    F = np.random.default_rng(31).standard_normal(og.shape) + 2.0
    dt = torch.float64 if precision == 0 else torch.float32
    Fd = cuda(F, dt)
    J = host(gg.outgoing_flux(Fd))
    Fo = host(Fd)                                    # the values the GPU saw
    JR2 = og.moments(Fo)[4]
    assert rel_l2(J, JR2) < tol
    _, _, _, _, J2 = gg.moments(Fd)
    assert rel_l2(J, host(J2)) < 1e-13
    gJ = np.array([0.5, -1.25, 2.0])
    lam = torch.full(og.shape, float("nan"), dtype=dt, device="cuda")
    T().ts_outgoing_flux_adjoint(gg.handle, cuda(gJ), lam)
    expect = np.zeros(og.shape)
    expect[:, -1] = gJ[:, None, None, None, None] * og.outgoing_flux_weights()[None]
    assert rel_l2(host(lam), expect) < (1e-15 if precision == 0 else 1e-7)
    assert np.all(host(lam)[:, :-1] == 0.0)


def test_outgoing_flux_backward_is_the_library_seed():
    from paper_1104_5330_gb300.autograd import outgoing_flux
    og, gg = pair(0.2, 1.0, 9, 6, 8, 6, 8, G=2)
    F = cuda(np.random.default_rng(5).standard_normal(og.shape)).requires_grad_()
    (outgoing_flux(gg, F) * torch.tensor([3.0, -1.0], dtype=torch.float64, device="cuda")).sum().backward()
    expect = np.zeros(og.shape)
    expect[:, -1] = np.array([3.0, -1.0])[:, None, None, None, None] * og.outgoing_flux_weights()[None]
    assert rel_l2(host(F.grad), expect) < 1e-15


@pytest.mark.parametrize("first", [False, True])
def test_ab2_adjoint_step_matches_oracle(first):
    """ts_adjoint_step_ab2 against the oracle's AB2 adjoint step (same F_n, lam,
    lam_prev): dObj/dF_n, the shifted level and both gradients."""
    og, gg = pair(0.2, 1.0, 11, 7, 10, 6, 12, G=2, scheme=2)
    kap, eta, ks, F0, gR1, gR2 = _workload(og)
    gg.set_coeffs(kap, eta, ks, gR1, gR2)
    op = OProblem(og, kap, eta, ks, gR1, gR2, scheme="ab2")
    rng = np.random.default_rng(41)
    lam, lp = rng.standard_normal(og.shape), rng.standard_normal(og.shape)
    dt = I.dt_rule(0.2, 1.0, og.Nr, 0.2)
    L, LP = cuda(lam), cuda(lp)
    gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
    ge = torch.zeros_like(gk)
    T().ts_adjoint_step_ab2(gg.handle, cuda(F0), L, LP, gk, ge, dt, first)
    lam_n, a, b = op.adjoint_step_ab2(F0, lam, lp, dt, first)
    assert rel_l2(host(L), lam_n) < 1e-12
    assert np.array_equal(host(LP), lam)
    assert rel_l2(host(gk), a) < 1e-12 and rel_l2(host(ge), b) < 1e-12


def test_ab2_gradients_match_oracle_adjoint_and_central_differences():
    """Gradients of the outgoing flux after 9 AB2 steps (checkpoint segments of 3:
    each recomputation resumes from (F_s, K_{s-1})) against the oracle's AB2
    adjoint chain (1e-12) and central finite differences of the GPU forward (1e-6)."""
    from paper_1104_5330_gb300.autograd import outgoing_flux
    og, gg = pair(0.2, 1.0, 11, 7, 10, 6, 12, G=2, scheme=2)
    kap, eta, ks, F0, gR1, gR2 = _workload(og)
    dt = I.dt_rule(0.2, 1.0, og.Nr, 0.2)
    n = 9
    J1, gk, ge, _ = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, n, segment=3)
    J2, gk2, ge2, _ = _grads(gg, F0, kap, eta, ks, gR1, gR2, dt, n, segment=n)
    assert rel_l2(host(gk), host(gk2)) < 1e-14 and rel_l2(host(ge), host(ge2)) < 1e-14
    op = OProblem(og, kap, eta, ks, gR1, gR2, scheme="ab2")
    Fs = [F0]
    for _ in range(n):
        Fs.append(op.step(Fs[-1], dt))
    lam = np.zeros(og.shape)
    lam[:, -1] = og.outgoing_flux_weights()
    lp = np.zeros_like(lam)
    GK, GE = np.zeros_like(kap), np.zeros_like(eta)
    for m in range(n - 1, -1, -1):
        ln, a, b = op.adjoint_step_ab2(Fs[m], lam, lp, dt, m == 0)
        lp, lam = lam, ln
        GK += a
        GE += b
    assert rel_l2(host(gk), GK) < 1e-12
    assert rel_l2(host(ge), GE) < 1e-12

    def J(k, e):
        gg.set_coeffs(k, e, ks, gR1, gR2)
        F = cuda(F0)
        gg.step(F, dt, n)
        return float(outgoing_flux(gg, F).sum())

    v = np.broadcast_to(I.seeded_smooth(og.r, og.theta, og.phi, None, None, 99, og.R1, og.R2,
                                        with_direction=False), kap.shape)
    for base, grad, which in ((kap, host(gk), "kappa"), (eta, host(ge), "eta")):
        eps = 1e-5 * np.linalg.norm(base) / np.linalg.norm(v)
        if which == "kappa":
            fd = (J(kap + eps * v, eta) - J(kap - eps * v, eta)) / (2 * eps)
        else:
            fd = (J(kap, eta + eps * v) - J(kap, eta - eps * v)) / (2 * eps)
        assert abs(fd - float(np.sum(grad * v))) <= 1e-6 * abs(fd), which
