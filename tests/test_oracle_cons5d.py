"""Pins of the conservative 5-D oracle (App. A, Eq. Cohercons) against facts the
paper and the mathematics fix, independent of the oracle's own arithmetic:

  * SymPy: for a Cartesian polynomial P the flux form applied to J P equals
    J omega.grad P (the streaming operator of Eq. prop2 times the volume element
    J = r^2 sin th sin Th), exactly on a grid that resolves J P;
  * the divergence theorem term by term (Eq. Cons): for EVERY grid function the
    r flux integrates to J_R2 - J_R1 and the ph, Th and Ph fluxes and the
    scattering term to zero; the th flux converges spectrally for smooth data;
  * closed forms: N of F = 1 is the phase-space volume (4 pi)^2 (R2^3 - R1^3)/3;
    the number and fluxes equal the plain form's moments of F = Fhat / J;
  * a homogeneous isotropic equilibrium (eta = kappa F) is a fixed point;
  * spherically symmetric data stay spherically symmetric, and RK4's number
    changes by exactly dt sum_s b_s (J_R1 - J_R2)(U_s) (no Tau rows);
  * without Tau rows both forms advance the same solution, their difference
    converging with N_r.
``test_planted_mistakes_fail_a_pin`` checks that plausible mistakes in the
conservative oracle make at least one of these fail.
"""
import numpy as np
import pytest
import sympy as sp

import analytic as A
from oracle import conservative5d as C
from oracle.transport import Grid, Problem
from paper_1104_5330_gb300 import inputs as I

POLY = ("x", "z", "wx", "wy*wz", "xy+wz", "x*wy-z^2", "cubic")


def _integral(g, T):
    W, _ = C.hat_weights(g)
    return np.einsum("gijlkm,ijlkm->g", T, W)


def _random(g, seed, strip_theta_modes=False):
    """Random Fhat; optionally without the Fourier modes (m = 0 in ph, M = +-1 in
    Ph), the only ones the th flux (sin Th cos Ph / r) Fhat brings into the
    ph and Ph trapezoid sums."""
    X = np.random.default_rng(seed).standard_normal(g.shape)
    if strip_theta_modes:
        c = np.fft.fft(np.fft.fft(X, axis=3), axis=5)
        c[:, :, :, 0, :, 1] = 0.0
        c[:, :, :, 0, :, -1] = 0.0
        X = np.real(np.fft.ifft(np.fft.ifft(c, axis=5), axis=3))
    return X


# ------------------------------------------------------------------ pin helpers
def pin_flux_form_polynomials(g):
    J = C.jacobian(g)
    worst = 0.0
    for name in POLY:
        P, adv = A.cartesian_case(name)
        E = J * A.on_grid(adv, g)
        L = C.liouville_hat(g, J * A.on_grid(P, g))
        worst = max(worst, np.abs(L - E).max() / max(1.0, np.abs(E).max()))
    return worst


def pin_term_balance(g, seed=1):
    """Largest term-by-term balance error (relative to the fluxes and number)
    over the r, ph, Th and Ph fluxes and the scattering term, random Fhat."""
    X = _random(g, seed)
    rng = np.random.default_rng(seed + 1)
    ks = 0.3 + rng.random((g.G, g.Nr, g.Nt, g.Np))
    pr = C.ConservativeProblem(g, kappa_s=ks, scatter_b=-0.3, scatter_c=0.75, bc="none")
    J1, J2 = pr.fluxes(X)
    scale = np.abs(J1).max() + np.abs(J2).max() + np.abs(pr.number(X)).max()
    t_r, t_th, t_ph, t_Th, t_Ph = C.liouville_terms(g, X)
    errs = [np.abs(_integral(g, t_r) - (J2 - J1)).max()]
    errs += [np.abs(_integral(g, t)).max() for t in (t_ph, t_Th, t_Ph)]
    errs.append(np.abs(pr.number(pr.collision(X))).max())
    # what is left of the balance is the th flux's integral
    errs.append(np.abs(pr.balance_residual(X) + _integral(g, t_th)).max())
    return max(errs) / scale


def pin_number_against_moments(g):
    X = _random(g, 4) + 3.0
    pr = C.ConservativeProblem(g)
    _, _, N, J1, J2 = g.moments(X / C.jacobian(g))
    N_h, (J1_h, J2_h) = pr.number(X), pr.fluxes(X)
    vol = (4 * np.pi) ** 2 * (g.R2 ** 3 - g.R1 ** 3) / 3.0
    one = pr.number(np.broadcast_to(C.jacobian(g), g.shape))
    return max(np.abs(N_h - N).max() / np.abs(N).max(),
               np.abs(J1_h - J1).max() / np.abs(J1).max(),
               np.abs(J2_h - J2).max() / np.abs(J2).max(),
               np.abs(one - vol).max() / vol)


def pin_equilibrium(g):
    rng = np.random.default_rng(5)
    kap = 0.5 + rng.random((g.G, g.Nr, g.Nt, g.Np))
    F = 2.5
    pr = C.ConservativeProblem(g, kappa=kap, eta=kap * F, kappa_s=kap, scatter_b=-0.2,
                               scatter_c=0.75)
    X = F * np.broadcast_to(C.jacobian(g), g.shape)
    return np.abs(pr.rhs(X)).max() / np.abs(X).max()


def pin_symmetric_rk4_balance(nsteps=6, dt=2e-3):
    """Spherically symmetric Fhat = J h(r, Th), h random (unresolved in r and Th):
    symmetry kept, and N_n - N_0 + dt sum b_s (J_R2 - J_R1)(U_s) = 0."""
    g = Grid(0.3, 1.0, 10, 6, 4, 8, 6)
    h = np.random.default_rng(6).standard_normal((1, g.Nr, 1, 1, g.NT, 1))
    X = C.jacobian(g) * h * np.ones(g.shape)
    ks = np.broadcast_to((0.5 + g.r)[None, :, None, None], (1, g.Nr, g.Nt, g.Np))
    pr = C.ConservativeProblem(g, kappa_s=ks, scatter_c=0.75, bc="none")
    N0 = pr.number(X)
    flux = 0.0
    for _ in range(nsteps):
        X, stages = pr.rk4_step(X, dt, keep_stages=True)
        for b, U in zip((1 / 6, 1 / 3, 1 / 3, 1 / 6), stages):
            J1, J2 = pr.fluxes(U)
            flux = flux + dt * b * (J2 - J1)
    hs = X / C.jacobian(g)
    sym = np.abs(hs - hs[:, :, :1, :1, :, :1]).max() / np.abs(hs).max()
    bal = np.abs(pr.number(X) - N0 + flux).max() / np.abs(N0).max()
    return max(sym, bal)


def pin_forms_agree(Nr, nsteps=5):
    g = Grid(0.2, 1.0, Nr, 12, 12, 12, 12)
    F0 = I.seeded_smooth(g.r, g.theta, g.phi, g.Theta, g.Phi, 7, g.R1, g.R2)[None]
    kap = np.full((1, Nr, 12, 12), 0.5)
    pp = Problem(g, kap, 0.3 * kap, 0.7 * kap, bc="none")
    ph = C.ConservativeProblem(g, kap, 0.3 * kap, 0.7 * kap, bc="none")
    dt = 0.4 * np.diff(g.r).min()
    Fp = pp.run(F0, dt, nsteps)
    Fh = ph.run(C.jacobian(g) * F0, dt, nsteps)
    return np.abs(Fh / C.jacobian(g) - Fp).max() / np.abs(Fp).max()


def theta_flux_integral(Nt):
    """Relative integral of the th flux for exp(0.7 x + z)(1 + wx + wz/2)."""
    expr = (sp.exp(0.7 * A.x + A.z) * (1 + A.wx + 0.5 * A.wz)).subs(A.SPH)
    g = Grid(0.2, 1.0, 12, Nt, 8, 8, 8)
    X = C.jacobian(g) * A.on_grid(expr, g)
    J1, J2 = C.ConservativeProblem(g).fluxes(X)
    return abs(_integral(g, C.liouville_terms(g, X)[1])[0]) / (abs(J1[0]) + abs(J2[0]))


# ------------------------------------------------------------------------ tests
def test_flux_form_is_jacobian_times_omega_dot_grad():
    assert pin_flux_form_polynomials(Grid(0.2, 1.0, 12, 10, 10, 10, 10)) < 1e-12
    assert pin_flux_form_polynomials(Grid(0.2, 1.0, 11, 7, 10, 6, 12)) < 1e-12


@pytest.mark.parametrize("dims", [(0.2, 1.0, 10, 8, 8, 8, 8), (0.2, 1.0, 11, 7, 10, 6, 12),
                                  (0.5, 1.5, 9, 6, 6, 10, 8)])
def test_every_flux_but_theta_integrates_exactly(dims):
    assert pin_term_balance(Grid(*dims, groups=2)) < 1e-13


def test_theta_flux_converges_spectrally():
    e = [theta_flux_integral(n) for n in (4, 8, 12)]
    assert e[0] > 1e-4 and e[1] < 1e-5 and e[2] < 1e-10
    assert e[2] < 1e-3 * e[1] < 1e-6 * e[0]


def test_number_and_fluxes_are_the_plain_moments():
    assert pin_number_against_moments(Grid(0.2, 1.0, 9, 6, 8, 8, 6, groups=2)) < 1e-13


def test_homogeneous_equilibrium_is_a_fixed_point():
    assert pin_equilibrium(Grid(0.4, 1.2, 7, 6, 6, 8, 8, groups=2)) < 1e-13


def test_balance_is_exact_without_theta_coupled_modes_and_the_plain_one_is_not():
    g = Grid(0.2, 1.0, 10, 8, 8, 8, 8, groups=2)
    X = _random(g, 3, strip_theta_modes=True)
    ks = 0.3 + np.random.default_rng(4).random((2, g.Nr, g.Nt, g.Np))
    ph = C.ConservativeProblem(g, kappa_s=ks, scatter_b=-0.3, scatter_c=0.75, bc="none")
    pp = Problem(g, kappa_s=ks, scatter_b=-0.3, scatter_c=0.75, bc="none")
    N, J1, J2, dN, S = ph.balance(X)
    scale = np.abs(J1).max() + np.abs(J2).max() + np.abs(N).max()
    assert np.abs(dN + J2 - J1 - S).max() < 1e-13 * scale
    Np_, J1p, J2p, dNp, Sp = C.plain_balance(pp, X / C.jacobian(g))
    assert np.abs(dNp + J2p - J1p - Sp).max() > 1e-3 * scale


def test_spherical_symmetry_and_rk4_number_balance():
    assert pin_symmetric_rk4_balance() < 1e-13


def test_forms_advance_the_same_solution():
    e13, e17 = pin_forms_agree(13), pin_forms_agree(17)
    assert e13 < 1e-4 and e17 < 0.1 * e13


def test_source_integral_and_the_conservative_state():
    g = Grid(0.3, 1.0, 7, 4, 4, 6, 4)
    rng = np.random.default_rng(8)
    kap = 0.5 + rng.random((1, g.Nr, g.Nt, g.Np))
    eta = rng.random((1, g.Nr, g.Nt, g.Np))
    pr = C.ConservativeProblem(g, kappa=kap, eta=eta, bc="none")
    X = _random(g, 9)
    F = pr.from_hat(X)
    np.testing.assert_allclose(pr.to_hat(F), X, rtol=1e-15, atol=1e-15)
    # S = int r^2 dr dOmega_x dOmega (eta - kappa F): the plain moments of eta - kappa F
    S = g.moments(eta[..., None, None] - kap[..., None, None] * F)[2]
    assert np.abs(pr.source(X) - S).max() < 1e-13 * np.abs(S).max()
    with pytest.raises(ValueError):
        C.ConservativeProblem(g, scheme="split")


# --------------------------------------------------------------- planted mistakes
MUTANTS = {}


def mutant(name):
    def deco(f):
        MUTANTS[name] = f
        return f
    return deco


@mutant("th continuation with +Fhat (the plain form's parity)")
def _c1(mp):
    def bad(g, Fh):
        ext = g._extend(Fh, 2, g._partner_th(Fh))
        return np.take(g._fourier_deriv(ext, 2), np.arange(g.Nt), axis=2)
    mp.setattr(C, "d_th_odd", bad)


@mutant("Th continuation with +Fhat")
def _c2(mp):
    def bad(g, Fh):
        ext = g._extend(Fh, 4, g._partner_Th(Fh))
        return np.take(g._fourier_deriv(ext, 4), np.arange(g.NT), axis=4)
    mp.setattr(C, "d_Th_odd", bad)


@mutant("Th term without the Nyquist projection")
def _c3(mp):
    mp.setattr(C, "nyquist_free_Th", lambda g, Fh: Fh)


@mutant("Ph flux as sin Ph dFhat/dPh (cos Ph Fhat dropped)")
def _c4(mp):
    orig = C.liouville_terms

    def bad(g, Fh):
        t = orig(g, Fh)
        th = g.theta.reshape(1, 1, -1, 1, 1, 1)
        Th = g.Theta.reshape(1, 1, 1, 1, -1, 1)
        Ph = g.Phi.reshape(1, 1, 1, 1, 1, -1)
        r = g.r.reshape(1, -1, 1, 1, 1, 1)
        t_Ph = -np.sin(Th) * np.cos(th) / (np.sin(th) * r) * np.sin(Ph) * g.d_Ph(Fh)
        return t[0], t[1], t[2], t[3], t_Ph
    mp.setattr(C, "liouville_terms", bad)


@mutant("collision not multiplied by the volume element")
def _c5(mp):
    mp.setattr(C.ConservativeProblem, "collision", lambda self, Fh: Problem.collision(self, Fh))


@mutant("number weights without 1/sin Th")
def _c6(mp):
    orig = C.hat_weights

    def bad(g):
        W, ws = orig(g)
        s = np.sin(g.Theta)[None, None, :, None]
        return W * s[None], ws * s
    mp.setattr(C, "hat_weights", bad)


@mutant("Th term's cos Th product with the wrong sign")
def _c7(mp):
    orig = C.nyquist_free_Th
    mp.setattr(C, "nyquist_free_Th", lambda g, Fh: -orig(g, Fh))


def _all_pins_pass():
    checks = [
        lambda: pin_flux_form_polynomials(Grid(0.2, 1.0, 11, 7, 10, 6, 12)) < 1e-12,
        lambda: pin_term_balance(Grid(0.2, 1.0, 10, 8, 8, 8, 8, groups=2)) < 1e-13,
        lambda: pin_number_against_moments(Grid(0.2, 1.0, 9, 6, 8, 8, 6, groups=2)) < 1e-13,
        lambda: pin_equilibrium(Grid(0.4, 1.2, 7, 6, 6, 8, 8, groups=2)) < 1e-13,
        lambda: pin_symmetric_rk4_balance(nsteps=2) < 1e-13,
    ]
    return all(c() for c in checks)


def test_pins_pass_on_the_oracle():
    assert _all_pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_fail_a_pin(name, monkeypatch):
    with monkeypatch.context() as mp:
        MUTANTS[name](mp)
        assert not _all_pins_pass(), f"no pin caught: {name}"
