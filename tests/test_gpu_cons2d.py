"""The conservative 2-D (r, Theta) variant of App. B (Fhat = r^2 sin Th F,
Eq. speccons) through the C ABI: right-hand sides and RK4 steps against the
FP64 oracle (1e-12), and the discrete number balance dN/dt + J_R2 - J_R1 = 0
(Eq. Cons) to rounding."""
import numpy as np
import pytest
import torch

from gpu_common import T, cuda, host, rel_l2
from oracle.conservative2d import Grid2D, Problem2D

pytestmark = pytest.mark.gpu

R1, R2 = 0.2, 1.0
SIZES = [(9, 8), (10, 8), (33, 24), (65, 32), (17, 6)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _data(Nr, NT, P, seed):
    g = Grid2D(R1, R2, Nr, NT)
    rng = np.random.default_rng(seed)
    ks = 0.3 + rng.uniform(0, 2, (P, 1)) * (1 + 0.5 * np.cos(2 * g.r))[None, :]
    m = np.arange(1, NT + 1)          # every sine mode, Nyquist included
    b = rng.standard_normal((P, Nr, NT)) * 0.7 ** m[None, None, :]
    X = np.einsum("pim,km->pik", b, np.sin(np.outer(g.Theta, m)))
    g1 = X[:, 0, :NT // 2].copy()
    g2 = X[:, -1, NT // 2:].copy()
    return g, ks, X, g1, g2


def _pair(Nr, NT, P, c, bc, ks, g1, g2):
    gg = T().Cons2D(R1, R2, Nr, NT, problems=P, scatter_c=c, bc=0 if bc == "tau" else 1)
    gg.set_coeffs(ks, g1, g2)
    return gg


def test_nodes_match_oracle():
    gg = T().Cons2D(R1, R2, 17, 12)
    r, th = gg.nodes()
    g = Grid2D(R1, R2, 17, 12)
    assert np.abs(r - g.r).max() < 1e-15 and np.abs(th - g.Theta).max() < 1e-15


@pytest.mark.parametrize("c", [0.0, 0.75])
@pytest.mark.parametrize("bc", ["tau", "none"])
@pytest.mark.parametrize("size", SIZES)
def test_rhs_parity(size, bc, c):
    Nr, NT = size
    g, ks, X, g1, g2 = _data(Nr, NT, 3, 11)
    gg = _pair(Nr, NT, 3, c, bc, ks, g1, g2)
    K = host(gg.rhs(cuda(X)))
    Ko = Problem2D(g, ks, c=c, form="hat", bc=bc).rhs(X)
    assert rel_l2(K, Ko) < 1e-12


@pytest.mark.parametrize("size", SIZES)
def test_steps_parity(size):
    Nr, NT = size
    g, ks, X, g1, g2 = _data(Nr, NT, 2, 12)
    gg = _pair(Nr, NT, 2, 0.75, "tau", ks, g1, g2)
    dt = 0.4 * 0.5 * (R2 - R1) * (1 - np.cos(np.pi / (Nr - 1)))
    Xg = cuda(X)
    gg.step(Xg, dt, 40)
    Xo = Problem2D(g, ks, c=0.75, form="hat", bc="tau").run(X, dt, 40)
    assert rel_l2(host(Xg), Xo) < 1e-12


@pytest.mark.parametrize("size", SIZES)
def test_discrete_number_balance(size):
    """Without boundary rows the operator conserves N to rounding (Nyquist sine
    mode of Fhat included), and N, J_R1, J_R2 match the oracle."""
    Nr, NT = size
    g, ks, X, g1, g2 = _data(Nr, NT, 4, 13)
    gg = _pair(Nr, NT, 4, 0.75, "none", ks, g1, g2)
    NJ, res = gg.balance(cuda(X))
    NJ, res = host(NJ), host(res)
    op = Problem2D(g, ks, c=0.75, form="hat", bc="none")
    J1, J2 = op.fluxes(X)
    N = op.number(X)
    scale = np.abs(NJ).max()
    assert np.abs(NJ[:, 0] - N).max() < 1e-13 * scale
    assert np.abs(NJ[:, 1] - J1).max() < 1e-13 * scale
    assert np.abs(NJ[:, 2] - J2).max() < 1e-13 * scale
    assert np.abs(res).max() < 1e-12 * scale
    assert np.abs(op.balance_residual(X)).max() < 1e-12 * scale


def test_shell_with_lambert_inflow_against_oracle():
    """The App. B setting: empty shell 0.5 <= r <= 1, Fhat(R1, Th) = cos Th sin Th
    on the outgoing directions, nothing entering at R2, Thomson scattering from
    a plasma vanishing at R2; 200 steps."""
    Nr, NT, P = 33, 24, 3
    g = Grid2D(0.5, 1.0, Nr, NT)
    tau = np.array([0.5, 2.0, 5.0])
    prof = (1 - (g.r - 0.5) / 0.5) ** 8
    ks = 9 * tau[:, None] / 0.5 * prof[None, :]
    g1 = np.tile(np.cos(g.Theta[:NT // 2]) * np.sin(g.Theta[:NT // 2]), (P, 1))
    gg = T().Cons2D(0.5, 1.0, Nr, NT, problems=P, scatter_c=0.75)
    gg.set_coeffs(ks, g1, None)
    Xg = gg.apply_inflow(torch.zeros((P, Nr, NT), dtype=torch.float64, device="cuda"))
    X0 = np.zeros((P, Nr, NT))
    X0[:, 0, :NT // 2] = g1
    assert np.array_equal(host(Xg), X0)
    dt = 0.4 * 0.25 * (1 - np.cos(np.pi / (Nr - 1)))
    gg.step(Xg, dt, 200)
    Xo = Problem2D(g, ks, c=0.75, form="hat", bc="tau").run(X0, dt, 200)
    assert rel_l2(host(Xg), Xo) < 1e-12


# ---------------------------------------------- the three-zone radial grid (App. B)
ZSIZES = [(5, 9, 8), (4, 10, 6), (30, 25, 24)]   # (nodes per edge zone, central nodes, NTheta)


def _zdata(nA, nB, NT, P, seed):
    Nr = 2 * (nA - 1) + nB
    g = Grid2D(R1, R2, Nr, NT, zone_nodes=nA, zone_width=0.1)
    rng = np.random.default_rng(seed)
    ks = 0.3 + rng.uniform(0, 2, (P, 1)) * (1 + 0.5 * np.cos(2 * g.r))[None, :]
    m = np.arange(1, NT + 1)
    b = rng.standard_normal((P, Nr, NT)) * 0.7 ** m[None, None, :]
    X = np.einsum("pim,km->pik", b, np.sin(np.outer(g.Theta, m)))
    return g, ks, X, X[:, 0, :NT // 2].copy(), X[:, -1, NT // 2:].copy()


def _zpair(nA, nB, NT, P, c, bc, ks, g1, g2):
    ts = T()
    gg = ts.Cons2D(R1, R2, 2 * (nA - 1) + nB, NT, problems=P, scatter_c=c,
                   bc=0 if bc == "tau" else 1, radial=ts.TS_RADIAL_ZONED, zone_nodes=nA,
                   zone_width=0.1)
    gg.set_coeffs(ks, g1, g2)
    return gg


def test_zoned_nodes_match_oracle():
    ts = T()
    gg = ts.Cons2D(R1, R2, 83, 24, radial=ts.TS_RADIAL_ZONED, zone_nodes=30, zone_width=0.1)
    r, th = gg.nodes()
    g = Grid2D(R1, R2, 83, 24, zone_nodes=30, zone_width=0.1)
    assert np.abs(r - g.r).max() < 1e-15 and np.abs(th - g.Theta).max() < 1e-15


@pytest.mark.parametrize("c", [0.0, 0.75])
@pytest.mark.parametrize("bc", ["tau", "none"])
@pytest.mark.parametrize("size", ZSIZES)
def test_zoned_rhs_parity(size, bc, c):
    nA, nB, NT = size
    g, ks, X, g1, g2 = _zdata(nA, nB, NT, 3, 21)
    gg = _zpair(nA, nB, NT, 3, c, bc, ks, g1, g2)
    K = host(gg.rhs(cuda(X)))
    Ko = Problem2D(g, ks, c=c, form="hat", bc=bc).rhs(X)
    assert rel_l2(K, Ko) < 1e-12


@pytest.mark.parametrize("size", ZSIZES)
def test_zoned_steps_and_balance_parity(size):
    """40 RK4 steps against the oracle; N, J_R1, J_R2 and the balance residual
    (no longer zero: the edge zones' first-order differences) equal the oracle's."""
    nA, nB, NT = size
    g, ks, X, g1, g2 = _zdata(nA, nB, NT, 2, 22)
    gg = _zpair(nA, nB, NT, 2, 0.75, "tau", ks, g1, g2)
    dt = 0.4 * np.diff(g.r).min()
    Xg = cuda(X)
    gg.step(Xg, dt, 40)
    Xo = Problem2D(g, ks, c=0.75, form="hat", bc="tau").run(X, dt, 40)
    assert rel_l2(host(Xg), Xo) < 1e-12
    gb = _zpair(nA, nB, NT, 2, 0.75, "none", ks, g1, g2)
    NJ, res = gb.balance(cuda(X))
    NJ, res = host(NJ), host(res)
    op = Problem2D(g, ks, c=0.75, form="hat", bc="none")
    J1, J2 = op.fluxes(X)
    scale = np.abs(NJ).max()
    assert np.abs(NJ[:, 0] - op.number(X)).max() < 1e-13 * scale
    assert np.abs(NJ[:, 1] - J1).max() < 1e-13 * scale
    assert np.abs(NJ[:, 2] - J2).max() < 1e-13 * scale
    assert np.abs(res - op.balance_residual(X)).max() < 1e-11 * max(scale, np.abs(res).max())


def test_zoned_shell_with_lambert_inflow_the_papers_zones():
    """App. B's run: (30 + 25 + 30) radial nodes (edge zones of width 0.1 (R2 -
    R1), shared interfaces: N_r = 83), 24 Theta nodes, Lambert inflow at R1,
    Thomson scattering from a plasma vanishing at R2; 200 steps against the oracle."""
    ts = T()
    nA, nB, NT, P = 30, 25, 24, 3
    Nr = 2 * (nA - 1) + nB
    g = Grid2D(0.5, 1.0, Nr, NT, zone_nodes=nA, zone_width=0.1)
    tau = np.array([0.5, 2.0, 5.0])
    prof = (1 - (g.r - 0.5) / 0.5) ** 8
    ks = 9 * tau[:, None] / 0.5 * prof[None, :]
    g1 = np.tile(np.cos(g.Theta[:NT // 2]) * np.sin(g.Theta[:NT // 2]), (P, 1))
    gg = ts.Cons2D(0.5, 1.0, Nr, NT, problems=P, scatter_c=0.75, radial=ts.TS_RADIAL_ZONED,
                   zone_nodes=nA, zone_width=0.1)
    gg.set_coeffs(ks, g1, None)
    Xg = gg.apply_inflow(torch.zeros((P, Nr, NT), dtype=torch.float64, device="cuda"))
    X0 = np.zeros((P, Nr, NT))
    X0[:, 0, :NT // 2] = g1
    dt = 0.4 * np.diff(g.r).min()
    gg.step(Xg, dt, 200)
    Xo = Problem2D(g, ks, c=0.75, form="hat", bc="tau").run(X0, dt, 200)
    assert rel_l2(host(Xg), Xo) < 1e-12
    assert np.abs(host(Xg)[:, 1:]).max() > 0.05   # the emitted front has left the inflow nodes
