"""Second-order Adams-Bashforth time marching (Sect. 5.1) on the GPU against the
FP64 oracle: F + dt (3/2 K_n - 1/2 K_{n-1}), forward-Euler first step, the
history kept by the grid between calls.

Bars: relative L2 <= 1e-12 (FP64) and <= 1e-5 (FP32 variants) after tens of
steps at dt = 0.2 x the smallest radial spacing (AB2's stability limit on these
grids is between 0.2 and 0.25 of it; RK4's rule of 0.4 diverges); history
handling bit for bit."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, pair, rel_l2
from oracle.transport import Problem as OProblem
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5
CFL = 0.2

RAGGED = (0.2, 1.0, 11, 7, 10, 6, 12)
SQUARE = (0.2, 1.0, 17, 16, 16, 16, 16)
WARP = (0.2, 1.0, 13, 6, 10, 8, 16)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _both(dims, G, precision=0, filter_on=False, aniso=False):
    ts = T()
    og, gg = pair(*dims, G=G, precision=precision, scheme=ts.TS_AB2, filter_on=filter_on)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    b = I.signed_field(og.r, og.theta, og.phi, G, 7, og.R1, og.R2) if aniso else None
    op = OProblem(og, kap, eta, 4.0 * ks, gR1, gR2, scheme="ab2", filter_on=filter_on,
                  scatter_b=b)
    gg.set_coeffs(kap, eta, 4.0 * ks, gR1, gR2)
    if aniso:
        gg.set_scattering_anisotropy(b)
    return og, gg, op, F0, I.dt_rule(dims[0], dims[1], dims[2], CFL)


@pytest.mark.parametrize("dims,G,n", [(RAGGED, 3, 40), (SQUARE, 2, 20), (WARP, 2, 30)])
def test_ab2_parity(dims, G, n):
    og, gg, op, F0, dt = _both(dims, G)
    Fg = cuda(F0)
    gg.step(Fg, dt, n)
    assert rel_l2(host(Fg), op.run(F0, dt, n)) < FP64_TOL


def test_ab2_full_size_33x16():
    og, gg, op, F0, dt = _both((0.2, 1.0, 33, 16, 16, 16, 16), 4)
    Fg = cuda(F0)
    gg.step(Fg, dt, 3)
    assert rel_l2(host(Fg), op.run(F0, dt, 3)) < FP64_TOL


def test_ab2_with_filter_and_anisotropic_scattering():
    og, gg, op, F0, dt = _both(RAGGED, 2, filter_on=True, aniso=True)
    Fg = cuda(F0)
    gg.step(Fg, dt, 25)
    assert rel_l2(host(Fg), op.run(F0, dt, 25)) < FP64_TOL


@pytest.mark.parametrize("precision", [1, 2, 3, 4])
def test_ab2_fp32_variants(precision):
    og, gg, op, F0, dt = _both(SQUARE, 2, precision=precision)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 20)
    assert rel_l2(host(Fg), op.run(F0, dt, 20)) < FP32_TOL


def test_ab2_history_between_calls_and_restarts():
    og, gg, op, F0, dt = _both(WARP, 2)
    a = cuda(F0)
    gg.step(a, dt, 4)
    gg.step(a, dt, 3)                   # history carried over
    b = cuda(F0)
    gg.step(b, dt, 7)                   # another field pointer: restarts by itself
    assert torch.equal(a, b)
    assert rel_l2(host(a), op.run(F0, dt, 7)) < FP64_TOL
    c = cuda(F0)
    gg.step(c, dt, 4)
    gg.reset_history()                  # explicit restart in the middle
    gg.step(c, dt, 3)
    op.reset_history()
    Fo = op.run(F0, dt, 4)
    op.reset_history()
    Fo = op.run(Fo, dt, 3)
    assert rel_l2(host(c), Fo) < FP64_TOL
    assert not torch.equal(a, c)


def test_ab2_host_entry_point_keeps_its_own_history():
    ts = T()
    og, gg, op, F0, dt = _both(RAGGED, 1)
    Fh = torch.as_tensor(F0, dtype=torch.float64).contiguous().pin_memory()
    ts.ts_step_host(gg.handle, Fh, dt, 3)
    ts.ts_step_host(gg.handle, Fh, dt, 2)
    assert rel_l2(Fh.numpy(), op.run(F0, dt, 5)) < FP64_TOL


def test_ab2_batches_are_not_mixed_and_the_rk4_adjoint_refuses_ab2():
    ts = T()
    d = ts.GridDesc(0.2, 1.0, 9, 4, 4, 4, 4, 1, 0, ts.TS_AB2, 0, 0, 36.0, 16)
    d4 = ts.GridDesc(0.2, 1.0, 9, 4, 4, 4, 4, 1, 0, ts.TS_RK4, 0, 0, 36.0, 16)
    with pytest.raises(RuntimeError):
        ts.Batch([d, d4], autotune=False)
    og, gg, op, F0, dt = _both(RAGGED, 1)
    lam = cuda(np.ones(og.shape))
    gk = torch.zeros(gg.coef_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        gg.adjoint_step(cuda(F0), lam, gk, torch.zeros_like(gk), dt)
