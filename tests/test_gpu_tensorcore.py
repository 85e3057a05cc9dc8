"""The tensor-core radial passes (tcgen05.mma with a TMEM accumulator):
TS_TF32X3 (operands x = hi + lo in TF32, products hi*hi + hi*lo + lo*hi) and
TS_BF16X3 (operands x = b0 + b1 + b2 in bf16, the six products of total order
<= 2), both accumulated in FP32. Bar: the FP32 bound (1e-5 relative L2)
against the FP64 oracle, and agreement with the FP32 SIMT passes."""
import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, pair, rel_l2, setup_both
from paper_1104_5330_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# 128-column tiles: whole (256 = 2 tiles), ragged (96 < 128, 192 = 1.5 tiles)
GRIDS = [(0.2, 1.0, 33, 8, 8, 16, 16), (0.2, 1.0, 17, 6, 4, 8, 12), (0.3, 1.2, 65, 4, 6, 16, 12),
         (0.2, 1.0, 9, 4, 4, 8, 8)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


TC = [3, 4]   # TS_TF32X3, TS_BF16X3


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("dims", GRIDS)
def test_tensor_core_rhs_and_steps_against_oracle(dims, prec):
    og, gg = pair(*dims, G=2, precision=prec)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = setup_both(og, gg, kap, eta, ks, gR1, gR2)
    F = F0 + 0.1 * np.random.default_rng(3).standard_normal(og.shape)
    K = host(gg.rhs(cuda(F, torch.float32)))
    T().ts_sync_status(gg.handle)
    assert rel_l2(K, op.rhs(F)) < 1e-5
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 20)
    T().ts_sync_status(gg.handle)
    assert rel_l2(host(Fg), op.run(F0, dt, 20)) < 1e-5


@pytest.mark.parametrize("prec", TC)
def test_tensor_core_radial_derivative_on_polynomial(prec):
    """cos(Theta) p'(r) for F = p(r) at 65 nodes through the tensor cores."""
    og, gg = pair(0.2, 1.0, 65, 4, 4, 16, 8, precision=prec)
    gg.set_coeffs()
    rng = np.random.default_rng(9)
    p = np.polynomial.Chebyshev(rng.standard_normal(30) * 0.8 ** np.arange(30), domain=[0.2, 1.0])
    F = np.ascontiguousarray(np.broadcast_to(p(og.r)[None, :, None, None, None, None], og.shape))
    LF = host(gg.liouville(cuda(F, torch.float32)))
    E = np.cos(og.Theta)[None, None, None, None, :, None] * p.deriv()(og.r)[None, :, None, None, None, None]
    assert rel_l2(LF, np.broadcast_to(E, og.shape)) < 1e-5


@pytest.mark.parametrize("prec", TC)
def test_tensor_core_agrees_with_simt_fp32(prec):
    dims = GRIDS[0]
    og, tc = pair(*dims, G=3, precision=prec)
    _, simt = pair(*dims, G=3, precision=1)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    for g in (tc, simt):
        g.set_coeffs(kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    a, b = cuda(F0, torch.float32), cuda(F0, torch.float32)
    tc.step(a, dt, 10)
    simt.step(b, dt, 10)
    T().ts_sync_status(tc.handle)
    assert rel_l2(host(a), host(b)) < 2e-6


@pytest.mark.parametrize("prec", TC)
def test_operand_wait_timeout_is_reported_and_the_grid_recovers(prec):
    """Failure detection without a fault: the tensor-core pass's operand wait is
    made to give up at once (ts_set_wait_limit < 0). Every CTA then issues no
    products, latches the grid's error flag, drains its own bulk copy with the
    full bound and frees its tensor memory; ts_sync_status reports
    TS_ERR_TIMEOUT once and clears the flag. With the default bound back, the
    next steps return TS_OK and match the oracle."""
    ts = T()
    dims = GRIDS[1]
    og, gg = pair(*dims, G=2, precision=prec)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = setup_both(og, gg, kap, eta, ks, gR1, gR2)
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    ts.ts_set_wait_limit(gg.handle, -1)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 1)
    with pytest.raises(ts.TSError) as e:
        ts.ts_sync_status(gg.handle)
    assert e.value.status == ts.TS_ERR_TIMEOUT
    ts.ts_sync_status(gg.handle)          # reported once, then cleared
    ts.ts_set_wait_limit(gg.handle, 0)
    Fg = cuda(F0, torch.float32)
    gg.step(Fg, dt, 5)
    ts.ts_sync_status(gg.handle)
    assert rel_l2(host(Fg), op.run(F0, dt, 5)) < 1e-5


# 16 x 16 direction blocks: the angular pass also runs on the tensor cores for
# TS_TF32X3 (8 blocks per tile; the last tile of these grids is ragged)
ANG16 = [(0.2, 1.0, 9, 3, 2, 16, 16), (0.2, 1.0, 17, 4, 6, 16, 16), (0.2, 1.0, 33, 16, 16, 16, 16)]


def _grid_tc_angular(dims, G, on):
    import os
    old = os.environ.get("TS_TC_ANGULAR")
    os.environ["TS_TC_ANGULAR"] = "1" if on else "0"
    try:
        return pair(*dims, G=G, precision=3)
    finally:
        if old is None:
            del os.environ["TS_TC_ANGULAR"]
        else:
            os.environ["TS_TC_ANGULAR"] = old


@pytest.mark.parametrize("dims", ANG16)
def test_tensor_core_angular_pass_against_oracle_and_simt(dims):
    G = 3 if dims[2] < 33 else 4
    og, tc = _grid_tc_angular(dims, G, True)
    _, simt = _grid_tc_angular(dims, G, False)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    op = setup_both(og, tc, kap, eta, ks, gR1, gR2)
    simt.set_coeffs(kap, eta, ks, gR1, gR2)
    F = F0 + 0.1 * np.random.default_rng(8).standard_normal(og.shape)
    Kt = host(tc.rhs(cuda(F, torch.float32)))
    T().ts_sync_status(tc.handle)
    assert rel_l2(Kt, op.rhs(F)) < 1e-5
    assert rel_l2(Kt, host(simt.rhs(cuda(F, torch.float32)))) < 2e-6
    LF = host(tc.liouville(cuda(F, torch.float32)))
    assert rel_l2(LF, og.liouville(F)) < 1e-5
    dt = I.dt_rule(dims[0], dims[1], dims[2])
    a, b = cuda(F0, torch.float32), cuda(F0, torch.float32)
    tc.step(a, dt, 10)
    simt.step(b, dt, 10)
    T().ts_sync_status(tc.handle)
    assert rel_l2(host(a), op.run(F0, dt, 10)) < 1e-5
    assert rel_l2(host(a), host(b)) < 2e-6
