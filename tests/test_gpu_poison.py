"""Uninitialised reads: every workspace field of the grid (U, K, Acc, and the
adjoint's fields) starts as NaN (TS_POISON_WORKSPACE=1), and one step of each
pass form -- FP64 even/odd, generic (TS_GENERIC_PASSES=1), FP32 fused and three
passes, FP32 + FP64 rows (both forms), the tensor-core radial forms, the split scheme, AB2,
the hybrid radial grid, the adjoint -- must give exactly the result of a grid
whose workspace starts as zero. A pass that read a workspace element before
writing it would carry the NaN into the result."""
import os

import numpy as np
import pytest
import torch

from gpu_common import T, absorber_workload, cuda, host, pair

pytestmark = pytest.mark.gpu

FORMS = [
    # (name, precision, scheme, env, dims)
    ("fp64", 0, 0, {}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("fp64 generic", 0, 0, {"TS_GENERIC_PASSES": "1"}, (0.2, 1.0, 11, 7, 10, 6, 12)),
    ("fp32 fused", 1, 0, {"TS_FUSED": "1"}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("fp32 three passes", 1, 0, {}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("fp32 + fp64 rows, split", 2, 1, {}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("fp32 + fp64 rows, split, fused", 2, 1, {"TS_FUSED": "1"}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("tf32x3", 3, 0, {}, (0.2, 1.0, 17, 6, 4, 8, 12)),
    ("bf16x3", 4, 0, {}, (0.2, 1.0, 17, 6, 4, 8, 12)),
    ("fp64 ab2", 0, 2, {}, (0.2, 1.0, 17, 8, 8, 8, 16)),
    ("fp32 fused ab2", 1, 2, {"TS_FUSED": "1"}, (0.2, 1.0, 17, 8, 8, 8, 16)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _make(dims, precision, scheme, env, poison, radial=0):
    saved = {k: os.environ.get(k) for k in list(env) + ["TS_POISON_WORKSPACE"]}
    os.environ.update(env)
    os.environ["TS_POISON_WORKSPACE"] = "1" if poison else "0"
    try:
        return T().Grid(*dims, groups=2, precision=precision, scheme=scheme, radial=radial)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("name,precision,scheme,env,dims", FORMS, ids=[f[0] for f in FORMS])
def test_poisoned_workspace_changes_nothing(name, precision, scheme, env, dims):
    og, _ = pair(*dims, G=2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    dt = 0.3 * (1.0 - np.cos(np.pi / (dims[2] - 1))) * 0.4
    out = []
    for poison in (False, True):
        gg = _make(dims, precision, scheme, env, poison)
        gg.set_coeffs(kap, eta, ks, gR1, gR2)
        F = cuda(F0, gg.dtype)
        gg.step(F, dt, 2)
        K = gg.rhs(F)
        out.append((host(F), host(K)))
    for a, b in zip(*out):
        assert np.isfinite(b).all(), name
        assert np.array_equal(a, b), name


def test_poisoned_workspace_hybrid_grid_and_adjoint():
    dims = (0.5, 1.0, 17, 8, 8, 8, 16)
    og, _ = pair(*dims, G=2)
    kap, eta, ks, F0, gR1, gR2 = absorber_workload(og)
    res = []
    for poison in (False, True):
        fd = _make(dims, 0, 0, {}, poison, radial=1)
        fd.set_coeffs(kap, eta, ks, gR1, gR2)
        F = cuda(F0)
        fd.step(F, 1e-3, 2)
        ch = _make(dims, 0, 0, {}, poison)
        ch.set_coeffs(kap, eta, ks, gR1, gR2)
        lam = cuda(np.random.default_rng(4).standard_normal(og.shape))
        gk = torch.zeros(ch.coef_shape, dtype=torch.float64, device="cuda")
        ge = torch.zeros_like(gk)
        ch.adjoint_step(cuda(F0), lam, gk, ge, 1e-3)
        res.append([host(F), host(lam), host(gk), host(ge)])
    for a, b in zip(*res):
        assert np.isfinite(b).all()
        assert np.array_equal(a, b)
