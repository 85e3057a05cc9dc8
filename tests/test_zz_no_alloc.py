"""ts_moments_noalloc, the entry point for callers that cannot allocate device
memory (a process whose device memory belongs to another allocator's pool, a
fixed device-memory budget, or a loop that cannot afford an allocation's
synchronisation). It must give ts_moments' outputs while its scratch lives in
a static device array shared by every call; two calls in a row with different
inputs check that no state from the first leaks into the second.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest
import torch

from gpu_common import T, cuda, host, pair, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1104_5330_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    yield


def _outputs(shape, G):
    z = lambda *s: torch.full(s, float("nan"), dtype=torch.float64, device="cuda")
    return z(*shape[:4]), z(3, *shape[:4]), z(G), z(G), z(G)


CASES = [
    # (dims, groups, precision): odd N_r (even number of Chebyshev intervals), the float
    # precisions, an even N_r (the Clenshaw-Curtis weights' odd-N branch), 64 direction
    # nodes per axis (the kernel's whole direction tables), and a grid whose scratch need
    # groups*Nr*Nt*Np + 2*groups*Nt*Np is exactly the static maximum 2^21
    ((0.2, 1.0, 11, 7, 10, 6, 12), 3, 0),
    ((0.2, 1.0, 11, 7, 10, 6, 12), 3, 1),
    ((0.2, 1.0, 11, 7, 10, 6, 12), 2, 2),
    ((0.2, 1.0, 11, 7, 10, 6, 12), 2, 3),
    ((0.2, 1.0, 12, 5, 6, 8, 8), 2, 0),
    ((0.2, 1.0, 5, 2, 2, 64, 64), 1, 0),
    ((0.2, 1.0, 126, 64, 64, 2, 2), 4, 0),
]


@pytest.mark.parametrize("dims,G,precision", CASES)
def test_noalloc_moments_match_ts_moments_twice(dims, G, precision):
    tol = 1e-12
    if dims[2] == 126:
        assert G * dims[2] * dims[3] * dims[4] + 2 * G * dims[3] * dims[4] == 1 << 21
    og, gg = pair(*dims, G=G, precision=precision)
    dt = torch.float64 if precision == 0 else torch.float32
    for call, seed in enumerate((21, 22)):
        F = cuda(np.random.default_rng(seed).standard_normal(og.shape) + 1.5 * call, dt)
        ref = gg.moments(F)                                   # existing entry point
        out = _outputs(og.shape, G)
        T().ts_moments_noalloc(gg.desc, F, *out)
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            assert rel_l2(host(a), host(b)) < tol, call


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    ts = T()
    d = ts.GridDesc(0.2, 1.0, 129, 64, 64, 2, 2, 8, 0, 0, 0, 0, 36.0, 16)   # 8*129*64*64 > 2^21
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TSError) as e:
        ts.ts_moments_noalloc(d, F)
    assert e.value.status == ts.TS_ERR_UNSUPPORTED
    assert "static maximum" in str(e.value)
