"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/ts.h declares, and rejects bad arguments before touching the
device (these calls return before any CUDA call)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def T():
    from paper_1104_5330_gb300 import build
    build.build()
    import paper_1104_5330_gb300.ts as T
    return T


def test_every_declared_symbol_is_exported(T):
    names = T.declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(T.LIB, n), n
    assert "sm_103a" in T.ts_version()


def _desc(T, **kw):
    d = dict(R1=0.2, R2=1.0, Nr=9, Ntheta=8, Nphi=8, NTheta=8, NPhi=8, groups=1,
             precision=T.TS_FP64, scheme=T.TS_RK4, bc=T.TS_BC_TAU_INFLOW, filter_on=0,
             filter_alpha=36.0, filter_order=16)
    d.update(kw)
    return T.GridDesc(**d)


@pytest.mark.parametrize("kw,status", [
    (dict(Nr=2), 2), (dict(Nr=200), 2), (dict(Nphi=7), 2), (dict(NTheta=5), 2),
    (dict(NPhi=3), 2), (dict(NTheta=66), 2), (dict(R1=0.0), 1), (dict(R2=0.1), 1),
    (dict(groups=0), 1), (dict(precision=9), 2), (dict(scheme=4), 2), (dict(bc=3), 2),
    (dict(radial=3), 2), (dict(radial=1, precision=3), 2), (dict(radial=1, precision=2), 2),
    (dict(radial=2), 2), (dict(radial=2, zone_nodes=1, zone_width=0.1), 2),
    (dict(radial=2, zone_nodes=5, zone_width=0.1), 2),
    (dict(radial=2, zone_nodes=3, zone_width=0.5), 2),
    (dict(radial=2, zone_nodes=3, zone_width=float("nan")), 2),
    (dict(radial=2, zone_nodes=3, zone_width=0.1, precision=4), 2),
    (dict(form=2), 2), (dict(form=1, precision=9), 2), (dict(form=1, scheme=1), 2),
    (dict(form=1, filter_on=1), 2), (dict(form=1, radial=1), 2),
])
def test_create_grid_rejects_bad_descriptors(T, kw, status):
    h = ctypes.c_void_p()
    st = T.LIB.ts_create_grid(ctypes.byref(_desc(T, **kw)), ctypes.byref(h))
    assert st == status
    assert h.value is None
    assert len(T.LIB.ts_last_error()) > 0


def test_null_arguments_are_rejected(T):
    assert T.LIB.ts_create_grid(None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_step(None, None, ctypes.c_double(0.1), 1, None) == T.TS_ERR_ARG
    assert T.LIB.ts_moments(None, None, None, None, None, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_adjoint_step(None, None, None, None, None, ctypes.c_double(0.1), None) == T.TS_ERR_ARG
    assert T.LIB.ts_number_balance(None, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_destroy_grid(None) == T.TS_OK
    assert T.LIB.ts_field_elems(None) == 0


def test_misaligned_fields_are_rejected_before_any_device_work(T):
    """Device fields must be 16-byte aligned (the passes use 16-byte vector
    accesses): an address 4 bytes past a boundary is refused with TS_ERR_ARG,
    which ts_moments_noalloc checks before touching the device."""
    d = _desc(T)
    st = T.LIB.ts_moments_noalloc(ctypes.byref(d), ctypes.c_void_p(0x10004), None, None, None,
                                  None, None, None)
    assert st == T.TS_ERR_ARG
    assert "aligned" in T.LIB.ts_last_error().decode()


def test_probe_widen_arguments(T):
    assert T.LIB.ts_probe_widen(None, None, 0, None) == T.TS_OK
    assert T.LIB.ts_probe_widen(None, None, 5, None) == T.TS_ERR_ARG


def test_new_entry_points_reject_null_grids(T):
    assert T.LIB.ts_set_scattering_anisotropy(None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_set_scattering_quadrupole(None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_reset_history(None) == T.TS_ERR_ARG
    assert T.LIB.ts_outgoing_flux(None, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_outgoing_flux_adjoint(None, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_set_wait_limit(None, 0) == T.TS_ERR_ARG
    assert T.LIB.ts_stable_dt(None, None, 10, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_adjoint_step_ab2(None, None, None, None, None, None, ctypes.c_double(0.1), 0,
                                     None) == T.TS_ERR_ARG
    assert T.LIB.ts_set_history(None, None, None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_cons2d_create(None, None) == T.TS_ERR_ARG
    assert T.LIB.ts_cons2d_step(None, None, ctypes.c_double(0.1), 1, None) == T.TS_ERR_ARG


def test_batches_refuse_ab2_before_touching_the_device(T):
    descs = (T.GridDesc * 2)(_desc(T), _desc(T, scheme=T.TS_AB2))
    h = ctypes.c_void_p()
    assert T.LIB.ts_batch_create(descs, 2, 0, ctypes.byref(h)) == T.TS_ERR_UNSUPPORTED
    assert h.value is None
    assert b"AB2" in T.LIB.ts_last_error()
    descs = (T.GridDesc * 1)(_desc(T, radial=T.TS_RADIAL_UPWIND_FD))
    assert T.LIB.ts_batch_create(descs, 1, 0, ctypes.byref(h)) == T.TS_ERR_UNSUPPORTED
    d = _desc(T, radial=T.TS_RADIAL_UPWIND_FD)
    assert T.LIB.ts_moments_noalloc(ctypes.byref(d), ctypes.c_void_p(0x10000), None, None, None,
                                    None, None, None) == T.TS_ERR_UNSUPPORTED
    # the conservative form: no batches, no allocation-free moments
    descs = (T.GridDesc * 1)(_desc(T, form=T.TS_FORM_CONSERVATIVE))
    assert T.LIB.ts_batch_create(descs, 1, 0, ctypes.byref(h)) == T.TS_ERR_UNSUPPORTED
    d = _desc(T, form=T.TS_FORM_CONSERVATIVE)
    assert T.LIB.ts_moments_noalloc(ctypes.byref(d), ctypes.c_void_p(0x10000), None, None, None,
                                    None, None, None) == T.TS_ERR_UNSUPPORTED
