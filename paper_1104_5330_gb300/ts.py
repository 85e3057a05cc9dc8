"""Thin Python binding of the C ABI in include/ts.h.

Every function here only marshals arguments (tensor data pointers, the
current CUDA stream) into the same-named C entry point of libts.so; all
arithmetic of the step runs in the library's CUDA kernels. There is no CPU
fallback: if libts.so cannot be loaded the import of this module raises.

Tensors are torch tensors on the CUDA device, contiguous, with the element
type of the grid (float64 for TS_FP64, float32 for TS_FP32); coefficient
fields, gradients and moments are float64. Layouts follow include/ts.h:
F[g][r][theta][phi][Theta][Phi], coefficients [g][r][theta][phi].
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libts.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ts.h")

TS_OK, TS_ERR_ARG, TS_ERR_UNSUPPORTED, TS_ERR_OOM, TS_ERR_CUDA, TS_ERR_TIMEOUT, TS_ERR_STATE = range(7)
TS_FP64, TS_FP32, TS_FP32_R64, TS_TF32X3, TS_BF16X3 = 0, 1, 2, 3, 4
TS_RK4, TS_RK4_SPLIT_IMPLICIT, TS_AB2 = 0, 1, 2
TS_BC_TAU_INFLOW, TS_BC_NONE = 0, 1
TS_RADIAL_CHEBYSHEV, TS_RADIAL_UPWIND_FD, TS_RADIAL_ZONED = 0, 1, 2
TS_FORM_ADVECTIVE, TS_FORM_CONSERVATIVE = 0, 1

STATUS_NAMES = ["TS_OK", "TS_ERR_ARG", "TS_ERR_UNSUPPORTED", "TS_ERR_OOM", "TS_ERR_CUDA",
                "TS_ERR_TIMEOUT", "TS_ERR_STATE"]


class TSError(RuntimeError):
    def __init__(self, status, where, text):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {text}")


class GridDesc(ctypes.Structure):
    _fields_ = [("R1", ctypes.c_double), ("R2", ctypes.c_double),
                ("Nr", ctypes.c_int), ("Ntheta", ctypes.c_int), ("Nphi", ctypes.c_int),
                ("NTheta", ctypes.c_int), ("NPhi", ctypes.c_int), ("groups", ctypes.c_int),
                ("precision", ctypes.c_int), ("scheme", ctypes.c_int), ("bc", ctypes.c_int),
                ("filter_on", ctypes.c_int), ("filter_alpha", ctypes.c_double),
                ("filter_order", ctypes.c_int), ("radial", ctypes.c_int),
                ("zone_nodes", ctypes.c_int), ("zone_width", ctypes.c_double),
                ("form", ctypes.c_int)]


class Cons2DDesc(ctypes.Structure):
    _fields_ = [("R1", ctypes.c_double), ("R2", ctypes.c_double), ("Nr", ctypes.c_int),
                ("NTheta", ctypes.c_int), ("problems", ctypes.c_int),
                ("scatter_c", ctypes.c_double), ("bc", ctypes.c_int),
                ("radial", ctypes.c_int), ("zone_nodes", ctypes.c_int),
                ("zone_width", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libts.so not built ({LIB_PATH}); run "
                          "python -m paper_1104_5330_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    sig = {
        "ts_create_grid": [ctypes.POINTER(GridDesc), ctypes.POINTER(P)],
        "ts_destroy_grid": [P],
        "ts_grid_nodes": [P, P, P, P, P, P],
        "ts_set_coeffs": [P, P, P, P, P, P, P],
        "ts_set_scattering_anisotropy": [P, P, P],
        "ts_set_scattering_quadrupole": [P, P, P],
        "ts_reset_history": [P],
        "ts_apply_inflow": [P, P, P],
        "ts_step": [P, P, D, I, P],
        "ts_step_host": [P, P, D, I, P],
        "ts_step_profile": [P, P, D, I, P, P, P],
        "ts_rhs": [P, P, P, P],
        "ts_liouville": [P, P, P, P],
        "ts_adjoint_step": [P, P, P, P, P, D, P],
        "ts_adjoint_step_ab2": [P, P, P, P, P, P, D, I, P],
        "ts_set_history": [P, P, P, P],
        "ts_flux_weights": [P, P, P],
        "ts_outgoing_flux": [P, P, P, P],
        "ts_outgoing_flux_adjoint": [P, P, P, P],
        "ts_moments": [P, P, P, P, P, P, P, P],
        "ts_number_balance": [P, P, P, P],
        "ts_moments_noalloc": [ctypes.POINTER(GridDesc), P, P, P, P, P, P, P],
        "ts_autotune": [P, P],
        "ts_tile_shape": [P, P, P, P],
        "ts_batch_create": [ctypes.POINTER(GridDesc), I, I, ctypes.POINTER(P)],
        "ts_batch_destroy": [P],
        "ts_batch_grid": [P, I, ctypes.POINTER(P)],
        "ts_batch_step": [P, P, P, I, P],
        "ts_sync_status": [P, P],
        "ts_set_wait_limit": [P, ctypes.c_longlong],
        "ts_stable_dt": [P, P, I, ctypes.POINTER(D), ctypes.POINTER(D), P],
        "ts_probe_fma_rate": [I, ctypes.POINTER(D), P],
        "ts_probe_widen": [P, P, ctypes.c_size_t, P],
        "ts_cons2d_create": [ctypes.POINTER(Cons2DDesc), ctypes.POINTER(P)],
        "ts_cons2d_destroy": [P],
        "ts_cons2d_nodes": [P, P, P],
        "ts_cons2d_set_coeffs": [P, P, P, P, P],
        "ts_cons2d_apply_inflow": [P, P, P],
        "ts_cons2d_rhs": [P, P, P, P],
        "ts_cons2d_step": [P, P, D, I, P],
        "ts_cons2d_balance": [P, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ts_last_error.restype = ctypes.c_char_p
    lib.ts_last_error.argtypes = []
    lib.ts_version.restype = ctypes.c_char_p
    lib.ts_version.argtypes = []
    lib.ts_field_elems.restype = S
    lib.ts_field_elems.argtypes = [P]
    return lib


LIB = _load()


def declared_functions(header: str = HEADER):
    """Names of the functions include/ts.h declares."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z_0-9]+)\s*\(", txt)))


def _check(status, where):
    if status != TS_OK:
        raise TSError(status, where, LIB.ts_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ts_version() -> str:
    return LIB.ts_version().decode()


def ts_probe_widen(x, out=None, stream=None):
    """float32 device tensor -> float64 by the library's integer-unit widening."""
    out = torch.empty(x.shape, dtype=torch.float64, device=x.device) if out is None else out
    _check(LIB.ts_probe_widen(_ptr(x), _ptr(out), x.numel(), _stream(stream)), "ts_probe_widen")
    return out


def ts_probe_fma_rate(precision: int, stream=None) -> float:
    """Measured FMA rate (TFLOP/s) of the current device for TS_FP64 or TS_FP32."""
    out = ctypes.c_double()
    _check(LIB.ts_probe_fma_rate(precision, ctypes.byref(out), _stream(stream)), "ts_probe_fma_rate")
    return out.value


def ts_create_grid(desc: GridDesc):
    h = ctypes.c_void_p()
    _check(LIB.ts_create_grid(ctypes.byref(desc), ctypes.byref(h)), "ts_create_grid")
    return h


def ts_destroy_grid(grid):
    _check(LIB.ts_destroy_grid(grid), "ts_destroy_grid")


def ts_field_elems(grid) -> int:
    return int(LIB.ts_field_elems(grid))


def ts_grid_nodes(grid, desc: GridDesc):
    import numpy as np
    out = [np.zeros(n) for n in (desc.Nr, desc.Ntheta, desc.Nphi, desc.NTheta, desc.NPhi)]
    _check(LIB.ts_grid_nodes(grid, *[o.ctypes.data_as(ctypes.c_void_p) for o in out]),
           "ts_grid_nodes")
    return out


def ts_set_coeffs(grid, kappa, eta, kappa_s, inflow_R1=None, inflow_R2=None, stream=None):
    _check(LIB.ts_set_coeffs(grid, _ptr(kappa), _ptr(eta), _ptr(kappa_s), _ptr(inflow_R1),
                             _ptr(inflow_R2), _stream(stream)), "ts_set_coeffs")


def nucleon_scattering(A_n, A_p):
    """Single kernel (kappa_s/4pi)(1 + b omega.omega') of neutrino scattering on
    neutrons and protons, sigma = A_n (1 - omega.omega'/3) + A_p (1 - omega.omega'/10)
    (Eqs. cross, crossnun, crossnup): kappa_s = 4 pi (A_n + A_p) and
    b = -(A_n/3 + A_p/10)/(A_n + A_p). Host arithmetic on numpy arrays."""
    A_n = np.asarray(A_n, dtype=np.float64)
    A_p = np.asarray(A_p, dtype=np.float64)
    return 4.0 * np.pi * (A_n + A_p), -(A_n / 3.0 + A_p / 10.0) / (A_n + A_p)


def ts_set_scattering_anisotropy(grid, b, stream=None):
    _check(LIB.ts_set_scattering_anisotropy(grid, _ptr(b), _stream(stream)),
           "ts_set_scattering_anisotropy")


def ts_set_scattering_quadrupole(grid, c, stream=None):
    _check(LIB.ts_set_scattering_quadrupole(grid, _ptr(c), _stream(stream)),
           "ts_set_scattering_quadrupole")


def ts_reset_history(grid):
    _check(LIB.ts_reset_history(grid), "ts_reset_history")


def ts_apply_inflow(grid, F, stream=None):
    _check(LIB.ts_apply_inflow(grid, _ptr(F), _stream(stream)), "ts_apply_inflow")


def ts_step(grid, F, dt, nsteps=1, stream=None):
    _check(LIB.ts_step(grid, _ptr(F), float(dt), int(nsteps), _stream(stream)), "ts_step")


def ts_step_profile(grid, F, dt, nsteps=1, stream=None):
    """Returns (pass_ms[4], launches[4]) summed over the steps: angular-block,
    plane, radial passes and other kernels."""
    import numpy as np
    ms = np.zeros(4)
    n = np.zeros(4, dtype=np.int32)
    _check(LIB.ts_step_profile(grid, _ptr(F), float(dt), int(nsteps),
                               ms.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                               _stream(stream)), "ts_step_profile")
    return ms, n


def ts_step_host(grid, F_host, dt, nsteps=1, stream=None):
    """F_host: a CPU tensor (pinned for full bandwidth), updated in place."""
    if F_host.is_cuda:
        raise ValueError("ts_step_host takes a host tensor")
    _check(LIB.ts_step_host(grid, _ptr(F_host), float(dt), int(nsteps), _stream(stream)),
           "ts_step_host")


def ts_rhs(grid, F, K, stream=None):
    _check(LIB.ts_rhs(grid, _ptr(F), _ptr(K), _stream(stream)), "ts_rhs")


def ts_liouville(grid, F, LF, stream=None):
    _check(LIB.ts_liouville(grid, _ptr(F), _ptr(LF), _stream(stream)), "ts_liouville")


def ts_adjoint_step(grid, F_n, lam, grad_kappa, grad_eta, dt, stream=None):
    _check(LIB.ts_adjoint_step(grid, _ptr(F_n), _ptr(lam), _ptr(grad_kappa), _ptr(grad_eta),
                               float(dt), _stream(stream)), "ts_adjoint_step")


def ts_adjoint_step_ab2(grid, F_n, lam, lam_prev, grad_kappa, grad_eta, dt, first, stream=None):
    _check(LIB.ts_adjoint_step_ab2(grid, _ptr(F_n), _ptr(lam), _ptr(lam_prev), _ptr(grad_kappa),
                                   _ptr(grad_eta), float(dt), int(bool(first)), _stream(stream)),
           "ts_adjoint_step_ab2")


def ts_set_history(grid, F, K_prev, stream=None):
    _check(LIB.ts_set_history(grid, _ptr(F), _ptr(K_prev), _stream(stream)), "ts_set_history")


def ts_flux_weights(grid, w, stream=None):
    _check(LIB.ts_flux_weights(grid, _ptr(w), _stream(stream)), "ts_flux_weights")


def ts_outgoing_flux(grid, F, J_R2, stream=None):
    _check(LIB.ts_outgoing_flux(grid, _ptr(F), _ptr(J_R2), _stream(stream)), "ts_outgoing_flux")


def ts_outgoing_flux_adjoint(grid, gJ, lam, stream=None):
    _check(LIB.ts_outgoing_flux_adjoint(grid, _ptr(gJ), _ptr(lam), _stream(stream)),
           "ts_outgoing_flux_adjoint")


def ts_moments(grid, F, F0=None, F1=None, N=None, J_R1=None, J_R2=None, stream=None):
    _check(LIB.ts_moments(grid, _ptr(F), _ptr(F0), _ptr(F1), _ptr(N), _ptr(J_R1), _ptr(J_R2),
                          _stream(stream)), "ts_moments")


def ts_number_balance(grid, F, out, stream=None):
    """out: a host float64 numpy array of 5 G values (N, J_R1, J_R2, dN/dt, S)."""
    _check(LIB.ts_number_balance(grid, _ptr(F), out.ctypes.data_as(ctypes.c_void_p),
                                 _stream(stream)), "ts_number_balance")


def ts_moments_noalloc(desc: GridDesc, F, F0=None, F1=None, N=None, J_R1=None, J_R2=None,
                       stream=None):
    """ts_moments without a grid and without device allocation (static scratch)."""
    _check(LIB.ts_moments_noalloc(ctypes.byref(desc), _ptr(F), _ptr(F0), _ptr(F1), _ptr(N),
                                  _ptr(J_R1), _ptr(J_R2), _stream(stream)), "ts_moments_noalloc")


def ts_autotune(grid, stream=None):
    _check(LIB.ts_autotune(grid, _stream(stream)), "ts_autotune")


def ts_tile_shape(grid):
    v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
    _check(LIB.ts_tile_shape(grid, *[ctypes.byref(x) for x in v]), "ts_tile_shape")
    return tuple(x.value for x in v)


def ts_batch_create(descs, autotune=True):
    arr = (GridDesc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(LIB.ts_batch_create(arr, len(descs), int(bool(autotune)), ctypes.byref(h)),
           "ts_batch_create")
    return h


def ts_batch_destroy(batch):
    _check(LIB.ts_batch_destroy(batch), "ts_batch_destroy")


def ts_batch_grid(batch, problem):
    h = ctypes.c_void_p()
    _check(LIB.ts_batch_grid(batch, int(problem), ctypes.byref(h)), "ts_batch_grid")
    return h


def ts_batch_step(batch, fields, dts, nsteps=1, stream=None):
    n = len(fields)
    ptrs = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fields])
    dt = (ctypes.c_double * n)(*[float(x) for x in dts])
    _check(LIB.ts_batch_step(batch, ptrs, dt, int(nsteps), _stream(stream)), "ts_batch_step")


def ts_stable_dt(grid, x0, iters=60, stream=None):
    """(rho, dt_max): power-iteration spectral radius of the stage operator's
    linear part from the start field x0, and the RK4 step 2.6 / rho."""
    rho, dtm = ctypes.c_double(), ctypes.c_double()
    _check(LIB.ts_stable_dt(grid, _ptr(x0), int(iters), ctypes.byref(rho), ctypes.byref(dtm),
                            _stream(stream)), "ts_stable_dt")
    return rho.value, dtm.value


def ts_set_wait_limit(grid, operand_wait_iterations):
    _check(LIB.ts_set_wait_limit(grid, int(operand_wait_iterations)), "ts_set_wait_limit")


def ts_sync_status(grid, stream=None):
    _check(LIB.ts_sync_status(grid, _stream(stream)), "ts_sync_status")


class Grid:
    """Owning handle around ts_create_grid/ts_destroy_grid with tensor helpers."""

    def __init__(self, R1=0.2, R2=1.0, Nr=17, Ntheta=8, Nphi=8, NTheta=8, NPhi=8, groups=1,
                 precision=TS_FP64, scheme=TS_RK4, bc=TS_BC_TAU_INFLOW, filter_on=False,
                 filter_alpha=36.0, filter_order=16, device=None, radial=TS_RADIAL_CHEBYSHEV,
                 zone_nodes=0, zone_width=0.0, form=TS_FORM_ADVECTIVE):
        self.desc = GridDesc(R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups, precision, scheme,
                             bc, int(filter_on), filter_alpha, filter_order, radial, zone_nodes,
                             zone_width, form)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.handle = ts_create_grid(self.desc)
        self._owns = True
        self._shapes()

    def _shapes(self):
        d = self.desc
        self.shape = (d.groups, d.Nr, d.Ntheta, d.Nphi, d.NTheta, d.NPhi)
        self.coef_shape = (d.groups, d.Nr, d.Ntheta, d.Nphi)
        self.inflow_shape = (d.groups, d.Ntheta, d.Nphi, d.NTheta // 2, d.NPhi)
        self.dtype = torch.float64 if d.precision == TS_FP64 else torch.float32

    @classmethod
    def borrowed(cls, handle, desc, device=None):
        """A view of a grid owned elsewhere (a batch's problem); never destroyed here."""
        g = cls.__new__(cls)
        g.desc = desc
        g.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        g.handle = handle
        g._owns = False
        g._shapes()
        return g

    def autotune(self):
        ts_autotune(self.handle)
        return ts_tile_shape(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            if getattr(self, "_owns", True):
                ts_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def points(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def nodes(self):
        return ts_grid_nodes(self.handle, self.desc)

    def empty(self):
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    def set_coeffs(self, kappa=None, eta=None, kappa_s=None, inflow_R1=None, inflow_R2=None):
        cv = lambda a, dt: None if a is None else torch.as_tensor(a, dtype=dt, device=self.device).contiguous()
        self._coeffs = [cv(kappa, torch.float64), cv(eta, torch.float64), cv(kappa_s, torch.float64),
                        cv(inflow_R1, self.dtype), cv(inflow_R2, self.dtype)]
        ts_set_coeffs(self.handle, *self._coeffs)

    def set_scattering_anisotropy(self, b=None):
        """b: [G][Nr][Ntheta][Nphi] anisotropy of the kernel (kappa_s/4pi)(1 + b omega.omega'),
        a scalar (broadcast) or None (isotropic)."""
        if b is None:
            self._scb = None
        else:
            self._scb = torch.broadcast_to(torch.as_tensor(b, dtype=torch.float64, device=self.device),
                                           self.coef_shape).contiguous()
        ts_set_scattering_anisotropy(self.handle, self._scb)

    def set_scattering_quadrupole(self, c=None):
        """c: [G][Nr][Ntheta][Nphi] coefficient of mu^2 - 1/3 in the kernel
        (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)), a scalar (broadcast) or None
        (no such term); Thomson scattering is c = 3/4 with b = 0."""
        if c is None:
            self._scc = None
        else:
            self._scc = torch.broadcast_to(torch.as_tensor(c, dtype=torch.float64, device=self.device),
                                           self.coef_shape).contiguous()
        ts_set_scattering_quadrupole(self.handle, self._scc)

    def apply_inflow(self, F):
        ts_apply_inflow(self.handle, F)
        return F

    def reset_history(self):
        """TS_AB2: the next step is a forward-Euler starting step."""
        ts_reset_history(self.handle)

    def step(self, F, dt, nsteps=1):
        ts_step(self.handle, F, dt, nsteps)
        return F

    def rhs(self, F, K=None):
        K = torch.empty_like(F) if K is None else K
        ts_rhs(self.handle, F, K)
        return K

    def liouville(self, F, LF=None):
        LF = torch.empty_like(F) if LF is None else LF
        ts_liouville(self.handle, F, LF)
        return LF

    def adjoint_step(self, F_n, lam, grad_kappa, grad_eta, dt):
        ts_adjoint_step(self.handle, F_n, lam, grad_kappa, grad_eta, dt)
        return lam

    def flux_weights(self):
        w = torch.empty(self.shape[2:], dtype=torch.float64, device=self.device)
        ts_flux_weights(self.handle, w)
        return w

    def outgoing_flux(self, F):
        """J_R2 per group (Eq. Flux), float64 [G]."""
        J = torch.empty(self.shape[0], dtype=torch.float64, device=self.device)
        ts_outgoing_flux(self.handle, F, J)
        return J

    def moments(self, F):
        G = self.shape[0]
        F0 = torch.empty(self.coef_shape, dtype=torch.float64, device=self.device)
        F1 = torch.empty((3,) + self.coef_shape, dtype=torch.float64, device=self.device)
        N = torch.empty(G, dtype=torch.float64, device=self.device)
        J1 = torch.empty(G, dtype=torch.float64, device=self.device)
        J2 = torch.empty(G, dtype=torch.float64, device=self.device)
        ts_moments(self.handle, F, F0, F1, N, J1, J2)
        return F0, F1, N, J1, J2

    def number_balance(self, F):
        """[G][5] float64 numpy: N, J_R1, J_R2, dN/dt (operator without Tau rows)
        and the absorption/emission integral S per group (ts_number_balance)."""
        out = np.zeros((self.shape[0], 5), dtype=np.float64)
        ts_number_balance(self.handle, F, out)
        return out


class Batch:
    """Owning handle around ts_batch_create/ts_batch_destroy; `grids[q]` are
    borrowed views of the per-problem grids (set_coeffs, nodes, moments...)."""

    def __init__(self, descs, autotune=True):
        self.descs = list(descs)
        self.handle = ts_batch_create(self.descs, autotune)
        self.grids = [Grid.borrowed(ts_batch_grid(self.handle, q), d)
                      for q, d in enumerate(self.descs)]

    def step(self, fields, dts, nsteps=1):
        ts_batch_step(self.handle, fields, dts, nsteps)
        return fields

    @property
    def points(self):
        return sum(g.points for g in self.grids)

    def close(self):
        if getattr(self, "handle", None) is not None:
            for g in self.grids:
                g.handle = None
            ts_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cons2D:
    """Owning handle of the conservative 2-D (r, Theta) variant (ts_cons2d_*):
    Fhat[P][Nr][NTheta] float64 tensors on the device."""

    def __init__(self, R1, R2, Nr, NTheta, problems=1, scatter_c=0.75, bc=TS_BC_TAU_INFLOW,
                 radial=TS_RADIAL_CHEBYSHEV, zone_nodes=0, zone_width=0.0):
        self.desc = Cons2DDesc(R1, R2, Nr, NTheta, problems, scatter_c, bc, radial, zone_nodes,
                               zone_width)
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _check(LIB.ts_cons2d_create(ctypes.byref(self.desc), ctypes.byref(h)), "ts_cons2d_create")
        self.handle = h
        self.shape = (problems, Nr, NTheta)

    def close(self):
        if getattr(self, "handle", None) is not None:
            _check(LIB.ts_cons2d_destroy(self.handle), "ts_cons2d_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nodes(self):
        r, th = np.zeros(self.desc.Nr), np.zeros(self.desc.NTheta)
        _check(LIB.ts_cons2d_nodes(self.handle, r.ctypes.data_as(ctypes.c_void_p),
                                   th.ctypes.data_as(ctypes.c_void_p)), "ts_cons2d_nodes")
        return r, th

    def set_coeffs(self, kappa_s=None, inflow_R1=None, inflow_R2=None):
        cv = lambda a: None if a is None else torch.as_tensor(
            a, dtype=torch.float64, device=self.device).contiguous()
        self._c = [cv(kappa_s), cv(inflow_R1), cv(inflow_R2)]
        _check(LIB.ts_cons2d_set_coeffs(self.handle, *[_ptr(x) for x in self._c],
                                        _stream(None)), "ts_cons2d_set_coeffs")

    def apply_inflow(self, Fh):
        _check(LIB.ts_cons2d_apply_inflow(self.handle, _ptr(Fh), _stream(None)),
               "ts_cons2d_apply_inflow")
        return Fh

    def rhs(self, Fh):
        K = torch.empty_like(Fh)
        _check(LIB.ts_cons2d_rhs(self.handle, _ptr(Fh), _ptr(K), _stream(None)), "ts_cons2d_rhs")
        return K

    def step(self, Fh, dt, nsteps=1):
        _check(LIB.ts_cons2d_step(self.handle, _ptr(Fh), float(dt), int(nsteps), _stream(None)),
               "ts_cons2d_step")
        return Fh

    def balance(self, Fh):
        """(N, J_R1, J_R2) [P][3] and the residual dN/dt + J_R2 - J_R1 [P]."""
        P = self.shape[0]
        NJ = torch.empty((P, 3), dtype=torch.float64, device=self.device)
        res = torch.empty(P, dtype=torch.float64, device=self.device)
        _check(LIB.ts_cons2d_balance(self.handle, _ptr(Fh), _ptr(NJ), _ptr(res), _stream(None)),
               "ts_cons2d_balance")
        return NJ, res
