"""Python binding of the GB300 boundary-integral library (libbie.so).

The functions below carry the names of the C ABI in include/bie.h and only
marshal arguments: tensors become device/host pointers, options become the C
structs.  Every step of the solve runs in the CUDA library; there is no
Python or CPU fallback, and importing the binding without a built library
raises at first use.

Typical use (torch only provides device memory and the stream):

    ctx = bie_create(0, torch.cuda.current_stream())
    bie_set_geometry(ctx, M, zeta, dzeta, d2zeta, zc)     # complex128 CUDA tensors
    bie_set_flow(ctx, V1, a)
    bie_assemble(ctx, BIE_FP32_IR)
    info = bie_solve(ctx, phit, omega, U, psi)
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbie.so")

# status codes (include/bie.h)
BIE_OK = 0
BIE_ERR_ARG = 1
BIE_ERR_GEOM = 2
BIE_ERR_OOM = 3
BIE_ERR_CUDA = 4
BIE_ERR_NOCONV = 5
BIE_ERR_NAN = 6
BIE_ERR_TIMEOUT = 7
BIE_ERR_STATE = 8
STATUS_NAMES = {0: "BIE_OK", 1: "BIE_ERR_ARG", 2: "BIE_ERR_GEOM", 3: "BIE_ERR_OOM",
                4: "BIE_ERR_CUDA", 5: "BIE_ERR_NOCONV", 6: "BIE_ERR_NAN",
                7: "BIE_ERR_TIMEOUT", 8: "BIE_ERR_STATE"}

# storage precisions
BIE_FP64 = 0
BIE_FP32_IR = 1
BIE_BF16_IR = 2
BIE_FP16_IR = 3
PRECISIONS = {"fp64": BIE_FP64, "fp32_ir": BIE_FP32_IR, "bf16_ir": BIE_BF16_IR,
              "fp16_ir": BIE_FP16_IR}


class BieError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bie_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("row_flip", ctypes.c_int), ("x0", ctypes.c_int)]


class bie_profile(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("n_gemv_inner", ctypes.c_int),
                ("ms_gemv_inner", ctypes.c_double), ("bytes_gemv_inner", ctypes.c_double),
                ("n_gemv_full", ctypes.c_int), ("ms_gemv_full", ctypes.c_double),
                ("bytes_gemv_full", ctypes.c_double), ("n_assemble", ctypes.c_int),
                ("ms_assemble", ctypes.c_double), ("n_velocity", ctypes.c_int),
                ("ms_velocity", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("n_gemv_hi", ctypes.c_int), ("ms_gemv_hi", ctypes.c_double),
                ("bytes_gemv_hi", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bie_evolve_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("solves", ctypes.c_int),
                ("gmres_iters", ctypes.c_longlong), ("max_rel_resid", ctypes.c_double)]

    def as_dict(self):
        return {"steps": self.steps, "solves": self.solves, "gmres_iters": self.gmres_iters,
                "max_rel_resid": self.max_rel_resid}


class bie_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_resid", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "cycles": self.cycles,
                "converged": bool(self.converged), "rel_resid": self.rel_resid}


class bie_grads(ctypes.Structure):
    _fields_ = [("g_zeta", ctypes.c_void_p), ("g_dzeta", ctypes.c_void_p),
                ("g_d2zeta", ctypes.c_void_p), ("g_zc", ctypes.c_void_p),
                ("g_phit", ctypes.c_void_p), ("g_node", ctypes.c_void_p),
                ("g_shape", ctypes.c_void_p), ("lambda_", ctypes.c_void_p)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_l = ctypes.c_long

# int exchange(void* user, int op, long long count, int elem_bytes, void* stream)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
                               ctypes.c_int, ctypes.c_void_p)
BIE_EXCH_ALLGATHER = 0
BIE_EXCH_ALLREDUCE_SUM = 1

# C signatures: name -> (restype, argtypes)
SIGNATURES = {
    "bie_default_opts": (None, [ctypes.POINTER(bie_solve_opts)]),
    "bie_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "bie_destroy": (None, [_vp]),
    "bie_last_error": (ctypes.c_char_p, [_vp]),
    "bie_set_geometry": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "bie_set_flow": (_i, [_vp, _d, _vp]),
    "bie_assemble": (_i, [_vp, _i]),
    "bie_rhs": (_i, [_vp, _vp, _vp]),
    "bie_matvec": (_i, [_vp, _i, _vp, _vp]),
    "bie_matmat": (_i, [_vp, _i, _vp, _vp]),
    "bie_matmat_full": (_i, [_vp, _i, _vp, _vp]),
    "bie_solve_multi": (_i, [_vp, _i, _i, _vp, _vp, _vp, ctypes.POINTER(bie_solve_opts),
                             ctypes.POINTER(bie_solve_info)]),
    "bie_pressure_rhs": (_i, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp]),
    "bie_boundary_potential": (_i, [_vp, _vp, _vp]),
    "bie_eval_potential": (_i, [_vp, _vp, ctypes.c_longlong, _vp, _vp]),
    "bie_solve_b": (_i, [_vp, _vp, _vp, ctypes.POINTER(bie_solve_opts),
                         ctypes.POINTER(bie_solve_info)]),
    "bie_graph_rhs": (_i, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i,
                           ctypes.POINTER(bie_solve_opts), _vp, _vp, _vp, _vp]),
    "bie_graph_evolve": (_i, [_vp, _vp, _vp, ctypes.c_double, _i, ctypes.c_double,
                              ctypes.c_double, _i, _i, ctypes.POINTER(bie_solve_opts), _vp,
                              ctypes.POINTER(bie_evolve_info)]),
    "bie_hls_rhs": (_i, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i,
                         ctypes.POINTER(bie_solve_opts), _vp, _vp, _vp, _vp]),
    "bie_hls_evolve": (_i, [_vp, _vp, _vp, ctypes.c_double, _i, ctypes.c_double,
                            ctypes.c_double, _i, _i, ctypes.POINTER(bie_solve_opts), _vp,
                            ctypes.POINTER(bie_evolve_info)]),
    "bie_hls_curve": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "bie_vs_graph_rhs": (_i, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i,
                              ctypes.POINTER(bie_solve_opts), _vp, _vp, _vp]),
    "bie_evolve": (_i, [_vp, _i, _i, _vp, _vp, ctypes.c_double, _i, ctypes.c_double,
                        ctypes.c_double, _i, _i, ctypes.POINTER(bie_solve_opts), _vp,
                        ctypes.POINTER(bie_evolve_info)]),
    "bie_energy": (_i, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                        ctypes.POINTER(ctypes.c_double)]),
    "bie_filter": (_i, [_vp, _vp]),
    "bie_assemble_psi": (_i, [_vp, _i]),
    "bie_min_separation": (_i, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "bie_set_min_separation": (_i, [_vp, ctypes.c_double]),
    "bie_solve_psi": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(bie_solve_opts),
                           ctypes.POINTER(bie_solve_info)]),
    "bie_sample_entries": (_i, [_vp, _i, _l, _vp, _vp, _vp]),
    "bie_normal_velocity": (_i, [_vp, _vp, _vp, _vp]),
    "bie_solve": (_i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(bie_solve_opts),
                       ctypes.POINTER(bie_solve_info)]),
    "bie_solve_host": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _i,
                            ctypes.POINTER(bie_solve_opts), _vp, _vp, _vp,
                            ctypes.POINTER(bie_solve_info)]),
    "bie_boundary_velocity": (_i, [_vp, _vp, _vp]),
    "bie_eval_velocity": (_i, [_vp, _vp, ctypes.c_longlong, _vp, _vp, _i, _d,
                               ctypes.POINTER(ctypes.c_longlong)]),
    "bie_normal_velocity_static": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp,
                                        _vp]),
    "bie_vs_normal_velocity": (_i, [_vp, _vp, _vp, _vp, _i, ctypes.POINTER(bie_solve_opts),
                                    ctypes.POINTER(bie_solve_info)]),
    "bie_backward": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(bie_grads),
                          ctypes.POINTER(bie_solve_opts), ctypes.POINTER(bie_solve_info)]),
    "bie_batch_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "bie_batch_destroy": (None, [_vp]),
    "bie_batch_last_error": (ctypes.c_char_p, [_vp]),
    "bie_batch_set_problem": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "bie_batch_run": (_i, [_vp, _i, _vp, _vp, _vp, _i, ctypes.POINTER(bie_solve_opts), _vp]),
    "bie_batch_tuning": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), _vp]),
    "bie_batch_resid_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "bie_test_grid_barrier": (_i, [_i, ctypes.c_uint, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "bie_set_partition": (_i, [_vp, _i, _i, _vp, ctypes.c_size_t, EXCHANGE_FN, _vp]),
    "bie_partition_rows": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                ctypes.POINTER(ctypes.c_longlong)]),
    "bie_set_profiling": (_i, [_vp, _i]),
    "bie_get_profile": (_i, [_vp, ctypes.POINTER(bie_profile)]),
}


def lib():
    """Load libbie.so (built by __graft_entry__.build() / _build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected one of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, name="array"):
    """Host pointer of a contiguous CPU tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    try:
        import torch
        if isinstance(t, torch.Tensor):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor")
            return ctypes.c_void_p(t.data_ptr())
    except ImportError:  # pragma: no cover
        pass
    import numpy as np
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(f"{name} must be a CPU tensor or numpy array")


def _check(ctx, status):
    if status != BIE_OK:
        msg = lib().bie_last_error(ctx).decode() if ctx else ""
        raise BieError(status, msg)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


_C128 = None


def _c128():
    global _C128
    if _C128 is None:
        import torch
        _C128 = (torch.complex128,)
    return _C128


def _f64():
    import torch
    return (torch.float64,)


def _i64():
    import torch
    return (torch.int64,)


# ---------------------------------------------------------------------------
# the C ABI, same names
# ---------------------------------------------------------------------------

def bie_default_opts(**overrides):
    o = bie_solve_opts()
    lib().bie_default_opts(ctypes.byref(o))
    names = {f[0] for f in bie_solve_opts._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"bie_default_opts: unknown option {k!r}")
        setattr(o, k, v)
    return o


def bie_create(device=0, stream=None):
    ctx = ctypes.c_void_p()
    st = lib().bie_create(ctypes.byref(ctx), int(device), _stream_handle(stream))
    if st != BIE_OK:
        raise BieError(st, "bie_create failed")
    return ctx


def bie_destroy(ctx):
    if ctx:
        lib().bie_destroy(ctx)


def bie_last_error(ctx):
    return lib().bie_last_error(ctx).decode()


def bie_set_geometry(ctx, M, zeta, dzeta, d2zeta, zc=None):
    """M: sequence of node counts; zeta, dzeta, d2zeta: complex128 CUDA tensors of
    length sum(M); zc: obstacle centres (host complex array, len(M)-2)."""
    import numpy as np
    Mh = np.ascontiguousarray(np.asarray(M, dtype=np.int32))
    zch = None
    if zc is not None and len(zc) > 0:
        zch = np.ascontiguousarray(np.asarray(zc, dtype=np.complex128))
    st = lib().bie_set_geometry(ctx, len(Mh), _hptr(Mh), _dptr(zeta, _c128(), "zeta"),
                                _dptr(dzeta, _c128(), "dzeta"), _dptr(d2zeta, _c128(), "d2zeta"),
                                _hptr(zch) if zch is not None else None)
    _check(ctx, st)


def bie_set_flow(ctx, V1, a=None):
    import numpy as np
    ah = None
    if a is not None and len(a) > 0:
        ah = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    _check(ctx, lib().bie_set_flow(ctx, float(V1), _hptr(ah) if ah is not None else None))


def bie_assemble(ctx, precision):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    _check(ctx, lib().bie_assemble(ctx, int(precision)))


def bie_rhs(ctx, phit, b):
    _check(ctx, lib().bie_rhs(ctx, _dptr(phit, _f64(), "phit"), _dptr(b, _f64(), "b")))


def bie_matvec(ctx, which, x, y):
    _check(ctx, lib().bie_matvec(ctx, int(which), _dptr(x, _f64(), "x"), _dptr(y, _f64(), "y")))


def bie_matmat(ctx, X, Y):
    """Y[r] = A X[r] for the rows r of X (float64 CUDA, nrhs x N) on the tensor cores."""
    _check(ctx, lib().bie_matmat(ctx, int(X.shape[0]), _dptr(X, _f64(), "X"), _dptr(Y, _f64(), "Y")))


RHS_PHIT, RHS_B = 0, 1


def bie_solve_multi(ctx, rhs, omega, U=None, opts=None, raise_on_noconv=True, kind="phit"):
    """Solve for every row of rhs (float64 CUDA): phi~ rows (nrhs x M_0, kind
    "phit", b from eq. Awb) or b rows (nrhs x N, kind "b").  Writes omega
    (nrhs x N) and, if given, U (nrhs x M_0); returns the per-column
    bie_solve_info list."""
    nrhs = int(rhs.shape[0])
    k = {"phit": RHS_PHIT, "b": RHS_B}[kind]
    infos = (bie_solve_info * max(nrhs, 1))()
    o = opts if opts is not None else bie_default_opts()
    st = lib().bie_solve_multi(ctx, nrhs, k, _dptr(rhs, _f64(), "rhs"),
                               _dptr(omega, _f64(), "omega"), _dptr(U, _f64(), "U"),
                               ctypes.byref(o), infos)
    if not (st == BIE_ERR_NOCONV and not raise_on_noconv):
        _check(ctx, st)
    return list(infos)[:nrhs]


def bie_pressure_rhs(ctx, phit, U, b, tau=0.1, g=1.0):
    """b (N) = auxiliary Dirichlet data of Phi_t - C (eq. pressure:d:prob)."""
    _check(ctx, lib().bie_pressure_rhs(ctx, _dptr(phit, _f64(), "phit"), _dptr(U, _f64(), "U"),
                                       float(tau), float(g), _dptr(b, _f64(), "b")))


def bie_boundary_potential(ctx, omega, phi):
    """phi (complex128, N) = Phi~ of eq. w123 on every boundary node from the
    fluid side (Plemelj); for omega^aux its real part is Phi_t - C."""
    _check(ctx, lib().bie_boundary_potential(ctx, _dptr(omega, _f64(), "omega"),
                                             _dptr(phi, _c128(), "phi")))


def bie_eval_potential(ctx, omega, z, phi):
    """phi (complex128, n) = Phi~(z) at the targets z (complex128, n) of the
    fluid (Helsing-Ojala with the Plemelj boundary values)."""
    _check(ctx, lib().bie_eval_potential(ctx, _dptr(omega, _f64(), "omega"), int(z.numel()),
                                         _dptr(z, _c128(), "z"), _dptr(phi, _c128(), "phi")))


def bie_solve_b(ctx, b, omega, opts=None):
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    _check(ctx, lib().bie_solve_b(ctx, _dptr(b, _f64(), "b"), _dptr(omega, _f64(), "omega"),
                                  ctypes.byref(o), ctypes.byref(info)))
    return info


def _prec(precision):
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def bie_graph_rhs(ctx, eta, phit, eta_t, phit_t, tau=0.1, g=1.0, precision="fp32_ir",
                  opts=None, omega=None, U=None):
    """One evaluation of eqs. graph:eta:t and phitileq (float64 CUDA vectors)."""
    o = opts if opts is not None else bie_default_opts()
    _check(ctx, lib().bie_graph_rhs(ctx, _dptr(eta, _f64(), "eta"), _dptr(phit, _f64(), "phit"),
                                    float(tau), float(g), _prec(precision), ctypes.byref(o),
                                    _dptr(eta_t, _f64(), "eta_t"), _dptr(phit_t, _f64(), "phit_t"),
                                    _dptr(omega, _f64(), "omega"), _dptr(U, _f64(), "U")))


def bie_graph_evolve(ctx, eta, phit, dt, nsteps, tau=0.1, g=1.0, filter=False,
                     precision="fp32_ir", opts=None, energies=True):
    """RK4 steps on (eta, phi~) in place; returns (energies or None, bie_evolve_info)."""
    import numpy as np
    o = opts if opts is not None else bie_default_opts()
    info = bie_evolve_info()
    E = np.zeros(int(nsteps) + 1) if energies else None
    _check(ctx, lib().bie_graph_evolve(ctx, _dptr(eta, _f64(), "eta"), _dptr(phit, _f64(), "phit"),
                                       float(dt), int(nsteps), float(tau), float(g),
                                       1 if filter else 0, _prec(precision), ctypes.byref(o),
                                       E.ctypes.data_as(ctypes.c_void_p) if E is not None else None,
                                       ctypes.byref(info)))
    return E, info


def bie_hls_rhs(ctx, Ptheta, phit, Ptheta_t, phit_t, tau=0.1, g=1.0, precision="fp32_ir",
                opts=None, omega=None, U=None):
    o = opts if opts is not None else bie_default_opts()
    _check(ctx, lib().bie_hls_rhs(ctx, _dptr(Ptheta, _f64(), "Ptheta"), _dptr(phit, _f64(), "phit"),
                                  float(tau), float(g), _prec(precision), ctypes.byref(o),
                                  _dptr(Ptheta_t, _f64(), "Ptheta_t"), _dptr(phit_t, _f64(), "phit_t"),
                                  _dptr(omega, _f64(), "omega"), _dptr(U, _f64(), "U")))


def bie_hls_evolve(ctx, Ptheta, phit, dt, nsteps, tau=0.1, g=1.0, filter=False,
                   precision="fp32_ir", opts=None, energies=True):
    import numpy as np
    o = opts if opts is not None else bie_default_opts()
    info = bie_evolve_info()
    E = np.zeros(int(nsteps) + 1) if energies else None
    _check(ctx, lib().bie_hls_evolve(ctx, _dptr(Ptheta, _f64(), "Ptheta"), _dptr(phit, _f64(), "phit"),
                                     float(dt), int(nsteps), float(tau), float(g),
                                     1 if filter else 0, _prec(precision), ctypes.byref(o),
                                     E.ctypes.data_as(ctypes.c_void_p) if E is not None else None,
                                     ctypes.byref(info)))
    return E, info


FORMULATIONS = {"graph": 0, "hls": 1, "vs_graph": 2}
INTEGRATORS = {"rk4": 0, "gbs8": 1, "dp8": 2}


def bie_evolve(ctx, y1, phit, dt, nsteps, formulation="graph", integrator="rk4", tau=0.1, g=1.0,
               filter=False, precision="fp32_ir", opts=None, energies=True):
    """Evolve (eta or P theta, phi~) in place; returns (energies or None, bie_evolve_info)."""
    import numpy as np
    o = opts if opts is not None else bie_default_opts()
    info = bie_evolve_info()
    E = np.zeros(int(nsteps) + 1) if energies else None
    _check(ctx, lib().bie_evolve(ctx, FORMULATIONS[formulation], INTEGRATORS[integrator],
                                 _dptr(y1, _f64(), "y1"), _dptr(phit, _f64(), "phit"), float(dt),
                                 int(nsteps), float(tau), float(g), 1 if filter else 0,
                                 _prec(precision), ctypes.byref(o),
                                 E.ctypes.data_as(ctypes.c_void_p) if E is not None else None,
                                 ctypes.byref(info)))
    return E, info


def bie_vs_graph_rhs(ctx, eta, gamma0, eta_t, gamma0_t, tau=0.1, g=1.0, precision="fp32_ir",
                     opts=None, U=None):
    o = opts if opts is not None else bie_default_opts()
    _check(ctx, lib().bie_vs_graph_rhs(ctx, _dptr(eta, _f64(), "eta"), _dptr(gamma0, _f64(), "gamma0"),
                                       float(tau), float(g), _prec(precision), ctypes.byref(o),
                                       _dptr(eta_t, _f64(), "eta_t"),
                                       _dptr(gamma0_t, _f64(), "gamma0_t"), _dptr(U, _f64(), "U")))


def bie_hls_curve(ctx, Ptheta, zeta=None, dzeta=None, d2zeta=None):
    _check(ctx, lib().bie_hls_curve(ctx, _dptr(Ptheta, _f64(), "Ptheta"), _dptr(zeta, _c128(), "zeta"),
                                    _dptr(dzeta, _c128(), "dzeta"), _dptr(d2zeta, _c128(), "d2zeta")))


def bie_energy(ctx, phit, omega, tau=0.1, g=1.0):
    E = ctypes.c_double(0.0)
    _check(ctx, lib().bie_energy(ctx, _dptr(phit, _f64(), "phit"), _dptr(omega, _f64(), "omega"),
                                 float(tau), float(g), ctypes.byref(E)))
    return E.value


def bie_min_separation(ctx):
    """(closest approach of two boundaries in local node spacings, node index)."""
    r, n = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(ctx, lib().bie_min_separation(ctx, ctypes.byref(r), ctypes.byref(n)))
    return r.value, n.value


def bie_set_min_separation(ctx, ratio):
    _check(ctx, lib().bie_set_min_separation(ctx, float(ratio)))


def save_state(path, geom, flow, phit, omega=None, U=None, **extra):
    """Write geometry, flow, phi~ and (optionally) omega, U and other arrays to
    an .npz file, for reproducible runs."""
    import numpy as np
    arrs = {"M": np.asarray(geom.M), "zeta": geom.zeta, "dzeta": geom.dzeta,
            "d2zeta": geom.d2zeta, "zc": np.asarray(geom.zc, dtype=np.complex128),
            "V1": np.float64(flow.V1), "a": np.asarray(flow.a, dtype=np.float64),
            "phit": np.asarray(phit)}
    if omega is not None:
        arrs["omega"] = np.asarray(omega)
    if U is not None:
        arrs["U"] = np.asarray(U)
    for k, v in extra.items():
        arrs[k] = np.asarray(v)
    np.savez(path, **arrs)


def load_state(path):
    """The arrays written by save_state, as a dict of numpy arrays."""
    import numpy as np
    with np.load(path) as d:
        return {k: d[k] for k in d.files}


def bie_assemble_psi(ctx, precision):
    _check(ctx, lib().bie_assemble_psi(ctx, _prec(precision)))


def bie_solve_psi(ctx, phic, psi_solid, omega, U=None, opts=None, nobs=0):
    """App. B solve; returns (the first nobs circulations a_j, bie_solve_info)."""
    import numpy as np
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    a = np.zeros(32)
    _check(ctx, lib().bie_solve_psi(ctx, _dptr(phic, _f64(), "phic"), _dptr(psi_solid, _f64(), "psi"),
                                    _dptr(omega, _f64(), "omega"), _dptr(U, _f64(), "U"),
                                    a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                                    ctypes.byref(info)))
    return a[:int(nobs)], info


def bie_filter(ctx, x):
    _check(ctx, lib().bie_filter(ctx, _dptr(x, _f64(), "x")))


def bie_matmat_full(ctx, X, Y):
    """Y[r] = A X[r] with the full-accuracy operator on the tensor cores (exact slices)."""
    _check(ctx, lib().bie_matmat_full(ctx, int(X.shape[0]), _dptr(X, _f64(), "X"),
                                      _dptr(Y, _f64(), "Y")))


def bie_sample_entries(ctx, which, rows, cols, out):
    n = rows.numel()
    _check(ctx, lib().bie_sample_entries(ctx, int(which), n, _dptr(rows, _i64(), "rows"),
                                         _dptr(cols, _i64(), "cols"), _dptr(out, _f64(), "out")))


def bie_normal_velocity(ctx, omega, U, psi=None):
    _check(ctx, lib().bie_normal_velocity(ctx, _dptr(omega, _f64(), "omega"),
                                          _dptr(U, _f64(), "U"), _dptr(psi, _f64(), "psi")))


def bie_boundary_velocity(ctx, omega, f):
    """f: complex128 CUDA tensor of length N (u - i v at every node)."""
    _check(ctx, lib().bie_boundary_velocity(ctx, _dptr(omega, _f64(), "omega"),
                                            _dptr(f, _c128(), "f")))


VEL_FAR, VEL_HELSING, VEL_AUTO = 0, 1, 2


def bie_eval_velocity(ctx, omega, z, uv, mode=VEL_AUTO, near_spacings=4.0, count_near=False):
    """z, uv: complex128 CUDA tensors (targets, output u - i v)."""
    nn = ctypes.c_longlong(0)
    _check(ctx, lib().bie_eval_velocity(ctx, _dptr(omega, _f64(), "omega"), z.numel(),
                                        _dptr(z, _c128(), "z"), _dptr(uv, _c128(), "uv"),
                                        int(mode), float(near_spacings),
                                        ctypes.byref(nn) if count_near else None))
    return nn.value if count_near else None


def bie_solve(ctx, phit, omega, U, psi=None, opts=None, raise_on_noconv=True):
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    st = lib().bie_solve(ctx, _dptr(phit, _f64(), "phit"), _dptr(omega, _f64(), "omega"),
                         _dptr(U, _f64(), "U"), _dptr(psi, _f64(), "psi"), ctypes.byref(o),
                         ctypes.byref(info))
    if st == BIE_ERR_NOCONV and not raise_on_noconv:
        return info
    _check(ctx, st)
    return info


def bie_solve_host(ctx, M, zeta, dzeta, d2zeta, zc, V1, a, phit, precision, omega, U,
                   psi=None, opts=None):
    """End-to-end call on host buffers (numpy arrays or CPU tensors, pinned is fastest)."""
    import numpy as np
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    Mh = np.ascontiguousarray(np.asarray(M, dtype=np.int32))
    zch = np.ascontiguousarray(np.asarray(zc if zc is not None else [], dtype=np.complex128))
    ah = np.ascontiguousarray(np.asarray(a if a is not None else [], dtype=np.float64))
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    st = lib().bie_solve_host(ctx, len(Mh), _hptr(Mh), _hptr(zeta, "zeta"), _hptr(dzeta, "dzeta"),
                              _hptr(d2zeta, "d2zeta"), _hptr(zch) if len(zch) else None,
                              float(V1), _hptr(ah) if len(ah) else None, _hptr(phit, "phit"),
                              int(precision), ctypes.byref(o), _hptr(omega, "omega"),
                              _hptr(U, "U"), _hptr(psi, "psi") if psi is not None else None,
                              ctypes.byref(info))
    _check(ctx, st)
    return info


STATIC_MAXN = 8192


def bie_normal_velocity_static(M, zeta, dzeta, d2zeta, zc, V1, a, omega, U, psi=None,
                               stream=None):
    """Allocation-free normal velocity (no context); N = sum(M) <= STATIC_MAXN."""
    import numpy as np
    Mh = np.ascontiguousarray(np.asarray(M, dtype=np.int32))
    zch = np.ascontiguousarray(np.asarray(zc if zc is not None else [], dtype=np.complex128))
    ah = np.ascontiguousarray(np.asarray(a if a is not None else [], dtype=np.float64))
    st = lib().bie_normal_velocity_static(
        len(Mh), _hptr(Mh), _dptr(zeta, _c128(), "zeta"), _dptr(dzeta, _c128(), "dzeta"),
        _dptr(d2zeta, _c128(), "d2zeta"), _hptr(zch) if len(zch) else None, float(V1),
        _hptr(ah) if len(ah) else None, _dptr(omega, _f64(), "omega"), _dptr(U, _f64(), "U"),
        _dptr(psi, _f64(), "psi"), _stream_handle(stream))
    if st != BIE_OK:
        raise BieError(st, "bie_normal_velocity_static failed")


def bie_vs_normal_velocity(ctx, gamma0, U, gamma=None, precision="fp32_ir", opts=None):
    """Vortex-sheet route: gamma0 (float64 CUDA, M_0) -> U (float64 CUDA, M_0);
    gamma (float64 CUDA, N - M_0, optional) receives the solid strengths."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    _check(ctx, lib().bie_vs_normal_velocity(ctx, _dptr(gamma0, _f64(), "gamma0"),
                                             _dptr(U, _f64(), "U"), _dptr(gamma, _f64(), "gamma"),
                                             int(precision), ctypes.byref(o), ctypes.byref(info)))
    return info


def bie_backward(ctx, omega, gU, ellipses=None, *, g_zeta=None, g_dzeta=None, g_d2zeta=None,
                 g_zc=None, g_phit=None, g_node=None, g_shape=None, lam=None, opts=None,
                 raise_on_noconv=True):
    """Backward pass for J(U): gU = dJ/dU (float64 CUDA, M_0).  Outputs are
    optional CUDA tensors: complex128 for g_zeta, g_dzeta, g_d2zeta, g_zc,
    g_node; float64 for g_phit, g_shape (5 per obstacle), lam (N).
    ellipses: host array (nb-2, 5) of (x, y, q, b, theta), needed for g_shape."""
    import numpy as np
    eh = None
    if ellipses is not None and len(ellipses) > 0:
        eh = np.ascontiguousarray(np.asarray(ellipses, dtype=np.float64).reshape(-1))
    g = bie_grads()
    g.g_zeta = _dptr(g_zeta, _c128(), "g_zeta")
    g.g_dzeta = _dptr(g_dzeta, _c128(), "g_dzeta")
    g.g_d2zeta = _dptr(g_d2zeta, _c128(), "g_d2zeta")
    g.g_zc = _dptr(g_zc, _c128(), "g_zc")
    g.g_phit = _dptr(g_phit, _f64(), "g_phit")
    g.g_node = _dptr(g_node, _c128(), "g_node")
    g.g_shape = _dptr(g_shape, _f64(), "g_shape")
    g.lambda_ = _dptr(lam, _f64(), "lam")
    info = bie_solve_info()
    o = opts if opts is not None else bie_default_opts()
    st = lib().bie_backward(ctx, _dptr(omega, _f64(), "omega"), _dptr(gU, _f64(), "gU"),
                            _hptr(eh) if eh is not None else None, ctypes.byref(g),
                            ctypes.byref(o), ctypes.byref(info))
    if st == BIE_ERR_NOCONV and not raise_on_noconv:
        return info
    _check(ctx, st)
    return info


def bie_batch_create(device=0, stream=None):
    b = ctypes.c_void_p()
    st = lib().bie_batch_create(ctypes.byref(b), int(device), _stream_handle(stream))
    if st != BIE_OK:
        raise BieError(st, "bie_batch_create failed")
    return b


def bie_batch_destroy(b):
    if b:
        lib().bie_batch_destroy(b)


def bie_batch_last_error(b):
    return lib().bie_batch_last_error(b).decode()


def _bcheck(b, status):
    if status != BIE_OK:
        raise BieError(status, lib().bie_batch_last_error(b).decode() if b else "")


def bie_batch_set_problem(b, p, M, zeta, dzeta, d2zeta, zc, V1, a):
    import numpy as np
    Mh = np.ascontiguousarray(np.asarray(M, dtype=np.int32))
    zch = np.ascontiguousarray(np.asarray(zc if zc is not None else [], dtype=np.complex128))
    ah = np.ascontiguousarray(np.asarray(a if a is not None else [], dtype=np.float64))
    _bcheck(b, lib().bie_batch_set_problem(
        b, int(p), len(Mh), _hptr(Mh), _dptr(zeta, _c128(), "zeta"), _dptr(dzeta, _c128(), "dzeta"),
        _dptr(d2zeta, _c128(), "d2zeta"), _hptr(zch) if len(zch) else None, float(V1),
        _hptr(ah) if len(ah) else None))


def bie_batch_run(b, nprob, phit_all, omega_all, U_all, precision, opts=None,
                  raise_on_noconv=True):
    """Packed float64 CUDA arrays in problem order; returns a list of bie_solve_info."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    infos = (bie_solve_info * int(nprob))()
    o = opts if opts is not None else bie_default_opts()
    st = lib().bie_batch_run(b, int(nprob), _dptr(phit_all, _f64(), "phit_all"),
                             _dptr(omega_all, _f64(), "omega_all"), _dptr(U_all, _f64(), "U_all"),
                             int(precision), ctypes.byref(o), ctypes.cast(infos, ctypes.c_void_p))
    if not (st == BIE_ERR_NOCONV and not raise_on_noconv):
        _bcheck(b, st)
    return list(infos)


def bie_batch_tuning(b):
    """(chosen GEMV unit bytes, [kernel ms per candidate]) of the batch's autotuner."""
    ub = ctypes.c_longlong(0)
    ms = (ctypes.c_float * 5)()
    _bcheck(b, lib().bie_batch_tuning(b, ctypes.byref(ub), ctypes.cast(ms, ctypes.c_void_p)))
    return ub.value, list(ms)


def bie_batch_resid_bytes(b):
    """Matrix bytes the last bie_batch_run's residual products read (all problems)."""
    v = ctypes.c_double()
    _bcheck(b, lib().bie_batch_resid_bytes(b, ctypes.byref(v)))
    return v.value


def bie_test_grid_barrier(device=0, spin_limit=1 << 14, stall=-1):
    """Returns (status, barriers passed summed over CTAs, error flag)."""
    passed, err = ctypes.c_int(0), ctypes.c_int(0)
    st = lib().bie_test_grid_barrier(int(device), int(spin_limit), int(stall), ctypes.byref(passed),
                                     ctypes.byref(err))
    return st, passed.value, err.value


def bie_set_profiling(ctx, on):
    _check(ctx, lib().bie_set_profiling(ctx, 1 if on else 0))


def bie_get_profile(ctx):
    p = bie_profile()
    _check(ctx, lib().bie_get_profile(ctx, ctypes.byref(p)))
    return p


# ---------------------------------------------------------------------------
# a small convenience wrapper (still pure marshalling)
# ---------------------------------------------------------------------------

class Problem:
    """Holds device copies of one geometry + flow + phi~ and a context."""

    def __init__(self, geom, flow, phit, device=0, stream=None):
        import torch
        self.geom, self.flow = geom, flow
        dev = torch.device("cuda", device)
        self.M = list(geom.M)
        self.N = int(sum(self.M))
        self.zeta = torch.as_tensor(geom.zeta, dtype=torch.complex128, device=dev).contiguous()
        self.dzeta = torch.as_tensor(geom.dzeta, dtype=torch.complex128, device=dev).contiguous()
        self.d2zeta = torch.as_tensor(geom.d2zeta, dtype=torch.complex128, device=dev).contiguous()
        self.phit = torch.as_tensor(phit, dtype=torch.float64, device=dev).contiguous()
        self.ctx = bie_create(device, stream if stream is not None else torch.cuda.current_stream(dev))
        bie_set_geometry(self.ctx, self.M, self.zeta, self.dzeta, self.d2zeta, geom.zc)
        bie_set_flow(self.ctx, flow.V1, flow.a)
        self.omega = torch.zeros(self.N, dtype=torch.float64, device=dev)
        self.U = torch.zeros(self.M[0], dtype=torch.float64, device=dev)
        self.psi = torch.zeros(max(1, len(self.M) - 2), dtype=torch.float64, device=dev)

    def assemble(self, precision):
        bie_assemble(self.ctx, precision)

    def solve(self, opts=None, **kw):
        o = opts if opts is not None else bie_default_opts(**kw)
        return bie_solve(self.ctx, self.phit, self.omega, self.U, self.psi, o)

    def close(self):
        if self.ctx:
            bie_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autograd: U as a differentiable function of the node data, centres and phi~
# ---------------------------------------------------------------------------

class Solver:
    """A context plus the settings the differentiable solve needs: node counts,
    flow (V1, a_j) and storage precision.  Geometry is passed per call."""

    def __init__(self, M, V1, a=None, precision="fp32_ir", device=0, stream=None, opts=None):
        import torch
        self.M = [int(m) for m in M]
        self.V1, self.a = float(V1), (list(a) if a is not None else [])
        self.precision = precision
        self.opts = opts
        dev = torch.device("cuda", device)
        self.device = dev
        self.ctx = bie_create(device, stream if stream is not None else torch.cuda.current_stream(dev))

    def close(self):
        if self.ctx:
            bie_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def _solve_u_function():
    import torch

    class SolveU(torch.autograd.Function):
        """U(zeta, zeta', zeta'', z_j, phi~): forward = bie_set_geometry +
        bie_set_flow + bie_assemble + bie_solve; backward = bie_backward."""

        @staticmethod
        def forward(fctx, zeta, dzeta, d2zeta, zc, phit, solver):
            ctx = solver.ctx
            zc_host = zc.detach().cpu().numpy() if zc.numel() else None
            zeta, dzeta, d2zeta = (t.detach().contiguous() for t in (zeta, dzeta, d2zeta))
            phit = phit.detach().contiguous()
            bie_set_geometry(ctx, solver.M, zeta, dzeta, d2zeta, zc_host)
            bie_set_flow(ctx, solver.V1, solver.a)
            bie_assemble(ctx, solver.precision)
            N = sum(solver.M)
            omega = torch.empty(N, dtype=torch.float64, device=zeta.device)
            U = torch.empty(solver.M[0], dtype=torch.float64, device=zeta.device)
            bie_solve(ctx, phit, omega, U, None, solver.opts)
            fctx.solver = solver
            fctx.zc_shape = (zc.shape, zc.device)
            fctx.save_for_backward(omega)
            return U

        @staticmethod
        def backward(fctx, gU):
            (omega,) = fctx.saved_tensors
            solver = fctx.solver
            N = sum(solver.M)
            dev = omega.device
            out = {k: torch.empty(N, dtype=torch.complex128, device=dev)
                   for k in ("g_zeta", "g_dzeta", "g_d2zeta")}
            nobs = len(solver.M) - 2
            gzc = torch.empty(max(nobs, 1), dtype=torch.complex128, device=dev)
            gphit = torch.empty(solver.M[0], dtype=torch.float64, device=dev)
            bie_backward(solver.ctx, omega, gU.contiguous().to(torch.float64), None,
                         g_zc=gzc, g_phit=gphit, opts=solver.opts, **out)
            shape, zdev = fctx.zc_shape
            g_zc = gzc[:nobs].reshape(shape).to(zdev)
            return out["g_zeta"], out["g_dzeta"], out["g_d2zeta"], g_zc, gphit, None

    return SolveU


_SOLVE_U = None


def solve_u(zeta, dzeta, d2zeta, zc, phit, solver):
    """Differentiable U (float64, M_0) of complex128 CUDA node data, centres
    (complex128 tensor, nb-2, any device) and phi~ (float64 CUDA)."""
    global _SOLVE_U
    if _SOLVE_U is None:
        _SOLVE_U = _solve_u_function()
    return _SOLVE_U.apply(zeta, dzeta, d2zeta, zc, phit, solver)


# ---------------------------------------------------------------------------
# row partition over cooperating contexts (one per GPU)
# ---------------------------------------------------------------------------

_EXCHANGE_REFS = {}


def bie_set_partition(ctx, nparts, part, stage=None, exchange=None):
    """Row partition of the stored operator: part `part` of `nparts` (see
    bie_set_partition in include/bie.h).  `stage` is a CUDA tensor of at least
    8 * nparts * R bytes (R from bie_partition_rows after the geometry is set;
    partition_stage_bytes gives the size) and `exchange(op, count,
    elem_bytes, stream)` the collective on it (DistExchange below for
    torch.distributed).  nparts = 1 clears the partition."""
    key = ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx
    if nparts <= 1:
        _check(ctx, lib().bie_set_partition(ctx, 1, 0, None, 0, EXCHANGE_FN(), None))
        _EXCHANGE_REFS.pop(key, None)
        return

    def _cb(user, op, count, elem_bytes, stream):
        try:
            return int(exchange(op, count, elem_bytes, stream) or 0)
        except Exception:                       # reported to the library as a failure
            import traceback
            traceback.print_exc()
            return 1

    fn = EXCHANGE_FN(_cb)
    _check(ctx, lib().bie_set_partition(ctx, int(nparts), int(part), _dptr(stage),
                                        int(stage.numel() * stage.element_size()), fn, None))
    _EXCHANGE_REFS[key] = (fn, exchange, stage)


def bie_partition_rows(ctx):
    """(row0, row1, rows per part) of a context with a geometry."""
    r0, r1, R = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(ctx, lib().bie_partition_rows(ctx, ctypes.byref(r0), ctypes.byref(r1), ctypes.byref(R)))
    return r0.value, r1.value, R.value


def partition_rows(N, nparts, part):
    """The rows [row0, row1) that part `part` of `nparts` holds, and the rows
    per part R: R = 32 ceil(N / (32 nparts)) (the library's rule)."""
    if nparts <= 1:
        return 0, N, N
    R = (N + 32 * nparts - 1) // (32 * nparts) * 32
    return min(N, part * R), min(N, (part + 1) * R), R


def partition_stage_bytes(N, nparts):
    """Bytes of the staging buffer bie_set_partition needs."""
    return 8 * nparts * partition_rows(N, nparts, 0)[2]


class DistExchange:
    """The exchange of a row partition over a torch.distributed process group
    (NCCL between GPUs; the same calls work on CPU tensors under gloo).  The
    staging buffer holds nparts segments; part p's rows sit in segment p.
    Allgather: every segment to every part.  Allreduce: element-wise sum."""

    def __init__(self, stage, nparts, part, group=None):
        self.stage, self.nparts, self.part, self.group = stage, int(nparts), int(part), group

    def _run(self, op, count, elem_bytes):
        import torch
        import torch.distributed as dist
        if op == BIE_EXCH_ALLGATHER:
            dt = torch.float32 if elem_bytes == 4 else torch.float64
            buf = self.stage.view(dt)[: self.nparts * count]
            mine = buf[self.part * count:(self.part + 1) * count].clone()
            dist.all_gather_into_tensor(buf, mine, group=self.group)
        elif op == BIE_EXCH_ALLREDUCE_SUM:
            buf = self.stage.view(torch.float64)[:count]
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
        else:
            return 1
        return 0

    def __call__(self, op, count, elem_bytes, stream):
        import torch
        if self.stage.is_cuda:
            dev = self.stage.device
            s = torch.cuda.ExternalStream(stream, device=dev) if stream else torch.cuda.default_stream(dev)
            with torch.cuda.stream(s):
                return self._run(op, count, elem_bytes)
        return self._run(op, count, elem_bytes)
