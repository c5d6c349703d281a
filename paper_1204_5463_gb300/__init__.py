"""Python binding of ``libdwsolve.so`` (include/dwsolve.h, include/dwsolve_dense.h).

Argument marshalling only: every function below forwards to the C ABI of the
CUDA library with the same name. Pointers may be given as integers, torch
tensors (``data_ptr()``) or numpy arrays (host buffers). There is no CPU
fallback: importing the package raises if the CUDA library is missing.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwsolve.so")

DW_OK, DW_EINVAL, DW_ECUDA, DW_ENOMEM, DW_ENOTCONV, DW_EBREAKDOWN, DW_ENONFINITE, DW_ETIMEOUT, DW_ECANCELLED = range(9)
DW_F64, DW_F32, DW_F16, DW_BF16, DW_DF64 = range(5)
DW_MAX_RHS = 16
PREC = {"f64": DW_F64, "f32": DW_F32, "f16": DW_F16, "bf16": DW_BF16, "df64": DW_DF64}

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)


class dw_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("block", ctypes.c_int * 4), ("m0", ctypes.c_double)]


class dw_solver_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("k", ctypes.c_int), ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("max_iterations", ctypes.c_int), ("sap_cycles", ctypes.c_int), ("mr_steps", ctypes.c_int),
                ("sap_prec", ctypes.c_int), ("matvec_prec", ctypes.c_int), ("clean_restart_t", ctypes.c_double),
                ("nrhs", ctypes.c_int), ("host_buffers", ctypes.c_int), ("use_x0", ctypes.c_int),
                ("outer_prec", ctypes.c_int)]


class dw_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("cycles", ctypes.c_int), ("clean_restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("explicit_residuals", ctypes.c_int),
                ("iterations_rhs", ctypes.c_int * DW_MAX_RHS), ("true_rel_res", ctypes.c_double * DW_MAX_RHS),
                ("time_s", ctypes.c_double)]


class dw_tune_entry(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int * 4), ("seconds", ctypes.c_double), ("iterations", ctypes.c_int),
                ("status", ctypes.c_int)]


class dw_tune_sap_entry(ctypes.Structure):
    _fields_ = [("sap_cycles", ctypes.c_int), ("mr_steps", ctypes.c_int), ("seconds", ctypes.c_double),
                ("iterations", ctypes.c_int), ("status", ctypes.c_int)]


class dw_request(ctypes.Structure):
    _fields_ = [("lattice", dw_lattice), ("U", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("params", dw_solver_params)]


class dw_server_status(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("in_use_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("running", ctypes.c_int), ("queued", ctypes.c_int), ("completed", ctypes.c_longlong),
                ("reused", ctypes.c_longlong), ("peak_running", ctypes.c_int)]


class dw_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "dw_create": ([ctypes.POINTER(dw_lattice), _P, ctypes.POINTER(_P)], _I),
    "dw_destroy": ([_P], None),
    "dw_set_mass": ([_P, ctypes.c_double], _I),
    "dw_set_gauge": ([_P, _P, _I], _I),
    "dw_set_clover": ([_P, ctypes.c_double], _I),
    "dw_apply": ([_P, _P, _P, _I, _I], _I),
    "sap_precondition": ([_P, _P, _P, _I, _I, _I, _I], _I),
    "dw_default_params": ([ctypes.POINTER(dw_solver_params)], None),
    "fgmresdr_solve": ([_P, _P, _P, ctypes.POINTER(dw_solver_params), ctypes.POINTER(dw_stats)], _I),
    "dw_last_error": ([], ctypes.c_char_p),
    "dw_cancel": ([_P], _I),
    "dw_debug_basis": ([_P, _I, _P, _P, _P, _I, ctypes.POINTER(_I)], _I),
    "dw_residual_history": ([_P, _I, _P, _I, ctypes.POINTER(_I)], _I),
    "dw_profile": ([_P, _I], _I),
    "dw_kernel_launches": ([], ctypes.c_longlong),
    "dw_profile_read": ([_P, ctypes.POINTER(dw_kernel_stat), _I, ctypes.POINTER(_I), _I], _I),
    "dw_autotune_block": ([ctypes.POINTER(dw_lattice), _P, _P, ctypes.POINTER(dw_solver_params), _P,
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dw_tune_entry), _I, ctypes.POINTER(_I)], _I),
    "dw_autotune_sap": ([ctypes.POINTER(dw_lattice), _P, _P, ctypes.POINTER(dw_solver_params), _P,
                         ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(dw_tune_sap_entry), _I,
                         ctypes.POINTER(_I)], _I),
    "dw_apply_f32_noalloc": ([ctypes.POINTER(ctypes.c_int), ctypes.c_double, _P, _P, _P, _P], _I),
    "dw_request_bytes": ([ctypes.POINTER(dw_request)], ctypes.c_size_t),
    "dw_server_create": ([ctypes.c_size_t, _I, ctypes.POINTER(_P)], _I),
    "dw_server_submit": ([_P, ctypes.POINTER(dw_request), ctypes.POINTER(ctypes.c_uint64)], _I),
    "dw_server_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(dw_stats),
                        ctypes.POINTER(ctypes.c_double)], _I),
    "dw_server_wait": ([_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_I), ctypes.POINTER(dw_stats),
                        ctypes.POINTER(ctypes.c_double)], _I),
    "dw_server_cancel": ([_P, ctypes.c_uint64], _I),
    "dw_server_info": ([_P, ctypes.POINTER(dw_server_status)], _I),
    "dw_server_destroy": ([_P], None),
    "dw_dense_eig": ([_I, _P, _P, _P], _I),
    "dw_dense_qr": ([_I, _I, _P, _P, _P], _I),
    "dw_dense_lstsq": ([_I, _I, _I, _P, _P, _P, _P], _I),
    "dw_dense_solve": ([_I, _P, _P], _I),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class DwError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed with code {code}: {dw_last_error()}")


def _ptr(x):
    """Raw address of an int / torch tensor / numpy array / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(rc: int, where: str, allow=(DW_OK,)):
    if rc not in allow:
        raise DwError(rc, where)
    return rc


def dw_last_error() -> str:
    return _lib.dw_last_error().decode()


def dw_create(dims, block, m0: float, stream=None) -> int:
    L = dw_lattice((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*block), float(m0))
    h = _P()
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib.dw_create(ctypes.byref(L), s, ctypes.byref(h)), "dw_create")
    return h.value


def dw_destroy(ctx) -> None:
    _lib.dw_destroy(ctx)


def dw_set_mass(ctx, m0: float) -> None:
    _check(_lib.dw_set_mass(ctx, float(m0)), "dw_set_mass")


def dw_set_gauge(ctx, U, on_device: bool) -> None:
    _check(_lib.dw_set_gauge(ctx, _ptr(U), int(bool(on_device))), "dw_set_gauge")


def dw_set_clover(ctx, csw: float) -> None:
    """Add the clover term with coefficient csw (0 restores plain Wilson)."""
    _check(_lib.dw_set_clover(ctx, float(csw)), "dw_set_clover")


def dw_apply(ctx, inp, out, prec: int = DW_F64, nrhs: int = 1) -> None:
    _check(_lib.dw_apply(ctx, _ptr(inp), _ptr(out), int(prec), int(nrhs)), "dw_apply")


def sap_precondition(ctx, v, z, ncycles: int, nmr: int, storage: int = DW_F32, nrhs: int = 1) -> None:
    _check(_lib.sap_precondition(ctx, _ptr(v), _ptr(z), int(ncycles), int(nmr), int(storage), int(nrhs)),
           "sap_precondition")


def dw_default_params(**overrides) -> dw_solver_params:
    P = dw_solver_params()
    _lib.dw_default_params(ctypes.byref(P))
    for k, v in overrides.items():
        if not hasattr(P, k):
            raise AttributeError(k)
        setattr(P, k, v)
    return P


def fgmresdr_solve(ctx, b, x, params: dw_solver_params, allow_notconv: bool = False,
                   allow_cancelled: bool = False) -> dw_stats:
    S = dw_stats()
    allow = (DW_OK, DW_ENOTCONV) if allow_notconv else (DW_OK,)
    if allow_cancelled:
        allow = allow + (DW_ECANCELLED,)
    rc = _lib.fgmresdr_solve(ctx, _ptr(b), _ptr(x), ctypes.byref(params), ctypes.byref(S))
    _check(rc, "fgmresdr_solve", allow)
    S.status = rc
    return S


def dw_cancel(ctx) -> None:
    _check(_lib.dw_cancel(ctx), "dw_cancel")


def dw_debug_basis(ctx, rhs: int, V_out=None, Z_out=None, H_out=None, max_cols: int = 64) -> int:
    """Copies the last cycle's bases of rhs (see include/dwsolve.h); returns the column count m'."""
    n = _I(0)
    _check(_lib.dw_debug_basis(ctx, int(rhs), _ptr(V_out), _ptr(Z_out), _ptr(H_out), int(max_cols), ctypes.byref(n)),
           "dw_debug_basis")
    return n.value


def dw_residual_history(ctx, rhs: int = 0):
    """[(steps, implicit rel. residual, explicit rel. residual)] per cycle of the last solve."""
    n = _I(0)
    _check(_lib.dw_residual_history(ctx, int(rhs), None, 0, ctypes.byref(n)), "dw_residual_history")
    buf = (ctypes.c_double * (3 * max(1, n.value)))()
    _check(_lib.dw_residual_history(ctx, int(rhs), buf, n.value, ctypes.byref(n)), "dw_residual_history")
    return [(int(buf[3 * i]), buf[3 * i + 1], buf[3 * i + 2]) for i in range(n.value)]


def dw_kernel_launches() -> int:
    return int(_lib.dw_kernel_launches())


def dw_profile(ctx, enable: bool) -> None:
    _check(_lib.dw_profile(ctx, int(bool(enable))), "dw_profile")


def dw_profile_read(ctx, reset: bool = False) -> dict:
    buf = (dw_kernel_stat * 64)()
    n = _I()
    _check(_lib.dw_profile_read(ctx, buf, 64, ctypes.byref(n), int(bool(reset))), "dw_profile_read")
    return {buf[i].name.decode(): dict(launches=buf[i].launches, total_ms=buf[i].total_ms, bytes=buf[i].bytes)
            for i in range(min(n.value, 64))}


def dw_autotune_block(dims, m0: float, U, b, params: dw_solver_params, stream=None, with_results: bool = True):
    """Best SAP domain block by calibration-solve time; returns (block, [(block, seconds, iterations, status)])."""
    L = dw_lattice((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(0, 0, 0, 0), float(m0))
    best = (ctypes.c_int * 4)()
    res = (dw_tune_entry * 256)() if with_results else None
    n = _I(0)
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib.dw_autotune_block(ctypes.byref(L), _ptr(U), _ptr(b), ctypes.byref(params), s, best,
                                  res, 256 if with_results else 0, ctypes.byref(n)), "dw_autotune_block")
    table = [(tuple(res[i].block), res[i].seconds, res[i].iterations, res[i].status)
             for i in range(min(n.value, 256))] if with_results else []
    return tuple(best), table


def dw_autotune_sap(dims, block, m0: float, U, b, params: dw_solver_params, stream=None, with_results: bool = True):
    """Best (sap_cycles, mr_steps) on this block by calibration-solve time;
    returns ((cycles, mr), [(cycles, mr, seconds, iterations, status)])."""
    L = dw_lattice((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*block), float(m0))
    c, m = _I(), _I()
    res = (dw_tune_sap_entry * 64)() if with_results else None
    n = _I(0)
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib.dw_autotune_sap(ctypes.byref(L), _ptr(U), _ptr(b), ctypes.byref(params), s, ctypes.byref(c),
                                ctypes.byref(m), res, 64 if with_results else 0, ctypes.byref(n)), "dw_autotune_sap")
    table = [(res[i].sap_cycles, res[i].mr_steps, res[i].seconds, res[i].iterations, res[i].status)
             for i in range(min(n.value, 64))] if with_results else []
    return (c.value, m.value), table


def dw_apply_f32_noalloc(dims, m0: float, U, inp, out, stream=None) -> None:
    """out = D in (FP32) without any device allocation (lattices up to 4096 sites)."""
    d = (ctypes.c_int * 4)(*dims)
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib.dw_apply_f32_noalloc(d, float(m0), _ptr(U), _ptr(inp), _ptr(out), s), "dw_apply_f32_noalloc")


def make_request(dims, block, m0, U, b, x, params: dw_solver_params) -> dw_request:
    """A request over host buffers (numpy arrays kept alive by the caller)."""
    L = dw_lattice((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*block), float(m0))
    return dw_request(L, _ptr(U), _ptr(b), _ptr(x), params)


def dw_request_bytes(req: dw_request) -> int:
    return int(_lib.dw_request_bytes(ctypes.byref(req)))


def dw_server_create(hbm_budget_bytes: int, max_slots: int) -> int:
    h = _P()
    _check(_lib.dw_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)), "dw_server_create")
    return h.value


def dw_server_submit(server, req: dw_request) -> int:
    rid = ctypes.c_uint64()
    _check(_lib.dw_server_submit(server, ctypes.byref(req), ctypes.byref(rid)), "dw_server_submit")
    return rid.value


def dw_server_poll(server, rid: int):
    done, status, lat = _I(), _I(), ctypes.c_double()
    S = dw_stats()
    _check(_lib.dw_server_poll(server, int(rid), ctypes.byref(done), ctypes.byref(status), ctypes.byref(S),
                               ctypes.byref(lat)), "dw_server_poll")
    return bool(done.value), status.value, S, lat.value


def dw_server_wait(server, rid: int, timeout_s: float = 600.0):
    status, lat = _I(), ctypes.c_double()
    S = dw_stats()
    _check(_lib.dw_server_wait(server, int(rid), float(timeout_s), ctypes.byref(status), ctypes.byref(S),
                               ctypes.byref(lat)), "dw_server_wait")
    return status.value, S, lat.value


def dw_server_cancel(server, rid: int) -> None:
    _check(_lib.dw_server_cancel(server, int(rid)), "dw_server_cancel")


def dw_server_info(server) -> dict:
    st = dw_server_status()
    _check(_lib.dw_server_info(server, ctypes.byref(st)), "dw_server_info")
    return {f: getattr(st, f) for f, _ in dw_server_status._fields_}


def dw_server_destroy(server) -> None:
    _lib.dw_server_destroy(server)


def dw_dense_eig(n: int, A, lam, vecs) -> None:
    _check(_lib.dw_dense_eig(int(n), _ptr(A), _ptr(lam), _ptr(vecs)), "dw_dense_eig")


def dw_dense_qr(rows: int, cols: int, G, Q, R=None) -> None:
    _check(_lib.dw_dense_qr(int(rows), int(cols), _ptr(G), _ptr(Q), _ptr(R)), "dw_dense_qr")


def dw_dense_lstsq(rows: int, cols: int, dense_rows: int, H, c, eta, residual) -> None:
    _check(_lib.dw_dense_lstsq(int(rows), int(cols), int(dense_rows), _ptr(H), _ptr(c), _ptr(eta), _ptr(residual)),
           "dw_dense_lstsq")


def dw_dense_solve(n: int, A, b) -> None:
    _check(_lib.dw_dense_solve(int(n), _ptr(A), _ptr(b)), "dw_dense_solve")


def lib_path() -> str:
    return LIB_PATH
