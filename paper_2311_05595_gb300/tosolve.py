"""Python binding of the tosolve C ABI (include/tosolve.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels
of libtosolve.so.  Functions keep the C names; device buffers are passed as
torch CUDA tensors (or raw integer addresses) and streams as torch streams.
There is no CPU fallback: if the library is missing, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtosolve.so")

OK, EINVAL, ENOMEM, ENOTCONV, EBREAKDOWN, ECUDA = range(6)
PREC_FP64, PREC_FP32, PREC_TF32, PREC_FP32X2, PREC_BF16, PREC_BF16X3, PREC_F16X3 = 0, 1, 2, 3, 4, 5, 6
SMOOTH_JACOBI, SMOOTH_CHEBYSHEV = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTCONV", 4: "EBREAKDOWN", 5: "ECUDA"}


class tosolve_desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("degree", C.c_int), ("n_mr", C.c_int), ("d_mr", C.c_int),
        ("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
        ("penal", C.c_double), ("rmin", C.c_double),
        ("mg_levels", C.c_int), ("precision", C.c_int),
        ("omega", C.c_double), ("cycle_gamma", C.c_int), ("max_rhs", C.c_int),
        ("family", C.c_int), ("prolongation", C.c_int), ("inner_its", C.c_int),
        ("smoother", C.c_int), ("cheb_degree", C.c_int),
    ]


class tosolve_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int), ("total_iterations", C.c_int),
        ("rel_residual", C.c_double), ("ms", C.c_double), ("status", C.c_int),
    ]


class tosolve_server_desc(C.Structure):
    _fields_ = [("slots", C.c_int), ("hbm_budget", C.c_size_t), ("rtol", C.c_double),
                ("maxit", C.c_int)]


class tosolve_request_result(C.Structure):
    _fields_ = [("request", C.c_longlong), ("design", C.c_int), ("status", C.c_int),
                ("iterations", C.c_int), ("cold", C.c_int), ("compliance", C.c_double),
                ("rel_residual", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_end", C.c_double)]


class tosolve_server_info(C.Structure):
    _fields_ = [("designs", C.c_int), ("resident_designs", C.c_int), ("pending", C.c_int),
                ("running", C.c_int), ("resident_bytes", C.c_size_t), ("builds", C.c_longlong),
                ("evictions", C.c_longlong), ("now", C.c_double)]


class TosolveError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"{_LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the solver has no CPU fallback)")
    lib = C.CDLL(_LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    sigs = {
        "tosolve_create": ([P(tosolve_desc), vp, vp, P(vp)], i),
        "tosolve_footprint": ([P(tosolve_desc), P(sz)], i),
        "tosolve_create_mixed": ([P(tosolve_desc), vp, vp, vp, P(vp)], i),
        "tosolve_free_dofs": ([vp, P(C.c_longlong)], i),
        "tosolve_set_densities": ([vp, vp], i),
        "tosolve_solve": ([vp, vp, i, vp, d, i, P(tosolve_info)], i),
        "tosolve_compliance_grad": ([vp, vp, vp, i, P(d), vp, vp], i),
        "tosolve_step_host": ([vp, vp, vp, i, d, i, i, vp, P(d), vp, P(tosolve_info)], i),
        "tosolve_level_dims": ([vp, i, P(i)], i),
        "tosolve_subcell_table": ([vp, vp], i),
        "tosolve_densities": ([vp, vp, vp], i),
        "tosolve_apply": ([vp, i, i, vp, vp], i),
        "tosolve_precondition": ([vp, vp, vp], i),
        "tosolve_tc_stage": ([vp, i, i, vp], i),
        "tosolve_smoother_lmax": ([vp, i, vp], i),
        "tosolve_tune": ([vp, i, vp, vp, vp, vp, i, C.c_double, i, i, vp, vp], i),
        "tosolve_tune_pick": ([vp, i, i, i, C.c_double, vp], i),
        "tosolve_batch_create": ([P(vp), i, P(i), P(vp), P(vp), P(vp)], i),
        "tosolve_batch_solve": ([vp, d, i, vp], i),
        "tosolve_batch_destroy": ([vp], None),
        "tosolve_compliance_noalloc": ([vp, vp, vp, sz, i, vp, vp], i),
        "tosolve_server_create": ([P(tosolve_server_desc), P(vp)], i),
        "tosolve_server_add_design": ([vp, i, P(tosolve_desc), vp, vp, i], i),
        "tosolve_server_submit": ([vp, i, vp, vp, P(C.c_longlong)], i),
        "tosolve_server_poll": ([vp, P(tosolve_request_result), i, i], i),
        "tosolve_server_stats": ([vp, P(tosolve_server_info)], i),
        "tosolve_server_last_error": ([], C.c_char_p),
        "tosolve_server_failure": ([vp, i], C.c_char_p),
        "tosolve_server_destroy": ([vp], None),
        "tosolve_trim_pool": ([sz], i),
        "tosolve_fix_variables": ([vp, vp, C.c_double, C.c_double, C.c_double, vp, P(C.c_longlong)], i),
        "tosolve_release_variables": ([vp], i),
        "tosolve_threshold_scratch_bytes": ([C.c_longlong], sz),
        "tosolve_heaviside": ([vp, C.c_longlong, C.c_double, vp, P(C.c_double), P(i), vp, sz, vp], i),
        "tosolve_threshold_density": ([vp, C.c_longlong, C.c_double, C.c_double, C.c_double, vp, C.c_double,
                                       vp, P(i), vp, sz, vp], i),
        "tosolve_threshold_gradient": ([vp, vp, C.c_longlong, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_double, vp, P(C.c_double), vp, sz, vp], i),
        "tosolve_last_error": ([vp], C.c_char_p),
        "tosolve_destroy": ([vp], None),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _check(h, status: int, what: str):
    if status != OK:
        msg = _lib.tosolve_last_error(h)
        raise TosolveError(status, f"{what}: {msg.decode() if msg else ''}")


FAMILY_LAGRANGE, FAMILY_SERENDIPITY = 0, 1


def make_desc(nx, ny, nz, *, degree=1, n_mr=1, d_mr=None, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0,
              rmin=0.0, mg_levels=0, precision=PREC_FP64, omega=0.0, cycle_gamma=1,
              max_rhs=1, family=FAMILY_LAGRANGE, prolongation=0, inner_its=0, smoother=SMOOTH_JACOBI,
              cheb_degree=0) -> tosolve_desc:
    return tosolve_desc(nx, ny, nz, degree, n_mr, d_mr or n_mr, E0, Emin, nu, penal, rmin, mg_levels,
                        precision, omega, cycle_gamma, max_rhs, family, prolongation, inner_its, smoother,
                        cheb_degree)


# ---- the C ABI, same names ----------------------------------------------------

def tosolve_footprint(desc: tosolve_desc) -> int:
    out = C.c_size_t(0)
    _check(None, _lib.tosolve_footprint(C.byref(desc), C.byref(out)), "tosolve_footprint")
    return out.value


def tosolve_create(desc: tosolve_desc, mask: np.ndarray, stream=None) -> int:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    h = C.c_void_p(0)
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    _check(None, _lib.tosolve_create(C.byref(desc), mask.ctypes.data, st, C.byref(h)),
           "tosolve_create")
    return h.value


def tosolve_create_mixed(desc: tosolve_desc, mask: np.ndarray, elem_q1: np.ndarray, stream=None) -> int:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    q1 = np.ascontiguousarray(elem_q1, dtype=np.uint8)
    h = C.c_void_p(0)
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    _check(None, _lib.tosolve_create_mixed(C.byref(desc), mask.ctypes.data, q1.ctypes.data, st,
                                           C.byref(h)), "tosolve_create_mixed")
    return h.value


def tosolve_free_dofs(h) -> int:
    n = C.c_longlong(0)
    _check(h, _lib.tosolve_free_dofs(h, C.byref(n)), "tosolve_free_dofs")
    return n.value


def tosolve_destroy(h) -> None:
    _lib.tosolve_destroy(h)


def tosolve_set_densities(h, x_dev) -> None:
    _check(h, _lib.tosolve_set_densities(h, _ptr(x_dev)), "tosolve_set_densities")


def tosolve_solve(h, f_dev, nrhs: int, u_dev, rtol: float, maxit: int, raise_on_error=True):
    info = tosolve_info()
    s = _lib.tosolve_solve(h, _ptr(f_dev), nrhs, _ptr(u_dev), rtol, maxit, C.byref(info))
    if raise_on_error:
        _check(h, s, "tosolve_solve")
    return info


def tosolve_compliance_grad(h, u_dev, f_dev, nrhs: int, dcdx_dev=None, dcdrho_dev=None):
    c = (C.c_double * nrhs)()
    _check(h, _lib.tosolve_compliance_grad(h, _ptr(u_dev), _ptr(f_dev), nrhs, c, _ptr(dcdx_dev),
                                           _ptr(dcdrho_dev)), "tosolve_compliance_grad")
    return np.array(c[:])


def tosolve_step_host(h, x_host: np.ndarray, f_host: np.ndarray, nrhs: int, rtol: float, maxit: int,
                      warm: int = 0, u_host: np.ndarray | None = None,
                      dcdx_host: np.ndarray | None = None):
    c = (C.c_double * nrhs)()
    info = tosolve_info()
    s = _lib.tosolve_step_host(h, _ptr(x_host), _ptr(f_host), nrhs, rtol, maxit, warm, _ptr(u_host),
                               c, _ptr(dcdx_host), C.byref(info))
    _check(h, s, "tosolve_step_host")
    return np.array(c[:]), info


def tosolve_batch_create(handles, nrhs, f_devs, u_devs) -> int:
    n = len(handles)
    if not (len(nrhs) == len(f_devs) == len(u_devs) == n):
        raise ValueError("handles, nrhs, f_devs and u_devs must have the same length")
    hv = (C.c_void_p * n)(*handles)
    rv = (C.c_int * n)(*nrhs)
    fv = (C.c_void_p * n)(*[_ptr(t) for t in f_devs])
    uv = (C.c_void_p * n)(*[_ptr(t) for t in u_devs])
    b = C.c_void_p(0)
    _check(None, _lib.tosolve_batch_create(hv, n, rv, fv, uv, C.byref(b)), "tosolve_batch_create")
    return b.value


def tosolve_batch_solve(b, rtol: float, maxit: int, count: int, raise_on_error=True):
    infos = (tosolve_info * count)()
    s = _lib.tosolve_batch_solve(b, rtol, maxit, infos)
    if raise_on_error:
        _check(None, s, "tosolve_batch_solve")
    return list(infos)


def tosolve_batch_destroy(b) -> None:
    _lib.tosolve_batch_destroy(b)


def _check_server(status: int, what: str):
    if status != OK:
        msg = _lib.tosolve_server_last_error()
        raise TosolveError(status, f"{what}: {msg.decode() if msg else ''}")


def tosolve_server_create(slots: int, hbm_budget: int, rtol: float, maxit: int) -> int:
    d = tosolve_server_desc(slots, hbm_budget, rtol, maxit)
    s = C.c_void_p(0)
    _check_server(_lib.tosolve_server_create(C.byref(d), C.byref(s)), "tosolve_server_create")
    return s.value


def tosolve_server_add_design(s, design: int, desc: tosolve_desc, mask: np.ndarray, f: np.ndarray,
                              nrhs: int) -> None:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check_server(_lib.tosolve_server_add_design(s, design, C.byref(desc), mask.ctypes.data,
                                                 f.ctypes.data, nrhs), "tosolve_server_add_design")


def tosolve_server_submit(s, design: int, x: np.ndarray, dcdx: np.ndarray | None = None) -> int:
    """x is copied at once; dcdx (if given) is written when the request
    completes and must stay alive until its result has been polled."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rid = C.c_longlong(0)
    _check_server(_lib.tosolve_server_submit(s, design, x.ctypes.data, _ptr(dcdx), C.byref(rid)),
                  "tosolve_server_submit")
    return rid.value


def tosolve_server_poll(s, max_results: int = 64, timeout_ms: int = 100) -> list:
    buf = (tosolve_request_result * max_results)()
    n = _lib.tosolve_server_poll(s, buf, max_results, timeout_ms)
    return [buf[k] for k in range(n)]


def tosolve_server_stats(s) -> tosolve_server_info:
    info = tosolve_server_info()
    _check_server(_lib.tosolve_server_stats(s, C.byref(info)), "tosolve_server_stats")
    return info


def tosolve_server_failures(s) -> list:
    """Messages of the most recent failed requests, newest first."""
    out = []
    while True:
        m = _lib.tosolve_server_failure(s, len(out))
        if not m:
            return out
        out.append(m.decode())


def tosolve_server_destroy(s) -> None:
    _lib.tosolve_server_destroy(s)


NOALLOC_MAX_RHS = 16


def tosolve_compliance_noalloc(f_dev, u_dev, mask_dev, ndof: int, nrhs: int, c_dev, stream=None) -> None:
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    _check(None, _lib.tosolve_compliance_noalloc(_ptr(f_dev), _ptr(u_dev), _ptr(mask_dev), ndof, nrhs,
                                                 _ptr(c_dev), st), "tosolve_compliance_noalloc")


def tosolve_fix_variables(h, dcdx_dev=None, rho_lo: float = 1e-6, rho_hi: float = 0.9,
                          eps_grad: float = 1e-6, fixed_dev=None) -> int:
    """Sec. 6.1 fixing; returns the number of suppressed DOFs."""
    n = C.c_longlong(0)
    _check(h, _lib.tosolve_fix_variables(h, _ptr(dcdx_dev), rho_lo, rho_hi, eps_grad, _ptr(fixed_dev),
                                         C.byref(n)), "tosolve_fix_variables")
    return n.value


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def tosolve_threshold_scratch_bytes(n: int) -> int:
    return int(_lib.tosolve_threshold_scratch_bytes(n))


def tosolve_heaviside(rho_dev, beta: float, out_dev, scratch_dev, stream=None) -> tuple[float, int]:
    """Sec. 5 Heaviside projection; returns (eta, Newton iterations)."""
    eta, its = C.c_double(0.0), C.c_int(0)
    _check(None, _lib.tosolve_heaviside(_ptr(rho_dev), rho_dev.numel(), beta, _ptr(out_dev), C.byref(eta),
                                        C.byref(its), _ptr(scratch_dev), scratch_dev.numel() * scratch_dev.element_size(),
                                        _stream_ptr(stream)), "tosolve_heaviside")
    return eta.value, its.value


def tosolve_threshold_density(rho_dev, vfrac: float, gradL_dev, out_dev, scratch_dev, round_lo: float = 0.05,
                              round_hi: float = 0.95, theta_max_deg: float = 89.9, stream=None) -> bool:
    acc = C.c_int(0)
    _check(None, _lib.tosolve_threshold_density(_ptr(rho_dev), rho_dev.numel(), vfrac, round_lo, round_hi,
                                                _ptr(gradL_dev), theta_max_deg, _ptr(out_dev), C.byref(acc),
                                                _ptr(scratch_dev), scratch_dev.numel() * scratch_dev.element_size(),
                                                _stream_ptr(stream)), "tosolve_threshold_density")
    return bool(acc.value)


def tosolve_threshold_gradient(rho_dev, gradL_dev, out_dev, scratch_dev, round_lo: float = 0.05,
                               round_hi: float = 0.95, vu_min: float = 0.3, vl_max: float = 0.7,
                               theta_max_deg: float = 89.9, stream=None) -> float:
    alpha = C.c_double(0.0)
    _check(None, _lib.tosolve_threshold_gradient(_ptr(rho_dev), _ptr(gradL_dev), rho_dev.numel(), round_lo,
                                                 round_hi, vu_min, vl_max, theta_max_deg, _ptr(out_dev),
                                                 C.byref(alpha), _ptr(scratch_dev),
                                                 scratch_dev.numel() * scratch_dev.element_size(),
                                                 _stream_ptr(stream)), "tosolve_threshold_gradient")
    return alpha.value


def tosolve_release_variables(h) -> None:
    _check(h, _lib.tosolve_release_variables(h), "tosolve_release_variables")


def tosolve_trim_pool(keep_bytes: int = 0) -> None:
    _check(None, _lib.tosolve_trim_pool(keep_bytes), "tosolve_trim_pool")


def tosolve_level_count(h) -> int:
    """Multigrid levels of a handle (the levels tosolve_level_dims accepts)."""
    dims = (C.c_int * 3)()
    n = 0
    while n < 8 and _lib.tosolve_level_dims(h, n, dims) == OK:
        n += 1
    return n


def tosolve_level_dims(h, level: int):
    dims = (C.c_int * 3)()
    _check(h, _lib.tosolve_level_dims(h, level, dims), "tosolve_level_dims")
    return tuple(dims[:])


def tosolve_subcell_table(h, table_dev) -> None:
    _check(h, _lib.tosolve_subcell_table(h, _ptr(table_dev)), "tosolve_subcell_table")


def tosolve_densities(h, rho_dev=None, w_dev=None) -> None:
    _check(h, _lib.tosolve_densities(h, _ptr(rho_dev), _ptr(w_dev)), "tosolve_densities")


def tosolve_apply(h, level: int, precision: int, x_dev, y_dev) -> None:
    _check(h, _lib.tosolve_apply(h, level, precision, _ptr(x_dev), _ptr(y_dev)), "tosolve_apply")


def tosolve_tc_stage(h, part: int, stages: int, x_dev=None) -> None:
    _check(h, _lib.tosolve_tc_stage(h, part, stages, _ptr(x_dev)),
           "tosolve_tc_stage")


def tosolve_smoother_lmax(h, level: int) -> float:
    v = C.c_double(0.0)
    _check(h, _lib.tosolve_smoother_lmax(h, level, C.byref(v)), "tosolve_smoother_lmax")
    return v.value


def tosolve_tune(cands, mask: np.ndarray, x_dev, f_dev, nrhs: int, rtol: float, maxit: int, reps: int,
                 stream=None, elem_q1=None) -> np.ndarray:
    """Times each candidate descriptor (a list of tosolve_desc) on one
    instance; returns ms[ncand, reps] (+inf where a candidate failed)."""
    n = len(cands)
    arr = (tosolve_desc * n)(*cands)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    eq = None if elem_q1 is None else np.ascontiguousarray(elem_q1, dtype=np.uint8)
    out = np.zeros(n * reps)
    st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(None, _lib.tosolve_tune(arr, n, _ptr(mask), _ptr(eq), _ptr(x_dev), _ptr(f_dev), nrhs, rtol, maxit,
                                   reps, st, _ptr(out)), "tosolve_tune")
    return out.reshape(n, reps)


def tosolve_tune_pick(ms: np.ndarray, min_gain: float) -> np.ndarray:
    """ms[nclass, ncand, reps] -> the chosen candidate per class (-1: none)."""
    ms = np.ascontiguousarray(ms, dtype=np.float64)
    k, c, r = ms.shape
    out = np.zeros(k, dtype=np.int32)
    _check(None, _lib.tosolve_tune_pick(_ptr(ms), k, c, r, min_gain, _ptr(out)), "tosolve_tune_pick")
    return out


def tosolve_precondition(h, b_dev, z_dev) -> None:
    _check(h, _lib.tosolve_precondition(h, _ptr(b_dev), _ptr(z_dev)), "tosolve_precondition")


def tosolve_last_error(h) -> str:
    msg = _lib.tosolve_last_error(h)
    return msg.decode() if msg else ""


class Solver:
    """Owns one handle; a convenience wrapper used by the tests and the
    benchmark (each method is one ABI call)."""

    def __init__(self, desc: tosolve_desc, mask: np.ndarray, stream=None, elem_q1=None):
        self.desc = desc
        self.h = (tosolve_create(desc, mask, stream) if elem_q1 is None
                  else tosolve_create_mixed(desc, mask, elem_q1, stream))

    def close(self):
        if self.h:
            tosolve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
