"""Python binding of the C ABI in include/pressure_projection.h.

Argument marshalling only: every step of the projection runs in the CUDA
library ``libpp_gb300.so`` built in-tree by ``build_ext.py``.  Field
arguments are float64, C-contiguous torch tensors (CUDA or CPU) or numpy
arrays; CPU/numpy buffers are host pointers, which the library stages
through its own device buffers.  Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpp_gb300.so")

PP_OK, PP_ERR_INVALID_ARG, PP_ERR_UNSUPPORTED, PP_ERR_NOT_CONVERGED = 0, 1, 2, 3
PP_ERR_NUMERIC, PP_ERR_CUDA, PP_ERR_OOM, PP_ERR_TOO_LARGE = 4, 5, 6, 7
PP_BC_PERIODIC, PP_BC_WALL = 0, 1
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_fp32": 1, "mixed_tc": 2, "mixed_z64": 3}
# iterations of Sec. 3.3.1: Method III (Eq. new_poisson), I (Eq. poisson_me1), II (Eq. poisson_laizet)
METHODS = {"III": 0, "I": 1, "II": 2}


class pp_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("zfaces", ctypes.POINTER(ctypes.c_double)), ("bc", ctypes.c_int * 3),
                ("yfaces", ctypes.POINTER(ctypes.c_double))]


class pp_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("res_l1_sum", ctypes.c_double), ("mean_S_removed", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pp_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double)]


class PressureError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {status_string(code)} (pp_status {code})")
        self.code = code


_lib = None

EXPORTS = ("pressure_plan_create", "pressure_plan_destroy", "pressure_plan_set_method",
           "pressure_plan_set_zsolve", "pressure_solve", "pressure_mixture_density", "pressure_correct", "pressure_solve_adjoint",
           "pressure_last_info", "pressure_profile_enable", "pressure_profile_read",
           "pressure_solve_noalloc", "pressure_batch_create", "pressure_batch_layout",
           "pressure_batch_correct", "pressure_batch_destroy", "pressure_batch_mixture_density",
           "pressure_p0_rate", "pressure_dp0dt_extrapolate", "pressure_divergence_source",
           "pressure_predictor",
           "pressure_status_string")


def lib():
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2005_11806_gb300.build_ext` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    pinfo = ctypes.POINTER(pp_info)
    L.pressure_plan_create.argtypes = [ctypes.POINTER(pp_grid), i, vp, ctypes.POINTER(vp)]
    L.pressure_plan_destroy.argtypes = [vp]
    L.pressure_plan_set_method.argtypes = [vp, i]
    L.pressure_plan_set_zsolve.argtypes = [vp, i]
    L.pressure_solve.argtypes = [vp, vp, vp, pinfo]
    L.pressure_mixture_density.argtypes = [vp, vp, d, d, vp]
    L.pressure_correct.argtypes = [vp, vp, vp, vp, vp, vp, d, vp, i, vp, vp, vp, d, i, pinfo]
    L.pressure_solve_adjoint.argtypes = [vp, vp, vp, d, vp, vp, vp, vp, vp, vp, vp, d, i, pinfo]
    L.pressure_last_info.argtypes = [vp, pinfo]
    L.pressure_profile_enable.argtypes = [vp, i]
    L.pressure_profile_read.argtypes = [vp, ctypes.POINTER(pp_kernel_time), i,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
    L.pressure_solve_noalloc.argtypes = [ctypes.POINTER(pp_grid), vp, vp, vp]
    ll = ctypes.c_longlong
    L.pressure_batch_create.argtypes = [ctypes.POINTER(pp_grid), i, i, vp, ctypes.POINTER(vp)]
    L.pressure_batch_layout.argtypes = [vp, ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(ll),
                                        ctypes.POINTER(ctypes.c_int)]
    L.pressure_batch_correct.argtypes = [vp, vp, vp, vp, vp, vp, d, vp, vp, vp, vp, d, i, pinfo]
    L.pressure_batch_destroy.argtypes = [vp]
    L.pressure_batch_mixture_density.argtypes = [vp, vp, d, d, vp]
    L.pressure_p0_rate.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, ctypes.POINTER(d)]
    L.pressure_dp0dt_extrapolate.argtypes = [d, d, d, d, ctypes.POINTER(d)]
    L.pressure_divergence_source.argtypes = [vp, vp, vp, vp, d, d, d, vp]
    L.pressure_predictor.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(d), d, d,
                                     ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.pressure_status_string.argtypes = [i]
    L.pressure_status_string.restype = ctypes.c_char_p
    for name in EXPORTS[:-1]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def status_string(code):
    return lib().pressure_status_string(int(code)).decode()


def _ptr(x):
    """Address of a float64 C-contiguous buffer (torch tensor or numpy)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy fields must be C-contiguous float64")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensor fields must be contiguous float64")
        return x.data_ptr()
    raise TypeError(f"unsupported field type {type(x)}")


def _stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return 0


def _check(code, what, allow=()):
    if code != PP_OK and code not in allow:
        raise PressureError(code, what)
    return code


# Cell and z-face counts of the plans this module created.  Fields are
# checked against them before a call: the library sees raw pointers, and a
# short buffer would be read or written past its end on the device.
_PLAN_SIZES = {}


def _sized(plan, *fields):
    """fields: (array or None, kind) pairs, kind "c" for a cell field
    ([nz][ny][nx]) and "w" for a z-face field ([nz+1][ny][nx])."""
    dims = _PLAN_SIZES.get(plan)
    if dims is None:
        return
    for x, kind in fields:
        if x is None:
            continue
        n = x.size if isinstance(x, np.ndarray) else getattr(x, "numel", lambda: None)()
        need = dims[0] if kind == "c" else dims[1]
        if n is not None and n < need:
            raise ValueError(f"a {'cell' if kind == 'c' else 'z-face'} field needs {need} elements, got {n}")


def pressure_plan_create(nx, ny, nz, lx, ly, lz, zfaces=None, precision="fp64", stream=None,
                         ywalls=False, yfaces=None):
    """Create a plan; returns an opaque handle (int).  ``zfaces``: None for a
    uniform z grid, else nz + 1 increasing face coordinates (host array).
    ``ywalls``: walls at y = 0 and y = ly instead of periodic y.  ``yfaces``
    (walls in y only): ny + 1 increasing face coordinates of a stretched y."""
    g = pp_grid()
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    g.lx, g.ly, g.lz = float(lx), float(ly), float(lz)
    keep = ykeep = None
    if zfaces is not None:
        keep = np.ascontiguousarray(zfaces, dtype=np.float64)
        if keep.shape != (int(nz) + 1,):
            raise ValueError("zfaces must hold nz + 1 values")
        g.zfaces = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if yfaces is not None:
        ykeep = np.ascontiguousarray(yfaces, dtype=np.float64)
        if ykeep.shape != (int(ny) + 1,):
            raise ValueError("yfaces must hold ny + 1 values")
        g.yfaces = ykeep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g.bc[0], g.bc[1], g.bc[2] = PP_BC_PERIODIC, PP_BC_WALL if ywalls else PP_BC_PERIODIC, PP_BC_WALL
    out = ctypes.c_void_p()
    _check(lib().pressure_plan_create(ctypes.byref(g), PRECISIONS[precision], _stream(stream),
                                      ctypes.byref(out)), "pressure_plan_create")
    _PLAN_SIZES[out.value] = (g.nx * g.ny * g.nz, g.nx * g.ny * (g.nz + 1))
    return out.value


def _grid(nx, ny, nz, lx, ly, lz, zfaces, ywalls=False):
    g = pp_grid()
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    g.lx, g.ly, g.lz = float(lx), float(ly), float(lz)
    keep = None
    if zfaces is not None:
        keep = np.ascontiguousarray(zfaces, dtype=np.float64)
        if keep.shape != (int(nz) + 1,):
            raise ValueError("zfaces must hold nz + 1 values")
        g.zfaces = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g.bc[0], g.bc[1], g.bc[2] = PP_BC_PERIODIC, PP_BC_WALL if ywalls else PP_BC_PERIODIC, PP_BC_WALL
    return g, keep


def pressure_solve_noalloc(nx, ny, nz, lx, ly, lz, f, p, zfaces=None, stream=None, ywalls=False):
    """FP64 constant-coefficient solve that allocates no device memory (see
    the header).  f, p: CUDA float64 tensors.  ``ywalls``: walls at y = 0 and
    y = ly.  Returns after enqueueing."""
    g, keep = _grid(nx, ny, nz, lx, ly, lz, zfaces, ywalls)
    n = int(nx) * int(ny) * int(nz)
    for x in (f, p):
        got = x.size if isinstance(x, np.ndarray) else getattr(x, "numel", lambda: None)()
        if got is not None and got < n:
            raise ValueError(f"a cell field needs {n} elements, got {got}")
    _check(lib().pressure_solve_noalloc(ctypes.byref(g), _ptr(f), _ptr(p), _stream(stream)),
           "pressure_solve_noalloc")
    del keep


def pressure_plan_destroy(plan):
    _PLAN_SIZES.pop(plan, None)
    _check(lib().pressure_plan_destroy(plan), "pressure_plan_destroy")


ZSOLVES = {"tridiag": 0, "cosine": 1}


def pressure_plan_set_zsolve(plan, zsolve):
    """zsolve: "tridiag" (default) or "cosine" (uniform z, FP64 plans)."""
    code = ZSOLVES[zsolve] if isinstance(zsolve, str) else int(zsolve)
    _check(lib().pressure_plan_set_zsolve(plan, code), "pressure_plan_set_zsolve")


def pressure_plan_set_method(plan, method):
    """method: "III" (default), "I" or "II" (or the pp_method integer)."""
    code = METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().pressure_plan_set_method(plan, code), "pressure_plan_set_method")


def pressure_solve(plan, f, p):
    _sized(plan, (f, "c"), (p, "c"))
    info = pp_info()
    _check(lib().pressure_solve(plan, _ptr(f), _ptr(p), ctypes.byref(info)), "pressure_solve")
    return info.as_dict()


def pressure_mixture_density(plan, phi, rho_g, rho_l, rho):
    _sized(plan, (phi, "c"), (rho, "c"))
    _check(lib().pressure_mixture_density(plan, _ptr(phi), float(rho_g), float(rho_l), _ptr(rho)),
           "pressure_mixture_density")


def pressure_correct(plan, us, vs, ws, rho, S, dt, p, u, v, w, rtol=1e-10, maxit=500,
                     warm_start=False, sync=True, allow_not_converged=False):
    """Method III projection.  With ``sync=False`` the call only enqueues the
    work (read the status later with ``pressure_last_info``)."""
    _sized(plan, (us, "c"), (vs, "c"), (ws, "w"), (rho, "c"), (S, "c"), (p, "c"), (u, "c"), (v, "c"), (w, "w"))
    info = pp_info()
    code = lib().pressure_correct(plan, _ptr(us), _ptr(vs), _ptr(ws), _ptr(rho), _ptr(S),
                                  float(dt), _ptr(p), int(bool(warm_start)), _ptr(u), _ptr(v),
                                  _ptr(w), float(rtol), int(maxit),
                                  ctypes.byref(info) if sync else None)
    allow = (PP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(code, "pressure_correct", allow)
    return info.as_dict() if sync else None


def pressure_p0_rate(plan, phi, kc, T, u, v, w, p0, gamma):
    """Eq. 30: the rate of the thermodynamic pressure (host float)."""
    _sized(plan, (phi, "c"), (kc, "c"), (T, "c"), (u, "c"), (v, "c"), (w, "w"))
    out = ctypes.c_double()
    _check(lib().pressure_p0_rate(plan, _ptr(phi), _ptr(kc), _ptr(T), _ptr(u), _ptr(v), _ptr(w), float(p0),
                                  float(gamma), ctypes.byref(out)), "pressure_p0_rate")
    return out.value


def pressure_dp0dt_extrapolate(rp_n, rp_nm1, dt_new, dt_old):
    out = ctypes.c_double()
    _check(lib().pressure_dp0dt_extrapolate(float(rp_n), float(rp_nm1), float(dt_new), float(dt_old),
                                            ctypes.byref(out)), "pressure_dp0dt_extrapolate")
    return out.value


def pressure_divergence_source(plan, phi, kc, T, p0, gamma, dp0dt, S):
    """Eq. 34: the divergence source S written into S (cell field)."""
    _sized(plan, (phi, "c"), (kc, "c"), (T, "c"), (S, "c"))
    _check(lib().pressure_divergence_source(plan, _ptr(phi), _ptr(kc), _ptr(T), float(p0), float(gamma),
                                            float(dp0dt), _ptr(S)), "pressure_divergence_source")


def pressure_predictor(plan, u, v, w, rho, mu, gravity, dt_new, u_star, dt_old=0.0, ru_prev=None,
                       ru_out=None, force=None):
    """Eqs. 29, 32: u_star = (u*, v*, w*) written in place; ru_out receives
    RU^n; ru_prev = RU^{n-1} (None: forward Euler).  Device tensors only."""
    _sized(plan, (u, "c"), (v, "c"), (w, "w"), (rho, "c"), (mu, "c"))
    for ts in (force, ru_prev, u_star, ru_out):
        if ts is not None:
            _sized(plan, *zip(ts, ("c", "c", "w")))
    trio = lambda ts: None if ts is None else (ctypes.c_void_p * 3)(*[_ptr(t) for t in ts])  # noqa: E731
    grav = (ctypes.c_double * 3)(*[float(x) for x in gravity])
    _check(lib().pressure_predictor(plan, _ptr(u), _ptr(v), _ptr(w), _ptr(rho), _ptr(mu), trio(force), grav,
                                    float(dt_new), float(dt_old), trio(ru_prev), trio(u_star), trio(ru_out)),
           "pressure_predictor")


def pressure_last_info(plan):
    info = pp_info()
    lib().pressure_last_info(plan, ctypes.byref(info))
    return info.as_dict()


def pressure_solve_adjoint(plan, rho, p, dt, gu, gv, gw, gus, gvs, gws, grho, rtol=1e-10, maxit=500,
                           allow_not_converged=False):
    _sized(plan, (rho, "c"), (p, "c"), (gu, "c"), (gv, "c"), (gw, "w"), (gus, "c"), (gvs, "c"), (gws, "w"),
           (grho, "c"))
    info = pp_info()
    code = lib().pressure_solve_adjoint(plan, _ptr(rho), _ptr(p), float(dt), _ptr(gu), _ptr(gv),
                                        _ptr(gw), _ptr(gus), _ptr(gvs), _ptr(gws), _ptr(grho),
                                        float(rtol), int(maxit), ctypes.byref(info))
    _check(code, "pressure_solve_adjoint", (PP_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return info.as_dict()


def pressure_profile_enable(plan, enable=True):
    _check(lib().pressure_profile_enable(plan, int(bool(enable))), "pressure_profile_enable")


def pressure_profile_read(plan):
    """Returns ({kernel: (launches, total_ms)}, total_launches)."""
    n = ctypes.c_int()
    tot = ctypes.c_longlong()
    _check(lib().pressure_profile_read(plan, None, 0, ctypes.byref(n), ctypes.byref(tot)),
           "pressure_profile_read")
    arr = (pp_kernel_time * max(n.value, 1))()
    _check(lib().pressure_profile_read(plan, arr, n.value, ctypes.byref(n), ctypes.byref(tot)),
           "pressure_profile_read")
    return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(n.value)}, tot.value


class Batch:
    """Batched projections of independent grids (packed field buffers).

    ``grids``: list of dicts with nx, ny, nz, lx, ly, lz and optional zfaces
    and ywalls (walls at y = 0 and y = ly).
    """

    def __init__(self, grids, precision="mixed", stream=None):
        self.n = len(grids)
        arr = (pp_grid * self.n)()
        self._keep = []
        for k, gd in enumerate(grids):
            g, keep = _grid(gd["nx"], gd["ny"], gd["nz"], gd["lx"], gd["ly"], gd["lz"], gd.get("zfaces"),
                            bool(gd.get("ywalls", False)))
            arr[k] = g
            self._keep.append(keep)
        out = ctypes.c_void_p()
        _check(lib().pressure_batch_create(arr, self.n, PRECISIONS[precision], _stream(stream),
                                           ctypes.byref(out)), "pressure_batch_create")
        self.handle = out.value
        co = (ctypes.c_longlong * self.n)()
        wo = (ctypes.c_longlong * self.n)()
        tot = (ctypes.c_longlong * 2)()
        tiles = (ctypes.c_int * 2)()
        _check(lib().pressure_batch_layout(self.handle, co, wo, tot, tiles), "pressure_batch_layout")
        self.cell_offset = list(co)
        self.wface_offset = list(wo)
        self.ncell, self.nwface = tot[0], tot[1]
        self.tiles = (tiles[0], tiles[1])
        _PLAN_SIZES[self.handle] = (self.ncell, self.nwface)   # packed buffers are checked like a plan's

    def mixture_density(self, phi, rho_g, rho_l, rho):
        _sized(self.handle, (phi, "c"), (rho, "c"))
        _check(lib().pressure_batch_mixture_density(self.handle, _ptr(phi), float(rho_g), float(rho_l),
                                                    _ptr(rho)), "pressure_batch_mixture_density")

    def correct(self, us, vs, ws, rho, S, dt, p, u, v, w, rtol=1e-10, maxit=500,
                allow_not_converged=False):
        _sized(self.handle, (us, "c"), (vs, "c"), (ws, "w"), (rho, "c"), (S, "c"), (p, "c"), (u, "c"),
               (v, "c"), (w, "w"))
        infos = (pp_info * self.n)()
        code = lib().pressure_batch_correct(self.handle, _ptr(us), _ptr(vs), _ptr(ws), _ptr(rho), _ptr(S),
                                            float(dt), _ptr(p), _ptr(u), _ptr(v), _ptr(w), float(rtol),
                                            int(maxit), infos)
        _check(code, "pressure_batch_correct", (PP_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return [infos[k].as_dict() for k in range(self.n)]

    def close(self):
        if getattr(self, "handle", None):
            _PLAN_SIZES.pop(self.handle, None)
            _check(lib().pressure_batch_destroy(self.handle), "pressure_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper of a plan handle."""

    def __init__(self, nx, ny, nz, lx, ly, lz, zfaces=None, precision="fp64", stream=None,
                 method="III", ywalls=False, zsolve="tridiag", yfaces=None):
        self.shape = (int(nz), int(ny), int(nx))
        self.wshape = (int(nz) + 1, int(ny), int(nx))
        self.handle = pressure_plan_create(nx, ny, nz, lx, ly, lz, zfaces, precision, stream, ywalls, yfaces)
        if method != "III":
            pressure_plan_set_method(self.handle, method)
        if zsolve != "tridiag":
            pressure_plan_set_zsolve(self.handle, zsolve)

    def close(self):
        if getattr(self, "handle", None):
            pressure_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
