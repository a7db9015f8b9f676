"""Host-side checks of the C ABI (no GPU): the shared library loads and
exports every function include/pressure_projection.h declares."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pressure_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    assert {"pressure_plan_create", "pressure_solve", "pressure_correct",
            "pressure_solve_adjoint"} <= _declared()


def test_library_exports_every_declared_symbol():
    from paper_2005_11806_gb300 import pressure
    if not os.path.exists(pressure.LIB_PATH):
        from paper_2005_11806_gb300 import build_ext
        build_ext.build()
    L = pressure.lib()
    for name in sorted(_declared()):
        assert hasattr(L, name), name
    assert set(pressure.EXPORTS) >= _declared()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2005_11806_gb300 import pressure
    monkeypatch.setattr(pressure, "_lib", None)
    monkeypatch.setattr(pressure, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pressure.lib()


def _lib_or_build():
    from paper_2005_11806_gb300 import pressure
    if not os.path.exists(pressure.LIB_PATH):
        from paper_2005_11806_gb300 import build_ext
        build_ext.build()
    return pressure


@pytest.mark.parametrize("dims,lens,prec,bc,code", [
    ((0, 8, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),      # empty grid
    ((8, 8, 0), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),
    ((8, 0, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),
    ((-2, 8, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),     # negative size
    ((8, 8, 8), (1, -1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),     # negative length
    ((8, 8, 8), (0, 1, 1), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),      # zero length
    ((8, 8, 8), (1, 1, 0), "fp64", (0, 0, 1), "PP_ERR_INVALID_ARG"),
    ((7, 8, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_UNSUPPORTED"),      # odd nx (two real rows per complex FFT)
    ((8, 7, 8), (1, 1, 1), "fp64", (0, 1, 1), "PP_ERR_UNSUPPORTED"),      # odd ny with walls in y
    ((8, 8, 8), (1, 1, 1), "fp64", (1, 0, 1), "PP_ERR_UNSUPPORTED"),      # walls in x
    ((8, 8, 8), (1, 1, 1), "fp64", (0, 0, 0), "PP_ERR_UNSUPPORTED"),      # periodic z
    ((4096, 8, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_UNSUPPORTED"),   # longer than one FFT block
    ((14, 8, 8), (1, 1, 1), "fp64", (0, 0, 1), "PP_ERR_UNSUPPORTED"),     # prime factor 7
    ((8, 8, 1024), (1, 1, 1), "mixed_tc", (0, 0, 1), "PP_ERR_UNSUPPORTED"),  # tensor-core z beyond 512
])
def test_plan_create_rejects_bad_descriptors(dims, lens, prec, bc, code):
    """Descriptor checks come before any CUDA call, so they run here."""
    import ctypes
    pressure = _lib_or_build()
    g = pressure.pp_grid()
    g.nx, g.ny, g.nz = dims
    g.lx, g.ly, g.lz = lens
    g.bc[0], g.bc[1], g.bc[2] = bc
    out = ctypes.c_void_p()
    got = pressure.lib().pressure_plan_create(ctypes.byref(g), pressure.PRECISIONS[prec], None, ctypes.byref(out))
    assert got == getattr(pressure, code)
    assert out.value is None


@pytest.mark.parametrize("ny,bc,faces,code", [
    (8, (0, 0, 1), "tanh", "PP_ERR_UNSUPPORTED"),     # stretched y needs walls in y
    (1025, (0, 1, 1), "tanh", "PP_ERR_UNSUPPORTED"),  # dense y step: ny <= 1024
    (8, (0, 1, 1), "flat", "PP_ERR_INVALID_ARG"),     # faces not increasing
    (8, (0, 1, 1), "short", "PP_ERR_INVALID_ARG"),    # faces do not span ly
])
def test_plan_create_rejects_bad_y_faces(ny, bc, faces, code):
    """The stretched-y descriptor checks also precede any CUDA call."""
    import ctypes
    import math
    pressure = _lib_or_build()
    yf = np.array([0.5 * (1 + math.tanh(1.5 * (2 * j / ny - 1)) / math.tanh(1.5)) for j in range(ny + 1)])
    if faces == "flat":
        yf[3] = yf[2]
    if faces == "short":
        yf = yf * 0.9
    g = pressure.pp_grid()
    g.nx, g.ny, g.nz = 8, ny, 8
    g.lx, g.ly, g.lz = 1.0, 1.0, 1.0
    g.bc[0], g.bc[1], g.bc[2] = bc
    keep = np.ascontiguousarray(yf)
    g.yfaces = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = ctypes.c_void_p()
    got = pressure.lib().pressure_plan_create(ctypes.byref(g), pressure.PRECISIONS["fp64"], None, ctypes.byref(out))
    assert got == getattr(pressure, code)
    assert out.value is None


def test_host_only_entry_points():
    pressure = _lib_or_build()
    # dp0/dt at t^{n+1} from two rates, linear in time (Sec. 3.3)
    assert pressure.pressure_dp0dt_extrapolate(2.0, 1.0, 1e-3, 2e-3) == pytest.approx(2.5)
    with pytest.raises(pressure.PressureError) as e:
        pressure.pressure_dp0dt_extrapolate(2.0, 1.0, 1e-3, 0.0)
    assert e.value.code == pressure.PP_ERR_INVALID_ARG
    assert pressure.status_string(pressure.PP_OK)
    assert pressure.status_string(pressure.PP_ERR_UNSUPPORTED) != pressure.status_string(pressure.PP_OK)


@pytest.mark.parametrize("dims,bc,code", [
    ((4096, 2, 1), (0, 0, 1), "PP_ERR_UNSUPPORTED"),   # one x line per FFT block: nx <= 2048
    ((2, 4096, 1), (0, 0, 1), "PP_ERR_UNSUPPORTED"),   # one y line per FFT block: ny <= 2048
    ((7, 4, 3), (0, 0, 1), "PP_ERR_UNSUPPORTED"),      # odd nx
    ((14, 4, 3), (0, 0, 1), "PP_ERR_UNSUPPORTED"),     # prime factor 7
    ((8, 7, 8), (0, 1, 1), "PP_ERR_UNSUPPORTED"),      # walls in y need an even ny
    ((8, 8, 8), (1, 1, 1), "PP_ERR_UNSUPPORTED"),      # walls in x
    ((0, 8, 8), (0, 0, 1), "PP_ERR_INVALID_ARG"),      # empty grid
])
def test_noalloc_rejects_bad_descriptors_before_any_cuda_call(dims, bc, code):
    """The allocation-free solve checks the grid before it touches the
    device, so these run without a GPU (the field pointers are never used)."""
    import ctypes
    pressure = _lib_or_build()
    g = pressure.pp_grid()
    g.nx, g.ny, g.nz = dims
    g.lx, g.ly, g.lz = 1.0, 1.0, 1.0
    g.bc[0], g.bc[1], g.bc[2] = bc
    buf = (ctypes.c_double * 8)()
    got = pressure.lib().pressure_solve_noalloc(ctypes.byref(g), ctypes.cast(buf, ctypes.c_void_p),
                                                ctypes.cast(buf, ctypes.c_void_p), None)
    assert got == getattr(pressure, code)


@pytest.mark.parametrize("dims,bc,yfaces,code", [
    ((8, 7, 8), (0, 1, 1), False, "PP_ERR_UNSUPPORTED"),   # walls in y need an even ny
    ((8, 8, 8), (1, 0, 1), False, "PP_ERR_UNSUPPORTED"),   # walls in x
    ((8, 8, 8), (0, 1, 1), True, "PP_ERR_UNSUPPORTED"),    # a stretched y is single-plan only
    ((8, 0, 8), (0, 0, 1), False, "PP_ERR_INVALID_ARG"),   # empty grid
])
def test_batch_rejects_bad_descriptors_before_any_cuda_call(dims, bc, yfaces, code):
    """pressure_batch_create checks every grid before it allocates."""
    import ctypes
    pressure = _lib_or_build()
    g = pressure.pp_grid()
    g.nx, g.ny, g.nz = dims
    g.lx, g.ly, g.lz = 1.0, 1.0, 1.0
    g.bc[0], g.bc[1], g.bc[2] = bc
    keep = np.linspace(0.0, 1.0, dims[1] + 1)
    if yfaces:
        g.yfaces = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    arr = (pressure.pp_grid * 1)(g)
    out = ctypes.c_void_p()
    got = pressure.lib().pressure_batch_create(arr, 1, pressure.PRECISIONS["mixed"], None, ctypes.byref(out))
    assert got == getattr(pressure, code)
    assert out.value is None


@pytest.mark.parametrize("faces", ["flat", "reversed", "nan", "inf"])
@pytest.mark.parametrize("entry", ["plan", "batch", "noalloc"])
def test_bad_z_faces_rejected_before_any_cuda_call(entry, faces):
    """z faces that are not finite and strictly increasing (the Sec. 3 grid
    needs positive cell widths dzf) are refused by every entry point that
    takes a grid, before it touches the device."""
    import ctypes
    pressure = _lib_or_build()
    zf = np.linspace(0.0, 1.0, 9)
    if faces == "flat":
        zf[3] = zf[2]
    elif faces == "reversed":
        zf = zf[::-1].copy()
    elif faces == "nan":
        zf[4] = np.nan
    else:
        zf[0] = -np.inf
    keep = np.ascontiguousarray(zf)
    g = pressure.pp_grid()
    g.nx, g.ny, g.nz = 8, 8, 8
    g.lx, g.ly, g.lz = 1.0, 1.0, 1.0
    g.bc[0], g.bc[1], g.bc[2] = 0, 0, 1
    g.zfaces = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = ctypes.c_void_p()
    L = pressure.lib()
    if entry == "plan":
        got = L.pressure_plan_create(ctypes.byref(g), pressure.PRECISIONS["fp64"], None, ctypes.byref(out))
    elif entry == "batch":
        arr = (pressure.pp_grid * 1)(g)
        got = L.pressure_batch_create(arr, 1, pressure.PRECISIONS["mixed"], None, ctypes.byref(out))
    else:
        buf = (ctypes.c_double * 8)()
        got = L.pressure_solve_noalloc(ctypes.byref(g), ctypes.cast(buf, ctypes.c_void_p),
                                       ctypes.cast(buf, ctypes.c_void_p), None)
    assert got == pressure.PP_ERR_INVALID_ARG
    assert out.value is None
