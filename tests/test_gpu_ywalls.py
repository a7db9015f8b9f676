"""Walls in y on the GPU (the cosine eigenbasis of the Neumann y difference,
through one complex FFT per column), through the C ABI, against the oracle.

Tolerances as for periodic y: FP64 paths match the oracle to a relative L2
error of 1e-11; mixed paths reach a relative residual <= 1e-10 (re-evaluated
by the oracle in FP64) and match the oracle's converged fields within 1e-9."""
import functools
import math

import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl
from tests.fp32_bounds import mixed_solve_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="module")
def pp():
    from paper_2005_11806_gb300 import pressure
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    pressure.lib()
    return pressure


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _plan(pp, g, precision="fp64", method="III"):
    return pp.Plan(g.nx, g.ny, g.nz, g.lx, g.ly, float(g.zf[-1] - g.zf[0]), zfaces=g.zf,
                   precision=precision, method=method, ywalls=True)


def _grid(w):
    return orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=True)


# --- constant-coefficient solve -------------------------------------------

@pytest.mark.parametrize("dims,stretch,precision", [
    ((32, 32, 32), None, "fp64"),
    ((24, 20, 17), 1.5, "fp64"),      # radix 5 in y, odd nz, stretched z
    ((16, 2, 8), None, "fp64"),       # the smallest walled y: two rows
    ((96, 30, 9), 2.0, "fp64"),       # ny = 30: radices 2, 3, 5
    ((64, 48, 40), 1.5, "mixed"),
    ((64, 48, 40), 1.5, "mixed_z64"),
])
def test_ywalls_constant_solve_vs_oracle(pp, dims, stretch, precision):
    nx, ny, nz = dims
    zf = wl.uniform_zfaces(nz, 1.2) if stretch is None else wl.tanh_zfaces(nz, 1.2, stretch)
    g = orc.Grid(nx, ny, nz, 1.0, 0.75, zf, ywalls=True)
    f = np.random.default_rng(nx * 5 + ny).standard_normal(g.shape)
    plan = _plan(pp, g, precision)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    # mixed plans: the FP32 rounding bound of one solve (tests/fp32_bounds.py)
    tol = FP64_TOL if precision == "fp64" else mixed_solve_bound(nx, ny, ywalls=True)
    err = _rel(host(p), orc.solve_constant(g, f))
    print(f"walled-y constant solve {dims} {precision}: rel. L2 error {err:.3e}, bound {tol:.3e}")
    assert err < tol


def test_ywalls_single_mode_closed_form_gpu(pp):
    """cos(2 pi a i/nx) cos(pi b (j + 1/2)/ny) cos(pi c (k + 1/2)/nz) is an
    eigenvector of the walled operator: p = f / lambda, no oracle involved."""
    nx, ny, nz, lx, ly, lz = 32, 24, 20, 1.0, 1.3, 0.6
    g = orc.Grid(nx, ny, nz, lx, ly, wl.uniform_zfaces(nz, lz), ywalls=True)
    a, b, c = 3, 5, 2
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    f = np.cos(2 * np.pi * a * i / nx + 0.4) * np.cos(np.pi * b * (j + 0.5) / ny) * np.cos(np.pi * c * (k + 0.5) / nz)
    lam = -(4 * (nx / lx) ** 2 * math.sin(math.pi * a / nx) ** 2
            + 4 * (ny / ly) ** 2 * math.sin(math.pi * b / (2 * ny)) ** 2
            + 4 * (nz / lz) ** 2 * math.sin(math.pi * c / (2 * nz)) ** 2)
    plan = _plan(pp, g)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    assert _rel(host(p), f / lam) < FP64_TOL


# --- variable-density projection ------------------------------------------

def _case(n, ny=None, nz=None, stretched=False, ratio=1000.0, seed=1202):
    w = wl.channel_bubble_case(n, ny, nz, seed=seed, rho_ratio=ratio, stretched=stretched)
    return w, orc.mixture_density(w.phi, w.rho_g, w.rho_l)


def _run(pp, w, rho, precision="fp64", rtol=1e-13, maxit=400, method="III", host_ptrs=False):
    plan = _plan(pp, _grid(w), precision, method)
    allow = rtol == 0.0
    if host_ptrs:
        p, u, v = (np.empty(w.shape) for _ in range(3))
        ww = np.empty((w.nz + 1, w.ny, w.nx))
        info = pp.pressure_correct(plan.handle, w.us, w.vs, w.ws, rho, w.S, w.dt, p, u, v, ww,
                                   rtol=rtol, maxit=maxit, allow_not_converged=allow)
        return info, p, u, v, ww
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=rtol, maxit=maxit, allow_not_converged=allow)
    return info, host(p), host(u), host(v), host(ww)


@pytest.mark.parametrize("dims,stretched,ratio,passes", [
    ((32, None, None), False, 1000.0, 40),
    ((24, 20, 18), True, 100.0, 30),
    ((40, 30, 25), True, 1000.0, 25),
])
def test_ywalls_iterates_vs_oracle(pp, dims, stretched, ratio, passes):
    """Algorithm 1 stopped after a fixed number of passes: the GPU iterate
    equals the oracle's (same s) to round-off, and the wall row of v is 0."""
    n, ny, nz = dims
    w, rho = _case(n, ny, nz, stretched, ratio)
    g = _grid(w)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    info, p, u, v, ww = _run(pp, w, rho, rtol=0.0, maxit=passes)
    assert info["iters"] == passes
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    assert _rel(p, p0) < FP64_TOL
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL
    assert np.all(v[:, 0, :] == 0.0)


def test_ywalls_converged_fp64_meets_the_divergence_target(pp):
    w, rho = _case(32, 24, 20, stretched=True)
    g = _grid(w)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-12, maxit=5000)
    info, p, u, v, ww = _run(pp, w, rho, rtol=1e-12, maxit=5000)
    assert info["status"] == 0 and info["res_final"] <= 1e-12
    assert abs(info["iters"] - oinfo["iters"]) <= 1
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-12 * np.linalg.norm(d0)


@functools.lru_cache(maxsize=1)
def _mixed_reference():
    """The oracle's converged projection of the 48 x 40 x 40 duct (3659
    passes to 1e-13; computed once for the three mixed plans)."""
    w, rho = _case(48, 40, 40, stretched=True)
    g = _grid(w)
    return w, rho, orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=6000)


@pytest.mark.parametrize("precision", ["mixed", "mixed_z64", "mixed_tc"])
def test_ywalls_mixed_vs_oracle(pp, precision):
    """Mixed precision with walls in y: residual <= 1e-10 in FP64, fields
    within 1e-9 of the oracle's converged projection."""
    w, rho, (p0, u0, v0, w0, _) = _mixed_reference()
    g = _grid(w)
    info, p, u, v, ww = _run(pp, w, rho, precision, rtol=1e-10, maxit=6000)
    assert info["status"] == 0 and info["res_final"] <= 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1e-10 * np.linalg.norm(d0) * 1.0001
    errs = [_rel(a, b) for a, b in ((u, u0), (v, v0), (ww, w0))]
    print(precision, "walled y vs oracle", errs, "iters", info["iters"])
    assert max(errs) < 1e-9
    assert np.all(v[:, 0, :] == 0.0)


@pytest.mark.parametrize("method", ["I", "II"])
def test_ywalls_methods_1_2_vs_oracle(pp, method):
    w, rho = _case(24, 20, 18, stretched=True, ratio=10.0)
    g = _grid(w)
    fn = orc.method1 if method == "I" else orc.method2
    passes = 20
    p0, u0, v0, w0, _ = fn(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    info, p, u, v, ww = _run(pp, w, rho, rtol=0.0, maxit=passes, method=method)
    assert info["iters"] == passes
    for a, b in ((p, p0), (u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL


def test_ywalls_host_pointers_and_wall_input_ignored(pp):
    """Host buffers give the device result; a nonzero wall row of v* is read
    as zero, as the oracle's D reads it."""
    w, rho = _case(16, 12, 10)
    a = _run(pp, w, rho, rtol=1e-11, maxit=2000)
    b = _run(pp, w, rho, rtol=1e-11, maxit=2000, host_ptrs=True)
    assert a[0]["iters"] == b[0]["iters"]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    w.vs[:, 0, :] = 0.3
    c = _run(pp, w, rho, rtol=1e-11, maxit=2000)
    for x, y in zip(a[1:], c[1:]):
        assert np.array_equal(x, y)


def test_ywalls_odd_ny_is_refused(pp):
    with pytest.raises(pp.PressureError) as e:
        pp.Plan(16, 9, 8, 1.0, 1.0, 1.0, ywalls=True)   # odd ny: the cosine transform by an even FFT
    assert e.value.code == pp.PP_ERR_UNSUPPORTED


def _adjoint_case():
    """12 x 8 x 10 duct, stretched z, 3 bubbles at ratio 100, a converged
    forward pressure and the gradient of ||u^{n+1} - target||^2."""
    w, rho = _case(12, 8, 10, stretched=True, seed=1211, ratio=100.0)
    g = _grid(w)
    p0, u, v, ww = orc.projection_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt)
    rng = np.random.default_rng(1211 + 20)
    gu = 2 * (u - 0.1 * rng.standard_normal(w.shape))
    gv = 2 * (v - 0.1 * rng.standard_normal(w.shape))
    gw = 2 * (ww - 0.1 * rng.standard_normal(ww.shape))
    gv[:, 0, :] = 0.7   # on the wall row: must be ignored
    return w, rho, g, p0, gu, gv, gw


def _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, rtol, maxit):
    g = _grid(w)
    plan = _plan(pp, g)
    out = [torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    out.append(torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda"))
    grho = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    info = pp.pressure_solve_adjoint(plan.handle, dev(rho), dev(p0), w.dt, dev(gu), dev(gv), dev(gw),
                                     out[0], out[1], out[2], grho, rtol=rtol, maxit=maxit,
                                     allow_not_converged=(rtol == 0.0))
    plan.close()
    return info, [host(x) for x in (*out, grho)]


def test_ywalls_adjoint_iterates_vs_oracle(pp):
    """Walls in y: the transposed solve stopped after 40 passes on both sides
    (Algorithm 1 on the adjoint system) gives the oracle's gradients to
    round-off; the wall row of the upstream v gradient is ignored."""
    w, rho, g, p0, gu, gv, gw = _adjoint_case()
    ref = orc.adjoint_method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw, rtol=0.0, maxit=40, p=p0)
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 0.0, 40)
    assert info["iters"] == 40
    for a, b in zip(got, ref[:4]):
        assert _rel(a, b) < FP64_TOL
    assert np.all(got[1][:, 0, :] == 0.0)


def test_ywalls_adjoint_converged_vs_direct(pp):
    """Walls in y: the converged adjoint against the oracle's literal
    sparse-transpose gradient (itself pinned by central differences)."""
    w, rho, g, p0, gu, gv, gw = _adjoint_case()
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 1e-12, 5000)
    assert info["status"] == 0
    ref = orc.adjoint_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw)
    errs = [_rel(a, b) for a, b in zip(got, ref)]
    print("walled-y adjoint vs direct", errs, "iters", info["iters"])
    assert max(errs) < 1e-8


@pytest.mark.slow
def test_ywalls_fullsize_duct256_iterates(pp):
    """256^3 duct (walls in y and z, ratio 1000): three FP64 passes against
    the oracle's three passes at every cell, and the mixed path's converged
    field meets the divergence target in FP64."""
    w, rho = _case(256, stretched=True, seed=1203)
    g = _grid(w)
    p0, u0, v0, w0, _ = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=3)
    info, p, u, v, ww = _run(pp, w, rho, rtol=0.0, maxit=3)
    for a, b in ((p, p0), (u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL
    info, p, u, v, ww = _run(pp, w, rho, "mixed", rtol=1e-10, maxit=20000)
    assert info["status"] == 0
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1e-10 * np.linalg.norm(d0) * 1.0001
    assert np.all(v[:, 0, :] == 0.0)
