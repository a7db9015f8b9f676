"""Methods I and II of Sec. 3.3.1 (Eqs. poisson_me1/poisson_me2 and
poisson_laizet) on the GPU, through the C ABI, against the oracle's literal
forms of the two equations; and the pass counts of the three methods on the
same frozen bubble field (the comparison of the rising-bubble figure in
Sec. 4, on a synthetic field)."""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
ORACLE = {"I": orc.method1, "II": orc.method2, "III": orc.method3}


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


def _bubbles(n, ratio, stretched=False, nz=None, ny=None, seed=1102):
    w = wl.small_bubble_case(n, seed=seed, rho_ratio=ratio, stretched=stretched, nz=nz, ny=ny)
    return w, orc.mixture_density(w.phi, w.rho_g, w.rho_l)


def _sphere(n, ratio):
    zf = wl.uniform_zfaces(n, 1.0)
    phi = wl.spheres_phi(n, n, n, 1.0, 1.0, zf, [(0.5, 0.5, 0.3, 0.15)])
    us, vs, ws = wl.random_faces(n, n, n, 0.1, 1002)
    w = wl.Workload(f"sphere {n}", n, n, n, 1.0, 1.0, zf, 1e-3, us, vs, ws, phi, 1.0, ratio,
                    wl.gas_source(phi))
    return w, orc.mixture_density(phi, 1.0, ratio)


def _gpu(pp, w, rho, method, precision="fp64", rtol=0.0, maxit=100):
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf,
                   precision=precision, method=method)
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u = torch.empty_like(p); v = torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=rtol, maxit=maxit, allow_not_converged=(rtol == 0.0))
    return info, host(p), host(u), host(v), host(ww)


@pytest.mark.parametrize("method,stretched,ratio,dims,passes", [
    ("I", False, 10.0, (32, None, None), 30),
    ("I", True, 100.0, (24, 20, 18), 25),     # ragged: radix 3/5 in x/y, stretched z
    ("II", False, 1000.0, (32, None, None), 30),
    ("II", True, 10.0, (40, 30, 25), 20),
])
def test_method_iterates_vs_oracle(pp, method, stretched, ratio, dims, passes):
    """After a fixed number of passes the GPU iterate and the corrected
    velocity (Method I: Eq. poisson_me2 with the second-to-last iterate)
    equal the oracle's to round-off.  The GPU runs the defect form
    p += L^-1 [r~ (D u^s - S_c)/dt], the oracle the equations as printed."""
    n, ny, nz = dims
    w, rho = _bubbles(n, ratio, stretched, nz=nz, ny=ny)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, oinfo = ORACLE[method](g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    info, p, u, v, ww = _gpu(pp, w, rho, method, rtol=0.0, maxit=passes)
    assert info["iters"] == passes
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    assert _rel(p, p0) < FP64_TOL
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL


def test_pass_counts_of_the_three_methods(pp):
    """Same frozen field (one gas sphere, ratio 10), relative residual 1e-10:
    the GPU needs the oracle's pass count for every method, and Method III
    needs fewer passes than II, which needs fewer than I (Sec. 4)."""
    w, rho = _sphere(32, 10.0)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    iters = {}
    for m in ("I", "II", "III"):
        *_, oinfo = ORACLE[m](g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-10, maxit=5000)
        info, *_ = _gpu(pp, w, rho, m, rtol=1e-10, maxit=5000)
        assert info["status"] == 0 and info["res_final"] <= 1e-10
        assert abs(info["iters"] - oinfo["iters"]) <= 1, (m, info["iters"], oinfo["iters"])
        iters[m] = info["iters"]
    print("passes to 1e-10:", iters)
    assert iters["III"] < iters["II"] < iters["I"]


@pytest.mark.parametrize("method,precision", [("I", "mixed"), ("II", "mixed"), ("II", "mixed_tc")])
def test_method_mixed_converged_vs_oracle(pp, method, precision):
    """Mixed precision with the FP64 residual reaches 1e-10 under Methods I and
    II too, and matches the oracle's converged velocity."""
    w, rho = _sphere(32, 10.0)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, _ = ORACLE[method](g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=5000)
    info, p, u, v, ww = _gpu(pp, w, rho, method, precision, rtol=1e-10, maxit=5000)
    assert info["status"] == 0 and info["res_final"] <= 1e-10
    errs = [_rel(a, b) for a, b in ((u, u0), (v, v0), (ww, w0))]
    assert max(errs) < 1e-8, errs


def test_set_method_rejects_unknown(pp):
    plan = pp.Plan(8, 8, 8, 1.0, 1.0, 1.0)
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_plan_set_method(plan.handle, 7)
    assert e.value.code == pp.PP_ERR_INVALID_ARG
    pp.pressure_plan_set_method(plan.handle, "II")
    pp.pressure_plan_set_method(plan.handle, "III")
