"""A stretched y between walls on the GPU (the y step as dense products with
the W-orthonormal eigenbasis computed at plan creation), through the C ABI,
against the oracle (whose eigenbasis comes from scipy's generalized
symmetric eigensolver, not from the library's Sturm bisection).

Tolerances: FP64 paths match the oracle to a relative L2 error of 1e-11;
mixed paths reach a relative residual <= 1e-10 (re-evaluated by the oracle
in FP64) and match the oracle's converged fields within 1e-9.  One mixed
constant solve is held to the FP32 rounding bound of its arithmetic
(tests/fp32_bounds.py, with the dense y products)."""
import functools

import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl
from tests.fp32_bounds import mixed_solve_bound_dense_y

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


_GRID = object()


def _plan(pp, g, precision="fp64", method="III", yfaces=_GRID):
    yf = g.yf if yfaces is _GRID else yfaces
    return pp.Plan(g.nx, g.ny, g.nz, g.lx, g.ly, float(g.zf[-1] - g.zf[0]), zfaces=g.zf,
                   precision=precision, method=method, ywalls=True, yfaces=yf)


def _sgrid(nx, ny, nz, ybeta, zbeta=None, ly=0.75, lz=1.2):
    zf = wl.uniform_zfaces(nz, lz) if zbeta is None else wl.tanh_zfaces(nz, lz, zbeta)
    yf = np.linspace(0.0, ly, ny + 1) if ybeta is None else wl.tanh_yfaces(ny, ly, ybeta)
    return orc.Grid(nx, ny, nz, 1.0, ly, zf, ywalls=True, yf=yf)


# --- constant-coefficient solve -------------------------------------------

@pytest.mark.parametrize("dims,ybeta,zbeta", [
    ((32, 24, 20), 1.5, None),
    ((24, 17, 12), 2.0, 1.5),     # odd ny, stretched z
    ((16, 2, 8), 1.0, None),      # two rows
    ((8, 300, 4), 1.5, 1.5),      # two output rows per thread of the dense step
    ((6, 1024, 3), 2.0, None),    # the largest ny: four rows per thread
])
def test_constant_solve_fp64_vs_oracle(pp, dims, ybeta, zbeta):
    g = _sgrid(*dims, ybeta, zbeta)
    f = np.random.default_rng(dims[0] * 7 + dims[1]).standard_normal(g.shape)
    plan = _plan(pp, g)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    err = _rel(host(p), orc.solve_constant(g, f))
    print(f"stretched-y constant solve {dims}: rel. L2 error {err:.3e}")
    assert err < FP64_TOL


def test_uniform_faces_match_the_cosine_plan(pp):
    """Uniform faces given as yfaces take the dense eigenbasis step; the
    result equals the plan without them (cosine transform by FFT)."""
    g = _sgrid(32, 20, 16, None, 1.5)
    gu = orc.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, ywalls=True)
    f = np.random.default_rng(4).standard_normal(g.shape)
    out = []
    for yf in (g.yf, None):
        plan = _plan(pp, g, yfaces=yf)
        p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        pp.pressure_solve(plan.handle, dev(f), p)
        out.append(host(p))
    assert _rel(out[0], out[1]) < FP64_TOL
    assert _rel(out[0], orc.solve_constant(gu, f)) < FP64_TOL


@pytest.mark.parametrize("precision", ["mixed", "mixed_z64", "mixed_tc"])
def test_constant_solve_mixed_vs_oracle(pp, precision):
    g = _sgrid(64, 48, 40, 1.5, 1.5)
    f = np.random.default_rng(77).standard_normal(g.shape)
    plan = _plan(pp, g, precision)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    tol = mixed_solve_bound_dense_y(g.nx, g.ny, g.dyf, tc=precision == "mixed_tc", nz=g.nz)
    err = _rel(host(p), orc.solve_constant(g, f))
    print(f"stretched-y constant solve {precision}: rel. L2 error {err:.3e}, bound {tol:.3e}")
    assert err < tol


# --- variable-density projection ------------------------------------------

def _case(n, ny, nz, ybeta=1.5, stretched=True, ratio=1000.0, seed=1302):
    w = wl.channel_bubble_case(n, ny, nz, seed=seed, rho_ratio=ratio, stretched=stretched, ybeta=ybeta)
    return w, orc.mixture_density(w.phi, w.rho_g, w.rho_l)


def _grid(w):
    return orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=True, yf=w.yf)


def _run(pp, w, rho, precision="fp64", rtol=1e-13, maxit=400, method="III"):
    plan = _plan(pp, _grid(w), precision, method)
    allow = rtol == 0.0
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=rtol, maxit=maxit, allow_not_converged=allow)
    return info, host(p), host(u), host(v), host(ww)


@pytest.mark.parametrize("dims,ybeta,ratio,passes", [
    ((32, 24, 20), 1.5, 1000.0, 30),
    ((24, 21, 18), 2.0, 100.0, 25),
])
def test_iterates_vs_oracle(pp, dims, ybeta, ratio, passes):
    """Algorithm 1 stopped after a fixed number of passes: the GPU iterate
    equals the oracle's (same s) to round-off; the wall row of v is 0."""
    w, rho = _case(*dims, ybeta=ybeta, ratio=ratio)
    g = _grid(w)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    info, p, u, v, ww = _run(pp, w, rho, rtol=0.0, maxit=passes)
    assert info["iters"] == passes
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    assert _rel(p, p0) < FP64_TOL
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL
    assert np.all(v[:, 0, :] == 0.0)


def test_converged_fp64_meets_the_divergence_target(pp):
    w, rho = _case(32, 24, 20)
    g = _grid(w)
    info, p, u, v, ww = _run(pp, w, rho, rtol=1e-12, maxit=5000)
    assert info["status"] == 0 and info["res_final"] <= 1e-12
    pd, ud, vd, wd = orc.projection_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt)
    for a, b in ((u, ud), (v, vd), (ww, wd)):
        assert _rel(a, b) < 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-12 * np.linalg.norm(d0)


@functools.lru_cache(maxsize=1)
def _mixed_reference():
    """The oracle's converged projection of a 40 x 36 x 32 duct with
    stretched y and z (computed once for the three mixed plans)."""
    w, rho = _case(40, 36, 32)
    g = _grid(w)
    return w, rho, orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-12, maxit=8000)


@pytest.mark.parametrize("precision", ["mixed", "mixed_z64", "mixed_tc"])
def test_mixed_vs_oracle(pp, precision):
    """Mixed precision on a stretched y: residual <= 1e-10 in FP64, fields
    within 1e-9 of the oracle's converged projection."""
    w, rho, (p0, u0, v0, w0, _) = _mixed_reference()
    g = _grid(w)
    info, p, u, v, ww = _run(pp, w, rho, precision, rtol=1e-10, maxit=8000)
    assert info["status"] == 0 and info["res_final"] <= 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1e-10 * np.linalg.norm(d0) * 1.0001
    errs = [_rel(a, b) for a, b in ((u, u0), (v, v0), (ww, w0))]
    print(precision, "stretched y vs oracle", errs, "iters", info["iters"])
    assert max(errs) < 1e-9
    assert np.all(v[:, 0, :] == 0.0)


@pytest.mark.parametrize("method", ["I", "II"])
def test_methods_1_2_vs_oracle(pp, method):
    w, rho = _case(24, 20, 18, ybeta=2.0, ratio=10.0)
    g = _grid(w)
    fn = orc.method1 if method == "I" else orc.method2
    passes = 20
    p0, u0, v0, w0, _ = fn(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    info, p, u, v, ww = _run(pp, w, rho, rtol=0.0, maxit=passes, method=method)
    assert info["iters"] == passes
    for a, b in ((p, p0), (u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL


def _adjoint_case():
    """A stretched duct, the direct forward pressure and the gradient of
    ||u^{n+1} - target||^2 (with a nonzero wall row of the v gradient, which
    must be ignored)."""
    w, rho = _case(12, 10, 8, ybeta=1.5, ratio=100.0, seed=1311)
    g = _grid(w)
    p0, u, v, ww = orc.projection_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt)
    rng = np.random.default_rng(1311 + 20)
    gu = 2 * (u - 0.1 * rng.standard_normal(w.shape))
    gv = 2 * (v - 0.1 * rng.standard_normal(w.shape))
    gw = 2 * (ww - 0.1 * rng.standard_normal(ww.shape))
    gv[:, 0, :] = 0.7
    return w, rho, g, p0, gu, gv, gw


def _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, rtol, maxit):
    plan = _plan(pp, _grid(w))
    out = [torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    out.append(torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda"))
    grho = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    info = pp.pressure_solve_adjoint(plan.handle, dev(rho), dev(p0), w.dt, dev(gu), dev(gv), dev(gw),
                                     out[0], out[1], out[2], grho, rtol=rtol, maxit=maxit,
                                     allow_not_converged=(rtol == 0.0))
    plan.close()
    return info, [host(x) for x in (*out, grho)]


def test_adjoint_iterates_vs_oracle(pp):
    """The transposed solve on a stretched y stopped after 30 passes on both
    sides equals the oracle's Algorithm-1 adjoint (face weights with the y
    metrics) to round-off; the wall row of the v gradient is 0."""
    w, rho, g, p0, gu, gv, gw = _adjoint_case()
    ref = orc.adjoint_method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw, rtol=0.0, maxit=30, p=p0)
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 0.0, 30)
    assert info["iters"] == 30
    for a, b in zip(got, ref[:4]):
        assert _rel(a, b) < FP64_TOL
    assert np.all(got[1][:, 0, :] == 0.0)


def test_adjoint_converged_vs_literal_transpose(pp):
    """The converged adjoint on a stretched y against the oracle's literal
    sparse-transpose gradient."""
    w, rho, g, p0, gu, gv, gw = _adjoint_case()
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 1e-12, 5000)
    assert info["status"] == 0
    ref = orc.adjoint_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw)
    for a, b in zip(got, ref):
        assert _rel(a, b) < 1e-9


def test_uniform_y_only_calls_refuse_a_stretched_y(pp):
    """The predictor is built for a uniform y: it returns PP_ERR_UNSUPPORTED
    before touching a field."""
    g = _sgrid(16, 12, 8, 1.5)
    plan = _plan(pp, g)
    c = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    fw = torch.zeros((g.nz + 1, g.ny, g.nx), dtype=torch.float64, device="cuda")
    ustar = (c.clone(), c.clone(), fw.clone())
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_predictor(plan.handle, c, c, fw, c + 1.0, c + 1e-3, (0.0, 0.0, -9.81), 1e-3, ustar)
    assert e.value.code == pp.PP_ERR_UNSUPPORTED
