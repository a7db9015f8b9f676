"""The z solve by the cosine basis (uniform walls in z: the eigenvectors of
the Neumann z difference are cos(pi m (k + 1/2) / nz)) on FP64 plans,
through the C ABI, against the oracle's Thomas-based solve: the same
discrete solution, relative L2 error <= 1e-11."""
import math

import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl

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


def _plan(pp, g, zfaces=True, **kw):
    return pp.Plan(g.nx, g.ny, g.nz, g.lx, g.ly, float(g.zf[-1] - g.zf[0]), zfaces=g.zf if zfaces else None,
                   ywalls=g.ywalls, zsolve="cosine", **kw)


@pytest.mark.parametrize("dims,ywalls,zfaces", [
    ((32, 32, 32), False, False),
    ((24, 20, 18), False, True),     # radices 3 and 5, faces passed explicitly
    ((16, 12, 10), True, False),     # cosine in y and in z
    ((96, 30, 40), True, True),
])
def test_zcosine_constant_solve_vs_oracle(pp, dims, ywalls, zfaces):
    nx, ny, nz = dims
    g = orc.Grid(nx, ny, nz, 1.0, 0.75, wl.uniform_zfaces(nz, 1.2), ywalls=ywalls)
    f = np.random.default_rng(nx + 3 * nz).standard_normal(g.shape)
    plan = _plan(pp, g, zfaces)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    assert _rel(host(p), orc.solve_constant(g, f)) < FP64_TOL


def test_zcosine_single_mode_closed_form(pp):
    nx, ny, nz, lx, ly, lz = 32, 24, 20, 1.0, 1.3, 0.6
    g = orc.Grid(nx, ny, nz, lx, ly, wl.uniform_zfaces(nz, lz))
    a, b, c = 3, 5, 7
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    f = np.cos(2 * np.pi * a * i / nx) * np.cos(2 * np.pi * b * j / ny + 0.3) * np.cos(np.pi * c * (k + 0.5) / nz)
    lam = -(4 * (nx / lx) ** 2 * math.sin(math.pi * a / nx) ** 2 + 4 * (ny / ly) ** 2 * math.sin(math.pi * b / ny) ** 2
            + 4 * (nz / lz) ** 2 * math.sin(math.pi * c / (2 * nz)) ** 2)
    plan = _plan(pp, g)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    assert _rel(host(p), f / lam) < FP64_TOL


@pytest.mark.parametrize("ywalls,ratio,passes", [(False, 1000.0, 40), (True, 100.0, 30)])
def test_zcosine_projection_iterates_vs_oracle(pp, ywalls, ratio, passes):
    """Algorithm 1 with the cosine z solve: the fixed-pass iterate equals the
    oracle's (which solves z by Thomas) to round-off."""
    if ywalls:
        w = wl.channel_bubble_case(32, 24, 20, seed=1202, rho_ratio=ratio)
    else:
        w = wl.small_bubble_case(32, seed=1102, rho_ratio=ratio)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=ywalls)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    plan = _plan(pp, g)
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=0.0, maxit=passes, allow_not_converged=True)
    assert info["iters"] == passes
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    for a, b in ((p, p0), (u, u0), (v, v0), (ww, w0)):
        assert _rel(host(a), b) < FP64_TOL


def test_zcosine_rejected_where_not_built(pp):
    g = orc.Grid(16, 16, 16, 1.0, 1.0, wl.tanh_zfaces(16, 1.0, 1.5))
    for kw, code in ((dict(), pp.PP_ERR_UNSUPPORTED),                      # stretched z
                     (dict(zfaces=False, precision="mixed"), pp.PP_ERR_UNSUPPORTED)):
        with pytest.raises(pp.PressureError) as e:
            _plan(pp, g, **kw)
        assert e.value.code == code
    with pytest.raises(pp.PressureError) as e:
        pp.Plan(16, 16, 15, 1.0, 1.0, 1.0, zsolve="cosine")           # odd nz
    assert e.value.code == pp.PP_ERR_UNSUPPORTED
    plan = pp.Plan(16, 16, 16, 1.0, 1.0, 1.0)
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_plan_set_zsolve(plan.handle, 5)
    assert e.value.code == pp.PP_ERR_INVALID_ARG
    pp.pressure_plan_set_zsolve(plan.handle, "cosine")
    pp.pressure_plan_set_zsolve(plan.handle, "tridiag")
