"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 paths match the oracle to a relative L2 error of 1e-11 when
both iterate to a relative residual of 1e-13; mixed-precision paths reach a
relative residual <= 1e-10 measured in FP64 and match the oracle to the
error that residual allows (checked against 1e-8)."""
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


def _plan(pp, nx, ny, nz, lx, ly, zf, precision="fp64"):
    return pp.Plan(nx, ny, nz, lx, ly, float(zf[-1] - zf[0]), zfaces=zf, precision=precision)


# --- constant-coefficient solve -------------------------------------------

@pytest.mark.parametrize("dims,stretch,precision", [
    ((32, 32, 32), None, "fp64"),       # 32^3 random-divergence workload
    ((8, 8, 8), None, "fp64"),          # the 8^3 sub-case
    ((24, 20, 17), 1.5, "fp64"),        # ragged: radix 3/5, odd nz, stretched z
    ((96, 30, 9), 2.0, "fp64"),
    ((64, 48, 40), 1.5, "mixed"),
    ((64, 16, 512), None, "mixed"),     # nz = 512 with well-conditioned FP32 z columns
    ((48, 30, 100), 1.5, "mixed"),      # radices 2, 3, 5 in y, stretched z
    ((64, 48, 40), 1.5, "mixed_z64"),   # FP64 z recurrences in every column
    ((48, 30, 100), 1.5, "mixed_z64"),
])
def test_constant_solve_vs_oracle(pp, dims, stretch, precision):
    nx, ny, nz = dims
    lx, ly, lz = 1.0, 0.75, 1.2
    zf = wl.uniform_zfaces(nz, lz) if stretch is None else wl.tanh_zfaces(nz, lz, stretch)
    g = orc.Grid(nx, ny, nz, lx, ly, zf)
    rng = np.random.default_rng(nx * 7 + nz)
    f = rng.standard_normal(g.shape)
    ref = orc.solve_constant(g, f)
    plan = _plan(pp, nx, ny, nz, lx, ly, zf, precision)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    # mixed plans: the FP32 rounding bound of one solve (tests/fp32_bounds.py)
    tol = FP64_TOL if precision == "fp64" else mixed_solve_bound(nx, ny)
    err = _rel(host(p), ref)
    print(f"constant solve {dims} {precision}: rel. L2 error {err:.3e}, bound {tol:.3e}")
    assert err < tol


def test_single_mode_closed_form_gpu(pp):
    """Discrete eigenmode (3, 5, 2) on the 32^3 grid: p = f / lambda."""
    n = 32
    zf = wl.uniform_zfaces(n, 1.0)
    i = np.arange(n)[None, None, :]; j = np.arange(n)[None, :, None]; k = np.arange(n)[:, None, None]
    f = np.cos(2 * np.pi * 3 * i / n) * np.cos(2 * np.pi * 5 * j / n) * np.cos(np.pi * 2 * (k + 0.5) / n)
    h = 1.0 / n
    lam = -4 / h ** 2 * (np.sin(np.pi * 3 / n) ** 2 + np.sin(np.pi * 5 / n) ** 2 + np.sin(np.pi * 2 / (2 * n)) ** 2)
    plan = _plan(pp, n, n, n, 1.0, 1.0, zf)
    p = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    assert _rel(host(p), f / lam) < FP64_TOL


# --- Method III projection -----------------------------------------------

def _case(n=32, stretched=False, ratio=1000.0, nz=None, ny=None, seed=1102):
    w = wl.small_bubble_case(n, seed=seed, rho_ratio=ratio, stretched=stretched, nz=nz, ny=ny)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    return w, rho


def _run_gpu(pp, w, rho, precision="fp64", rtol=1e-13, maxit=400, host_ptrs=False):
    allow = rtol == 0.0
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, precision)
    if host_ptrs:
        p = np.empty(w.shape); u = np.empty(w.shape); v = np.empty(w.shape)
        ww = np.empty((w.nz + 1, w.ny, w.nx))
        info = pp.pressure_correct(plan.handle, w.us, w.vs, w.ws, rho, w.S, w.dt, p, u, v, ww,
                                   rtol=rtol, maxit=maxit, allow_not_converged=allow)
        return info, p, u, v, ww
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u = torch.empty_like(p); v = torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=rtol, maxit=maxit, allow_not_converged=allow)
    return info, host(p), host(u), host(v), host(ww)


@pytest.mark.parametrize("stretched,ratio,dims,passes", [
    (False, 1000.0, (32, None, None), 40),
    (True, 1000.0, (32, None, None), 40),
    (False, 10.0, (24, 20, 18), 25),
    (True, 100.0, (40, 30, 25), 30),
])
def test_projection_fp64_iterates_vs_oracle(pp, stretched, ratio, dims, passes):
    """Algorithm 1 stopped after a fixed number of passes: the GPU iterate
    equals the oracle's iterate (same s) to round-off."""
    n, ny, nz = dims
    w, rho = _case(n, stretched, ratio, nz=nz, ny=ny)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=passes)
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=0.0, maxit=passes, allow_not_converged=True)
    assert info["iters"] == passes
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    assert abs(info["res_l1_sum"] - oinfo["res_l1_sum"]) <= 1e-9 * oinfo["res_l1_sum"]
    assert abs(info["mean_S_removed"] - oinfo["mean_S_removed"]) <= 1e-14 * max(1.0, abs(oinfo["mean_S_removed"]))
    assert _rel(host(p), p0) < FP64_TOL
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(host(a), b) < FP64_TOL


def _sphere_case(n, ratio, stretched=False, nz=None):
    nz = nz or n
    zf = wl.tanh_zfaces(nz, 1.0, 1.5) if stretched else wl.uniform_zfaces(nz, 1.0)
    phi = wl.spheres_phi(n, n, nz, 1.0, 1.0, zf, [(0.5, 0.5, 0.3, 0.15)])
    us, vs, ws = wl.random_faces(n, n, nz, 0.1, 1002)
    w = wl.Workload(f"sphere {n}", n, n, nz, 1.0, 1.0, zf, 1e-3, us, vs, ws, phi, 1.2, ratio,
                    wl.gas_source(phi))
    return w, orc.mixture_density(phi, 1.2, ratio)


@pytest.mark.parametrize("n,ratio,stretched,nz", [(32, 1000.0, False, None), (24, 100.0, True, 20)])
def test_projection_fp64_converged_vs_oracle(pp, n, ratio, stretched, nz):
    """Converged projection (relative residual 1e-12 on both sides)."""
    w, rho = _sphere_case(n, ratio, stretched, nz)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-12, maxit=2000)
    info, *_ = _run_gpu(pp, w, rho, "fp64", rtol=1e-12, maxit=2000)
    assert info["status"] == 0 and info["res_final"] <= 1e-12
    assert abs(info["iters"] - oinfo["iters"]) <= 1
    # same pass count on both sides: the converged fields agree to round-off
    info, p, u, v, ww = _run_gpu(pp, w, rho, "fp64", rtol=0.0, maxit=oinfo["iters"])
    assert _rel(p, p0) < FP64_TOL
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < FP64_TOL
    # the corrected field meets the divergence target (oracle's D, FP64)
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-12 * np.linalg.norm(d0)


@pytest.mark.parametrize("stretched,precision", [(False, "mixed"), (True, "mixed"), (True, "mixed_z64")])
def test_projection_mixed_vs_oracle(pp, stretched, precision):
    """Mixed precision + FP64 residual: reaches 1e-10 and matches the FP64
    oracle's converged solution (mixed_z64: FP64 recurrences in every z
    column)."""
    w, rho = _sphere_case(48, 1000.0, stretched, 40)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, _ = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=3000)
    info, p, u, v, ww = _run_gpu(pp, w, rho, precision, rtol=1e-10, maxit=3000)
    assert info["status"] == 0 and info["res_final"] <= 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    # residual re-evaluated by the oracle in FP64
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1e-10 * np.linalg.norm(d0) * 1.0001
    errs = [_rel(a, b) for a, b in ((u, u0), (v, v0), (ww, w0))]
    print("mixed vs oracle rel errors", errs, "iters", info["iters"])
    assert max(errs) < 1e-9


@pytest.mark.parametrize("dims,precision", [
    ((512, 15, 7), "mixed_z64"),    # 512-point x lines in registers; odd row count (a half-empty pair)
    ((16, 512, 6), "mixed"),        # 512-point y lines in registers
    ((512, 512, 3), "mixed_z64"),   # both, several row groups per block
])
def test_register_transforms_vs_oracle(pp, dims, precision):
    """The 512-point FP32 transforms (residual + forward x, inverse x +
    update, y) against the oracle: a constant solve within the FP32 bound,
    then a projection that crosses the exact / updated residual cycle (50
    passes) and converges to 1e-10 with the oracle's fields."""
    nx, ny, nz = dims
    zf = wl.tanh_zfaces(nz, 0.7, 1.5)
    g = orc.Grid(nx, ny, nz, 1.0, 0.8, zf)
    f = np.random.default_rng(nx + 3 * ny + nz).standard_normal(g.shape)
    plan = _plan(pp, nx, ny, nz, 1.0, 0.8, zf, precision)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    err = _rel(host(p), orc.solve_constant(g, f))
    bound = mixed_solve_bound(nx, ny)
    print(f"register transforms {dims} {precision}: constant solve {err:.3e} (bound {bound:.3e})")
    assert err < bound
    rng = np.random.default_rng(5)
    phi = np.zeros(g.shape)
    phi[:, ny // 4:ny // 2 + 1, nx // 3:nx // 2] = 1.0
    rho = orc.mixture_density(phi, 1.0, 100.0)
    us, vs = rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1
    ws = rng.standard_normal((nz + 1, ny, nx)) * 0.1
    ws[0] = ws[-1] = 0.0
    S = wl.gas_source(phi)
    dt = 1e-3
    p0, u0, v0, w0, _ = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-12, maxit=3000)
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((nz + 1, ny, nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(us), dev(vs), dev(ws), dev(rho), dev(S), dt, p, u, v, ww,
                               rtol=1e-10, maxit=3000)
    assert info["status"] == 0 and info["res_final"] <= 1e-10 and info["iters"] > 45
    Sc = S - orc.volume_mean(g, S)
    d0 = orc.divergence(g, us, vs, ws) - Sc
    assert np.linalg.norm(orc.divergence(g, host(u), host(v), host(ww)) - Sc) <= 1e-10 * np.linalg.norm(d0) * 1.0001
    errs = [_rel(host(a), b) for a, b in ((u, u0), (v, v0), (ww, w0))]
    print(f"register transforms {dims} {precision}: converged fields vs oracle {errs}, iters {info['iters']}")
    assert max(errs) < 1e-8


@pytest.mark.parametrize("dims", [(512, 512, 16), (512, 512, 17), (512, 64, 96)])
def test_register_transforms_many_lines_per_block(pp, dims):
    """The persistent 512-point kernels with several lines (x) and tiles (y)
    per block, the next tile's values loaded during the current transform:
    constant solves against the oracle within the FP32 bound, both mixed
    plans."""
    nx, ny, nz = dims
    zf = wl.tanh_zfaces(nz, 1.0, 1.5)
    g = orc.Grid(nx, ny, nz, 2.0, 2.0, zf)
    f = np.random.default_rng(nz).standard_normal(g.shape)
    ref = orc.solve_constant(g, f)
    bound = mixed_solve_bound(nx, ny)
    for precision in ("mixed_z64", "mixed"):
        plan = _plan(pp, nx, ny, nz, 2.0, 2.0, zf, precision)
        p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        pp.pressure_solve(plan.handle, dev(f), p)
        err = _rel(host(p), ref)
        print(f"register transforms {dims} {precision}: constant solve {err:.3e} (bound {bound:.3e})")
        assert err < bound
        plan.close()


def test_host_pointers_match_device(pp):
    w, rho = _case(24, True, 10.0)
    a = _run_gpu(pp, w, rho, "fp64", rtol=1e-11)
    b = _run_gpu(pp, w, rho, "fp64", rtol=1e-11, host_ptrs=True)
    assert a[0]["iters"] == b[0]["iters"]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_constant_density_single_pass(pp):
    w, _ = _case(16, False, 1.0)
    rho = np.full(w.shape, 2.5)
    info, *_ = _run_gpu(pp, w, rho, "fp64", rtol=1e-12)
    assert info["iters"] == 1


def test_not_converged_status(pp):
    w, rho = _case(16, False, 1000.0)
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    u, v = torch.empty_like(p), torch.empty_like(p)
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt,
                               p, u, v, ww, rtol=1e-14, maxit=2, allow_not_converged=True)
    assert info["status"] == pp.PP_ERR_NOT_CONVERGED and info["iters"] == 2
    with pytest.raises(pp.PressureError):
        pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), -1.0,
                            p, u, v, ww)


def test_mixture_density_gpu(pp):
    w, _ = _case(16, False, 1000.0)
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_mixture_density(plan.handle, dev(w.phi), 1.2, 1000.0, rho)
    assert np.array_equal(host(rho), orc.mixture_density(w.phi, 1.2, 1000.0))


# --- adjoint --------------------------------------------------------------

def _adjoint_inputs():
    w = wl.droplets_case(24, 24, 16, seed=1005, beta=2.0)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    ut = w.extra["target"]
    p0, u0, v0, w0, _ = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-12, maxit=3000)
    gu, gv, gw = 2 * (u0 - ut[0]), 2 * (v0 - ut[1]), 2 * (w0 - ut[2])
    return w, rho, g, p0, gu, gv, gw


def _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, rtol, maxit, precision="fp64"):
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, precision)
    outs = [torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    gws = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    grho = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    info = pp.pressure_solve_adjoint(plan.handle, dev(rho), dev(p0), w.dt, dev(gu), dev(gv), dev(gw),
                                     outs[0], outs[1], gws, grho, rtol=rtol, maxit=maxit,
                                     allow_not_converged=(rtol == 0.0))
    return info, [host(outs[0]), host(outs[1]), host(gws), host(grho)]


def test_adjoint_iterates_vs_oracle(pp):
    """Transposed solve stopped after 60 passes on both sides: gradients agree
    to round-off (stretched z, 4 droplets, ratio 100)."""
    w, rho, g, p0, gu, gv, gw = _adjoint_inputs()
    ref = orc.adjoint_method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw, rtol=0.0, maxit=60, p=p0)
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 0.0, 60)
    assert info["iters"] == 60
    for a, b in zip(got, ref[:4]):
        assert _rel(a, b) < FP64_TOL


def test_adjoint_converged_vs_direct(pp):
    """Converged adjoint (relative residual 1e-12) against the oracle's
    literal sparse-transpose gradient."""
    w, rho, g, p0, gu, gv, gw = _adjoint_inputs()
    info, got = _gpu_adjoint(pp, w, rho, p0, gu, gv, gw, 1e-12, 3000)
    assert info["status"] == 0
    ref = orc.adjoint_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt, gu, gv, gw)
    errs = [_rel(a, b) for a, b in zip(got, ref)]
    print("adjoint vs direct", errs, "iters", info["iters"])
    assert max(errs) < 1e-8


def test_autograd_function_matches_oracle_gradient(pp):
    """torch.autograd through ProjectFunction: dL/du*, dL/drho equal the
    oracle's literal-transpose gradient (L = ||u^{n+1} - u_target||^2)."""
    from paper_2005_11806_gb300.autograd import project
    w, rho, g, p0, gu, gv, gw = _adjoint_inputs()
    ut = w.extra["target"]
    plan = _plan(pp, w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    us, vs, ws, r = (dev(a).requires_grad_() for a in (w.us, w.vs, w.ws, rho))
    u, v, ww, p = project(us, vs, ws, r, plan, dev(w.S), w.dt, rtol=1e-12, maxit=3000)
    tgt = [dev(a) for a in ut]
    loss = ((u - tgt[0]) ** 2).sum() + ((v - tgt[1]) ** 2).sum() + ((ww[1:-1] - tgt[2][1:-1]) ** 2).sum()
    loss.backward()
    ref = orc.adjoint_direct(g, w.us, w.vs, w.ws, rho, w.S, w.dt, 2 * (host(u) - ut[0]),
                             2 * (host(v) - ut[1]), 2 * (host(ww) - ut[2]))
    for got, exp in ((us.grad, ref[0]), (vs.grad, ref[1]), (ws.grad, ref[2]), (r.grad, ref[3])):
        assert _rel(host(got), exp) < 1e-8


# --- tensor-core z solve (eigenvector expansion along z, BF16x3 products) --

@pytest.mark.parametrize("dims,stretch", [((32, 32, 40), 1.5), ((48, 40, 128), 2.0), ((64, 64, 64), None)])
def test_tc_constant_solve_vs_oracle(pp, dims, stretch):
    """The tensor-core z expansion solves the constant-coefficient equation;
    its error is that of BF16x3 products (2^-16 relative per product)."""
    nx, ny, nz = dims
    zf = wl.uniform_zfaces(nz, 1.0) if stretch is None else wl.tanh_zfaces(nz, 1.0, stretch)
    g = orc.Grid(nx, ny, nz, 1.0, 1.0, zf)
    f = np.random.default_rng(nz).standard_normal(g.shape)
    ref = orc.solve_constant(g, f)
    plan = _plan(pp, nx, ny, nz, 1.0, 1.0, zf, "mixed_tc")
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    pp.pressure_solve(plan.handle, dev(f), p)
    err = _rel(host(p), ref)
    print("tc constant solve rel err", dims, err)
    assert err < 1e-3


@pytest.mark.parametrize("stretched", [False, True])
def test_projection_tc_vs_oracle(pp, stretched):
    """Method III with the tensor-core z solve still reaches a relative
    residual of 1e-10 (evaluated in FP64) and the FP64 oracle's solution."""
    w, rho = _sphere_case(48, 1000.0, stretched, 40)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=3000)
    info, p, u, v, ww = _run_gpu(pp, w, rho, "mixed_tc", rtol=1e-10, maxit=3000)
    print("tc projection iters", info["iters"], "oracle(1e-13)", oinfo["iters"])
    assert info["status"] == 0 and info["res_final"] <= 1e-10
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
    assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-10 * np.linalg.norm(d0)
    for a, b in ((u, u0), (v, v0), (ww, w0)):
        assert _rel(a, b) < 1e-9
