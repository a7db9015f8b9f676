"""The momentum predictor (Eqs. 29, 32) on the GPU, through the C ABI,
against the oracle: FP64, 1e-12 relative L2 on u*, v*, w* and on RU."""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def _state(w, seed):
    """Two-phase properties from the volume fraction, a previous RU and a
    body force, all seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    mu = 1.8e-5 * w.phi + 1e-3 * (1.0 - w.phi)
    prev = (rng.standard_normal(w.shape), rng.standard_normal(w.shape), rng.standard_normal((w.nz + 1, w.ny, w.nx)))
    prev[2][0] = prev[2][-1] = 0.0
    force = (0.1 * rng.standard_normal(w.shape), 0.1 * rng.standard_normal(w.shape),
             0.1 * rng.standard_normal((w.nz + 1, w.ny, w.nx)))
    return rho, mu, prev, force


def _gpu(pp, w, rho, mu, grav, dt_new, dt_old=0.0, prev=None, force=None, ywalls=False):
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf, ywalls=ywalls)
    out = [torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    out.append(torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda"))
    ru = [torch.empty_like(t) for t in out]
    pp.pressure_predictor(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(mu), grav, dt_new, out,
                          dt_old=dt_old, ru_prev=None if prev is None else [dev(a) for a in prev], ru_out=ru,
                          force=None if force is None else [dev(a) for a in force])
    return [host(t) for t in out], [host(t) for t in ru]


@pytest.mark.parametrize("dims,stretched,ab2", [((32, None, None), False, True), ((24, 20, 18), True, True),
                                                ((40, 30, 25), True, False)])
def test_predictor_vs_oracle(pp, dims, stretched, ab2):
    n, ny, nz = dims
    w = wl.small_bubble_case(n, seed=1102, rho_ratio=1000.0, stretched=stretched, nz=nz, ny=ny)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho, mu, prev, force = _state(w, 1106)
    grav = (0.0, 0.3, -9.81)
    kw = dict(dt_old=1e-3, prev=prev) if ab2 else {}
    out, ru = _gpu(pp, w, rho, mu, grav, 1.3e-3, force=force, **kw)
    (ue, ve, we), rue = orc.predictor(g, w.us, w.vs, w.ws, rho, mu, grav, 1.3e-3,
                                      dt_old=1e-3 if ab2 else None, ru_prev=prev if ab2 else None, force=force)
    errs = [_rel(a, b) for a, b in zip(out + ru, (ue, ve, we) + tuple(rue))]
    print("predictor vs oracle:", errs)
    assert max(errs) < TOL
    assert np.all(out[2][0] == 0.0) and np.all(out[2][-1] == 0.0)


@pytest.mark.parametrize("dims,ab2", [((24, 16, 18), True), ((40, 30, 25), False)])
def test_predictor_with_walls_in_y_vs_oracle(pp, dims, ab2):
    """No-slip walls in y (a duct, stretched z): u*, v*, w* and RU against
    the oracle's walled-y predictor (itself pinned by Poiseuille profiles
    and its reduction to the periodic stencil away from the walls).  A
    nonzero wall row of v^n is read as zero; the wall row of v* and of RU_y
    is written as zero."""
    nx, ny, nz = dims
    w = wl.channel_bubble_case(nx, ny, nz, seed=1206, rho_ratio=1000.0, stretched=True)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=True)
    rho, mu, prev, force = _state(w, 1107)
    w.vs[:, 0, :] = 0.4
    grav = (0.2, 0.3, -9.81)
    kw = dict(dt_old=1e-3, prev=prev) if ab2 else {}
    out, ru = _gpu(pp, w, rho, mu, grav, 1.3e-3, force=force, ywalls=True, **kw)
    (ue, ve, we), rue = orc.predictor(g, w.us, w.vs, w.ws, rho, mu, grav, 1.3e-3,
                                      dt_old=1e-3 if ab2 else None, ru_prev=prev if ab2 else None, force=force)
    errs = [_rel(a, b) for a, b in zip(out + ru, (ue, ve, we) + tuple(rue))]
    print("walled-y predictor vs oracle:", errs)
    assert max(errs) < TOL
    assert np.all(out[1][:, 0, :] == 0.0) and np.all(ru[1][:, 0, :] == 0.0)
    assert np.all(out[2][0] == 0.0) and np.all(out[2][-1] == 0.0)


def test_predictor_rejects_host_pointers(pp):
    w = wl.small_bubble_case(16, seed=1102)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf)
    out = [torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    out.append(torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda"))
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_predictor(plan.handle, w.us, dev(w.vs), dev(w.ws), dev(np.ones(w.shape)),
                              dev(np.ones(w.shape)), (0, 0, 0), 1e-3, out)
    assert e.value.code == pp.PP_ERR_INVALID_ARG


def test_predictor_then_projection(pp):
    """One time step of the solver's order: predictor, then the Method III
    projection of u* (D u^{n+1} = 0 to 1e-12 with S = 0)."""
    w = wl.small_bubble_case(24, seed=1102, rho_ratio=100.0, stretched=True, nz=20)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho, mu, _, _ = _state(w, 1107)
    (us, vs, ws), _ = _gpu(pp, w, rho, mu, (0.0, 0.0, -9.81), 1e-3)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf)
    p, u, v = (torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(3))
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(us), dev(vs), dev(ws), dev(rho), None, 1e-3, p, u, v, ww,
                               rtol=1e-12, maxit=5000)
    assert info["status"] == 0
    d0 = np.linalg.norm(orc.divergence(g, us, vs, ws).ravel())
    assert np.linalg.norm(orc.divergence(g, host(u), host(v), host(ww)).ravel()) <= 1.0001e-12 * d0


@pytest.mark.slow
def test_predictor_fullsize_sphere256(pp):
    """256^3 sphere workload (ratio 1000 : 1.2), Adams-Bashforth step with a
    body force, every face against the oracle."""
    w = wl.single_sphere_case(n=256, seed=1002)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho, mu, prev, force = _state(w, 1108)
    out, ru = _gpu(pp, w, rho, mu, (0.0, 0.0, -9.81), 1e-3, dt_old=1.1e-3, prev=prev, force=force)
    (ue, ve, we), rue = orc.predictor(g, w.us, w.vs, w.ws, rho, mu, (0.0, 0.0, -9.81), 1e-3, dt_old=1.1e-3,
                                      ru_prev=prev, force=force)
    errs = [_rel(a, b) for a, b in zip(out + ru, (ue, ve, we) + tuple(rue))]
    print("256^3 predictor vs oracle:", errs)
    assert max(errs) < TOL
