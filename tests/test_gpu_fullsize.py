"""Parity at the benchmark's full sizes, through the C ABI.

At these sizes the oracle cannot run a converged projection (a 512^3 pass
takes it about 16 s, and the benchmark needs 2448 passes).  So each case
checks what the oracle can afford, plus properties that hold at any size:

* The first Algorithm 1 passes are compared element by element with the
  oracle's passes on the same input, covering the residual, every transform,
  the z solve, the update of p and the correction.
* The converged projection must satisfy D u^{n+1} = S_c to the tolerance, as
  the oracle's FP64 divergence evaluates it.  The returned u and p must be
  consistent: u = u* - dt beta G p (Eq. corr), evaluated by the oracle.  And
  p has zero volume-weighted mean.
* The adjoint is checked against central finite differences of the converged
  projection on sampled entries, and against the dot-product identity.

Tolerances:

* FP64 paths: 1e-11 relative L2 for iterates.
* Mixed paths: the first two passes carry the FP32 rounding of the
  transforms and of the z solve's stored values.  The bound is the model of
  tests/fp32_bounds.py: per solve 2^-24 x (1 narrowing + 3 per Stockham pass
  x 3 passes x 4 transforms of length 512 + 2 z stores) = 39 u, times 2
  passes: 4.6e-6 (measured: 0.8e-6 in p, 1.8e-6 in the velocities, for
  both the FP64-recurrence and the hybrid z solve).  Converged mixed results
  satisfy the 1e-10 residual in FP64.
"""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl
from tests.fp32_bounds import mixed_solve_bound

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64_TOL = 1e-11
MIXED_PASS_TOL = mixed_solve_bound(512, 512, passes=2)


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


class Runner:
    """One plan and its device buffers for repeated projections."""

    def __init__(self, pp, w, precision):
        self.pp, self.w = pp, w
        self.plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf,
                            precision=precision)
        self.p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        self.u = torch.empty_like(self.p)
        self.v = torch.empty_like(self.p)
        self.ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")

    def run(self, us, vs, ws, rho, S, rtol, maxit):
        info = self.pp.pressure_correct(self.plan.handle, us, vs, ws, rho, S, self.w.dt, self.p, self.u,
                                        self.v, self.ww, rtol=rtol, maxit=maxit,
                                        allow_not_converged=(rtol == 0.0))
        return info


def _check_converged(g, w, rho, p, u, v, ww, tol, label):
    """Properties of a converged projection, evaluated by the oracle in FP64."""
    Sc = w.S - orc.volume_mean(g, w.S)
    d0 = np.linalg.norm((orc.divergence(g, w.us, w.vs, w.ws) - Sc).ravel())
    d = np.linalg.norm((orc.divergence(g, u, v, ww) - Sc).ravel())
    print(f"{label}: ||D u - S_c|| / ||D u* - S_c|| = {d / d0:.3e}")
    assert d <= tol * d0 * 1.0001
    ue, ve, we = orc.correct_velocity(g, w.us, w.vs, w.ws, rho, p, w.dt)
    errs = [_rel(a, b) for a, b in ((u, ue), (v, ve), (ww, we))]
    print(f"{label}: u vs u* - dt beta G p: {errs}")
    assert max(errs) < 1e-12
    assert abs(orc.volume_mean(g, p)) <= 1e-12 * max(1.0, float(np.max(np.abs(p))))


def test_bubbles512_mixed(pp):
    """The benchmark workload (512^3, 200 bubbles, tanh z, ratio 1000): the
    plan bench.py times (mixed_z64: FP64 z recurrences in every column) and
    the hybrid-z plan.  Each: two passes against the oracle's (computed
    once), then the converged projection's properties."""
    w = wl.bubbles_case(n=512, nbubbles=200, seed=1003, beta=1.5, rho_g=1.0, rho_l=1000.0)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=2)
    args = [dev(a) for a in (w.us, w.vs, w.ws, rho, w.S)]
    for precision in ("mixed_z64", "mixed"):
        R = Runner(pp, w, precision)
        info = R.run(*args, rtol=0.0, maxit=2)
        assert info["iters"] == 2
        errs = [_rel(host(a), b) for a, b in ((R.p, p0), (R.u, u0), (R.v, v0), (R.ww, w0))]
        print(f"512^3 {precision}, 2 passes vs oracle:", errs, "bound", MIXED_PASS_TOL,
              "res", info["res_final"], oinfo["res_hist"][-1])
        assert max(errs) < MIXED_PASS_TOL
        info = R.run(*args, rtol=1e-10, maxit=50000)
        assert info["status"] == 0 and info["res_final"] <= 1e-10
        _check_converged(g, w, rho, host(R.p), host(R.u), host(R.v), host(R.ww), 1e-10, f"512^3 {precision}")
        R.plan.close()
        del R


def test_sphere256_fp64(pp):
    """256^3 unit cube, one gas sphere at ratio 1000 : 1.2, FP64: three passes
    equal the oracle's to round-off; the converged projection meets 1e-12."""
    w = wl.single_sphere_case(n=256, seed=1002)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    R = Runner(pp, w, "fp64")
    args = [dev(a) for a in (w.us, w.vs, w.ws, rho, w.S)]
    info = R.run(*args, rtol=0.0, maxit=3)
    assert info["iters"] == 3
    p0, u0, v0, w0, oinfo = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=0.0, maxit=3)
    errs = [_rel(host(a), b) for a, b in ((R.p, p0), (R.u, u0), (R.v, v0), (R.ww, w0))]
    print("256^3 fp64, 3 passes vs oracle:", errs)
    assert max(errs) < FP64_TOL
    assert abs(info["res_final"] - oinfo["res_hist"][-1]) <= 1e-9 * oinfo["res_hist"][-1]
    info = R.run(*args, rtol=1e-12, maxit=20000)
    assert info["status"] == 0 and info["res_final"] <= 1e-12
    _check_converged(g, w, rho, host(R.p), host(R.u), host(R.v), host(R.ww), 1e-12, "256^3 fp64")


def test_batch96_converged_properties(pp):
    """The 96-grid batch (one graph launch): every grid converges to 1e-10,
    and a seeded sample of 16 grids is checked by the oracle."""
    cases = wl.batch_case(count=96, seed=1004, ratio=1000.0)
    grids = [dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, lz=float(c.zf[-1]), zfaces=c.zf) for c in cases]
    B = pp.Batch(grids)
    cat = lambda arrs: dev(np.concatenate([a.ravel() for a in arrs]))  # noqa: E731
    us, vs, ws = cat([c.us for c in cases]), cat([c.vs for c in cases]), cat([c.ws for c in cases])
    phi, S = cat([c.phi for c in cases]), cat([c.S for c in cases])
    rho = torch.empty_like(phi)
    p, u, v = (torch.empty(B.ncell, dtype=torch.float64, device="cuda") for _ in range(3))
    w = torch.empty(B.nwface, dtype=torch.float64, device="cuda")
    B.mixture_density(phi, cases[0].rho_g, cases[0].rho_l, rho)
    infos = B.correct(us, vs, ws, rho, S, cases[0].dt, p, u, v, w, rtol=1e-10, maxit=50000)
    assert all(i["status"] == 0 and i["res_final"] <= 1e-10 for i in infos)
    hp, hu, hv, hw, hr = host(p), host(u), host(v), host(w), host(rho)
    pick = np.random.Generator(np.random.PCG64(1004 + 30)).choice(len(cases), 16, replace=False)
    for k in sorted(pick):
        c = cases[k]
        co, wo, nc, nw = B.cell_offset[k], B.wface_offset[k], c.nx * c.ny * c.nz, c.nx * c.ny * (c.nz + 1)
        sl = lambda a: a[co:co + nc].reshape(c.shape)  # noqa: E731
        g = orc.Grid(c.nx, c.ny, c.nz, c.lx, c.ly, c.zf)
        r = sl(hr)
        assert np.array_equal(r, orc.mixture_density(c.phi, c.rho_g, c.rho_l)) or \
            _rel(r, orc.mixture_density(c.phi, c.rho_g, c.rho_l)) < 1e-15
        _check_converged(g, c, r, sl(hp), sl(hu), sl(hv), hw[wo:wo + nw].reshape((c.nz + 1, c.ny, c.nx)),
                         1e-10, f"batch grid {k}")


def test_adjoint_droplets_fd(pp):
    """256 x 256 x 128, stretched z (beta = 2), 4 droplets at ratio 100, FP64.
    L = ||u^{n+1} - u_target||^2.  The adjoint's dL/du* and dL/drho are checked
    against central finite differences (eps = 1e-6, scaled by the entry) on 32
    seeded entries, and against the dot-product identity <J d, g> =
    <d, J^T g> along one random direction of (u*, rho)."""
    w = wl.droplets_case(256, 256, 128, seed=1005, beta=2.0)
    rho = orc.mixture_density(w.phi, w.rho_g, w.rho_l)
    ut = w.extra["target"]
    R = Runner(pp, w, "fp64")
    base = {"us": w.us, "vs": w.vs, "ws": w.ws, "rho": rho}
    d = {k: dev(a) for k, a in base.items()}
    S = dev(w.S)
    tgt = [dev(a) for a in ut]

    def project(fields):
        info = R.run(fields["us"], fields["vs"], fields["ws"], fields["rho"], S, rtol=1e-13, maxit=50000)
        assert info["status"] == 0
        return R.u.clone(), R.v.clone(), R.ww.clone(), R.p.clone()

    u, v, ww, p = project(d)
    gu, gv, gw = 2 * (u - tgt[0]), 2 * (v - tgt[1]), 2 * (ww - tgt[2])
    gw[0] = 0.0
    gw[-1] = 0.0
    gus, gvs = torch.empty_like(u), torch.empty_like(u)
    gws, grho = torch.empty_like(ww), torch.empty_like(u)
    info = pp.pressure_solve_adjoint(R.plan.handle, d["rho"], p, w.dt, gu, gv, gw, gus, gvs, gws, grho,
                                     rtol=1e-13, maxit=50000)
    assert info["status"] == 0
    grads = {"us": gus, "vs": gvs, "ws": gws, "rho": grho}

    def dloss(plus, minus):
        # L(+) - L(-) summed as (a - b)(a + b - 2 t): no cancellation of large L
        s = 0.0
        for a, b, t in zip(plus[:3], minus[:3], tgt):
            if a.shape[0] == w.nz + 1:
                a, b, t = a[1:-1], b[1:-1], t[1:-1]
            s += float(((a - b) * (a + b - 2 * t)).sum())
        return s

    rng = np.random.Generator(np.random.PCG64(1005 + 30))
    worst = 0.0
    scale = {k: float(grads[k].abs().max()) for k in grads}
    for name, count in (("us", 8), ("vs", 8), ("ws", 8), ("rho", 8)):
        shape = base[name].shape
        for _ in range(count):
            kk = int(rng.integers(1, shape[0] - 1)) if name == "ws" else int(rng.integers(0, shape[0]))
            idx = (kk, int(rng.integers(0, shape[1])), int(rng.integers(0, shape[2])))
            x0 = float(base[name][idx])
            eps = 1e-6 * max(1.0, abs(x0))
            fp = dict(d); fp[name] = d[name].clone(); fp[name][idx] = x0 + eps
            plus = project(fp)
            fm = dict(d); fm[name] = d[name].clone(); fm[name][idx] = x0 - eps
            minus = project(fm)
            fd = dloss(plus, minus) / (2 * eps)
            err = abs(fd - float(grads[name][idx])) / scale[name]
            worst = max(worst, err)
    print("adjoint vs central differences, worst error / max|grad|:", worst)
    assert worst < 1e-5

    # dot-product identity along one random direction of (u*, rho)
    dirs = {k: torch.from_numpy(rng.standard_normal(base[k].shape)).cuda() for k in base}
    dirs["ws"][0] = 0.0
    dirs["ws"][-1] = 0.0
    dirs["rho"] *= 1e-3 * float(d["rho"].abs().mean())
    eps = 1e-6
    plus = project({k: d[k] + eps * dirs[k] for k in d})
    minus = project({k: d[k] - eps * dirs[k] for k in d})
    gbar = [torch.from_numpy(rng.standard_normal(a.shape)).cuda() for a in (w.us, w.vs, w.ws)]
    jd = [(a - b) / (2 * eps) for a, b in zip(plus[:3], minus[:3])]
    lhs = sum(float((x[1:-1] * y[1:-1]).sum()) if x.shape[0] == w.nz + 1 else float((x * y).sum())
              for x, y in zip(jd, gbar))
    gbar[2][0] = 0.0
    gbar[2][-1] = 0.0
    info = pp.pressure_solve_adjoint(R.plan.handle, d["rho"], p, w.dt, gbar[0], gbar[1], gbar[2], gus, gvs,
                                     gws, grho, rtol=1e-13, maxit=50000)
    assert info["status"] == 0
    rhs = float((dirs["us"] * gus).sum() + (dirs["vs"] * gvs).sum() + (dirs["ws"] * gws).sum()
                + (dirs["rho"] * grho).sum())
    print("dot-product identity:", lhs, rhs, abs(lhs - rhs) / abs(rhs))
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs)
