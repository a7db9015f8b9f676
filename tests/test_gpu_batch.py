"""Batched projections (one graph launch for several grids of different
sizes) against single-grid plans and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    from paper_2005_11806_gb300 import pressure
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    pressure.lib()
    return pressure


def _cases(ratio):
    specs = [(16, 16, 24, None, 1), (24, 20, 16, 1.5, 2), (32, 32, 40, None, 3), (20, 30, 12, 2.0, 4),
             (48, 40, 36, 1.5, 5)]
    out = []
    for nx, ny, nz, beta, seed in specs:
        w = wl.small_bubble_case(nx, seed=1200 + seed, rho_ratio=ratio, stretched=beta is not None,
                                 nz=nz, ny=ny, nbubbles=1)
        out.append((w, orc.mixture_density(w.phi, w.rho_g, w.rho_l)))
    return out


def _pack(batch, cases):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    cell = lambda attr: dev(np.concatenate([getattr(w, attr).ravel() for w, _ in cases]))  # noqa: E731
    us, vs, S = cell("us"), cell("vs"), cell("S")
    ws = dev(np.concatenate([w.ws.ravel() for w, _ in cases]))
    rho = dev(np.concatenate([r.ravel() for _, r in cases]))
    assert us.numel() == batch.ncell and ws.numel() == batch.nwface
    return us, vs, ws, rho, S


def _unpack(batch, cases, p, u, v, w):
    out = []
    for k, (wk, _) in enumerate(cases):
        c0, w0 = batch.cell_offset[k], batch.wface_offset[k]
        nc, nw = wk.npts, (wk.nz + 1) * wk.ny * wk.nx
        out.append((p[c0:c0 + nc].reshape(wk.shape).cpu().numpy(), u[c0:c0 + nc].reshape(wk.shape).cpu().numpy(),
                    v[c0:c0 + nc].reshape(wk.shape).cpu().numpy(),
                    w[w0:w0 + nw].reshape(wk.nz + 1, wk.ny, wk.nx).cpu().numpy()))
    return out


def _run_batch(pp, cases, rtol, maxit):
    grids = [dict(nx=w.nx, ny=w.ny, nz=w.nz, lx=w.lx, ly=w.ly, lz=float(w.zf[-1]), zfaces=w.zf, ywalls=w.ywalls)
             for w, _ in cases]
    batch = pp.Batch(grids)
    us, vs, ws, rho, S = _pack(batch, cases)
    p, u, v = (torch.empty(batch.ncell, dtype=torch.float64, device="cuda") for _ in range(3))
    w = torch.empty(batch.nwface, dtype=torch.float64, device="cuda")
    infos = batch.correct(us, vs, ws, rho, S, cases[0][0].dt, p, u, v, w, rtol=rtol, maxit=maxit,
                          allow_not_converged=(rtol == 0.0))
    res = _unpack(batch, cases, p, u, v, w)
    batch.close()
    return infos, res


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_batch_matches_single_grid_plans(pp):
    """Fixed pass count: each batch member equals a single-grid mixed plan."""
    cases = _cases(1000.0)
    infos, res = _run_batch(pp, cases, 0.0, 30)
    for k, (w, rho) in enumerate(cases):
        assert infos[k]["iters"] == 30
        plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1]), zfaces=w.zf, precision="mixed")
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        u, v = torch.empty_like(p), torch.empty_like(p)
        ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
        pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt, p, u, v, ww,
                            rtol=0.0, maxit=30, allow_not_converged=True)
        for got, ref in zip(res[k], (p, u, v, ww)):
            assert _rel(got, ref.cpu().numpy()) < 1e-12, k
        plan.close()


def test_batch_converged_vs_oracle(pp):
    """Every member reaches rel. residual 1e-10 (checked in FP64 by the
    oracle's divergence) and matches the oracle's converged projection."""
    cases = _cases(10.0)
    infos, res = _run_batch(pp, cases, 1e-10, 2000)
    for k, (w, rho) in enumerate(cases):
        assert infos[k]["status"] == 0 and infos[k]["res_final"] <= 1e-10
        g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
        p0, u0, v0, w0, _ = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=3000)
        Sc = w.S - orc.volume_mean(g, w.S)
        d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
        _, u, v, ww = res[k]
        assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-10 * np.linalg.norm(d0)
        for a, b in ((u, u0), (v, v0), (ww, w0)):
            assert _rel(a, b) < 1e-9


def _mixed_wall_cases(ratio):
    """Periodic and walled-y grids in one batch (ducts: walls in y and z)."""
    out = _cases(ratio)[:2]
    for nx, ny, nz, stretched, seed in ((24, 20, 18, True, 1), (32, 30, 16, False, 2), (16, 12, 20, True, 3)):
        w = wl.channel_bubble_case(nx, ny, nz, seed=1300 + seed, rho_ratio=ratio, stretched=stretched)
        out.append((w, orc.mixture_density(w.phi, w.rho_g, w.rho_l)))
    return out


def test_batch_walls_in_y_match_single_grid_plans(pp):
    """A batch that mixes periodic and walled-y grids (the cosine y basis for
    the latter): fixed pass count, each member equals its single-grid plan."""
    cases = _mixed_wall_cases(1000.0)
    infos, res = _run_batch(pp, cases, 0.0, 25)
    for k, (w, rho) in enumerate(cases):
        assert infos[k]["iters"] == 25
        plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1]), zfaces=w.zf, precision="mixed",
                       ywalls=w.ywalls)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        p = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        u, v = torch.empty_like(p), torch.empty_like(p)
        ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
        pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), dev(rho), dev(w.S), w.dt, p, u, v, ww,
                            rtol=0.0, maxit=25, allow_not_converged=True)
        for got, ref in zip(res[k], (p, u, v, ww)):
            assert _rel(got, ref.cpu().numpy()) < 1e-12, k
        if w.ywalls:
            assert np.all(res[k][2][:, 0, :] == 0.0)
        plan.close()


def test_batch_walls_in_y_converged_vs_oracle(pp):
    cases = _mixed_wall_cases(10.0)
    infos, res = _run_batch(pp, cases, 1e-10, 3000)
    for k, (w, rho) in enumerate(cases):
        assert infos[k]["status"] == 0 and infos[k]["res_final"] <= 1e-10
        g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=w.ywalls)
        p0, u0, v0, w0, _ = orc.method3(g, w.us, w.vs, w.ws, rho, w.S, w.dt, rtol=1e-13, maxit=4000)
        Sc = w.S - orc.volume_mean(g, w.S)
        d0 = orc.divergence(g, w.us, w.vs, w.ws) - Sc
        _, u, v, ww = res[k]
        assert np.linalg.norm(orc.divergence(g, u, v, ww) - Sc) <= 1.0001e-10 * np.linalg.norm(d0)
        for a, b in ((u, u0), (v, v0), (ww, w0)):
            assert _rel(a, b) < 1e-9
