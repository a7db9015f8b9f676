"""The divergence source from the thermodynamics on the GPU (Eq. 30 for the
rate of p0, Eq. v_gas, the extrapolation of dp0/dt in Sec. 3.3, Eq. 34 for
S), through the C ABI, against the oracle.  FP64 throughout: 1e-12
relative (L2 for S, absolute-relative for the scalar rate)."""
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


def _fields(w, seed):
    """Temperature and conductivity: warm gas, cool liquid, smooth noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = 1.0 + 0.3 * w.phi + 0.05 * rng.standard_normal(w.shape)
    kc = 0.02 + 0.5 * (1.0 - w.phi) + 0.01 * rng.uniform(0, 1, w.shape)
    return T, kc


@pytest.mark.parametrize("dims,stretched", [((32, None, None), False), ((24, 20, 18), True), ((40, 30, 25), True)])
def test_p0_rate_and_source_vs_oracle(pp, dims, stretched):
    n, ny, nz = dims
    w = wl.small_bubble_case(n, seed=1102, rho_ratio=1000.0, stretched=stretched, nz=nz, ny=ny)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    T, kc = _fields(w, 1103)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf)
    gamma, p0 = 1.4, 1.05
    rp = pp.pressure_p0_rate(plan.handle, dev(w.phi), dev(kc), dev(T), dev(w.us), dev(w.vs), dev(w.ws), p0, gamma)
    rp0 = orc.p0_rate(g, w.phi, kc, T, w.us, w.vs, w.ws, p0, gamma)
    assert abs(rp - rp0) <= TOL * max(abs(rp0), 1e-300) * 10
    dp0dt = pp.pressure_dp0dt_extrapolate(rp, 0.9 * rp, 1.2e-3, 1e-3)
    assert dp0dt == pytest.approx(orc.dp0dt_extrapolate(rp, 0.9 * rp, 1.2e-3, 1e-3), rel=1e-15)
    S = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_divergence_source(plan.handle, dev(w.phi), dev(kc), dev(T), p0, gamma, dp0dt, S)
    S0 = orc.divergence_source(g, w.phi, kc, T, p0, gamma, dp0dt)
    assert _rel(host(S), S0) < TOL
    # host pointers: staged through the plan, same result
    Sh = np.empty(w.shape)
    pp.pressure_divergence_source(plan.handle, w.phi, kc, T, p0, gamma, dp0dt, Sh)
    assert np.array_equal(Sh, host(S))
    rph = pp.pressure_p0_rate(plan.handle, w.phi, kc, T, w.us, w.vs, w.ws, p0, gamma)
    assert rph == rp


@pytest.mark.parametrize("dims", [(24, 16, 18), (40, 30, 25)])
def test_p0_rate_and_source_with_walls_in_y(pp, dims):
    """Walls in y (a duct, stretched z): the rate of p0 and S against the
    oracle, whose conduction has no flux through the y walls and whose
    divergence reads the wall row of v as zero (set to 0.7 here, ignored)."""
    nx, ny, nz = dims
    w = wl.channel_bubble_case(nx, ny, nz, seed=1204, rho_ratio=1000.0, stretched=True)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=True)
    T, kc = _fields(w, 1105)
    vs = w.vs.copy()
    vs[:, 0, :] = 0.7
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf, ywalls=True)
    gamma, p0 = 1.4, 0.95
    rp = pp.pressure_p0_rate(plan.handle, dev(w.phi), dev(kc), dev(T), dev(w.us), dev(vs), dev(w.ws), p0, gamma)
    rp0 = orc.p0_rate(g, w.phi, kc, T, w.us, vs, w.ws, p0, gamma)
    assert abs(rp - rp0) <= TOL * max(abs(rp0), 1e-300) * 10
    S = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_divergence_source(plan.handle, dev(w.phi), dev(kc), dev(T), p0, gamma, 0.3 * rp, S)
    assert _rel(host(S), orc.divergence_source(g, w.phi, kc, T, p0, gamma, 0.3 * rp)) < TOL


@pytest.mark.parametrize("dims,ybeta", [((24, 16, 18), 1.5), ((20, 21, 12), 2.0)])
def test_p0_rate_and_source_on_a_stretched_y(pp, dims, ybeta):
    """A duct with tanh-clustered y faces: the conduction takes the row
    widths and centre distances, the volume sums the row widths (the
    oracle's D, G and cell volumes on the same faces)."""
    nx, ny, nz = dims
    w = wl.channel_bubble_case(nx, ny, nz, seed=1206, rho_ratio=1000.0, stretched=True, ybeta=ybeta)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf, ywalls=True, yf=w.yf)
    T, kc = _fields(w, 1107)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf, ywalls=True,
                   yfaces=w.yf)
    gamma, p0 = 1.4, 1.1
    rp = pp.pressure_p0_rate(plan.handle, dev(w.phi), dev(kc), dev(T), dev(w.us), dev(w.vs), dev(w.ws), p0, gamma)
    rp0 = orc.p0_rate(g, w.phi, kc, T, w.us, w.vs, w.ws, p0, gamma)
    assert abs(rp - rp0) <= TOL * max(abs(rp0), 1e-300) * 10
    S = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_divergence_source(plan.handle, dev(w.phi), dev(kc), dev(T), p0, gamma, 0.2 * rp, S)
    assert _rel(host(S), orc.divergence_source(g, w.phi, kc, T, p0, gamma, 0.2 * rp)) < TOL


def test_source_feeds_the_projection(pp):
    """S from Eq. 34 is the divergence the projection then imposes:
    D u^{n+1} = S_c to 1e-12 (oracle divergence)."""
    w = wl.small_bubble_case(24, seed=1102, rho_ratio=100.0, stretched=True, nz=20)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    T, kc = _fields(w, 1104)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf)
    S = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_divergence_source(plan.handle, dev(w.phi), dev(kc), dev(T), 1.0, 1.4, 1e-2, S)
    rho = dev(orc.mixture_density(w.phi, w.rho_g, w.rho_l))
    p, u, v = (torch.empty(w.shape, dtype=torch.float64, device="cuda") for _ in range(3))
    ww = torch.empty((w.nz + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    info = pp.pressure_correct(plan.handle, dev(w.us), dev(w.vs), dev(w.ws), rho, S, w.dt, p, u, v, ww,
                               rtol=1e-12, maxit=5000)
    assert info["status"] == 0
    Sh = host(S)
    Sc = Sh - orc.volume_mean(g, Sh)
    d0 = np.linalg.norm((orc.divergence(g, w.us, w.vs, w.ws) - Sc).ravel())
    d = np.linalg.norm((orc.divergence(g, host(u), host(v), host(ww)) - Sc).ravel())
    assert d <= 1.0001e-12 * d0


def test_no_gas_and_bad_arguments(pp):
    w = wl.small_bubble_case(16, seed=1102)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf)
    z = dev(np.zeros(w.shape))
    wz = dev(np.zeros((w.nz + 1, w.ny, w.nx)))
    one = dev(np.ones(w.shape))
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_p0_rate(plan.handle, z, one, one, z, z, wz, 1.0, 1.4)
    assert e.value.code == pp.PP_ERR_NUMERIC
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_divergence_source(plan.handle, one, one, one, 0.0, 1.4, 0.0, z)
    assert e.value.code == pp.PP_ERR_INVALID_ARG
    with pytest.raises(pp.PressureError) as e:
        pp.pressure_dp0dt_extrapolate(1.0, 1.0, 1e-3, 0.0)
    assert e.value.code == pp.PP_ERR_INVALID_ARG


@pytest.mark.slow
def test_fullsize_bubbles512_source(pp):
    """512^3 benchmark field: with a uniform temperature, Eq. 34 gives the
    benchmark's own source (gas only, rate 1e-2, gamma 1.4, p0 1); with
    the conduction term, S and the rate match the oracle at every cell."""
    w = wl.bubbles_case(n=512, nbubbles=200, seed=1003, beta=1.5, rho_g=1.0, rho_l=1000.0)
    g = orc.Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.zf)
    plan = pp.Plan(w.nx, w.ny, w.nz, w.lx, w.ly, float(w.zf[-1] - w.zf[0]), zfaces=w.zf, precision="mixed")
    phi = dev(w.phi)
    S = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    pp.pressure_divergence_source(plan.handle, phi, dev(np.ones(w.shape)), dev(np.full(w.shape, 1.3)), 1.0, 1.4,
                                  1e-2, S)
    assert _rel(host(S), w.S) < 1e-15
    T, kc = _fields(w, 1105)
    pp.pressure_divergence_source(plan.handle, phi, dev(kc), dev(T), 1.0, 1.4, 1e-2, S)
    assert _rel(host(S), orc.divergence_source(g, w.phi, kc, T, 1.0, 1.4, 1e-2)) < TOL
    rp = pp.pressure_p0_rate(plan.handle, phi, dev(kc), dev(T), dev(w.us), dev(w.vs), dev(w.ws), 1.0, 1.4)
    rp0 = orc.p0_rate(g, w.phi, kc, T, w.us, w.vs, w.ws, 1.0, 1.4)
    assert abs(rp - rp0) <= 1e-10 * abs(rp0)
