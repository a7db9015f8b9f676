"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each test names the plausible mistake it would catch.
"""
import math

import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl
from tests import dense_reference as dr


def _grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, beta=None):
    zf = wl.uniform_zfaces(nz, lz) if beta is None else wl.tanh_zfaces(nz, lz, beta)
    return orc.Grid(nx, ny, nz, lx, ly, zf)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# --- constant-coefficient solve -------------------------------------------

@pytest.mark.parametrize("dims,mode,phase", [
    ((32, 32, 32), (3, 5, 2), (0.0, 0.0)),
    ((24, 20, 16), (3, 2, 1), (0.3, -1.1)),
    ((17, 12, 9), (4, 5, 7), (0.7, 0.2)),      # odd nx, Nyquist-free
])
def test_single_mode_closed_form(dims, mode, phase):
    """Discrete eigenmode: L f = lambda f exactly, so p = f / lambda.  Catches
    wrong modified wavenumbers, a swapped axis, a wrong Neumann end row or a
    wrong DFT sign/normalisation."""
    nx, ny, nz = dims
    lx, ly, lz = 1.0, 1.5, 0.7
    g = _grid(nx, ny, nz, lx, ly, lz)
    a, b, c = mode
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    f = (np.cos(2 * np.pi * a * i / nx + phase[0]) * np.cos(2 * np.pi * b * j / ny + phase[1])
         * np.cos(np.pi * c * (k + 0.5) / nz))
    dx, dy, dz = lx / nx, ly / ny, lz / nz
    lam = -(4 / dx ** 2 * math.sin(math.pi * a / nx) ** 2 + 4 / dy ** 2 * math.sin(math.pi * b / ny) ** 2
            + 4 / dz ** 2 * math.sin(math.pi * c / (2 * nz)) ** 2)
    p = orc.solve_constant(g, f)
    assert _rel(p, f / lam) < 1e-12
    assert _rel(orc.laplacian(g, f), lam * f) < 1e-12


@pytest.mark.parametrize("dims,beta", [((8, 8, 8), None), ((8, 8, 8), 1.5), ((6, 5, 7), 2.0)])
def test_constant_solve_vs_dense_lu(dims, beta):
    """Dense LU of the 7-point matrix assembled entry by entry; catches any
    error in the z coefficients on stretched grids and in the zero-mode gauge."""
    nx, ny, nz = dims
    lx, ly, lz = 1.0, 0.8, 1.3
    g = _grid(nx, ny, nz, lx, ly, lz, beta)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(g.shape)
    A = dr.assemble_variable(nx, ny, nz, lx, ly, g.zf, None)
    wts = dr.cell_weights(nx, ny, nz, g.zf)
    fc = f.ravel() - np.dot(wts, f.ravel()) / wts.sum()
    p_lu = dr.bordered_solve(A, fc, wts).reshape(g.shape)
    p = orc.solve_constant(g, f)
    assert _rel(p, p_lu) < 1e-12
    # residual of the 7-point equation, evaluated with the assembled matrix
    assert np.linalg.norm(A @ p.ravel() - fc) / np.linalg.norm(fc) < 1e-12


def test_operator_identities_stretched():
    """Linear fields: D of w = z_face is exactly 1, G of p = z_centre is
    exactly 1 on interior z faces and 0 on the walls; G of a constant is 0.
    Catches dzf/dzc mix-ups and an off-by-one face index."""
    g = _grid(6, 5, 9, beta=1.5)
    zero = np.zeros(g.shape)
    w = np.broadcast_to(g.zf[:, None, None], (g.nz + 1, g.ny, g.nx)).copy()
    assert np.allclose(orc.divergence(g, zero, zero, w), 1.0, rtol=0, atol=1e-12)
    p = np.broadcast_to(g.zc[:, None, None], g.shape).copy()
    gx, gy, gz = orc.gradient(g, p)
    assert np.allclose(gz[1:-1], 1.0, atol=1e-12) and np.all(gz[0] == 0) and np.all(gz[-1] == 0)
    assert np.allclose(gx, 0) and np.allclose(gy, 0)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(g.shape)
    v = rng.standard_normal(g.shape)
    w = rng.standard_normal((g.nz + 1, g.ny, g.nx))
    ref = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, u, v, w)
    assert np.allclose(orc.divergence(g, u, v, w), ref, rtol=0, atol=1e-10)


def test_summation_by_parts_weights():
    """sum_f W_f (G p) y = -sum_c W_c p (D y) for y with no wall flux: the
    weighted transpose relation D^T = -W_f G W_c^{-1} used by the adjoint."""
    g = _grid(5, 6, 7, beta=2.0)
    rng = np.random.default_rng(11)
    p = rng.standard_normal(g.shape)
    yu, yv = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    yw = rng.standard_normal((g.nz + 1, g.ny, g.nx))
    yw[0] = yw[-1] = 0
    gx, gy, gz = orc.gradient(g, p)
    wl_ = g.dzf[:, None, None]
    wz = np.ones(g.nz + 1); wz[1:-1] = g.dzc[1:-1]
    lhs = np.sum(wl_ * gx * yu) + np.sum(wl_ * gy * yv) + np.sum(wz[:, None, None] * gz * yw)
    rhs = -np.sum(wl_ * p * orc.divergence(g, yu, yv, yw))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


# --- variable-density projection ------------------------------------------

def _small_case(nx, ny, nz, beta=None, ratio=1000.0, seed=5, S_on=True, lz=1.0):
    g = _grid(nx, ny, nz, 1.0, ny / nx, lz, beta)
    rng = np.random.default_rng(seed)
    phi = np.zeros(g.shape)
    # a blob of gas plus one interface layer
    phi[nz // 4:nz // 2 + 1, ny // 4:ny // 2 + 1, nx // 3:2 * nx // 3 + 1] = 1.0
    phi[nz // 2 + 1, ny // 4:ny // 2, nx // 3:2 * nx // 3] = 0.4
    rho = orc.mixture_density(phi, 1.0, ratio)
    us, vs, ws = (rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1,
                  rng.standard_normal((nz + 1, ny, nx)) * 0.1)
    ws[0] = ws[-1] = 0
    S = wl.gas_source(phi) if S_on else np.zeros(g.shape)
    return g, us, vs, ws, rho, S


def test_mixture_density_endpoints():
    assert np.allclose(orc.mixture_density(np.array([0.0, 1.0, 0.25]), 1.2, 1000.0),
                       [1000.0, 1.2, 0.25 * 1.2 + 0.75 * 1000.0])


@pytest.mark.parametrize("beta", [None, 1.5])
def test_projection_direct_vs_dense(beta):
    """Plain definition (sparse) vs a dense LU of D(beta G) assembled entry by
    entry with arithmetic face densities; catches a harmonic/other face
    average, a missing 1/dt or a wrong correction sign."""
    g, us, vs, ws, rho, S = _small_case(5, 4, 6, beta)
    dt = 1e-3
    p, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    A = dr.assemble_variable(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, rho)
    wts = dr.cell_weights(g.nx, g.ny, g.nz, g.zf)
    Sc = S.ravel() - np.dot(wts, S.ravel()) / wts.sum()
    div = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, us, vs, ws).ravel()
    p_lu = dr.bordered_solve(A, (div - Sc) / dt, wts).reshape(g.shape)
    assert _rel(p, p_lu) < 1e-11
    # the corrected field meets the divergence target exactly
    dnew = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, u, v, w).ravel()
    assert np.max(np.abs(dnew - Sc)) < 1e-11 * np.max(np.abs(div))


@pytest.mark.parametrize("beta,ratio", [(None, 1000.0), (1.5, 1000.0), (None, 10.0)])
def test_method3_reaches_direct_solution(beta, ratio):
    """Algorithm 1 converges to the plain definition (its fixed point is the
    discrete Eq. lap_p exactly, as the paper states for Method III)."""
    g, us, vs, ws, rho, S = _small_case(12, 10, 14, beta, ratio)
    dt = 1e-3
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-13)
    assert info["res_hist"][-1] <= 1e-13
    pd, ud, vd, wd = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    assert _rel(p, pd) < 1e-10
    for a, b in ((u, ud), (v, vd), (w, wd)):
        assert _rel(a, b) < 1e-11


def test_projection_invariants():
    """D u^{n+1} = S_c, sum S_c dV = 0, idempotence and rho_f-weighted
    orthogonality of the correction (S = 0)."""
    g, us, vs, ws, rho, S = _small_case(16, 16, 16, 1.5, 1000.0)
    dt = 1e-3
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-13)
    Sc = S - orc.volume_mean(g, S)
    assert abs(np.sum(Sc * g.cell_volume())) < 1e-15 * np.sum(np.abs(S))
    d0 = orc.divergence(g, us, vs, ws)
    assert np.max(np.abs(orc.divergence(g, u, v, w) - Sc)) < 1e-12 * np.max(np.abs(d0))
    # S = 0: orthogonality and idempotence
    zero = np.zeros(g.shape)
    p1, u1, v1, w1, _ = orc.method3(g, us, vs, ws, rho, zero, dt, rtol=1e-13)
    rx, ry, rz = orc.face_density(g, rho)
    wl_ = g.dzf[:, None, None]
    wz = np.ones(g.nz + 1); wz[1:-1] = g.dzc[1:-1]
    dot = (np.sum(wl_ * rx * (us - u1) * u1) + np.sum(wl_ * ry * (vs - v1) * v1)
           + np.sum(wz[:, None, None] * rz * (ws - w1) * w1))
    scale = np.sum(wl_ * rx * u1 * u1) + np.sum(wl_ * ry * v1 * v1)
    assert abs(dot) < 1e-11 * scale
    # u1 already meets the constraint to round-off: projecting it again
    # (a few passes) leaves it unchanged and gives a vanishing pressure.
    p2, u2, v2, w2, info2 = orc.method3(g, u1, v1, w1, rho, zero, dt, rtol=1e-10, maxit=3)
    assert _rel(u2, u1) < 1e-12
    assert np.max(np.abs(p2)) < 1e-10 * np.max(np.abs(p1))


def test_constant_density_one_iteration():
    """rho = const: Method III's right-hand side is exact after one pass and
    equals the constant-coefficient projection with p scaled by rho."""
    g = _grid(16, 12, 10, beta=1.5)
    rng = np.random.default_rng(2)
    us, vs = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    ws = rng.standard_normal((g.nz + 1, g.ny, g.nx)); ws[0] = ws[-1] = 0
    rho = np.full(g.shape, 3.0)
    S = np.zeros(g.shape)
    dt = 1e-3
    p, u, v, wv, info = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-12)
    assert info["iters"] == 1
    pc = orc.solve_constant(g, orc.divergence(g, us, vs, ws) / dt) * 3.0
    assert _rel(p, pc) < 1e-12


@pytest.mark.parametrize("method", ["method1", "method2"])
def test_methods_1_2_reach_direct_solution(method):
    """Methods I and II converge to the same discrete solution (their fixed
    point is Eq. lap_p too); Method I's modified correction then agrees with
    Eq. corr to the tolerance."""
    g, us, vs, ws, rho, S = _small_case(12, 10, 14, 1.5, 10.0)
    dt = 1e-3
    p, u, v, w, info = getattr(orc, method)(g, us, vs, ws, rho, S, dt, rtol=1e-13)
    assert info["res_hist"][-1] <= 1e-13
    pd, ud, vd, wd = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    assert _rel(p, pd) < 1e-10
    for a, b in ((u, ud), (v, vd), (w, wd)):
        assert _rel(a, b) < 1e-10


def test_methods_share_first_pass_with_constant_density():
    """rho = const: all three scalings coincide and one pass is exact."""
    g = _grid(10, 8, 12, beta=1.5)
    rng = np.random.default_rng(12)
    us, vs = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    ws = rng.standard_normal((g.nz + 1, g.ny, g.nx)); ws[0] = ws[-1] = 0
    rho = np.full(g.shape, 2.0)
    S = np.zeros(g.shape)
    out = [f(g, us, vs, ws, rho, S, 1e-3, rtol=1e-12) for f in (orc.method1, orc.method2, orc.method3)]
    for p, u, v, w, info in out:
        assert info["iters"] == 1
        assert _rel(p, out[2][0]) < 1e-12


# --- adjoint --------------------------------------------------------------

def _loss(g, us, vs, ws, rho, S, dt, tgt):
    _, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    return float(np.sum((u - tgt[0]) ** 2) + np.sum((v - tgt[1]) ** 2)
                 + np.sum((w[1:-1] - tgt[2][1:-1]) ** 2))


def test_adjoint_central_differences():
    """adjoint_direct vs central differences of the projection (eps = 1e-6
    relative), on entries of u*, v*, w* and rho."""
    g, us, vs, ws, rho, S = _small_case(5, 4, 6, 2.0, 100.0, seed=9, lz=0.5)
    dt = 1e-3
    rng = np.random.default_rng(21)
    tgt = (rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1,
           rng.standard_normal((g.nz + 1, g.ny, g.nx)) * 0.1)
    _, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    gu, gv, gw = 2 * (u - tgt[0]), 2 * (v - tgt[1]), 2 * (w - tgt[2])
    gus, gvs, gws, grho = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    checks = [("u", (1, 2, 3)), ("v", (4, 1, 0)), ("w", (3, 2, 2)), ("rho", (2, 1, 2)),
              ("rho", (1, 1, 1)), ("rho", (3, 3, 4))]
    for name, idx in checks:
        arrs = {"u": us, "v": vs, "w": ws, "rho": rho}
        base = arrs[name]
        h = 1e-6 * max(1.0, abs(base[idx]))
        plus = base.copy(); plus[idx] += h
        minus = base.copy(); minus[idx] -= h
        args_p = dict(us=us, vs=vs, ws=ws, rho=rho); args_m = dict(args_p)
        key = {"u": "us", "v": "vs", "w": "ws", "rho": "rho"}[name]
        args_p[key] = plus; args_m[key] = minus
        fd = (_loss(g, args_p["us"], args_p["vs"], args_p["ws"], args_p["rho"], S, dt, tgt)
              - _loss(g, args_m["us"], args_m["vs"], args_m["ws"], args_m["rho"], S, dt, tgt)) / (2 * h)
        an = {"u": gus, "v": gvs, "w": gws, "rho": grho}[name][idx]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.max(np.abs(gus))), (name, idx, fd, an)


def test_adjoint_dot_product_and_method3():
    """<P d, g> = <d, P^T g> for the velocity part, and the Algorithm-1 form
    of the adjoint (weighted transposes) equals the literal sparse one."""
    g, us, vs, ws, rho, S = _small_case(8, 6, 10, 2.0, 100.0, seed=4, lz=0.5)
    dt = 1e-3
    rng = np.random.default_rng(8)
    gu, gv = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    gw = rng.standard_normal((g.nz + 1, g.ny, g.nx)); gw[0] = gw[-1] = 0
    du, dv = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    dw = rng.standard_normal((g.nz + 1, g.ny, g.nx)); dw[0] = dw[-1] = 0
    zero = np.zeros(g.shape)
    _, pu, pv, pw = orc.projection_direct(g, du, dv, dw, rho, zero, dt)
    a1, a2, a3, grho = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    lhs = np.sum(pu * gu) + np.sum(pv * gv) + np.sum(pw * gw)
    rhs = np.sum(du * a1) + np.sum(dv * a2) + np.sum(dw * a3)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    b1, b2, b3, brho, _ = orc.adjoint_method3(g, us, vs, ws, rho, S, dt, gu, gv, gw, rtol=1e-13)
    for x, y in ((b1, a1), (b2, a2), (b3, a3), (brho, grho)):
        assert _rel(x, y) < 1e-9


# --- planted mistakes: the pins above must catch them ---------------------

def test_planted_harmonic_face_density_is_caught(monkeypatch):
    orig = orc.face_density

    def planted(g, rho):
        rx = 2.0 / (1.0 / rho + 1.0 / np.roll(rho, 1, axis=2))
        _, ry, rz = orig(g, rho)
        return rx, ry, rz
    monkeypatch.setattr(orc, "face_density", planted)
    with pytest.raises(AssertionError):
        test_projection_direct_vs_dense(None)


def test_planted_gradient_sign_is_caught(monkeypatch):
    orig = orc.gradient

    def planted(g, p):
        gx, gy, gz = orig(g, p)
        return gx, gy, -gz
    monkeypatch.setattr(orc, "gradient", planted)
    with pytest.raises(AssertionError):
        test_single_mode_closed_form((24, 20, 16), (3, 2, 1), (0.3, -1.1))


# --- divergence source from the thermodynamics (Eqs. 30, 34, v_gas) -------

def test_conduction_single_mode_closed_form():
    """Constant k on a uniform grid: D(k G T) of a discrete eigenmode is k
    times its modified-wavenumber eigenvalue (Neumann cosine in z)."""
    nx, ny, nz, a, b, c, kap = 16, 12, 10, 3, 2, 4, 2.5
    g = _grid(nx, ny, nz)
    i = np.arange(nx)[None, None, :]; j = np.arange(ny)[None, :, None]; k = np.arange(nz)[:, None, None]
    T = np.cos(2 * np.pi * a * i / nx) * np.cos(2 * np.pi * b * j / ny) * np.cos(np.pi * c * (k + 0.5) / nz)
    lam = -4 * (nx ** 2 * np.sin(np.pi * a / nx) ** 2 + ny ** 2 * np.sin(np.pi * b / ny) ** 2
                + nz ** 2 * np.sin(np.pi * c / (2 * nz)) ** 2)
    got = orc.conduction(g, np.full(g.shape, kap), T)
    assert _rel(got, kap * lam * T) < 1e-12


def test_conduction_matches_dense_assembly():
    """Variable k, stretched z: the array operator equals the matrix assembled
    entry by entry from the stencil definition."""
    nx, ny, nz = 6, 5, 7
    g = _grid(nx, ny, nz, 1.0, 0.8, 0.6, beta=1.5)
    rng = np.random.default_rng(30)
    kc = rng.uniform(0.5, 3.0, g.shape)
    T = rng.standard_normal(g.shape)
    A = dr.assemble_conduction(nx, ny, nz, 1.0, 0.8, g.zf, kc)
    assert _rel(orc.conduction(g, kc, T).ravel(), A @ T.ravel()) < 1e-13


def test_heat_is_conserved_in_a_closed_gas_box():
    """Adiabatic walls, periodic x/y: sum of div(k grad T) dV vanishes, so a
    box full of gas (Phi = 1) with no net dilatation has dp0/dt = 0."""
    g, us, vs, ws, rho, S = _small_case(12, 10, 9, beta=1.5)
    rng = np.random.default_rng(31)
    kc = rng.uniform(0.2, 2.0, g.shape)
    T = rng.uniform(0.5, 2.0, g.shape)
    cond = orc.conduction(g, kc, T)
    dv = g.cell_volume()
    assert abs(np.sum(cond * dv)) <= 1e-13 * np.sum(np.abs(cond) * dv)
    rp = orc.p0_rate(g, np.ones(g.shape), kc, T, us, vs, ws, p0=1.3, gamma=1.4)
    scale = (1.4 / orc.gas_volume(g, np.ones(g.shape))) * np.sum(np.abs(cond) * dv)
    assert abs(rp) <= 1e-13 * scale


def test_p0_rate_is_the_heat_flux_through_the_interface():
    """Gas below a flat interface (Phi = 1 for k < m, 0 above), u = 0: Eq. 30
    gives (gamma - 1)/V_g times the heat flowing into the gas through the
    interface faces, summed here face by face (discrete Gauss theorem)."""
    nx, ny, nz, m = 8, 6, 10, 4
    g = _grid(nx, ny, nz, 1.0, 0.75, 1.0, beta=1.5)
    rng = np.random.default_rng(32)
    kc = rng.uniform(0.5, 2.0, g.shape)
    T = rng.uniform(0.5, 2.0, g.shape)
    phi = np.zeros(g.shape); phi[:m] = 1.0
    zero = np.zeros(g.shape)
    gamma, p0 = 1.4, 0.9
    flux = 0.0
    for j in range(ny):
        for i in range(nx):
            kf = 0.5 * (kc[m, j, i] + kc[m - 1, j, i])
            flux += kf * (T[m, j, i] - T[m - 1, j, i]) / (g.zc[m] - g.zc[m - 1]) * g.dx * g.dy
    vg = float(np.sum(g.dzf[:m])) * g.lx * g.ly
    assert abs(orc.gas_volume(g, phi) - vg) <= 1e-14 * vg
    rp = orc.p0_rate(g, phi, kc, T, zero, zero, np.zeros((nz + 1, ny, nx)), p0, gamma)
    assert rp == pytest.approx((gamma - 1.0) / vg * flux, rel=1e-12)


def test_dp0dt_extrapolation_is_exact_for_a_linear_history():
    """The extrapolation of Sec. 3.3 reproduces a rate linear in time."""
    a, b, t, dt_old, dt_new = 0.3, -1.7, 2.0, 0.01, 0.013
    rp_n, rp_nm1 = a + b * t, a + b * (t - dt_old)
    assert orc.dp0dt_extrapolate(rp_n, rp_nm1, dt_new, dt_old) == pytest.approx(a + b * (t + dt_new), rel=1e-13)
    assert orc.dp0dt_extrapolate(0.25, 0.25, dt_new, dt_old) == pytest.approx(0.25, rel=1e-15)


def test_divergence_source_special_cases():
    """Eq. 34: zero in the liquid; a uniform temperature leaves only the
    pressure-rate term; the conduction term enters with (gamma - 1)/gamma."""
    g = _grid(8, 8, 8)
    rng = np.random.default_rng(33)
    phi = rng.uniform(0, 1, g.shape); phi[0] = 0.0
    kc = rng.uniform(0.5, 2.0, g.shape)
    gamma, p0, r = 1.4, 1.1, 0.02
    S = orc.divergence_source(g, phi, kc, np.full(g.shape, 1.7), p0, gamma, r)
    assert np.all(S[0] == 0.0)
    assert _rel(S, -phi * r / (gamma * p0)) < 1e-14
    T = rng.uniform(0.5, 2.0, g.shape)
    S0 = orc.divergence_source(g, phi, kc, T, p0, gamma, 0.0)
    assert _rel(S0 * p0, (gamma - 1) / gamma * phi * (dr.assemble_conduction(8, 8, 8, 1.0, 1.0, g.zf, kc)
                                                        @ T.ravel()).reshape(g.shape)) < 1e-12


# --- momentum predictor (Eqs. 29, 32; Newton-Stokes stress) -----------------

def _curl_field(g, seed):
    """A discretely divergence-free MAC field: the discrete curl of a vector
    potential on the cell edges, zero on the wall edges so that w = 0 on the
    walls."""
    nx, ny, nz = g.nx, g.ny, g.nz
    rng = np.random.default_rng(seed)
    Ax = rng.standard_normal((nz + 1, ny, nx)); Ay = rng.standard_normal((nz + 1, ny, nx))
    Az = rng.standard_normal((nz, ny, nx))
    Ax[0] = Ax[-1] = 0.0; Ay[0] = Ay[-1] = 0.0
    dzf = g.dzf[:, None, None]
    u = (np.roll(Az, -1, axis=1) - Az) / g.dy - (Ay[1:] - Ay[:-1]) / dzf
    v = (Ax[1:] - Ax[:-1]) / dzf - (np.roll(Az, -1, axis=2) - Az) / g.dx
    w = (np.roll(Ay, -1, axis=2) - Ay) / g.dx - (np.roll(Ax, -1, axis=1) - Ax) / g.dy
    return u, v, w


def test_convection_conserves_momentum_and_energy():
    """For a divergence-free field, the central divergence form conserves x
    and y momentum and the kinetic energy (uniform grid, the paper's)."""
    g = _grid(12, 10, 9, 1.0, 0.8, 0.6)
    u, v, w = _curl_field(g, 40)
    assert np.abs(orc.divergence(g, u, v, w)).max() < 1e-10
    cx, cy, cz = orc.convection(g, u, v, w)
    dv = g.cell_volume()
    dvw = (g.dx * g.dy * g.dzc)[:, None, None]
    scale = np.sum(np.abs(u * cx) * dv)
    assert abs(np.sum(cx * dv)) < 1e-13 * np.sum(np.abs(cx) * dv)
    assert abs(np.sum(cy * dv)) < 1e-13 * np.sum(np.abs(cy) * dv)
    energy = np.sum(u * cx * dv) + np.sum(v * cy * dv) + np.sum(w * cz * dvw)
    assert abs(energy) < 1e-13 * scale


def test_viscous_term_is_mu_laplacian_for_a_solenoidal_mode():
    """Constant mu, a divergence-free single Fourier mode in x and y with no
    z dependence: away from the walls div tau = mu * lambda * u with the
    modified-wavenumber eigenvalue (the transpose and -2/3 div u parts cancel)."""
    nx, ny, nz, a, b, mu = 16, 12, 6, 3, 2, 0.7
    g = _grid(nx, ny, nz, 1.0, 0.75, 0.5)
    xe = (np.arange(nx) - 0.5) * g.dx; ye = (np.arange(ny) - 0.5) * g.dy     # edge coordinates
    psi = np.sin(2 * np.pi * a * xe[None, None, :] / g.lx) * np.sin(2 * np.pi * b * ye[None, :, None] / g.ly)
    psi = np.broadcast_to(psi, (nz, ny, nx)).copy()
    u = (np.roll(psi, -1, axis=1) - psi) / g.dy
    v = -(np.roll(psi, -1, axis=2) - psi) / g.dx
    w = np.zeros((nz + 1, ny, nx))
    lam = -4 / g.dx ** 2 * np.sin(np.pi * a / nx) ** 2 - 4 / g.dy ** 2 * np.sin(np.pi * b / ny) ** 2
    fx, fy, fz = orc.viscous(g, np.full(g.shape, mu), u, v, w)
    assert _rel(fx[1:-1], mu * lam * u[1:-1]) < 1e-12
    assert _rel(fy[1:-1], mu * lam * v[1:-1]) < 1e-12
    assert np.abs(fz).max() < 1e-9 * np.abs(fx).max()


def test_viscous_shear_flow_is_the_conduction_operator():
    """u = u(z), v = w = 0, mu = mu(z): away from the walls the x component
    of div tau is d/dz(mu du/dz), the same operator as the pinned conduction
    term with k = mu (stretched z)."""
    nx, ny, nz = 6, 5, 12
    g = _grid(nx, ny, nz, 1.0, 1.0, 0.8, beta=1.5)
    rng = np.random.default_rng(41)
    uz = rng.standard_normal(nz); muz = rng.uniform(0.5, 2.0, nz)
    u = np.broadcast_to(uz[:, None, None], g.shape).copy()
    mu = np.broadcast_to(muz[:, None, None], g.shape).copy()
    zero = np.zeros(g.shape)
    fx, fy, fz = orc.viscous(g, mu, u, zero, np.zeros((nz + 1, ny, nx)))
    ref = orc.conduction(g, mu, u)
    assert _rel(fx[1:-1], ref[1:-1]) < 1e-12
    assert np.abs(fy).max() < 1e-12 and np.abs(fz).max() < 1e-12


def test_poiseuille_profile_gives_constant_viscous_force():
    """u = z (Lz - z), uniform z, constant mu and rho: no convection, and the
    viscous force is -2 mu in every layer off the walls (second differences
    are exact for a quadratic), so RU = -2 mu / rho + g there."""
    nx, ny, nz, mu, rho, lz = 8, 6, 10, 0.3, 2.0, 1.0
    g = _grid(nx, ny, nz, 1.0, 1.0, lz)
    u = np.broadcast_to((g.zc * (lz - g.zc))[:, None, None], g.shape).copy()
    zero = np.zeros(g.shape); wz = np.zeros((nz + 1, ny, nx))
    cx, cy, cz = orc.convection(g, u, zero, wz)
    assert max(np.abs(cx).max(), np.abs(cy).max(), np.abs(cz).max()) < 1e-14
    ru, rv, rw = orc.predictor_rhs(g, u, zero, wz, np.full(g.shape, rho), np.full(g.shape, mu), (0.1, 0.0, -9.81))
    assert np.allclose(ru[1:-1], -2 * mu / rho + 0.1, rtol=1e-12, atol=1e-12)
    assert np.allclose(rv, 0.0, atol=1e-13)
    assert np.allclose(rw[1:-1], -9.81, rtol=1e-13)
    assert rw[0].max() == 0.0 and rw[-1].max() == 0.0


def test_predictor_time_stepping():
    """Eq. 29: forward Euler on the first step; Adams-Bashforth with a
    constant RU history reduces to u + dt RU; a fluid at rest with variable
    density only feels gravity (rho g / rho = g)."""
    g = _grid(8, 8, 6, beta=1.5)
    rng = np.random.default_rng(42)
    rho = rng.uniform(1.0, 1000.0, g.shape); mu = rng.uniform(1e-3, 1.0, g.shape)
    zero = np.zeros(g.shape); wz = np.zeros((g.nz + 1, g.ny, g.nx))
    grav = (0.0, 0.5, -9.81)
    (us, vs, ws), ru = orc.predictor(g, zero, zero, wz, rho, mu, grav, 1e-3)
    assert np.allclose(us, 0.0) and np.allclose(vs, 0.5e-3, rtol=1e-14) and np.allclose(ws[1:-1], -9.81e-3, rtol=1e-14)
    u, v, w = _curl_field(g, 43)
    (a1, b1, c1), ru1 = orc.predictor(g, u, v, w, rho, mu, grav, 2e-3, 1e-3, ru_prev=orc.predictor_rhs(g, u, v, w, rho, mu, grav))
    assert _rel(a1, u + 2e-3 * ru1[0]) < 1e-14 and _rel(c1[1:-1], w[1:-1] + 2e-3 * ru1[2][1:-1]) < 1e-14


# --- walls in y ------------------------------------------------------------

def _ygrid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, beta=None):
    zf = wl.uniform_zfaces(nz, lz) if beta is None else wl.tanh_zfaces(nz, lz, beta)
    return orc.Grid(nx, ny, nz, lx, ly, zf, ywalls=True)


@pytest.mark.parametrize("dims,mode", [((16, 12, 10), (3, 5, 2)), ((10, 7, 6), (2, 6, 5)),
                                       ((8, 16, 8), (0, 1, 0))])
def test_ywalls_single_mode_closed_form(dims, mode):
    """cos(pi b (j + 1/2) / ny) is an eigenvector of the y second difference
    with Neumann ends, eigenvalue -(4/dy^2) sin^2(pi b / (2 ny)).  Catches the
    periodic wavenumber left in place, a DCT of the wrong type or scale, and
    the wall flux left open."""
    nx, ny, nz = dims
    lx, ly, lz = 1.0, 1.3, 0.6
    g = _ygrid(nx, ny, nz, lx, ly, lz)
    a, b, c = mode
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    f = np.cos(2 * np.pi * a * i / nx + 0.4) * np.cos(np.pi * b * (j + 0.5) / ny) * np.cos(np.pi * c * (k + 0.5) / nz)
    dx, dy, dz = lx / nx, ly / ny, lz / nz
    lam = -(4 / dx ** 2 * math.sin(math.pi * a / nx) ** 2 + 4 / dy ** 2 * math.sin(math.pi * b / (2 * ny)) ** 2
            + 4 / dz ** 2 * math.sin(math.pi * c / (2 * nz)) ** 2)
    assert _rel(orc.laplacian(g, f), lam * f) < 1e-12
    assert _rel(orc.solve_constant(g, f), f / lam) < 1e-12


@pytest.mark.parametrize("beta", [None, 1.5])
def test_ywalls_solve_is_the_even_extension_of_a_periodic_solve(beta):
    """Neumann walls in y are the mirror symmetry of a periodic problem of
    twice the width: reflect f about y = ly, solve periodically on 2 ny rows,
    keep the first ny.  No cosine transform on the right-hand side, so this
    pins the wall solve through the periodic one."""
    nx, ny, nz = 12, 10, 9
    g = _ygrid(nx, ny, nz, 1.0, 0.9, 1.0, beta)
    gp = orc.Grid(nx, 2 * ny, nz, 1.0, 1.8, g.zf)
    f = np.random.default_rng(21).standard_normal(g.shape)
    fe = np.concatenate([f, f[:, ::-1, :]], axis=1)
    assert _rel(orc.solve_constant(g, f), orc.solve_constant(gp, fe)[:, :ny, :]) < 1e-12


@pytest.mark.parametrize("dims,beta", [((6, 5, 4), None), ((4, 6, 5), 2.0)])
def test_ywalls_constant_solve_vs_dense_lu(dims, beta):
    """Dense LU of the 7-point matrix with no flux through the y walls,
    assembled entry by entry."""
    nx, ny, nz = dims
    lx, ly, lz = 1.0, 0.8, 1.3
    g = _ygrid(nx, ny, nz, lx, ly, lz, beta)
    f = np.random.default_rng(8).standard_normal(g.shape)
    A = dr.assemble_variable(nx, ny, nz, lx, ly, g.zf, None, ywalls=True)
    wts = dr.cell_weights(nx, ny, nz, g.zf)
    fc = f.ravel() - np.dot(wts, f.ravel()) / wts.sum()
    p = orc.solve_constant(g, f)
    assert _rel(p, dr.bordered_solve(A, fc, wts).reshape(g.shape)) < 1e-12


def _ywall_case(nx, ny, nz, beta=None, ratio=1000.0, seed=5):
    g, us, vs, ws, rho, S = _small_case(nx, ny, nz, beta, ratio, seed)
    g = orc.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, ywalls=True)
    vs[:, 0, :] = 0.0
    return g, us, vs, ws, rho, S


@pytest.mark.parametrize("beta", [None, 1.5])
def test_ywalls_projection_direct_vs_dense(beta):
    """The variable-density definition with y walls against a dense LU of
    D(beta G) assembled entry by entry; the corrected field has no flux
    through the y walls and meets the divergence target."""
    g, us, vs, ws, rho, S = _ywall_case(5, 6, 4, beta)
    dt = 1e-3
    p, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    A = dr.assemble_variable(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, rho, ywalls=True)
    wts = dr.cell_weights(g.nx, g.ny, g.nz, g.zf)
    Sc = S.ravel() - np.dot(wts, S.ravel()) / wts.sum()
    div = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, us, vs, ws, ywalls=True).ravel()
    assert _rel(p, dr.bordered_solve(A, (div - Sc) / dt, wts).reshape(g.shape)) < 1e-11
    assert np.all(v[:, 0, :] == 0.0)
    dnew = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, u, v, w, ywalls=True).ravel()
    assert np.max(np.abs(dnew - Sc)) < 1e-11 * np.max(np.abs(div))


@pytest.mark.parametrize("beta,ratio", [(None, 1000.0), (1.5, 100.0)])
def test_ywalls_method3_reaches_direct_solution(beta, ratio):
    """Algorithm 1 with the wall eigenbasis in y converges to the plain
    definition."""
    g, us, vs, ws, rho, S = _ywall_case(12, 10, 14, beta, ratio)
    dt = 1e-3
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-13, maxit=3000)
    assert info["res_hist"][-1] <= 1e-13
    pd, ud, vd, wd = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    assert _rel(p, pd) < 1e-10
    for a, b in ((u, ud), (v, vd), (w, wd)):
        assert _rel(a, b) < 1e-11


@pytest.mark.parametrize("method", ["method1", "method2"])
def test_ywalls_methods_1_2_reach_direct_solution(method):
    """Methods I and II with y walls reach the same discrete solution."""
    g, us, vs, ws, rho, S = _ywall_case(12, 10, 14, 1.5, 10.0)
    dt = 1e-3
    p, u, v, w, info = getattr(orc, method)(g, us, vs, ws, rho, S, dt, rtol=1e-13)
    assert info["res_hist"][-1] <= 1e-13
    pd, ud, vd, wd = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    assert _rel(p, pd) < 1e-10
    for a, b in ((u, ud), (v, vd), (w, wd)):
        assert _rel(a, b) < 1e-10


def test_ywalls_y_independent_field_matches_periodic():
    """A right-hand side constant in y meets both the periodic and the wall
    conditions, so the two solves agree."""
    g = _ygrid(10, 8, 7, beta=1.5)
    gp = orc.Grid(10, 8, 7, 1.0, 1.0, g.zf)
    f = np.broadcast_to(np.random.default_rng(4).standard_normal((7, 1, 10)), g.shape).copy()
    assert _rel(orc.solve_constant(g, f), orc.solve_constant(gp, f)) < 1e-12



def test_ywalls_operator_identities():
    """D against the loop definition with a nonzero wall row in v (no flux
    crosses a wall whatever the array holds); G of p = y_centre is exactly 1
    on the interior y faces and 0 on the wall row.  Catches an open wall in
    D or G and an off-by-one wall row."""
    g = _ygrid(6, 7, 5, ly=0.7, beta=1.5)
    rng = np.random.default_rng(12)
    u, v = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    w = rng.standard_normal((g.nz + 1, g.ny, g.nx))
    w[0] = w[-1] = 0
    ref = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, u, v, w, ywalls=True)
    assert np.allclose(orc.divergence(g, u, v, w), ref, rtol=0, atol=1e-10)
    yc = (np.arange(g.ny) + 0.5) * g.dy
    p = np.broadcast_to(yc[None, :, None], g.shape).copy()
    gx, gy, gz = orc.gradient(g, p)
    assert np.allclose(gy[:, 1:, :], 1.0, rtol=0, atol=1e-12) and np.all(gy[:, 0, :] == 0)
    assert np.allclose(gx, 0) and np.allclose(gz, 0)


@pytest.mark.parametrize("n,beta,ratio,ywalls", [(32, 1.5, 1000.0, False), (32, None, 10.0, False),
                                                 (48, 1.5, 1000.0, False), (32, 1.5, 1000.0, True)])
def test_method3_matches_preconditioned_cg(n, beta, ratio, ywalls):
    """Beyond the reach of the direct solve: W_c D(beta G) is symmetric
    (D^T = -W_f G W_c^-1), so the variable-density equation is solved
    independently by Jacobi-preconditioned conjugate gradients on
    -W_c A p = -W_c rhs, and Algorithm 1's converged p and u must match it.
    Catches a fixed point that differs from Eq. lap_p by a small term (a
    wrong face average, a dropped u . grad rho part) that the tiny-grid
    pins might not resolve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    g, us, vs, ws, rho, S = (_ywall_case if ywalls else _small_case)(n, n, n, beta, ratio)
    dt = 1e-3
    D, G = orc._sparse_operators(g)
    rx, ry, rz = orc.face_density(g, rho)
    bf = 1.0 / np.concatenate([rx.ravel(), ry.ravel(), rz.ravel()])
    A = (D @ sp.diags(bf) @ G).tocsr()
    Sc = S - orc.volume_mean(g, S)
    rhs = (D @ np.concatenate([us.ravel(), vs.ravel(), ws.ravel()]) - Sc.ravel()) / dt
    wc = np.broadcast_to(g.cell_volume(), g.shape).ravel()
    K = -(sp.diags(wc) @ A).tocsr()
    assert abs(K - K.T).max() <= 1e-12 * abs(K).max()
    x, info = spla.cg(K, -(wc * rhs), rtol=1e-14, maxiter=20000, M=sp.diags(1.0 / K.diagonal()))
    assert info == 0
    x = x.reshape(g.shape)
    x -= orc.volume_mean(g, x)
    p, u, v, w, oinfo = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-13, maxit=20000)
    assert oinfo["res_hist"][-1] <= 1e-13
    assert _rel(p, x) < 1e-10
    for a, b in zip((u, v, w), orc.correct_velocity(g, us, vs, ws, rho, x, dt)):
        assert _rel(a, b) < 1e-11


def test_degenerate_divergence_free_input_takes_no_pass():
    """u* that already meets the target exactly (a uniform flow along the
    periodic directions: D u* = S_c = 0 with no round-off): Algorithm 1
    stops before its first pass with p = 0 and u = u*.  (A field that is
    divergence-free only to round-off is iterated on that noise, as the
    relative stopping rule defines.)"""
    g = _grid(8, 6, 5, beta=1.5)
    rng = np.random.default_rng(31)
    us = np.full(g.shape, 0.37)
    vs = np.full(g.shape, -1.25)
    ws = np.zeros((g.nz + 1, g.ny, g.nx))
    assert np.all(orc.divergence(g, us, vs, ws) == 0.0)
    rho = orc.mixture_density(rng.uniform(0, 1, g.shape), 1.0, 1000.0)
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, np.zeros(g.shape), 1e-3)
    assert info["iters"] == 0 and info["res0"] == 0.0
    assert np.all(p == 0.0) and np.array_equal(u, us) and np.array_equal(v, vs) and np.array_equal(w, ws)


def test_single_layer_is_the_two_dimensional_problem():
    """nz = 1: no z coupling, so a mode cos(2 pi a i/nx) cos(2 pi b j/ny) has
    the 2-D eigenvalue, and the (0, 0) mode is the pinned mean."""
    nx, ny = 16, 12
    g = _grid(nx, ny, 1, 1.0, 0.8, 0.3)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    f = np.cos(2 * np.pi * 3 * i / nx) * np.cos(2 * np.pi * 2 * j / ny + 0.5)
    lam = -(4 * (nx / 1.0) ** 2 * math.sin(math.pi * 3 / nx) ** 2 + 4 * (ny / 0.8) ** 2 * math.sin(math.pi * 2 / ny) ** 2)
    assert _rel(orc.solve_constant(g, f), f / lam) < 1e-12
    assert np.max(np.abs(orc.solve_constant(g, np.ones(g.shape)))) < 1e-14
