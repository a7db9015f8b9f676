"""Pins of the oracle's convection term, the Adams-Bashforth weights of the
predictor (Eqs. 29, 32), Method I's modified correction (Eq. poisson_me2)
and the constant densities of Methods I and II (Eqs. poisson_me1,
poisson_laizet), each against something other than the oracle itself:
closed forms of the discrete stencils worked out by hand for special
fields, the exactness of a second-order multistep formula, and dense
matrices assembled entry by entry (tests/dense_reference.py).  The last
section plants a mistake in each and checks that a pin fails.  CPU only.
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


def _bcast(a, shape):
    return np.broadcast_to(a, shape).copy()


# --- convection C(u) = div(u u) - u div(u) -----------------------------------

def test_convection_shear_by_a_uniform_cross_velocity():
    """u = sin(kappa y) on the x faces (y of the face centre (j + 1/2) dy) is
    carried by a uniform v = V0: div u = 0, and the only term left is the xy
    edge flux, whose centred difference is the closed form
    C_x = V0 cos(kappa y_j) sin(kappa dy) / dy (a sine's central difference).
    The same with the roles of x and y exchanged for C_y.  Fixes the sign and
    scale of the cross terms (the conservation pins are blind to both)."""
    nx, ny, nz, lx, ly, V0 = 6, 16, 5, 0.7, 1.3, 0.37
    g = _grid(nx, ny, nz, lx, ly, 0.9, beta=1.5)
    kap = 2 * math.pi / ly
    yj = (np.arange(ny) + 0.5) * g.dy
    u = _bcast(np.sin(kap * yj)[None, :, None], g.shape)
    v = np.full(g.shape, V0)
    w = np.zeros((nz + 1, ny, nx))
    cx, cy, cz = orc.convection(g, u, v, w)
    ref = _bcast((V0 * np.cos(kap * yj) * math.sin(kap * g.dy) / g.dy)[None, :, None], g.shape)
    assert _rel(cx, ref) < 1e-13
    assert np.abs(cy).max() < 1e-13 and np.abs(cz).max() < 1e-13

    nx, ny = 18, 4
    g = _grid(nx, ny, nz, lx, ly, 0.9)
    kap = 2 * math.pi / lx
    xi = (np.arange(nx) + 0.5) * g.dx
    U0 = -0.81
    v = _bcast(np.sin(kap * xi)[None, None, :], g.shape)
    u = np.full(g.shape, U0)
    cx, cy, cz = orc.convection(g, u, v, np.zeros((nz + 1, ny, nx)))
    ref = _bcast((U0 * np.cos(kap * xi) * math.sin(kap * g.dx) / g.dx)[None, None, :], g.shape)
    assert _rel(cy, ref) < 1e-13
    assert np.abs(cx).max() < 1e-13 and np.abs(cz).max() < 1e-13


def _compressive_closed_form(n, d):
    """A single sine u_i = sin(theta_i) on the faces of one direction,
    theta_i = 2 h i (h = half the phase step), nothing else moving.  With
    a_i = (u_i + u_{i+1})/2 = cos h sin(theta_i + h) and the divergence
    D_i = 2 sin h cos(theta_i + h) / d, the centred
    (a_i^2 - a_{i-1}^2)/d - u_i (D_i + D_{i-1})/2 reduces to
    sin(4h) sin(2 theta_i) / (4 d); the continuous limit is u u' = k sin(2kx)/2."""
    return lambda theta, h: math.sin(4 * h) * np.sin(2 * theta) / (4 * d)


def test_convection_compressive_single_modes():
    """Compressive single modes along x, y and z (uniform z, w zero on the
    walls): the closed form above fixes the normal flux and the -u div(u)
    term, which vanishes on every divergence-free field the conservation
    pins use."""
    nx, ny, nz, lx, ly, lz = 12, 10, 8, 1.1, 0.8, 0.6
    g = _grid(nx, ny, nz, lx, ly, lz)
    z3 = np.zeros((nz + 1, ny, nx))
    zc = np.zeros(g.shape)
    # x: faces at x = i dx
    th = 2 * math.pi * np.arange(nx) / nx
    u = _bcast(np.sin(th)[None, None, :], g.shape)
    cx, cy, cz = orc.convection(g, u, zc, z3)
    ref = _bcast(_compressive_closed_form(nx, g.dx)(th, math.pi / nx)[None, None, :], g.shape)
    assert _rel(cx, ref) < 1e-12
    assert np.abs(cy).max() < 1e-13 and np.abs(cz).max() < 1e-13
    # y: faces at y = j dy
    th = 2 * math.pi * np.arange(ny) / ny
    v = _bcast(np.sin(th)[None, :, None], g.shape)
    cx, cy, cz = orc.convection(g, zc, v, z3)
    ref = _bcast(_compressive_closed_form(ny, g.dy)(th, math.pi / ny)[None, :, None], g.shape)
    assert _rel(cy, ref) < 1e-12
    assert np.abs(cx).max() < 1e-13 and np.abs(cz).max() < 1e-13
    # z: faces at z = k dz, k = 0 .. nz, w = sin(pi k / nz) vanishes on both walls
    dz = lz / nz
    th = math.pi * np.arange(nz + 1) / nz
    w = _bcast(np.sin(th)[:, None, None], (nz + 1, ny, nx))
    cx, cy, cz = orc.convection(g, zc, zc, w)
    ref = _bcast(_compressive_closed_form(nz, dz)(th, math.pi / (2 * nz))[:, None, None], (nz + 1, ny, nx))
    ref[0] = ref[-1] = 0.0
    assert _rel(cz, ref) < 1e-12
    assert np.abs(cx).max() < 1e-13 and np.abs(cy).max() < 1e-13


def test_convection_by_a_uniform_wall_normal_velocity_stretched():
    """u = u(z) arbitrary on a stretched z, w = W0 on every interior z face
    (0 on the walls), v = 0.  Worked out by hand from the stencil: the xz
    edge flux is W0 times the face mean of u, so in the interior layers
    C_x = W0 (u_{k+1} - u_{k-1}) / (2 dzf_k); in the two wall layers the
    divergence is +-W0/dzf and the -u div(u) term turns the one-sided flux
    into W0 (u_1 - u_0) / (2 dzf_0) and W0 (u_{n-1} - u_{n-2}) / (2 dzf_{n-1}).
    For w itself: the centre values of w are W0/2 in the wall layers and W0
    inside, so C_z on face 1 is W0^2 (3/(4 dzc_1) - 1/(2 dzf_0)), on face
    nz - 1 it is W0^2 (1/(2 dzf_{n-1}) - 3/(4 dzc_{n-1})), and 0 between.
    Fixes the xz edge term, the z interpolation of div(u) and their signs."""
    nx, ny, nz, W0 = 4, 3, 9, 0.6
    g = _grid(nx, ny, nz, 1.0, 1.0, 0.8, beta=2.0)
    rng = np.random.default_rng(77)
    uz = rng.standard_normal(nz)
    u = _bcast(uz[:, None, None], g.shape)
    w = np.full((nz + 1, ny, nx), W0)
    w[0] = w[-1] = 0.0
    cx, cy, cz = orc.convection(g, u, np.zeros(g.shape), w)
    dzf = g.dzf
    ref = np.empty(nz)
    ref[1:-1] = W0 * (uz[2:] - uz[:-2]) / (2 * dzf[1:-1])
    ref[0] = W0 * (uz[1] - uz[0]) / (2 * dzf[0])
    ref[-1] = W0 * (uz[-1] - uz[-2]) / (2 * dzf[-1])
    assert _rel(cx, _bcast(ref[:, None, None], g.shape)) < 1e-13
    assert np.abs(cy).max() < 1e-13
    refz = np.zeros(nz + 1)
    refz[1] = W0 ** 2 * (3 / (4 * g.dzc[1]) - 1 / (2 * dzf[0]))
    refz[nz - 1] = W0 ** 2 * (1 / (2 * dzf[-1]) - 3 / (4 * g.dzc[nz - 1]))
    assert _rel(cz, _bcast(refz[:, None, None], (nz + 1, ny, nx))) < 1e-13


# --- Adams-Bashforth weights (Eq. 29) ----------------------------------------

def test_adams_bashforth_is_exact_for_a_linear_history():
    """A second-order two-step formula integrates a right-hand side that is
    linear in time exactly, for any step ratio r: with RU(t) = RU^n + beta
    (t - t_n), int_{t_n}^{t_n + dt_new} RU = dt_new (RU^n + beta dt_new / 2).
    Feeding RU^{n-1} = RU^n - beta dt_old must give that increment.  The
    history differs from RU^n and r = 2.5 != 1, so any weights other than
    Eq. 29's (1 + r/2, r/2) fail, e.g. (1 + r, r) or a - b = 1 pairs."""
    g = _grid(8, 6, 7, beta=1.5)
    rng = np.random.default_rng(91)
    rho = rng.uniform(1.0, 50.0, g.shape)
    mu = rng.uniform(1e-3, 0.1, g.shape)
    u, v = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    w = rng.standard_normal((g.nz + 1, g.ny, g.nx)); w[0] = w[-1] = 0.0
    grav = (0.1, 0.0, -9.81)
    dt_old, dt_new = 1e-3, 2.5e-3
    ru = orc.predictor_rhs(g, u, v, w, rho, mu, grav)
    beta = (rng.standard_normal(g.shape), rng.standard_normal(g.shape),
            rng.standard_normal((g.nz + 1, g.ny, g.nx)))
    prev = tuple(q - b * dt_old for q, b in zip(ru, beta))
    (a1, b1, c1), ru_out = orc.predictor(g, u, v, w, rho, mu, grav, dt_new, dt_old, ru_prev=prev)
    for out, x, q, b in zip((a1, b1, c1), (u, v, w), ru, beta):
        ref = x + dt_new * (q + 0.5 * b * dt_new)
        if out.shape[0] == g.nz + 1:
            ref = ref.copy(); ref[0] = ref[-1] = 0.0
        assert _rel(out, ref) < 1e-14


# --- Methods I and II: dense restatements on a tiny grid ----------------------

def _case(ratio=10.0):
    """5 x 4 x 6 cells, stretched z, a gas block with pure gas and pure
    liquid cells (so min rho = rho_g and max rho = rho_l), a thin interface
    layer, a random u* and a gas source."""
    nx, ny, nz = 5, 4, 6
    zf = wl.tanh_zfaces(nz, 0.8, 1.5)
    g = orc.Grid(nx, ny, nz, 1.0, 0.9, zf)
    phi = np.zeros(g.shape)
    phi[1:4, 1:3, 1:3] = 1.0
    phi[4, 1:3, 1:3] = 0.35
    rho_g, rho_l = 1.0, ratio
    rho = orc.mixture_density(phi, rho_g, rho_l)
    rng = np.random.default_rng(23)
    us, vs = rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1
    ws = rng.standard_normal((nz + 1, ny, nx)) * 0.1; ws[0] = ws[-1] = 0.0
    S = wl.gas_source(phi)
    return g, zf, us, vs, ws, rho, S, rho_g, rho_l


def _dense(g, zf, rho):
    A = dr.assemble_variable(g.nx, g.ny, g.nz, g.lx, g.ly, zf, rho)
    Lp = dr.pseudo_inverse_laplacian(g.nx, g.ny, g.nz, g.lx, g.ly, zf)
    wts = dr.cell_weights(g.nx, g.ny, g.nz, zf)
    return A, Lp, wts


def _b(g, zf, us, vs, ws, S, wts, dt):
    d = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, zf, us, vs, ws).ravel()
    Sc = S.ravel() - (wts @ S.ravel()) / wts.sum()
    return (d - Sc) / dt


def test_method1_modified_correction_after_two_passes():
    """Stop Method I after two passes and rebuild both iterates and
    Eq. poisson_me2 from the dense operators: p1 = L+ (rho0 b),
    p2 = L+ [D((1 - rho0 beta) G p1) + rho0 b] (Eq. poisson_me1, L+ the
    zero-mean inverse of D G), then
    u = u* - dt [ (1/rho0) G p2 + (beta - 1/rho0) G p1 ].
    Two passes, so p2 != p1 and a correction that swaps p and p^q (or uses
    Eq. corr) differs by dt (2/rho0 - beta) G (p1 - p2)."""
    g, zf, us, vs, ws, rho, S, rho_g, _ = _case(10.0)
    dt = 1e-3
    A, Lp, wts = _dense(g, zf, rho)
    b = _b(g, zf, us, vs, ws, S, wts, dt)
    rho0 = rho_g                      # Eq. poisson_me1: the smallest density
    sh = g.shape
    p1 = Lp @ (rho0 * b)
    bx, by, bz = dr.face_beta_loops(g.nx, g.ny, g.nz, rho)
    gx, gy, gz = dr.gradient_loops(g.nx, g.ny, g.nz, g.lx, g.ly, zf, p1.reshape(sh))
    dflux = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, zf, (1 - rho0 * bx) * gx,
                                (1 - rho0 * by) * gy, (1 - rho0 * bz) * gz).ravel()
    p2 = Lp @ (dflux + rho0 * b)
    g2 = dr.gradient_loops(g.nx, g.ny, g.nz, g.lx, g.ly, zf, p2.reshape(sh))
    g1 = (gx, gy, gz)
    ref = [x - dt * (q2 / rho0 + (bb - 1 / rho0) * q1) for x, q2, q1, bb in
           zip((us, vs, ws), g2, g1, (bx, by, bz))]
    ref[2][0] = ref[2][-1] = 0.0
    p, u, v, w, info = orc.method1(g, us, vs, ws, rho, S, dt, rtol=0.0, maxit=2)
    assert info["iters"] == 2
    assert _rel(p.ravel(), p2) < 1e-12
    for a, r in zip((u, v, w), ref):
        assert _rel(a, r) < 1e-12
    # the swap is not a rounding-level change here
    swapped = us - dt * (g1[0] / rho0 + (bx - 1 / rho0) * g2[0])
    assert _rel(swapped, ref[0]) > 1e-3


def _dense_residuals(A, Lp, scale, b, npass):
    """Relative residual norms of the defect-correction iteration
    r^{s+1} = (I - A L+ diag(scale)) r^s, r^0 = b (Sec. 3.3.1: each method
    adds L+ (rho~ times the residual) to p; A = D(beta G))."""
    M = np.eye(len(b)) - A @ Lp @ np.diag(scale)
    r, out = b.copy(), []
    for _ in range(npass):
        r = M @ r
        out.append(float(np.linalg.norm(r) / np.linalg.norm(b)))
    return np.array(out), M


def _spectral_radius_on_compatible(M, wts):
    """Largest |eigenvalue| of M on the residuals with zero weighted sum
    (the space it maps into itself); orthonormal basis Q of that space."""
    n = len(wts)
    Q, _ = np.linalg.qr(np.column_stack([wts, np.eye(n)[:, :n - 1]]))
    Q = Q[:, 1:]
    return float(np.max(np.abs(np.linalg.eigvals(Q.T @ M @ Q))))


@pytest.mark.parametrize("method", ["method1", "method2", "method3"])
def test_residual_history_is_the_dense_iteration(method):
    """The constant density decides how fast each method contracts, so it is
    pinned through the residual history.  The dense iteration uses the
    paper's definitions directly: Method I's smallest density
    (Eq. poisson_me1), Method II's harmonic mean of the two phase
    densities (Eq. poisson_laizet), Method III's cell density
    (Eq. new_poisson).  The oracle's relative residuals after each pass must
    equal the dense iteration's, and the late contraction per pass must
    approach the spectral radius of the error-propagation matrix."""
    g, zf, us, vs, ws, rho, S, rho_g, rho_l = _case(10.0)
    dt = 1e-3
    A, Lp, wts = _dense(g, zf, rho)
    b = _b(g, zf, us, vs, ws, S, wts, dt)
    n = len(b)
    scale = {"method1": np.full(n, rho_g),
             "method2": np.full(n, 2.0 / (1.0 / rho_g + 1.0 / rho_l)),
             "method3": rho.ravel()}[method]
    npass = 60
    ref, M = _dense_residuals(A, Lp, scale, b, npass)
    _, _, _, _, info = getattr(orc, method)(g, us, vs, ws, rho, S, dt, rtol=0.0, maxit=npass)
    hist = np.array(info["res_hist"])
    assert len(hist) == npass
    # pass by pass while the residual is far above the rounding floor
    k = int(np.searchsorted(-ref, -1e-6))
    assert k >= 8
    assert np.max(np.abs(hist[:k] / ref[:k] - 1.0)) < 1e-8
    # late contraction, measured down to 1e-11, against the spectral radius
    kl = int(np.searchsorted(-ref, -1e-11))
    rad = _spectral_radius_on_compatible(M, wts)
    assert rad < 1.0
    late = (hist[kl - 1] / hist[kl - 7]) ** (1.0 / 6.0)
    assert abs(late - rad) < 0.03 * rad, (late, rad)


# --- planted mistakes: each must make a pin above fail ------------------------

def test_planted_convection_sign_is_caught(monkeypatch):
    orig = orc.convection
    monkeypatch.setattr(orc, "convection", lambda g, u, v, w: tuple(-c for c in orig(g, u, v, w)))
    with pytest.raises(AssertionError):
        test_convection_shear_by_a_uniform_cross_velocity()
    with pytest.raises(AssertionError):
        test_convection_compressive_single_modes()


def test_planted_convection_scale_is_caught(monkeypatch):
    orig = orc.convection
    monkeypatch.setattr(orc, "convection", lambda g, u, v, w: tuple(0.5 * c for c in orig(g, u, v, w)))
    with pytest.raises(AssertionError):
        test_convection_shear_by_a_uniform_cross_velocity()


def test_planted_dropped_u_div_u_is_caught(monkeypatch):
    """C without its -u div(u) part (divergence form only)."""
    orig = orc.convection

    def planted(g, u, v, w):
        cx, cy, cz = orig(g, u, v, w)
        D = orc.divergence(g, u, v, w)
        Dz = np.zeros((g.nz + 1, g.ny, g.nx))
        Dz[1:-1] = 0.5 * (D[1:] + D[:-1])
        return (cx + u * 0.5 * (D + np.roll(D, 1, axis=2)), cy + v * 0.5 * (D + np.roll(D, 1, axis=1)),
                cz + w * Dz)
    monkeypatch.setattr(orc, "convection", planted)
    # the divergence-free conservation pins cannot see it ...
    from tests.test_oracle_pins import test_convection_conserves_momentum_and_energy
    test_convection_conserves_momentum_and_energy()
    # ... the compressive closed forms do
    with pytest.raises(AssertionError):
        test_convection_compressive_single_modes()
    with pytest.raises(AssertionError):
        test_convection_by_a_uniform_wall_normal_velocity_stretched()


def test_planted_adams_bashforth_weights_are_caught(monkeypatch):
    """The dp0/dt extrapolation's weights (1 + r, r) in place of Eq. 29's."""
    monkeypatch.setattr(orc, "ab2_weights", lambda dn, do: (1.0 + dn / do, dn / do))
    with pytest.raises(AssertionError):
        test_adams_bashforth_is_exact_for_a_linear_history()


def test_planted_swapped_method1_iterates_are_caught(monkeypatch):
    orig = orc.method1_correction
    monkeypatch.setattr(orc, "method1_correction",
                        lambda g, us, vs, ws, rho, rho0, p, p_q, dt: orig(g, us, vs, ws, rho, rho0, p_q, p, dt))
    with pytest.raises(AssertionError):
        test_method1_modified_correction_after_two_passes()


@pytest.mark.parametrize("name,method,planted", [
    ("method2_rho_tilde", "method2", lambda rho: 0.5 * (float(np.min(rho)) + float(np.max(rho)))),
    ("method2_rho_tilde", "method2", lambda rho: float(np.min(rho))),
    ("method1_rho_tilde", "method1", lambda rho: 2.0 / (1.0 / float(np.min(rho)) + 1.0 / float(np.max(rho)))),
])
def test_planted_constant_density_is_caught(monkeypatch, name, method, planted):
    monkeypatch.setattr(orc, name, planted)
    with pytest.raises(AssertionError):
        test_residual_history_is_the_dense_iteration(method)


# --- adjoint with walls in y -------------------------------------------------

def _duct_case():
    """6 x 4 x 5 duct (walls in y and z), stretched z, a gas block at ratio
    100, v* zero on the wall row."""
    nx, ny, nz = 6, 4, 5
    zf = wl.tanh_zfaces(nz, 0.5, 2.0)
    g = orc.Grid(nx, ny, nz, 1.0, 0.8, zf, ywalls=True)
    phi = np.zeros(g.shape)
    phi[1:3, 1:3, 2:4] = 1.0
    phi[3, 1:3, 2:4] = 0.5
    rho = orc.mixture_density(phi, 1.0, 100.0)
    rng = np.random.default_rng(61)
    us, vs = rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1
    ws = rng.standard_normal((nz + 1, ny, nx)) * 0.1
    vs[:, 0, :] = 0.0
    ws[0] = ws[-1] = 0.0
    tgt = (rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1,
           rng.standard_normal((nz + 1, ny, nx)) * 0.1)
    return g, us, vs, ws, rho, wl.gas_source(phi), tgt


def _duct_loss(g, us, vs, ws, rho, S, dt, tgt):
    """L = ||u^{n+1} - target||^2 over the unknowns: the wall planes of w and
    the wall row of v are not unknowns (zero by the walls)."""
    _, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    return float(np.sum((u - tgt[0]) ** 2) + np.sum((v[:, 1:] - tgt[1][:, 1:]) ** 2)
                 + np.sum((w[1:-1] - tgt[2][1:-1]) ** 2))


def test_ywalls_adjoint_central_differences_and_dot_product():
    """With walls in y: adjoint_direct against central differences of the
    projection (eps = 1e-6 relative) on entries of u*, v* (off the wall row),
    w* and rho; the dot-product identity <P d, g> = <d, P^T g> with d and g
    zero on the wall faces; and the Algorithm-1 form of the adjoint against
    the literal sparse transpose."""
    g, us, vs, ws, rho, S, tgt = _duct_case()
    dt = 1e-3
    _, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    gu, gv, gw = 2 * (u - tgt[0]), 2 * (v - tgt[1]), 2 * (w - tgt[2])
    gv[:, 0, :] = 0.0
    gus, gvs, gws, grho = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    assert np.all(gvs[:, 0, :] == 0.0) and np.all(gws[0] == 0.0) and np.all(gws[-1] == 0.0)
    arrs = {"us": us, "vs": vs, "ws": ws, "rho": rho}
    grads = {"us": gus, "vs": gvs, "ws": gws, "rho": grho}
    for key, idx in (("us", (1, 2, 3)), ("vs", (2, 1, 4)), ("vs", (3, 3, 0)), ("ws", (2, 2, 1)),
                     ("rho", (2, 1, 2)), ("rho", (3, 2, 3)), ("rho", (0, 0, 5))):
        base = arrs[key]
        h = 1e-6 * max(1.0, abs(base[idx]))
        plus, minus = dict(arrs), dict(arrs)
        plus[key] = base.copy(); plus[key][idx] += h
        minus[key] = base.copy(); minus[key][idx] -= h
        fd = (_duct_loss(g, plus["us"], plus["vs"], plus["ws"], plus["rho"], S, dt, tgt)
              - _duct_loss(g, minus["us"], minus["vs"], minus["ws"], minus["rho"], S, dt, tgt)) / (2 * h)
        an = grads[key][idx]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.max(np.abs(gus))), (key, idx, fd, an)
    rng = np.random.default_rng(62)
    du, dv = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    dw = rng.standard_normal((g.nz + 1, g.ny, g.nx))
    dv[:, 0, :] = 0.0
    dw[0] = dw[-1] = 0.0
    zero = np.zeros(g.shape)
    _, pu, pv, pw = orc.projection_direct(g, du, dv, dw, rho, zero, dt)
    pv[:, 0, :] = 0.0
    a1, a2, a3, _ = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    lhs = np.sum(pu * gu) + np.sum(pv * gv) + np.sum(pw[1:-1] * gw[1:-1])
    rhs = np.sum(du * a1) + np.sum(dv * a2) + np.sum(dw * a3)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    b1, b2, b3, brho, _ = orc.adjoint_method3(g, us, vs, ws, rho, S, dt, gu, gv, gw, rtol=1e-13)
    for x, y in ((b1, gus), (b2, gvs), (b3, gws), (brho, grho)):
        assert _rel(x, y) < 1e-9
    # an upstream gradient on the wall row (not an unknown) is ignored
    gv_wall = gv.copy()
    gv_wall[:, 0, :] = rng.standard_normal((g.nz, g.nx))
    for fn in (lambda: orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv_wall, gw),
               lambda: orc.adjoint_method3(g, us, vs, ws, rho, S, dt, gu, gv_wall, gw, rtol=1e-13)[:4]):
        for x, y in zip(fn(), (gus, gvs, gws, grho)):
            assert _rel(x, y) < 1e-9


def test_planted_ywall_gradient_kept_is_caught(monkeypatch):
    """The wall row of v treated as an unknown (its upstream gradient kept)."""
    monkeypatch.setattr(orc, "_zero_ywall_row", lambda g, gv: np.array(gv, dtype=np.float64, copy=True))
    with pytest.raises(AssertionError):
        test_ywalls_adjoint_central_differences_and_dot_product()


# --- the divergence source with walls in y (Eqs. 30, 34) ---------------------

def test_ywalls_conduction_matches_dense_assembly_and_conserves_heat():
    """With walls in y the conduction operator D(k_f G T) equals the matrix
    assembled entry by entry with no flux through the y walls (variable k,
    stretched z), and a closed duct full of gas loses no heat:
    sum div(k grad T) dV = 0, so dp0/dt = 0 with no dilatation (Eq. 30)."""
    nx, ny, nz = 6, 5, 7
    zf = wl.tanh_zfaces(nz, 0.6, 1.5)
    g = orc.Grid(nx, ny, nz, 1.0, 0.8, zf, ywalls=True)
    rng = np.random.default_rng(71)
    kc = rng.uniform(0.5, 3.0, g.shape)
    T = rng.standard_normal(g.shape)
    A = dr.assemble_conduction(nx, ny, nz, 1.0, 0.8, zf, kc, ywalls=True)
    cond = orc.conduction(g, kc, T)
    assert _rel(cond.ravel(), A @ T.ravel()) < 1e-13
    dv = g.cell_volume()
    assert abs(np.sum(cond * dv)) <= 1e-13 * np.sum(np.abs(cond) * dv)
    zero = np.zeros(g.shape)
    rp = orc.p0_rate(g, np.ones(g.shape), kc, T, zero, zero, np.zeros((nz + 1, ny, nx)), 1.0, 1.4)
    assert abs(rp) <= 1e-13 * (1.4 / orc.gas_volume(g, np.ones(g.shape))) * np.sum(np.abs(cond) * dv)


def test_planted_open_y_wall_in_conduction_is_caught(monkeypatch):
    """Heat flowing through the y walls (the periodic faces used by both G
    and D, i.e. a periodic y)."""
    orig_g, orig_d = orc.gradient, orc.divergence

    def periodic(g):
        return orc.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, ywalls=False)
    monkeypatch.setattr(orc, "gradient", lambda g, p: orig_g(periodic(g), p))
    monkeypatch.setattr(orc, "divergence", lambda g, u, v, w: orig_d(periodic(g), u, v, w))
    with pytest.raises(AssertionError):
        test_ywalls_conduction_matches_dense_assembly_and_conserves_heat()


# --- the momentum predictor with walls in y (Eqs. 29, 32) --------------------

def _ygrid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
    return orc.Grid(nx, ny, nz, lx, ly, wl.uniform_zfaces(nz, lz), ywalls=True)


def test_ywalls_poiseuille_profiles_give_the_wall_closed_form():
    """No-slip y walls.  u = y (ly - y) at the cell centres (zero on both
    walls), constant mu: the second difference is exact for a quadratic, so
    div tau = -2 mu in every row off the walls; in the two wall rows the
    shear at the wall is mu u_0 / (dy/2) = mu (ly - dy/2) while the exact
    slope is ly, and the discrete force is exactly -1.5 mu there (layers
    off the z walls, whose shear adds to the two layers next to them).  The
    same for w = y (ly - y) on the z faces away from the z walls.  No convection
    in either.  Fixes the half-cell wall distance, the wall velocity and
    both walls' edge rows."""
    nx, ny, nz, mu, ly = 4, 10, 8, 0.7, 1.3
    g = _ygrid(nx, ny, nz, 1.0, ly, 0.9)
    yc = (np.arange(ny) + 0.5) * g.dy
    prof = yc * (ly - yc)
    expect = np.full(ny, -2.0 * mu)
    expect[0] = expect[-1] = -1.5 * mu
    zero = np.zeros(g.shape)
    wz = np.zeros((nz + 1, ny, nx))
    u = _bcast(prof[None, :, None], g.shape)
    fx, fy, fz = orc.viscous(g, np.full(g.shape, mu), u, zero, wz)
    # layers next to the z walls also feel the z-wall shear
    assert np.allclose(fx[1:-1], _bcast(expect[None, :, None], fx[1:-1].shape), rtol=1e-12, atol=1e-12)
    assert np.abs(fy).max() < 1e-12 and np.abs(fz).max() < 1e-12
    cx, cy, cz = orc.convection(g, u, zero, wz)
    assert max(np.abs(cx).max(), np.abs(cy).max(), np.abs(cz).max()) < 1e-13
    w = np.zeros((nz + 1, ny, nx))
    w[1:-1] = prof[None, :, None]
    fx, fy, fz = orc.viscous(g, np.full(g.shape, mu), zero, zero, w)
    assert np.allclose(fz[2:-2], _bcast(expect[None, :, None], fz[2:-2].shape), rtol=1e-12, atol=1e-12)
    assert np.abs(fx).max() < 1e-12


def test_ywalls_compressive_mode_and_wall_row():
    """v = sin(pi j / ny) on the y faces (zero on both walls), nothing else
    moving: C_y off the wall row is the compressive closed form
    sin(4h) sin(2 theta) / (4 dy), h = pi / (2 ny); the wall row of C_y, of
    RU_y and of the predicted v is zero."""
    nx, ny, nz = 4, 12, 5
    g = _ygrid(nx, ny, nz, 1.0, 0.9, 0.7)
    th = np.pi * np.arange(ny) / ny
    v = _bcast(np.sin(th)[None, :, None], g.shape)
    zero = np.zeros(g.shape)
    wz = np.zeros((nz + 1, ny, nx))
    cx, cy, cz = orc.convection(g, zero, v, wz)
    ref = _bcast(_compressive_closed_form(ny, g.dy)(th, np.pi / (2 * ny))[None, :, None], g.shape)
    assert _rel(cy[:, 1:], ref[:, 1:]) < 1e-12
    assert np.all(cy[:, 0] == 0.0) and np.abs(cx).max() < 1e-13 and np.abs(cz).max() < 1e-13
    rho = np.full(g.shape, 2.0)
    (us, vs, ws), ru = orc.predictor(g, zero, v, wz, rho, np.full(g.shape, 0.1), (0.0, 1.0, 0.0), 1e-3)
    assert np.all(vs[:, 0] == 0.0) and np.all(ru[1][:, 0] == 0.0)


def test_planted_ywall_shear_mistakes_are_caught(monkeypatch):
    """A full cell (not half a cell) to the y wall, and free-slip y walls."""
    orig = orc._viscous_ywalls

    def full_cell(g, mu, u, v, w):
        fx, fy, fz = orig(g, mu, u, v, w)
        # the wall rows' shear halved: as if the wall were dy away
        mux = 0.5 * (mu + np.roll(mu, 1, axis=2))
        fx = fx.copy()
        fx[:, 0] -= 0.5 * mux[:, 0] * u[:, 0] / (0.5 * g.dy) / g.dy
        fx[:, -1] -= 0.5 * mux[:, -1] * u[:, -1] / (0.5 * g.dy) / g.dy
        return fx, fy, fz

    def free_slip(g, mu, u, v, w):
        fx, fy, fz = orig(g, mu, u, v, w)
        mux = 0.5 * (mu + np.roll(mu, 1, axis=2))
        fx = fx.copy()
        fx[:, 0] += mux[:, 0] * u[:, 0] / (0.5 * g.dy) / g.dy
        fx[:, -1] += mux[:, -1] * u[:, -1] / (0.5 * g.dy) / g.dy
        return fx, fy, fz
    for planted in (full_cell, free_slip):
        monkeypatch.setattr(orc, "_viscous_ywalls", planted)
        with pytest.raises(AssertionError):
            test_ywalls_poiseuille_profiles_give_the_wall_closed_form()


def test_ywalls_predictor_terms_reduce_to_periodic_away_from_the_walls():
    """Fields that vanish in the two rows next to each y wall never reach the
    walls: the walled-y convection and viscous terms must then equal the
    periodic ones everywhere (variable mu, stretched z).  Checks the interior
    indexing of the walled code (edge rows, means of mu) against the pinned
    periodic operators."""
    nx, ny, nz = 5, 10, 6
    zf = wl.tanh_zfaces(nz, 0.7, 1.5)
    gw_ = orc.Grid(nx, ny, nz, 1.0, 0.9, zf, ywalls=True)
    gp = orc.Grid(nx, ny, nz, 1.0, 0.9, zf)
    rng = np.random.default_rng(81)
    u, v = rng.standard_normal(gp.shape), rng.standard_normal(gp.shape)
    w = rng.standard_normal((nz + 1, ny, nx))
    w[0] = w[-1] = 0.0
    for a in (u, v, w):
        a[:, :2] = 0.0
        a[:, -2:] = 0.0
    v[:, 2] = 0.0   # the face below row 2 borders row 1
    mu = rng.uniform(0.1, 1.0, gp.shape)
    for fn in (lambda g: orc.convection(g, u, v, w), lambda g: orc.viscous(g, mu, u, v, w)):
        for a, b in zip(fn(gw_), fn(gp)):
            assert np.allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(b).max())
