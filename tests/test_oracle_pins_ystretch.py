"""Pins of the oracle with a stretched y between walls (Sec. 3.3.1: the
eigenexpansion needs homogeneous boundary conditions, not uniform spacing;
the y step becomes a W-orthonormal eigenbasis found numerically).  Each is
checked against something other than the oracle itself: dense LU solves of
operators assembled entry by entry (tests/dense_reference.py), the DCT path
of a uniform y (scipy's cosine transform), exact identities of D and G on
linear fields, and the projection invariants.  The last section plants a
mistake in each piece and checks that a pin fails.  CPU only.
"""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl
from tests import dense_reference as dr


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _grid(nx, ny, nz, ybeta, zbeta=None, lx=1.0, ly=0.8, lz=1.0):
    zf = wl.uniform_zfaces(nz, lz) if zbeta is None else wl.tanh_zfaces(nz, lz, zbeta)
    yf = np.linspace(0.0, ly, ny + 1) if ybeta is None else wl.tanh_yfaces(ny, ly, ybeta)
    return orc.Grid(nx, ny, nz, lx, ly, zf, ywalls=True, yf=yf)


def _case(nx, ny, nz, ybeta, zbeta=None, ratio=1000.0, seed=7):
    g = _grid(nx, ny, nz, ybeta, zbeta)
    rng = np.random.default_rng(seed)
    phi = np.zeros(g.shape)
    phi[nz // 4:nz // 2 + 1, 1:ny // 2 + 1, nx // 3:2 * nx // 3 + 1] = 1.0
    phi[nz // 2 + 1, 1:ny // 2, nx // 3:2 * nx // 3] = 0.3
    rho = orc.mixture_density(phi, 1.0, ratio)
    us, vs, ws = (rng.standard_normal(g.shape) * 0.1, rng.standard_normal(g.shape) * 0.1,
                  rng.standard_normal((nz + 1, ny, nx)) * 0.1)
    ws[0] = ws[-1] = 0.0
    vs[:, 0, :] = 0.0
    return g, us, vs, ws, rho, wl.gas_source(phi)


# --- constant-coefficient solve -----------------------------------------------

@pytest.mark.parametrize("dims,zbeta", [((6, 8, 5), None), ((4, 10, 6), 1.5)])
def test_uniform_faces_reduce_to_the_cosine_solve(dims, zbeta):
    """Uniform y faces given explicitly take the eigenbasis path; its result
    equals the DCT-II path of the uniform walled y (scipy's cosine
    transform: the eigenvectors cos(pi m (j + 1/2) / ny) in closed form)."""
    nx, ny, nz = dims
    gs = _grid(nx, ny, nz, None, zbeta)
    gu = orc.Grid(nx, ny, nz, gs.lx, gs.ly, gs.zf, ywalls=True)
    f = np.random.default_rng(3).standard_normal(gs.shape)
    assert gs.ystretched and not gu.ystretched
    assert _rel(orc.solve_constant(gs, f), orc.solve_constant(gu, f)) < 1e-13


@pytest.mark.parametrize("dims,ybeta,zbeta", [((6, 8, 5), 1.5, None), ((5, 6, 7), 2.0, 1.5),
                                              ((4, 9, 3), 1.0, 2.0)])
def test_constant_solve_vs_dense_lu(dims, ybeta, zbeta):
    """solve_constant on a stretched walled y against a bordered dense LU of
    D G assembled entry by entry (odd ny included)."""
    nx, ny, nz = dims
    g = _grid(nx, ny, nz, ybeta, zbeta)
    f = np.random.default_rng(11).standard_normal(g.shape)
    L = dr.assemble_variable(nx, ny, nz, g.lx, g.ly, g.zf, None, ywalls=True, yf=g.yf)
    wts = dr.cell_weights(nx, ny, nz, g.zf, yf=g.yf)
    fc = f.ravel() - np.dot(wts, f.ravel()) / wts.sum()
    ref = dr.bordered_solve(L, fc, wts).reshape(g.shape)
    assert _rel(orc.solve_constant(g, f), ref) < 1e-11


def test_cell_volumes_and_mean():
    """The cell volumes tile the box; the volume mean of a field linear in
    the centre y is the mid-height value."""
    g = _grid(5, 12, 4, 2.0, 1.5)
    vol = np.broadcast_to(g.cell_volume(), g.shape)
    assert abs(vol.sum() - g.lx * g.ly * g.lz) < 1e-14
    yc = 0.5 * (g.yf[1:] + g.yf[:-1])
    f = np.broadcast_to(yc[None, :, None], g.shape)
    # each row's centre is its volume's centroid, so the mean is ly / 2
    assert abs(orc.volume_mean(g, f) - 0.5 * g.ly) < 1e-14


# --- D and G -----------------------------------------------------------------

def test_operator_identities():
    """G of the centre coordinate y is 1 on every interior y face and 0 on
    the wall row; D of the face coordinate (wall faces at rest) is 1 in every
    cell away from the top wall; both equal the loop definitions on random
    fields."""
    g = _grid(5, 10, 4, 1.8, 1.2)
    nx, ny, nz = g.nx, g.ny, g.nz
    yc = 0.5 * (g.yf[1:] + g.yf[:-1])
    p = np.broadcast_to(yc[None, :, None], g.shape).copy()
    _, gy, _ = orc.gradient(g, p)
    assert np.max(np.abs(gy[:, 1:] - 1.0)) < 1e-13 and np.all(gy[:, 0] == 0.0)
    v = np.broadcast_to(g.yf[None, :-1, None], g.shape).copy()
    u = np.zeros(g.shape)
    w = np.zeros((nz + 1, ny, nx))
    d = orc.divergence(g, u, v, w)
    # cell 0 sees the wall (y = 0 = yf[0]) below; the top cell sees the wall above
    assert np.max(np.abs(d[:, :-1] - 1.0)) < 1e-13
    rng = np.random.default_rng(5)
    u, v, w = rng.standard_normal(g.shape), rng.standard_normal(g.shape), rng.standard_normal((nz + 1, ny, nx))
    ref = dr.divergence_loops(nx, ny, nz, g.lx, g.ly, g.zf, u, v, w, ywalls=True, yf=g.yf)
    assert _rel(orc.divergence(g, u, v, w), ref) < 1e-14
    p = rng.standard_normal(g.shape)
    for a, b in zip(orc.gradient(g, p), dr.gradient_loops(nx, ny, nz, g.lx, g.ly, g.zf, p, ywalls=True,
                                                            yf=g.yf)):
        assert _rel(a, b) < 1e-14


# --- the variable-density projection --------------------------------------------

@pytest.mark.parametrize("ybeta,zbeta", [(1.5, None), (2.0, 1.5)])
def test_projection_direct_vs_dense(ybeta, zbeta):
    """The definition with a stretched walled y against a dense LU of
    D(beta G) assembled entry by entry; the corrected field meets the
    divergence target and has no flux through the y walls."""
    g, us, vs, ws, rho, S = _case(5, 8, 4, ybeta, zbeta)
    dt = 1e-3
    p, u, v, w = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    A = dr.assemble_variable(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, rho, ywalls=True, yf=g.yf)
    wts = dr.cell_weights(g.nx, g.ny, g.nz, g.zf, yf=g.yf)
    Sc = S.ravel() - np.dot(wts, S.ravel()) / wts.sum()
    div = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, us, vs, ws, ywalls=True, yf=g.yf).ravel()
    assert _rel(p, dr.bordered_solve(A, (div - Sc) / dt, wts).reshape(g.shape)) < 1e-11
    assert np.all(v[:, 0, :] == 0.0)
    dnew = dr.divergence_loops(g.nx, g.ny, g.nz, g.lx, g.ly, g.zf, u, v, w, ywalls=True, yf=g.yf).ravel()
    assert np.max(np.abs(dnew - Sc)) < 1e-11 * np.max(np.abs(div))


@pytest.mark.parametrize("ybeta,zbeta,ratio", [(1.5, None, 1000.0), (2.0, 1.5, 100.0)])
def test_method3_reaches_direct_solution(ybeta, zbeta, ratio):
    """Algorithm 1 with the eigenbasis y step converges to the direct
    solution (the eigenexpansion solve is exact, so the fixed point is the
    variable-density definition).  The numerical eigenbasis is orthonormal
    to a few ulps, which sets a floor near 2e-13 on the relative residual at
    ratio 1000 (the cosine basis of a uniform y reaches 1e-13)."""
    g, us, vs, ws, rho, S = _case(8, 12, 10, ybeta, zbeta, ratio)
    dt = 1e-3
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, S, dt, rtol=1e-12, maxit=4000)
    assert info["res_hist"][-1] <= 1e-12
    pd, ud, vd, wd = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    assert _rel(p, pd) < 1e-10
    for a, b in ((u, ud), (v, vd), (w, wd)):
        assert _rel(a, b) < 1e-11


def test_adjoint_direct_dot_product():
    """adjoint_direct on a stretched y: <g, J du*> = <J^T g, du*> for the
    linear map u* -> u^{n+1} (a forward difference of projection_direct is
    exact for it), and the y-wall row of the gradient is zero."""
    g, us, vs, ws, rho, S = _case(4, 6, 4, 1.5, 1.5, 100.0)
    dt = 1e-3
    rng = np.random.default_rng(9)
    gu, gv, gw = rng.standard_normal(g.shape), rng.standard_normal(g.shape), rng.standard_normal(ws.shape)
    gw[0] = gw[-1] = 0.0
    gv[:, 0, :] = 0.0
    au, av, aw, _ = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    du, dv, dw = rng.standard_normal(g.shape), rng.standard_normal(g.shape), rng.standard_normal(ws.shape)
    dw[0] = dw[-1] = 0.0
    dv[:, 0, :] = 0.0
    _, u0, v0, w0 = orc.projection_direct(g, us, vs, ws, rho, S, dt)
    _, u1, v1, w1 = orc.projection_direct(g, us + du, vs + dv, ws + dw, rho, S, dt)
    lhs = np.sum(gu * (u1 - u0)) + np.sum(gv * (v1 - v0)) + np.sum(gw * (w1 - w0))
    rhs = np.sum(au * du) + np.sum(av * dv) + np.sum(aw * dw)
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
    assert np.all(av[:, 0, :] == 0.0)


@pytest.mark.parametrize("ybeta,zbeta", [(1.5, None), (2.0, 1.5)])
def test_adjoint_method3_equals_the_literal_transpose(ybeta, zbeta):
    """The Algorithm-1 form of the adjoint (W-weighted transposes, the
    gradient of mu through the projection loop) on a stretched y equals the
    implicit differentiation of the definition with literal sparse
    transposes, for u* and for rho; the y-wall row of the gradient is 0."""
    g, us, vs, ws, rho, S = _case(6, 8, 5, ybeta, zbeta, ratio=100.0)
    dt = 1e-3
    rng = np.random.default_rng(21)
    gu, gv, gw = rng.standard_normal(g.shape), rng.standard_normal(g.shape), rng.standard_normal(ws.shape)
    ref = orc.adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw)
    got = orc.adjoint_method3(g, us, vs, ws, rho, S, dt, gu, gv, gw, rtol=1e-13, maxit=3000)
    for a, b in zip(got[:4], ref):
        assert _rel(a, b) < 1e-9
    assert np.all(got[1][:, 0, :] == 0.0)


def test_uniform_only_terms_refuse_a_stretched_y():
    g, us, vs, ws, rho, S = _case(4, 6, 4, 1.5)
    with pytest.raises(NotImplementedError):
        orc.convection(g, us, vs, ws)
    with pytest.raises(NotImplementedError):
        orc.viscous(g, np.ones(g.shape), us, vs, ws)
    with pytest.raises(ValueError):
        orc.Grid(4, 6, 4, 1.0, 0.8, g.zf, ywalls=False, yf=g.yf)


# --- planted mistakes: each must make a pin above fail ------------------------

def test_planted_unweighted_eigenbasis_is_caught(monkeypatch):
    """Eigenvectors of T alone (orthonormal in the plain dot product) in
    place of the W-orthonormal ones of T v = lambda W v."""
    import scipy.linalg as sla

    def planted(g):
        ny = g.ny
        T = np.zeros((ny, ny))
        for j in range(1, ny):
            c = 1.0 / g.dyc[j]
            T[j, j] -= c
            T[j - 1, j - 1] -= c
            T[j, j - 1] = T[j - 1, j] = c
        lam, V = sla.eigh(T)
        order = np.argsort(-lam)
        return lam[order], V[:, order] / np.sqrt(g.dyf)[:, None]
    monkeypatch.setattr(orc, "_y_eigenbasis", planted)
    with pytest.raises(AssertionError):
        test_constant_solve_vs_dense_lu((6, 8, 5), 1.5, None)


def test_planted_face_width_for_centre_distance_is_caught(monkeypatch):
    """The y gradient divided by the row width dyf instead of the centre
    distance dyc."""
    orig = orc.gradient

    def planted(g, p):
        gx, gy, gz = orig(g, p)
        if g.ystretched:
            gy = gy * np.where(g.dyc > 0, g.dyc, 1.0)[None, :, None] / g.dyf[None, :, None]
        return gx, gy, gz
    monkeypatch.setattr(orc, "gradient", planted)
    with pytest.raises(AssertionError):
        test_operator_identities()
    # Algorithm 1 corrects with G: its fixed point leaves the direct solution
    with pytest.raises(AssertionError):
        test_method3_reaches_direct_solution(2.0, 1.5, 100.0)


def test_planted_uniform_volumes_are_caught(monkeypatch):
    """Cell volumes with the mean spacing ly/ny in place of dyf."""
    monkeypatch.setattr(orc.Grid, "cell_volume", lambda self: (self.dx * self.dy * self.dzf)[:, None, None])
    with pytest.raises(AssertionError):
        test_cell_volumes_and_mean()
    with pytest.raises(AssertionError):
        test_constant_solve_vs_dense_lu((6, 8, 5), 1.5, None)


def test_planted_uniform_adjoint_weights_are_caught(monkeypatch):
    """The adjoint's face weights without the y metrics (dzf on every x/y
    face, as on a uniform y)."""
    def planted(g, us, vs, ws, rho, S, dt, gu, gv, gw, rtol=1e-13, maxit=1000, p=None):
        gw = orc._zero_walls(gw)
        gv = orc._zero_ywall_row(g, gv)
        rx, ry, rz = orc.face_density(g, rho)
        wlay = g.dzf[:, None, None]
        wz = np.ones(g.nz + 1)
        wz[1:-1] = g.dzc[1:-1]
        wz = wz[:, None, None]
        zero = np.zeros(g.shape)
        mu = orc.method3(g, -dt * gu / (rx * wlay), -dt * gv / (ry * wlay), -dt * gw / (rz * wz), rho, zero, dt,
                         rtol=rtol, maxit=maxit)[0]
        gx, gy, gz = orc.gradient(g, mu)
        gus = gu + wlay * gx
        gvs = orc._zero_ywall_row(g, gv + wlay * gy)
        gws = orc._zero_walls(gw + wz * gz)
        pp = orc.method3(g, us, vs, ws, rho, S, dt, rtol=rtol, maxit=maxit)[0]
        px, py, pz = orc.gradient(g, pp)
        gbeta = orc._face_vector(-dt * px * gus, -dt * py * gvs, -dt * pz * gws)
        beta = 1.0 / orc._face_vector(rx, ry, rz)
        return gus, gvs, gws, orc._beta_to_rho(g, beta, gbeta), {}
    monkeypatch.setattr(orc, "adjoint_method3", planted)
    with pytest.raises(AssertionError):
        test_adjoint_method3_equals_the_literal_transpose(1.5, None)
