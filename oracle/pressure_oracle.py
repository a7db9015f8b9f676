"""FP64 CPU oracle for the pressure step of the low-Mach two-phase solver of
Dalla Barba, Scapin, Rosti, Picano and Brandt, "An interface capturing method
for liquid-gas flows at low-Mach number" (arXiv:2005.11806).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path: it imports numpy/scipy only, and nothing from the product
package.  It is deliberately plain and slow: numpy array expressions, numpy's
FFT and dense/sparse library solves as single steps, no fusion, no blocking.

Discretisation (Sec. 3, "Numerical methodology": a Cartesian marker-and-cell
grid, velocities on faces, scalar fields at cell centres):

* arrays are ``[nz][ny][nx]``, x fastest;
* ``u[k, j, i]`` lives on the x-face at ``i - 1/2`` (periodic in x),
  ``v[k, j, i]`` on the y-face at ``j - 1/2`` (periodic in y),
  ``w[k, j, i]`` (shape ``[nz + 1][ny][nx]``) on the z-face ``k``; faces 0 and
  nz are the no-penetration walls;
* z may be stretched: ``zf`` holds the nz + 1 face coordinates, the cell
  centre is the midpoint of its faces, ``dzf[k]`` is the width of cell k and
  ``dzc[k]`` the distance between the centres that share the z-face k;
* with ``ywalls`` the y direction is bounded by two no-penetration walls
  instead of being periodic.  ``v`` keeps its ``[nz][ny][nx]`` shape: row j
  is still the face at ``j - 1/2``, and row 0 stands for both walls
  (``y = 0`` and ``y = ly``), whose normal velocity is zero;
* a bounded y may be stretched: ``yf`` holds the ny + 1 face coordinates,
  ``dyf[j]`` is the width of row j and ``dyc[j]`` the distance between the
  centres that share the y-face j (j = 1 .. ny - 1).  The y step of the
  eigenexpansion solve is then the eigenbasis of the y part of L, found
  numerically (Sec. 3.3.1 needs only homogeneous conditions, not uniform
  spacing).

Readings of points the paper leaves open:

* the density on a face is the arithmetic mean of its two cells, so the
  centred form of ``u . grad(rho)`` used by Method III is
  ``D(rho_f u) - rho_c D u``;
* the pressure satisfies homogeneous Neumann conditions at the z walls (and
  at the y walls when y is bounded) and is periodic in the other directions;
  it is fixed to zero volume-weighted mean;
* the divergence target ``S`` (Eq. 34) is made compatible with the closed box
  by removing its volume-weighted mean;
* Algorithm 1 is read as: iteration s uses ``u^s`` (``u^0 = u*``) to produce
  ``p^{s+1}`` and ``u^{s+1}``; it stops on the relative L2 norm of
  ``D u^{s+1} - S_c`` (the paper's L1 sum is reported too);
* the conduction term ``div(k grad T)`` of Eqs. 30 and 34 is ``D(k_f G T)``
  with the arithmetic face mean of k (the same operator as the pressure's);
  the z walls are adiabatic (zero heat flux), x and y periodic;
* the momentum predictor (Eqs. 29, 32) has no-slip z walls (and no-slip y
  walls when y is bounded); the density on a face and the viscosity on an
  edge are arithmetic means of the cells around them; a velocity is carried to an edge by the mean of its two
  values in x, y or z;
  the surface-tension force of the VOF model is out of scope (a caller
  force may stand in for it); the first step is forward Euler.

Pins (tests/test_oracle_pins.py): the single-mode closed form, dense LU
solves of systems assembled entry by entry, exact-linear-field identities of
D and G, the projection invariants, the constant-density reduction and the
agreement of Algorithm 1 with the direct sparse solve.  With y walls: the
cosine eigenmode in y, the even extension to a periodic problem of twice the
width, dense LU with closed walls and the y-independent reduction.  ``adjoint_*`` is
pinned by central finite differences of ``projection_direct`` and by the
dot-product identity.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "Grid", "mixture_density", "divergence", "gradient", "face_density",
    "volume_mean", "laplacian", "solve_constant", "method3", "projection_direct",
    "correct_velocity", "adjoint_direct", "adjoint_method3", "method1", "method2",
    "conduction", "gas_volume", "p0_rate", "dp0dt_extrapolate", "divergence_source",
    "convection", "viscous", "predictor_rhs", "predictor", "method1_rho_tilde",
    "method1_correction", "method2_rho_tilde", "ab2_weights",
]


# Threads of scipy's FFTs (the batch of 1-D transforms is split among them;
# the arithmetic of each transform does not depend on it).  The rest of the
# oracle is plain single-threaded numpy.
WORKERS = os.cpu_count() or 1


class Grid:
    """MAC grid: nx x ny cells of uniform width in x and y, nz cells in z with
    face coordinates ``zf`` (length nz + 1, increasing).  Sec. 3 uses uniform
    spacing; a stretched ``zf`` is allowed.  x is periodic, z has walls, y is
    periodic unless ``ywalls``.  With ``ywalls``, ``yf`` (ny + 1 increasing
    face coordinates spanning ``ly``) makes the y spacing non-uniform too."""

    def __init__(self, nx, ny, nz, lx, ly, zf, ywalls=False, yf=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.ywalls = bool(ywalls)
        self.lx, self.ly = float(lx), float(ly)
        zf = np.asarray(zf, dtype=np.float64)
        if zf.shape != (self.nz + 1,) or np.any(np.diff(zf) <= 0):
            raise ValueError("zf must hold nz + 1 increasing face coordinates")
        self.zf = zf
        self.dx = self.lx / self.nx
        self.dy = self.ly / self.ny
        self.ystretched = yf is not None
        if self.ystretched:
            yf = np.asarray(yf, dtype=np.float64)
            if not self.ywalls:
                raise ValueError("a stretched y needs walls in y")
            if yf.shape != (self.ny + 1,) or np.any(np.diff(yf) <= 0):
                raise ValueError("yf must hold ny + 1 increasing face coordinates")
            if abs((yf[-1] - yf[0]) - self.ly) > 1e-12 * self.ly:
                raise ValueError("yf must span ly")
            self.yf = yf
            self.dyf = yf[1:] - yf[:-1]                 # width of row j
            yc = 0.5 * (yf[1:] + yf[:-1])
            self.dyc = np.zeros(self.ny)                # centre distance across y-face j
            self.dyc[1:] = yc[1:] - yc[:-1]             # (face 0: the walls)
        self.dzf = zf[1:] - zf[:-1]                     # width of cell k
        self.zc = 0.5 * (zf[1:] + zf[:-1])              # centre of cell k
        self.dzc = np.zeros(self.nz + 1)                # centre distance across z-face k
        self.dzc[1:-1] = self.zc[1:] - self.zc[:-1]
        self.lz = zf[-1] - zf[0]

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def cell_volume(self):
        """Delta V of every cell, broadcastable to the cell shape."""
        if self.ystretched:
            return (self.dx * self.dyf)[None, :, None] * self.dzf[:, None, None]
        return (self.dx * self.dy * self.dzf)[:, None, None]


def mixture_density(phi, rho_g, rho_l):
    """Eq. 22 with the indicator H replaced by the cell volume fraction Phi:
    rho = rho_g Phi + rho_l (1 - Phi)."""
    phi = np.asarray(phi, dtype=np.float64)
    return rho_g * phi + rho_l * (1.0 - phi)


def divergence(g, u, v, w):
    """Discrete divergence D: faces -> cell centres (Sec. 3, MAC grid).  With
    y walls no flux crosses them: the wall row of v counts as zero."""
    if g.ywalls:
        v = np.array(v, dtype=np.float64, copy=True)
        v[:, 0, :] = 0.0
    dyf = g.dyf[None, :, None] if g.ystretched else g.dy
    return ((np.roll(u, -1, axis=2) - u) / g.dx
            + (np.roll(v, -1, axis=1) - v) / dyf
            + (w[1:] - w[:-1]) / g.dzf[:, None, None])


def gradient(g, p):
    """Discrete gradient G: cell centres -> faces.  The wall faces carry a
    zero gradient (homogeneous Neumann pressure at no-penetration walls)."""
    gx = (p - np.roll(p, 1, axis=2)) / g.dx
    if g.ystretched:
        gy = np.zeros(g.shape)
        gy[:, 1:] = (p[:, 1:] - p[:, :-1]) / g.dyc[None, 1:, None]
    else:
        gy = (p - np.roll(p, 1, axis=1)) / g.dy
    if g.ywalls:
        gy[:, 0, :] = 0.0
    gz = np.zeros((g.nz + 1, g.ny, g.nx))
    gz[1:-1] = (p[1:] - p[:-1]) / g.dzc[1:-1, None, None]
    return gx, gy, gz


def face_density(g, rho):
    """Density on the faces: arithmetic mean of the two cells sharing the face.
    The wall z-faces take the value of their only cell (it never enters: both
    G p and the velocity vanish there)."""
    rx = 0.5 * (rho + np.roll(rho, 1, axis=2))
    ry = 0.5 * (rho + np.roll(rho, 1, axis=1))
    rz = np.empty((g.nz + 1, g.ny, g.nx))
    rz[1:-1] = 0.5 * (rho[1:] + rho[:-1])
    rz[0] = rho[0]
    rz[-1] = rho[-1]
    return rx, ry, rz


def volume_mean(g, f):
    """Volume-weighted mean of a cell field."""
    dv = g.cell_volume()
    if g.ystretched:
        return float(np.sum(f * dv) / (np.sum(dv) * g.nx))
    return float(np.sum(f * dv) / (np.sum(dv) * g.nx * g.ny))


def laplacian(g, p):
    """L = D G, the compact 7-point operator."""
    return divergence(g, *gradient(g, p))


def _z_coefficients(g):
    """Sub- and super-diagonal of the z part of L in one column:
    (L_z p)_k = a_k p_{k-1} - (a_k + c_k) p_k + c_k p_{k+1}, with no flux
    through the walls."""
    a = np.zeros(g.nz)
    c = np.zeros(g.nz)
    a[1:] = 1.0 / (g.dzc[1:-1] * g.dzf[1:])
    c[:-1] = 1.0 / (g.dzc[1:-1] * g.dzf[:-1])
    return a, c


def _y_eigenbasis(g):
    """Eigenpairs of the y part of L on a stretched y bounded by walls.

    (L_y p)_j = [(p_{j+1} - p_j)/dyc_{j+1} - (p_j - p_{j-1})/dyc_j] / dyf_j,
    with the wall terms absent, is W^{-1} T with W = diag(dyf) and T
    symmetric tridiagonal, so its eigenvectors solve T v = lambda W v:
    scipy's generalized symmetric eigensolver returns them W-orthonormal
    (V^T W V = I).  Ordered from lambda = 0 (the constant vector, written
    exactly) to the most negative."""
    ny = g.ny
    T = np.zeros((ny, ny))
    for j in range(1, ny):
        c = 1.0 / g.dyc[j]
        T[j, j] -= c
        T[j - 1, j - 1] -= c
        T[j, j - 1] = c
        T[j - 1, j] = c
    lam, V = sla.eigh(T, np.diag(g.dyf))
    order = np.argsort(-lam)
    lam, V = lam[order].copy(), V[:, order].copy()
    lam[0] = 0.0
    V[:, 0] = 1.0 / np.sqrt(g.ly)
    return lam, V


def solve_constant(g, f):
    """Constant-coefficient pressure solve by the eigenexpansion method
    (Sec. 3.3.1: homogeneous pressure boundary conditions, solved exactly).

    Returns the zero-mean p with ``D G p = f - <f>_V``.  Steps: real DFT in x,
    complex DFT in y (scipy's FFT), one tridiagonal system per (kx, ky) along
    z with the eigenvalues of the periodic second difference on its diagonal
    (Thomas algorithm), the singular (0, 0) column by a bordered dense solve
    that fixes its zero weighted mean, then the inverse DFTs.

    With y walls the y step is the eigenbasis of the Neumann second
    difference on cell centres, cos(pi m (j + 1/2) / ny), m = 0 .. ny - 1,
    with eigenvalues -(4 / dy^2) sin^2(pi m / (2 ny)): scipy's DCT-II and its
    inverse.  On a stretched y it is the W-orthonormal eigenbasis V of
    ``_y_eigenbasis``: coefficients V^T W f forward, V c back.
    """
    nx, ny, nz = g.nx, g.ny, g.nz
    fc = f - volume_mean(g, f)
    kx = np.arange(nx // 2 + 1)
    ky = np.arange(ny)
    if g.ystretched:
        lam_y, V = _y_eigenbasis(g)
        fh = sfft.rfft(fc, axis=2, workers=WORKERS)
        fh = np.einsum("mj,kji->kmi", V.T * g.dyf[None, :], fh)
    elif g.ywalls:
        fh = sfft.rfft(fc, axis=2, workers=WORKERS)
        fh = (sfft.dct(fh.real, type=2, axis=1, workers=WORKERS)
              + 1j * sfft.dct(fh.imag, type=2, axis=1, workers=WORKERS))
        lam_y = -4.0 / g.dy ** 2 * np.sin(np.pi * ky / (2 * ny)) ** 2
    else:
        fh = sfft.rfft2(fc, axes=(1, 2), workers=WORKERS)   # [nz, ny, nx//2 + 1]
        lam_y = -4.0 / g.dy ** 2 * np.sin(np.pi * ky / ny) ** 2
    lam = (-4.0 / g.dx ** 2 * np.sin(np.pi * kx / nx) ** 2)[None, :] + lam_y[:, None]
    a, c = _z_coefficients(g)
    lam_safe = lam.copy()
    lam_safe[0, 0] = -1.0                               # replaced below
    # Thomas algorithm, vectorised over all (kx, ky) columns.
    dprime = np.empty((nz,) + lam.shape)
    y = np.empty_like(fh)
    dprime[0] = -(a[0] + c[0]) + lam_safe
    y[0] = fh[0]
    for k in range(1, nz):
        m = a[k] / dprime[k - 1]
        dprime[k] = (-(a[k] + c[k]) + lam_safe) - m * c[k - 1]
        y[k] = fh[k] - m * y[k - 1]
    ph = np.empty_like(fh)
    ph[nz - 1] = y[nz - 1] / dprime[nz - 1]
    for k in range(nz - 2, -1, -1):
        ph[k] = (y[k] - c[k] * ph[k + 1]) / dprime[k]
    # (kx, ky) = (0, 0): L_z x + mu 1 = f, sum_k dzf_k x_k = 0.
    lz = np.zeros((nz + 1, nz + 1))
    for k in range(nz):
        lz[k, k] = -(a[k] + c[k])
        if k > 0:
            lz[k, k - 1] = a[k]
        if k < nz - 1:
            lz[k, k + 1] = c[k]
        lz[k, nz] = 1.0
        lz[nz, k] = g.dzf[k]
    rhs = np.zeros(nz + 1, dtype=np.complex128)
    rhs[:nz] = fh[:, 0, 0]
    ph[:, 0, 0] = np.linalg.solve(lz, rhs)[:nz]
    if g.ystretched:
        ph = np.einsum("jm,kmi->kji", V, ph)
        p = sfft.irfft(ph, n=nx, axis=2, workers=WORKERS)
    elif g.ywalls:
        ph = (sfft.idct(ph.real, type=2, axis=1, workers=WORKERS)
              + 1j * sfft.idct(ph.imag, type=2, axis=1, workers=WORKERS))
        p = sfft.irfft(ph, n=nx, axis=2, workers=WORKERS)
    else:
        p = sfft.irfft2(ph, s=(ny, nx), axes=(1, 2), workers=WORKERS)
    return p - volume_mean(g, p)


def correct_velocity(g, us, vs, ws, rho, p, dt):
    """Correction step, Eq. (eqn:corr): u = u* - (dt / rho_f) G p.  Wall
    faces carry zero normal velocity."""
    rx, ry, rz = face_density(g, rho)
    gx, gy, gz = gradient(g, p)
    v = vs - dt * gy / ry
    if g.ywalls:
        v[:, 0, :] = 0.0
    return us - dt * gx / rx, v, ws - dt * gz / rz


def method3(g, us, vs, ws, rho, S, dt, rtol=1e-13, maxit=1000):
    """Method III, Algorithm 1 (Sec. 3.3.1), in the paper's order.

    The two loop-invariant terms of Eq. (eqn:new_poisson), D(rho u*) and
    rho D u^{n+1} with D u^{n+1} = S_c, are formed once before the loop, as
    the paper notes.  Each pass builds the right-hand side with the current
    ``u^s . grad(rho)`` (centred: ``D(rho_f u^s) - rho_c D u^s``), solves the
    constant-coefficient equation, applies the correction step and evaluates
    the residual ``D u^{s+1} - S_c``.

    Returns ``(p, u, v, w, info)`` with ``info`` holding the iteration count,
    the relative L2 residual history and the paper's L1 sum.
    """
    Sc = S - volume_mean(g, S)
    rx, ry, rz = face_density(g, rho)
    pre = divergence(g, rx * us, ry * vs, rz * ws) - rho * Sc
    res0 = np.linalg.norm((divergence(g, us, vs, ws) - Sc).ravel())
    u, v, w = us, vs, ws
    p = np.zeros(g.shape)
    hist = []
    eps_l1 = float(np.sum(np.abs(divergence(g, us, vs, ws) - Sc)))
    if res0 == 0.0:
        return p, u, v, w, {"iters": 0, "res_hist": [], "res_l1_sum": eps_l1,
                            "res0": 0.0, "mean_S_removed": volume_mean(g, S)}
    s = 0
    while s < maxit:
        conv = divergence(g, rx * u, ry * v, rz * w) - rho * divergence(g, u, v, w)
        rhs = (pre - conv) / dt
        p = solve_constant(g, rhs)
        u, v, w = correct_velocity(g, us, vs, ws, rho, p, dt)
        d = divergence(g, u, v, w) - Sc
        eps_l1 = float(np.sum(np.abs(d)))
        hist.append(float(np.linalg.norm(d.ravel()) / res0))
        s += 1
        if hist[-1] <= rtol:
            break
    info = {"iters": s, "res_hist": hist, "res_l1_sum": eps_l1, "res0": float(res0),
            "mean_S_removed": volume_mean(g, S)}
    return p, u, v, w, info


def method1(g, us, vs, ws, rho, S, dt, rtol=1e-13, maxit=5000):
    """Method I (Sec. 3.3.1, Eqs. poisson_me1 and poisson_me2), written as
    the paper states it: with rho0 = min rho,
        L p^{s+1} = D((1 - rho0/rho_f) G p^s) + (rho0/dt)(D u* - S_c),
    iterated from p^0 = 0; then the modified correction
        u = u* - dt [ (1/rho0) G p^{n+1} + (1/rho_f - 1/rho0) G p^{n+1,q} ]
    with p^{n+1,q} the second-to-last iterate.  The stopping rule is the one
    used for Method III (relative L2 norm of D u - S_c, u from Eq. corr at the
    current iterate) so that iteration counts compare; the paper's own
    measure ||p^{s+1} - p^s|| is reported in the history."""
    Sc = S - volume_mean(g, S)
    rx, ry, rz = face_density(g, rho)
    rho0 = method1_rho_tilde(rho)
    pre = (rho0 / dt) * (divergence(g, us, vs, ws) - Sc)
    res0 = np.linalg.norm((divergence(g, us, vs, ws) - Sc).ravel())
    p = np.zeros(g.shape)
    p_prev = p
    hist, dp_hist = [], []
    s = 0
    while s < maxit and res0 > 0:
        gx, gy, gz = gradient(g, p)
        rhs = divergence(g, (1.0 - rho0 / rx) * gx, (1.0 - rho0 / ry) * gy, (1.0 - rho0 / rz) * gz) + pre
        p_prev, p = p, solve_constant(g, rhs)
        u, v, w = correct_velocity(g, us, vs, ws, rho, p, dt)
        hist.append(float(np.linalg.norm((divergence(g, u, v, w) - Sc).ravel()) / res0))
        dp_hist.append(float(np.linalg.norm((p - p_prev).ravel())))
        s += 1
        if hist[-1] <= rtol:
            break
    u, v, w = method1_correction(g, us, vs, ws, rho, rho0, p, p_prev, dt)
    return p, u, v, w, {"iters": s, "res_hist": hist, "dp_hist": dp_hist, "rho_tilde": rho0}


def method1_rho_tilde(rho):
    """Eq. poisson_me1: the constant density of Method I is the smallest
    density in the domain."""
    return float(np.min(rho))


def method1_correction(g, us, vs, ws, rho, rho0, p, p_q, dt):
    """Eq. poisson_me2, Method I's modified correction:
    u = u* - dt [ (1/rho0) G p + (1/rho_f - 1/rho0) G p^q ], with p the last
    iterate and p^q the one before it."""
    rx, ry, rz = face_density(g, rho)
    gx, gy, gz = gradient(g, p)
    qx, qy, qz = gradient(g, p_q)
    u = us - dt * (gx / rho0 + (1.0 / rx - 1.0 / rho0) * qx)
    v = vs - dt * (gy / rho0 + (1.0 / ry - 1.0 / rho0) * qy)
    w = ws - dt * (gz / rho0 + (1.0 / rz - 1.0 / rho0) * qz)
    return u, v, w


def method2_rho_tilde(rho):
    """Eq. poisson_laizet: the harmonic mean of the two phase densities,
    taken as the smallest and largest density in the domain (reading R17)."""
    rmin, rmax = float(np.min(rho)), float(np.max(rho))
    return 2.0 * rmin * rmax / (rmin + rmax)


def method2(g, us, vs, ws, rho, S, dt, rtol=1e-13, maxit=5000):
    """Method II (Sec. 3.3.1, Eq. poisson_laizet), written as the paper
    states it: with rho~ the harmonic mean of the two phase densities (here
    of min rho and max rho),
        L p^{s+1} = L p^s + rho~ [ (D u* - S_c)/dt - D(rho_f^{-1} G p^s) ],
    from p^0 = 0, then the correction of Eq. corr.  Same stopping rule as
    method3."""
    Sc = S - volume_mean(g, S)
    rx, ry, rz = face_density(g, rho)
    rt = method2_rho_tilde(rho)
    b = (divergence(g, us, vs, ws) - Sc) / dt
    res0 = np.linalg.norm((b * dt).ravel())
    p = np.zeros(g.shape)
    hist = []
    s = 0
    while s < maxit and res0 > 0:
        gx, gy, gz = gradient(g, p)
        rhs = laplacian(g, p) + rt * (b - divergence(g, gx / rx, gy / ry, gz / rz))
        p = solve_constant(g, rhs)
        u, v, w = correct_velocity(g, us, vs, ws, rho, p, dt)
        hist.append(float(np.linalg.norm((divergence(g, u, v, w) - Sc).ravel()) / res0))
        s += 1
        if hist[-1] <= rtol:
            break
    u, v, w = correct_velocity(g, us, vs, ws, rho, p, dt)
    return p, u, v, w, {"iters": s, "res_hist": hist, "rho_tilde": rt}


# ---------------------------------------------------------------------------
# Direct solve of the variable-coefficient equation (small grids)
# ---------------------------------------------------------------------------

def _index(g):
    return np.arange(g.nx * g.ny * g.nz).reshape(g.shape)


def _sparse_operators(g):
    """Sparse D (cells x faces) and G (faces x cells).  Face unknowns are
    ordered [u (nz*ny*nx), v (nz*ny*nx), w (nz+1)*ny*nx]."""
    nx, ny, nz = g.nx, g.ny, g.nz
    nc = nx * ny * nz
    cid = _index(g)
    nu = nc
    nw = (nz + 1) * ny * nx
    fid_u = cid
    fid_v = nu + cid
    fid_w = 2 * nu + np.arange(nw).reshape(nz + 1, ny, nx)
    rows, cols, vals = [], [], []

    def add(r, cidx, val):
        rows.append(r.ravel()); cols.append(cidx.ravel())
        vals.append(np.broadcast_to(val, r.shape).ravel())

    # D: (u_{i+1} - u_i)/dx + (v_{j+1} - v_j)/dy + (w_{k+1} - w_k)/dzf_k;
    # with y walls the wall row of v (row 0, both walls) gets no entries.
    vopen = np.ones(g.shape)
    if g.ywalls:
        vopen[:, 0, :] = 0.0
    add(cid, np.roll(fid_u, -1, axis=2), 1.0 / g.dx)
    add(cid, fid_u, -1.0 / g.dx)
    if g.ystretched:
        dyf = np.broadcast_to(g.dyf[None, :, None], g.shape)
        add(cid, np.roll(fid_v, -1, axis=1), np.roll(vopen, -1, axis=1) / dyf)
        add(cid, fid_v, -vopen / dyf)
    else:
        add(cid, np.roll(fid_v, -1, axis=1), np.roll(vopen, -1, axis=1) / g.dy)
        add(cid, fid_v, -vopen / g.dy)
    inv_dzf = np.broadcast_to((1.0 / g.dzf)[:, None, None], g.shape)
    add(cid, fid_w[1:], inv_dzf)
    add(cid, fid_w[:-1], -inv_dzf)
    D = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nc, 2 * nu + nw))
    rows, cols, vals = [], [], []
    # G: x-face i: (p_i - p_{i-1})/dx; y likewise; interior z-face k:
    # (p_k - p_{k-1})/dzc_k; wall z-faces: no rows (zero gradient).
    add(fid_u, cid, 1.0 / g.dx)
    add(fid_u, np.roll(cid, 1, axis=2), -1.0 / g.dx)
    if g.ystretched:
        # y-face j (j >= 1): (p_j - p_{j-1})/dyc_j; the wall row has no entries
        dyc = np.broadcast_to(np.where(g.dyc > 0, g.dyc, 1.0)[None, :, None], g.shape)
        add(fid_v, cid, vopen / dyc)
        add(fid_v, np.roll(cid, 1, axis=1), -vopen / dyc)
    else:
        add(fid_v, cid, vopen / g.dy)
        add(fid_v, np.roll(cid, 1, axis=1), -vopen / g.dy)
    inv_dzc = np.broadcast_to((1.0 / g.dzc[1:-1])[:, None, None], (nz - 1, ny, nx))
    add(fid_w[1:-1], cid[1:], inv_dzc)
    add(fid_w[1:-1], cid[:-1], -inv_dzc)
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * nu + nw, nc))
    return D, G


def _face_vector(u, v, w):
    return np.concatenate([u.ravel(), v.ravel(), w.ravel()])


def _split_faces(g, x):
    nc = g.nx * g.ny * g.nz
    return (x[:nc].reshape(g.shape), x[nc:2 * nc].reshape(g.shape),
            x[2 * nc:].reshape(g.nz + 1, g.ny, g.nx))


def _beta_vector(g, rho):
    rx, ry, rz = face_density(g, rho)
    return 1.0 / _face_vector(rx, ry, rz)


def _bordered_solve(g, A, rhs):
    """Solve A p = rhs - mu (mu a scalar) with sum dV p = 0.  A has the
    constant vector as null vector; mu takes up any incompatible part."""
    n = A.shape[0]
    dv = np.broadcast_to(g.cell_volume(), g.shape).ravel()
    K = sp.bmat([[A, sp.csr_matrix(np.ones((n, 1)))],
                 [sp.csr_matrix(dv[None, :]), None]], format="csc")
    sol = spla.spsolve(K, np.concatenate([rhs, [0.0]]))
    return sol[:n]


def projection_direct(g, us, vs, ws, rho, S, dt):
    """The plain definition the projection reaches: the zero-mean p with
    D(rho_f^{-1} G p) = (D u* - S_c)/dt (Eq. lap_p with the target
    divergence S_c), and u^{n+1} = u* - dt rho_f^{-1} G p (Eq. corr).
    Sparse direct solve; for grids up to about 24^3."""
    D, G = _sparse_operators(g)
    beta = _beta_vector(g, rho)
    A = (D @ sp.diags(beta) @ G).tocsr()
    Sc = S - volume_mean(g, S)
    rhs = (D @ _face_vector(us, vs, ws) - Sc.ravel()) / dt
    p = _bordered_solve(g, A, rhs)
    un = _face_vector(us, vs, ws) - dt * beta * (G @ p)
    u, v, w = _split_faces(g, un)
    return p.reshape(g.shape), u, v, w


# ---------------------------------------------------------------------------
# Adjoint of the converged projection
# ---------------------------------------------------------------------------
#
# With beta = 1/rho_f (face-wise), B = diag(beta), A = D B G and the
# gauge-fixed solve of A p = (D u* - S_c)/dt, the projection is
#     u^{n+1} = u* - dt B G p.
# For an upstream gradient g = dL/du^{n+1} (wall z-faces excluded: they are
# not unknowns, w = 0 there), implicit differentiation gives
#     g_u*   = g - D^T lambda,        A^T lambda = G^T B g,  sum(lambda) = 0,
#     g_beta = -dt (G p) * g_u*       (face-wise),
#     g_rho  = sum over the faces of a cell of g_beta * (-beta^2 / 2)
# (beta_f = 2/(rho_a + rho_b) on interior faces; wall faces do not depend on
# rho).  rho_c's role as the scaling inside Algorithm 1 does not change the
# fixed point, so it contributes nothing.


def _zero_walls(gw):
    gw = np.array(gw, dtype=np.float64, copy=True)
    gw[0] = 0.0
    gw[-1] = 0.0
    return gw


def _zero_ywall_row(g, gv):
    """With y walls the wall row of v (row 0, both walls) is not an unknown
    either: its gradient is defined as zero, like the wall planes of w."""
    gv = np.array(gv, dtype=np.float64, copy=True)
    if g.ywalls:
        gv[:, 0, :] = 0.0
    return gv


def _bordered_solve_transposed(g, A, rhs):
    """Solve A^T x = rhs with sum(x) = 0.  A^T has the volume vector as null
    vector and the constant vector as left null vector, so a compatible rhs
    has zero plain sum; the bordering scalar takes up round-off."""
    n = A.shape[0]
    dv = np.broadcast_to(g.cell_volume(), g.shape).ravel()
    K = sp.bmat([[A.T.tocsr(), sp.csr_matrix(dv[:, None])],
                 [sp.csr_matrix(np.ones((1, n))), None]], format="csc")
    sol = spla.spsolve(K, np.concatenate([rhs, [0.0]]))
    return sol[:n]


def _beta_to_rho(g, beta, gbeta):
    """Pull a face gradient w.r.t. beta_f = 2/(rho_a + rho_b) back to the
    cells: d beta_f / d rho = -beta_f^2 / 2 for both cells of the face."""
    bu, bv, bw = _split_faces(g, beta)
    gu, gv, gw = _split_faces(g, gbeta)
    tu = -0.5 * bu ** 2 * gu
    tv = -0.5 * bv ** 2 * gv
    tw = -0.5 * bw ** 2 * gw
    tw[0] = 0.0
    tw[-1] = 0.0
    # x-face i touches cells i-1 and i; y likewise; z-face k touches k-1, k.
    out = tu + np.roll(tu, -1, axis=2) + tv + np.roll(tv, -1, axis=1)
    return out + tw[:-1] + tw[1:]


def adjoint_direct(g, us, vs, ws, rho, S, dt, gu, gv, gw):
    """Gradients of L(u^{n+1}) w.r.t. u* and rho_c by implicit
    differentiation of the plain definition (``projection_direct``), with
    literal sparse transposes.  Small grids only.  Returns
    ``(g_us, g_vs, g_ws, g_rho)``; wall entries of ``g_ws`` (and, with y
    walls, the wall row of ``g_vs``) are zero."""
    D, G = _sparse_operators(g)
    beta = _beta_vector(g, rho)
    A = (D @ sp.diags(beta) @ G).tocsr()
    Sc = S - volume_mean(g, S)
    rhs = (D @ _face_vector(us, vs, ws) - Sc.ravel()) / dt
    p = _bordered_solve(g, A, rhs)
    gvec = _face_vector(gu, _zero_ywall_row(g, gv), _zero_walls(gw))
    lam = _bordered_solve_transposed(g, A, G.T @ (beta * gvec))
    gus = gvec - D.T @ lam
    u, v, w = _split_faces(g, gus)
    w = _zero_walls(w)
    v = _zero_ywall_row(g, v)
    gus = _face_vector(u, v, w)
    grho = _beta_to_rho(g, beta, -dt * (G @ p) * gus)
    return u, v, w, grho


def adjoint_method3(g, us, vs, ws, rho, S, dt, gu, gv, gw, rtol=1e-13, maxit=1000, p=None):
    """The same gradients for any grid size, with Algorithm 1 as the solver.

    With W_c = diag(dzf) on cells and W_f = diag(dzf of the layer) on x/y
    faces, diag(dzc) on z faces (on a stretched y: W_c = diag(dzf dyf), and
    dzf dyf, dzf dyc, dzc dyf on x, y, z faces), the discrete operators satisfy
    D^T = -W_f G W_c^{-1} and G^T = -W_c D W_f^{-1}; hence
    A^T = W_c A W_c^{-1}, and lambda = W_c mu with
        A mu = -D(B W_f^{-1} g),
    which is the projection equation with u* = -dt B W_f^{-1} g and S = 0.
    Then g_u* = g + W_f G mu (the gauge of mu does not matter).
    ``p`` is the converged pressure of the forward projection (computed
    here with the same tolerance when not given).
    """
    gw = _zero_walls(gw)
    gv = _zero_ywall_row(g, gv)
    rx, ry, rz = face_density(g, rho)
    wlay = g.dzf[:, None, None]
    wz = np.ones(g.nz + 1)
    wz[1:-1] = g.dzc[1:-1]
    wz = wz[:, None, None]
    if g.ystretched:
        # W_c = diag(dzf dyf) and the face weights of D^T = -W_f G W_c^{-1}
        # on a stretched y: dzf dyf on x faces, dzf dyc on y faces (the wall
        # row carries no unknown), dzc dyf on z faces
        dyc = np.where(g.dyc > 0, g.dyc, 1.0)[None, :, None]
        wx = wlay * g.dyf[None, :, None]
        wy = wlay * dyc
        wz = wz * g.dyf[None, :, None]
    else:
        wx = wy = wlay
    ya, yb, yc = gu / (rx * wx), gv / (ry * wy), gw / (rz * wz)
    zero = np.zeros(g.shape)
    mu, _, _, _, info_adj = method3(g, -dt * ya, -dt * yb, -dt * yc, rho, zero, dt,
                                    rtol=rtol, maxit=maxit)
    gx, gy, gz = gradient(g, mu)
    gus, gvs, gws = gu + wx * gx, gv + wy * gy, gw + wz * gz
    gws = _zero_walls(gws)
    gvs = _zero_ywall_row(g, gvs)
    info_fwd = None
    if p is None:
        p, _, _, _, info_fwd = method3(g, us, vs, ws, rho, S, dt, rtol=rtol, maxit=maxit)
    px, py, pz = gradient(g, p)
    gbeta = _face_vector(-dt * px * gus, -dt * py * gvs, -dt * pz * gws)
    beta = 1.0 / _face_vector(rx, ry, rz)
    grho = _beta_to_rho(g, beta, gbeta)
    return gus, gvs, gws, grho, {"fwd": info_fwd, "adj": info_adj}


# ---------------------------------------------------------------------------
# The divergence source from the thermodynamics (Sec. 2, final_p0; Sec. 3.2,
# Eqs. 30 and v_gas; Sec. 3.3, Eq. 34 and the extrapolation of dp0/dt)

def conduction(g, kc, T):
    """div(k grad T) at the cell centres, second-order central: D(k_f G T)
    with k_f the arithmetic mean of the two cells of a face; G T is zero on
    the z walls (adiabatic walls)."""
    kx, ky, kz = face_density(g, kc)
    gx, gy, gz = gradient(g, T)
    return divergence(g, kx * gx, ky * gy, kz * gz)


def gas_volume(g, phi):
    """Eq. v_gas: V_g = sum of Phi dV over the cells (dV = dx dy dzf_k)."""
    return float(np.sum(phi * g.cell_volume()))


def p0_rate(g, phi, kc, T, u, v, w, p0, gamma):
    """Eq. 30 (final_p0 with the volume integrals as cell sums):
    RP = (gamma / V_g) [ (gamma - 1)/gamma sum Phi div(k grad T) dV
                         - p0 sum Phi div(u) dV ]."""
    dv = g.cell_volume()
    vg = gas_volume(g, phi)
    a = float(np.sum(phi * conduction(g, kc, T) * dv))
    b = float(np.sum(phi * divergence(g, u, v, w) * dv))
    return gamma / vg * ((gamma - 1.0) / gamma * a - p0 * b)


def dp0dt_extrapolate(rp_n, rp_nm1, dt_new, dt_old):
    """Sec. 3.3: (dp0/dt)^{n+1} ~ (1 + dt^{n+1}/dt^n) RP^n - (dt^{n+1}/dt^n) RP^{n-1}."""
    r = dt_new / dt_old
    return (1.0 + r) * rp_n - r * rp_nm1


def divergence_source(g, phi, kc, T, p0, gamma, dp0dt):
    """Eq. 34: S = (1/p0) [ (gamma - 1)/gamma div(k grad T) - (1/gamma) dp0/dt ] Phi."""
    return ((gamma - 1.0) / gamma * conduction(g, kc, T) - dp0dt / gamma) * phi / p0


# ---------------------------------------------------------------------------
# Momentum predictor (Sec. 3.3, Eqs. 29 and 32): u* = u^n + dt [(1 + r/2) RU^n
# - (r/2) RU^{n-1}], RU = -C(u) + (1/rho_f)[div tau(mu, u) + f] + g, with the
# Newton-Stokes stress tau = mu [(grad u + grad u^T) - (2/3)(div u) I] (Sec. 2)
# and the convection in divergence form C(u) = div(u u) - u div(u).  Central
# second-order differences on the MAC grid; z walls are no-slip.

def _zinterp(g, a):
    """Layered a (nz layers) carried to the interior z-faces 1..nz-1 by the
    mean of the two layers (returned with nz + 1 planes, wall planes zero).
    On the paper's uniform grid this is the central interpolation and keeps
    the convection term energy-conserving; on a stretched z it stays second
    order for smooth stretching."""
    out = np.zeros((g.nz + 1,) + a.shape[1:])
    out[1:-1] = 0.5 * (a[1:] + a[:-1])
    return out


def convection(g, u, v, w):
    """C(u) = div(u u) - u div(u) at the u, v and w points (w: interior faces;
    the wall planes are zero).  Products live at cell centres (normal terms)
    and at cell edges (cross terms); a velocity is carried to an edge by the
    mean of its two values in x, y or z.  With y walls the wall row of v is
    zero (no-penetration), so every product on a y-wall edge vanishes, and
    the wall row of C_y is zero.  Uniform y only."""
    if g.ystretched:
        raise NotImplementedError("convection: uniform y only")
    if g.ywalls:
        v = np.array(v, dtype=np.float64, copy=True)
        v[:, 0, :] = 0.0
    D = divergence(g, u, v, w)
    # normal fluxes at cell centres
    fxx = (0.5 * (u + np.roll(u, -1, axis=2))) ** 2
    fyy = (0.5 * (v + np.roll(v, -1, axis=1))) ** 2
    wc = 0.5 * (w[1:] + w[:-1])
    fzz = wc ** 2
    # cross fluxes at edges: xy edge (i-1/2, j-1/2), xz edge (i-1/2, k-1/2), yz edge (j-1/2, k-1/2)
    fxy = 0.5 * (u + np.roll(u, 1, axis=1)) * 0.5 * (v + np.roll(v, 1, axis=2))
    fxz = _zinterp(g, u) * 0.5 * (w + np.roll(w, 1, axis=2))
    fyz = _zinterp(g, v) * 0.5 * (w + np.roll(w, 1, axis=1))
    dzf = g.dzf[:, None, None]
    cx = ((fxx - np.roll(fxx, 1, axis=2)) / g.dx + (np.roll(fxy, -1, axis=1) - fxy) / g.dy
          + (fxz[1:] - fxz[:-1]) / dzf - u * 0.5 * (D + np.roll(D, 1, axis=2)))
    cy = ((np.roll(fxy, -1, axis=2) - fxy) / g.dx + (fyy - np.roll(fyy, 1, axis=1)) / g.dy
          + (fyz[1:] - fyz[:-1]) / dzf - v * 0.5 * (D + np.roll(D, 1, axis=1)))
    cz = np.zeros((g.nz + 1, g.ny, g.nx))
    dzc = g.dzc[1:-1, None, None]
    cz[1:-1] = ((np.roll(fxz[1:-1], -1, axis=2) - fxz[1:-1]) / g.dx
                + (np.roll(fyz[1:-1], -1, axis=1) - fyz[1:-1]) / g.dy
                + (fzz[1:] - fzz[:-1]) / dzc - w[1:-1] * _zinterp(g, D)[1:-1])
    if g.ywalls:
        cy[:, 0, :] = 0.0
    return cx, cy, cz


def viscous(g, mu, u, v, w):
    """div tau at the u, v and w points, tau = mu [(grad u + grad u^T) -
    (2/3)(div u) I].  Normal stresses at cell centres with mu of the cell;
    shear stresses at edges with the mean mu of the (up to) four cells
    around the edge.  No-slip z walls: the wall velocity is zero, so the
    wall shear uses the half-cell distance to the wall.  With y walls the
    same holds there (``_viscous_ywalls``).  Uniform y only."""
    if g.ystretched:
        raise NotImplementedError("viscous: uniform y only")
    if g.ywalls:
        return _viscous_ywalls(g, mu, u, v, w)
    D = divergence(g, u, v, w)
    dzf = g.dzf[:, None, None]
    txx = mu * (2.0 * (np.roll(u, -1, axis=2) - u) / g.dx - 2.0 / 3.0 * D)
    tyy = mu * (2.0 * (np.roll(v, -1, axis=1) - v) / g.dy - 2.0 / 3.0 * D)
    tzz = mu * (2.0 * (w[1:] - w[:-1]) / dzf - 2.0 / 3.0 * D)
    mxy = 0.25 * (mu + np.roll(mu, 1, axis=2) + np.roll(mu, 1, axis=1) + np.roll(np.roll(mu, 1, axis=1), 1, axis=2))
    txy = mxy * ((u - np.roll(u, 1, axis=1)) / g.dy + (v - np.roll(v, 1, axis=2)) / g.dx)

    def edge_z(a, axis):
        """Shear tau_az at the edges between the a-faces and the z-faces
        (nz + 1 planes): interior planes from the two layers, wall planes
        from the first layer and the zero wall velocity."""
        m2 = 0.5 * (mu + np.roll(mu, 1, axis=axis))          # mean over the two cells in x (or y)
        t = np.empty((g.nz + 1, g.ny, g.nx))
        dwd = (w - np.roll(w, 1, axis=axis)) / (g.dx if axis == 2 else g.dy)
        t[1:-1] = 0.5 * (m2[1:] + m2[:-1]) * ((a[1:] - a[:-1]) / g.dzc[1:-1, None, None] + dwd[1:-1])
        t[0] = m2[0] * (a[0] - 0.0) / (g.zc[0] - g.zf[0])
        t[-1] = m2[-1] * (0.0 - a[-1]) / (g.zf[-1] - g.zc[-1])
        return t

    txz = edge_z(u, 2)
    tyz = edge_z(v, 1)
    fx = ((txx - np.roll(txx, 1, axis=2)) / g.dx + (np.roll(txy, -1, axis=1) - txy) / g.dy
          + (txz[1:] - txz[:-1]) / dzf)
    fy = ((np.roll(txy, -1, axis=2) - txy) / g.dx + (tyy - np.roll(tyy, 1, axis=1)) / g.dy
          + (tyz[1:] - tyz[:-1]) / dzf)
    fz = np.zeros((g.nz + 1, g.ny, g.nx))
    fz[1:-1] = ((np.roll(txz[1:-1], -1, axis=2) - txz[1:-1]) / g.dx
                + (np.roll(tyz[1:-1], -1, axis=1) - tyz[1:-1]) / g.dy
                + (tzz[1:] - tzz[:-1]) / g.dzc[1:-1, None, None])
    return fx, fy, fz


def _viscous_ywalls(g, mu, u, v, w):
    """div tau with no-slip walls in y as well as in z.  The wall row of v
    is zero.  Shear stresses on the y-wall edges use the zero wall velocity
    and the half-cell distance to the wall (as at the z walls), so the two
    walls need separate edge rows: tau_xy and tau_yz are kept on ny + 1 edge
    rows (row 0 the wall y = 0, row ny the wall y = ly, rows 1 .. ny - 1
    between cells).  The edges where a y wall meets a z wall carry no shear
    (both velocities vanish there)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    v = np.array(v, dtype=np.float64, copy=True)
    v[:, 0, :] = 0.0
    D = divergence(g, u, v, w)
    dzf = g.dzf[:, None, None]
    txx = mu * (2.0 * (np.roll(u, -1, axis=2) - u) / g.dx - 2.0 / 3.0 * D)
    vtop = np.concatenate([v, np.zeros((nz, 1, nx))], axis=1)      # v on the ny + 1 y-face rows
    tyy = mu * (2.0 * (vtop[:, 1:] - vtop[:, :-1]) / g.dy - 2.0 / 3.0 * D)
    tzz = mu * (2.0 * (w[1:] - w[:-1]) / dzf - 2.0 / 3.0 * D)
    mux = 0.5 * (mu + np.roll(mu, 1, axis=2))                      # mean over the two cells in x
    # tau_xy on the (i - 1/2, j - 1/2) edges, j = 0 .. ny
    txy = np.zeros((nz, ny + 1, nx))
    mxy = 0.5 * (mux[:, 1:] + mux[:, :-1])
    txy[:, 1:-1] = mxy * ((u[:, 1:] - u[:, :-1]) / g.dy + (v[:, 1:] - np.roll(v[:, 1:], 1, axis=2)) / g.dx)
    txy[:, 0] = mux[:, 0] * (u[:, 0] - 0.0) / (0.5 * g.dy)
    txy[:, -1] = mux[:, -1] * (0.0 - u[:, -1]) / (0.5 * g.dy)
    # tau_xz on the (i - 1/2, k - 1/2) edges (as in the periodic case)
    txz = np.empty((nz + 1, ny, nx))
    dwdx = (w - np.roll(w, 1, axis=2)) / g.dx
    txz[1:-1] = 0.5 * (mux[1:] + mux[:-1]) * ((u[1:] - u[:-1]) / g.dzc[1:-1, None, None] + dwdx[1:-1])
    txz[0] = mux[0] * (u[0] - 0.0) / (g.zc[0] - g.zf[0])
    txz[-1] = mux[-1] * (0.0 - u[-1]) / (g.zf[-1] - g.zc[-1])
    # tau_yz on the (j - 1/2, k - 1/2) edges, j = 0 .. ny, k = 0 .. nz
    tyz = np.zeros((nz + 1, ny + 1, nx))
    muz = np.zeros((nz + 1, ny, nx))                               # mean over the two cells in z
    muz[1:-1] = 0.5 * (mu[1:] + mu[:-1])
    myz = 0.5 * (muz[:, 1:] + muz[:, :-1])
    dvdz = (v[1:] - v[:-1]) / g.dzc[1:-1, None, None]
    tyz[1:-1, 1:-1] = myz[1:-1] * (dvdz[:, 1:] + (w[1:-1, 1:] - w[1:-1, :-1]) / g.dy)
    tyz[1:-1, 0] = muz[1:-1, 0] * (w[1:-1, 0] - 0.0) / (0.5 * g.dy)
    tyz[1:-1, -1] = muz[1:-1, -1] * (0.0 - w[1:-1, -1]) / (0.5 * g.dy)
    my2 = 0.5 * (mu + np.roll(mu, 1, axis=1))                      # y faces between cells (row 0 unused)
    tyz[0, 1:-1] = my2[0, 1:] * (v[0, 1:] - 0.0) / (g.zc[0] - g.zf[0])
    tyz[-1, 1:-1] = my2[-1, 1:] * (0.0 - v[-1, 1:]) / (g.zf[-1] - g.zc[-1])
    fx = ((txx - np.roll(txx, 1, axis=2)) / g.dx + (txy[:, 1:] - txy[:, :-1]) / g.dy
          + (txz[1:] - txz[:-1]) / dzf)
    fy = np.zeros((nz, ny, nx))
    fy[:, 1:] = ((np.roll(txy[:, 1:-1], -1, axis=2) - txy[:, 1:-1]) / g.dx
                 + (tyy[:, 1:] - tyy[:, :-1]) / g.dy + (tyz[1:, 1:-1] - tyz[:-1, 1:-1]) / dzf)
    fz = np.zeros((nz + 1, ny, nx))
    fz[1:-1] = ((np.roll(txz[1:-1], -1, axis=2) - txz[1:-1]) / g.dx
                + (tyz[1:-1, 1:] - tyz[1:-1, :-1]) / g.dy
                + (tzz[1:] - tzz[:-1]) / g.dzc[1:-1, None, None])
    return fx, fy, fz


def predictor_rhs(g, u, v, w, rho, mu, grav, force=None):
    """Eq. 32 without the surface-tension force of the VOF model (out of
    scope): RU = -C(u) + (1/rho_f)[div tau + f] + g, with f an optional
    force on the faces (fx, fy, fz) given by the caller.  The w wall planes
    are zero."""
    cx, cy, cz = convection(g, u, v, w)
    vx, vy, vz = viscous(g, mu, u, v, w)
    rx, ry, rz = face_density(g, rho)
    if force is not None:
        vx, vy, vz = vx + force[0], vy + force[1], vz + force[2]
    ru = -cx + vx / rx + grav[0]
    rv = -cy + vy / ry + grav[1]
    rw = -cz + vz / rz + grav[2]
    rw[0] = 0.0
    rw[-1] = 0.0
    if g.ywalls:
        rv[:, 0, :] = 0.0
    return ru, rv, rw


def predictor(g, u, v, w, rho, mu, grav, dt_new, dt_old=None, ru_prev=None, force=None):
    """Eq. 29 (Adams-Bashforth): u* = u^n + dt [(1 + r/2) RU^n - (r/2) RU^{n-1}],
    r = dt_new/dt_old; the first step (no RU^{n-1}) is forward Euler.
    Returns (u*, v*, w*) and RU^n."""
    ru = predictor_rhs(g, u, v, w, rho, mu, grav, force)
    if ru_prev is None:
        a, b = 1.0, 0.0
        ru_prev = (0.0, 0.0, 0.0)
    else:
        a, b = ab2_weights(dt_new, dt_old)
    out = tuple(x + dt_new * (a * q - b * qp) for x, q, qp in zip((u, v, w), ru, ru_prev))
    out[2][0] = 0.0
    out[2][-1] = 0.0
    if g.ywalls:
        out[1][:, 0, :] = 0.0
    return out, ru


def ab2_weights(dt_new, dt_old):
    """Eq. 29's Adams-Bashforth weights for a step dt_new after a step dt_old:
    u* = u^n + dt_new [a RU^n - b RU^{n-1}], a = 1 + r/2, b = r/2,
    r = dt_new / dt_old."""
    r = dt_new / dt_old
    return 1.0 + 0.5 * r, 0.5 * r
