"""Seeded synthetic inputs for the pressure projection.

This module holds no arithmetic of the method: it only draws random fields,
builds grid face coordinates and samples volume fractions of spheres.  The
tests feed the same arrays to the CUDA path and to the CPU oracle.

The paper's own cases (Sec. 4) are two-dimensional whole-solver runs; these
three-dimensional stand-ins follow their structure: a liquid (rho_l) holding
gas bubbles or droplets (rho_g) described by a volume fraction Phi (Eq. 2),
a predicted velocity u*, and a divergence target S that is non-zero only in
the gas (Eq. 34 with uniform temperature: S = -Phi (dp0/dt) / (gamma p0)).

Seeds: workload c uses 1000 + c; sub-seeds add 1 (u), 2 (v), 3 (w),
10 (bubbles), 20 (target velocity), 30 (probe entries).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA_G = 1.4          # ratio of specific heats of the gas (unstated; air)
P0 = 1.0               # thermodynamic pressure (non-dimensional)
DP0_DT = 1e-2          # thermodynamic-pressure rate


def uniform_zfaces(nz: int, lz: float) -> np.ndarray:
    return np.linspace(0.0, lz, nz + 1)


def tanh_zfaces(nz: int, lz: float, beta: float) -> np.ndarray:
    """Faces clustered at both walls: z(xi) = lz/2 (1 + tanh(beta (2 xi - 1)) / tanh(beta))."""
    xi = np.arange(nz + 1) / nz
    z = 0.5 * lz * (1.0 + np.tanh(beta * (2.0 * xi - 1.0)) / math.tanh(beta))
    z[0], z[-1] = 0.0, lz
    return z


def tanh_yfaces(ny: int, ly: float, beta: float) -> np.ndarray:
    """The same clustering for a y bounded by walls (y faces 0 .. ny)."""
    return tanh_zfaces(ny, ly, beta)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    zf: np.ndarray
    dt: float = 1e-3
    us: np.ndarray | None = None
    vs: np.ndarray | None = None
    ws: np.ndarray | None = None
    phi: np.ndarray | None = None
    rho_g: float = 1.0
    rho_l: float = 1.0
    S: np.ndarray | None = None
    extra: dict = field(default_factory=dict)
    ywalls: bool = False      # walls at y = 0 and y = ly (v row 0 is the wall face)
    yf: np.ndarray | None = None  # y face coordinates of a stretched y (walls in y only)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def npts(self):
        return self.nx * self.ny * self.nz


def random_faces(nx, ny, nz, sigma, seed, remove_mean=False, dtype=np.float64, ywalls=False):
    """Face velocities drawn i.i.d. N(0, sigma^2); wall z-faces set to zero
    (and, with ``ywalls``, the wall row 0 of v).  With ``remove_mean`` each
    component's mean over its non-wall faces is subtracted."""
    out = []
    for comp, shape in ((1, (nz, ny, nx)), (2, (nz, ny, nx)), (3, (nz + 1, ny, nx))):
        rng = np.random.Generator(np.random.PCG64(seed + comp))
        a = rng.standard_normal(shape, dtype=np.float64) * sigma
        if comp == 3:
            a[0] = 0.0
            a[-1] = 0.0
            if remove_mean:
                a[1:-1] -= a[1:-1].mean()
        elif comp == 2 and ywalls:
            a[:, 0, :] = 0.0
            if remove_mean:
                a[:, 1:, :] -= a[:, 1:, :].mean()
        elif remove_mean:
            a -= a.mean()
        out.append(a.astype(dtype, copy=False))
    return tuple(out)


def spheres_phi(nx, ny, nz, lx, ly, zf, spheres, nsub=4, yf=None):
    """Volume fraction of a union of non-overlapping spheres: the fraction of
    the nsub^3 sub-cell centres of each cell inside a sphere (values m/nsub^3).
    x and y are periodic; z is bounded by the walls (and y too when its face
    coordinates ``yf`` are given: a stretched y between walls).  ``spheres``
    is a list of (cx, cy, cz, r).  Cells whose every sub-cell centre is
    provably inside (or outside) are set to 1 (or 0) without sampling."""
    phi = np.zeros((nz, ny, nx))
    dx, dy = lx / nx, ly / ny
    off = (np.arange(nsub) + 0.5) / nsub
    for (cx, cy, cz, r) in spheres:
        k0 = max(int(np.searchsorted(zf, cz - r, side="right")) - 1, 0)
        k1 = min(int(np.searchsorted(zf, cz + r, side="left")), nz)
        i0, i1 = int(math.floor((cx - r) / dx)), int(math.floor((cx + r) / dx)) + 1
        if yf is None:
            j0, j1 = int(math.floor((cy - r) / dy)), int(math.floor((cy + r) / dy)) + 1
        else:
            j0 = max(int(np.searchsorted(yf, cy - r, side="right")) - 1, 0)
            j1 = min(int(np.searchsorted(yf, cy + r, side="left")), ny)
        ii = np.arange(i0, i1)
        jj = np.arange(j0, j1)
        kk = np.arange(k0, k1)
        dzk = zf[kk + 1] - zf[kk]
        # cell-centre distances and the largest sub-cell-centre offset
        xc = (ii + 0.5) * dx - cx
        if yf is None:
            dyj = np.full(len(jj), dy)
            yc = (jj + 0.5) * dy - cy
        else:
            ylo, dyj = yf[jj], yf[jj + 1] - yf[jj]
            yc = ylo + 0.5 * dyj - cy
        zc = 0.5 * (zf[kk] + zf[kk + 1]) - cz
        dist = np.sqrt(zc[:, None, None] ** 2 + yc[None, :, None] ** 2 + xc[None, None, :] ** 2)
        reach = (0.5 - 0.5 / nsub) * np.sqrt(dzk[:, None, None] ** 2 + dyj[None, :, None] ** 2 + dx * dx)
        frac = np.zeros(dist.shape)
        frac[dist + reach <= r] = 1.0
        edge = np.argwhere((dist + reach > r) & (dist - reach <= r))
        if len(edge):
            ke, je, ie = edge[:, 0], edge[:, 1], edge[:, 2]
            sx = (ii[ie][:, None] + off[None, :]) * dx - cx                       # (m, nsub)
            if yf is None:
                sy = (jj[je][:, None] + off[None, :]) * dy - cy
            else:
                sy = ylo[je][:, None] + off[None, :] * dyj[je][:, None] - cy
            sz = zf[kk[ke]][:, None] + off[None, :] * dzk[ke][:, None] - cz
            inside = (sz[:, :, None, None] ** 2 + sy[:, None, :, None] ** 2
                      + sx[:, None, None, :] ** 2) <= r * r
            frac[ke, je, ie] = inside.reshape(len(edge), -1).sum(axis=1) / float(nsub ** 3)
        phi[np.ix_(kk, jj % ny, ii % nx)] += frac
    return np.minimum(phi, 1.0)


def batch_case(count=96, seed=1004, ratio=1000.0, dt=1e-3, sizes=(64, 96, 128, 160, 192)):
    """Independent grids for batched solves: N drawn from ``sizes`` for x and
    y, nz = N a with a ~ U[1, 2] rounded up to a multiple of 8, unit x/y
    period, lz = nz/N (cubic cells), walls in z.  Each grid holds one liquid
    droplet (radius U[0.1, 0.25] of the period) in gas at ratio ``ratio``:1
    and a random-divergence predicted velocity (N(0, 1) faces, mean-removed);
    S = 0."""
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    out = []
    for gi in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        a = rng.uniform(1.0, 2.0)
        nz = int(math.ceil(n * a / 8.0) * 8)
        lz = nz / n
        zf = uniform_zfaces(nz, lz)
        r = rng.uniform(0.1, 0.25)
        h = 1.0 / n
        c = (rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(r + 2 * h, lz - r - 2 * h))
        drop = spheres_phi(n, n, nz, 1.0, 1.0, zf, [(c[0], c[1], c[2], r)])
        us, vs, ws = random_faces(n, n, nz, 1.0, seed + 100 * (gi + 1), remove_mean=True)
        out.append(Workload(f"batch grid {gi}: {n}x{n}x{nz}, droplet r={r:.3f}", n, n, nz, 1.0, 1.0, zf,
                            dt, us, vs, ws, 1.0 - drop, 1.0, ratio, np.zeros((nz, n, n))))
    return out


def gas_source(phi):
    """Divergence target in the gas (Eq. 34, uniform temperature)."""
    return -phi * (DP0_DT / (GAMMA_G * P0))


def random_divergence_case(n=32, seed=1001, dt=1e-3):
    """Constant density, RHS = divergence of mean-removed N(0,1) faces / dt
    (unit cube, periodic x/y, walls in z)."""
    us, vs, ws = random_faces(n, n, n, 1.0, seed, remove_mean=True)
    return Workload(f"random-divergence {n}^3, rho=1", n, n, n, 1.0, 1.0,
                    uniform_zfaces(n, 1.0), dt, us, vs, ws,
                    np.zeros((n, n, n)), 1.0, 1.0, np.zeros((n, n, n)))


def single_sphere_case(n=256, seed=1002, dt=1e-3, radius=0.15, centre=(0.5, 0.5, 0.3),
                       rho_g=1.2, rho_l=1000.0):
    """One gas sphere in liquid, unit cube, N(0, 0.1) predicted velocity."""
    zf = uniform_zfaces(n, 1.0)
    us, vs, ws = random_faces(n, n, n, 0.1, seed)
    phi = spheres_phi(n, n, n, 1.0, 1.0, zf, [(centre[0], centre[1], centre[2], radius)])
    return Workload(f"gas sphere {n}^3, rho {rho_l:g}:{rho_g:g}", n, n, n, 1.0, 1.0, zf, dt,
                    us, vs, ws, phi, rho_g, rho_l, gas_source(phi))


def place_bubbles(count, lx, ly, lz, nx, nz_min_cell, rmin, rmax, rng, gap_cells=2.0,
                  max_tries=200000, ywalls=False):
    """Non-overlapping bubbles, centres uniform with rejection: at least
    ``gap_cells`` cells apart (periodic in x/y) and r + gap from the walls
    (the z walls, and the y walls with ``ywalls``)."""
    h = lx / nx
    out = []
    tries = 0
    while len(out) < count and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = (rng.uniform(0, lx), rng.uniform(0, ly), rng.uniform(0, lz))
        if c[2] - r < gap_cells * nz_min_cell or c[2] + r > lz - gap_cells * nz_min_cell:
            continue
        if ywalls and (c[1] - r < gap_cells * h or c[1] + r > ly - gap_cells * h):
            continue
        ok = True
        for (ox, oy, oz, orr) in out:
            ddx = abs(c[0] - ox); ddx = min(ddx, lx - ddx)
            ddy = abs(c[1] - oy)
            if not ywalls:
                ddy = min(ddy, ly - ddy)
            if math.sqrt(ddx * ddx + ddy * ddy + (c[2] - oz) ** 2) < r + orr + gap_cells * h:
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
    if len(out) < count:
        raise RuntimeError("could not place the requested bubbles")
    return out


def bubbles_case(n=512, nbubbles=200, seed=1003, dt=1e-3, beta=1.5, rmin=0.05, rmax=0.12,
                 rho_g=1.0, rho_l=1000.0, lz=2 * math.pi, nz=None):
    """Bubbly field in a (2 pi)^3 box with tanh-stretched z (n^2 x nz cells,
    nz = n by default)."""
    L = 2 * math.pi
    nz = nz or n
    zf = tanh_zfaces(nz, lz, beta)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    spheres = place_bubbles(nbubbles, L, L, lz, n, float(np.min(np.diff(zf))), rmin, rmax, rng)
    phi = spheres_phi(n, n, nz, L, L, zf, spheres)
    us, vs, ws = random_faces(n, n, nz, 0.1, seed)
    size = f"{n}^3" if nz == n else f"{n}x{n}x{nz}"
    return Workload(f"{nbubbles} bubbles {size} tanh(beta={beta:g}) z, rho {rho_l:g}:{rho_g:g}",
                    n, n, nz, L, L, zf, dt, us, vs, ws, phi, rho_g, rho_l, gas_source(phi),
                    extra={"spheres": spheres})


def droplets_case(nx=256, ny=256, nz=128, seed=1005, dt=1e-3, beta=2.0, ndrops=4,
                  rho_g=1.0, rho_l=100.0, lz=0.5):
    """Four droplets (liquid, rho_l) in gas; stretched z; adds a target
    velocity N(0, 0.1) for the loss ||u^{n+1} - u_target||^2."""
    zf = tanh_zfaces(nz, lz, beta)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    spheres = place_bubbles(ndrops, 1.0, 1.0, lz, nx, float(np.min(np.diff(zf))), 0.06, 0.12, rng)
    drop = spheres_phi(nx, ny, nz, 1.0, 1.0, zf, spheres)
    phi = 1.0 - drop                      # Phi is the gas fraction
    us, vs, ws = random_faces(nx, ny, nz, 0.1, seed)
    ut = random_faces(nx, ny, nz, 0.1, seed + 20 - 1)
    return Workload(f"{ndrops} droplets {nx}x{ny}x{nz} tanh(beta={beta:g}) z, rho {rho_l:g}:{rho_g:g}",
                    nx, ny, nz, 1.0, 1.0, zf, dt, us, vs, ws, phi, rho_g, rho_l,
                    np.zeros((nz, ny, nx)), extra={"target": ut, "spheres": spheres})


def small_bubble_case(n=32, seed=1102, rho_ratio=1000.0, stretched=False, nz=None, ny=None,
                      nbubbles=3, dt=1e-3):
    """Small multi-bubble case for parity tests (several tiles, ragged sizes
    allowed through nx != ny != nz)."""
    nx = n
    ny = ny or n
    nz = nz or n
    zf = tanh_zfaces(nz, 1.0, 1.5) if stretched else uniform_zfaces(nz, 1.0)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    spheres = place_bubbles(nbubbles, 1.0, ny / nx, 1.0, nx, float(np.min(np.diff(zf))),
                            0.08, 0.16, rng, gap_cells=1.0)
    phi = spheres_phi(nx, ny, nz, 1.0, ny / nx, zf, spheres)
    us, vs, ws = random_faces(nx, ny, nz, 0.1, seed)
    return Workload(f"{nbubbles} bubbles {nx}x{ny}x{nz}", nx, ny, nz, 1.0, ny / nx, zf, dt,
                    us, vs, ws, phi, 1.0, rho_ratio, gas_source(phi))


def channel_bubble_case(nx=32, ny=None, nz=None, seed=1202, rho_ratio=1000.0, stretched=False,
                        nbubbles=3, dt=1e-3, ybeta=None):
    """Bubbles in a duct: periodic in x, walls in y and z.  The bubbles keep
    a cell's gap from every wall; v* is zero on the y walls (row 0) as w* is
    on the z walls.  ``ybeta``: y faces clustered at the walls by
    ``tanh_yfaces`` with that beta (a stretched y)."""
    ny = ny or nx
    nz = nz or nx
    ly = ny / nx
    zf = tanh_zfaces(nz, 1.0, 1.5) if stretched else uniform_zfaces(nz, 1.0)
    yf = None if ybeta is None else tanh_yfaces(ny, ly, ybeta)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    spheres = place_bubbles(nbubbles, 1.0, ly, 1.0, nx, float(np.min(np.diff(zf))),
                            0.08, 0.16, rng, gap_cells=1.0, ywalls=True)
    phi = spheres_phi(nx, ny, nz, 1.0, ly, zf, spheres, yf=yf)
    us, vs, ws = random_faces(nx, ny, nz, 0.1, seed, ywalls=True)
    name = f"{nbubbles} bubbles in a duct {nx}x{ny}x{nz}" + ("" if yf is None else f", tanh({ybeta:g}) y")
    return Workload(name, nx, ny, nz, 1.0, ly, zf, dt,
                    us, vs, ws, phi, 1.0, rho_ratio, gas_source(phi), ywalls=True, yf=yf)
