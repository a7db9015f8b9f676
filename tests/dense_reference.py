"""Entry-by-entry assembly of the discrete operators with plain Python loops,
written directly from the stencil definitions (Sec. 3 MAC grid), for dense
LU pins on tiny grids.  Independent of the oracle's array code."""
import numpy as np


def metrics(nz, zf):
    dzf = [zf[k + 1] - zf[k] for k in range(nz)]
    zc = [0.5 * (zf[k + 1] + zf[k]) for k in range(nz)]
    return dzf, zc


def y_metrics(ny, ly, yf):
    """Row widths and centres of y: uniform (yf None) or from the ny + 1 face
    coordinates yf."""
    if yf is None:
        dy = ly / ny
        return [dy] * ny, [(j + 0.5) * dy for j in range(ny)]
    dyf = [yf[j + 1] - yf[j] for j in range(ny)]
    yc = [0.5 * (yf[j + 1] + yf[j]) for j in range(ny)]
    return dyf, yc


def assemble_variable(nx, ny, nz, lx, ly, zf, rho, ywalls=False, yf=None):
    """Matrix of p -> D(beta G p) with beta = 2/(rho_a + rho_b) on each face,
    zero flux through the z walls, periodic x, and y periodic or (ywalls)
    bounded by walls with zero flux.  rho=None means beta=1.  yf (walls in
    y only): y face coordinates of a stretched y."""
    dx, dy = lx / nx, ly / ny
    dzf, zc = metrics(nz, zf)
    dyf, yc = y_metrics(ny, ly, yf)
    n = nx * ny * nz

    def idx(i, j, k):
        return (k * ny + (j % ny)) * nx + (i % nx)

    def beta(c1, c2):
        if rho is None:
            return 1.0
        return 2.0 / (rho[c1] + rho[c2])

    A = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                cell = (k, j, i)
                # x faces: right face between (i, i+1), left face between (i-1, i)
                for di in (+1, -1):
                    nb = (k, j, (i + di) % nx)
                    b = beta(cell, nb) / (dx * dx)
                    A[r, idx(i + di, j, k)] += b
                    A[r, r] -= b
                for dj in (+1, -1):
                    if ywalls and not 0 <= j + dj < ny:
                        continue  # y wall: no flux
                    nb = (k, (j + dj) % ny, i)
                    if yf is None:
                        b = beta(cell, nb) / (dy * dy)
                    else:
                        b = beta(cell, nb) / (abs(yc[j + dj] - yc[j]) * dyf[j])
                    A[r, idx(i, j + dj, k)] += b
                    A[r, r] -= b
                for dk in (+1, -1):
                    kk = k + dk
                    if kk < 0 or kk >= nz:
                        continue  # wall: no flux
                    nb = (kk, j, i)
                    dist = abs(zc[kk] - zc[k])
                    b = beta(cell, nb) / (dist * dzf[k])
                    A[r, idx(i, j, kk)] += b
                    A[r, r] -= b
    return A


def bordered_solve(A, rhs, weights):
    """Solve A x + mu 1 = rhs with weights . x = 0 (dense LU)."""
    n = A.shape[0]
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = A
    K[:n, n] = 1.0
    K[n, :n] = weights
    sol = np.linalg.solve(K, np.concatenate([rhs, [0.0]]))
    return sol[:n]


def cell_weights(nx, ny, nz, zf, yf=None):
    """Cell volumes over dx dy (uniform y) or over dx (stretched y, yf)."""
    dzf, _ = metrics(nz, zf)
    if yf is None:
        return np.repeat(np.array(dzf), nx * ny)
    dyf, _ = y_metrics(ny, None, yf)
    return np.array([dzf[k] * dyf[j] for k in range(nz) for j in range(ny) for _ in range(nx)])


def divergence_loops(nx, ny, nz, lx, ly, zf, u, v, w, ywalls=False, yf=None):
    """With ywalls, v[k, j, i] is the face below cell j and both wall faces
    (below cell 0, above cell ny - 1) carry no flux.  yf: stretched y."""
    dx = lx / nx
    dzf, _ = metrics(nz, zf)
    dyf, _ = y_metrics(ny, ly, yf)
    out = np.zeros((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                vlo = 0.0 if (ywalls and j == 0) else v[k, j, i]
                vhi = 0.0 if (ywalls and j == ny - 1) else v[k, (j + 1) % ny, i]
                out[k, j, i] = ((u[k, j, (i + 1) % nx] - u[k, j, i]) / dx
                                + (vhi - vlo) / dyf[j]
                                + (w[k + 1, j, i] - w[k, j, i]) / dzf[k])
    return out


def assemble_conduction(nx, ny, nz, lx, ly, zf, kc, ywalls=False):
    """Matrix of T -> D(k_f G T) with k_f the arithmetic mean of the two
    cells of a face (kc indexed [k][j][i]); no flux through the z walls,
    periodic x, and y periodic or (ywalls) bounded by walls with no flux."""
    dx, dy = lx / nx, ly / ny
    dzf, zc = metrics(nz, zf)
    n = nx * ny * nz

    def idx(i, j, k):
        return (k * ny + (j % ny)) * nx + (i % nx)

    A = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                for di in (+1, -1):
                    kf = 0.5 * (kc[k][j][i] + kc[k][j][(i + di) % nx])
                    A[r, idx(i + di, j, k)] += kf / (dx * dx)
                    A[r, r] -= kf / (dx * dx)
                for dj in (+1, -1):
                    if ywalls and not 0 <= j + dj < ny:
                        continue  # adiabatic y wall
                    kf = 0.5 * (kc[k][j][i] + kc[k][(j + dj) % ny][i])
                    A[r, idx(i, j + dj, k)] += kf / (dy * dy)
                    A[r, r] -= kf / (dy * dy)
                for dk in (+1, -1):
                    kk = k + dk
                    if kk < 0 or kk >= nz:
                        continue  # adiabatic wall
                    kf = 0.5 * (kc[k][j][i] + kc[kk][j][i])
                    b = kf / (abs(zc[kk] - zc[k]) * dzf[k])
                    A[r, idx(i, j, kk)] += b
                    A[r, r] -= b
    return A


def gradient_loops(nx, ny, nz, lx, ly, zf, p, ywalls=False, yf=None):
    """G p on the faces, cell by cell: x faces (i - 1/2), y faces (j - 1/2),
    z faces k = 0 .. nz (the wall faces 0 and nz carry no gradient); with
    ywalls the wall row j = 0 of the y faces carries none either.  yf:
    stretched y (walls only)."""
    dx, dy = lx / nx, ly / ny
    _, zc = metrics(nz, zf)
    _, yc = y_metrics(ny, ly, yf)
    gx = np.zeros((nz, ny, nx))
    gy = np.zeros((nz, ny, nx))
    gz = np.zeros((nz + 1, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                gx[k, j, i] = (p[k, j, i] - p[k, j, (i - 1) % nx]) / dx
                if not (ywalls and j == 0):
                    dist = dy if yf is None else yc[j] - yc[j - 1]
                    gy[k, j, i] = (p[k, j, i] - p[k, (j - 1) % ny, i]) / dist
                if k > 0:
                    gz[k, j, i] = (p[k, j, i] - p[k - 1, j, i]) / (zc[k] - zc[k - 1])
    return gx, gy, gz


def face_beta_loops(nx, ny, nz, rho):
    """1 / rho_f on the faces with rho_f the arithmetic mean of the two cells
    of a face (x, y faces periodic; z faces 1 .. nz - 1; the wall planes of z
    hold 0, where the gradient vanishes anyway)."""
    bx = np.zeros((nz, ny, nx))
    by = np.zeros((nz, ny, nx))
    bz = np.zeros((nz + 1, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                bx[k, j, i] = 2.0 / (rho[k, j, i] + rho[k, j, (i - 1) % nx])
                by[k, j, i] = 2.0 / (rho[k, j, i] + rho[k, (j - 1) % ny, i])
                if k > 0:
                    bz[k, j, i] = 2.0 / (rho[k, j, i] + rho[k - 1, j, i])
    return bx, by, bz


def pseudo_inverse_laplacian(nx, ny, nz, lx, ly, zf):
    """Dense matrix of f -> the zero-mean p with L p = f - <f>_V (L = D G, the
    constant-coefficient operator), one bordered LU solve per unit vector."""
    L = assemble_variable(nx, ny, nz, lx, ly, zf, None)
    wts = cell_weights(nx, ny, nz, zf)
    n = L.shape[0]
    out = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        out[:, c] = bordered_solve(L, e - (wts @ e) / wts.sum(), wts)
    return out
