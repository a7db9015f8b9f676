"""Writes tests/golden/oracle_regression.txt from the oracle alone.

The paper prints no worked numbers for the pressure step, so no fixture here
holds a value from it.  This file records the oracle's own results on fixed,
seeded small cases, so that a later change to the oracle's arithmetic shows
up as a failing test (and must name the passage or reading that justifies
it).  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.pressure_oracle as orc  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.txt")
SAMPLES = [(0, 0, 0), (1, 2, 3), (4, 3, 2), (3, 5, 7), (2, 1, 6)]  # (k, j, i)


def _tanh_faces(n, lz, beta):
    xi = np.arange(n + 1) / n
    return 0.5 * lz * (1.0 + np.tanh(beta * (2.0 * xi - 1.0)) / np.tanh(beta))


def cases():
    """Yields (name, grid, f) for the constant solve and (name, grid, fields)
    for the projection.  Inputs are built here from numpy's PCG64 only."""
    g = orc.Grid(8, 6, 5, 1.0, 0.8, _tanh_faces(5, 1.3, 1.5))
    f = np.random.Generator(np.random.PCG64(7001)).standard_normal(g.shape)
    yield "solve_stretched_8x6x5", g, f
    gy = orc.Grid(8, 6, 5, 1.0, 0.8, _tanh_faces(5, 1.3, 1.5), ywalls=True)
    yield "solve_ywalls_8x6x5", gy, f


def projection_case():
    g = orc.Grid(8, 6, 8, 1.0, 0.75, _tanh_faces(8, 1.0, 1.5))
    rng = np.random.Generator(np.random.PCG64(7002))
    phi = np.zeros(g.shape)
    phi[2:5, 1:4, 2:6] = 1.0
    phi[5, 1:3, 2:5] = 0.5
    rho = orc.mixture_density(phi, 1.0, 1000.0)
    us = 0.1 * rng.standard_normal(g.shape)
    vs = 0.1 * rng.standard_normal(g.shape)
    ws = 0.1 * rng.standard_normal((g.nz + 1, g.ny, g.nx))
    ws[0] = ws[-1] = 0.0
    S = -phi * 1e-2 / 1.4
    return g, us, vs, ws, rho, S


def compute():
    rows = []
    for name, g, f in cases():
        p = orc.solve_constant(g, f)
        for (k, j, i) in SAMPLES:
            if k < g.nz and j < g.ny and i < g.nx:
                rows.append((name, f"p[{k},{j},{i}]", p[k, j, i]))
    g, us, vs, ws, rho, S = projection_case()
    p, u, v, w, info = orc.method3(g, us, vs, ws, rho, S, 1e-3, rtol=1e-12, maxit=5000)
    rows.append(("method3_8x6x8_ratio1000", "iters", float(info["iters"])))
    for (k, j, i) in SAMPLES:
        rows.append(("method3_8x6x8_ratio1000", f"p[{k},{j},{i}]", p[k, j, i]))
        rows.append(("method3_8x6x8_ratio1000", f"u[{k},{j},{i}]", u[k, j, i]))
        rows.append(("method3_8x6x8_ratio1000", f"w[{k},{j},{i}]", w[k, j, i]))
    return rows


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        fh.write("# case  quantity  value  (written by tests/golden/make_golden.py from oracle/ only)\n")
        for name, q, val in compute():
            fh.write(f"{name} {q} {float(val):.17g}\n")
    print("wrote", OUT)
