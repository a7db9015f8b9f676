"""The allocation-free constant-coefficient solve (pressure_solve_noalloc)
against the plan-based pressure_solve and the CPU oracle, through the C ABI.

Callers that cannot call cudaMalloc (device memory owned by an external pool
or budget, loops that must not enter an allocator) use this entry point; its
working memory is a fixed device array inside the library that every call
reuses.  This file is collected last so that a run stopping at the first
failure has run every other test first; it also passes when run alone in a
fresh process.
"""
import numpy as np
import pytest

import oracle.pressure_oracle as orc
from paper_2005_11806_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11  # the FP64 tolerance of the parity tests


@pytest.fixture(scope="module")
def pp():
    from paper_2005_11806_gb300 import pressure
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    pressure.lib()
    return pressure


def _plan_solve(pp, dims, lengths, zf, f, ywalls=False):
    plan = pp.Plan(*dims, *lengths, zfaces=zf, precision="fp64", ywalls=ywalls)
    p = torch.empty_like(f)
    pp.pressure_solve(plan.handle, f, p)
    torch.cuda.synchronize()
    plan.close()
    return p


def test_noalloc_matches_plan_solve_twice(pp):
    """Two calls in a row (different grids, so the second overwrites every
    table the first left in the shared array); each matches pressure_solve."""
    cases = [((32, 32, 32), (1.0, 1.0, 1.0), None, 1),
             ((24, 20, 17), (1.0, 0.75, 1.2), 1.5, 2)]
    for dims, lengths, stretch, seed in cases:
        nx, ny, nz = dims
        zf = wl.uniform_zfaces(nz, lengths[2]) if stretch is None else wl.tanh_zfaces(nz, lengths[2], stretch)
        f = torch.from_numpy(np.random.default_rng(seed).standard_normal((nz, ny, nx))).cuda()
        p = torch.full_like(f, float("nan"))
        pp.pressure_solve_noalloc(nx, ny, nz, *lengths, f, p, zfaces=zf)
        torch.cuda.synchronize()
        ref = _plan_solve(pp, dims, lengths, zf, f)
        err = float(torch.linalg.vector_norm(p - ref) / torch.linalg.vector_norm(ref))
        assert err < FP64_TOL, (dims, err)
        g = orc.Grid(nx, ny, nz, lengths[0], lengths[1], zf)
        po = orc.solve_constant(g, f.cpu().numpy())
        err_o = float(np.linalg.norm(p.cpu().numpy() - po) / np.linalg.norm(po))
        assert err_o < FP64_TOL, (dims, err_o)


def test_noalloc_walls_in_y(pp):
    """Walls in y (the cosine y basis): the same solve as an FP64 plan with
    walls in y and as the oracle, including a grid with radix-3 and radix-5
    y lengths; a periodic call after it still matches (the tables are
    rebuilt every call)."""
    cases = [((32, 24, 16), (1.0, 0.8, 1.0), 1.5, 5, True),
             ((20, 30, 9), (1.0, 1.3, 0.7), None, 6, True),
             ((16, 12, 10), (1.0, 0.9, 1.1), None, 7, False)]
    for dims, lengths, stretch, seed, ywalls in cases:
        nx, ny, nz = dims
        zf = wl.uniform_zfaces(nz, lengths[2]) if stretch is None else wl.tanh_zfaces(nz, lengths[2], stretch)
        f = torch.from_numpy(np.random.default_rng(seed).standard_normal((nz, ny, nx))).cuda()
        p = torch.full_like(f, float("nan"))
        pp.pressure_solve_noalloc(nx, ny, nz, *lengths, f, p, zfaces=zf, ywalls=ywalls)
        torch.cuda.synchronize()
        ref = _plan_solve(pp, dims, lengths, zf, f, ywalls)
        err = float(torch.linalg.vector_norm(p - ref) / torch.linalg.vector_norm(ref))
        assert err < FP64_TOL, (dims, err)
        g = orc.Grid(nx, ny, nz, lengths[0], lengths[1], zf, ywalls=ywalls)
        po = orc.solve_constant(g, f.cpu().numpy())
        err_o = float(np.linalg.norm(p.cpu().numpy() - po) / np.linalg.norm(po))
        assert err_o < FP64_TOL, (dims, err_o)


def test_noalloc_rejects_grids_beyond_the_scratch(pp):
    f = torch.zeros((64, 256, 256), dtype=torch.float64, device="cuda")
    p = torch.empty_like(f)
    with pytest.raises(pp.PressureError) as ei:
        pp.pressure_solve_noalloc(256, 256, 64, 1.0, 1.0, 1.0, f, p)
    assert ei.value.code == pp.PP_ERR_TOO_LARGE


def test_noalloc_input_checks_return_before_any_launch(pp):
    """Argument errors come back as status codes from the host-side checks,
    with nothing enqueued: the output keeps its NaN fill."""
    f = torch.zeros(4096 * 2, dtype=torch.float64, device="cuda")
    p = torch.full_like(f, float("nan"))
    bad = [
        (dict(nx=7, ny=4, nz=3), pp.PP_ERR_UNSUPPORTED),        # odd nx (two real rows per transform)
        (dict(nx=4096, ny=2, nz=1), pp.PP_ERR_UNSUPPORTED),     # one x line per block: nx <= 2048
        (dict(nx=2, ny=4096, nz=1), pp.PP_ERR_UNSUPPORTED),     # one y line per block: ny <= 2048
        (dict(nx=14, ny=4, nz=3), pp.PP_ERR_UNSUPPORTED),       # prime factor 7
    ]
    for dims, code in bad:
        with pytest.raises(pp.PressureError) as ei:
            pp.pressure_solve_noalloc(dims["nx"], dims["ny"], dims["nz"], 1.0, 1.0, 1.0, f, p)
        assert ei.value.code == code, dims
    zf = np.array([0.0, 0.5, 0.4, 1.0])                          # not increasing
    with pytest.raises(pp.PressureError) as ei:
        pp.pressure_solve_noalloc(4, 4, 3, 1.0, 1.0, 1.0, f, p, zfaces=zf)
    assert ei.value.code == pp.PP_ERR_INVALID_ARG
    fh = np.zeros(4 * 4 * 3)                                     # a host array as f
    with pytest.raises(pp.PressureError) as ei:
        pp.pressure_solve_noalloc(4, 4, 3, 1.0, 1.0, 1.0, fh, p)
    assert ei.value.code == pp.PP_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool(torch.isnan(p).all())
