"""The allocation-free constant-coefficient solve (pressure_solve_noalloc)
against the plan-based pressure_solve, through the C ABI.

Callers that cannot call cudaMalloc use this entry point; its working memory
is a fixed device array inside the library that every call reuses.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

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


def _plan_solve(pp, dims, lengths, zf, f):
    plan = pp.Plan(*dims, *lengths, zfaces=zf, precision="fp64")
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


def test_noalloc_rejects_grids_beyond_the_scratch(pp):
    f = torch.zeros((64, 256, 256), dtype=torch.float64, device="cuda")
    p = torch.empty_like(f)
    with pytest.raises(pp.PressureError) as ei:
        pp.pressure_solve_noalloc(256, 256, 64, 1.0, 1.0, 1.0, f, p)
    assert ei.value.code == pp.PP_ERR_TOO_LARGE
