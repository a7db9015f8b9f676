"""Host-side argument checks of the Python binding (no GPU): fields shorter
than the plan's cell or z-face count are refused before any library call,
so no kernel ever sees a short buffer."""
import numpy as np
import pytest

from paper_2005_11806_gb300 import pressure


class _FakeLib:
    """Stands in for the CUDA library: records the calls, returns PP_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return pressure.PP_OK
        return call


@pytest.fixture
def fake(monkeypatch):
    f = _FakeLib()
    monkeypatch.setattr(pressure, "_lib", f)
    handle = 0x5EED
    nx, ny, nz = 6, 5, 4
    monkeypatch.setitem(pressure._PLAN_SIZES, handle, (nx * ny * nz, nx * ny * (nz + 1)))
    return f, handle, (nz, ny, nx), (nz + 1, ny, nx)


def test_full_size_fields_reach_the_library(fake):
    f, h, cs, ws = fake
    c = lambda: np.zeros(cs)  # noqa: E731
    w = lambda: np.zeros(ws)  # noqa: E731
    pressure.pressure_solve(h, c(), c())
    pressure.pressure_mixture_density(h, c(), 1.0, 1000.0, c())
    pressure.pressure_correct(h, c(), c(), w(), c(), None, 1e-3, c(), c(), c(), w())
    pressure.pressure_solve_adjoint(h, c(), c(), 1e-3, c(), c(), w(), c(), c(), w(), c())
    pressure.pressure_divergence_source(h, c(), c(), c(), 1.0, 1.4, 0.0, c())
    pressure.pressure_p0_rate(h, c(), c(), c(), c(), c(), w(), 1.0, 1.4)
    assert f.calls == ["pressure_solve", "pressure_mixture_density", "pressure_correct",
                       "pressure_solve_adjoint", "pressure_divergence_source", "pressure_p0_rate"]


@pytest.mark.parametrize("which", ["cell", "zface"])
def test_short_fields_are_refused(fake, which):
    f, h, cs, ws = fake
    c, w = np.zeros(cs), np.zeros(ws)
    short_c = np.zeros(cs)[:, :-1].copy()
    with pytest.raises(ValueError, match="cell"):
        pressure.pressure_solve(h, c, short_c)
    if which == "cell":
        with pytest.raises(ValueError, match="cell"):
            pressure.pressure_correct(h, c, short_c, w, c, None, 1e-3, c, c, c, w)
    else:
        # a cell-shaped array where a z-face field belongs is one plane short
        with pytest.raises(ValueError, match="z-face"):
            pressure.pressure_correct(h, c, c, c, c, None, 1e-3, c, c, c, w)
        with pytest.raises(ValueError, match="z-face"):
            pressure.pressure_solve_adjoint(h, c, c, 1e-3, c, c, w, c, c, c, c)
    assert f.calls == []


def test_unknown_handles_are_not_checked(fake):
    """Handles from elsewhere (not made by this module) pass through."""
    f, h, cs, ws = fake
    pressure.pressure_solve(h + 1, np.zeros(3), np.zeros(3))
    assert f.calls == ["pressure_solve"]


def test_destroy_forgets_the_plan(fake):
    f, h, cs, ws = fake
    pressure.pressure_plan_destroy(h)
    assert h not in pressure._PLAN_SIZES
    assert f.calls == ["pressure_plan_destroy"]


def test_batch_buffers_are_checked(monkeypatch):
    """The packed buffers of a batch are checked against its total cell and
    z-face counts."""
    f = _FakeLib()
    monkeypatch.setattr(pressure, "_lib", f)
    b = pressure.Batch.__new__(pressure.Batch)
    b.handle, b.n, b.ncell, b.nwface = 0xBA7C, 2, 100, 120
    monkeypatch.setitem(pressure._PLAN_SIZES, b.handle, (b.ncell, b.nwface))
    c, w = np.zeros(100), np.zeros(120)
    b.correct(c, c, w, c, c, 1e-3, c, c, c, w)
    with pytest.raises(ValueError, match="z-face"):
        b.correct(c, c, c, c, c, 1e-3, c, c, c, w)
    with pytest.raises(ValueError, match="cell"):
        b.mixture_density(np.zeros(99), 1.0, 1000.0, c)
    assert f.calls == ["pressure_batch_correct"]
    b.close()
    assert b.handle is None and 0xBA7C not in pressure._PLAN_SIZES


def test_noalloc_fields_are_checked(monkeypatch):
    f = _FakeLib()
    monkeypatch.setattr(pressure, "_lib", f)
    pressure.pressure_solve_noalloc(4, 4, 4, 1.0, 1.0, 1.0, np.zeros(64), np.zeros(64))
    with pytest.raises(ValueError, match="cell"):
        pressure.pressure_solve_noalloc(4, 4, 4, 1.0, 1.0, 1.0, np.zeros(64), np.zeros(63))
    assert f.calls == ["pressure_solve_noalloc"]
