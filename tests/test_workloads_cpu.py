"""The seeded input generators (no GPU): determinism, the wall conditions of
the face velocities, and the bubbles' clearance from the walls."""
import numpy as np

from paper_2005_11806_gb300 import workloads as wl


def test_generators_are_deterministic():
    a = wl.channel_bubble_case(16, 12, 10, seed=1202, stretched=True)
    b = wl.channel_bubble_case(16, 12, 10, seed=1202, stretched=True)
    for x, y in ((a.us, b.us), (a.vs, b.vs), (a.ws, b.ws), (a.phi, b.phi), (a.S, b.S)):
        assert np.array_equal(x, y)
    c = wl.small_bubble_case(16, seed=1102)
    d = wl.small_bubble_case(16, seed=1102)
    assert np.array_equal(c.phi, d.phi) and np.array_equal(c.us, d.us)


def test_wall_faces_are_zero():
    w = wl.small_bubble_case(16, ny=12, nz=10)
    assert np.all(w.ws[0] == 0) and np.all(w.ws[-1] == 0) and not w.ywalls
    d = wl.channel_bubble_case(16, 12, 10)
    assert d.ywalls
    assert np.all(d.vs[:, 0, :] == 0) and np.all(d.ws[0] == 0) and np.all(d.ws[-1] == 0)
    assert np.count_nonzero(d.vs[:, 1:, :]) == d.vs[:, 1:, :].size


def test_duct_bubbles_clear_the_walls():
    """Every bubble keeps a cell's gap from the y and z walls, so the wall
    rows and planes are pure liquid; the gas volume is positive."""
    for seed in (1202, 1203, 1204):
        d = wl.channel_bubble_case(32, 24, 20, seed=seed, stretched=True)
        assert d.phi.sum() > 0
        assert np.all(d.phi[:, 0, :] == 0) and np.all(d.phi[:, -1, :] == 0)
        assert np.all(d.phi[0] == 0) and np.all(d.phi[-1] == 0)
        assert np.all((d.phi >= 0) & (d.phi <= 1))
        # the source lives in the gas only (Eq. 34 with uniform T)
        assert np.all(d.S[d.phi == 0] == 0) and np.all(d.S[d.phi > 0] < 0)


def test_random_faces_mean_removal_skips_walls():
    u, v, w = wl.random_faces(8, 6, 5, 1.0, 77, remove_mean=True, ywalls=True)
    assert abs(u.mean()) < 1e-14
    assert np.all(v[:, 0, :] == 0) and abs(v[:, 1:, :].mean()) < 1e-14
    assert np.all(w[0] == 0) and np.all(w[-1] == 0) and abs(w[1:-1].mean()) < 1e-14
