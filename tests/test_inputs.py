"""The seeded input recipes (paper_1602_02675_gb300/inputs.py) hold the shapes
and distributions the workloads state: the shock tube of Section V.C, the
batch of tubes (lengths uniform in 256..16384, pressure ratio log-uniform in
[2, 100], density ratio uniform in [1, 10]), and the random fields of the
parity tests.  They are deterministic for a seed."""
import math

import numpy as np

from paper_1602_02675_gb300 import inputs as I


def test_sod_workloads():
    assert I.SOD_1D.nx == 1000 and I.SOD_1D.t_end == 0.2
    assert I.SOD_2D.nx == 4096 and I.SOD_2D.ny == 512
    assert I.SOD_LEFT == (1.0, 0.0, 1.0) and I.SOD_RIGHT == (0.125, 0.0, 0.1)
    c = I.CYLINDER_2D
    assert (c.nx, c.ny, c.steps, c.radius, c.bc_x, c.bc_y) == \
        (8192, 8192, 2000, 0.4, 2, 2)


def test_tubes_batch_recipe():
    tubes = I.tubes_batch()
    assert len(tubes) == 4096
    ns = np.array([t.n for t in tubes])
    assert ns.min() >= 256 and ns.max() <= 16384
    assert abs(ns.mean() - (256 + 16384) / 2) < 300
    pr = np.array([t.left[2] / t.right[2] for t in tubes])
    dr = np.array([t.left[0] / t.right[0] for t in tubes])
    assert pr.min() >= 2.0 - 1e-12 and pr.max() <= 100.0 + 1e-9
    # log-uniform: log pr uniform on [log 2, log 100]
    lp = np.log(pr)
    assert abs(lp.mean() - (math.log(2) + math.log(100)) / 2) < 0.05
    assert dr.min() >= 1.0 and dr.max() <= 10.0
    assert abs(dr.mean() - 5.5) < 0.15
    assert all(t.left == (1.0, 0.0, 1.0) for t in tubes)
    assert all(t.right[1] == 0.0 for t in tubes)
    again = I.tubes_batch()
    assert [(t.n, t.right) for t in again] == [(t.n, t.right) for t in tubes]


def test_hot_tubes_take_a_smaller_lattice_speed():
    """lambda0 = (max p/rho)^(-1/2) for a side hotter than Sod's left state,
    then whole steps to t = 0.2."""
    for t in I.tubes_batch(count=256, seed=5):
        steps, lam = t.steps_and_lambda()
        hot = max(t.left[2] / t.left[0], t.right[2] / t.right[0], 1.0)
        assert lam * lam * hot <= 1.0 + 1e-12
        assert math.isclose(steps * lam / t.n, 0.2, rel_tol=1e-12)


def test_random_fields_are_seeded_and_physical():
    for dim, nx, ny in ((1, 300, 1), (2, 40, 30)):
        a = I.random_smooth_prims(dim, nx, ny, seed=4)
        b = I.random_smooth_prims(dim, nx, ny, seed=4)
        for x, y in zip(a, b):
            if x is None:
                continue
            assert np.array_equal(x, y)
        rho, p = a[0], a[3]
        assert np.all(rho > 0) and np.all(p > 0)
        assert rho.size == nx * ny
    prims = I.random_node_prims(2, 500, seed=8)
    assert np.all(prims[0] >= 0) and np.all(prims[3] >= 0)
