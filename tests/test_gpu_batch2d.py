"""Batched small 2-D grids (lbm_batch2d_*): every grid of a batch of
different sizes, boundaries, time steps, initial states and step counts
equals, bit for bit, the same grid stepped alone on a handle (whose FP32
square-lattice results the parity tests check against the oracle)."""
import numpy as np
import pytest

from paper_1602_02675_gb300 import lbm as L

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "mx", "my", "rhoE")
SOD = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1))
HOT = ((1.0, 0.0, 0.0, 10.0), (0.25, 0.0, 0.0, 0.5))


def _grids(kahan):
    """(config, inner, outer, geom, a0, a1, radius, nsteps) per grid."""
    T, R, P = L.TRANSMISSIVE, L.REFLECTING, L.PERIODIC
    spec = [
        (96, 64, T, R, 1.0, SOD, L.PLANAR_X, 0.5, 0.5, 0.0, 40, 1),
        (128, 128, P, P, 1.0, SOD, L.CIRCLE, 0.5, 0.5, 0.3, 30, 0),
        (200, 50, T, T, 0.5, HOT, L.PLANAR_X, 0.4, 0.5, 0.0, 55, 1),
        (64, 64, R, R, 1.0, SOD, L.CIRCLE, 0.3, 0.6, 0.2, 0, 1),
        (300, 40, P, R, 0.8, HOT, L.CIRCLE, 0.5, 0.5, 0.25, 25, 3),
        (61, 49, T, P, 1.0, SOD, L.PLANAR_X, 0.55, 0.5, 0.0, 47, 1),
    ]
    out = []
    for nx, ny, bx, by, lam, (inner, outer), geom, a0, a1, r, k, every in spec:
        cfg = L.make_config(2, nx, ny, dt=lam / nx, precision=L.F32, bc_x=bx,
                            bc_y=by, kahan=kahan, cons_every=every)
        out.append((cfg, inner, outer, geom, a0, a1, r, k))
    return out


def _alone(cfg, inner, outer, geom, a0, a1, r, k):
    with L.Solver(cfg) as s:
        s.init_riemann(inner, outer, geom, a0, a1, r)
        s.step(k)
        return s.moments()


@pytest.mark.parametrize("kahan", [0, 1])
def test_batch2d_grids_equal_grids_alone(kahan):
    specs = _grids(kahan)
    grids = [L.make_grid2d(c, i, o, g, a0, a1, r, k)
             for c, i, o, g, a0, a1, r, k in specs]
    with L.Batch2D(grids) as b:
        b.run()
        assert b.steps() == max(s[-1] for s in specs)
        got = [b.moments(j) for j in range(len(specs))]
    for j, sp in enumerate(specs):
        ref = _alone(*sp)
        for f in FIELDS:
            assert np.array_equal(got[j][f], ref[f]), (j, f)


def test_batch2d_partial_runs_compose():
    specs = _grids(0)
    grids = [L.make_grid2d(c, i, o, g, a0, a1, r, k)
             for c, i, o, g, a0, a1, r, k in specs]
    with L.Batch2D(grids) as b:
        b.run()
        whole = [b.moments(j) for j in range(len(specs))]
    with L.Batch2D(grids) as b:
        for part in (7, 1, 13, -1):
            b.run(part)
        pieces = [b.moments(j) for j in range(len(specs))]
    for j in range(len(specs)):
        for f in FIELDS:
            assert np.array_equal(pieces[j][f], whole[j][f]), (j, f)


def test_batch2d_rejects_grids_outside_the_deposit_kernel():
    cfg = L.make_config(2, 32, 32, precision=L.F64)
    with pytest.raises(L.LbmError):
        L.Batch2D([L.make_grid2d(cfg, SOD[0], SOD[1], nsteps=3)])
    cfg = L.make_config(2, 32, 32, precision=L.F32, max_reach=8)
    with pytest.raises(L.LbmError):
        L.Batch2D([L.make_grid2d(cfg, SOD[0], SOD[1], nsteps=3)])
    a = L.make_config(2, 32, 32, precision=L.F32, kahan=0)
    b = L.make_config(2, 32, 32, precision=L.F32, kahan=1)
    with pytest.raises(L.LbmError):
        L.Batch2D([L.make_grid2d(a, SOD[0], SOD[1], nsteps=3),
                   L.make_grid2d(b, SOD[0], SOD[1], nsteps=3)])
