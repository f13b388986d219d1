"""lbm_step_noalloc: the allocation-free step for callers that cannot call
cudaMalloc (code under an allocator it does not own, services that reserve
all memory up front, real-time loops that must not stall on an allocation).

It is checked through the C ABI against the regular handle path
(lbm_create / lbm_step) on two calls in a row, within the tolerances the
parity tests use: bit-exact for FP64, mean |error| <= 1e-5 of each field's
range for FP32.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1602_02675_gb300 import inputs as I
from paper_1602_02675_gb300 import lbm as L

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "mx", "my", "rhoE")


def _close(a, b, prec):
    if prec == L.F64:
        return np.array_equal(a, b)
    rng = np.max(b) - np.min(b)
    scale = rng if rng > 0 else max(np.max(np.abs(b)), 1e-300)
    return np.mean(np.abs(a - b)) / scale <= 1e-5


@pytest.mark.parametrize("dim,prec,shape,bcs", [
    (1, L.F64, (1000, 1), (L.TRANSMISSIVE, 0)),
    (1, L.F32, (777, 1), (L.PERIODIC, 0)),
    # long enough for the 256-node tiles of the 1-D kernel (reach limit 64)
    (1, L.F64, (80000, 1), (L.TRANSMISSIVE, 0)),
    (2, L.F64, (70, 21), (L.TRANSMISSIVE, L.REFLECTING)),
    (2, L.F32, (96, 40), (L.PERIODIC, L.PERIODIC)),
])
def test_noalloc_matches_handle_step_twice(dim, prec, shape, bcs):
    import torch
    assert torch.cuda.is_available()
    nx, ny = shape
    n = nx * ny
    prims = I.random_smooth_prims(dim, nx, ny, seed=900 + nx + dim)
    # lambda = 1, so the handle's physical moments are the lattice moments
    cfg = L.make_config(dim, nx, ny, precision=prec, bc_x=bcs[0], bc_y=bcs[1])
    dt = torch.float64 if prec == L.F64 else torch.float32
    with L.Solver(cfg) as h:
        h.set_primitives(*prims)
        m0 = h.moments()
        dev = [torch.tensor(m0[f], dtype=dt, device="cuda")
               if (f != "my" or dim == 2) else None for f in FIELDS]
        outs = [torch.empty(n, dtype=dt, device="cuda")
                if (f != "my" or dim == 2) else None for f in FIELDS]
        totals = torch.zeros(4, dtype=torch.float64, device="cuda")
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        desc = L.lbm_noalloc_desc(dim, prec, bcs[0], bcs[1], nx,
                                  ny if dim == 2 else 1, 1.4,
                                  0.5 if dim == 1 else 0.0)
        addr = lambda ts: [t.data_ptr() if t is not None else 0 for t in ts]
        for call in range(2):
            src, dst = (dev, outs) if call == 0 else (outs, dev)
            L.lbm_step_noalloc(desc, addr(src), addr(dst),
                               totals=totals.data_ptr(),
                               flags=flags.data_ptr())
            torch.cuda.synchronize()
            h.step(1)
            ref = h.moments()
            for f, t in zip(FIELDS, dst):
                if t is None:
                    continue
                got = t.double().cpu().numpy()
                assert _close(got, ref[f], prec), (call, f)
            assert int(flags.item()) == 0
            # the call's FP64 totals against the exactly rounded sum of the
            # state it wrote
            import math
            tot = totals.cpu().numpy()
            for k, t in enumerate(dst):
                if t is None:
                    continue
                v = t.double().cpu().numpy()
                want = math.fsum(v.tolist())
                scale = math.fsum(np.abs(v).tolist())
                assert abs(tot[k] - want) <= 1e-12 * scale, (call, k)


def test_noalloc_rejects_grids_beyond_its_scratch():
    desc = L.lbm_noalloc_desc(2, L.F32, L.PERIODIC, L.PERIODIC, 8192, 8192,
                              1.4, 0.0)
    fake = [1 << 20] * 4  # never dereferenced: the size check comes first
    with pytest.raises(L.LbmError) as e:
        L.lbm_step_noalloc(desc, fake, fake)
    assert e.value.status == L.EINVAL
    assert "at most" in str(e.value)


@pytest.mark.parametrize("dim,prec", [(2, L.F32), (2, L.F64), (1, L.F64)])
def test_noalloc_reach_beyond_limit_reports_and_leaves_out(dim, prec):
    """A state whose migration reach exceeds the limit (2-D 6, 1-D 64): the
    step does not run, flags carries LBM_EREACH (bit 1), out keeps what it
    held and totals stay zero.  The kernel only returns early here."""
    import torch
    nx, ny = (48, 16) if dim == 2 else (300, 1)
    n = nx * ny
    dt = torch.float64 if prec == L.F64 else torch.float32
    V = 6.0 if dim == 2 else 70.0       # lattice speed: reach > the limit
    rho = torch.ones(n, dtype=dt, device="cuda")
    mx = torch.full((n,), V, dtype=dt, device="cuda")
    my = torch.zeros(n, dtype=dt, device="cuda") if dim == 2 else None
    rhoE = torch.full((n,), 1.0 / 0.4 + 0.5 * V * V, dtype=dt, device="cuda")
    outs = [torch.full((n,), 7.0, dtype=dt, device="cuda")
            if (f != "my" or dim == 2) else None for f in FIELDS]
    totals = torch.full((4,), 5.0, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    reach = torch.zeros(1, dtype=torch.int32, device="cuda")
    desc = L.lbm_noalloc_desc(dim, prec, L.PERIODIC, L.PERIODIC, nx, ny,
                              1.4, 0.5 if dim == 1 else 0.0)
    addr = lambda ts: [t.data_ptr() if t is not None else 0 for t in ts]
    L.lbm_step_noalloc(desc, addr([rho, mx, my, rhoE]), addr(outs),
                       totals=totals.data_ptr(), reach=reach.data_ptr(),
                       flags=flags.data_ptr())
    torch.cuda.synchronize()
    assert int(flags.item()) == 2
    for t in outs:
        if t is not None:
            assert bool(torch.all(t == 7.0))
    assert bool(torch.all(totals == 0.0))
    assert int(reach.item()) > (6 if dim == 2 else 64)
