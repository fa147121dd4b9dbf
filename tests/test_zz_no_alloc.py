"""The allocation-free p-adaptive action (sfx_padaptive_action_noalloc).

It is meant for callers that cannot allocate device memory when they need the
action (a memory pool owns the device, or allocation is allowed only at
start-up).  Its scratch is a fixed device array inside the library that every
call reuses, so each test makes two calls in a row: the second call checks
that the call clears what it must.  The result is compared with the FP64
oracle cell by cell, and with the plan entry point.  A cell whose offsets
break the rules is flagged on the device and skipped, and the other cells
still come out right."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def oracle_blocks(orc, degree, off, dims, X, x, form, nrhs, params=None):
    """y[off[c]:off[c+1]] = b^K of the oracle's DQ_p action on cell c."""
    ncell = len(degree)
    y = np.zeros((off[-1], nrhs))
    for p in np.unique(degree):
        cells = np.flatnonzero(degree == p)
        n3 = (int(p) + 1) ** 3
        xp = np.zeros((ncell * n3, nrhs))
        for c in cells:
            xp[c * n3:(c + 1) * n3] = x[off[c]:off[c + 1]]
        b = orc.cell_vectors("DQ", form, int(p), dims, X, xp, cells, params=params)
        b = b.reshape(len(cells), n3, nrhs)
        for k, c in enumerate(cells):
            y[off[c]:off[c + 1]] = b[k]
    return y


def test_noalloc_matches_oracle_and_plan_twice(gpu, orc):
    sfx, torch, ctx = gpu
    dims = (10, 9, 8)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    degree = inputs.padaptive_degrees(int(np.prod(dims)), 8, seed=2)
    nrhs = 2
    for form, seed in (("laplace", 3), ("helmholtz", 4), ("mass", 5)):
        plan = sfx.Plan(ctx, mesh, degree, [form], nrhs=nrhs)
        xh = inputs.random_vector(plan.ndof, nrhs, seed=seed)
        x = torch.from_numpy(xh.reshape(-1)).cuda()
        ref = torch.empty_like(x)
        plan.execute(x, [ref])
        yo = oracle_blocks(orc, degree, plan.cell_offset, dims, X, xh, form, nrhs)
        deg_d = torch.from_numpy(degree).cuda()
        off_d = torch.from_numpy(plan.cell_offset).cuda()
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            sfx.sfx_padaptive_action_noalloc(ctx, mesh, deg_d, off_d, form, x, y, nrhs=nrhs)
            torch.cuda.synchronize()
            yh = y.cpu().numpy().reshape(-1, nrhs)
            err_orc = np.abs(yh - yo).max() / np.abs(yo).max()
            assert err_orc <= TOL, (form, err_orc)
            err_plan = ((y - ref).abs().max() / ref.abs().max()).item()
            assert err_plan <= TOL, (form, err_plan)
        assert ctx.sync_status() == 0


def test_noalloc_skips_and_flags_bad_offsets(gpu, orc):
    sfx, torch, ctx = gpu
    dims = (4, 3, 5)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    degree = inputs.padaptive_degrees(int(np.prod(dims)), 4, seed=2)
    off = np.concatenate([[0], np.cumsum((degree.astype(np.int64) + 1) ** 3)])
    xh = inputs.random_vector(int(off[-1]), 1, seed=6)
    yo = oracle_blocks(orc, degree, off, dims, X, xh.reshape(-1, 1), "laplace", 1)[:, 0]
    bad = off.copy()
    bad[7] += 1  # cells 6 and 7 now have spans that do not match their degrees
    x = torch.from_numpy(xh).cuda()
    for _ in range(2):
        y = torch.full_like(x, 7.0)
        assert ctx.sync_status() == 0
        sfx.sfx_padaptive_action_noalloc(ctx, mesh, torch.from_numpy(degree).cuda(), torch.from_numpy(bad).cuda(),
                                         "laplace", x, y)
        assert ctx.sync_status() == sfx.DEV_BADCELL
        yh = y.cpu().numpy()
        good = np.ones(len(yh), dtype=bool)
        good[off[6]:off[8]] = False
        assert np.all(yh[~good] == 7.0)  # the skipped cells' blocks are left as they were
        assert np.abs(yh[good] - yo[good]).max() <= TOL * np.abs(yo).max()


def test_noalloc_rejects_too_many_cells(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 65, 64, 64)  # 266240 cells > 262144
    n = 65 * 64 * 64
    deg = torch.ones(n, dtype=torch.int32, device="cuda")
    off = torch.arange(0, 8 * (n + 1), 8, dtype=torch.int64, device="cuda")
    x = torch.zeros(8 * n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_padaptive_action_noalloc(ctx, mesh, deg, off, "mass", x, y)
    assert e.value.code == -5
