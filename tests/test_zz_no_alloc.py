"""The allocation-free p-adaptive action (sfx_padaptive_action_noalloc) gives
the same result as the plan entry point, on two calls in a row.  It is meant
for callers that cannot allocate device memory when they need the action; its
scratch is a fixed device array inside the library that every call reuses, so
the second call also checks that the call clears what it must."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_matches_plan_twice(gpu):
    sfx, torch, ctx = gpu
    dims = (10, 9, 8)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    degree = inputs.padaptive_degrees(int(np.prod(dims)), 8, seed=2)
    nrhs = 2
    for form, seed in (("laplace", 3), ("helmholtz", 4)):
        plan = sfx.Plan(ctx, mesh, degree, [form], nrhs=nrhs)
        x = torch.from_numpy(inputs.random_vector(plan.ndof, nrhs, seed=seed).reshape(-1)).cuda()
        ref = torch.empty_like(x)
        plan.execute(x, [ref])
        deg_d = torch.from_numpy(degree).cuda()
        off_d = torch.from_numpy(plan.cell_offset).cuda()
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            sfx.sfx_padaptive_action_noalloc(ctx, mesh, deg_d, off_d, form, x, y, nrhs=nrhs)
            torch.cuda.synchronize()
            err = ((y - ref).abs().max() / ref.abs().max()).item()
            assert err <= TOL, (form, err)
        assert ctx.sync_status() == 0


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
