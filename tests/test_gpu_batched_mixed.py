"""The split-precision p-adaptive batch (sfx_plan_create_padaptive_prec with
TF32x3 / BF16x3 tile bodies): one persistent graph-captured launch over cells
of every degree, several forms and right-hand sides, against the FP64 oracle
cell by cell at the split-precision bars of the scalar actions (TF32x3 2e-5,
BF16x3 2e-3, normwise per form), and bitwise against its own per-launch mode
(one launch per form and degree) and against the split-precision action of a
uniform DQ_p space (the same tile body)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

from test_gpu_batched import oracle_reference

pytestmark = pytest.mark.gpu
TOL = {"tf32x3": 2e-5, "bf16x3": 2e-3}


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_mixed_plan_matches_oracle(gpu, orc, prec, nrhs):
    sfx, torch, ctx = gpu
    dims = (7, 6, 5)
    X = inputs.box_coords(*dims)
    mesh = sfx.Mesh.structured(ctx, *dims, X)
    degree = inputs.padaptive_degrees(np.prod(dims), 8, seed=2)
    forms = ["laplace", "mass", "helmholtz"]
    plan = sfx.Plan(ctx, mesh, degree, forms, nrhs=nrhs, precision=prec)
    x = inputs.random_vector(plan.ndof, nrhs, seed=0)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ys = [torch.full_like(xd, float("nan")) for _ in forms]
    plan.execute(xd, ys, mode="graph")
    x2 = x.reshape(plan.ndof, nrhs)
    for f, y in zip(forms, ys):
        ref = oracle_reference(orc, degree, plan.cell_offset, dims, X, x2, f, nrhs)
        got = y.cpu().numpy().reshape(plan.ndof, nrhs)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL[prec], (f, err)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("nrhs", [1, 4, 16])
def test_mixed_plan_graph_per_launch_bitwise(gpu, nrhs):
    sfx, torch, ctx = gpu
    dims = (9, 8, 8)
    mesh = sfx.Mesh.box(ctx, *dims)
    degree = inputs.padaptive_degrees(np.prod(dims), 8, seed=2)
    forms = ["laplace", "mass"]
    plan = sfx.Plan(ctx, mesh, degree, forms, nrhs=nrhs, precision="tf32x3")
    xd = torch.from_numpy(inputs.random_vector(plan.ndof, nrhs, seed=1).reshape(-1)).cuda()
    ya = [torch.full_like(xd, float("nan")) for _ in forms]
    yb = [torch.full_like(xd, float("nan")) for _ in forms]
    plan.execute(xd, ya, mode="graph")
    plan.execute(xd, ya, mode="graph")
    plan.execute(xd, yb, mode="per_launch")
    torch.cuda.synchronize()
    for a, b in zip(ya, yb):
        assert torch.equal(a, b)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("p", [1, 4, 7, 8])
def test_mixed_plan_uniform_degree_equals_action(gpu, p):
    """All cells of one degree: the plan's dof numbering is the DQ_p space's, so
    the batch must equal the split-precision DQ_p action bitwise (same tile
    body, same staging of the factors for several RHS)."""
    sfx, torch, ctx = gpu
    dims = (6, 5, 4)
    mesh = sfx.Mesh.box(ctx, *dims)
    degree = np.full(np.prod(dims), p, dtype=np.int32)
    nrhs = 2
    plan = sfx.Plan(ctx, mesh, degree, ["helmholtz"], nrhs=nrhs, precision="tf32x3",
                    params=[(1.0, -1.0, 0.0, 0.0)])
    sp = sfx.Space(mesh, "DQ", p)
    assert sp.ndof == plan.ndof
    xd = torch.from_numpy(inputs.random_vector(plan.ndof, nrhs, seed=3).reshape(-1)).cuda()
    yp = [torch.empty_like(xd)]
    plan.execute(xd, yp)
    old = sfx.sfx_tune_get_warp_specialised(p)
    sfx.sfx_tune_set_warp_specialised(p, False)  # the one-role kernel: the plan's tile body
    try:
        ya = torch.empty_like(xd)
        sfx.sfx_assemble_action(ctx, "helmholtz", sp, xd, ya, nrhs=nrhs, precision="tf32x3",
                                params=(1.0, -1.0, 0.0, 0.0))
        torch.cuda.synchronize()
    finally:
        sfx.sfx_tune_set_warp_specialised(p, old)
    assert torch.equal(yp[0], ya)
    assert ctx.sync_status() == 0


def test_mixed_plan_tile_sizes_bitwise(gpu):
    """Cells per tile (kind 11) change only the launch geometry."""
    sfx, torch, ctx = gpu
    dims = (8, 7, 6)
    mesh = sfx.Mesh.box(ctx, *dims)
    degree = inputs.padaptive_degrees(np.prod(dims), 8, seed=4)
    outs = []
    try:
        for cb in (0, 1, 3):
            for p in range(1, 9):
                sfx.sfx_tune_set_cells_per_cta("batched_mixed", p, cb)
            plan = sfx.Plan(ctx, mesh, degree, ["laplace"], nrhs=2, precision="tf32x3")
            xd = torch.from_numpy(inputs.random_vector(plan.ndof, 2, seed=5).reshape(-1)).cuda()
            y = [torch.empty_like(xd)]
            plan.execute(xd, y)
            torch.cuda.synchronize()
            outs.append(y[0])
            plan.close()
    finally:
        for p in range(1, 9):
            sfx.sfx_tune_set_cells_per_cta("batched_mixed", p, 0)
    for y in outs[1:]:
        assert torch.equal(outs[0], y)
    assert ctx.sync_status() == 0


def test_mixed_plan_argument_errors(gpu):
    """An unknown precision is an argument error; a degree out of range too."""
    import ctypes as C
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    deg = np.full(8, 2, dtype=np.int32)
    forms = (C.c_int * 1)(sfx.FORM["laplace"])
    h = C.c_void_p()
    rc = sfx.lib().sfx_plan_create_padaptive_prec(ctx.h, mesh.h, deg.ctypes.data_as(C.c_void_p), 1,
                                                  C.cast(forms, C.c_void_p), None, 1, 7, C.byref(h))
    assert rc != 0 and not h.value
    with pytest.raises(sfx.SfxError):
        sfx.Plan(ctx, mesh, np.full(8, 9, dtype=np.int32), ["mass"], precision="tf32x3")
