"""Batched execution on a p-adaptive DQ mesh (persistent graph-captured launch
and the one-launch-per-(form, degree, RHS) mode) against the FP64 oracle,
cell by cell: cell c of degree p is a DQ_p cell (Gauss nodes, (p+1)^3 dofs)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def oracle_reference(orc, degree, off, dims, X, x, form, nrhs):
    """y[off[c] + l, r] = b^K_l of the oracle's DQ_p action on that cell."""
    ncell = len(degree)
    y = np.zeros((off[-1], nrhs))
    for p in np.unique(degree):
        cells = np.flatnonzero(degree == p)
        n3 = (p + 1) ** 3
        xp = np.zeros((ncell * n3, nrhs))
        for c in cells:
            xp[c * n3:(c + 1) * n3] = x[off[c]:off[c + 1]]
        b = orc.cell_vectors("DQ", form, int(p), dims, X, xp, cells)
        for k, c in enumerate(cells):
            y[off[c]:off[c + 1]] = b[k]
    return y


@pytest.mark.parametrize("nrhs", [1, 3])
def test_plan_matches_oracle(gpu, orc, nrhs):
    sfx, torch, ctx = gpu
    dims = (7, 6, 5)
    X = inputs.box_coords(*dims)
    mesh = sfx.Mesh.structured(ctx, *dims, X)
    degree = inputs.padaptive_degrees(np.prod(dims), 8, seed=2)
    forms = ["laplace", "mass", "helmholtz"]
    plan = sfx.Plan(ctx, mesh, degree, forms, nrhs=nrhs)
    n3 = (degree.astype(np.int64) + 1) ** 3
    assert plan.ndof == n3.sum()
    np.testing.assert_array_equal(plan.cell_offset, np.concatenate([[0], np.cumsum(n3)]))
    x = inputs.random_vector(plan.ndof, nrhs, seed=0)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ys = [torch.empty_like(xd) for _ in forms]
    plan.execute(xd, ys, mode="graph")
    x2 = x.reshape(plan.ndof, nrhs)
    for f, y in zip(forms, ys):
        ref = oracle_reference(orc, degree, plan.cell_offset, dims, X, x2, f, nrhs)
        got = y.cpu().numpy().reshape(plan.ndof, nrhs)
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max(), f
    assert ctx.sync_status() == 0


def test_graph_replay_and_per_launch_bitwise(gpu):
    """Replays of the captured graph and the per-launch mode run the same
    per-cell arithmetic: results are bitwise identical; a new x pointer is
    re-captured."""
    sfx, torch, ctx = gpu
    dims = (9, 8, 8)
    mesh = sfx.Mesh.box(ctx, *dims)
    degree = inputs.padaptive_degrees(np.prod(dims), 8, seed=2)
    forms = ["laplace", "mass"]
    plan = sfx.Plan(ctx, mesh, degree, forms, nrhs=4)
    xd = torch.from_numpy(inputs.random_vector(plan.ndof, 4, seed=1).reshape(-1)).cuda()
    ya = [torch.empty_like(xd) for _ in forms]
    yb = [torch.empty_like(xd) for _ in forms]
    yc = [torch.empty_like(xd) for _ in forms]
    plan.execute(xd, ya, mode="graph")
    plan.execute(xd, ya, mode="graph")   # replay into the same buffers
    plan.execute(xd, yb, mode="per_launch")
    x2 = xd.clone()
    plan.execute(x2, yc, mode="graph")   # new pointers: captured again
    torch.cuda.synchronize()
    for a, b, c in zip(ya, yb, yc):
        assert torch.equal(a, b) and torch.equal(a, c)
    assert ctx.sync_status() == 0


def test_plan_argument_errors(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    with pytest.raises(sfx.SfxError):
        sfx.Plan(ctx, mesh, np.full(8, 9, dtype=np.int32), ["mass"])
    with pytest.raises(sfx.SfxError):
        sfx.Plan(ctx, mesh, np.full(8, 2, dtype=np.int32), ["nce_curlcurl"])
