"""GPU parity: scalar forms (mass, Laplace, Helmholtz) on Q_p and DQ_p through
the C ABI against the FP64 oracle (Sec. 1.1 / Sec. 3.3 definitions).

Bar: normwise relative error (inf-norm) <= 1e-12 for the FP64 path."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    # several CTAs and a ragged tail in every colour pass
    return (9, 8, 7) if p <= 3 else (6, 5, 4)


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("form", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("p", range(1, 9))
def test_action_parity(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    nrhs = 2 if p in (2, 5) else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (0.7, -1.3, 0, 0) if form == "helmholtz" else None
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, params=prm)
    y = yd.cpu().numpy()
    yref = orc.action(fam, form, p, d, X, x, params=prm)
    assert rel(y, yref) <= TOL
    assert ctx.sync_status() == 0


def test_accumulate_and_box_mesh(gpu, orc):
    sfx, torch, ctx = gpu
    d, p = (4, 4, 4), 2
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    X = inputs.box_coords(*d)
    sp = sfx.Space(mesh, "Q", p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    y0 = inputs.random_vector(sp.ndof, 1, seed=9)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y0.copy()).cuda()
    sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd, accumulate=True)
    assert rel(yd.cpu().numpy(), y0 + orc.action("Q", "laplace", p, d, X, x)) <= TOL


@pytest.mark.parametrize("fam,p", [("Q", 8), ("DQ", 8), ("Q", 3)])
def test_full_size_sampled(gpu, orc, fam, p):
    """64^3 mesh in the launch configuration the benchmark times: sampled dofs
    y_j = sum over the cells containing j of the oracle's b^K_j, and the
    constant vector in the Laplace kernel."""
    sfx, torch, ctx = gpu
    d = (64, 64, 64)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    X = inputs.box_coords(*d)
    sp = sfx.Space(mesh, fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd)
    m = sp.cell_map()
    rng = np.random.default_rng(3)
    owners = {}
    for c in rng.choice(sp.ncell, 6, replace=False):
        ci = np.unravel_index(c, d)
        nb = [np.ravel_multi_index(t, d) for t in np.ndindex(3, 3, 3)
              if all(0 <= ci[k] + t[k] - 1 < d[k] for k in range(3))
              for t in [tuple(ci[k] + t[k] - 1 for k in range(3))]]
        for j in rng.choice(m[c], 7, replace=False):
            owners[int(j)] = [n for n in nb if (m[n] == j).any()]
    dofs = list(owners)
    allc = np.unique(np.concatenate([np.array(v) for v in owners.values()]))
    b = orc.cell_vectors(fam, "laplace", p, d, X, x, allc)
    row = {c: i for i, c in enumerate(allc)}
    y = yd.cpu().numpy()
    for j in dofs:
        ref = sum(b[row[c]][np.flatnonzero(m[c] == j)[0]] for c in owners[j])
        assert abs(y[j] - ref) <= TOL * max(np.abs(b).max(), 1e-300), (j, y[j], ref)
    one = torch.ones_like(xd)
    sfx.sfx_assemble_action(ctx, "laplace", sp, one, yd)
    assert yd.abs().max().item() < 1e-12 * np.abs(y).max()
    sfx.sfx_assemble_action(ctx, "mass", sp, one, yd)
    assert abs(yd.sum().item() - 1.0) < 1e-11


def test_cell_vectors_and_flags(gpu, orc):
    sfx, torch, ctx = gpu
    d, p = (5, 4, 3), 3
    X = inputs.box_coords(*d)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "Q", p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    cells = np.array([0, 7, 59, 31, 7], dtype=np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, "helmholtz", sp, torch.from_numpy(x).cuda(),
                                  torch.from_numpy(cells).cuda(), b)
    ref = orc.cell_vectors("Q", "helmholtz", p, d, X, x, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL
    assert ctx.sync_status() == 0
    # an out-of-range cell id is skipped and flagged, never dereferenced
    bad = torch.tensor([1, 60, -1], dtype=torch.int64, device="cuda")
    b2 = torch.full((3 * sp.nloc,), 7.0, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, "laplace", sp, torch.from_numpy(x).cuda(), bad, b2)
    assert ctx.sync_status() == sfx.DEV_BADCELL
    b2 = b2.cpu().numpy().reshape(3, -1)
    assert np.all(b2[1:] == 7.0) and not np.all(b2[0] == 7.0)


def test_inverted_cell_flag(gpu):
    """A cell turned inside out (det J < 0) sets the status bit and contributes
    nothing; the context stays usable."""
    sfx, torch, ctx = gpu
    d = (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.0)
    centre = (1 * 3 + 1) * 3 + 1
    X[centre] = [1.2, 1.2, 1.2]  # pushes the centre vertex through the far corner
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "Q", 1)
    xd = torch.ones(sp.ndof, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, "mass", sp, xd, yd)
    assert ctx.sync_status() & sfx.DEV_INVERTED
    assert torch.isfinite(yd).all()
    sfx.sfx_assemble_action(ctx, "mass", sfx.Space(sfx.Mesh.box(ctx, 2, 2, 2), "Q", 1),
                            xd, yd)
    assert ctx.sync_status() == 0
