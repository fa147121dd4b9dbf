"""GPU parity: the weighted Laplace form int kappa grad u . grad v (Sec. 1.1,
Eq. weighted_laplace) on Q_p / DQ_p through the C ABI against the oracle.

Bar: 1e-12 normwise (FP64).  Larger meshes: properties that hold at any size
(constant kappa scales the Laplace action; the energy |a|^2 int kappa of a
linear field with a linear coefficient)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    return (9, 8, 7) if p <= 3 else (6, 5, 4)


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", range(1, 9))
def test_weighted_action_parity(gpu, orc, fam, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    kappa = 1.0 + 0.5 * inputs.random_vector(sp.ndof, 1, seed=7)
    nrhs = 2 if p in (2, 5) else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    kd = torch.from_numpy(kappa).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_weighted_action(ctx, sp, kd, xd, yd, nrhs=nrhs)
    yref = orc.weighted_action(fam, p, d, X, kappa, x)
    assert rel(yd.cpu().numpy(), yref) <= TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam", ["Q", "DQ"])
@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_weighted_cell_matrices_parity(gpu, orc, fam, p):
    sfx, torch, ctx = gpu
    d = (3, 2, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=3)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, fam, p)
    kappa = 1.0 + 0.5 * inputs.random_vector(sp.ndof, 1, seed=8)
    A = torch.empty(sp.ncell * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_weighted_cell_matrices(ctx, sp, torch.from_numpy(kappa).cuda(), 0, sp.ncell, A)
    Ag = A.cpu().numpy().reshape(sp.ncell, sp.nloc, sp.nloc)
    Aref = orc.weighted_cell_matrices(fam, p, d, X, kappa)
    for c in range(sp.ncell):
        assert np.abs(Ag[c] - Aref[c]).max() <= TOL * np.abs(Aref[c]).max()


@pytest.mark.parametrize("fam", ["Q", "DQ"])
def test_weighted_full_size_constant_kappa(gpu, fam):
    """64^3, p = 8, the benchmark's mesh: kappa = 2.5 everywhere gives 2.5 x
    the (separately tested) Laplace action."""
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 64, 64, 64, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, 8)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
    kd = torch.full_like(x, 2.5)
    y, yl = torch.empty_like(x), torch.empty_like(x)
    sfx.sfx_assemble_weighted_action(ctx, sp, kd, x, y)
    sfx.sfx_assemble_action(ctx, "laplace", sp, x, yl)
    assert ((y - 2.5 * yl).abs().max() / (2.5 * yl).abs().max()).item() <= TOL
    assert ctx.sync_status() == 0


def test_weighted_energy_of_linear_field(gpu, orc):
    """u = a.x, kappa = b + c.x on a 32^3 perturbed mesh, Q_4: u . A_kappa u =
    |a|^2 int kappa = |a|^2 (b + c . (1/2, 1/2, 1/2)) exactly."""
    sfx, torch, ctx = gpu
    d, p = (32, 32, 32), 4
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "Q", p)
    xn = orc.q_node_coords(p, d, X)
    a, b, c = np.array([0.4, -0.9, 1.3]), 1.7, np.array([0.3, -0.5, 0.8])
    u = torch.from_numpy(xn @ a).cuda()
    kd = torch.from_numpy(b + xn @ c).cuda()
    y = torch.empty_like(u)
    sfx.sfx_assemble_weighted_action(ctx, sp, kd, u, y)
    assert abs((u @ y).item() - (a @ a) * (b + c @ np.array([0.5, 0.5, 0.5]))) <= 1e-10


def test_weighted_errors(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    sp = sfx.Space(mesh, "Q", 2)
    x = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    k = torch.ones_like(x)
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_weighted_action(ctx, sp, k, x, x)
    assert e.value.code == -1
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_weighted_action(ctx, sp, k, x, torch.empty_like(x), precision="tf32x3")
    assert e.value.code == -2
    spv = sfx.Space(mesh, "NCF", 2)
    xv = torch.zeros(spv.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_weighted_action(ctx, spv, torch.ones_like(xv), xv, torch.empty_like(xv))
    assert e.value.code == -1
