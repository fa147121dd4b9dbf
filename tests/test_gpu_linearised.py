"""GPU parity: the linearised hyperelastic operator K(u) du on vector Q_p
(sfx_assemble_linearised_action, the Jacobian of the Sec. 4.1 residual)
through the C ABI against the oracle.

Bar: normwise relative error <= 1e-12 (FP64).  At 48^3 (the hyperelastic mesh
of the structured-element workload) sampled cells are compared one by one."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    return (5, 4, 3) if p <= 3 else ((3, 2, 2) if p <= 6 else (2, 1, 2))


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", range(1, 9))
def test_linearised_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    sp = sfx.Space(mesh, "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)
    nrhs = 2 if p in (2, 5) else 1
    du = inputs.random_vector(sp.ndof, nrhs, seed=2)
    ud = torch.from_numpy(u).cuda()
    dd = torch.from_numpy(np.ascontiguousarray(du)).cuda()
    yd = torch.empty_like(dd)
    sfx.sfx_assemble_linearised_action(ctx, form, sp, ud, dd, yd, nrhs=nrhs)
    yref = orc.linearised_action(form, p, d, X, u, du)
    assert rel(yd.cpu().numpy(), yref) <= TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("form", ["neohooke", "svk"])
def test_linearised_matches_gpu_residual_differences(gpu, form):
    """K(u) du against central differences of the GPU residual (two different
    kernels): the difference is O(e^2) (2e-9 at e = 1e-6 on the CPU oracle for
    this state and direction)."""
    sfx, torch, ctx = gpu
    d, p = (4, 3, 3), 3
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", p)
    u = torch.from_numpy(inputs.displacement(sp.ndof, p, d[0], seed=1, amplitude=0.1)).cuda()
    du = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=3)).cuda()
    k = torch.empty_like(du)
    sfx.sfx_assemble_linearised_action(ctx, form, sp, u, du, k)
    eps = 1e-6
    rp, rm = torch.empty_like(du), torch.empty_like(du)
    sfx.sfx_assemble_action(ctx, form, sp, u + eps * du, rp)
    sfx.sfx_assemble_action(ctx, form, sp, u - eps * du, rm)
    fd = (rp - rm) / (2 * eps)
    assert ((k - fd).abs().max() / k.abs().max()).item() <= 1e-7


@pytest.mark.parametrize("form,p", [("svk", 4), ("neohooke", 6)])
def test_linearised_full_size_sampled(gpu, orc, form, p):
    """48^3, the launch configuration of the benchmark: per-cell vectors of a
    seeded sample of cells against the oracle's, and the assembled action at
    the dofs interior to one sampled cell (owned by that cell alone for p >= 2)
    against that cell's vector."""
    sfx, torch, ctx = gpu
    d = (48, 48, 48)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, "VQ", p)
    u = inputs.displacement(sp.ndof, p, d[0], seed=1)
    du = inputs.random_vector(sp.ndof, 1, seed=2)
    ud, dd = torch.from_numpy(u).cuda(), torch.from_numpy(du).cuda()
    cells = np.random.default_rng(7).choice(sp.ncell, 64, replace=False).astype(np.int64)
    b = torch.empty(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_vectors(ctx, form, sp, ud, dd, torch.from_numpy(cells).cuda(), b)
    bref = orc.linearised_cell_vectors(form, p, d, X, u, du, cells)
    bg = b.cpu().numpy().reshape(len(cells), sp.nloc)
    for k in range(len(cells)):
        assert np.abs(bg[k] - bref[k]).max() <= TOL * np.abs(bref[k]).max()
    y = torch.empty_like(dd)
    sfx.sfx_assemble_linearised_action(ctx, form, sp, ud, dd, y)
    cmap = sp.cell_map()
    n = p + 1
    inner = [(i1 * n + i2) * n + i3 for i1 in range(1, p) for i2 in range(1, p) for i3 in range(1, p)]
    inner = [c * n ** 3 + l for c in range(3) for l in inner]
    yh = y.cpu().numpy()
    for k, c in enumerate(cells[:8]):
        assert np.abs(yh[cmap[c, inner]] - bg[k, inner]).max() <= TOL * np.abs(bg[k]).max()
    assert ctx.sync_status() == 0


def test_linearised_errors(gpu):
    sfx, torch, ctx = gpu
    mesh = sfx.Mesh.box(ctx, 2, 2, 2)
    sp = sfx.Space(mesh, "VQ", 2)
    u = torch.zeros(sp.ndof, dtype=torch.float64, device="cuda")
    du = torch.zeros_like(u)
    y = torch.empty_like(u)
    A = torch.empty(sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:  # tangent matrices: FP64 only
        sfx.sfx_assemble_linearised_cell_matrices(ctx, "neohooke", sp, u, 0, 1, A, precision="tf32x3")
    assert e.value.code == -2
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_action(ctx, "neohooke", sp, u, du, du)
    assert e.value.code == -1
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_action(ctx, "laplace", sp, u, du, y)
    assert e.value.code == -1
    spq = sfx.Space(mesh, "Q", 2)
    uq = torch.zeros(spq.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError) as e:
        sfx.sfx_assemble_linearised_action(ctx, "svk", spq, uq, uq.clone(), torch.empty_like(uq))
    assert e.value.code == -1
