"""Element-matrix parity at the sizes the benchmark and the configurations use
(Sec. 3.2, Eqs. opt1_product / opt2_product; Sec. 4.1, the Laplace matrix
assembly of fig. poisson_assembly).  Bar: 1e-12 per cell,
max|A - A_ref| / max|A_ref|.

* The 4x4x4 Q_2 case exactly as configured: perturbed mesh (seed 0), all 64
  local 27x27 Laplace matrices, and the Laplace action with x from seed 1.
* The 32^3 meshes of the benchmark's element-matrix block, in its launch
  configuration (one call over a chunk of cells sized to about 1 GB of
  output): seeded sampled cells, including the first and the last of the
  chunk, for Q_p Laplace p = 1..8 and NCF/NCE p = 1..5.
* Cell ranges that start mid-mesh at large degree."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, r):
    return np.abs(a - r).max() / np.abs(r).max()


def test_config1_q2_laplace_4cube(gpu, orc):
    sfx, torch, ctx = gpu
    d = (4, 4, 4)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    assert np.array_equal(mesh.coords(), X)
    sp = sfx.Space(mesh, "Q", 2)
    assert sp.ndof == 729 and sp.nloc == 27 and sp.ncell == 64
    A = torch.empty(64 * 27 * 27, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp, 0, 64, A)
    R = orc.cell_matrices("Q", "laplace", 2, d, X)
    Ag = A.cpu().numpy().reshape(64, 27, 27)
    for c in range(64):
        assert rel(Ag[c], R[c]) <= TOL, c
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    y = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "laplace", sp, torch.from_numpy(x).cuda(), y)
    yr = orc.action("Q", "laplace", 2, d, X, x)
    assert rel(y.cpu().numpy(), yr) <= TOL
    assert ctx.sync_status() == 0


CASES = [("Q", "laplace", p) for p in range(1, 9)] + \
        [("NCF", "ncf_mass_divdiv", p) for p in range(1, 6)] + [("NCE", "nce_curlcurl", p) for p in range(1, 6)]


@pytest.fixture(scope="module")
def mesh32(gpu):
    sfx, torch, ctx = gpu
    return sfx.Mesh.box(ctx, 32, 32, 32, perturb=0.1, seed=0), inputs.box_coords(32, 32, 32, perturb=0.1, seed=0)


@pytest.mark.parametrize("fam,form,p", CASES)
def test_bench_chunk_sampled_32cube(gpu, orc, mesh32, fam, form, p):
    sfx, torch, ctx = gpu
    mesh, X = mesh32
    d = (32, 32, 32)
    sp = sfx.Space(mesh, fam, p)
    nc = int(min(sp.ncell, max(8, (1 << 30) // (sp.nloc * sp.nloc * 8))))  # the benchmark's chunk
    A = torch.empty(nc * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, 0, nc, A)
    assert ctx.sync_status() == 0
    rng = np.random.default_rng(100 + p)
    ns = 14 if sp.nloc <= 300 else 4
    cells = sorted({0, nc - 1} | set(int(c) for c in rng.choice(nc, ns, replace=False)))
    Av = A.view(nc, sp.nloc, sp.nloc)
    for c in cells:
        R = orc.cell_matrices(fam, form, p, d, X, c, c + 1)[0]
        assert rel(Av[c].cpu().numpy(), R) <= TOL, (c, nc)


@pytest.mark.parametrize("fam,form,p", [("Q", "helmholtz", 8), ("DQ", "laplace", 7), ("NCE", "nce_curlcurl", 6)])
def test_mid_mesh_range(gpu, orc, mesh32, fam, form, p):
    sfx, torch, ctx = gpu
    mesh, X = mesh32
    sp = sfx.Space(mesh, fam, p)
    c0, c1 = 16411, 16414
    prm = (1.0, -1.0, 0.0, 0.0) if form == "helmholtz" else None
    A = torch.empty((c1 - c0) * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_matrices(ctx, form, sp, c0, c1, A, params=prm)
    R = orc.cell_matrices(fam, form, p, (32, 32, 32), X, c0, c1, params=prm)
    Ag = A.cpu().numpy().reshape(R.shape)
    for k in range(c1 - c0):
        assert rel(Ag[k], R[k]) <= TOL, k
    assert ctx.sync_status() == 0
