"""The README's usage example runs as written (64^3 mesh, Q_4 split-precision
Laplace action, vector Q_3 residual and tangent matrices of 100 cells), with
no device-detected condition, and its outputs agree with the FP64 path and with
the symmetry of the tangent."""
import pytest

pytestmark = pytest.mark.gpu


def test_readme_example(gpu):
    sfx, torch, ctx = gpu
    from paper_1711_02473_gb300 import inputs
    mesh = sfx.Mesh.box(ctx, 64, 64, 64, perturb=0.1, seed=0)
    V = sfx.Space(mesh, "Q", 4)
    x = torch.from_numpy(inputs.random_vector(V.ndof, 1, seed=1)).cuda()
    y = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", V, x, y, precision="tf32x3")

    W = sfx.Space(mesh, "VQ", 3)
    u = torch.from_numpy(inputs.displacement(W.ndof, 3, 64, seed=1)).cuda()
    r = torch.empty_like(u)
    sfx.sfx_assemble_action(ctx, "neohooke", W, u, r)
    A = torch.empty(100 * W.nloc * W.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_linearised_cell_matrices(ctx, "neohooke", W, u, 0, 100, A)
    assert ctx.sync_status() == 0

    y64 = torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, "laplace", V, x, y64)
    assert ((y - y64).abs().max() / y64.abs().max()).item() <= 2e-5
    A = A.view(100, W.nloc, W.nloc)
    assert torch.isfinite(A).all() and torch.isfinite(r).all()
    assert ((A - A.transpose(1, 2)).abs().max() / A.abs().max()).item() <= 1e-12
