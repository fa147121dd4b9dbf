"""GPU parity of the H(div)/H(curl) actions (NCF_p mass + div-div, NCE_p
curl-curl, Sec. 2.7 and Eq. curl_curl_form) and the vector-Q_p hyperelastic
residuals (Sec. 4.1) against the FP64 oracle.  FP64 bar: 1e-12 normwise."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    return (5, 4, 4) if p <= 3 else (4, 4, 3)


@pytest.mark.parametrize("fam,form", [("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")])
@pytest.mark.parametrize("p", range(1, 9))
def test_hdivcurl_action_parity(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    nrhs = 2 if p == 2 else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (0.8, 1.3, 0, 0)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, params=prm)
    assert rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm)) <= TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam,form", [("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")])
@pytest.mark.parametrize("prm", [(1, 0, 0, 0), (0, 1, 0, 0)])
def test_hdivcurl_parts(gpu, orc, fam, form, prm):
    """each part of the form separately (mass only / div-div or curl-curl only)"""
    sfx, torch, ctx = gpu
    d, p = (3, 3, 2), 3
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=4)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.from_numpy(x).cuda(), yd, params=prm)
    assert rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm)) <= TOL


def test_exact_sequence_on_gpu(gpu, orc):
    """curl-curl of a gradient and div-div of a curl vanish on the GPU too."""
    sfx, torch, ctx = gpu
    d, p = (3, 3, 3), 3
    X = inputs.box_coords(*d, seed=2)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    nq, _ = orc.space_size("Q", p, d)
    g = orc.interp_grad_q_to_nce(p, d, inputs.random_vector(nq, 1, seed=5))
    sp = sfx.Space(mesh, "NCE", p)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "nce_curlcurl", sp, torch.from_numpy(g).cuda(), yd, params=(0, 1, 0, 0))
    assert yd.abs().max().item() < 1e-11 * np.abs(g).max()
    c = orc.interp_curl_nce_to_ncf(p, d, inputs.random_vector(sp.ndof, 1, seed=6))
    spf = sfx.Space(mesh, "NCF", p)
    yf = torch.empty(spf.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "ncf_mass_divdiv", spf, torch.from_numpy(c).cuda(), yf, params=(0, 1, 0, 0))
    assert yf.abs().max().item() < 1e-10 * np.abs(c).max()


@pytest.mark.parametrize("form", ["neohooke", "svk"])
@pytest.mark.parametrize("p", range(1, 9))
def test_hyperelastic_residual_parity(gpu, orc, form, p):
    sfx, torch, ctx = gpu
    d = (4, 4, 3) if p <= 4 else (3, 3, 2)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), "VQ", p)
    u = inputs.displacement(sp.ndof, p, max(d), seed=1)
    if form == "svk" and p <= 3:
        u = inputs.random_vector(sp.ndof, 1, seed=1, lo=-0.05, hi=0.05)  # the unscaled distribution
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.from_numpy(u).cuda(), yd)
    assert rel(yd.cpu().numpy(), orc.action("VQ", form, p, d, X, u)) <= TOL
    assert ctx.sync_status() == 0


def test_detf_flag(gpu):
    """A displacement that folds the material (det F <= 0) is flagged, the
    points contribute zero and the output stays finite."""
    sfx, torch, ctx = gpu
    d, p = (2, 2, 2), 2
    sp = sfx.Space(sfx.Mesh.box(ctx, *d), "VQ", p)
    u = inputs.random_vector(sp.ndof, 1, seed=3, lo=-2.0, hi=2.0)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, "neohooke", sp, torch.from_numpy(u).cuda(), yd)
    assert ctx.sync_status() == sfx.DEV_DETF
    assert torch.isfinite(yd).all()


@pytest.mark.parametrize("fam,form,p", [("NCF", "ncf_mass_divdiv", 4), ("NCE", "nce_curlcurl", 2),
                                        ("VQ", "neohooke", 3)])
def test_cell_vectors(gpu, orc, fam, form, p):
    sfx, torch, ctx = gpu
    d = (4, 3, 3)
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    x = (inputs.displacement(sp.ndof, p, 4) if fam == "VQ" else inputs.random_vector(sp.ndof, 1, seed=1))
    cells = np.array([35, 0, 12, 7], dtype=np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_cell_vectors(ctx, form, sp, torch.from_numpy(x).cuda(), torch.from_numpy(cells).cuda(), b)
    ref = orc.cell_vectors(fam, form, p, d, X, x, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL


@pytest.mark.parametrize("fam,form,p", [("NCE", "nce_curlcurl", 6), ("VQ", "neohooke", 6),
                                        ("NCF", "ncf_mass_divdiv", 6)])
def test_full_size_sampled(gpu, orc, fam, form, p):
    """Full-size meshes of the structured-element configuration (32^3 for
    NCF/NCE, 48^3 for vector Q): sampled cells' b^K against the oracle, in
    the per-cell output mode, plus a global property on the real launch:
    curl-curl of a discrete gradient vanishes; the residual of zero is zero."""
    sfx, torch, ctx = gpu
    d = (48, 48, 48) if fam == "VQ" else (32, 32, 32)
    mesh = sfx.Mesh.box(ctx, *d)
    X = inputs.box_coords(*d)
    sp = sfx.Space(mesh, fam, p)
    x = inputs.displacement(sp.ndof, p, d[0]) if fam == "VQ" else inputs.random_vector(sp.ndof, 1, seed=1)
    rng = np.random.default_rng(8)
    cells = rng.choice(sp.ncell, 12, replace=False).astype(np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    xd = torch.from_numpy(x).cuda()
    sfx.sfx_assemble_cell_vectors(ctx, form, sp, xd, torch.from_numpy(cells).cuda(), b)
    ref = orc.cell_vectors(fam, form, p, d, X, x, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd)
    assert ctx.sync_status() == 0
    assert torch.isfinite(yd).all()
    if fam == "VQ":
        sfx.sfx_assemble_action(ctx, form, sp, torch.zeros_like(xd), yd)
        assert yd.abs().max().item() == 0.0
