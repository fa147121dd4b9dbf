"""GPU parity of the split-precision (TF32x3 / BF16x3 tensor-core) NCF_p and
NCE_p actions (mass + div-div, mass + curl-curl; Secs. 2.6-2.7, 3.5, Eq.
curl_curl_form) against the FP64 oracle.  Each action runs up to 24 (NCF) or
36 (NCE) one-dimensional contraction stages, at most four deep from a dof to
a point and back to a dof, each with the FP32 accumulator's rounding and the
split's representation error (TF32x3 ~2^-22, BF16x3 ~2^-16 per operand), so
the normwise relative error bar is that of the scalar split-precision
actions: 2e-5 (TF32x3) and 2e-3 (BF16x3)."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"tf32x3": 2e-5, "bf16x3": 2e-3}
FORMS = [("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")]


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dims_for(p):
    # several CTAs and a ragged last one in every colour pass
    return (6, 5, 4) if p <= 3 else (4, 4, 3)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("fam,form", FORMS)
@pytest.mark.parametrize("p", range(1, 9))
def test_hdivcurl_mixed_parity(gpu, orc, prec, fam, form, p):
    sfx, torch, ctx = gpu
    d = dims_for(p)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    nrhs = 2 if p == 2 else 1
    x = inputs.random_vector(sp.ndof, nrhs, seed=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    prm = (0.8, 1.3, 0, 0)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, nrhs=nrhs, precision=prec, params=prm)
    err = rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm))
    assert err <= TOL[prec], err
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("fam,form", FORMS)
@pytest.mark.parametrize("prm", [(1, 0, 0, 0), (0, 1, 0, 0)])
@pytest.mark.parametrize("p", [3, 6])
def test_hdivcurl_mixed_parts(gpu, orc, fam, form, prm, p):
    """the mass part alone, and the div-div / curl-curl part alone"""
    sfx, torch, ctx = gpu
    d = (3, 3, 2)
    X = inputs.box_coords(*d)
    sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=4)
    yd = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    sfx.sfx_assemble_action(ctx, form, sp, torch.from_numpy(x).cuda(), yd, params=prm, precision="tf32x3")
    assert rel(yd.cpu().numpy(), orc.action(fam, form, p, d, X, x, params=prm)) <= TOL["tf32x3"]


def test_exact_sequence_mixed(gpu, orc):
    """curl-curl of a discrete gradient and div-div of a discrete curl vanish
    up to the split-precision error (relative to the same operator applied to
    a generic vector of the same size)."""
    sfx, torch, ctx = gpu
    d, p = (3, 3, 3), 3
    X = inputs.box_coords(*d, seed=2)
    mesh = sfx.Mesh.structured(ctx, *d, X)
    nq, _ = orc.space_size("Q", p, d)
    sp = sfx.Space(mesh, "NCE", p)
    g = orc.interp_grad_q_to_nce(p, d, inputs.random_vector(nq, 1, seed=5))
    r = inputs.random_vector(sp.ndof, 1, seed=7) * np.abs(g).max()
    yg = torch.empty(sp.ndof, dtype=torch.float64, device="cuda")
    yr = torch.empty_like(yg)
    sfx.sfx_assemble_action(ctx, "nce_curlcurl", sp, torch.from_numpy(g).cuda(), yg, params=(0, 1, 0, 0),
                            precision="tf32x3")
    sfx.sfx_assemble_action(ctx, "nce_curlcurl", sp, torch.from_numpy(r).cuda(), yr, params=(0, 1, 0, 0),
                            precision="tf32x3")
    assert yg.abs().max().item() < 1e-4 * yr.abs().max().item()
    spf = sfx.Space(mesh, "NCF", p)
    c = orc.interp_curl_nce_to_ncf(p, d, inputs.random_vector(sp.ndof, 1, seed=6))
    rf = inputs.random_vector(spf.ndof, 1, seed=8) * np.abs(c).max()
    yc = torch.empty(spf.ndof, dtype=torch.float64, device="cuda")
    yf = torch.empty_like(yc)
    sfx.sfx_assemble_action(ctx, "ncf_mass_divdiv", spf, torch.from_numpy(c).cuda(), yc, params=(0, 1, 0, 0),
                            precision="tf32x3")
    sfx.sfx_assemble_action(ctx, "ncf_mass_divdiv", spf, torch.from_numpy(rf).cuda(), yf, params=(0, 1, 0, 0),
                            precision="tf32x3")
    assert yc.abs().max().item() < 1e-4 * yf.abs().max().item()


def test_hdivcurl_mixed_inverted_cell(gpu):
    """a cell turned inside out is flagged and contributes nothing"""
    sfx, torch, ctx = gpu
    d = (2, 2, 2)
    X = inputs.box_coords(*d, perturb=0.0)
    X[(1 * 3 + 1) * 3 + 1] = [1.2, 1.2, 1.2]
    for fam, form in FORMS:
        sp = sfx.Space(sfx.Mesh.structured(ctx, *d, X), fam, 3)
        xd = torch.ones(sp.ndof, dtype=torch.float64, device="cuda")
        yd = torch.empty_like(xd)
        sfx.sfx_assemble_action(ctx, form, sp, xd, yd, precision="tf32x3")
        assert ctx.sync_status() & sfx.DEV_INVERTED
        assert torch.isfinite(yd).all()


@pytest.mark.parametrize("fam,form", FORMS)
@pytest.mark.parametrize("p", [1, 6])
def test_hdivcurl_mixed_full_size_sampled(gpu, orc, fam, form, p):
    """The 32^3 mesh of the structured-element configuration in the
    benchmark's launch configuration: sampled cells' b^K (per-cell output
    mode, first and last cell included) against the oracle, and a finite
    global action with no device flag."""
    sfx, torch, ctx = gpu
    d = (32, 32, 32)
    mesh = sfx.Mesh.box(ctx, *d)
    X = inputs.box_coords(*d)
    sp = sfx.Space(mesh, fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    rng = np.random.default_rng(8)
    cells = np.concatenate([[0, sp.ncell - 1], rng.choice(sp.ncell, 10, replace=False)]).astype(np.int64)
    b = torch.zeros(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
    xd = torch.from_numpy(x).cuda()
    sfx.sfx_assemble_cell_vectors(ctx, form, sp, xd, torch.from_numpy(cells).cuda(), b, precision="tf32x3")
    ref = orc.cell_vectors(fam, form, p, d, X, x, cells)
    assert rel(b.cpu().numpy().reshape(ref.shape), ref) <= TOL["tf32x3"]
    yd = torch.empty_like(xd)
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, precision="tf32x3")
    assert ctx.sync_status() == 0
    assert torch.isfinite(yd).all()
