"""The cells-per-CTA knob changes only the launch geometry: every cell's
arithmetic is the same, so results are bitwise identical for every value,
including ragged last CTAs; and the autotuner picks one of its candidates."""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,prec,stored", [("fp64", "fp64", False), ("mixed", "tf32x3", False),
                                              ("mixed_stored", "tf32x3", True), ("mixed", "bf16x3", False)])
@pytest.mark.parametrize("p", [1, 3, 6])
def test_cells_per_cta_bitwise(gpu, kind, prec, stored, p):
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 7, 6, 5), "Q", p)
    q = sfx.QData(ctx, sp, "fp32") if stored else None
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    outs = []
    ws = p >= 3 and sfx.sfx_tune_get_warp_specialised(p)
    if ws and kind == "mixed":
        sfx.sfx_tune_set_warp_specialised(p, False)  # the one-role kernel whose knob this is
    try:
        for cb in (1, 2, 3, 5, 16):
            sfx.sfx_tune_set_cells_per_cta(kind, p, cb)
            y = torch.empty_like(x)
            if stored:
                sfx.sfx_assemble_action_stored(ctx, "helmholtz", sp, q, x, y, precision=prec)
            else:
                sfx.sfx_assemble_action(ctx, "helmholtz", sp, x, y, precision=prec)
            outs.append(y)
    finally:
        sfx.sfx_tune_set_cells_per_cta(kind, p, 0)
        if ws:
            sfx.sfx_tune_set_warp_specialised(p, True)
    for y in outs[1:]:
        assert torch.equal(outs[0], y)


@pytest.mark.parametrize("p", [4, 8])
@pytest.mark.parametrize("form", ["laplace", "helmholtz"])
def test_ws_cells_per_batch_bitwise(gpu, p, form):
    """Warp-specialised kernel: cells per batch (and so the persistent grid's
    batch count and the contraction tiles' cell mix) change nothing."""
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 9, 7, 6), "Q", p)
    x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    old = sfx.sfx_tune_get_warp_specialised(p)
    sfx.sfx_tune_set_warp_specialised(p, True)
    outs = []
    try:
        for cb in (1, 2, 3, 0):
            sfx.sfx_tune_set_cells_per_cta("mixed_ws", p, cb)
            y = torch.empty_like(x)
            sfx.sfx_assemble_action(ctx, form, sp, x, y, precision="tf32x3")
            outs.append(y)
    finally:
        sfx.sfx_tune_set_cells_per_cta("mixed_ws", p, 0)
        sfx.sfx_tune_set_warp_specialised(p, old)
    assert ctx.sync_status() == 0
    for y in outs[1:]:
        assert torch.equal(outs[0], y)


def test_batched_tile_sizes_bitwise(gpu):
    """The persistent p-adaptive batch: cells per tile (tuned per degree,
    clamped to the layout's count) change nothing."""
    sfx, torch, ctx = gpu
    dims = (6, 5, 7)
    mesh = sfx.Mesh.box(ctx, *dims)
    deg = inputs.padaptive_degrees(int(np.prod(dims)), 8, seed=2)
    outs, ntiles = [], []
    try:
        for cb in (1, 3, 1000, 0):
            for p in range(1, 9):
                sfx.sfx_tune_set_cells_per_cta("batched", p, min(cb, 64))
            plan = sfx.Plan(ctx, mesh, deg, ["laplace", "mass"], nrhs=2)
            x = torch.from_numpy(inputs.random_vector(plan.ndof * 2, 1, seed=3)).cuda()
            ys = [torch.empty_like(x) for _ in range(2)]
            plan.execute(x, ys)
            outs.append(ys)
            ntiles.append(plan.ntiles)
    finally:
        for p in range(1, 9):
            sfx.sfx_tune_set_cells_per_cta("batched", p, 0)
    assert ctx.sync_status() == 0
    assert ntiles[0] > ntiles[1] >= ntiles[2] == ntiles[3]
    for ys in outs[1:]:
        assert torch.equal(outs[0][0], ys[0]) and torch.equal(outs[0][1], ys[1])


def test_autotune_small(gpu):
    sfx, torch, ctx = gpu
    from paper_1711_02473_gb300 import autotune
    try:
        table = autotune.tune(ctx, degrees=[2], kinds=("fp64", "mixed"), dims=(8, 8, 8), reps=1)
        for kind in ("fp64", "mixed"):
            best = table[kind][2]["best"]
            assert best in autotune.candidates(kind, 2)
            assert sfx.sfx_tune_get_cells_per_cta(kind, 2) == best
    finally:
        for kind in ("fp64", "mixed"):
            sfx.sfx_tune_set_cells_per_cta(kind, 2, 0)


def test_autotune_other_kinds_small(gpu):
    """Every other kind tunes without flagging the device status (the
    hyperelastic states keep det F > 0) and sets one of its candidates."""
    sfx, torch, ctx = gpu
    from paper_1711_02473_gb300 import autotune
    kinds = ("hdivcurl", "elastic", "linearised", "linearised_mixed", "hdivcurl_mixed", "batched", "batched_mixed",
             "mixed", "mixed_ws")
    try:
        table = autotune.tune(ctx, degrees=[3], kinds=kinds, dims=(8, 8, 8), reps=1)
        assert ctx.sync_status() == 0
        for kind in kinds:
            assert table[kind][3]["best"] in autotune.candidates(kind, 3), kind
    finally:
        for kind in kinds:
            autotune.set_value(kind, 3, 0)
        sfx.sfx_tune_set_warp_specialised(3, False)


@pytest.mark.parametrize("kind,fam,form,prec", [("hdivcurl", "NCF", "ncf_mass_divdiv", "fp64"),
                                               ("hdivcurl", "NCE", "nce_curlcurl", "fp64"),
                                               ("elastic", "VQ", "neohooke", "fp64"),
                                               ("linearised", "VQ", "svk", "fp64"),
                                               ("linearised_mixed", "VQ", "neohooke", "tf32x3"),
                                               ("hdivcurl_mixed", "NCF", "ncf_mass_divdiv", "tf32x3"),
                                               ("hdivcurl_mixed", "NCE", "nce_curlcurl", "bf16x3")])
@pytest.mark.parametrize("p", [1, 3])
def test_structured_cells_per_cta_bitwise(gpu, kind, fam, form, prec, p):
    """H(div)/H(curl) and hyperelastic kernels: cells per CTA (tuned, clamped
    to the team limit and shared memory) change nothing."""
    sfx, torch, ctx = gpu
    sp = sfx.Space(sfx.Mesh.box(ctx, 5, 4, 3), fam, p)
    x = torch.from_numpy(inputs.displacement(sp.ndof, p, 5, seed=2) if fam == "VQ"
                         else inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
    d = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=3)).cuda()
    outs = []
    try:
        for cb in (1, 2, 3, 64, 0):
            sfx.sfx_tune_set_cells_per_cta(kind, p, cb)
            y = torch.empty_like(x)
            if kind.startswith("linearised"):
                sfx.sfx_assemble_linearised_action(ctx, form, sp, x, d, y, precision=prec)
            else:
                sfx.sfx_assemble_action(ctx, form, sp, x, y, precision=prec)
            outs.append(y)
    finally:
        sfx.sfx_tune_set_cells_per_cta(kind, p, 0)
    assert ctx.sync_status() == 0
    for y in outs[1:]:
        assert torch.equal(outs[0], y)
