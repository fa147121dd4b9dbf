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
    for y in outs[1:]:
        assert torch.equal(outs[0], y)


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
