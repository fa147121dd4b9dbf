"""Full-size parity in the launch configurations the benchmark times, on
sampled outputs the oracle computes one by one.

* The 64^3 action sweep in split precision (one right-hand side, geometry at
  the point, the built-in cells per CTA): sampled dofs y_j = sum over the cells
  containing j of the oracle's b^K_j.  Bars: TF32x3 2e-5, BF16x3 2e-3 relative
  to the largest sampled |b|.
* The p-adaptive batch (200,000 cells on 40x50x100, p in 1..8 with P(p) ~ 1/p,
  16 right-hand sides, Laplace + mass, one graph launch): every sampled cell's
  block of y against the oracle on a one-cell mesh made of that cell's eight
  corners (DQ dofs belong to one cell), FP64 bar 1e-12.
"""
import numpy as np
import pytest

from paper_1711_02473_gb300 import inputs

pytestmark = pytest.mark.gpu
HELM = (1.0, -1.0, 0.0, 0.0)
TOL = {"tf32x3": 2e-5, "bf16x3": 2e-3}


def neighbours(c, d):
    ci = np.unravel_index(c, d)
    out = []
    for t in np.ndindex(3, 3, 3):
        q = tuple(ci[k] + t[k] - 1 for k in range(3))
        if all(0 <= q[k] < d[k] for k in range(3)):
            out.append(int(np.ravel_multi_index(q, d)))
    return out


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("fam,p", [("Q", 8), ("DQ", 8), ("Q", 3)])
@pytest.mark.parametrize("form", ["laplace", "helmholtz"])
def test_split_precision_64cube_sampled(gpu, orc, prec, fam, p, form):
    sfx, torch, ctx = gpu
    d = (64, 64, 64)
    mesh = sfx.Mesh.box(ctx, *d, perturb=0.1, seed=0)
    X = inputs.box_coords(*d, perturb=0.1, seed=0)
    sp = sfx.Space(mesh, fam, p)
    x = inputs.random_vector(sp.ndof, 1, seed=1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    prm = HELM if form == "helmholtz" else None
    sfx.sfx_assemble_action(ctx, form, sp, xd, yd, precision=prec, params=prm)
    assert ctx.sync_status() == 0
    m = sp.cell_map()
    rng = np.random.default_rng(5)
    owners = {}
    for c in list(rng.choice(sp.ncell, 5, replace=False)) + [0, sp.ncell - 1]:
        nb = neighbours(int(c), d)
        for j in rng.choice(m[c], 6, replace=False):
            owners[int(j)] = [n for n in nb if (m[n] == j).any()]
    allc = np.unique(np.concatenate([np.array(v) for v in owners.values()]))
    b = orc.cell_vectors(fam, form, p, d, X, x, allc, params=prm)
    row = {c: i for i, c in enumerate(allc)}
    y = yd.cpu().numpy()
    scale = np.abs(b).max()
    for j, cs in owners.items():
        ref = sum(b[row[c]][np.flatnonzero(m[c] == j)[0]] for c in cs)
        assert abs(y[j] - ref) <= TOL[prec] * scale, (j, y[j], ref)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("tf32x3", 2e-5)])
def test_padaptive_200k_cells_16rhs_sampled(gpu, orc, prec, tol):
    sfx, torch, ctx = gpu
    dims = (40, 50, 100)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    deg = inputs.padaptive_degrees(int(np.prod(dims)), 8, seed=2)
    forms, R = ["laplace", "mass"], 16
    plan = sfx.Plan(ctx, mesh, deg, forms, nrhs=R, precision=prec)
    x = np.stack([inputs.random_vector(plan.ndof, 1, seed=r) for r in range(R)], axis=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(-1)
    ys = [torch.empty_like(xd) for _ in forms]
    plan.execute(xd, ys, mode="graph")
    assert ctx.sync_status() == 0
    off = plan.cell_offset
    rng = np.random.default_rng(11)
    cells = sorted(set(int(c) for c in rng.choice(len(deg), 10, replace=False)) |
                   {0, len(deg) - 1} | {int(np.flatnonzero(deg == p)[-1]) for p in range(1, 9)})
    ny, nz = dims[1], dims[2]
    for c in cells:
        ci, cj, ck = np.unravel_index(c, dims)
        vids = [(I * (ny + 1) + J) * (nz + 1) + K for I in (ci, ci + 1) for J in (cj, cj + 1) for K in (ck, ck + 1)]
        Xc = X[vids]
        p = int(deg[c])
        xl = x[off[c]:off[c + 1]]
        for f, y in zip(forms, ys):
            ref = orc.cell_vectors("DQ", f, p, (1, 1, 1), Xc, xl, [0])[0]
            got = y[off[c] * R:off[c + 1] * R].cpu().numpy().reshape(-1, R)
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (c, p, f)
