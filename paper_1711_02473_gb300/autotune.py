"""Autotuner for the cells-per-CTA of the scalar action kernels.

For each kernel kind ("fp64", "mixed", "mixed_stored", "mixed_ws", "batched", "batched_mixed", and the
structured-element kinds "hdivcurl", "elastic", "linearised", "linearised_mixed", "hdivcurl_mixed") and
degree it times
the Q_p Laplace action on a tuning mesh for every candidate value (median of a
few CUDA-event timings, L2 flushed between runs), keeps the fastest, and sets
it in the library with sfx_tune_set_cells_per_cta.  For "mixed_ws" (the
warp-specialised split-precision kernel, p >= 3) the candidates are cells per
batch plus -1, which switches that kernel off for the degree in favour of the
one-role kernel; "mixed" is timed with it off.  The table can be saved per
GPU name and re-applied.  Only launch geometry changes: results are the same
sums (the per-cell arithmetic does not depend on how many cells share a CTA).
"""
import json
import os

import numpy as np

from . import (Context, Mesh, QData, Space, TUNE_KERNEL, sfx_assemble_action, sfx_assemble_action_stored,
               sfx_tune_get_warp_specialised, sfx_tune_set_cells_per_cta, sfx_tune_set_warp_specialised)
from . import inputs

_BUILD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")


def candidates(kind, p):
    n2 = (p + 1) ** 2
    if kind == "fp64":
        top = max(1, 256 // n2)
        return sorted({max(1, top // d) for d in (1, 2, 3, 4, 6)})
    if kind == "mixed_ws":
        return [-1, 1, 2, 3, 4, 6, 8] if p >= 3 else []
    if kind in ("batched", "batched_mixed"):
        return [1, 2, 4, 8, 16, 32]
    if kind in ("hdivcurl", "elastic", "linearised"):  # teams of (p+1)^2 threads, at most 256 threads
        top = max(1, 256 // n2)
        return sorted({c for c in (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64) if c <= top})
    if kind in ("linearised_mixed", "hdivcurl_mixed"):
        return [1, 2, 4, 8, 16]
    return [2, 4, 6, 8, 12, 16, 24, 32] if p <= 2 else [1, 2, 3, 4, 6, 8, 12, 16]


def _time(torch, fn, reps, flush):
    fn()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def set_value(kind, p, cb):
    """Apply one table entry (mixed_ws: -1 = off, else on with cb cells)."""
    if kind == "mixed_ws":
        if p < 3:
            return
        sfx_tune_set_warp_specialised(p, cb >= 0)
        sfx_tune_set_cells_per_cta(kind, p, max(cb, 0))
    else:
        sfx_tune_set_cells_per_cta(kind, p, cb)


def tune(ctx, degrees=range(1, 9), kinds=("fp64", "mixed", "mixed_stored"), dims=(32, 32, 32), reps=3):
    """Returns {kind: {p: {"best": cb, "ms": {cb: t}}}} and applies the winners."""
    import torch
    mesh = Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    flush = torch.empty((256 << 20) // 4, dtype=torch.float32, device="cuda")
    table = {}
    for bk, prec in (("batched", "fp64"), ("batched_mixed", "tf32x3")):
        if bk in kinds:
            table[bk] = tune_batched(ctx, degrees, torch, flush, reps, kind=bk, precision=prec)
            kinds = [k for k in kinds if k != bk]
    for k in [k for k in kinds if k in STRUCTURED]:
        table[k] = tune_structured(ctx, k, degrees, torch, flush, reps)
    kinds = [k for k in kinds if k not in STRUCTURED]
    for p in degrees:
        if not kinds:
            break
        sp = Space(mesh, "Q", p)
        x = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        y = torch.empty_like(x)
        qd = QData(ctx, sp, "fp32") if "mixed_stored" in kinds else None
        ws_was = sfx_tune_get_warp_specialised(p)
        for kind in sorted(kinds, key=lambda k: k == "mixed_ws"):  # the one-role kernel first
            if kind == "mixed_ws" and p < 3:
                continue
            if kind == "fp64":
                fn = lambda: sfx_assemble_action(ctx, "laplace", sp, x, y)
            elif kind in ("mixed", "mixed_ws"):
                fn = lambda: sfx_assemble_action(ctx, "laplace", sp, x, y, precision="tf32x3")
            else:
                fn = lambda: sfx_assemble_action_stored(ctx, "laplace", sp, qd, x, y, precision="tf32x3")
            if kind == "mixed" and p >= 3:
                sfx_tune_set_warp_specialised(p, False)
            res = {}
            for cb in candidates(kind, p):
                set_value(kind, p, cb)
                res[cb] = _time(torch, fn, reps, flush)
            best = min(res, key=res.get)
            set_value(kind, p, best)
            if kind == "mixed" and p >= 3:
                sfx_tune_set_warp_specialised(p, ws_was)
            table.setdefault(kind, {})[p] = {"best": best, "ms": {str(k): round(v, 4) for k, v in res.items()}}
        if qd is not None:
            qd.close()
        del x, y, sp
    return table


# kind -> (family, forms timed, precision, degrees it has, tuning mesh)
# (meshes large enough that a colour launch fills the GPU at every candidate: on a
# smaller one the fewest cells per CTA win only because they give more CTAs)
STRUCTURED = {"hdivcurl": ("NCF", ("ncf_mass_divdiv",), "fp64", range(1, 9), (32, 32, 32)),
              "elastic": ("VQ", ("neohooke",), "fp64", range(1, 9), (24, 24, 24)),
              "linearised": ("VQ", ("svk",), "fp64", range(1, 9), (24, 24, 24)),
              "linearised_mixed": ("VQ", ("svk",), "tf32x3", range(1, 9), (24, 24, 24)),
              "hdivcurl_mixed": ("NCE", ("nce_curlcurl",), "tf32x3", range(1, 9), (32, 32, 32))}


def tune_structured(ctx, kind, degrees, torch, flush, reps):
    """Cells per CTA of the NCF / NCE and hyperelastic kernels, per degree
    (NCF and NCE share the H(div)/H(curl) kernel's table; the NCF action is
    timed)."""
    from . import sfx_assemble_linearised_action
    fam, forms, prec, ps, dims = STRUCTURED[kind]
    mesh = Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    out = {}
    for p in degrees:
        if p not in ps:
            continue
        sp = Space(mesh, fam, p)
        # a displacement small enough that det F > 0 everywhere (the residual's recipe)
        x = torch.from_numpy(inputs.displacement(sp.ndof, p, dims[0], seed=1) if fam == "VQ"
                             else inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        d = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=2)).cuda()
        y = torch.empty_like(x)
        if kind.startswith("linearised"):
            fn = lambda: sfx_assemble_linearised_action(ctx, forms[0], sp, x, d, y, precision=prec)
        else:
            fn = lambda: sfx_assemble_action(ctx, forms[0], sp, x, y, precision=prec)
        res = {}
        for cb in candidates(kind, p):
            sfx_tune_set_cells_per_cta(kind, p, cb)
            res[cb] = _time(torch, fn, reps, flush)
        best = min(res, key=res.get)
        sfx_tune_set_cells_per_cta(kind, p, best)
        out[p] = {"best": best, "ms": {str(k): round(v, 4) for k, v in res.items()}}
        del x, d, y, sp
    if ctx.sync_status() != 0:
        raise RuntimeError("device status flagged while tuning " + kind)
    return out


def tune_batched(ctx, degrees, torch, flush, reps, dims=(20, 20, 20), nrhs=4, kind="batched", precision="fp64"):
    """Cells per tile of the persistent p-adaptive batch, per degree: a DQ_p
    mesh of that single degree, Laplace + mass on nrhs right-hand sides, one
    graph launch per candidate (a plan per candidate: tiles are cut when the
    plan is made)."""
    from . import Plan
    mesh = Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    ncell = dims[0] * dims[1] * dims[2]
    out = {}
    for p in degrees:
        res = {}
        deg = np.full(ncell, p, dtype=np.int32)
        for cb in candidates(kind, p):
            sfx_tune_set_cells_per_cta(kind, p, cb)
            plan = Plan(ctx, mesh, deg, ["laplace", "mass"], nrhs=nrhs, precision=precision)
            x = torch.from_numpy(inputs.random_vector(plan.ndof * nrhs, 1, seed=1)).cuda()
            ys = [torch.empty_like(x) for _ in range(2)]
            res[cb] = _time(torch, lambda: plan.execute(x, ys), reps, flush)
            plan.close()
        best = min(res, key=res.get)
        sfx_tune_set_cells_per_cta(kind, p, best)
        out[p] = {"best": best, "ms": {str(k): round(v, 4) for k, v in res.items()}}
    return out


def apply(table):
    for kind, per in table.items():
        for p, rec in per.items():
            set_value(kind, int(p), int(rec["best"]))


def cache_dir():
    """Directory of the per-GPU tables: $SFX_AUTOTUNE_CACHE if set, else the
    package's build directory."""
    return os.environ.get("SFX_AUTOTUNE_CACHE") or _BUILD


def cache_path(gpu_name):
    safe = "".join(c if c.isalnum() else "_" for c in gpu_name)
    return os.path.join(cache_dir(), "autotune_%s.json" % safe)


def save(table, gpu_name):
    os.makedirs(cache_dir(), exist_ok=True)
    with open(cache_path(gpu_name), "w") as f:
        json.dump({"gpu": gpu_name, "table": table}, f, indent=1)


def load(gpu_name):
    path = cache_path(gpu_name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)["table"]


def ensure(ctx, gpu_name, degrees=range(1, 9), kinds=("fp64", "mixed", "mixed_stored"), **kw):
    """Apply the cached table for this GPU, tuning (and caching) only the
    (kind, degree) entries it lacks.  Later runs on the same machine then use
    identical launch shapes without tuning again."""
    table = load(gpu_name) or {}
    table = {k: {int(p): v for p, v in per.items()} for k, per in table.items()}
    apply(table)
    missing = [(k, p) for k in kinds for p in degrees
               if p not in table.get(k, {}) and not (k == "mixed_ws" and p < 3)]
    if missing:
        new = tune(ctx, degrees=sorted({p for _, p in missing}), kinds=sorted({k for k, _ in missing}), **kw)
        for k, per in new.items():
            for p, rec in per.items():
                table.setdefault(k, {})[p] = rec
        save(table, gpu_name)
        apply(table)
    return {k: {p: v for p, v in per.items() if p in degrees} for k, per in table.items() if k in kinds}


__all__ = ["tune", "apply", "save", "load", "ensure", "candidates", "cache_dir", "cache_path", "TUNE_KERNEL",
           "Context"]
