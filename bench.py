"""Benchmark: sum-factorised operator action on a 64^3 perturbed hexahedral mesh.

Workload (one "step"): the mass, Laplace and Helmholtz (k = 1) actions on
Q_p and DQ_p for every requested degree (default p = 1..8), (p+1)^3 Gauss
points, input vectors uniform[-1, 1) (seed 1), mesh interior vertices
perturbed by uniform(+-0.1 h) (seed 0).  Metric: DoFs/s = sum of global DoFs
of all actions in a step / step time (the paper's N/t, Sec. 4).

Output: detail lines first (one JSON object per section, tagged "detail":
per-case times, the other arms, the sampled error against the oracle, the
other workloads), then ONE compact headline JSON line, the last line of
stdout.  ``--impl reference`` times the FP64 CPU oracle (the reference arm)
on a bounded sample of cells of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (64, 64, 64)
FORMS = ("mass", "laplace", "helmholtz")
HELM = (1.0, -1.0, 0.0, 0.0)  # alpha * laplace + beta * mass, beta = -k^2, k = 1
# nominal GB300 FP64 pipe: 152 SMs x 2 FP64 operations (add, multiply or FMA) per
# clock x 2.07 GHz; as flops (FMA = 2) this is the 1.26 TFLOP/s nominal figure
FP64_PEAK_GOPS = 152 * 2 * 2.07
L2_FLUSH_BYTES = 256 << 20
HBM_GBS = 6788.3             # GB300 HBM bandwidth, measured by a STREAM-style copy (GB/s)
METRIC = "DoFs/s for sum-factorised action (mixed vs FP64, same GB300, stated error); % roofline"
# DRAM bytes (read + write) per cell of one colour launch, from the ncu captures of
# the 32^3, p = 8 cases (dram__bytes_read.sum + dram__bytes_write.sum of the first
# colour launch of the form / 4096 cells), keyed by kernel, family, degree and form;
# the full-size launch processes 8x the cells, and the traffic of these kernels grows
# in proportion (x, map, y and coordinates are per cell).  Only the kernels as they
# are now: a kernel without an entry reports traffic null.  (The FP64 kernel's first
# colour stores every dof it writes, so later colours read more of y.)
NCU_DRAM_BYTES_PER_CELL = {("k_action_scalar_fp64", "Q", 8, "laplace"): (66.470400e6 + 11.927552e6) / 4096,
                           ("k_action_scalar_mixed_ws", "Q", 8, "helmholtz"): (93.733120e6 + 3.786240e6) / 4096}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfx", choices=["sfx", "reference"])
    ap.add_argument("--degrees", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--families", default="Q,DQ")
    ap.add_argument("--precision", default="tf32x3,fp64,tf32x3:stored,fp64:stored",
                    help="comma list of arms; the first is the headline, the others are timed beside it. "
                         "':stored' arms apply the operator with geometric factors stored once per space "
                         "(their setup time is reported separately)")
    ap.add_argument("--dims", default="64,64,64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in cells-per-CTA instead of tuning them first (untimed)")
    ap.add_argument("--extras-only", default="",
                    help="comma list of extra workloads (names of the 'extras' keys) to measure alone, without "
                         "the sweep; prints their JSON")
    ap.add_argument("--no-oracle-err", action="store_true",
                    help="skip the sampled per-cell comparison of each arm against the oracle")
    ap.add_argument("--detail-file", default="",
                    help="also write the full result (every section) to this JSON file")
    ap.add_argument("--padaptive-dims", default="40,50,100",
                    help="box of the p-adaptive batch extra (the configuration's 200,000 cells by default)")
    ap.add_argument("--small-extras", action="store_true",
                    help="run the other workloads on meshes 1/8 the size per axis, first two degrees each "
                         "(exercises the full output path quickly)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements of the other configurations (structured elements, "
                         "p-adaptive batching, naive kernels, element matrices)")
    return ap.parse_args()


def cases(args):
    ps = [int(p) for p in args.degrees.split(",")]
    fams = args.families.split(",")
    return [(f, p, form) for p in ps for f in fams for form in FORMS]


def fp64_ops_per_cell(fam, p, form):
    """Algorithmic FP64 operations (an add, multiply or FMA each counts one: the
    FP64 pipe issues any of them at the same rate) of the FP64 sum-factorised
    action per cell, one RHS, q = n = p+1, as the kernel computes it:
    1D contractions n^4 FMAs each -- B (3 forward, 3 back; none for DQ) and the
    collocation derivative Dq (3 + 3, Laplace part); the Jacobian column tables
    (78 per (a, b) entry); per point for the Laplace part the adjugate rows (3
    cross products, 18), det J (3), the weight (1, +1 for Helmholtz), a two-step
    Newton reciprocal (4), the flux t R (R^T g) (21), and for the mass part
    w S u (3; 12 with det J when alone).  The scatter's adds run in L2
    (red.global.add.f64), off the FP64 pipe, and are not counted."""
    n = p + 1
    lap = form != "mass"
    mas = form != "laplace"
    ncontr = (0 if fam == "DQ" else 6) + (6 if lap else 0)
    pt = (47 + (1 if form == "helmholtz" else 0) if lap else 0) + ((3 if lap else 12) if mas else 0)
    return ncontr * n ** 4 + 78 * n ** 2 + pt * n ** 3


def probe_rates(sfx, torch, target_ms=20.0):
    """Throughput of the units the roofline divides by, measured in this run
    with the library's probe kernels (independent chains, 4 CTAs of 256
    threads per SM): DFMA and FFMA in G FMA/s (one FP64-pipe operation per
    DFMA), the mma.sync forms in TFLOP/s.  Each probe is calibrated to about
    target_ms and timed with CUDA events (median of 3)."""
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = 4 * nsm, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    out = {}
    for kind, scale, unit in (("dfma", 1e9, "G FMA/s"), ("ffma", 1e9, "G FMA/s"), ("mma_tf32", 1e12, "TFLOP/s"),
                              ("mma_bf16", 1e12, "TFLOP/s"), ("dmma", 1e12, "TFLOP/s")):
        iters = 16
        for _ in range(12):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sfx.sfx_probe_launch(kind, blocks, threads, iters, sink)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            if t >= 0.5 * target_ms or iters >= 1 << 26:
                break
            iters = int(iters * min(64.0, max(2.0, target_ms / max(t, 1e-3))))
        ts, ops = [], 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = sfx.sfx_probe_launch(kind, blocks, threads, iters, sink)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[kind] = {"rate": round(ops / (float(np.median(ts)) * 1e-3) / scale, 2), "unit": unit}
    return out


def arm_dtype(arm):
    """The arithmetic an arm computes in."""
    prec = arm.split(":")[0]
    if prec == "fp64":
        return "f64"
    return ("%s contractions (split operands, fp32 accumulate); f64 geometry, quadrature scaling and scatter"
            % prec)


def launches_per_action(fam):
    return 1 if fam == "DQ" else 8


# --small-extras: the other workloads on meshes 1/8 the size per axis and their
# first two degrees (a quick run of the full output path; not a measurement)
SMALL_EXTRAS = False
PADAPTIVE_DIMS = (40, 50, 100)


def _d(*dims):
    return tuple(max(2, v // 8) for v in dims) if SMALL_EXTRAS else tuple(dims)


def _ps(seq):
    seq = list(seq)
    return seq[:2] if SMALL_EXTRAS else seq


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 8:
                continue
            for name, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def reduce_max_ms(ms, ws, device="cuda"):
    """Max over ranks of a rank's timed interval (the slowest rank sets the
    job's time); identity on one rank."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(dofs_per_step, ws, ms_step):
    """Whole-job throughput: every rank processes dofs_per_step per step
    (replicas, weak scaling)."""
    return dofs_per_step * ws / (ms_step * 1e-3)


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_sample(orc, inputs, wl_cases, dims, X, seconds, rng_seed=5, xs=None):
    """Time the oracle's per-cell assembly on seeded samples of cells per case
    and extrapolate to the whole mesh.  Each call of the oracle tabulates its
    dense 3D tables first, a fixed cost per call: a one-cell call measures it,
    then a sample grown until its per-cell part fills the case's share of the
    time budget gives the per-cell cost; full-mesh time per case = fixed cost
    + per-cell cost x cells.  Returns (DoFs/s, desc, threads)."""
    ncell = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(rng_seed)
    per_case = seconds / max(1, len(wl_cases))
    tot_dofs, tot_time, sampled = 0, 0.0, 0
    xs = {} if xs is None else xs  # input vectors by space, reusable across calls
    for fam, p, form in wl_cases:
        ndof, nloc = orc.space_size(fam, p, dims)
        key = (fam, p)
        if key not in xs:
            xs[key] = inputs.random_vector(ndof, 1, seed=1)
        prm = HELM if form == "helmholtz" else None

        def timed(m):
            cells = rng.choice(ncell, m, replace=False)
            t0 = time.perf_counter()
            orc.cell_vectors(fam, form, p, dims, X, xs[key], cells, params=prm)
            return time.perf_counter() - t0

        t1 = timed(1)
        m = 8
        while True:
            t = timed(m)
            sampled += m
            if t - t1 >= 0.5 * per_case or m >= ncell:
                break
            m = min(ncell, max(2 * m, int(m * 0.6 * per_case / max(t - t1, 1e-4))))
        per_cell = max(t - t1, 1e-9) / (m - 1)
        fixed = max(0.0, t1 - per_cell)
        tot_dofs += ndof
        tot_time += fixed + per_cell * ncell
        sampled += 1
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = ("oracle per-cell assembly timed on %d seeded cells in total across %d cases; per case a one-cell call "
            "gives the call's fixed cost (dense tabulation) and a sample grown to ~%.2f s of per-cell work gives the "
            "per-cell cost; full-mesh time = fixed + per-cell cost x all %d cells; scatter not timed"
            % (sampled, len(wl_cases), 0.5 * per_case, ncell))
    return tot_dofs / tot_time, desc, threads


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle as orc
    from paper_1711_02473_gb300 import inputs
    dims = tuple(int(v) for v in args.dims.split(","))
    X = inputs.box_coords(*dims, perturb=0.1, seed=0)
    wl = cases(args)
    orc.lib()
    secs = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    xs = {}  # seeded input vectors, generated once (before the timed steps)
    for fam, p, _ in wl:
        if (fam, p) not in xs:
            xs[(fam, p)] = inputs.random_vector(orc.space_size(fam, p, dims)[0], 1, seed=1)
    for _ in range(args.warmup):
        cpu_sample(orc, inputs, wl[:1], dims, X, 0.2, xs=xs)
    vals, t0 = [], time.perf_counter()
    for s in range(args.steps):
        v, desc, thr = cpu_sample(orc, inputs, wl, dims, X, secs, rng_seed=100 + s, xs=xs)
        vals.append(v)
    wall = time.perf_counter() - t0
    val = float(np.median(vals))
    out = {"impl": "reference", "metric": METRIC,
           "value": val, "unit": "DoF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": wall / max(1, args.steps) * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "operator-action sweep: mass/laplace/helmholtz on Q_p and DQ_p, "
                                  "p=%s, %dx%dx%d perturbed hex mesh, (p+1)^3 Gauss points" % (args.degrees, *dims),
                      "precision": "fp64 (CPU oracle, naive quadrature)", "families": args.families,
                      "degrees": args.degrees},
           "cpu_baseline": {"value": val, "unit": "DoF/s", "cores": thr, "kind": "oracle", "sample": desc},
           "e2e": {"value": val, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_setup(args)
    global SMALL_EXTRAS
    SMALL_EXTRAS = args.small_extras
    global PADAPTIVE_DIMS
    PADAPTIVE_DIMS = tuple(int(v) for v in args.padaptive_dims.split(","))
    import torch
    import paper_1711_02473_gb300 as sfx
    from paper_1711_02473_gb300 import inputs
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sfx.build()
    ctx = sfx.Context(local)
    if args.extras_only:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        only = set(args.extras_only.split(","))
        unknown = only - set(EXTRAS)
        if unknown:
            raise SystemExit("unknown extras: %s (known: %s)" % (sorted(unknown), ", ".join(EXTRAS)))
        print(json.dumps(run_extras(sfx, torch, ctx, inputs, flush, torch.cuda.current_stream(), only=only)),
              flush=True)
        return
    dims = tuple(int(v) for v in args.dims.split(","))
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    wl = cases(args)
    spaces, xs, ys = {}, {}, {}
    for fam, p, form in wl:
        if (fam, p) not in spaces:
            sp = sfx.Space(mesh, fam, p)
            spaces[(fam, p)] = sp
            xs[(fam, p)] = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
            ys[(fam, p)] = torch.empty_like(xs[(fam, p)])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    precs = args.precision.split(",")
    tuning = None
    if not args.no_autotune:
        from paper_1711_02473_gb300 import autotune
        kinds = sorted({("fp64" if pr.startswith("fp64") else ("mixed_stored" if pr.endswith(":stored") else "mixed"))
                        for pr in precs} - {"fp64"} | ({"fp64"} if any(pr.startswith("fp64") for pr in precs) else set()))
        if "mixed" in kinds:
            kinds = kinds + ["mixed_ws"]  # after "mixed": the warp-specialised kernel or the one-role one, per degree
        if not args.no_extras:
            # the other workloads' kernels: tiles of the p-adaptive batch (config 5), cells per CTA of the
            # H(div)/H(curl) and hyperelastic kernels (config 3 and the linearised operator)
            kinds = kinds + ["batched", "batched_mixed", "hdivcurl", "elastic", "linearised", "linearised_mixed",
                             "hdivcurl_mixed"]
        degrees = sorted({p for _, p, _ in wl})
        tuning = autotune.ensure(ctx, torch.cuda.get_device_name(local), degrees=degrees, kinds=kinds)
    probes = probe_rates(sfx, torch)
    arms = {pr: time_arm(args, sfx, torch, ctx, spaces, xs, ys, wl, pr, flush, stream, ws, local)
            for pr in precs}
    prec = precs[0]
    head = arms[prec]
    ms_step = head["ms_step"]
    dofs_step = sum(spaces[(f, p)].ndof for f, p, _ in wl)
    value = job_value(dofs_step, ws, ms_step)
    # error of each arm against the FP64 arm, per case (the FP64 path matches
    # the oracle to <= 1e-12 in the GPU tests)
    if "fp64" in arms and prec != "fp64":
        for c_head, c64 in zip(head["per_case"], arms["fp64"]["per_case"]):
            c_head["rel_err_vs_fp64"] = rel_err_case(sfx, torch, ctx, spaces, xs, c_head, prec.split(":")[0])
    mesh_cells = dims[0] * dims[1] * dims[2]
    dom = max(head["per_case"], key=lambda c: c["ms"])
    fam, p, form = dom["family"], dom["p"], dom["form"]
    if prec == "fp64":
        ops = fp64_ops_per_cell(fam, p, form) * mesh_cells
        achieved = ops / (dom["ms"] * 1e-3) / 1e9
        tpc = NCU_DRAM_BYTES_PER_CELL.get(("k_action_scalar_fp64", fam, p, form))
        roofline = {"bound": "alu", "kernel": "k_action_scalar_fp64 %s p=%d %s" % (fam, p, form),
                    "achieved": round(achieved, 2), "peak": round(FP64_PEAK_GOPS, 1), "unit": "G FP64 op/s",
                    "frac": round(achieved / FP64_PEAK_GOPS, 4),
                    "dfma_probe": probes["dfma"]["rate"],
                    "frac_of_dfma_probe": round(achieved / probes["dfma"]["rate"], 4),
                    "traffic": round(tpc * mesh_cells / launches_per_action(fam)) if tpc else None,
                    "note": "algorithmic FP64 operations per action (all colour launches; add, multiply or FMA "
                            "= 1) / event time; peak = 152 SMs x 2 FP64 op/clk x 2.07 GHz, of nominal"}
    else:
        ops = mixed_fp64_ops_per_cell(fam, p, form) * mesh_cells
        achieved = ops / (dom["ms"] * 1e-3) / 1e9
        # which kernel ran the dominant case: the warp-specialised one (Laplace part, geometry in the
        # kernel, switched on for this degree) or the one-role one
        kname = ("k_action_scalar_mixed_ws" if ":" not in prec and form != "mass" and p >= 3
                 and sfx.sfx_tune_get_warp_specialised(p) else "k_action_scalar_mixed")
        tpc = NCU_DRAM_BYTES_PER_CELL.get((kname, fam, p, form)) if ":" not in prec else None
        roofline = {"bound": "alu", "kernel": "%s %s p=%d %s %s" % (kname, fam, p, form, prec),
                    "achieved": round(achieved, 2), "peak": round(FP64_PEAK_GOPS, 1), "unit": "G FP64 op/s",
                    "frac": round(achieved / FP64_PEAK_GOPS, 4),
                    "dfma_probe": probes["dfma"]["rate"],
                    "frac_of_dfma_probe": round(achieved / probes["dfma"]["rate"], 4),
                    "traffic": round(tpc * mesh_cells / launches_per_action(fam)) if tpc else None,
                    "note": "binding resource = FP64 pipe (adjugate rows, det J, w/S and the factor scaling per "
                            "point, the FP64 scatter; the contractions run on the tensor cores); achieved = "
                            "those algorithmic FP64 operations / event time, peak = 152 SMs x 2 FP64 op/clk x "
                            "2.07 GHz, of nominal; traffic = DRAM bytes per colour launch, scaled from a 32^3 "
                            "capture"}

    out = {"metric": METRIC, "value": value, "unit": "DoF/s",
           "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": arm_dtype(prec),
           "data": "synthetic",
           "config": {"workload": "operator-action sweep: mass/laplace/helmholtz on Q_p and DQ_p, p=%s, "
                                  "%dx%dx%d perturbed hex mesh, (p+1)^3 Gauss points" % (args.degrees, *dims),
                      "precision": prec, "families": args.families, "degrees": args.degrees,
                      "l2": "flushed between cases (256 MiB write)", "parallelism": "replicas" if ws > 1 else "1 GPU"},
           # kernel launches of the headline arm's timed steps (one per colour pass: 8 per Q_p action,
           # 1 per DQ_p action); the other arms are timed in their own regions
           "gpu_launches": sum(launches_per_action(f) for f, _, _ in wl) * args.steps,
           "clocks": head["clocks"], "roofline": roofline, "per_case": head["per_case"],
           "probes": probes,
           "autotune": ({k: {str(p): v["best"] for p, v in per.items()} for k, per in tuning.items()}
                        if tuning else None),
           "arms": {pr: {"value": dofs_step * ws / (arms[pr]["ms_step"] * 1e-3), "ms_per_step": arms[pr]["ms_step"],
                         "clocks": arms[pr]["clocks"], "speedup_vs_fp64": (arms["fp64"]["ms_step"] / arms[pr]["ms_step"]
                                                                           if "fp64" in arms else None),
                         **({"geometry_setup_ms": arms[pr]["geometry_setup_ms"]} if "geometry_setup_ms" in arms[pr]
                            else {})} for pr in precs}}
    for pr in precs[1:]:
        out["arms"][pr]["per_case"] = arms[pr]["per_case"]
    if "fp64" in arms and prec != "fp64":
        out["speedup_vs_fp64"] = arms["fp64"]["ms_step"] / ms_step

    if not args.no_e2e:
        out["e2e"] = e2e(args, sfx, torch, ctx, spaces, wl, prec, stream)
    if rank == 0 and not args.no_oracle_err:
        X = mesh.coords()
        out["err_vs_oracle"] = oracle_err_sample(sfx, torch, ctx, spaces, xs, wl, precs, dims, X)
    if not args.no_extras and ws == 1:
        del spaces, xs, ys
        torch.cuda.empty_cache()
        out["extras"] = run_extras(sfx, torch, ctx, inputs, flush, stream)
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as orc
        X = mesh.coords()
        v, desc, thr = cpu_sample(orc, inputs, wl, dims, X, args.cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": "DoF/s", "cores": thr, "kind": "oracle", "sample": desc}
    if rank == 0:
        emit(out, args.detail_file)
    if ws > 1:
        torch.distributed.destroy_process_group()


def headline(out):
    """The compact JSON line printed last (under 2,000 characters): the
    contract's keys, the headline arm's roofline, the FP64 arm beside it with
    the speed-up, the measured error against the oracle, the end-to-end rate
    and the CPU oracle's rate.  Everything else goes on the detail lines."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks")
    h = {k: out[k] for k in keep if k in out}
    rf = dict(out["roofline"])
    rf.pop("note", None)
    h["roofline"] = rf
    arms = out.get("arms", {})
    if "fp64" in arms and out["config"]["precision"] != "fp64":
        h["fp64_value"] = arms["fp64"]["value"]
        h["speedup_vs_fp64"] = round(out.get("speedup_vs_fp64", 0.0), 4)
    ev = out.get("err_vs_oracle")
    if ev:
        h["max_rel_err_vs_oracle"] = {arm: ev["max"][arm] for arm in ev["max"]}
        h["err_sample"] = ev["sample"]
    if "e2e" in out:
        h["e2e"] = {k: out["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
    if "cpu_baseline" in out:
        cb = dict(out["cpu_baseline"])
        cb["sample"] = cb["sample"].split(";")[0]
        h["cpu_baseline"] = cb
    h["detail"] = "per-case times, the other arms and the other workloads are on the preceding stdout lines"
    return h


def emit(out, detail_file=None):
    """Detail lines first (one JSON object per section, each tagged
    "detail"), then the compact headline as the last line of stdout."""
    sections = {"per_case": out.get("per_case"), "arms": out.get("arms"), "autotune": out.get("autotune"),
                "probes": out.get("probes"),
                "err_vs_oracle": out.get("err_vs_oracle"), "roofline_note": out.get("roofline", {}).get("note")}
    for name, fn in (out.get("extras") or {}).items():
        sections["extras." + name] = fn
    for name, val in sections.items():
        if val is not None:
            print(json.dumps({"detail": name, "data": val}), flush=True)
    if detail_file:
        with open(detail_file, "w") as f:
            json.dump(out, f)
    line = json.dumps(headline(out))
    print(line, flush=True)


def oracle_err_sample(sfx, torch, ctx, spaces, xs, wl, precs, dims, X, nsample=8, seed=11):
    """Normwise relative error of each arm's per-cell vectors b^K against the
    oracle's, on a seeded sample of cells per case (the first and the last cell
    of the mesh plus nsample - 2 drawn ones): max |b - b_ref| / max |b_ref|
    over the sample.  The stored-factor arms apply the same contractions as
    their plain arm and are not sampled separately."""
    import oracle as orc
    ncell = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(seed)
    arms = [a for a in precs if ":" not in a]
    rows, mx = [], {a: 0.0 for a in arms}
    xh = {}
    for fam, p, form in wl:
        key = (fam, p)
        if key not in xh:
            xh[key] = xs[key].cpu().numpy()
        cells = np.unique(np.concatenate([[0, ncell - 1], rng.choice(ncell, nsample - 2, replace=False)]))
        prm = HELM if form == "helmholtz" else None
        ref = orc.cell_vectors(fam, form, p, dims, X, xh[key], cells, params=prm)
        cd = torch.from_numpy(cells.astype(np.int64)).cuda()
        sp = spaces[key]
        row = {"family": fam, "p": p, "form": form}
        for a in arms:
            b = torch.empty(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
            sfx.sfx_assemble_cell_vectors(ctx, form, sp, xs[key], cd, b, precision=a, params=prm)
            e = float(np.abs(b.cpu().numpy().reshape(ref.shape) - ref).max() / np.abs(ref).max())
            row[a] = e
            mx[a] = max(mx[a], e)
        rows.append(row)
    if ctx.sync_status() != 0:
        raise RuntimeError("device status flagged while sampling cell vectors")
    return {"per_case": rows, "max": mx,
            "sample": "%d cells per case (first, last, %d seeded), per-cell vectors vs the FP64 oracle, "
                      "max|b-b_ref|/max|b_ref|" % (nsample, nsample - 2)}


def mixed_fp64_ops_per_cell(fam, p, form):
    """FP64 operations per cell left in the split-precision action (the
    contractions run on the tensor cores, the flux in FP32).  n >= 4: staged
    adjugate-row tables per cell -- edge vectors (126), 1D vectors (108 per
    point, 42 for mass alone), 2D tables (22 per (a, b) entry, 10 for mass) --
    then per point the rows (9), det J (3), the weight (1), a one-step Newton
    reciprocal (2), t = w/S (1, +1 for Helmholtz) and the scaling of R^T g by
    t (3; the flux R (t R^T g) runs in FP32 otherwise); mass adds w S (2), or
    9 with det J when alone.  n <= 3: the Jacobian column tables (78 per
    entry) and cross products at the point (29 / 13).  The scatter's adds
    run in L2 (red.global.add.f64), off the FP64 pipe, and are not counted."""
    n = p + 1
    lap = form != "mass"
    mas = form != "laplace"
    helm = 1 if form == "helmholtz" else 0
    if n >= 4:
        tables = 126 + (108 if lap else 42) * n + (22 if lap else 10) * n ** 2
        pt = (19 + helm if lap else 0) + ((2 if lap else 9) if mas else 0)
    else:
        tables = 78 * n ** 2
        pt = (29 + helm if lap else 0) + ((2 if lap else 13) if mas else 0)
    return tables + pt * n ** 3


def time_arm(args, sfx, torch, ctx, spaces, xs, ys, wl, arm, flush, stream, ws, local):
    prec, _, mode = arm.partition(":")
    stored = mode == "stored"
    qd, setup_ms = {}, 0.0
    if stored:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for key, sp in spaces.items():
            qd[key] = sfx.QData(ctx, sp, "fp64" if prec == "fp64" else "fp32", stream=stream)
        setup_ms = (time.perf_counter() - t0) * 1e3

    def run_case(fam, p, form):
        prm = HELM if form == "helmholtz" else None
        if stored:
            sfx.sfx_assemble_action_stored(ctx, form, spaces[(fam, p)], qd[(fam, p)], xs[(fam, p)], ys[(fam, p)],
                                           precision=prec, params=prm, stream=stream)
        else:
            sfx.sfx_assemble_action(ctx, form, spaces[(fam, p)], xs[(fam, p)], ys[(fam, p)], precision=prec,
                                    params=prm, stream=stream)

    ev = {c: [] for c in wl}

    def step(record):
        for c in wl:
            flush.fill_(1.0)  # evict L2 between cases
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run_case(*c)
                e1.record(stream)
                ev[c].append((e0, e1))
            else:
                run_case(*c)

    for _ in range(max(3, args.warmup)):
        step(False)
    torch.cuda.synchronize()
    if ctx.sync_status() != 0:
        raise RuntimeError("device status flagged during warm-up")
    clk = ClockSampler(local)
    clk.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms_total = reduce_max_ms(t0.elapsed_time(t1), ws)
    ncell = next(iter(spaces.values())).ncell
    per_case = []
    for c in wl:
        t = float(np.median([a.elapsed_time(b) for a, b in ev[c]]))
        fam, p, form = c
        nd = spaces[(fam, p)].ndof
        ops = (fp64_ops_per_cell if prec == "fp64" else mixed_fp64_ops_per_cell)(fam, p, form)
        per_case.append({"family": fam, "p": p, "form": form, "ms": round(t, 4), "dofs_per_s": nd / (t * 1e-3),
                         "gops_fp64_alg": ops * ncell / (t * 1e-3) / 1e9 if not stored else None})
    for q in qd.values():
        q.close()
    out = {"ms_step": ms_total / args.steps, "per_case": per_case, "clocks": clocks}
    if stored:
        out["geometry_setup_ms"] = setup_ms
    return out


def rel_err_case(sfx, torch, ctx, spaces, xs, case, prec):
    """Normwise (inf) relative error of the `prec` action against the FP64 one."""
    fam, p, form = case["family"], case["p"], case["form"]
    sp, x = spaces[(fam, p)], xs[(fam, p)]
    prm = HELM if form == "helmholtz" else None
    y64, ym = torch.empty_like(x), torch.empty_like(x)
    sfx.sfx_assemble_action(ctx, form, sp, x, y64, params=prm)
    sfx.sfx_assemble_action(ctx, form, sp, x, ym, precision=prec, params=prm)
    return float((ym - y64).abs().max() / y64.abs().max())


def _time(torch, stream, flush, fn, reps=3, warm=2):
    """median CUDA-event time (ms) of fn(), L2 flushed before every run"""
    for _ in range(warm):
        flush.fill_(1.0)
        fn()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def dq_multi_ops(p, form, nrhs):
    """FP64 operations (add, multiply or FMA = 1) of the DQ action for one
    cell and nrhs right-hand sides in the persistent kernel: the Jacobian
    column tables (78 per entry) and the staged factors once per cell (Laplace:
    rows 18, det J 3, weight and w/S 2, reciprocal 4, six dot products 18 and
    their scaling 6; mass: w S 2, or 11 with det J when alone), then per RHS
    the Dq contractions (6 n^4, Laplace), the flux (9 per point, Laplace;
    1 for mass) and the scatter (1 per dof)."""
    n = p + 1
    lap = form != "mass"
    geo = 78 * n ** 2 + ((51 + 2) if lap else 11) * n ** 3
    per_rhs = (6 * n ** 4 if lap else 0) + ((9 if lap else 1) + 1) * n ** 3
    return geo + per_rhs * nrhs


def matrix_flops(p, fam):
    """FP64 flops of the sum-factorised element matrix of the scalar Laplace
    form per cell: stages q1 (9 terms, n^5), q2 (9 terms, n^6), q3 (4 groups,
    n^7), 3 flops per multiply-add with a table product."""
    n = p + 1
    return 3 * (9 * n ** 5 + 9 * n ** 6 + 4 * n ** 7)


def extra_structured(sfx, torch, ctx, inputs, flush, stream):
    """NCF mass + div-div and NCE curl-curl on 32^3 (p = 1..6), neo-Hookean
    residual on 48^3 (p = 2..6), FP64."""
    rows = []
    for fam, form, dims, ps in [("NCF", "ncf_mass_divdiv", _d(32, 32, 32), _ps(range(1, 7))),
                                ("NCE", "nce_curlcurl", _d(32, 32, 32), _ps(range(1, 7))),
                                ("VQ", "neohooke", _d(48, 48, 48), _ps(range(2, 7)))]:
        mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
        for p in ps:
            sp = sfx.Space(mesh, fam, p)
            x = (inputs.displacement(sp.ndof, p, dims[0], seed=1) if fam == "VQ"
                 else inputs.random_vector(sp.ndof, 1, seed=1))
            xd = torch.from_numpy(x).cuda()
            yd = torch.empty_like(xd)
            t = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, form, sp, xd, yd, stream=stream))
            rows.append({"family": fam, "form": form, "p": p, "mesh": "%dx%dx%d" % dims, "ndof": sp.ndof,
                         "ms": round(t, 4), "dofs_per_s": sp.ndof / (t * 1e-3)})
            del xd, yd, sp
        del mesh
    return {"rows": rows, "device_status": ctx.sync_status()}


def extra_hdivcurl_mixed(sfx, torch, ctx, inputs, flush, stream):
    """NCF_p mass + div-div and NCE_p curl-curl on 32^3, p = 1..6 (the
    structured-element configuration): FP64, TF32x3 and BF16x3 (split-precision
    contractions on the tensor cores, FP64 geometry and scaling), each with its
    speed-up over FP64 and its error against the oracle on six sampled cells
    (first, last and four seeded) and against the FP64 GPU action."""
    import oracle as orc
    rows = []
    dims = _d(32, 32, 32)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    X = mesh.coords()
    rng = np.random.default_rng(19)
    for fam, form in (("NCF", "ncf_mass_divdiv"), ("NCE", "nce_curlcurl")):
        for p in _ps(range(1, 7)):
            sp = sfx.Space(mesh, fam, p)
            x = inputs.random_vector(sp.ndof, 1, seed=1)
            xd = torch.from_numpy(x).cuda()
            cells = np.unique(np.concatenate([[0, sp.ncell - 1], rng.choice(sp.ncell, 4, replace=False)]))
            ref = orc.cell_vectors(fam, form, p, dims, X, x, cells)
            cd = torch.from_numpy(cells.astype(np.int64)).cuda()
            row = {"family": fam, "form": form, "p": p, "mesh": "%dx%dx%d" % dims, "ndof": sp.ndof}
            ys = {}
            for prec in ("fp64", "tf32x3", "bf16x3"):
                ys[prec] = torch.empty_like(xd)
                t = _time(torch, stream, flush,
                          lambda: sfx.sfx_assemble_action(ctx, form, sp, xd, ys[prec], precision=prec, stream=stream))
                row[prec + "_ms"] = round(t, 4)
                row[prec + "_dofs_per_s"] = sp.ndof / (t * 1e-3)
                b = torch.empty(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
                sfx.sfx_assemble_cell_vectors(ctx, form, sp, xd, cd, b, precision=prec)
                row[prec + "_rel_err_vs_oracle_sampled"] = float(np.abs(b.cpu().numpy().reshape(ref.shape) - ref).max()
                                                                 / np.abs(ref).max())
                if prec != "fp64":
                    row[prec + "_speedup_vs_fp64"] = row["fp64_ms"] / row[prec + "_ms"]
                    row[prec + "_rel_err_vs_fp64"] = float((ys[prec] - ys["fp64"]).abs().max()
                                                           / ys["fp64"].abs().max())
            rows.append(row)
            del xd, ys, sp
    del mesh
    return {"rows": rows, "device_status": ctx.sync_status()}


def extra_linearised(sfx, torch, ctx, inputs, flush, stream):
    """Linearised hyperelastic operator K(u) du (the Jacobian of the residual;
    the operator whose matrices Sec. 4.1 assembles and whose action Sec. 4.2 times), vector Q_p on 48^3, p = 2..6,
    state = the residual's displacement: FP64 and TF32x3 (split-precision
    contractions), the speed-up, the error against the FP64 GPU action and
    against the oracle on six sampled cells (first, last and four seeded)."""
    rows = []
    dims = _d(48, 48, 48)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    import oracle as orc
    X = mesh.coords()
    rng = np.random.default_rng(17)
    for form in ("svk", "neohooke"):
        for p in _ps(range(2, 7)):
            sp = sfx.Space(mesh, "VQ", p)
            u = inputs.displacement(sp.ndof, p, dims[0], seed=1)
            du = inputs.random_vector(sp.ndof, 1, seed=2)
            ud, dd = torch.from_numpy(u).cuda(), torch.from_numpy(du).cuda()
            row = {"family": "VQ", "form": form + "_linearised", "p": p, "mesh": "%dx%dx%d" % dims, "ndof": sp.ndof}
            ys = {}
            cells = np.unique(np.concatenate([[0, sp.ncell - 1], rng.choice(sp.ncell, 4, replace=False)]))
            ref = orc.linearised_cell_vectors(form, p, dims, X, u, du, cells)
            cd = torch.from_numpy(cells.astype(np.int64)).cuda()
            for prec in ("fp64", "tf32x3"):
                ys[prec] = torch.empty_like(dd)
                t = _time(torch, stream, flush,
                          lambda: sfx.sfx_assemble_linearised_action(ctx, form, sp, ud, dd, ys[prec], precision=prec,
                                                                     stream=stream))
                row[prec + "_ms"] = round(t, 4)
                row[prec + "_dofs_per_s"] = sp.ndof / (t * 1e-3)
                b = torch.empty(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
                sfx.sfx_assemble_linearised_cell_vectors(ctx, form, sp, ud, dd, cd, b, precision=prec)
                row[prec + "_rel_err_vs_oracle_sampled"] = float(np.abs(b.cpu().numpy().reshape(ref.shape) - ref).max()
                                                                 / np.abs(ref).max())
            row["tf32x3_speedup_vs_fp64"] = row["fp64_ms"] / row["tf32x3_ms"]
            row["tf32x3_rel_err_vs_fp64"] = float((ys["tf32x3"] - ys["fp64"]).abs().max() / ys["fp64"].abs().max())
            rows.append(row)
            del ud, dd, ys, sp
    del mesh
    return {"rows": rows, "device_status": ctx.sync_status()}


def extra_padaptive(sfx, torch, ctx, inputs, flush, stream):
    """p-adaptive batching: 200,000 cells (40x50x100), p in 1..8 with
    P(p) ~ 1/p, DQ_p per cell, Laplace + mass on 16 RHS (seeds 0..15): one
    graph-captured persistent launch vs one launch per (form, degree, RHS), in
    FP64 and with the TF32x3 tile body."""
    dims = _d(*PADAPTIVE_DIMS)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    deg = inputs.padaptive_degrees(int(np.prod(dims)), 8, seed=2)
    forms, R = ["laplace", "mass"], 16
    plan = sfx.Plan(ctx, mesh, deg, forms, nrhs=R)
    x = np.stack([inputs.random_vector(plan.ndof, 1, seed=r) for r in range(R)], axis=1)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(-1)
    del x
    ys = [torch.empty_like(xd) for _ in forms]
    tg = _time(torch, stream, flush, lambda: plan.execute(xd, ys, mode="graph", stream=stream))
    tl = _time(torch, stream, flush, lambda: plan.execute(xd, ys, mode="per_launch", stream=stream), reps=2, warm=1)
    work = plan.ndof * R * len(forms)
    ndeg = len(np.unique(deg))
    fl = sum(dq_multi_ops(int(p), f, R) * int((deg == p).sum()) for p in np.unique(deg) for f in forms)
    out = {
        "cells": int(np.prod(dims)), "ndof": int(plan.ndof), "nrhs": R, "forms": forms, "tiles": int(plan.ntiles),
        "graph_ms": round(tg, 3), "per_launch_ms": round(tl, 3),
        "graph_dofs_per_s": work / (tg * 1e-3), "per_launch_dofs_per_s": work / (tl * 1e-3),
        "speedup_graph_vs_per_launch": tl / tg, "launches_graph": 1, "launches_per_launch": ndeg * R * len(forms),
        "roofline": {"bound": "alu", "achieved": round(fl / (tg * 1e-3) / 1e9, 2), "peak": round(FP64_PEAK_GOPS, 1),
                     "unit": "G FP64 op/s", "frac": round(fl / (tg * 1e-3) / 1e9 / FP64_PEAK_GOPS, 4)},
        "tile_cells_tuned": {str(p): sfx.sfx_tune_get_cells_per_cta("batched", p) for p in range(1, 9)}}
    # the same batch with the split-precision tile body (TF32x3): one graph
    # launch, its speed-up over the FP64 batch and its error against it
    ref = [y.clone() for y in ys]
    plan.close()
    planm = sfx.Plan(ctx, mesh, deg, forms, nrhs=R, precision="tf32x3")
    tm = _time(torch, stream, flush, lambda: planm.execute(xd, ys, mode="graph", stream=stream))
    tml = _time(torch, stream, flush, lambda: planm.execute(xd, ys, mode="per_launch", stream=stream), reps=2, warm=1)
    planm.execute(xd, ys, mode="graph", stream=stream)
    torch.cuda.synchronize()
    out["tf32x3"] = {"graph_ms": round(tm, 3), "per_launch_ms": round(tml, 3), "graph_dofs_per_s": work / (tm * 1e-3),
                     "speedup_vs_fp64_graph": tg / tm, "launches_per_launch": ndeg * len(forms),
                     "rel_err_vs_fp64": max(float((y - r).abs().max() / r.abs().max()) for y, r in zip(ys, ref)),
                     "tile_cells_tuned": {str(p): sfx.sfx_tune_get_cells_per_cta("batched_mixed", p)
                                          for p in range(1, 9)}}
    planm.close()
    del xd, ys, ref, mesh
    return out


def extra_naive(sfx, torch, ctx, inputs, flush, stream):
    """Naive (un-factorised) vs sum-factorised action, Q_p Laplace, 32^3."""
    mesh = sfx.Mesh.box(ctx, *_d(32, 32, 32), perturb=0.1, seed=0)
    rows = []
    for p in _ps(range(1, 9)):
        sp = sfx.Space(mesh, "Q", p)
        xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        yd = torch.empty_like(xd)
        ts = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd, stream=stream))
        tn = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd, algo="naive",
                                                                         stream=stream), reps=2, warm=1)
        rows.append({"p": p, "sumfact_ms": round(ts, 4), "naive_ms": round(tn, 4), "speedup": tn / ts,
                     "sumfact_dofs_per_s": sp.ndof / (ts * 1e-3), "naive_dofs_per_s": sp.ndof / (tn * 1e-3)})
        del xd, yd, sp
    return rows


def extra_weighted(sfx, torch, ctx, inputs, flush, stream):
    """Weighted Laplace int kappa grad u . grad v (Sec. 1.1, Eq.
    weighted_laplace), FP64, Q_p on 64^3, beside the plain Laplace action."""
    mesh = sfx.Mesh.box(ctx, *_d(64, 64, 64), perturb=0.1, seed=0)
    rows = []
    for p in _ps(range(1, 9)):
        sp = sfx.Space(mesh, "Q", p)
        xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        kd = 1.0 + 0.5 * torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=7)).cuda()
        yd = torch.empty_like(xd)
        tw = _time(torch, stream, flush, lambda: sfx.sfx_assemble_weighted_action(ctx, sp, kd, xd, yd, stream=stream))
        tl = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd, stream=stream))
        rows.append({"p": p, "ndof": sp.ndof, "weighted_ms": round(tw, 4), "laplace_ms": round(tl, 4),
                     "weighted_dofs_per_s": sp.ndof / (tw * 1e-3), "overhead": tw / tl})
        del xd, kd, yd, sp
    return rows


def extra_matrices(sfx, torch, ctx, inputs, flush, stream):
    """Element matrices (FP64): Q_p Laplace p = 1..8 and NCF/NCE p = 1..5 on
    32^3, on a chunk of cells sized to ~1 GB of output; sum-factorised and,
    p <= 4, naive."""
    mesh = sfx.Mesh.box(ctx, *_d(32, 32, 32), perturb=0.1, seed=0)
    rows = []
    for fam, form, ps in [("Q", "laplace", _ps(range(1, 9))), ("NCF", "ncf_mass_divdiv", _ps(range(1, 6))),
                          ("NCE", "nce_curlcurl", _ps(range(1, 6)))]:
        for p in ps:
            sp = sfx.Space(mesh, fam, p)
            nc = int(min(sp.ncell, max(8, (1 << 30) // (sp.nloc * sp.nloc * 8))))
            A = torch.empty(nc * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
            t = _time(torch, stream, flush,
                      lambda: sfx.sfx_assemble_cell_matrices(ctx, form, sp, 0, nc, A, stream=stream), reps=2, warm=1)
            row = {"family": fam, "form": form, "p": p, "cells": nc, "nloc": sp.nloc, "ms": round(t, 4),
                   "cells_per_s": nc / (t * 1e-3),
                   "dofs_per_s_paper": sp.ndof * (nc / sp.ncell) / (t * 1e-3),
                   "gb_per_s_written": nc * sp.nloc ** 2 * 8 / (t * 1e-3) / 1e9}
            if fam == "Q":
                row["gflops_fp64"] = matrix_flops(p, fam) * nc / (t * 1e-3) / 1e9
            if p <= 4:
                tn = _time(torch, stream, flush,
                           lambda: sfx.sfx_assemble_cell_matrices(ctx, form, sp, 0, nc, A, algo="naive",
                                                                  stream=stream), reps=1, warm=1)
                row["naive_ms"] = round(tn, 4)
                row["speedup_vs_naive"] = tn / t
            rows.append(row)
            del A, sp
            torch.cuda.empty_cache()
    return rows


def extra_tangent(sfx, torch, ctx, inputs, flush, stream):
    """Tangent (element) matrices of the hyperelastic residual, vector Q_p on
    the 48^3 hyperelastic mesh, p = 1..6, both laws, state = the residual's
    displacement, FP64, on a chunk of cells sized to ~1 GB of output."""
    dims = _d(48, 48, 48)
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    rows = []
    for form in ("svk", "neohooke"):
        for p in _ps(range(1, 7)):
            sp = sfx.Space(mesh, "VQ", p)
            ud = torch.from_numpy(inputs.displacement(sp.ndof, p, dims[0], seed=1)).cuda()
            nc = int(min(sp.ncell, max(8, (1 << 30) // (sp.nloc * sp.nloc * 8))))
            A = torch.empty(nc * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
            t = _time(torch, stream, flush,
                      lambda: sfx.sfx_assemble_linearised_cell_matrices(ctx, form, sp, ud, 0, nc, A, stream=stream),
                      reps=2, warm=1)
            rows.append({"family": "VQ", "form": form + "_tangent", "p": p, "cells": nc, "nloc": sp.nloc,
                         "ms": round(t, 4), "cells_per_s": nc / (t * 1e-3),
                         "dofs_per_s_paper": sp.ndof * (nc / sp.ncell) / (t * 1e-3),
                         "gb_per_s_written": nc * sp.nloc ** 2 * 8 / (t * 1e-3) / 1e9})
            del A, ud, sp
            torch.cuda.empty_cache()
    del mesh
    return {"rows": rows, "device_status": ctx.sync_status()}


# the other workloads, by name (in the order the default run measures them)
EXTRAS = {
    "structured_fp64": extra_structured,
    "linearised_hyperelastic_fp64": extra_linearised,
    "hdivcurl_mixed_32cube": extra_hdivcurl_mixed,
    "precision_64cube": lambda *a: precision_block(*a),
    "padaptive_batched_fp64": extra_padaptive,
    "naive_vs_sumfact_Q_laplace_32cube": extra_naive,
    "weighted_laplace_fp64_64cube": extra_weighted,
    "underintegration": lambda *a: underint_block(*a),
    "matvec_vs_action": lambda *a: matvec_block(*a),
    "cell_matrices_fp64_32cube": extra_matrices,
    "tangent_matrices_fp64_48cube": extra_tangent,
}


def run_extras(sfx, torch, ctx, inputs, flush, stream, only=None):
    ex = {}
    for name, fn in EXTRAS.items():
        if only and name not in only:
            continue
        ex[name] = fn(sfx, torch, ctx, inputs, flush, stream)
        torch.cuda.empty_cache()
    ex["note"] = ("extras are measured once per configuration with CUDA events (median of 1-3 runs, L2 "
                  "flushed); DoFs/s follows the paper's N/t; dofs_per_s_paper for matrices scales N by the "
                  "fraction of cells assembled")
    return ex


def matvec_block(sfx, torch, ctx, inputs, flush, stream):
    """Assembled CSR matrix (pattern untimed, as the paper excludes sparsity
    creation) vs matrix-free action, Q_p Laplace.  SpMV bytes per product:
    12 per nonzero (value + column) + 24 per row (x, y, row pointer); the
    achieved rate is against the measured HBM bandwidth."""
    rows = []
    for p, n in _ps([(1, 64), (2, 48), (3, 32), (4, 24), (5, 20), (6, 16)]):
        mesh = sfx.Mesh.box(ctx, *_d(n, n, n), perturb=0.1, seed=0)
        sp = sfx.Space(mesh, "Q", p)
        csr = sfx.Csr(sp)
        vals = torch.empty(csr.nnz, dtype=torch.float64, device="cuda")
        xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        yd = torch.empty_like(xd)
        ta = _time(torch, stream, flush, lambda: sfx.sfx_csr_assemble(ctx, "laplace", csr, vals, stream=stream),
                   reps=2, warm=1)
        tm = _time(torch, stream, flush, lambda: sfx.sfx_csr_spmv(ctx, csr, vals, xd, yd, stream=stream))
        tf = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd, stream=stream))
        tt = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd,
                                                                         precision="tf32x3", stream=stream))
        spmv_bytes = 12 * csr.nnz + 24 * csr.nrows
        rows.append({"p": p, "mesh": "%d^3" % n, "ndof": sp.ndof, "nnz": csr.nnz,
                     "assembly_ms": round(ta, 4), "spmv_ms": round(tm, 4), "action_fp64_ms": round(tf, 4),
                     "action_tf32x3_ms": round(tt, 4), "spmv_dofs_per_s": sp.ndof / (tm * 1e-3),
                     "action_fp64_dofs_per_s": sp.ndof / (tf * 1e-3),
                     "action_tf32x3_dofs_per_s": sp.ndof / (tt * 1e-3),
                     "spmv_gb_per_s": spmv_bytes / (tm * 1e-3) / 1e9,
                     "spmv_frac_of_hbm": spmv_bytes / (tm * 1e-3) / 1e9 / HBM_GBS})
        del vals, xd, yd, csr, sp, mesh
        torch.cuda.empty_cache()
    return {"rows": rows, "device_status": ctx.sync_status(),
            "note": "pattern built on the host, untimed; assembly = sum-factorised element matrices + coloured "
                    "scatter into the CSR values"}


def underint_block(sfx, torch, ctx, inputs, flush, stream):
    """Collocated (GLL) vs Gauss rule: Laplace action DoF/s on 64^3, p = 1..8,
    FP64 and TF32x3; Laplace element matrices on the first cells of a 32^3
    mesh (about 1 GB of output), delta-cancelled vs sum-factorised, with the
    bytes written per second (the collocated kernel's dense n^6 output)."""
    mesh = sfx.Mesh.box(ctx, *_d(64, 64, 64), perturb=0.1, seed=0)
    acts = []
    for p in _ps(range(1, 9)):
        sp = sfx.Space(mesh, "Q", p)
        xd = torch.from_numpy(inputs.random_vector(sp.ndof, 1, seed=1)).cuda()
        yd = torch.empty_like(xd)
        row = {"p": p, "ndof": sp.ndof}
        for prec in ("fp64", "tf32x3"):
            for algo in ("collocated", "sumfact"):
                t = _time(torch, stream, flush, lambda: sfx.sfx_assemble_action(ctx, "laplace", sp, xd, yd,
                                                                                precision=prec, algo=algo,
                                                                                stream=stream))
                row["%s_%s_ms" % (algo, prec)] = round(t, 4)
                row["%s_%s_dofs_per_s" % (algo, prec)] = sp.ndof / (t * 1e-3)
            row["speedup_collocated_vs_gauss_" + prec] = row["sumfact_%s_ms" % prec] / row["collocated_%s_ms" % prec]
        acts.append(row)
        del xd, yd, sp
    del mesh
    torch.cuda.empty_cache()
    mesh = sfx.Mesh.box(ctx, *_d(32, 32, 32), perturb=0.1, seed=0)
    mats = []
    for p in _ps(range(1, 9)):
        sp = sfx.Space(mesh, "Q", p)
        nc = int(min(sp.ncell, max(8, (1 << 30) // (sp.nloc * sp.nloc * 8))))
        A = torch.empty(nc * sp.nloc * sp.nloc, dtype=torch.float64, device="cuda")
        tc = _time(torch, stream, flush, lambda: sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp, 0, nc, A,
                                                                                algo="collocated", stream=stream))
        ts = _time(torch, stream, flush, lambda: sfx.sfx_assemble_cell_matrices(ctx, "laplace", sp, 0, nc, A,
                                                                                stream=stream), reps=2, warm=1)
        gbs = nc * sp.nloc ** 2 * 8 / (tc * 1e-3) / 1e9
        mats.append({"p": p, "cells": nc, "nloc": sp.nloc, "collocated_ms": round(tc, 4), "sumfact_ms": round(ts, 4),
                     "speedup": ts / tc, "collocated_cells_per_s": nc / (tc * 1e-3),
                     "collocated_gb_per_s_written": gbs, "collocated_write_frac_of_hbm": gbs / HBM_GBS})
        del A, sp
        torch.cuda.empty_cache()
    status = ctx.sync_status()
    return {"action_64cube": acts, "matrices_32cube": mats, "device_status": status,
            "note": "collocated = (p+1)-point Gauss-Lobatto rule on the GLL nodes (B = I): fewer contractions "
                    "and a different (under-integrated) operator; matrices: dense n^3 x n^3 output per cell"}


def precision_block(sfx, torch, ctx, inputs, flush, stream, dims=None, degrees=None,
                    precs=("fp64", "tf32x3", "bf16x3")):
    """Per (form, p): event time of each precision, DoF/s, speedup over FP64,
    the normwise (inf) relative error against the FP64 GPU action (which the
    GPU tests hold at 1e-12 of the oracle) and each precision's error against
    the oracle itself on six sampled cells (first, last and four seeded):
    max |b - b_ref| / max |b_ref| over their per-cell vectors.  The
    displacement for degree p is the first ndof draws of stream 1 scaled by
    0.05 h / p, exactly what inputs.displacement returns; it is generated once
    at the largest size and sliced, since the stream is counter-based."""
    import oracle as orc
    dims = dims or _d(64, 64, 64)
    degrees = degrees or _ps(range(3, 9))
    mesh = sfx.Mesh.box(ctx, *dims, perturb=0.1, seed=0)
    X = mesh.coords()
    rng = np.random.default_rng(23)
    rows = []
    for fam, form in [("Q", "laplace"), ("VQ", "neohooke")]:
        spaces = {p: sfx.Space(mesh, fam, p) for p in degrees}
        base = torch.from_numpy(inputs.random_vector(max(sp.ndof for sp in spaces.values()), 1, seed=1)).cuda()
        for p in degrees:
            sp = spaces[p]
            xd = base[:sp.ndof] * (0.05 / (dims[0] * p)) if fam == "VQ" else base[:sp.ndof]
            ys = {pr: torch.empty_like(xd) for pr in precs}
            row = {"family": fam, "form": form, "p": p, "ndof": sp.ndof}
            for pr in precs:
                t = _time(torch, stream, flush,
                          lambda: sfx.sfx_assemble_action(ctx, form, sp, xd, ys[pr], precision=pr, stream=stream))
                row[pr + "_ms"] = round(t, 4)
                row[pr + "_dofs_per_s"] = sp.ndof / (t * 1e-3)
            for pr in precs[1:]:
                row[pr + "_speedup_vs_fp64"] = row["fp64_ms"] / row[pr + "_ms"]
                row[pr + "_rel_err_vs_fp64"] = float((ys[pr] - ys["fp64"]).abs().max() / ys["fp64"].abs().max())
            del ys
            cells = np.unique(np.concatenate([[0, sp.ncell - 1], rng.choice(sp.ncell, 4, replace=False)]))
            ref = orc.cell_vectors(fam, form, p, dims, X, xd.cpu().numpy(), cells)
            cd = torch.from_numpy(cells.astype(np.int64)).cuda()
            for pr in precs:
                b = torch.empty(len(cells) * sp.nloc, dtype=torch.float64, device="cuda")
                sfx.sfx_assemble_cell_vectors(ctx, form, sp, xd, cd, b, precision=pr)
                row[pr + "_rel_err_vs_oracle_sampled"] = float(np.abs(b.cpu().numpy().reshape(ref.shape) - ref).max()
                                                               / np.abs(ref).max())
            rows.append(row)
            del xd
        del base, spaces
        torch.cuda.empty_cache()
    status = ctx.sync_status()
    return {"rows": rows, "mesh": "%dx%dx%d" % dims, "device_status": status,
            "note": "TF32x3/BF16x3: 1D contractions on the tensor cores (mma.sync, three split products, FP32 "
                    "accumulation); geometry, neo-Hookean stress and scatter in FP64"}


def e2e(args, sfx, torch, ctx, spaces, wl, prec, stream):
    """Same sweep through the public call with host buffers: every case copies
    its input from pinned host memory, runs the action and copies the result
    back, all inside the timed region.  The cases are pipelined over three
    streams -- input copies, compute, output copies -- so that one case's
    copies overlap another case's action; events order every reuse of a
    buffer (device buffers per case, pinned host buffers per space)."""
    hx, hy, dx, dy = {}, {}, [], []
    for key, sp in spaces.items():
        hx[key] = torch.empty(sp.ndof, dtype=torch.float64, pin_memory=True)
        hx[key].copy_(torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, sp.ndof)))
        hy[key] = torch.empty(sp.ndof, dtype=torch.float64, pin_memory=True)
    for fam, p, _ in wl:
        nd = spaces[(fam, p)].ndof
        dx.append(torch.empty(nd, dtype=torch.float64, device="cuda"))
        dy.append(torch.empty(nd, dtype=torch.float64, device="cuda"))
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    n = len(wl)
    ev_in = [torch.cuda.Event() for _ in range(n)]
    ev_comp = [torch.cuda.Event() for _ in range(n)]
    ev_out = [torch.cuda.Event() for _ in range(n)]
    started = [False] * n

    def step():
        for i, (fam, p, form) in enumerate(wl):
            k = (fam, p)
            if started[i]:
                s_in.wait_event(ev_comp[i])      # the previous step's action has read dx[i]
            with torch.cuda.stream(s_in):
                dx[i].copy_(hx[k], non_blocking=True)
            ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            if started[i]:
                stream.wait_event(ev_out[i])     # the previous step's result has left dy[i]
            sfx.sfx_assemble_action(ctx, form, spaces[k], dx[i], dy[i], precision=prec,
                                    params=HELM if form == "helmholtz" else None, stream=stream)
            ev_comp[i].record(stream)
            s_out.wait_event(ev_comp[i])
            with torch.cuda.stream(s_out):
                hy[k].copy_(dy[i], non_blocking=True)
            ev_out[i].record(s_out)
            started[i] = True

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    nb = sum(spaces[(f, p)].ndof * 8 for f, p, _ in wl)
    dofs = sum(spaces[(f, p)].ndof for f, p, _ in wl)
    del dx, dy
    torch.cuda.empty_cache()
    return {"value": dofs / dt, "unit": "DoF/s", "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
            "note": "cases pipelined over three streams (input copy, action, output copy)"}


if __name__ == "__main__":
    main()
