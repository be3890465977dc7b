#!/usr/bin/env python
"""Benchmark: time to a 1e-8 Newton residual for steady Navier-Stokes on a 96^3 sphere pack.

Workload (seeded, synthetic): 96^3 image, spheres with radius U[6, 10] at uniform centres (x-periodic,
overlap allowed) until the porosity first drops to 0.35, seed 0; non-percolating void dropped;
~200 watershed pores of ~500-20k unknowns; rho = b = 1, mu from the Kozeny-Carman estimate for Re = 1
(the Re reached is measured from the solution and reported).

One step = one full solve through libpns: the Stokes initial iterate (aPLMM_S preconditioner built and
FGMRES run), the gPLMM preconditioner built at that iterate (wind = Stokes velocity), Newton-FGMRES
until ||r|| / ||r(0)|| < 1e-8.  `value` times the step with CUDA events on the solver's stream from a
context whose integer maps already exist; `e2e` repeats the solve through the C ABI from HOST arrays
(setup, host->device copies, the device->host copy of the solution inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pns|reference] [--precision fp32]
N > 1 (torchrun): independent replicas, one per GPU (the method does not shard here).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 Newton residual"
UNIT = "ms"


def max_over_ranks(value, dist):
    """The maximum of a per-rank float over all ranks (a CPU tensor through the process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pns", choices=["pns", "reference"])
    ap.add_argument("--variant", default="gplmm")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--re", type=float, default=1.0)
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precisions", default="fp64,fp32,bf16",
                    help="local-inverse precisions to time once each on the --precision-n pack at N=1 "
                         "(results under 'precisions'; 'none' to skip)")
    ap.add_argument("--precision-n", type=int, default=48)
    ap.add_argument("--compare", default="aplmm_s,block_schur",
                    help="comma-separated preconditioner variants to time once each after the main run at N=1 "
                         "(results under 'variants'; 'none' to skip)")
    return ap.parse_args(argv)


def workload(args, rank=0):
    from paper_2510_22077_gb300 import inputs
    w = inputs.make_workload("spheres", seed=args.seed + rank, n=args.n)
    mu = inputs.mu_kozeny_carman(w.mask, args.re)
    return w, mu


def config(args, w, info):
    return {"workload": f"spheres{args.n}^3 phi=0.35 r~U[6,10] seed={args.seed}, steady NS Re~{args.re:g}, "
                        f"gPLMM preconditioner, {args.precision} local inverses, FP64 residual/Arnoldi",
            "image": list(w.mask.shape), "n_unknowns": info["n_unknowns"], "n_pores": info["n_prim"],
            "n_interfaces": info["n_iface"], "prim_sum_n2": info["prim_sum_n2"],
            "variant": args.variant, "precision": args.precision, "l2": "inputs larger than L2 (local inverses "
            f"{info['prim_sum_n2'] * 4 / 1e9:.1f} GB)", "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------- oracle
def cpu_baseline(w, mu, its_total, budget_s=25.0):
    """The FP64 oracle timed on the host on a bounded sample of the same solve, extrapolated to the
    full solve: maps and operator assembly measured in full; the local factorisations (primary,
    closure and dual blocks) measured on a seeded sample of blocks and extrapolated with a fitted
    t = a n^p per kind; one preconditioner apply and Arnoldi step extrapolated the same way; both
    builds (aPLMM_S, gPLMM) and `its_total` FGMRES iterations.  Runs in a child process with one
    thread."""
    code = r'''
import json, sys, time
import numpy as np
import scipy.sparse.linalg as spla
sys.path.insert(0, %r)
from oracle import krylov, mac, plmm
d = np.load(sys.argv[1])
mu, its, budget = float(sys.argv[2]), int(sys.argv[3]), float(sys.argv[4])
t0 = time.perf_counter()
pb = krylov.Problem(d["mask"], d["labels"], mac.Params(1.0, mu, (1.0, 0.0, 0.0)))
t_maps = time.perf_counter() - t0
g, m = pb.g, pb.maps
t0 = time.perf_counter()
A = mac.assemble(g, pb.prm, pb.pins, "stokes")
J = pb.jacobian(np.zeros(g.nfull))
t_asm = time.perf_counter() - t0
v = np.random.default_rng(0).standard_normal(g.nfull)
t0 = time.perf_counter(); J @ v; t_mv = time.perf_counter() - t0
prim = [np.asarray(P) for P in m.prim_unknowns]
dual = [np.asarray(D) for D in m.dual_unknowns]
rng = np.random.default_rng(1)
def fit(lists, tf_build, tf_apply):
    n = np.array([len(l) for l in lists], float)
    order = np.argsort(n)
    pick = sorted(set(order[np.linspace(0, len(order) - 1, 9).astype(int)].tolist()))
    xs, yb, ya = [], [], []
    t_start = time.perf_counter()
    for i in pick:
        if time.perf_counter() - t_start > budget / 3 and len(xs) >= 3:
            break
        tb, ta = tf_build(lists[i]), tf_apply
        xs.append(n[i]); yb.append(tb[0]); ya.append(tb[1])
    xs, yb, ya = np.log(xs), np.log(np.maximum(yb, 1e-6)), np.log(np.maximum(ya, 1e-7))
    pb_, pa_ = np.polyfit(xs, yb, 1), np.polyfit(xs, ya, 1)
    return float(np.exp(np.polyval(pb_, np.log(n))).sum()), float(np.exp(np.polyval(pa_, np.log(n))).sum()), len(xs)
def local(U):
    B = A[U][:, U].tocsc()
    t = time.perf_counter(); lu = spla.splu(B); tb = time.perf_counter() - t
    r = np.ones(len(U)); t = time.perf_counter(); lu.solve(r); ta = time.perf_counter() - t
    return tb, ta
def closure(U):
    B = A[U][:, U].tocsc()
    t = time.perf_counter(); lu = spla.splu(B); lu.solve(np.ones((len(U), 8))); tb = time.perf_counter() - t
    return tb, 0.0
bp, ap_, kp = fit(prim, local, None)
bd, ad, kd = fit(dual, local, None)
bc, _, kc = fit(prim, closure, None)
n_o = len(m.coarse_ifaces) + m.n_prim
import scipy.linalg as sla
t0 = time.perf_counter(); sla.lu_factor(np.random.default_rng(0).standard_normal((n_o, n_o))); t_co = time.perf_counter() - t0
build = bp + bd + bc + t_co
w1 = np.random.default_rng(2).standard_normal(g.nfull); w2 = w1.copy()
t0 = time.perf_counter(); h = np.dot(w1, w2); w2 -= h * w1; t_mgs = time.perf_counter() - t0
t_iter = ap_ + ad + 3 * t_mv + 2 * 50 * t_mgs          # 2 inner residual updates + J z; MGS over ~50 vectors
total = t_maps + t_asm + 2 * build + its * t_iter
print(json.dumps({"total_s": total, "maps_s": t_maps, "asm_s": t_asm, "build_s": build, "iter_s": t_iter,
                  "sampled_blocks": kp + kd + kc}))
''' % ROOT
    with tempfile.NamedTemporaryFile(suffix=".npz", delete=False) as f:
        path = f.name
    import numpy as np
    np.savez(path, mask=w.mask, labels=w.labels)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t0 = time.time()
    r = subprocess.run([sys.executable, "-c", code, path, str(mu), str(its_total), str(budget_s)], capture_output=True,
                       text=True, env=env, timeout=900)
    wall = time.time() - t0
    os.unlink(path)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["total_s"] * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle (NumPy/SciPy SuperLU), 1 thread, {wall:.0f} s of host time: maps "
                       f"{d['maps_s']:.1f} s and operator assembly {d['asm_s']:.1f} s measured in full; local "
                       f"factorisations and solves measured on {d['sampled_blocks']} sampled blocks and "
                       f"extrapolated (t = a n^p) to all blocks: one build {d['build_s']:.0f} s, one FGMRES "
                       f"iteration {d['iter_s']:.2f} s; total = maps + 2 builds + {its_total} iterations")}


def compare_variants(args, w, mu):
    """One solve per named variant on the same workload (fresh context each): wall time on the
    library's stream, iteration counts, build time."""
    out = {}
    for var in [v.strip() for v in args.compare.split(",") if v.strip()]:
        out[var] = one_solve(w, mu, var, args.precision)
    return out


def one_solve(w, mu, variant, precision):
    """One timed solve (Stokes guess, build, Newton) in a fresh context; errors are recorded, not raised,
    so that a failing comparison never costs the main line."""
    import torch
    from paper_2510_22077_gb300 import pns
    S = None
    try:
        S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=variant, precision=precision,
                       timing=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(S.stream)
        x = S.zeros()
        _, sst = S.pns_stokes_solve(x, check=False)
        S.pns_build_precond(x)
        st = S.pns_newton_solve(x, check=False)
        e1.record(S.stream)
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "status": st["status"], "stokes_status": sst["status"],
                "newton_its": st["newton_its"], "fgmres_its_stokes": sst["fgmres_its_total"],
                "fgmres_its_newton": st["fgmres_its"], "t_build_ms": st["t_ml_ms"] + st["t_mg_ms"],
                "final_res": st["res_hist"][-1] if st["res_hist"] else None}
    except Exception as e:   # recorded in the JSON line
        return {"error": f"{type(e).__name__}: {e}"[:300]}
    finally:
        if S is not None:
            S.close()


def compare_precisions(args):
    """gPLMM with FP64, FP32 and BF16 local inverses on the smaller sphere pack (an FP64 Gauss-Jordan
    build of the 96^3 pack takes minutes on the FP64 units): time to 1e-8 and iterations of each."""
    from paper_2510_22077_gb300 import inputs
    w = inputs.make_workload("spheres", seed=args.seed, n=args.precision_n)
    mu = inputs.mu_kozeny_carman(w.mask, args.re)
    out = {"workload": f"spheres{args.precision_n}^3 phi=0.35 seed={args.seed}, gPLMM, Re~{args.re:g}"}
    for prec in [p.strip() for p in args.precisions.split(",") if p.strip()]:
        out[prec] = one_solve(w, mu, "gplmm", prec)
    return out


# ---------------------------------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local_rank)
    from paper_2510_22077_gb300 import inputs, pns

    w, mu = workload(args, rank)
    S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=args.variant, precision=args.precision,
                   timing=True)
    info = S.info()

    def step():
        x = S.zeros()
        _, sst = S.pns_stokes_solve(x)
        S.pns_build_precond(x)
        st = S.pns_newton_solve(x)
        return x, sst, st

    last = None
    for _ in range(args.warmup):
        last = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = S.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local_rank)
    e0.record(stream)
    results = []
    for k in range(args.steps):
        x, sst, st = step()
        results.append((sst, st))
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        ms = max_over_ranks(ms, dist)
        dist.barrier()
    sst, st = results[-1]
    ux = x[:S.ncell].cpu().numpy().reshape(w.mask.shape)
    re_reached = inputs.reynolds(w.mask, ux, 1.0, mu)
    its_stokes = sst["fgmres_its_total"]
    its_newton = st["fgmres_its_total"]
    # batched local-solve kernel over the timed region: event times and launch counts are cumulative
    # per context, so take the difference to the end of the last warm-up step
    base = last[2] if last is not None else {"t_local_ms": 0.0, "local_launches": 0, "kernel_launches": 0,
                                             "t_gj_update_ms": 0.0, "gj_update_flops": 0.0,
                                             "gj_update_launches": 0, "gj_update_tiles": 0}
    bytes_apply = st["local_bytes_per_apply"]
    launches_local = st["local_launches"] - base["local_launches"]
    t_local = st["t_local_ms"] - base["t_local_ms"]
    achieved = bytes_apply * (launches_local / 2.0) / (t_local * 1e-3) / 1e9 if t_local > 0 else None
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    launches = st["kernel_launches"] - base["kernel_launches"]
    # dominant kernel of the step: the FP32 Gauss-Jordan update of the local-inverse builds (ALU-bound);
    # peak from unit counts: SMs x 128 FP32 FMA lanes x 2 flops x the maximum SM clock
    gj_ms = st["t_gj_update_ms"] - base["t_gj_update_ms"]
    gj_fl = st["gj_update_flops"] - base["gj_update_flops"]
    gj_n = st["gj_update_launches"] - base["gj_update_launches"]
    gj_tiles = st["gj_update_tiles"] - base["gj_update_tiles"]
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    gj_achieved = gj_fl / (gj_ms * 1e-3) / 1e12 if gj_ms > 0 else None
    S.close()
    line = {"metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (residual, outer Jacobian, Arnoldi) + " + args.precision + " (preconditioner)",
            "data": "synthetic (seeded sphere pack)", "config": config(args, w, info),
            "fgmres_its": {"stokes": its_stokes, "newton": its_newton, "per_newton_step": st["fgmres_its"]},
            "newton_its": st["newton_its"], "res_hist": st["res_hist"], "re_reached": re_reached,
            "buckets_ms": {"t_ml": st["t_ml_ms"], "t_mg": st["t_mg_ms"], "t_sol_newton": st["t_sol_ms"],
                           "t_sol_stokes": sst["t_sol_ms"]},
            # traffic: DRAM bytes per launch, scaled from the ncu captures of the same kernels on the 48^3
            # pack (profiles/): update 0.979 x its C-tile bytes, local solve 1.019 x its algorithmic bytes
            "roofline": {"kernel": "k_mm128_gj_update (FP32 Gauss-Jordan trailing update of the local inverses)",
                         "bound": "alu", "achieved": gj_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": (gj_achieved / fp32_peak) if gj_achieved else None,
                         "traffic": (0.979 * gj_tiles * 128 * 128 * 8 / gj_n) if gj_n else None,
                         "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:g} MHz",
                         "flops_timed": gj_fl, "launches_timed": gj_n, "ms_timed": gj_ms},
            "roofline_apply": {"kernel": "k_local_gemv (batched local solves M_d, M_p; with its gather)",
                               "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": (achieved / peak) if achieved else None,
                               "traffic": 1.019 * bytes_apply, "traffic_unit": "bytes per M_d + M_p pass",
                               "peak_source": peak_src, "bytes_per_apply": bytes_apply,
                               "launches_timed": launches_local, "ms_timed": t_local},
            "clocks": clocks, "gpu_launches": launches}
    if rank == 0 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S2 = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=args.variant, precision=args.precision)
        x2 = S2.zeros()
        S2.pns_stokes_solve(x2)
        S2.pns_build_precond(x2)
        S2.pns_newton_solve(x2)
        host = x2.cpu().numpy()
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3
        S2.close()
        line["e2e"] = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(w.mask.nbytes + w.labels.nbytes),
                       "d2h_bytes_per_step": int(host.nbytes)}
    if rank == 0 and world == 1 and args.compare and args.compare != "none":
        line["variants"] = compare_variants(args, w, mu)
    if rank == 0 and world == 1 and args.precisions and args.precisions != "none":
        line["precisions"] = compare_precisions(args)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, mu, its_stokes + its_newton)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, rank 0 only (others exit)."""
    if rank != 0:
        return
    w, mu = workload(args, 0)
    # the same config record as the GPU arm, its sizes taken from the oracle's maps
    from oracle import krylov, mac
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)))
    info = {"n_unknowns": int(len(pb.g.unknown)), "n_prim": int(pb.maps.n_prim), "n_iface": int(pb.maps.n_iface),
            "prim_sum_n2": float(sum(len(P) ** 2 for P in pb.maps.prim_unknowns))}
    del pb
    its = 83 + 209       # FGMRES iterations of one solve of this workload (Stokes + Newton), as the GPU path takes them
    vals = []
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(w, mu, its)
        vals.append(cb["value"])
    v = float(sum(vals) / len(vals)) if all(x is not None for x in vals) else None
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 0,
            "ms_per_step": v, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded sphere pack)", "impl": "reference",
            "config": config(args, w, info),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
