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
# DRAM bytes measured by ncu per algorithmic byte, for the kernels of the current build (profiles/*.md); a
# kernel missing here has no capture of its current version and reports no traffic
TRAFFIC_RATIO = {"k_local_gemv_p": 1.008, "k_gj_update_tcp": 1.008}
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
    ap.add_argument("--gj", type=int, default=None,
                    help="Gauss-Jordan update of the FP32 local inverses: 0 FMA units, 1 mma.sync, 2 tcgen05 "
                         "(default: the library's)")
    ap.add_argument("--jac-only", action="store_true",
                    help="time only the FP64 Jacobian apply (pns_setup + pns_jacobian_apply; no preconditioner)")
    ap.add_argument("--learned", action="store_true",
                    help="the learned-initial-guess experiment instead of the main line: solver-generated samples, "
                         "U-Net training on the GPU, Newton from the Stokes vs the guarded learned start on "
                         "held-out images")
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--sample-n", type=int, default=64)
    ap.add_argument("--kinds", default="spheres", help="image kinds of the learned-guess samples (spheres,grf)")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--heldout", default="64:9000-9007,96:9000-9001",
                    help="held-out images as size:first-last seed ranges")
    ap.add_argument("--autotune", action="store_true",
                    help="run the local-solve autotuner on the workload's gPLMM preconditioner and print its table "
                         "(the table the library ships, paper_2510_22077_gb300/tuning_gb300.json, came from this)")
    ap.add_argument("--transient", action="store_true",
                    help="the transient configuration instead of the main line: 128^3 sphere pack at porosity 0.40 "
                         "(labeller target 1400 pores), Re 50, dt for CFL 1, backward Euler from rest with one "
                         "aPLMM_NS build reused for every step")
    ap.add_argument("--be-steps", type=int, default=50)
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
# The FP64 oracle timed on the host cores.  Every figure is a measured run of the oracle's own steps
# (oracle/: maps, operator assembly, SuperLU factorisations of the local and closure blocks as
# oracle.plmm.Plmm makes them, their solves, a Jacobian apply, one Gram-Schmidt pass).  The local blocks
# are split into N_STRATA strata (dealt in snake order over the size ranking, primary and dual grids alike);
# a bounded sample measures some strata in full, and the build and apply times of the sample are scaled
# by N_STRATA / (strata measured): with all strata measured (the reference arm at --steps >= N_STRATA)
# the whole build is measured and nothing is scaled.
N_STRATA = 20
SOLVE_GOLDEN = os.path.join(ROOT, "tests", "golden", "spheres96_solve.json")


def _oracle_setup(spec):
    import numpy as np
    from oracle import krylov, mac
    d = np.load(spec["npz"])
    t0 = time.perf_counter()
    pb = krylov.Problem(d["mask"], d["labels"], mac.Params(1.0, spec["mu"], (1.0, 0.0, 0.0)))
    t_maps = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = pb.build_matrix("aplmm_s", None)
    t_asm = time.perf_counter() - t0
    return pb, A, t_maps, t_asm


def _strata(pb, n_strata):
    import numpy as np
    m = pb.maps
    kinds = [("p", i, len(P)) for i, P in enumerate(m.prim_unknowns)] + \
            [("d", j, len(D)) for j, D in enumerate(m.dual_unknowns)]
    kinds.sort(key=lambda t: (-t[2], t[0], t[1]))
    # snake order over the size ranking (0..S-1, S-1..0, ...): every stratum gets blocks of every size and
    # about the same share of the work
    strata = [[] for _ in range(n_strata)]
    for r, kd in enumerate(kinds):
        q, m = divmod(r, n_strata)
        strata[m if q % 2 == 0 else n_strata - 1 - m].append(kd)
    return strata, np


def _time_blocks(pb, A, blocks):
    """Oracle build and one solve of the given blocks: (build seconds, solve seconds)."""
    import numpy as np
    import scipy.sparse.linalg as spla
    from oracle import plmm
    m = pb.maps
    tb = ts = 0.0
    for kind, i, _ in blocks:
        U = m.prim_unknowns[i] if kind == "p" else m.dual_unknowns[i]
        t = time.perf_counter()
        lu = spla.splu(A[U][:, U].tocsc())
        if kind == "p":
            lub = spla.splu(plmm.closure_block(A, m, i))
            lub.solve(np.ones((len(U), len(m.C[i]) + 1)))
        tb += time.perf_counter() - t
        r = np.ones(len(U))
        t = time.perf_counter()
        lu.solve(r)
        ts += time.perf_counter() - t
    return tb, ts


_POOL = {}


def _pool_init(spec):
    pb, A, _, _ = _oracle_setup(spec)
    _POOL["pb"], _POOL["A"] = pb, A


def _pool_task(blocks):
    return _time_blocks(_POOL["pb"], _POOL["A"], blocks)


def oracle_worker(spec):
    """Child-process entry (bench.py --oracle-worker JSON): prints one JSON line per measured stratum, then
    a summary line with the fixed costs."""
    import numpy as np
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    pb, A, t_maps, t_asm = _oracle_setup(spec)
    g = pb.g
    strata, _ = _strata(pb, spec["n_strata"])
    rng = np.random.default_rng(0)
    v = np.zeros(g.nfull)
    v[g.unknown] = rng.standard_normal(len(g.unknown))
    J = pb.jacobian(v)
    t0 = time.perf_counter()
    for _ in range(3):
        J @ v
    t_jac = (time.perf_counter() - t0) / 3
    V = rng.standard_normal((50, g.nfull))
    w = v.copy()
    t0 = time.perf_counter()
    for i in range(50):                      # one modified Gram-Schmidt pass against 50 basis vectors
        w -= np.dot(w, V[i]) * V[i]
    t_orth = time.perf_counter() - t0
    import scipy.linalg as sla
    n_o = len(pb.maps.coarse_ifaces) + pb.maps.n_prim
    t0 = time.perf_counter()
    sla.lu_factor(rng.standard_normal((n_o, n_o)))
    t_coarse = time.perf_counter() - t0
    for k in range(spec.get("warmup", 0)):
        _time_blocks(pb, A, strata[k % len(strata)][-2:])
    for s in spec["strata"]:
        t0 = time.perf_counter()
        tb, ts = _time_blocks(pb, A, strata[s])
        print(json.dumps({"stratum": s, "build_s": tb, "solve_s": ts, "blocks": len(strata[s]),
                          "wall_s": time.perf_counter() - t0}), flush=True)
    out = {"maps_s": t_maps, "asm_s": t_asm, "jac_s": t_jac, "orth50_s": t_orth, "coarse_lu_s": t_coarse,
           "n_o": n_o, "n_blocks": sum(len(x) for x in strata)}
    if spec.get("mt_workers", 0) > 1:
        import multiprocessing as mp
        jobs = [strata[s][q::spec["mt_workers"]] for s in spec["strata"] for q in range(spec["mt_workers"])]
        ctx = mp.get_context("spawn")
        with ctx.Pool(spec["mt_workers"], initializer=_pool_init, initargs=(spec,)) as pool:
            pool.map(_pool_task, [jobs[0][:1]] * spec["mt_workers"])      # workers ready
            t0 = time.perf_counter()
            res = pool.map(_pool_task, jobs)
            out["mt_build_wall_s"] = time.perf_counter() - t0
            out["mt_build_cpu_s"] = float(sum(r[0] + r[1] for r in res))
        out["mt_workers"] = spec["mt_workers"]
    print(json.dumps({"summary": out}), flush=True)


def oracle_iterations():
    """FGMRES iterations of the oracle's own solve of the 96^3 benchmark workload (Stokes + Newton), from
    the stored oracle run (tests/golden/make_spheres96_solve.py calls only the oracle)."""
    try:
        d = json.load(open(SOLVE_GOLDEN))
        return int(sum(d["stokes_fgmres_its"]) + sum(d["newton_fgmres_its"])), "oracle's own solve of this workload"
    except (OSError, KeyError, ValueError):
        return None, None


def run_oracle(w, mu, strata, warmup=0, mt_workers=0, timeout=1800):
    """Run the oracle timing child; returns (per-stratum records, summary)."""
    import numpy as np
    with tempfile.NamedTemporaryFile(suffix=".npz", delete=False) as f:
        path = f.name
    np.savez(path, mask=w.mask, labels=w.labels)
    spec = {"npz": path, "mu": mu, "n_strata": N_STRATA, "strata": list(strata), "warmup": warmup,
            "mt_workers": mt_workers}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-worker", json.dumps(spec)],
                       capture_output=True, text=True, env=env, timeout=timeout)
    os.unlink(path)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-400:])
    recs, summ = [], None
    for line in r.stdout.splitlines():
        if line.startswith("{"):
            d = json.loads(line)
            if "summary" in d:
                summ = d["summary"]
            else:
                recs.append(d)
    return recs, summ


def compose_oracle(recs, summ, its, its_src):
    """Time to 1e-8 of the oracle from measured parts: maps + assembly + two builds (aPLMM_S for the Stokes
    iterate, gPLMM at it; each build = the local and closure factorisations + the coarse LU) + `its` FGMRES
    iterations (each: the local solves, three Jacobian-sized sparse products, one Gram-Schmidt pass)."""
    scale = N_STRATA / len(recs)
    build = scale * sum(r["build_s"] for r in recs) + summ["coarse_lu_s"]
    solves = scale * sum(r["solve_s"] for r in recs)
    it = solves + 3 * summ["jac_s"] + summ["orth50_s"]
    total = summ["maps_s"] + summ["asm_s"] + 2 * build + its * it
    return total, build, it, scale


def cpu_baseline(w, mu, its_gpu, strata=(9, 10), mt=True, stored_its=True):
    """The FP64 oracle on one host core on a bounded sample of the workload: the strata given (2 of 20:
    a tenth of the local blocks, every size represented; the two middle strata of the snake order, whose
    blocks sit mid-rank in every group of 20, so that the heavy tail of block sizes is not over-weighted)
    measured in full, scaled to all blocks; plus the same sample on all host cores (process pool) as a
    labelled multi-threaded figure.  The reference arm measures every stratum."""
    its, its_src = oracle_iterations() if stored_its else (None, None)
    if its is None:
        its, its_src = its_gpu, "FGMRES iterations of this run's GPU solve (no stored oracle solve)"
    cores = os.cpu_count() or 1
    try:
        recs, summ = run_oracle(w, mu, strata, mt_workers=cores if mt else 0)
    except Exception as e:   # recorded, never fatal for the main line
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    total, build, it, scale = compose_oracle(recs, summ, its, its_src)
    wall = sum(r["wall_s"] for r in recs)
    out = {"value": total * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"FP64 oracle (NumPy/SciPy, SuperLU per block as oracle.plmm builds them), 1 thread; measured "
                      f"in full: maps {summ['maps_s']:.1f} s, operator assembly {summ['asm_s']:.1f} s, one Jacobian "
                      f"apply {summ['jac_s'] * 1e3:.0f} ms, one Gram-Schmidt pass over 50 vectors "
                      f"{summ['orth50_s'] * 1e3:.0f} ms, the coarse LU; local and closure factorisations and one "
                      f"solve of each measured in full on {len(recs)} of {N_STRATA} strata (snake order over the sizes) "
                      f"({sum(r['blocks'] for r in recs)} of {summ['n_blocks']} blocks, {wall:.0f} s) and scaled x"
                      f"{scale:g}: one build {build:.0f} s, one FGMRES iteration {it:.2f} s; total = maps + assembly "
                      f"+ 2 builds + {its} iterations ({its_src})"),
           "parts_s": {"maps": summ["maps_s"], "assembly": summ["asm_s"], "build": build, "iteration": it,
                       "jacobian_apply": summ["jac_s"], "iterations": its}}
    if "mt_build_wall_s" in summ:
        mt_build = scale * summ["mt_build_wall_s"] + summ["coarse_lu_s"]
        mt_total = summ["maps_s"] + summ["asm_s"] + 2 * mt_build + its * it
        out["multi_threaded"] = {"value": mt_total * 1e3, "unit": UNIT, "cores": summ["mt_workers"],
                                 "sample": (f"the same sample with the block factorisations spread over "
                                            f"{summ['mt_workers']} processes ({summ['mt_build_wall_s']:.1f} s wall); "
                                            f"iterations kept serial")}
    return out


def time_jacobian(S, info, reps=40, sets=4, peak=None, seed=0):
    """Mean time of pns_jacobian_apply over `reps` launches on the solver's stream (CUDA events), cycling
    through `sets` different (state, v, y) triples so that the inputs of consecutive launches (4 full-layout
    FP64 vectors per triple) exceed the L2 cache.  Bytes: the algorithmic count 8 (2 N + n_f) + N of a
    packed layout, and what the image-shaped layout moves (v and y over every cell slot, the face state,
    one flag byte per cell)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    xs = [torch.randn(S.nfull, dtype=torch.float64, device="cuda", generator=g) for _ in range(sets)]
    vs = [torch.randn(S.nfull, dtype=torch.float64, device="cuda", generator=g) for _ in range(sets)]
    ys = [S.zeros() for _ in range(sets)]
    for q in range(sets):
        S.pns_jacobian_apply(xs[q], vs[q], ys[q])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(S.stream)
    for r in range(reps):
        q = r % sets
        S.pns_jacobian_apply(xs[q], vs[q], ys[q])
    e1.record(S.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    N, nf, nc, dim = info["n_unknowns"], info["n_faces"], info["ncell"], info["dim"]
    alg = 8.0 * (2 * N + nf) + N
    lay = 8.0 * (2 * (dim + 1) * nc + dim * nc) + nc
    out = {"kernel": "k_apply<double> (FP64 Jacobian apply, pns_jacobian_apply)", "bound": "hbm",
           "ms_per_apply": ms, "bytes_algorithmic": alg, "bytes_layout": lay,
           "achieved": alg / (ms * 1e-3) / 1e9, "achieved_layout": lay / (ms * 1e-3) / 1e9, "unit": "GB/s",
           "launches_timed": reps, "l2": f"{sets} rotating input sets of {4 * S.nfull * 8 / 1e6:.0f} MB"}
    if peak:
        out["peak"] = peak
        out["frac"] = out["achieved"] / peak
        out["frac_layout"] = out["achieved_layout"] / peak
    return out


def compare_variants(args, w, mu):
    """One solve per named variant on the same workload (fresh context each): wall time on the
    library's stream, iteration counts, build time."""
    out = {}
    for var in [v.strip() for v in args.compare.split(",") if v.strip()]:
        out[var] = one_solve(w, mu, var, args.precision, args.gj)
    return out


def one_solve(w, mu, variant, precision, gj=None):
    """One timed solve (Stokes guess, build, Newton) in a fresh context; errors are recorded, not raised,
    so that a failing comparison never costs the main line."""
    import torch
    from paper_2510_22077_gb300 import pns
    S = None
    try:
        S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=variant, precision=precision,
                       timing=True, gj_tensor_cores=gj)
        tt, _ = load_tuning()
        if tt:
            S.pns_set_tuning(tt)
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
        out[prec] = one_solve(w, mu, "gplmm", prec, args.gj)
    return out


def run_transient(args):
    """Backward Euler through the library: the aPLMM_NS preconditioner built once at the state of rest and
    reused by the Newton solve of every time step (Sec. 8.2); each step timed with CUDA events."""
    import numpy as np
    import torch
    from paper_2510_22077_gb300 import inputs, pns
    n = args.n if args.n != 96 else 128
    w = inputs.make_workload("spheres", seed=args.seed, n=n, porosity=0.40, target=1400)
    re = 50.0
    mu = inputs.mu_kozeny_carman(w.mask, re)
    U = re * mu / inputs.characteristic_length(w.mask)
    dt = 1.0 / U
    S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), dt, variant="aplmm_ns", precision=args.precision,
                   timing=True, gj_tensor_cores=args.gj)
    tt, _ = load_tuning()
    if tt:
        S.pns_set_tuning(tt)
    info = S.info()
    print(json.dumps({"transient_setup": info}), file=sys.stderr, flush=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x_prev = S.zeros()
    torch.cuda.synchronize()
    e0.record(S.stream)
    S.pns_build_precond(x_prev)
    e1.record(S.stream)
    torch.cuda.synchronize()
    t_build = e0.elapsed_time(e1)
    steps = []
    clk = ClockSampler(0)
    for k in range(args.be_steps):
        x = x_prev.clone()
        e0.record(S.stream)
        st = S.pns_newton_solve(x, x_prev, check=False)
        e1.record(S.stream)
        torch.cuda.synchronize()
        steps.append({"ms": e0.elapsed_time(e1), "newton_its": st["newton_its"], "fgmres_its": st["fgmres_its"],
                      "status": st["status"]})
        print(json.dumps({"be_step": k, **steps[-1]}), file=sys.stderr, flush=True)
        x_prev = x
        if st["status"] != "PNS_OK":
            break
    clocks = clk.stop()
    ux = x_prev[:S.ncell].cpu().numpy().reshape(w.mask.shape)
    its = [i for s_ in steps for i in s_["fgmres_its"]]
    line = {"metric": "transient NS: time per backward-Euler step", "value": float(np.mean([s_["ms"] for s_ in steps])),
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": len(steps),
            "dtype": "f64 (residual, outer Jacobian, Arnoldi) + " + args.precision + " (preconditioner)",
            "data": "synthetic (seeded sphere pack)",
            "config": {"workload": f"spheres{n}^3 phi=0.40 r~U[6,10] seed={args.seed}, labeller target 1400 pores, "
                                   f"Re {re:g} (Kozeny-Carman mu), dt = h/U = {dt:.4g} (CFL 1), backward Euler from "
                                   f"rest, aPLMM_NS built once at rest and reused", "n_unknowns": info["n_unknowns"],
                       "n_pores": info["n_prim"], "n_interfaces": info["n_iface"], "max_block": info["max_block"],
                       "prim_sum_n2": info["prim_sum_n2"], "dual_sum_n2": info["dual_sum_n2"], "dt": dt, "mu": mu},
            "build_ms": t_build, "newton_its_per_step": [s_["newton_its"] for s_ in steps],
            "fgmres_its_per_newton_step_mean": float(np.mean(its)) if its else None,
            "fgmres_its_per_step": [s_["fgmres_its"] for s_ in steps], "ms_per_step": [s_["ms"] for s_ in steps],
            "status_last": steps[-1]["status"] if steps else None,
            "re_reached_last": inputs.reynolds(w.mask, ux, 1.0, mu), "clocks": clocks}
    S.close()
    print(json.dumps(line), flush=True)


TUNING = os.path.join(ROOT, "paper_2510_22077_gb300", "tuning_gb300.json")


def load_tuning():
    """The committed local-solve tuning table (one shape id per block-size bin), or None."""
    try:
        d = json.load(open(TUNING))
        return [int(v) for v in d["table"]], d
    except (OSError, KeyError, ValueError):
        return None, None


def run_autotune(args):
    """Autotune the persistent local-solve launch on this workload (gPLMM built at the Stokes iterate) and
    print the table with the time of every (bin, shape)."""
    from paper_2510_22077_gb300 import pns
    w, mu = workload(args)
    S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=args.variant, precision=args.precision,
                   gj_tensor_cores=args.gj)
    x, _ = S.pns_stokes_solve()
    S.pns_build_precond(x)
    table, ms = S.pns_autotune()
    out = {"table": table, "ms": ms.tolist(), "shapes": pns.TUNE_SHAPES, "bin_edges": pns.TUNE_BIN_EDGES,
           "workload": config(args, w, S.info())["workload"],
           "how": "pns_autotune: best of five launches after one warm-up per (bin, shape), primary and dual sets "
                  "summed, CUDA events, one GB300"}
    S.close()
    print(json.dumps(out), flush=True)


def run_learned(args):
    """The learned Newton initial guess (BASELINE config 5 at reduced scale, stated in the line): samples
    generated by the solver, the U-Net trained on the GPU, then on held-out images Newton from the Stokes
    solution and from the guarded learned start, each timed with CUDA events."""
    import numpy as np
    import torch
    from paper_2510_22077_gb300 import learned, pns
    t0 = time.time()
    n = args.sample_n
    net = pns.UNet(channels=(16, 32, 64, 64), in_ch=6, out_ch=4, batch=4, shape=(n, n, n), seed=args.seed)
    log = lambda m: print(m, file=sys.stderr, flush=True)   # noqa: E731
    kinds = tuple(args.kinds.split(","))
    data = learned.Dataset(net, args.samples, n=n, seed0=1000, log=log, kinds=kinds)
    t_data = time.time() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(net.stream)
    hist = learned.train(net, data, epochs=args.epochs, batch=4, lr=args.lr, seed=args.seed, log=log)
    e1.record(net.stream)
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1) / 1e3
    evals = []
    for spec in args.heldout.split(","):
        size, rng_ = spec.split(":")
        lo, hi = (int(v) for v in rng_.split("-"))
        for seed in range(lo, hi + 1):
            kind = kinds[seed % len(kinds)]
            w, phi = learned._image(kind, seed, int(size))
            re = float(np.random.default_rng(seed + 7).uniform(1.0, 100.0))
            if int(size) != n:
                # the network is fully convolutional: run it at the held-out size
                net_eval = pns.UNet(channels=(16, 32, 64, 64), in_ch=6, out_ch=4, batch=1,
                                    shape=w.mask.shape, seed=0)
                net_eval.set_params(net.get_params())
            else:
                net_eval = net
            try:
                r = learned.compare_on(w, re, net_eval, gain=data.gain)
                log(f"held-out {size}^3 seed {seed}: {r}")
            except Exception as ex:   # recorded
                r = {"error": f"{type(ex).__name__}: {ex}"[:200]}
            evals.append({"size": int(size), "seed": seed, "kind": kind, "phi": phi, "re": re, **r})
            if net_eval is not net:
                net_eval.close()
    ok = [e for e in evals if "stokes" in e and e["stokes"]["status"] == "PNS_OK" and e["learned"]["status"] == "PNS_OK"]
    line = {"metric": "learned Newton initial guess: Newton iterations and time to 1e-8, Stokes start vs learned start",
            "unit": "ms", "data": "synthetic (seeded sphere packs and Gaussian fields)",
            "config": {"workload": f"3D U-Net (16/32/64/64, BF16, FP32 master, Adam) trained on {data.m} solver-generated "
                                   f"{n}^3 samples ({'/'.join(kinds)}; {data.skipped} images skipped: failed solves), "
                                   f"{args.epochs} epochs; held-out {args.heldout}", "samples": data.m,
                       "skipped": data.skipped, "re_range": [1, 100], "kinds": list(kinds)},
            "seconds": {"samples": t_data, "train": t_train}, "loss_per_epoch": hist,
            "heldout": evals,
            "summary": {"images": len(ok),
                        "newton_its_stokes": float(np.mean([e["stokes"]["newton_its"] for e in ok])) if ok else None,
                        "newton_its_learned": float(np.mean([e["learned"]["newton_its"] for e in ok])) if ok else None,
                        "ms_stokes": float(np.mean([e["stokes"]["ms"] for e in ok])) if ok else None,
                        "ms_learned": float(np.mean([e["learned"]["ms"] for e in ok])) if ok else None,
                        "network_used": int(sum(e["learned"]["used_network"] for e in ok))}}
    print(json.dumps(line), flush=True)
    net.close()


# ---------------------------------------------------------------------------------------- main
def main():
    if len(sys.argv) > 2 and sys.argv[1] == "--oracle-worker":
        return oracle_worker(json.loads(sys.argv[2]))
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.learned:
        return run_learned(args)
    if args.autotune:
        return run_autotune(args)
    if args.transient:
        return run_transient(args)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local_rank)
    from paper_2510_22077_gb300 import inputs, pns

    w, mu = workload(args, rank)
    S = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=args.variant, precision=args.precision,
                   timing=True, gj_tensor_cores=args.gj)
    info = S.info()
    tune_table, tune_rec = load_tuning()
    if tune_table:
        S.pns_set_tuning(tune_table)
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    if args.jac_only:
        rj = time_jacobian(S, info, peak=peak)
        rj["peak_source"] = peak_src
        rj["workload"] = config(args, w, info)["workload"]
        print(json.dumps({"jacobian": rj}), flush=True)
        S.close()
        if dist:
            dist.destroy_process_group()
        return

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
                                             "t_gj_update_ms": 0.0, "gj_update_flops": 0.0, "gj_update_bytes": 0.0,
                                             "gj_update_launches": 0, "gj_update_tiles": 0}
    bytes_apply = st["local_bytes_per_apply"]
    launches_local = st["local_launches"] - base["local_launches"]
    t_local = st["t_local_ms"] - base["t_local_ms"]
    achieved = bytes_apply * (launches_local / 2.0) / (t_local * 1e-3) / 1e9 if t_local > 0 else None
    launches = st["kernel_launches"] - base["kernel_launches"]
    # dominant kernel of the step: the FP32 Gauss-Jordan update of the local-inverse builds (ALU-bound);
    # peak from unit counts: SMs x 128 FP32 FMA lanes x 2 flops x the maximum SM clock
    gj_ms = st["t_gj_update_ms"] - base["t_gj_update_ms"]
    gj_fl = st["gj_update_flops"] - base["gj_update_flops"]
    gj_by = st["gj_update_bytes"] - base.get("gj_update_bytes", 0.0)
    gj_n = st["gj_update_launches"] - base["gj_update_launches"]
    gj_tiles = st["gj_update_tiles"] - base["gj_update_tiles"]
    gj_kind = {0: "fma", 1: "mma.sync", 2: "tcgen05", 3: "tcgen05-tile"}.get(args.gj if args.gj is not None else 2)
    gj_achieved = gj_fl / (gj_ms * 1e-3) / 1e12 if gj_ms > 0 else None
    gj_gbs = gj_by / (gj_ms * 1e-3) / 1e9 if gj_ms > 0 else None
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16_peak, bf16_src = pk["bf16_tflops"], "measured"
    except (OSError, KeyError, ValueError):
        bf16_peak, bf16_src = 1900.0, "fallback"
    # TF32 dense rate = the measured BF16 rate x the nominal TF32 / BF16 ratio (1.1 / 2.25); the update runs
    # three TF32 products per FP32 product, so its FP32-equivalent tensor ceiling is a third of that
    tf32_peak = bf16_peak * 1.1 / 2.25
    fp32_eq_peak = tf32_peak / 3.0
    roof_gj = {"kernel": "k_gj_update_tcp (FP32 Gauss-Jordan trailing update of the local inverses, tcgen05 "
                         "kind::tf32 with a 3-term split, persistent)" if gj_kind == "tcgen05" else
                         f"Gauss-Jordan trailing update ({gj_kind})",
               "bound": "hbm", "achieved": gj_gbs, "peak": peak, "unit": "GB/s",
               "frac": (gj_gbs / peak) if gj_gbs else None,
               "traffic": (TRAFFIC_RATIO["k_gj_update_tcp"] * gj_by / gj_n
                           if TRAFFIC_RATIO.get("k_gj_update_tcp") and gj_n and gj_kind == "tcgen05" else None),
               "peak_source": peak_src,
               "bytes_timed": gj_by, "flops_timed": gj_fl, "launches_timed": gj_n, "ms_timed": gj_ms,
               "tensor": {"achieved": gj_achieved, "unit": "TFLOP/s (FP32 products)", "peak": fp32_eq_peak,
                          "frac": (gj_achieved / fp32_eq_peak) if gj_achieved else None,
                          "peak_source": f"{bf16_src} BF16 {bf16_peak:g} TFLOP/s x 1.1/2.25 (TF32) / 3 products"}}
    roof_jac = time_jacobian(S, info, peak=peak)
    roof_jac["peak_source"] = peak_src
    S.close()
    line = {"metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (residual, outer Jacobian, Arnoldi) + " + args.precision + " (preconditioner)",
            "data": "synthetic (seeded sphere pack)", "config": config(args, w, info),
            "fgmres_its": {"stokes": its_stokes, "newton": its_newton, "per_newton_step": st["fgmres_its"]},
            "newton_its": st["newton_its"], "res_hist": st["res_hist"], "re_reached": re_reached,
            "buckets_ms": {"t_ml": st["t_ml_ms"], "t_mg": st["t_mg_ms"], "t_sol_newton": st["t_sol_ms"],
                           "t_sol_stokes": sst["t_sol_ms"],
                           "t_mg_parts": dict(zip(["closure_solves", "coarse_matrix", "coarse_inverse"],
                                                  st["t_mg_parts_ms"]))},
            # traffic: DRAM bytes per unit, scaled from the ncu captures of the same kernels on the 48^3 pack
            # (profiles/) by the units processed (TRAFFIC_RATIO: measured DRAM bytes / algorithmic bytes)
            "roofline": roof_gj,
            "roofline_apply": {"kernel": "k_local_gemv_p (persistent size-binned local solves M_d, M_p; with their "
                                         "gather and refinement residual)",
                               "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": (achieved / peak) if achieved else None,
                               "traffic": (TRAFFIC_RATIO["k_local_gemv_p"] * bytes_apply
                                           if TRAFFIC_RATIO.get("k_local_gemv_p") else None),
                               "traffic_unit": "bytes per M_d + M_p pass",
                               "peak_source": peak_src, "bytes_per_apply": bytes_apply,
                               "launches_timed": launches_local, "ms_timed": t_local},
            "roofline_jac": roof_jac, "clocks": clocks, "gpu_launches": launches,
            "local_solve_tuning": {"table": tune_table, "shapes": [list(v) for v in pns.TUNE_SHAPES],
                                   "bin_edges": pns.TUNE_BIN_EDGES,
                                   "source": "paper_2510_22077_gb300/tuning_gb300.json" if tune_table else
                                   "library default"}}
    if rank == 0 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S2 = pns.Solver(w.mask, w.labels, 1.0, mu, (1.0, 0.0, 0.0), variant=args.variant, precision=args.precision,
                        gj_tensor_cores=args.gj)
        if tune_table:
            S2.pns_set_tuning(tune_table)
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
        line["cpu_baseline"] = cpu_baseline(w, mu, its_stokes + its_newton, stored_its=(args.n == 96 and args.seed == 0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, rank 0 only (others exit).  Step k measures,
    in full, stratum k mod 20 of the local blocks (their factorisations and one solve each); the fixed
    costs (maps, assembly, Jacobian apply, Gram-Schmidt pass, coarse LU) are measured once before the
    steps.  `value` composes the time to 1e-8 from the measured parts (with --steps >= 20 every block of
    the build is measured, nothing scaled); `ms_per_step` is the measured time of one step."""
    if rank != 0:
        return
    w, mu = workload(args, 0)
    from oracle import krylov, mac
    pb = krylov.Problem(w.mask, w.labels, mac.Params(1.0, mu, (1.0, 0.0, 0.0)))
    info = {"n_unknowns": int(len(pb.g.unknown)), "n_prim": int(pb.maps.n_prim), "n_iface": int(pb.maps.n_iface),
            "prim_sum_n2": float(sum(len(P) ** 2 for P in pb.maps.prim_unknowns))}
    del pb
    its, its_src = oracle_iterations() if args.n == 96 and args.seed == 0 else (None, None)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded sphere pack)", "impl": "reference", "config": config(args, w, info)}
    if its is None:
        line.update({"value": None, "ms_per_step": None,
                     "unavailable": "no stored oracle solve of this workload (tests/golden/spheres96_solve.json "
                                    "covers the 96^3 pack, seed 0) to take the oracle's iteration count from"})
        print(json.dumps(line), flush=True)
        return
    strata = [k % N_STRATA for k in range(max(1, args.steps))]
    uniq = sorted(set(strata))
    recs, summ = run_oracle(w, mu, uniq, warmup=args.warmup, mt_workers=0, timeout=7200)
    by = {r["stratum"]: r for r in recs}
    step_s = [by[k]["wall_s"] for k in strata]
    total, build, it, scale = compose_oracle([by[k] for k in uniq], summ, its, its_src)
    ms_step = 1e3 * sum(step_s) / len(step_s)
    v = total * 1e3
    cb = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": (f"each step: one of {N_STRATA} strata of the local blocks (dealt in snake order over the size "
                     f"ranking) factorised and solved in full by the oracle, 1 thread; {len(uniq)} strata measured "
                     f"({'all blocks, nothing scaled' if scale == 1 else f'scaled x{scale:g}'}); fixed costs measured "
                     f"once: maps {summ['maps_s']:.1f} s, assembly {summ['asm_s']:.1f} s, Jacobian apply "
                     f"{summ['jac_s'] * 1e3:.0f} ms, Gram-Schmidt pass {summ['orth50_s'] * 1e3:.0f} ms; value = maps + "
                     f"assembly + 2 builds ({build:.0f} s each) + {its} FGMRES iterations ({it:.2f} s each; {its_src})")}
    line.update({"value": v, "ms_per_step": ms_step, "cpu_baseline": cb,
                 "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
