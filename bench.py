"""Benchmark: CIC deposit + ten-equation constraint solve to relative residual 1e-8.

One step = deposit of the resident particles, reset of the ten fields to the
plain guess (psi = alpha psi = 1, vectors 0) and the full solve.  The
headline path is the mixed-precision solve (defect correction with the fine
residual in double-float, FP32 correction V-cycles); the plain FP64 GPU
solve of the same step is timed next to it, and so is the same solve started by
one full multigrid cycle per equation (a classical non-learned warm start),
the composite solve with two static nested refinement patches (128^3 at
2x and 4x the base resolution, centred on the densest cell), and the full
timestep of the time loop (deposit with the previous conformal factor, solve
from the previous solution, kicks and drift of the particles).  The CPU
oracle's bounded sample and its own time to residual run in a separate
process that never initialises CUDA.
Multi-GPU runs are independent replicas (one problem per rank, different
seeds: weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec mixed_df|mixed|fp64]
                    [--no-fp64] [--no-fmg] [--no-e2e] [--no-learned] [--no-patches] [--no-cpu]
                    [--no-cpu-solve] [--no-timestep]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-residual-1e-8 per 10-eq solve & Gcell-updates/s: learned+FP32 vs plain FP64"
UNIT = "Gcell-updates/s"
DEFAULT_WORKLOAD = "zeldovich512_lognormal5"

# algorithmic bytes per finest-level cell and launch, per profiled kernel
# class and equation kind (split layout: a colour pass touches half the cells)
BYTES = {
    # class: {kind: bytes per finest-level cell}
    "sweep32": {"poisson": 6.0, "helm": 8.0},  # one colour pass
    "smooth3": {"poisson": 10.0, "helm": 14.0},  # three colour passes fused: other colour + f (+ inv) in, e out
    "sweep64": {"poisson": 12.0, "helm": 16.0, "psi": 24.0},
    "resid_restrict32": {"poisson": 9.0, "helm": 13.0},
    "resid_restrict32_red": {"poisson": 7.0, "helm": 9.0},  # red children only, after a black pass
    "resid_restrict64": {"poisson": 18.0, "helm": 26.0, "psi": 35.0},
    "prolong32": {"any": 4.5},  # black children only (a red pass follows)
    "prolong64": {"any": 17.0},
    "mixed_resid": {"poisson": 20.0, "helm": 28.0, "psi": 44.0},
    "df_resid": {"poisson": 22.0, "helm": 32.0, "psi": 46.0},  # + the first red pass of the next cycle
    "mixed_update": {"any": 20.0},
    "df_black_update": {"poisson": 20.0, "helm": 22.0},  # last black pass + update of both colours
    "norm64": {"poisson": 16.0, "helm": 24.0, "psi": 32.0},
}
EQ_KIND = ["poisson"] * 4 + ["psi", "helm"] + ["poisson"] * 4
EQ_KIND32 = ["poisson"] * 4 + ["helm", "helm"] + ["poisson"] * 4


def class_bytes(cls, cycles, n, nu1, nu2, prec, fused=False):
    """Algorithmic bytes of every finest-level launch of one profiled class
    over a solve with the given per-equation cycle counts (n >= 8, nu1, nu2 >= 1).
    In the double-float mode the residual kernel also makes the first red
    pass of each cycle and the last black pass is fused with the update.
    fused: three of the colour passes of each smoothing (nu1 = nu2 = 2) run as
    one fused launch (class smooth3)."""
    mixed, dfm = prec != "fp64", prec == "mixed_df"
    cells = float(n) ** 3
    total = 0.0
    for eq, cyc in enumerate(cycles):
        k64, k32 = EQ_KIND[eq], EQ_KIND32[eq]
        if cls == "sweep32" and mixed:
            passes = 2 * (nu1 + nu2) - (2 if dfm else 0) - (6 if fused else 0)
            total += cyc * passes * BYTES["sweep32"][k32] * cells
        elif cls == "smooth3" and mixed and fused:
            total += cyc * 2 * BYTES["smooth3"][k32] * cells
        elif cls == "sweep64" and not mixed:
            total += cyc * 2 * (nu1 + nu2) * BYTES["sweep64"][k64] * cells
        elif cls == "resid_restrict":
            key = "resid_restrict32_red" if mixed else "resid_restrict64"
            total += cyc * BYTES[key][k32 if mixed else k64] * cells
        elif cls == "prolong":
            total += cyc * BYTES["prolong32" if mixed else "prolong64"]["any"] * cells
        elif cls == "mixed_resid" and mixed:
            total += (cyc + 1) * BYTES["df_resid" if dfm else "mixed_resid"][k64] * cells
        elif cls == "mixed_update" and mixed:
            total += cyc * (BYTES["df_black_update"][k32] if dfm else BYTES["mixed_update"]["any"]) * cells
        elif cls == "norm64" and not mixed:
            total += (cyc + 1) * BYTES["norm64"][k64] * cells
    return total


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 7:
                continue
            try:
                sm.append(float(row[0]))
                smax = float(row[1])
            except ValueError:
                continue
            for nm, v in zip(names, row[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(n, src_np, rho_hat, cycles=1, repeats=3, warm=True):
    """Time the FP64 CPU oracle (as it stands) on a bounded sample of the
    workload: `cycles` V(2,2) cycles of the V_x and psi equations at the full
    grid, from the plain guess.  One untimed sample warms the host (page
    faults, thread start-up) unless warm is False, then `repeats` timed samples; returns
    (median Gcell-updates/s, seconds of the median sample, threads, all rates)."""
    import numpy as np

    import oracle

    cells_per_cycle = sum(4 * (n >> l) ** 3 for l in range(0, int(math.log2(n)) - 1)) + 32 * 8
    fld = oracle.initial_fields(n)
    setups = [oracle.eq_setup(eq, src_np, fld, rho_hat) for eq in (0, 4)]
    rates, secs = [], []
    first = 0 if warm else 1
    for rep in range(first, repeats + 1):
        t_total, updates = 0.0, 0
        for kind, f, c0, c1, ref in setups:
            u = np.zeros((n, n, n))
            t0 = time.perf_counter()
            for _ in range(cycles):
                oracle.vcycle(kind, u, f, c0, c1, rho_hat)
            t_total += time.perf_counter() - t0
            updates += cycles * cells_per_cycle
        if rep:  # the first sample is the untimed warm-up
            rates.append(updates / t_total / 1e9)
            secs.append(t_total)
    order = sorted(range(repeats), key=lambda i: rates[i])
    mid = order[repeats // 2]
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return rates[mid], secs[mid], threads, rates


def oracle_time_to_residual(src_np, rho_hat, tol):
    """The FP64 CPU oracle's ten-equation solve of the bench's own sources from
    the plain guess to relative residual tol (every field): wall seconds,
    cycles and the cell updates it made (same counting as the GPU report)."""
    import oracle

    n = src_np["s0"].shape[0]
    fld = oracle.initial_fields(n)
    t0 = time.perf_counter()
    st, rep = oracle.solve_constraints(src_np, fld, rho_hat, tol=tol, max_cycles=60)
    secs = time.perf_counter() - t0
    per_cycle = sum(4 * (n >> l) ** 3 for l in range(0, int(math.log2(n)) - 1)) + 32 * 8
    updates = sum(rep["cycles"]) * per_cycle
    return st, secs, rep["cycles"], updates


def profile_case(case, n=None):
    """One small workload for an ncu capture (two or three repetitions after the
    set-up; prints one line of CUDA-event timings, not a bench value):
      mixed      the headline double-float solve at n^3 (default 128), lognormal rms 5, tol 1e-8
      fp64       the plain FP64 solve at n^3 (default 128: lognormal rms 1, rms |u| 0.003, tol 1e-10)
      unet       three inferences of the trained network at 128^3 (held-out seed 5000)
      particles  three particle updates and three deposits with the metric at n^3 (default 512)
      fma        the FP64 and FP32 FMA issue rates of the GPU (gr_fma_rate)"""
    import torch

    from paper_1905_08890_gb300 import gr, learn, synth

    torch.cuda.set_device(0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = []

    def timed(fn, reps):
        for _ in range(reps):
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize()
            out.append(round(ev[0].elapsed_time(ev[1]), 3))

    if case == "fma":
        # FMA issue rates (FP64, FP32) over the whole GPU: the denominators of
        # the ALU-bound rooflines
        rates = {k: round(gr.gr_fma_rate(k == "fp64", 1 << 17) / 1e12, 3) for k in ("fp64", "fp32")}
        print(json.dumps({"case": case, "fma_tflops": rates}))
        return
    if case == "unet":
        ctx = gr.Context(learn.N)
        net = learn.load(learn.WEIGHTS)
        src, rho = learn.sources(ctx, 5000)
        fld = ctx.initial_fields()
        timed(lambda: net.infer(src, fld, rho, learn.V_RMS), 3)
        print(json.dumps({"case": case, "n": learn.N, "inference_ms": out}))
        return
    fp64 = case == "fp64"
    n = n or (512 if case == "particles" else 128)
    seed, sigma, tol = (2, 1.0, 1e-10) if fp64 else (4, 5.0, 1e-8)
    x, u, mass = synth.zeldovich_torch(n, seed, sigma, 0.003, True)
    ctx = gr.Context(n)
    src = ctx.deposit(x, u, mass)
    opts = dict(tol=tol, max_cycles=60, prec="fp64" if fp64 else "mixed_df", rho_hat=mass * n ** 3)
    fld = ctx.initial_fields()
    if case in ("mixed", "fp64"):
        timed(lambda: ctx.solve(src, ctx.initial_fields(), **opts), 2)
        print(json.dumps({"case": case, "n": n, "solve_ms": out}))
        return
    ctx.solve(src, fld, **opts)
    dt = 0.05 / n / 0.003
    timed(lambda: ctx.particle_update(x, u, fld, dt), 3)
    timed(lambda: ctx.deposit_metric(x, u, mass, fld["psi"], src), 3)
    print(json.dumps({"case": case, "n": n, "particle_update_ms": out[:3], "deposit_metric_ms": out[3:]}))


def cpu_worker(folder):
    """The CPU legs in a process of their own that never touches CUDA (so the
    oracle runs on the host as it does in the reference arm): the bounded
    sample and, if asked, the full time-to-residual solve, on the sources
    saved in folder; prints one JSON line."""
    import numpy as np

    meta = json.load(open(os.path.join(folder, "meta.json")))
    src = {k: np.load(os.path.join(folder, k + ".npy")) for k in ("s0", "sx", "sy", "sz", "sigma")}
    n = src["s0"].shape[0]
    val, secs, thr, rates = oracle_sample(n, src, meta["rho_hat"])
    res = {"value": val, "secs": secs, "threads": thr, "rates": rates}
    if meta["solve"]:
        st, osecs, ocyc, oupd = oracle_time_to_residual(src, meta["rho_hat"], meta["tol"])
        res.update(solve_status=st, solve_secs=osecs, solve_cycles=ocyc, solve_updates=oupd)
    print(json.dumps(res), flush=True)


def cpu_legs(src, rho_hat, tol, n, gpu_solve_ms, solve):
    """Save the bench's sources, run cpu_worker in a fresh interpreter, and
    shape its results into the cpu_baseline / cpu_time_to_residual keys."""
    import shutil
    import tempfile

    import numpy as np

    folder = tempfile.mkdtemp(prefix="gr_cpu_")
    try:
        for k, v in src.items():
            np.save(os.path.join(folder, k + ".npy"), v.cpu().numpy())
        json.dump({"rho_hat": rho_hat, "tol": tol, "solve": bool(solve)}, open(os.path.join(folder, "meta.json"), "w"))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", folder], capture_output=True,
                           text=True, env=dict(os.environ))
        if r.returncode != 0:
            return {"cpu_baseline": {"error": r.stderr[-500:]}}
        w = json.loads(r.stdout.strip().splitlines()[-1])
    finally:
        shutil.rmtree(folder, ignore_errors=True)
    out = {"cpu_baseline": {"value": round(w["value"], 5), "unit": UNIT, "cores": w["threads"], "kind": "oracle",
                            "sample": f"one V(2,2) cycle each of the V_x and psi equations at {n}^3 from the plain "
                                      f"guess, median of {len(w['rates'])} after one untimed sample ({w['secs']:.1f} s "
                                      f"each; rates {[round(x, 4) for x in w['rates']]}), in a process without CUDA"}}
    if solve:
        out["cpu_time_to_residual"] = {
            "ms": round(1e3 * w["solve_secs"], 1), "status": w["solve_status"], "cycles": w["solve_cycles"],
            "threads": w["threads"], "n": n, "gcell_updates_per_s": round(w["solve_updates"] / w["solve_secs"] / 1e9, 4),
            "vs_gpu_time_to_residual": round(1e3 * w["solve_secs"] / gpu_solve_ms, 1),
            "what": f"FP64 CPU oracle, ten-equation solve of this workload's sources to {tol:g} from the plain guess"}
    return out


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="mixed_df", choices=["mixed_df", "mixed", "fp64"])
    ap.add_argument("--no-fmg", action="store_true", help="skip the full multigrid start comparison")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-cpu-solve", action="store_true",
                    help="skip the CPU oracle's full time-to-residual solve (about a minute at 512^3)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-timestep", action="store_true", help="skip the full timestep (deposit, solve, particle update)")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--case", default=None, choices=["mixed", "fp64", "unet", "particles", "fma"],
                    help="run one small profiling case instead of the bench (the commands of profiles/*.md)")
    ap.add_argument("--n", type=int, default=None, help="grid of --case")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-guess comparison at 128^3")
    ap.add_argument("--no-patches", action="store_true",
                    help="skip the composite solve with two nested 128^3 refinement patches")
    args = ap.parse_args()
    if args.cpu_worker:
        return cpu_worker(args.cpu_worker)
    if args.case:
        return profile_case(args.case, args.n)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

    from paper_1905_08890_gb300 import synth

    w = synth.WORKLOADS[args.workload]
    n, tol = w["n"], w["tol"]
    config = {"workload": args.workload, "n": n, "particles": n ** 3, "delta": ("lognormal" if w["lognormal"] else
              "gaussian") + f" rms {w['sigma']}", "v_rms": w["v_rms"], "tol": tol, "cycle": "V(2,2) red-black GS",
              "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        return run_reference(args, rank, world, n, w, config)

    import torch

    from paper_1905_08890_gb300 import gr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    p = synth.zeldovich(n, replica_seed(w["seed"], rank), w["sigma"], w["v_rms"], w["lognormal"])
    ctx = gr.Context(n)
    x = torch.from_numpy(p.x).cuda()
    u = torch.from_numpy(p.u).cuda()
    src = ctx.new_sources()
    fld = ctx.initial_fields()
    opts = dict(tol=tol, max_cycles=60, prec=args.prec, rho_hat=p.rho_hat)

    dep_ev = []

    def step(profile=0):
        if profile:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.deposit(x, u, p.mass, src)
            e1.record()
            dep_ev.append((e0, e1))
        else:
            ctx.deposit(x, u, p.mass, src)
        fld["psi"].fill_(1.0)
        fld["apsi"].fill_(1.0)
        for k in ("Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b"):
            fld[k].zero_()
        return ctx.solve(src, fld, profile=profile, **opts)

    for _ in range(args.warmup):
        step()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)  # let the sampler start before the timed region
    barrier()
    launches0 = gr.gr_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    reps = [step(profile=1) for _ in range(args.steps)]
    ev1.record()
    barrier()
    clk = clocks.stop()
    launches = gr.gr_kernel_launches() - launches0
    value, ms = job_throughput(sum(r["cell_updates"] for r in reps), ev0.elapsed_time(ev1), dist, "cuda")
    solve_ms = 1e3 * sum(sum(r["eq_seconds"]) for r in reps) / len(reps)

    # per-class roofline over the timed region
    mixed = args.prec != "fp64"
    hbm, peak_kind = peaks()
    kernels = {}
    fused = any(r["prof"]["smooth3"]["launches"] > 0 for r in reps)
    for cls, d in reps[0]["prof"].items():
        tot_ms = sum(r["prof"][cls]["ms"] for r in reps)
        launches_c = sum(r["prof"][cls]["launches"] for r in reps)
        if launches_c == 0:
            continue
        if cls in ("setup", "coarse", "patch"):
            kernels[cls] = {"launches": launches_c, "ms": round(tot_ms, 3), "share_of_step": round(tot_ms / ms, 3)}
            continue
        byt = sum(class_bytes(cls, r["cycles"], n, 2, 2, args.prec, fused) for r in reps)
        gbs = byt / (tot_ms * 1e-3) / 1e9
        kernels[cls] = {"launches": launches_c, "ms": round(tot_ms, 3), "avg_us": round(1e3 * tot_ms / launches_c, 2),
                        "algorithmic_GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm, 3),
                        "share_of_step": round(tot_ms / ms, 3)}
    dep_ms = sum(a.elapsed_time(b) for a, b in dep_ev)
    kernels["deposit"] = {"launches": len(dep_ev), "ms": round(dep_ms, 3),
                          "avg_us": round(1e3 * dep_ms / max(len(dep_ev), 1), 2),
                          "algorithmic_GBps": round((48 + 40) * n ** 3 * len(dep_ev) / (dep_ms * 1e-3) / 1e9, 1),
                          "frac_hbm": round((48 + 40) * n ** 3 * len(dep_ev) / (dep_ms * 1e-3) / 1e9 / hbm, 3),
                          "share_of_step": round(dep_ms / ms, 3)}
    dom = (max((k for k in kernels if k not in ("coarse", "deposit", "patch")), key=lambda k: kernels[k]["ms"])
           if kernels else None)
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if dom and os.path.exists(tpath):
        tj = json.load(open(tpath))
        ent = tj.get(dom)
        if ent and ent.get("n") == n and ent.get("source_hash") == _source_hash(ent.get("files"), ent.get("function")):
            traffic = ent["bytes_per_launch"]
    roofline = None
    if dom:
        avg_bytes = class_bytes(dom, reps[0]["cycles"], n, 2, 2, args.prec, fused) / reps[0]["prof"][dom]["launches"]
        roofline = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["algorithmic_GBps"], "peak": hbm,
                    "unit": "GB/s", "frac": kernels[dom]["frac_hbm"], "traffic": traffic,
                    "algorithmic_bytes_per_launch": round(avg_bytes), "peak_source": f"{peak_kind} hbm_gbs"}

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"mixed_df": "f32 pairs + f32", "mixed": "f64 + f32", "fp64": "f64"}[args.prec],
           "data": "synthetic (seeded Zel'dovich particles)", "config": config,
           "time_to_residual_ms": round(solve_ms, 3), "path": args.prec, "learned": None,
           "cycles": reps[-1]["cycles"], "res": [float(f"{r:.3e}") for r in reps[-1]["res"]],
           # the same cell updates over the solve alone (no deposit, no field reset), and the
           # fine-equivalent rate: n^3 cells times the cycles of all ten equations per solve second
           "solve_gcell_updates_per_s": round(sum(r["cell_updates"] for r in reps) / len(reps)
                                              / (solve_ms * 1e-3) / 1e9 * world, 3),
           "fine_equivalent_gcells_per_s": round(float(n) ** 3 * sum(reps[-1]["cycles"]) / (solve_ms * 1e-3) / 1e9
                                                 * world, 3),
           "gpu_launches": int(launches), "roofline": roofline, "kernels": kernels, "clocks": clk}

    # the end-to-end measurement runs first, on the state the timed steps left
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_measure(ctx, p, n, opts, world, max(args.steps, 5))

    if rank == 0 and not args.no_fp64 and mixed:
        mixed_fields = {k: v.clone() for k, v in fld.items()}
        o64 = dict(opts, prec="fp64")
        ctx.deposit(x, u, p.mass, src)
        fld64 = ctx.initial_fields()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        r64 = ctx.solve(src, fld64, **o64)
        t1.record()
        torch.cuda.synchronize()
        ms64 = t0.elapsed_time(t1)
        diff = {k: float((mixed_fields[k] - fld64[k]).abs().max() / fld64[k].abs().max().clamp_min(1e-300))
                for k in fld64}
        out["fp64"] = {"time_to_residual_ms": round(ms64, 3),
                       "gcell_updates_per_s": round(r64["cell_updates"] / (ms64 * 1e-3) / 1e9, 3),
                       "cycles": r64["cycles"], "speedup_mixed_vs_fp64": round(ms64 / solve_ms, 3),
                       "max_rel_linf_mixed_vs_fp64": max(diff.values())}
        del fld64, mixed_fields

    if rank == 0 and not args.no_fmg and mixed:
        out["fmg_start"] = fmg_measure(ctx, x, u, p, src, fld, opts)

    if rank == 0 and mixed and not args.no_timestep:
        out["timestep"] = timestep_measure(ctx, x, u, p, fld, opts, n)

    if rank == 0 and not args.no_patches and n >= 256:
        out["patches"] = patches_measure(ctx, x, u, p, src, fld, opts, n)

    if rank == 0 and not args.no_learned:
        out["learned"] = learned_measure(args.prec)
        if mixed and n > 128:
            ctx.deposit(x, u, p.mass, src)
            out["learned_full"] = learned_full_measure(ctx, p, src, fld, opts, n)

    if rank == 0 and world == 1 and not args.no_cpu:
        out.update(cpu_legs(src, p.rho_hat, tol, n, solve_ms, not args.no_cpu_solve))
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank solves its own problem (weak scaling): rank r draws seed base + 1000 r."""
    return base_seed + 1000 * rank


def job_throughput(cell_updates: int, ms: float, dist=None, device="cpu"):
    """Whole-job Gcell-updates/s: cell updates summed over the ranks divided by
    the slowest rank's time (max over ranks).  Returns (value, max ms)."""
    if dist is not None:
        import torch

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([float(cell_updates)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, cell_updates = float(t.item()), float(u.item())
    return cell_updates / (ms * 1e-3) / 1e9, ms


def e2e_measure(ctx, p, n, opts, world, steps):
    """The same metric through the public API with host buffers: each step
    hands the particles in pinned host memory to gr_deposit (which streams
    them to the GPU in chunks, each copy overlapping the previous chunk's
    deposit) and solves with gr_opts.host_out, so that each field is read back
    into pinned host memory while the later equations solve; the step ends
    when the last field has arrived (stream synchronisation)."""
    import torch

    xh = torch.from_numpy(p.x).pin_memory()
    uh = torch.from_numpy(p.u).pin_memory()
    host_out = {k: torch.empty((n, n, n), dtype=torch.float64).pin_memory() for k in
                ("psi", "apsi", "Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b")}
    src = ctx.new_sources()
    fld = ctx.initial_fields()  # device fields, reset to the plain guess in every step
    o = dict(opts, host_out=host_out)
    # host link rates seen by this run (the copies share the machine's host links with other jobs)
    probe_d = torch.empty_like(host_out["psi"], device="cuda")
    rates = {}
    for name, (dst, srcb) in {"h2d_GBps": (probe_d, host_out["psi"]), "d2h_GBps": (host_out["psi"], probe_d)}.items():
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(srcb, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            best = max(best, dst.numel() * 8 / (a.elapsed_time(b) * 1e-3) / 1e9)
        rates[name] = round(best, 1)
    del probe_d
    ctx.deposit(xh, uh, p.mass, src)  # untimed: the context allocates its staging buffers on first use
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    updates = 0
    per_step, phases = [], []
    for _ in range(steps):
        ts = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        ctx.deposit(xh, uh, p.mass, src)
        ev[1].record()
        fld["psi"].fill_(1.0)
        fld["apsi"].fill_(1.0)
        for k in ("Vx", "Vy", "Vz", "U", "Bx", "By", "Bz", "b"):
            fld[k].zero_()
        r = ctx.solve(src, fld, **o)
        ev[2].record()  # after the solve's stream has waited for the last host_out copy
        updates += r["cell_updates"]
        torch.cuda.current_stream().synchronize()
        per_step.append(round(1e3 * (time.perf_counter() - ts), 1))
        dep, rest = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        solve = 1e3 * sum(r["eq_seconds"])
        phases.append({"deposit_from_host_ms": round(dep, 1), "solve_ms": round(solve, 1),
                       "copy_tail_ms": round(max(rest - solve, 0.0), 1)})
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    med = sorted(per_step)[len(per_step) // 2]
    return {"value": round(updates * world / dt / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": 48 * n ** 3,
            "d2h_bytes_per_step": 80 * n ** 3, "steps": steps, "ms_per_step": round(1e3 * dt / steps, 3),
            "ms_each_step": per_step, "median_ms_per_step": med, "phases_each_step": phases,
            "link_rates_before_steps": rates, "clocks": clk}


def fmg_measure(ctx, x, u, p, src, fld, opts):
    """The same workload with the full multigrid start (gr_opts.fmg, a
    classical non-learned warm start): one untimed and one timed solve from
    the plain guess, CUDA events; fields compared with the headline solve's."""
    import torch

    ref = {k: v.clone() for k, v in fld.items()}
    o = dict(opts, fmg=1)
    for it in range(2):
        ctx.deposit(x, u, p.mass, src)
        f2 = ctx.initial_fields()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        rep = ctx.solve(src, f2, **o)
        t1.record()
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    diff = max(float((f2[k] - ref[k]).abs().max() / ref[k].abs().max().clamp_min(1e-300)) for k in ref)
    del f2, ref
    return {"time_to_residual_ms": round(ms, 3), "cycles": rep["cycles"],
            "gcell_updates_per_s": round(rep["cell_updates"] / (ms * 1e-3) / 1e9, 3),
            "max_rel_linf_vs_headline": diff}


def patches_measure(ctx, x, u, p, src, fld, opts, n, sizes=(128, 128)):
    """The full-scale configuration with static nested refinement patches:
    two 128^3 patches at 2x and 4x the base resolution centred on the densest
    base cell, composite solve to the same tolerance.
    One untimed and one timed run from the plain guess (CUDA events), next to
    the base-only headline solve's fields."""
    import torch

    from paper_1905_08890_gb300 import gr

    ctx.deposit(x, u, p.mass, src)
    c = int(torch.argmax(src["s0"]).item())
    centre = (c // (n * n), (c // n) % n, c % n)
    chain = gr.centred_chain(n, centre, sizes)
    ctx.initial_patch_fields(chain)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for it in range(2):
        for q in chain:
            for k, v in q["fld"].items():
                v.fill_(1.0 if k in ("psi", "apsi") else 0.0)
        f2 = ctx.initial_fields()
        torch.cuda.synchronize()
        ev[0].record()
        ctx.deposit_patches(chain, x, u, p.mass)
        ev[1].record()
        ev[2].record()
        rep = ctx.solve(src, f2, patches=chain, **opts)
        ev[3].record()
        torch.cuda.synchronize()
    dep_ms, ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    # a third run with the per-class CUDA events, for the patches' share (not the timed number)
    for q in chain:
        for k, v in q["fld"].items():
            v.fill_(1.0 if k in ("psi", "apsi") else 0.0)
    f3 = ctx.initial_fields()
    prof = ctx.solve(src, f3, patches=chain, profile=1, **opts)["prof"]
    del f3
    diff = max(float((f2[k] - fld[k]).abs().max() / fld[k].abs().max().clamp_min(1e-300)) for k in fld)
    psi2 = chain[-1]["fld"]["psi"]
    out = {"chain": [{"n": q["n"], "origin": q["origin"]} for q in chain], "centre_cell": list(centre),
           "time_to_residual_ms": round(ms, 3), "deposit_patches_ms": round(dep_ms, 3), "cycles": rep["cycles"],
           "patch_kernels_ms": round(prof["patch"]["ms"], 3), "patch_launches": prof["patch"]["launches"],
           "res_max_per_level": [float(f"{max(r[l] for r in rep['res_level']):.3e}") for l in range(len(sizes) + 1)],
           "base_fields_max_rel_change_vs_no_patches": diff,
           "finest_patch_psi_range": [float(psi2.min()), float(psi2.max())],
           "base_psi_range": [float(f2["psi"].min()), float(f2["psi"].max())]}
    # the plain FP64 composite solve (the comparator of the full-scale configuration), one timed run
    for q in chain:
        for k, v in q["fld"].items():
            v.fill_(1.0 if k in ("psi", "apsi") else 0.0)
    f4 = ctx.initial_fields()
    torch.cuda.synchronize()
    ev[0].record()
    rep64 = ctx.solve(src, f4, patches=chain, **dict(opts, prec="fp64"))
    ev[1].record()
    torch.cuda.synchronize()
    out["fp64_time_to_residual_ms"] = round(ev[0].elapsed_time(ev[1]), 3)
    out["fp64_cycles"] = rep64["cycles"]
    out["speedup_mixed_vs_fp64"] = round(out["fp64_time_to_residual_ms"] / ms, 3)
    del f4
    # the learned base guess (the network on the sources averaged down to its grid, interpolated
    # back up); the patches start from the plain guess; one untimed and one timed run
    net = _load_net()
    if net is not None:
        from paper_1905_08890_gb300 import learn

        for it in range(2):
            for q in chain:
                for k, v in q["fld"].items():
                    v.fill_(1.0 if k in ("psi", "apsi") else 0.0)
            f5 = ctx.initial_fields()
            torch.cuda.synchronize()
            ev[0].record()
            net.guess(n, src, f5, p.rho_hat, learn.V_RMS)
            ev[1].record()
            rep5 = ctx.solve(src, f5, patches=chain, **opts)
            ev[2].record()
            torch.cuda.synchronize()
        out["learned_time_to_residual_ms"] = round(ev[0].elapsed_time(ev[2]), 3)
        out["learned_inference_ms"] = round(ev[0].elapsed_time(ev[1]), 3)
        out["learned_cycles"] = rep5["cycles"]
        del f5
        net.close()
    del f2, chain
    return out


def _load_net():
    from paper_1905_08890_gb300 import learn

    return learn.load(learn.WEIGHTS) if os.path.exists(learn.WEIGHTS) else None


def learned_full_measure(ctx, p, src, fld, opts, n):
    """The learned initial guess at the headline grid: the 128^3 network runs
    on the sources averaged down to its grid and its ten fields are
    interpolated back to n^3 (gr_net_guess); the solve then starts from them
    with the per-equation guess check.  Against the plain guess and the full
    multigrid start, same sources, one untimed and one timed pass (CUDA
    events); the guess's error per field against the converged solution."""
    import torch

    from paper_1905_08890_gb300 import learn

    net = _load_net()
    if net is None:
        return {"unavailable": "no trained weights"}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    for it in range(2):
        fp = ctx.initial_fields()
        fl = ctx.initial_fields()
        ff = ctx.initial_fields()
        torch.cuda.synchronize()
        ev[0].record()
        rp = ctx.solve(src, fp, **opts)
        ev[1].record()
        net.guess(n, src, fl, p.rho_hat, learn.V_RMS)
        ev[2].record()
        guess = {k: v.clone() for k, v in fl.items()}
        ev[3].record()
        rl = ctx.solve(src, fl, check_guess=1, **opts)
        ev[4].record()
        rf = ctx.solve(src, ff, fmg=1, **opts)
        ev[5].record()
        torch.cuda.synchronize()

    def dev(k, t):
        return t - 1.0 if k in ("psi", "apsi") else t

    err = {k: float((dev(k, guess[k]) - dev(k, fp[k])).abs().max() / dev(k, fp[k]).abs().max().clamp_min(1e-300))
           for k in fp}
    inf_ms = ev[1].elapsed_time(ev[2])
    out = {"workload": "the headline workload; 128^3 network on sources averaged 4^3, fields interpolated back",
           "time_to_residual_ms_plain": round(ev[0].elapsed_time(ev[1]), 3),
           "time_to_residual_ms_learned": round(inf_ms + ev[3].elapsed_time(ev[4]), 3),
           "inference_ms": round(inf_ms, 3), "time_to_residual_ms_fmg_start": round(ev[4].elapsed_time(ev[5]), 3),
           "vcycles_plain": sum(rp["cycles"]), "vcycles_learned": sum(rl["cycles"]), "vcycles_fmg": sum(rf["cycles"]),
           "cycles_learned": rl["cycles"], "guesses_rejected": sum(rl["guess_rejected"]),
           "guess_rel_linf_error_of_deviation": {k: float(f"{v:.3g}") for k, v in err.items()}}
    del fp, fl, ff, guess
    net.close()
    return out


def timestep_measure(ctx, x, u, p, fld, opts, n, steps=5, shift_cells=0.05):
    """The full timestep of the method's time loop (Sec. 4.2 steps 3 and 5-8)
    on copies of the bench's particles: the deposit with the previous psi in
    the Lorentz factor (gr_deposit_metric), the ten-equation solve started
    from the previous solution, and the particle update (synchronising kick,
    opening kick, drift: gr_particle_update), with dt set so that particles
    at the rms speed move shift_cells cells.  One untimed opening step, then
    `steps` timed steps (CUDA events per phase on the context's stream)."""
    import torch

    from paper_1905_08890_gb300 import gr

    xs, us = x.clone(), u.clone()
    W = torch.sqrt(1.0 + (us * us).sum(0))
    dt = shift_cells / n / float(torch.sqrt(((us / W) ** 2).sum(0).mean()))
    src = ctx.new_sources()
    ctx.deposit(xs, us, p.mass, src)
    f = {k: t.clone() for k, t in fld.items()}
    ctx.solve(src, f, **opts)
    ctx.particle_update(xs, us, f, dt, gr.GR_KICK_OPEN | gr.GR_DRIFT)
    rows = []
    for it in range(steps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record()
        ctx.deposit_metric(xs, us, p.mass, f["psi"], src)
        ev[1].record()
        rep = ctx.solve(src, f, **opts)
        ev[2].record()
        ctx.particle_update(xs, us, f, dt)
        ev[3].record()
        torch.cuda.synchronize()
        if it:  # the first pass warms the update's scratch allocation
            rows.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                         ev[0].elapsed_time(ev[3]), rep["cycles"]))
    k = len(rows)
    upd_ms = sum(r[2] for r in rows) / k
    # algorithmic bytes of the update: per particle x, u read and written (96 B); per cell the
    # fields read for alpha, beta (48 B) and the FP64 scratch written (32 B), that scratch read
    # (40 B) and the 20 FP32 quantities written (80 B), and those read once by the gather (80 B)
    upd_bytes = 96 * x.shape[1] + 280 * n ** 3
    del xs, us, f, src
    return {"dt": dt, "rms_shift_cells": shift_cells, "steps": k,
            "ms_per_timestep": round(sum(r[3] for r in rows) / k, 3),
            "deposit_metric_ms": round(sum(r[0] for r in rows) / k, 3),
            "solve_ms": round(sum(r[1] for r in rows) / k, 3), "particle_update_ms": round(upd_ms, 3),
            "particle_update_algorithmic_GBps": round(upd_bytes / (upd_ms * 1e-3) / 1e9, 1),
            "cycles_each_step": [r[4] for r in rows]}


def learned_measure(prec, seeds=(5000, 5001, 5002, 5003)):
    """The learned initial guess on its own workload (128^3, lognormal rms
    delta U[0.3, 3], held-out seeds): time to residual 1e-8 and V-cycles from
    the plain guess and from the network's guess (inference included, guess
    check on), CUDA events."""
    import torch

    from paper_1905_08890_gb300 import gr, learn

    if not os.path.exists(learn.WEIGHTS):
        return {"unavailable": "no trained weights"}
    ctx = gr.Context(learn.N)
    net = learn.load(learn.WEIGHTS)
    src = ctx.new_sources()
    kw = dict(prec=prec)
    res = {"plain_ms": 0.0, "learned_ms": 0.0, "inference_ms": 0.0, "cycles_plain": 0, "cycles_learned": 0,
           "rejected": 0, "fmg_ms": 0.0, "cycles_fmg": 0}
    for rep_i in range(2):  # first pass warms up
        for k in res:
            res[k] = 0
        for seed in seeds:
            src, rho = learn.sources(ctx, seed, src)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            e[0].record()
            _, rp = learn.solve(ctx, src, rho, **kw)
            e[1].record()
            guess = ctx.initial_fields()
            e[2].record()
            _, rw, t_inf = learn.warm_solve(ctx, net, src, rho, **kw)
            e[3].record()
            e[4].record()
            _, rf = learn.solve(ctx, src, rho, fmg=1, **kw)
            e[5].record()
            torch.cuda.synchronize()
            res["plain_ms"] += e[0].elapsed_time(e[1])
            res["learned_ms"] += e[2].elapsed_time(e[3])
            res["fmg_ms"] += e[4].elapsed_time(e[5])
            res["cycles_fmg"] += sum(rf["cycles"])
            res["inference_ms"] += 1e3 * t_inf
            res["cycles_plain"] += sum(rp["cycles"])
            res["cycles_learned"] += sum(rw["cycles"])
            res["rejected"] += sum(rw["guess_rejected"])
            del guess
    k = len(seeds)
    out = {"workload": "zeldovich128, lognormal rms delta U[0.3,3], rms|u| 0.003, tol 1e-8, held-out seeds 5000-5003",
           "time_to_residual_ms_plain": round(res["plain_ms"] / k, 3),
           "time_to_residual_ms_learned": round(res["learned_ms"] / k, 3),
           "inference_ms": round(res["inference_ms"] / k, 3),
           "vcycles_plain": res["cycles_plain"] / k, "vcycles_learned": res["cycles_learned"] / k,
           "guesses_rejected": res["rejected"],
           "time_to_residual_ms_fmg_start": round(res["fmg_ms"] / k, 3), "cycles_fmg_start": res["cycles_fmg"] / k,
           "path": prec}
    net.close()
    ctx.close()
    return out


def _source_hash(files=None, kernel=None):
    """Hash of the CUDA sources a profile was taken with: the named files
    under csrc/ (all of them by default), or only the definition of one
    kernel in them.  A traffic figure is used only while that text is
    unchanged."""
    import hashlib

    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1905_08890_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        text = open(os.path.join(d, f), "rb").read()
        if kernel:
            k = text.find(f"{kernel}(".encode())
            if k < 0:
                continue
            text = text[k:text.find(b"\n}\n", k) + 3]
        h.update(text)
    return h.hexdigest()[:12]


def run_reference(args, rank, world, n, w, config):
    """The FP64 CPU oracle as it stands, on the host cores: each step is the
    bounded sample of oracle_sample (one V(2,2) cycle of V_x and psi)."""
    if rank != 0:
        return
    from paper_1905_08890_gb300 import synth

    import oracle

    p = synth.zeldovich(n, w["seed"], w["sigma"], w["v_rms"], w["lognormal"])
    src_np = oracle.deposit(n, p.x, p.u, p.mass)
    for _ in range(args.warmup):
        oracle_sample(n, src_np, p.rho_hat, repeats=1, warm=False)
    t_sum, v_sum = 0.0, []
    for _ in range(args.steps):
        v, secs, thr, _ = oracle_sample(n, src_np, p.rho_hat, repeats=1, warm=False)
        t_sum += secs
        v_sum.append(v)
    value = sum(v_sum) / len(v_sum)
    sample = f"one V(2,2) cycle each of the V_x and psi equations at {n}^3 from the plain guess"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_sum / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Zel'dovich particles)", "config": config,
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": thr, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
