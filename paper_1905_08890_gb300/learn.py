"""The learned initial guess: training set, training and warm-started solves.

Training pairs are (sources -> converged fields) at 128^3 from the seeded
Zel'dovich generator with lognormal rms delta drawn uniformly in [0.3, 3] per
seed and rms |u| = 0.003; the targets come from the library's own solver
(double-float mixed precision, relative residual 1e-8).  Train, validation
and test seeds are disjoint (1000-2799, 2800-2999, 5000-5099).  Sources are
regenerated from their seeds at every use (particle drawing and deposit take
milliseconds on the GPU); targets are kept on the GPU in BF16.

    python -m paper_1905_08890_gb300.learn --train 1800 --epochs 12 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import gr, synth

N = 128
V_RMS = 0.003
SIGMA_RANGE = (0.3, 3.0)
TRAIN_SEEDS = range(1000, 2800)
VAL_SEEDS = range(2800, 3000)
TEST_SEEDS = range(5000, 5100)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet128.npz")
SOLVE_OPTS = dict(tol=1e-8, max_cycles=60, prec="mixed_df")


def sigma_of(seed: int) -> float:
    lo, hi = SIGMA_RANGE
    return float(np.random.default_rng(seed + 7919).uniform(lo, hi))


def sources(ctx: gr.Context, seed: int, src=None):
    """Deposit the particles of one seed; returns (sources, rho_hat)."""
    x, u, mass = synth.zeldovich_torch(ctx.n, seed, sigma_of(seed), V_RMS, True)
    src = ctx.deposit(x, u, mass, src)
    return src, mass * ctx.n ** 3


def solve(ctx: gr.Context, src, rho, guess=None, **kw):
    fld = guess if guess is not None else ctx.initial_fields()
    opts = dict(SOLVE_OPTS, rho_hat=rho)
    opts.update(kw)
    rep = ctx.solve(src, fld, allow_noconv=True, **opts)
    return fld, rep


def _dev_stack(fld):
    import torch

    chans = [fld["psi"] - 1.0, fld["apsi"] - 1.0] + [fld[k] for k in gr.FIELDS[2:]]
    return torch.stack([c.reshape(-1) for c in chans])


def build_targets(ctx, seeds, log=print):
    """Solve every seed; returns BF16 targets [len, 10, n^3] (deviations),
    per-channel output and input statistics."""
    import torch

    n3 = ctx.n ** 3
    tg = torch.empty((len(seeds), 10, n3), dtype=torch.bfloat16, device="cuda")
    s_out, s2_out = torch.zeros(10, dtype=torch.float64, device="cuda"), torch.zeros(10, dtype=torch.float64,
                                                                                      device="cuda")
    s_in, s2_in = torch.zeros(4, dtype=torch.float64, device="cuda"), torch.zeros(4, dtype=torch.float64,
                                                                                   device="cuda")
    src = ctx.new_sources()
    t0 = time.time()
    for k, seed in enumerate(seeds):
        src, rho = sources(ctx, seed, src)
        fld, rep = solve(ctx, src, rho)
        d = _dev_stack(fld)
        tg[k] = d.to(torch.bfloat16)
        s_out += d.mean(dim=1)
        s2_out += (d * d).mean(dim=1)
        xin = torch.stack([torch.log(0.01 + src["s0"].reshape(-1) / rho)] +
                          [src[c].reshape(-1) / (rho * V_RMS) for c in ("sx", "sy", "sz")])
        s_in += xin.mean(dim=1)
        s2_in += (xin * xin).mean(dim=1)
        if log and (k + 1) % 200 == 0:
            log(f"targets {k + 1}/{len(seeds)} ({time.time() - t0:.0f} s)")
    m = len(seeds)
    out_mean = (s_out / m).cpu().numpy()
    out_std = np.sqrt(np.maximum((s2_out / m).cpu().numpy() - out_mean ** 2, 1e-60))
    in_mean = (s_in / m).cpu().numpy()
    in_std = np.sqrt(np.maximum((s2_in / m).cpu().numpy() - in_mean ** 2, 1e-30))
    return tg, dict(in_mean=in_mean, in_std=in_std, out_mean=out_mean, out_std=out_std)


def _target_fields(ctx, row, out):
    for k, name in enumerate(gr.FIELDS):
        v = row[k].to(out[name].dtype).reshape(out[name].shape)
        out[name].copy_(v + 1.0 if k < 2 else v)
    return out


def train(net: gr.Net, ctx: gr.Context, seeds, targets, epochs=3, lr=1e-3, max_seconds=None, log=print, val=None):
    """Adam on the standardised MSE, cosine learning-rate decay; returns the
    per-epoch mean training loss (and validation loss when val=(seeds, targets))."""
    import torch

    rng = np.random.default_rng(0)
    total = epochs * len(seeds)
    step = 0
    hist = []
    src = ctx.new_sources()
    tgt = ctx.initial_fields()
    t0 = time.time()
    for ep in range(epochs):
        losses = []
        for i in rng.permutation(len(seeds)):
            src, rho = sources(ctx, seeds[i], src)
            _target_fields(ctx, targets[i], tgt)
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            losses.append(net.train_step(src, tgt, rho, V_RMS, max(cur, 1e-6)))
            step += 1
            if max_seconds and time.time() - t0 > max_seconds:
                break
        entry = {"epoch": ep, "train_loss": float(np.mean(losses)), "steps": step, "seconds": time.time() - t0}
        if val is not None:
            entry["val_loss"] = validate(net, ctx, *val)
        hist.append(entry)
        if log:
            log(json.dumps(entry))
        if max_seconds and time.time() - t0 > max_seconds:
            break
    torch.cuda.synchronize()
    return hist


def validate(net, ctx, seeds, targets):
    src = ctx.new_sources()
    tgt = ctx.initial_fields()
    ls = []
    for i, seed in enumerate(seeds):
        src, rho = sources(ctx, seed, src)
        _target_fields(ctx, targets[i], tgt)
        ls.append(net.loss_grad(src, tgt, rho, V_RMS, want_grads=False)[0])
    return float(np.mean(ls))


def save(path, net: gr.Net, stats: dict, meta: dict | None = None):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez_compressed(path, params=net.get_params(), meta=json.dumps(meta or {}), **stats)


def load(path, n=N, seed=0) -> gr.Net:
    d = np.load(path)
    net = gr.Net(n, seed=seed)
    net.set_params(d["params"])
    net.set_norm(d["in_mean"], d["in_std"], d["out_mean"], d["out_std"])
    return net


def warm_solve(ctx, net, src, rho, **kw):
    """Network guess, then the solve with the guess check (fallback to the
    plain guess per equation); returns (fields, report, inference seconds)."""
    import torch

    fld = ctx.initial_fields()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.infer(src, fld, rho, V_RMS)
    e1.record()
    torch.cuda.synchronize()
    t_inf = e0.elapsed_time(e1) * 1e-3
    fld, rep = solve(ctx, src, rho, guess=fld, check_guess=1, **kw)
    return fld, rep, t_inf


def evaluate(ctx, net, seeds, log=print):
    """Per held-out seed: V-cycles and solve time from the plain guess and
    from the network's guess (with fallback), and the network's error
    against the plain solve per field (relative L-infinity)."""
    import torch

    rows = []
    src = ctx.new_sources()
    for seed in seeds:
        src, rho = sources(ctx, seed, src)
        t0 = time.perf_counter()
        ref, rp = solve(ctx, src, rho)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        guess = ctx.initial_fields()
        net.infer(src, guess, rho, V_RMS)
        err = {k: float(((guess[k] - ref[k]).abs().max() / (ref[k] - (1.0 if k in ("psi", "apsi") else 0.0)).abs()
                         .max().clamp_min(1e-300)).item()) for k in gr.FIELDS}
        t0 = time.perf_counter()
        fld, rw, t_inf = warm_solve(ctx, net, src, rho)
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t0
        diff = max(float(((fld[k] - ref[k]).abs().max() / ref[k].abs().max().clamp_min(1e-300)).item())
                   for k in gr.FIELDS)
        rows.append({"seed": seed, "sigma": sigma_of(seed), "cycles_plain": sum(rp["cycles"]),
                     "cycles_warm": sum(rw["cycles"]), "rejected": sum(rw["guess_rejected"]),
                     "s_plain": t_plain, "s_warm": t_warm, "s_infer": t_inf, "net_rel_err": err,
                     "max_rel_diff_solutions": diff})
        if log:
            log(json.dumps({k: rows[-1][k] for k in ("seed", "cycles_plain", "cycles_warm", "rejected",
                                                      "s_plain", "s_warm")}))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=len(TRAIN_SEEDS))
    ap.add_argument("--val", type=int, default=40)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--max-minutes", type=float, default=None)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    import torch

    ctx = gr.Context(N)
    t0 = time.time()
    train_seeds = list(TRAIN_SEEDS)[:args.train]
    val_seeds = list(VAL_SEEDS)[:args.val]
    targets, stats = build_targets(ctx, train_seeds)
    vtargets, _ = build_targets(ctx, val_seeds, log=None)
    t_data = time.time() - t0
    net = gr.Net(N, seed=1)
    net.set_norm(stats["in_mean"], stats["in_std"], stats["out_mean"], stats["out_std"])
    hist = train(net, ctx, train_seeds, targets, epochs=args.epochs, lr=args.lr,
                 max_seconds=args.max_minutes * 60 if args.max_minutes else None, val=(val_seeds, vtargets))
    t_train = time.time() - t0 - t_data
    meta = {"train_seeds": [train_seeds[0], train_seeds[-1]], "epochs": hist[-1]["epoch"] + 1 if hist else 0,
            "history": hist, "data_seconds": t_data, "train_seconds": t_train, "n": N, "v_rms": V_RMS,
            "sigma_range": SIGMA_RANGE}
    save(args.out, net, stats, meta)
    del targets, vtargets
    torch.cuda.empty_cache()
    rows = evaluate(ctx, net, list(TEST_SEEDS)[:args.test])
    untrained = gr.Net(N, seed=2)
    untrained.set_norm(stats["in_mean"], stats["in_std"], stats["out_mean"], stats["out_std"])
    rows_u = evaluate(ctx, untrained, list(TEST_SEEDS)[:min(args.test, 5)], log=None)
    summary = {"meta": meta, "test": rows, "untrained": rows_u}
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(summary, fh)
    print(json.dumps({"cycles_plain": sum(r["cycles_plain"] for r in rows),
                      "cycles_warm": sum(r["cycles_warm"] for r in rows),
                      "cycles_warm_untrained": sum(r["cycles_warm"] for r in rows_u),
                      "s_plain": sum(r["s_plain"] for r in rows), "s_warm": sum(r["s_warm"] for r in rows),
                      "data_s": t_data, "train_s": t_train}))


if __name__ == "__main__":
    main()
