"""Training data, training and evaluation of the learned tile picker.

The paper picks its spreading method and tiles by hand-tuned rules (Sec. 4.1
remark; method advice of Sec. 5.4).  The library's picker (nufft_picker_* in
include/nufft_gb300.h) is a 12 -> 64 -> 64 -> 1 perceptron that predicts
log2(execute ms) of a problem under one candidate tiling; this module

* draws problems (`sample_problems`): 2D / 3D, type 1 / 2, N_i log-uniform in
  [32, 1024], M log-uniform in [1e4, 3e7], points uniform, wrapped Gaussian
  (sigma_g log-uniform in [0.01 pi, 0.5 pi]) or an 8-component Gaussian mixture,
  eps log-uniform in [1e-12, 1e-2], single precision for eps >= 1e-6; problems
  over a work bound are redrawn so that timing every candidate stays short;
* times every candidate tiling of each problem with nufft_autotune, at the
  upsampling factor sigma = 2 and, where the plan's precision reaches eps there,
  at sigma = 1.25 (`collect`), and stores one JSON line per problem;
* trains the perceptron on the 80 % of problems whose seed is not 0 mod 5
  (`train`), and compares, on the other 20 %, the execute time of the picker's
  choice (over both factors) with the heuristic (sigma = 2, default tiles) and
  the fastest candidate (`evaluate`).

sigma needs no feature of its own: it enters through the kernel width w and the
fine-grid size n_tot (features 3 and 4), the two quantities it trades against
each other (spreading work ~ M w^d against FFT work ~ n_tot log n_tot).

Usage:
    python -m paper_2102_08463_gb300.picker collect --count 200 --out trials.jsonl
    python -m paper_2102_08463_gb300.picker train --data trials.jsonl --out picker.txt
    python -m paper_2102_08463_gb300.picker evaluate --data trials.jsonl --weights picker.txt
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "picker_weights_gb300.txt")
DEFAULT_TRIALS = os.path.join(HERE, "data", "picker_trials_gb300.jsonl")
PROBLEM_SEED = wl.BASE_SEED + 5

# Work bound: M * w^d (x16 in double precision, whose arithmetic is far slower)
# and the fine-grid size, so that one execute stays within tens of ms.
MAX_WORK = 2.0e10
MAX_NFTOT = 1 << 26


def is_heldout(seed: int) -> bool:
    """The 20 % evaluation split, by problem seed."""
    return seed % 5 == 0


def sample_problems(count: int, first_seed: int = 0, max_work: float = MAX_WORK,
                    max_nftot: int = MAX_NFTOT, heldout=None):
    """`count` problems with seeds first_seed, first_seed + 1, ... (redrawn past
    the work bound; heldout True / False keeps only that split)."""
    from . import binding
    out = []
    s = first_seed
    while len(out) < count:
        seed = s
        s += 1
        if heldout is not None and is_heldout(seed) != heldout:
            continue
        u = wl.uniform01(PROBLEM_SEED, 12, stream=1000 + seed)
        dim = 2 if u[0] < 0.5 else 3
        tp = 1 if u[1] < 0.5 else 2
        lo, hi = math.log(32), math.log(1024)
        N = tuple(int(round(math.exp(lo + u[2 + d] * (hi - lo)))) for d in range(dim))
        M = int(round(math.exp(math.log(1e4) + u[5] * (math.log(3e7) - math.log(1e4)))))
        kind = "rand" if u[6] < 1 / 3 else ("gauss" if u[6] < 2 / 3 else "mixture")
        spread = math.exp(math.log(0.01 * math.pi) + u[7] * math.log(50.0))
        eps = 10.0 ** (-12.0 + 10.0 * u[8])
        prec = 0 if eps >= 1e-6 else 1
        f = binding.picker_features(tp, N, eps, M, 0.0, "sm", prec=prec)
        w = int(round(f[3] * 16))
        nftot = 2.0 ** (f[4] * 32)
        w125 = sigma125_width(tp, N, eps, M, prec)
        work = M * max(w, w125 or 0) ** dim * (16 if prec else 1)
        if work > max_work or nftot > max_nftot * 1.0001:
            continue
        out.append(dict(seed=seed, type=tp, dim=dim, N=list(N), M=M, kind=kind,
                        spread=spread, eps=eps, prec=prec, w=w))
    return out


def sigma125_width(tp, N, eps, M, prec):
    """Kernel width of the sigma = 1.25 plan at this precision, or None where that
    plan does not reach eps (single precision below 1e-4, w over 16)."""
    from . import binding
    try:
        f = binding.picker_features(tp, N, eps, M, 0.0, "sm", prec=prec, upsampfac=1.25)
    except binding.NufftError:
        return None
    return int(round(f[3] * 16))


def _inputs(pr, torch):
    dt = np.float32 if pr["prec"] == 0 else np.float64
    ct = np.complex64 if pr["prec"] == 0 else np.complex128
    pts = wl.points(pr["kind"], pr["dim"], pr["M"], PROBLEM_SEED + 7 * pr["seed"], dt,
                    spread=pr["spread"])
    pts = [torch.from_numpy(a).cuda() for a in pts]
    if pr["type"] == 1:
        c = torch.from_numpy(wl.strengths(pr["M"], PROBLEM_SEED + 7 * pr["seed"] + 1, ct)).cuda()
        f = torch.zeros(tuple(reversed(pr["N"])), dtype=c.dtype, device="cuda")
    else:
        f = torch.from_numpy(wl.modes(pr["N"], PROBLEM_SEED + 7 * pr["seed"] + 2, ct)).cuda()
        c = torch.zeros(pr["M"], dtype=f.dtype, device="cuda")
    return pts, c, f


def collect(problems, reps: int = 2, out=None, log=None, seconds=None):
    """Time every candidate tiling of each problem at sigma = 2 and, where it
    reaches eps, sigma = 1.25; returns one dict per problem (its fields, skew,
    heuristic tiles and trials [method, bin x3, M_sub, threads, sigma, ms]) and
    appends JSON lines to out.  Stops after `seconds` of wall time if given."""
    import torch
    from . import binding
    rows = []
    fh = open(out, "a") if out else None
    start = time.time()
    try:
        for i, pr in enumerate(problems):
            if seconds is not None and time.time() - start > seconds:
                break
            t0 = time.time()
            pts, c, f = _inputs(pr, torch)
            skew = binding.point_skew(*pts)
            with binding.Plan(pr["type"], pr["N"], pr["eps"], prec=pr["prec"]) as p:
                heur = p.tiles()
            sigmas = [2.0]
            if sigma125_width(pr["type"], pr["N"], pr["eps"], pr["M"], pr["prec"]):
                sigmas.append(1.25)
            rec, best_ms = [], float("inf")
            for sg in sigmas:
                base = binding.default_opts()
                base.upsampfac = sg
                _, ms, trials = binding.autotune(
                    pr["type"], pr["N"], pr["eps"], pr["M"], pts[0], pts[1],
                    pts[2] if pr["dim"] == 3 else None, c, f, prec=pr["prec"], reps=reps,
                    base=base)
                best_ms = min(best_ms, ms)
                rec += [[t["method"]] + list(t["bin"]) + [t["msub"], t["threads"], sg,
                                                          round(t["exec_ms"], 5)]
                        for t in trials]
            binding.tune_cache_clear()
            row = dict(pr, skew=skew, heuristic=[heur["method"]] + list(heur["bin"]) +
                       [heur["msub"], heur["threads"]], trials=rec)
            rows.append(row)
            if fh:
                fh.write(json.dumps(row) + "\n")
                fh.flush()
            if log:
                log("problem %d/%d seed %d: %dD type %d N=%s M=%d eps=%.1e %s -> best %.3f ms "
                    "(%d trials, %.1f s)" % (i + 1, len(problems), pr["seed"], pr["dim"],
                                             pr["type"], pr["N"], pr["M"], pr["eps"], pr["kind"],
                                             best_ms, len(rec), time.time() - t0))
            del pts, c, f
    finally:
        if fh:
            fh.close()
    return rows


def load_rows(path):
    with open(path) as fh:
        return [json.loads(ln) for ln in fh if ln.strip()]


def trial_sigma(t):
    """Upsampling factor of a stored trial (rows without one were timed at 2)."""
    return t[6] if len(t) == 8 else 2.0


def features(row):
    """Feature matrix [n_trials, 12] and targets log2(ms) of one problem's trials."""
    from . import binding
    X, T = [], []
    for t in row["trials"]:
        m, b0, b1, b2, msub, th = t[:6]
        X.append(binding.picker_features(row["type"], row["N"], row["eps"], row["M"], row["skew"],
                                         m, bins=(b0, b1, b2)[:row["dim"]], msub=msub, threads=th,
                                         prec=row["prec"], upsampfac=trial_sigma(t)))
        T.append(math.log2(max(t[-1], 1e-4)))
    return np.asarray(X, dtype=np.float32), np.asarray(T, dtype=np.float32)


def train(rows, epochs: int = 300, batch: int = 256, lr: float = 2e-3, seed: int = 1):
    """A picker trained on the rows of the training split; returns (picker, loss)."""
    import torch
    from . import binding
    Xs, Ts = [], []
    for r in rows:
        if is_heldout(r["seed"]):
            continue
        X, T = features(r)
        Xs.append(X)
        Ts.append(T)
    X = torch.from_numpy(np.concatenate(Xs)).cuda()
    T = torch.from_numpy(np.concatenate(Ts)).cuda()
    p = binding.Picker(seed=seed)
    loss = p.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return p, loss


def evaluate(picker, rows):
    """Per-problem and total execute times of the picker's choice, the heuristic
    tiles and the fastest candidate over the held-out rows."""
    import torch
    tot = dict(picker=0.0, heuristic=0.0, best=0.0)
    per = []
    for r in rows:
        if not is_heldout(r["seed"]):
            continue
        X, _ = features(r)
        pred = picker.predict(torch.from_numpy(X).cuda()).cpu().numpy()
        ms = np.asarray([t[-1] for t in r["trials"]])
        k = int(np.argmin(pred))
        heur = [t[-1] for t in r["trials"]
                if t[:6] == r["heuristic"] and trial_sigma(t) == 2.0]
        if not heur:
            continue
        tot["picker"] += float(ms[k])
        tot["heuristic"] += float(heur[0])
        tot["best"] += float(ms.min())
        per.append(dict(seed=r["seed"], picker=float(ms[k]), heuristic=float(heur[0]),
                        best=float(ms.min()), choice=r["trials"][k][:6],
                        sigma=trial_sigma(r["trials"][k])))
    tot["problems"] = len(per)
    tot["picked_sigma125"] = sum(1 for q in per if q["sigma"] != 2.0)
    tot["regret"] = tot["picker"] / tot["best"] - 1.0 if tot["best"] > 0 else None
    tot["speedup_vs_heuristic"] = tot["heuristic"] / tot["picker"] if tot["picker"] > 0 else None
    return tot, per


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("collect")
    a.add_argument("--count", type=int, default=200)
    a.add_argument("--first-seed", type=int, default=0)
    a.add_argument("--reps", type=int, default=2)
    a.add_argument("--seconds", type=float, default=None)
    a.add_argument("--out", default=DEFAULT_TRIALS)
    a = sub.add_parser("train")
    a.add_argument("--data", default=DEFAULT_TRIALS)
    a.add_argument("--out", default=DEFAULT_WEIGHTS)
    a.add_argument("--epochs", type=int, default=300)
    a.add_argument("--batch", type=int, default=256)
    a.add_argument("--lr", type=float, default=2e-3)
    a.add_argument("--seed", type=int, default=1)
    a = sub.add_parser("evaluate")
    a.add_argument("--data", default=DEFAULT_TRIALS)
    a.add_argument("--weights", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    from . import binding
    if args.cmd == "collect":
        probs = sample_problems(args.count, args.first_seed)
        collect(probs, reps=args.reps, out=args.out, log=lambda s: print(s, flush=True),
                seconds=args.seconds)
    elif args.cmd == "train":
        rows = load_rows(args.data)
        t0 = time.time()
        p, loss = train(rows, args.epochs, args.batch, args.lr, args.seed)
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        p.save(args.out)
        tot, _ = evaluate(p, rows)
        print(json.dumps(dict(train_loss=loss, seconds=round(time.time() - t0, 2), heldout=tot)))
    else:
        rows = load_rows(args.data)
        p = binding.Picker(path=args.weights)
        tot, per = evaluate(p, rows)
        print(json.dumps(dict(heldout=tot, per_problem=per)))


if __name__ == "__main__":
    main()
