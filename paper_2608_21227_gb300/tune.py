"""Auto-tuning driver: sweeps, the installed table, batched buckets, the cost model.

    python -m paper_2608_21227_gb300.tune sweep  --sizes 1024 2048 4096 8192 --dtypes f32 f64 \
        --cache tuned/sweep.csv --table tuned/gb300.kt --summary tuned/sweep.json
    python -m paper_2608_21227_gb300.tune sweep  --sizes 768 1536 --shapes 4096x1024 --no-pipeline \
        --cache tuned/sweep.csv                       (more training rows for the cost model)
    python -m paper_2608_21227_gb300.tune batched --table tuned/gb300.kt --summary tuned/batched.json
    python -m paper_2608_21227_gb300.tune mlp --cache tuned/sweep.csv --holdout 3072 6144 12288 \
        --model tuned/mlp.bin --summary tuned/mlp.json

sweep:   for every size, dtype, side (QR / LQ trailing update) and band width,
         exhaustive kernel-level search (Eq. 1) of one full-size trailing-update
         launch; then the band width is chosen at pipeline level (whole SVD
         timed per band with that band's best kernel configurations); the best
         configurations are appended to the table read by kt_load_config.
batched: for each size bucket, the threads-per-matrix value that runs a batch
         of that bucket fastest.
mlp:     trains the cost model on the sweep cache (held-out sizes excluded), then
         on each held-out size compares the best of the model's top 5% with the
         exhaustive optimum, a random 5% sample (20 seeds) and the default.
All work runs on the GPU through libnla.so.
"""
from __future__ import annotations

import argparse
import csv
import json
import math
import os
import time

import numpy as np

from . import kt, nla

DT = {"f64": nla.F64, "f32": nla.F32}
SIDES = {0: kt.KT_TRAIL_LEFT, 1: kt.KT_TRAIL_RIGHT}
DEFAULT = (32, 64, 128, 2, 1)


def parse_shapes(args):
    shapes = [(n, n) for n in args.sizes]
    for s in args.shapes:
        m, n = (int(x) for x in s.lower().split("x"))
        shapes.append((max(m, n), min(m, n)))
    return shapes


def sweep(args):
    summary = []
    os.makedirs(os.path.dirname(os.path.abspath(args.cache)), exist_ok=True)
    for dname in args.dtypes:
        dt = DT[dname]
        for m, n in parse_shapes(args):
            per_band = {}
            for side, kern in SIDES.items():
                for band in args.bands:
                    t0 = time.time()
                    r = kt.tune(kern, m, n, dt, band=band, reps=args.reps, cache=args.cache, seed=n)
                    r.update({"m": m, "n": n, "dtype": dname, "side": side, "band": band,
                              "seconds": time.time() - t0, "opt_over_median": r["median_ms"] / r["best_ms"],
                              "default_over_opt": (r["default_ms"] / r["best_ms"]) if r["default_ms"] == r["default_ms"] else None})
                    summary.append(r)
                    per_band.setdefault(band, {})[side] = r
                    print(json.dumps(r), flush=True)
            if args.no_pipeline:
                continue
            pipe = kt.tune(kt.KT_GESVD, m, n, dt, reps=2, cache=args.cache, seed=n)
            band = pipe["best"][0]
            rec = {"m": m, "n": n, "dtype": dname, "pipeline": pipe,
                   "tuned_over_default": pipe["default_ms"] / pipe["best_ms"]}
            summary.append(rec)
            print(json.dumps(rec), flush=True)
            if args.table:
                for side in (0, 1):
                    best = per_band[band][side]
                    kt.write_table(args.table, side, m, n, dt, 0, best["best"], best["best_ms"])
    # mixed-precision forms: only the band width is a free parameter (pipeline level)
    for n in args.mixed_sizes:
        for upd in (nla.UPD_TF32, nla.UPD_BF16):
            pipe = kt.tune(kt.KT_GESVD, n, n, nla.F64, update=upd, reps=2, seed=n)
            rec = {"n": n, "dtype": "f64", "update": upd, "pipeline": pipe}
            summary.append(rec)
            print(json.dumps(rec), flush=True)
            if args.table:
                for side in (0, 1):
                    kt.write_table(args.table, side, n, n, nla.F64, upd, pipe["best"], pipe["best_ms"])
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(summary, f, indent=1)


def batched(args):
    import torch

    from . import inputs

    # bucket b holds matrices with m*n in ((48K >> (4 - b)), 48K >> (3 - b)]; representative batches
    elems = 48 * 1024
    bounds = [0, elems // 8, elems // 4, elems // 2, elems, 1 << 30]
    min_group = [32, 64, 128, 256, 128]  # the largest bucket: threads per matrix of the large-matrix kernel
    ms, ns = inputs.batch_shapes(20000, seed=args.seed)
    out = []
    for b in range(5):
        sel = [i for i in range(len(ms)) if bounds[b] < ms[i] * ns[i] <= bounds[b + 1]][: args.count]
        if not sel:
            continue
        mats = [torch.from_numpy(np.ascontiguousarray(inputs.gaussian(int(ms[i]), int(ns[i]), [args.seed, i],
                                                                      dtype=np.float32).T)).cuda() for i in sel]
        bt = nla.Batch(mats)
        best = None
        for g in [x for x in (32, 64, 128, 256) if x >= min_group[b]]:
            tmp = args.table + f".tmp{g}"
            with open(tmp, "w") as f:
                f.write(f"2 {b} 0 1 0 {g} 0 0 0 0 0\n")
            kt.load_config(tmp)
            os.remove(tmp)
            for _ in range(2):
                nla.gesvd_vals_batched(bt)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                nla.gesvd_vals_batched(bt)
            e1.record()
            torch.cuda.synchronize()
            ms_ = e0.elapsed_time(e1) / 5
            rec = {"bucket": b, "group": g, "count": len(sel), "ms": ms_}
            print(json.dumps(rec), flush=True)
            out.append(rec)
            if best is None or ms_ < best[1]:
                best = (g, ms_)
        kt.load_config(None)
        kt.write_table(args.table, 2, b, 0, nla.F32, 0, (best[0], 0, 0, 0, 0), best[1])
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(out, f, indent=1)


def read_cache(path):
    rows = []
    with open(path) as f:
        for r in csv.DictReader(f):
            extra = r.pop(None, None)  # (a row with the objective column under an older header)
            r = {k: (float(v) if k == "median_ms" else int(v)) for k, v in r.items() if v is not None}
            if extra:
                r["objective"] = int(extra[0])
            if r["status"] == 0 and r["kernel"] in (0, 1) and r["median_ms"] > 0 and r.get("objective", 0) == 0:
                rows.append(r)
    return rows


def mlp(args):
    rows = read_cache(args.cache)
    hold = set(args.holdout)
    train = [r for r in rows if r["m"] not in hold]
    X = np.stack([kt.features(r["kernel"], r["m"], r["n"], r["dtype"], r["update"],
                              (r["band"], r["tile"], r["threads"], r["cpb"], r["unroll"])) for r in train])
    y = np.log(np.array([r["median_ms"] for r in train], dtype=np.float64)).astype(np.float32)
    t0 = time.time()
    loss = kt.mlp_train(X, y, epochs=args.epochs, batch=256, lr=args.lr, seed=args.seed, model_path=args.model)
    train_s = time.time() - t0
    report = {"train_rows": int(len(train)), "final_loss": loss, "train_seconds": train_s, "cases": []}
    print(json.dumps({k: v for k, v in report.items() if k != "cases"}), flush=True)
    for dname in args.dtypes:
        dt = DT[dname]
        for n in args.holdout:
            for side, kern in SIDES.items():
                for band in args.bands:
                    ex = kt.tune(kern, n, n, dt, band=band, reps=3, cache=args.cache, seed=n)
                    t0 = time.time()
                    mo = kt.tune(kern, n, n, dt, band=band, reps=3, strategy=kt.KT_MODEL_TOPK, budget_frac=0.05,
                                 model=args.model, seed=n)
                    t_model = time.time() - t0
                    rnd = [kt.tune(kern, n, n, dt, band=band, reps=3, strategy=kt.KT_RANDOM, budget_frac=0.05,
                                   cache=args.cache, seed=1000 + s)["best_ms"] for s in range(args.random_seeds)]
                    case = {"n": n, "dtype": dname, "side": side, "band": band, "exhaustive_ms": ex["best_ms"],
                            "exhaustive_evaluated": ex["evaluated"], "model_ms": mo["best_ms"],
                            "model_evaluated": mo["evaluated"], "model_seconds": t_model,
                            "model_over_opt": mo["best_ms"] / ex["best_ms"],
                            "random_mean_over_opt": float(np.mean(rnd)) / ex["best_ms"],
                            "default_over_opt": ex["default_ms"] / ex["best_ms"] if ex["default_ms"] == ex["default_ms"] else None,
                            "median_over_opt": ex["median_ms"] / ex["best_ms"]}
                    report["cases"].append(case)
                    print(json.dumps(case), flush=True)
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(report, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("sweep")
    s.add_argument("--sizes", type=int, nargs="*", default=[1024, 2048, 4096, 8192])
    s.add_argument("--shapes", nargs="*", default=[], help="rectangular problems MxN (m >= n)")
    s.add_argument("--no-pipeline", action="store_true", help="kernel-level sweeps only (training data)")
    s.add_argument("--dtypes", nargs="+", default=["f32", "f64"])
    s.add_argument("--bands", type=int, nargs="+", default=[16, 32, 64])
    s.add_argument("--reps", type=int, default=5)
    s.add_argument("--mixed-sizes", type=int, nargs="*", default=[])
    s.add_argument("--cache", required=True)
    s.add_argument("--table")
    s.add_argument("--summary")
    b = sub.add_parser("batched")
    b.add_argument("--table", required=True)
    b.add_argument("--count", type=int, default=800)
    b.add_argument("--seed", type=int, default=3)
    b.add_argument("--summary")
    m = sub.add_parser("mlp")
    m.add_argument("--cache", required=True)
    m.add_argument("--holdout", type=int, nargs="+", default=[3072, 6144, 12288])
    m.add_argument("--dtypes", nargs="+", default=["f32"])
    m.add_argument("--bands", type=int, nargs="+", default=[32])
    m.add_argument("--model", required=True)
    m.add_argument("--epochs", type=int, default=80)
    m.add_argument("--lr", type=float, default=2e-3)
    m.add_argument("--seed", type=int, default=1)
    m.add_argument("--random-seeds", type=int, default=20)
    m.add_argument("--summary")
    args = ap.parse_args()
    {"sweep": sweep, "batched": batched, "mlp": mlp}[args.cmd](args)


if __name__ == "__main__":
    main()
