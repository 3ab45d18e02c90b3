"""Measurement drivers beside the benchmark: mixed-precision accuracy / speed and small-case latency.

    python -m paper_2608_21227_gb300.experiments mixed --table tuned/gb300.kt --out tuned/mixed_gb300.json
    python -m paper_2608_21227_gb300.experiments latency --out tuned/latency_gb300.json

mixed:   A = U diag(sigma) V^T stored in FP64 with Haar-random U, V and sigma_i =
         kappa^(-(i-1)/(p-1)), kappa in {1, 1e4, 1e8}, shapes 16384^2 and 32768 x 8192.
         The FP64-native path runs untuned (default configuration); the TF32 and BF16
         forms run with the tuned table (--table).  For each: the error max_i |s_i - sigma_i|
         / sigma_1 against the prescribed sigma (the input is formed in FP64, so its own
         singular values are within ~1e-14 sigma_1 of sigma), the error against the FP64
         path, the median relative error over sigma_i >= 1e-3 sigma_1, and the time (CUDA
         events) with the speedup over FP64-native.
peaks:   FP32 FMA, FP64 FMA and tensor-core (kind::tf32) throughput from long chains of
         independent operations (nla_pipe_selftest), CUDA events, SM clock sampled.
latency: the 256 x 256 FP64 N(0,1) case (tile 32, band 32, default configuration): one
         call captured into a CUDA graph, median of 20 replays.
case:    one workload run `--reps` times, for profilers that capture single launches:
         a dense SVD (--n, --dtype, --update; U[-1,1] entries, seed 7), a batch of the
         batched workload's shapes (--batched COUNT), or cost-model forward/backward and
         Adam steps (--mlp ROWS).
All work runs on the GPU through libnla.so; inputs are generated on the GPU with seeded
torch generators (input generation only, not part of the timed library call).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import nla


def haar(m, n, gen, device):
    """m x n with orthonormal columns, Haar distributed (QR of a Gaussian with the sign fix)."""
    import torch

    G = torch.randn(m, n, generator=gen, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    return Q * torch.sign(torch.diagonal(R)).unsqueeze(0)


def prescribed(m, n, kappa, seed, device):
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    p = min(m, n)
    sigma = torch.tensor(kappa ** (-np.arange(p) / max(p - 1, 1)), dtype=torch.float64, device=device)
    U = haar(m, p, gen, device)
    V = haar(n, p, gen, device)
    A = (U * sigma.unsqueeze(0)) @ V.T  # row-major m x n == column-major A^T (same singular values)
    del U, V
    return A.contiguous(), sigma


def timed_call(A, update, reps, table=None):
    import torch

    from . import kt

    kt.load_config(table)  # None: untuned defaults
    ts, S = [], None
    for _ in range(reps):
        B = A.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        S, info = nla.gesvd_vals(B, update=update)
        e1.record()
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        ts.append(e0.elapsed_time(e1))
        del B
    return float(np.median(ts)), S.double().cpu().numpy()


def mixed(args):
    import torch

    dev = torch.device("cuda", 0)
    out = []
    for (m, n) in [tuple(map(int, s.split("x"))) for s in args.shapes]:
        for kappa in args.kappas:
            seed = 400 + 10 * (m // 1024) + int(round(np.log10(kappa)))
            A, sigma = prescribed(m, n, kappa, seed, dev)
            sig = sigma.cpu().numpy()
            reps = args.reps if kappa == args.kappas[0] else 1
            t64, s64 = timed_call(A, nla.UPD_NATIVE, reps)
            rec = {"m": m, "n": n, "kappa": kappa, "seed": seed, "fp64_ms": t64, "fp64_config": "default",
                   "mixed_config": "tuned table" if args.table else "default",
                   "fp64_err_vs_sigma": float(np.max(np.abs(s64 - sig)) / sig[0])}
            mask = sig >= 1e-3 * sig[0]
            for name, upd in (("tf32", nla.UPD_TF32), ("bf16", nla.UPD_BF16), ("tf32x3", nla.UPD_TF32X3),
                              ("bf16x3", nla.UPD_BF16X3)):
                # the compensated forms have no tuned entries of their own: they take the
                # table's TF32 band when the table is installed (same kernels, three products)
                t, s = timed_call(A, upd, reps, args.table)
                rec[name] = {"ms": t, "speedup_vs_fp64": t64 / t,
                             "err_vs_sigma": float(np.max(np.abs(s - sig)) / sig[0]),
                             "err_vs_fp64": float(np.max(np.abs(s - s64)) / s64[0]),
                             "median_rel_err_top": float(np.median(np.abs(s[mask] - sig[mask]) / sig[mask]))}
            print(json.dumps(rec), flush=True)
            out.append(rec)
            del A
            torch.cuda.empty_cache()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)


def latency(args):
    import torch

    from . import inputs

    dev = torch.device("cuda", 0)
    A0 = torch.from_numpy(np.ascontiguousarray(inputs.gaussian(256, 256, 1).T)).to(dev)
    m, n, _ = nla.col_major_view(A0)
    cfg = nla.Cfg.make(band=32, tile=64, threads=128, cols_per_block=2, unroll=1)
    need = nla.gesvd_vals_workspace(m, n, nla.F64, cfg=cfg, preserve_a=True)
    work = nla.workspace(need, dev)
    S = torch.empty(n, dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream(dev)
    with torch.cuda.stream(st):
        for _ in range(3):
            nla.gesvd_vals(A0, cfg=cfg, preserve_a=True, work=work, S=S, info=info, stream=st)
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            nla.gesvd_vals(A0, cfg=cfg, preserve_a=True, work=work, S=S, info=info, stream=st)
        ts = []
        for _ in range(20):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g.replay()
            e1.record(st)
            st.synchronize()
            ts.append(e0.elapsed_time(e1))
    assert int(info.item()) == 0
    flops = 4.0 * 256 ** 3 - 4.0 * 256 ** 3 / 3
    rec = {"case": "256x256 FP64 N(0,1) seed 1, band 32, default configuration, CUDA graph replay",
           "median_ms": float(np.median(ts)), "min_ms": float(np.min(ts)),
           "gflops": flops / (float(np.median(ts)) / 1e3) / 1e9}
    print(json.dumps(rec), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rec, f, indent=1)


def case(args):
    import torch

    from . import inputs, kt

    dev = torch.device("cuda", 0)
    if args.tuned:
        import os

        kt.load_config(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned", "gb300.kt"))
    if args.batched:
        ms, ns = inputs.batch_shapes(args.batched, seed=3)
        mats = [torch.from_numpy(np.ascontiguousarray(inputs.gaussian(int(ms[i]), int(ns[i]), [3, i],
                                                                      dtype=np.float32).T)).to(dev)
                for i in range(args.batched)]
        bt = nla.Batch(mats)
        for _ in range(args.reps):
            _, info = nla.gesvd_vals_batched(bt)
        torch.cuda.synchronize()
        assert int(info.abs().max().item()) == 0
        print(json.dumps({"case": "batched", "count": args.batched}))
        return
    if args.mlp:
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        npar = kt.mlp_param_count()
        params = torch.randn(npar, generator=g, device=dev) * 0.05
        X = torch.randn(args.mlp, kt.FEATURES, generator=g, device=dev)
        y = torch.randn(args.mlp, generator=g, device=dev)
        mom, var = torch.zeros_like(params), torch.zeros_like(params)
        for t in range(1, args.reps + 1):
            _, grads = kt.mlp_forward_backward(params, X, y)
            kt.mlp_adam_step(params, grads, mom, var, t, 1e-3)
        torch.cuda.synchronize()
        print(json.dumps({"case": "mlp", "rows": args.mlp}))
        return
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    A0 = inputs.uniform_device(args.n, args.n, 7, dtype=tdt, device=dev)
    upd = {"native": nla.UPD_NATIVE, "tf32": nla.UPD_TF32, "bf16": nla.UPD_BF16}[args.update]
    for _ in range(args.reps):
        A = A0.clone()
        S, info = nla.gesvd_vals(A, update=upd)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
    print(json.dumps({"case": "gesvd", "n": args.n, "dtype": args.dtype, "update": args.update,
                      "sigma_max": float(S[0].item())}))


def peaks(args):
    """FP32 FMA, FP64 FMA and tcgen05 kind::tf32 throughput of this GPU (nla_pipe_selftest),
    timed with CUDA events while nvidia-smi samples the SM clock (read-only)."""
    import ctypes
    import subprocess
    import threading

    import torch

    L = nla.lib()
    L.nla_pipe_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    L.nla_pipe_selftest.restype = ctypes.c_int
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.zeros(sms * 8 * 256, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    lines = []
    proc = subprocess.Popen(["nvidia-smi", "-i", "0", "--query-gpu=clocks.sm,clocks.max.sm,power.draw",
                             "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                            stderr=subprocess.DEVNULL, text=True)
    reader = threading.Thread(target=lambda: [lines.append(x.strip()) for x in proc.stdout], daemon=True)
    reader.start()
    res = {}
    # kind: (name, blocks, iters, flops per launch)
    runs = [("fp32_fma", 0, sms * 8, 200000, lambda b, it: 2.0 * 8 * it * b * 256),
            ("fp64_fma", 1, sms * 8, 20000, lambda b, it: 2.0 * 8 * it * b * 256),
            ("tf32_tcgen05", 2, sms, 200000, lambda b, it: 2.0 * 128 * 256 * 8 * it * b)]
    for name, kind, blocks, iters, fl in runs:
        st = torch.cuda.current_stream().cuda_stream
        for _ in range(2):  # warm-up
            assert L.nla_pipe_selftest(kind, blocks, max(iters // 10, 1), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(info.data_ptr()), ctypes.c_void_p(st)) == 0
        torch.cuda.synchronize()
        best = None
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            assert L.nla_pipe_selftest(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(info.data_ptr()), ctypes.c_void_p(st)) == 0
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        assert int(info.item()) == 0
        res[name] = {"tflops": round(fl(blocks, iters) / (best / 1e3) / 1e12, 2), "ms": round(best, 3),
                     "blocks": blocks, "iters": iters}
        print(json.dumps({name: res[name]}), flush=True)
    proc.terminate()
    reader.join(timeout=2)
    mhz = [float(x.split(",")[0]) for x in lines if x and x.split(",")[0].strip().replace(".", "").isdigit()]
    res["clocks"] = {"sm_mhz_median": float(np.median(mhz)) if mhz else None, "samples": len(mhz),
                     "sm_max_mhz": float(lines[0].split(",")[1]) if lines else None}
    res["sms"] = sms
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    m = sub.add_parser("mixed")
    m.add_argument("--shapes", nargs="+", default=["16384x16384", "32768x8192"])
    m.add_argument("--kappas", type=float, nargs="+", default=[1.0, 1e4, 1e8])
    m.add_argument("--reps", type=int, default=2)
    m.add_argument("--table", help="tuned table for the TF32 / BF16 forms")
    m.add_argument("--out")
    la = sub.add_parser("latency")
    la.add_argument("--out")
    c = sub.add_parser("case")
    c.add_argument("--n", type=int, default=2048)
    c.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    c.add_argument("--update", choices=["native", "tf32", "bf16"], default="native")
    c.add_argument("--batched", type=int, default=0)
    c.add_argument("--mlp", type=int, default=0)
    c.add_argument("--reps", type=int, default=2)
    c.add_argument("--tuned", action="store_true", help="install the tuned table first")
    pk = sub.add_parser("peaks")
    pk.add_argument("--reps", type=int, default=5)
    pk.add_argument("--out")
    args = ap.parse_args()
    t0 = time.time()
    {"mixed": mixed, "latency": latency, "case": case, "peaks": peaks}[args.cmd](args)
    print(json.dumps({"seconds": round(time.time() - t0, 1)}))


if __name__ == "__main__":
    main()
