#!/usr/bin/env python3
"""Time to a 1e-12 relative residual per frontal solve, HODLR-preconditioned GMRES.

Workload (default): the n = 4096 plane front -- the exact Schur complement onto
the middle plane of a 7-point lognormal (sigma = 0.5) diffusion operator on a
64 x 64 x 65 grid (32 planes on each side, Dirichlet), 4 N(0,1) right-hand
sides, leaf 128, ACA tol 1e-4.  One step = hodlr_build + hodlr_factor +
gmres_solve to 1e-12 for the 4 right-hand sides, with A and B resident in HBM.
The headline arm factors in FP32 (GMRES in FP64); the plain FP64 HODLR path on
the same GPU is timed beside it.

`--impl reference` times the CPU FP64 oracle on the same workload (host cores).
Multi-GPU (torchrun): every rank solves its own copy of the front (replicas);
value = max-over-ranks time / (steps x ranks).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402



def _scratch_dir():
    """Where the benchmark's scratch files go: $HODLR_FRONT_CACHE (the front
    cache's directory) when set, else the system's temporary directory."""
    d = os.environ.get("HODLR_FRONT_CACHE")
    if not d:
        return tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d

METRIC = "time to 1e-12 relative residual per frontal solve"
# arithmetic of the path per --precision: preconditioner storage + factor, then the FP64 Krylov loop
DTYPE = {"fp32": "f32+f64", "bf16": "bf16+f32+f64", "fp16": "f16+f32+f64", "fp64": "f64"}
WORKLOADS = {
    "plane4096": dict(nx=64, ny=64, below=32, above=32, field="lognormal", sigma=0.5, leaf=128, seed=0, nrhs=4),
    "plane576": dict(nx=24, ny=24, below=8, above=8, field="lognormal", sigma=0.5, leaf=64, seed=0, nrhs=1),
    # the large front (run with --precision fp16 --tol 1e-3 --no-cpu-baseline)
    "plane32768": dict(nx=128, ny=256, below=4, above=4, field="lognormal", sigma=0.5, leaf=256, seed=0, nrhs=32),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p.get("bf16_tflops"), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampler for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv", dir=_scratch_dir())
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic(kernel, workload, precision):
    """DRAM bytes per launch unit of `kernel` from the committed ncu summary
    (profiles/dram_traffic.txt), or None when it holds no figure for this case."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                p = line.split()
                if len(p) >= 4 and not line.startswith("#") and p[:3] == [kernel, workload, precision]:
                    return float(p[3])
    except OSError:
        pass
    return None


def make_inputs(wl, device):
    import frontgen as fg
    w = dict(WORKLOADS[wl])
    nrhs = w.pop("nrhs")
    F = fg.make_front(**w, device=device, cache=True)
    B = fg.rhs(F.n, nrhs, seed=1)
    return F, B


def oracle_solve(A, B, leaf, bounds, method, tol, graph):
    from oracle import hodlr_oracle as O
    tree = O.make_tree(A.shape[0], leaf, bounds)
    t0 = time.perf_counter()
    _, _, P = O.hodlr_precond(A, tree, method, tol, graph=graph, symmetric=True)
    res = [O.gmres(A, B[:, r], prec=P, tol=1e-12) for r in range(B.shape[1])]
    return time.perf_counter() - t0, res


def _oracle_subprocess(path, leaf, method, tol, reps):
    """Run the oracle single-threaded in a child process; returns seconds per solve."""
    code = (
        "import sys, json, numpy as np; sys.path.insert(0, %r)\n"
        "import bench\n"
        "d = np.load(%r)\n"
        "ts = []\n"
        "for _ in range(%d):\n"
        "    t, res = bench.oracle_solve(d['A'], d['B'], %d, d['bounds'], %r, %r, (d['rowptr'], d['colind']))\n"
        "    ts.append(t)\n"
        "print(json.dumps({'t': ts, 'iters': [r.iters for r in res], 'relres': [r.true_relres for r in res]}))\n"
    ) % (ROOT, path, reps, leaf, method, tol)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=3000)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _save_inputs(F, B):
    fd, path = tempfile.mkstemp(suffix=".npz", dir=_scratch_dir())
    os.close(fd)
    A = F.A if isinstance(F.A, np.ndarray) else F.A.cpu().numpy()
    np.savez(path, A=A, B=B, bounds=F.bounds, rowptr=F.rowptr, colind=F.colind)
    return path


def job_time(total_ms, steps, world, device):
    """The timed region's length over the whole job: the maximum over ranks (an
    all-reduce when world > 1), the time per step, and the value, time per
    frontal solve, every rank solving its own front in each step."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return total_ms, ms_per_step, ms_per_step / world


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    F, B = make_inputs(args.workload, dev)
    path = _save_inputs(F, B)
    leaf = WORKLOADS[args.workload]["leaf"]
    try:
        r = _oracle_subprocess(path, leaf, args.method, args.tol, args.warmup + args.steps)
    finally:
        os.unlink(path)
    ts = r["t"][args.warmup:]
    ms = 1e3 * sum(ts) / len(ts)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, F),
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"full oracle solve (ACA build, recursive factor, GMRES x{B.shape[1]} rhs) per step"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_iters": r["iters"], "oracle_true_relres": r["relres"],
    }
    print(json.dumps(line))


def run_batch(args):
    """The 585 octree fronts of a 64^3 lognormal (sigma = 1) grid solved as one
    batch per step (1 right-hand side each): batched build, factor and GMRES.
    value = batch time / number of fronts."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    import frontgen as fg
    torch.cuda.set_device(0)
    boxes = fg.octree_boxes(64, 8)
    As, leaves = [], []
    for s_, org in boxes:
        leaf = 128 if s_ * s_ >= 1024 else 64
        F = fg.make_octree_front(s_, org, leaf, sigma=1.0, seed=0, device="cuda")
        As.append(F.A if torch.is_tensor(F.A) else torch.as_tensor(F.A, device="cuda"))
        leaves.append(leaf)
    Bs = [torch.as_tensor(np.ascontiguousarray(fg.rhs(A.shape[0], 1, seed=1 + f).T), device="cuda")
          for f, A in enumerate(As)]
    ctx = H.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(marks=None):
        hs = H.hodlr_build_batched(ctx, As, leaves, args.tol, "aca", precision=args.precision)
        if marks:
            marks[0].record()
        H.hodlr_factor_batched(hs)
        if marks:
            marks[1].record()
        res = H.gmres_solve_batched(ctx, As, Bs, hs, tol=1e-12)
        if marks:
            marks[2].record()
        for h in hs:
            h.close()
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = H.hodlr_launch_count()
    tot = 0.0
    ph = np.zeros(4)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e0.record()
        res = step(marks)
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
        ev = [e0] + marks + [e1]
        ph += [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
    l1 = H.hodlr_launch_count()
    ms = tot / args.steps
    ph /= args.steps
    its = np.array([int(r[1].iters[0]) for r in res])
    tr = np.array([float(r[1].true_relres[0]) for r in res])
    line = {"metric": METRIC, "value": ms / len(As), "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "octree585: the 585 octree fronts of a 64^3 lognormal (sigma 1) grid, "
                                   "sizes 4096, 1024 x8, 256 x64, 64 x512, 1 rhs each, solved as one batch",
                       "fronts": len(As), "tol": args.tol, "precision": args.precision, "gmres_tol": 1e-12,
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas x1"},
            "converged": bool(np.all(tr <= 1e-12)), "iters_max": int(its.max()), "iters_mean": float(its.mean()),
            "true_relres_max": float(tr.max()), "gpu_launches": l1 - l0,
            "gpu_launches_per_step": (l1 - l0) / args.steps,
            "phases_ms": {"build_batched": ph[0], "factor_batched": ph[1], "gmres_solve_batched": ph[2],
                          "close": ph[3]}}
    print(json.dumps(line))


def run_kernels(args):
    """Component timings of one front: each call timed alone (median of reps)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    F, Bh = make_inputs(args.workload, "cuda")
    A = F.A
    leaf = WORKLOADS[args.workload]["leaf"]
    graph = (F.rowptr, F.colind)
    B = torch.as_tensor(np.ascontiguousarray(Bh.T), device="cuda")
    ctx = H.Context(0)

    def timed(fn, reps=10, setup=None):
        ts = []
        for i in range(reps + 3):
            if setup is not None:
                arg = setup()
                fn_i = (lambda a=arg: fn(a))
            else:
                fn_i = fn
            torch.cuda.synchronize()
            last = i == reps + 2
            if last:
                torch.cuda.nvtx.range_push("kernels")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn_i()
            e1.record()
            torch.cuda.synchronize()
            if last:
                torch.cuda.nvtx.range_pop()
            if i >= 3:
                ts.append(e0.elapsed_time(e1) * 1e3)
        return statistics.median(ts)

    out = {"workload": args.workload, "precision": args.precision, "method": args.method, "tol": args.tol}
    # the build factors each level once it is compressed; the factorisation
    # alone is timed on builds that defer it
    out["build_us"] = timed(lambda: H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph,
                                                  precision=args.precision).close(), 5)
    out["build_deferred_us"] = timed(lambda: H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph,
                                                           precision=args.precision, defer_factor=True).close(), 5)
    deferred = []

    def fresh():
        deferred.append(H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph,
                                      precision=args.precision, defer_factor=True))
        return deferred[-1]

    out["factor_us"] = timed(H.hodlr_factor, 5, setup=fresh)
    for d in deferred:
        d.close()
    h = H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph, precision=args.precision)
    X = B.clone()
    out["apply_us"] = timed(lambda: H.hodlr_solve(h, X))
    out["matvec_us"] = timed(lambda: H.hodlr_matvec(ctx, A, B))
    out["gmres_us"] = timed(lambda: H.gmres_solve(ctx, A, B, h, tol=1e-12), 3)
    _, info = H.gmres_solve(ctx, A, B, h, tol=1e-12)
    out["iters"] = info.iters.tolist()
    out["true_relres"] = info.true_relres.tolist()
    out["ranks_max"] = h.stats()["rank_max"]
    print(json.dumps(out))


def _config(args, F):
    return {"workload": f"{args.workload}: n={F.n} plane front of a {F.nx}x{F.ny}x{F.meta['nz']} lognormal "
                        f"7-point operator, {WORKLOADS[args.workload]['nrhs']} rhs",
            "n": int(F.n), "nrhs": WORKLOADS[args.workload]["nrhs"], "leaf": WORKLOADS[args.workload]["leaf"],
            "method": args.method, "tol": args.tol, "precision": args.precision, "gmres_tol": 1e-12,
            "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plane4096", choices=sorted(WORKLOADS) + ["octree585"])
    ap.add_argument("--method", default="aca", choices=["aca", "bdlr"])
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--nvtx", action="store_true", help="wrap every timed step in an NVTX range 'bench_step'")
    ap.add_argument("--kernels", action="store_true",
                    help="time each component alone (build, factor, apply, matvec, GMRES) with CUDA events; "
                         "the last repetition of each runs inside an NVTX range 'kernels' for ncu")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernels:
        return run_kernels(args)
    if args.workload == "octree585":
        return run_batch(args)

    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H

    F, Bh = make_inputs(args.workload, "cuda")
    A = F.A
    n = F.n
    leaf = WORKLOADS[args.workload]["leaf"]
    graph = (F.rowptr, F.colind)
    B = torch.as_tensor(np.ascontiguousarray(Bh.T), device="cuda")
    ctx = H.Context(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(prec, A_dev=A, B_dev=B):
        h = H.hodlr_build(ctx, A_dev, leaf, args.tol, args.method, graph=graph, precision=prec)
        H.hodlr_factor(h)
        X, info = H.gmres_solve(ctx, A_dev, B_dev, h, tol=1e-12)
        st = h.stats()
        h.close()
        return X, info, st

    launches = [0, 0]

    def timed(prec, k, w):
        for _ in range(w):
            step(prec)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        tot = 0.0
        infos = []
        launches[0] = H.hodlr_launch_count()
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if args.nvtx:
                torch.cuda.nvtx.range_push("bench_step")
            X, info, st = step(prec)
            if args.nvtx:
                torch.cuda.nvtx.range_pop()
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
            infos.append((info, st))
        launches[1] = H.hodlr_launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        return tot, infos, X

    clocks = Clocks(local)
    clocks.start()
    total_ms, infos, X = timed(args.precision, args.steps, args.warmup)
    clk = clocks.stop()
    n_launches = launches[1] - launches[0]
    total_ms, ms_per_step, value = job_time(total_ms, args.steps, world, "cuda")
    info, st = infos[-1]
    converged = bool(info.converged and np.all(info.true_relres <= 1e-12))

    # ---- the dominant kernels, timed alone with CUDA events on the launching stream
    hbm, _, peak_kind = _peaks()
    comp_ms = statistics.median(s["ms_compress"] for _, s in infos)
    w = 8 if args.precision == "fp64" else 4   # compression precision (FP32 below FP64)
    ranks = st["rank_mean"]
    # ACA reads each pivot row/column of A once (FP64) and writes u_k, v_k once:
    # sum over levels of (2^l nodes) * rank * (m + n) * (8 + w), m = n = n/2^l per block.
    aca_bytes = sum((2 ** l) * ranks[l - 1] * 2 * (n / 2 ** l) * (8 + w) for l in range(1, st["levels"] + 1))
    Z = torch.randn(WORKLOADS[args.workload]["nrhs"], n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        H.hodlr_matvec(ctx, A, Z)
    torch.cuda.synchronize()
    mv = []
    for _ in range(10):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.hodlr_matvec(ctx, A, Z)
        e1.record()
        torch.cuda.synchronize()
        mv.append(e0.elapsed_time(e1))
    mv_ms = statistics.median(mv)
    nz = Z.shape[0]
    if nz >= 16:
        # hodlr_matvec with 16+ rhs: A's digit split (two reads of A, 7 BF16
        # slices written) and the slice product (the slices read once), Z read
        # twice and its slices written, W written
        np_, kp_ = -(-n // 128) * 128, -(-n // 64) * 64
        mv_name = "oz_split_and_gemm"
        mv_bytes = 16.0 * n * n + 2 * 14.0 * np_ * kp_ + 16.0 * n * nz + 14.0 * kp_ * nz + 8.0 * n * nz
    else:
        mv_name = "df_matvec_kernel"
        mv_bytes = 8.0 * n * n + 8.0 * n * nz * 2
    n_mv = int(np.max(info.iters)) + 1 + info.restarts
    # the apply, on a factored preconditioner of the same front
    hp = H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph, precision=args.precision)
    H.hodlr_factor(hp)
    Xa = torch.empty_like(Z)
    ap = []
    for it in range(13):
        Xa.copy_(Z)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.hodlr_solve(hp, Xa)
        e1.record()
        torch.cuda.synchronize()
        if it >= 3:
            ap.append(e0.elapsed_time(e1))
    ap_ms = statistics.median(ap)
    pst = hp.stats()
    hp.close()
    ew = 8 if args.precision == "fp64" else (2 if args.precision in ("bf16", "fp16") else 4)
    wtot = sum(pst["rank_pad"])
    # V (n x rp) and E (n x 2 rp) of every level, the leaf inverses' rows, X in and out
    ap_bytes = (3.0 * n * wtot * ew + n * WORKLOADS[args.workload]["leaf"] * (8 if args.precision == "fp64" else 4)
                + 16.0 * n * Z.shape[0])
    n_ap = int(np.max(info.iters)) + info.restarts
    kernels = {
        "aca_kernel": {"ms_per_step": comp_ms, "launch_ms": comp_ms, "bytes": aca_bytes},
        mv_name: {"ms_per_step": mv_ms * n_mv, "launch_ms": mv_ms, "bytes": mv_bytes},
        "apply_fused_kernel": {"ms_per_step": ap_ms * n_ap, "launch_ms": ap_ms, "bytes": ap_bytes},
    }
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    kd = kernels[dom]
    achieved = kd["bytes"] / (kd["launch_ms"] * 1e-3) / 1e9
    traffic = _traffic(dom, args.workload, args.precision)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_kind, "traffic": traffic,
                "share_of_step": kd["ms_per_step"] / ms_per_step,
                "others": {k: {"launch_ms": v["launch_ms"], "GBs": v["bytes"] / (v["launch_ms"] * 1e-3) / 1e9,
                               "ms_per_step": v["ms_per_step"]} for k, v in kernels.items()}}

    # ---- the plain FP64 HODLR path on the same GPU
    compare = None
    if not args.no_compare and args.precision != "fp64":
        t64, inf64, _ = timed("fp64", 2, 1)
        compare = {"fp64_ms_per_step": t64 / 2, "fp64_iters": inf64[-1][0].iters.tolist(),
                   "speedup_vs_fp64": (t64 / 2) / ms_per_step}

    # ---- end to end through the public API with host buffers
    A_host = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    A_host.copy_(A)
    B_host = torch.empty_like(B, device="cpu").pin_memory()
    B_host.copy_(B)
    X_host = torch.empty_like(B_host).pin_memory()
    e2e = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Ad = A_host.to("cuda", non_blocking=True)
        Bd = B_host.to("cuda", non_blocking=True)
        Xd, _, _ = step(args.precision, Ad, Bd)
        X_host.copy_(Xd, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e.append(e0.elapsed_time(e1))
        del Ad, Bd
    e2e_ms = sum(e2e) / len(e2e)

    # ---- CPU oracle on the host cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        path = _save_inputs(F, Bh)
        try:
            r = _oracle_subprocess(path, leaf, args.method, args.tol, 1)
            cpu = {"value": 1e3 * r["t"][0], "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": f"one full oracle solve of the same front and {Bh.shape[1]} rhs "
                             f"(build + recursive factor + GMRES), single-threaded BLAS",
                   "oracle_iters": r["iters"]}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
        finally:
            os.unlink(path)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": _config(args, F),
            "converged": converged, "iters": info.iters.tolist(), "true_relres": info.true_relres.tolist(),
            "ranks_max": st["rank_max"], "ms_compress": comp_ms,
            # compression and factorisation overlap (level l is factored while
            # the levels above it are compressed): each phase is its own span
            "phases_ms": {"compress": comp_ms,
                          "factor": statistics.median(s["ms_factor"] for _, s in infos),
                          "gmres": statistics.median(i.ms_total for i, _ in infos),
                          "build_and_factor": ms_per_step - statistics.median(i.ms_total for i, _ in infos)},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "e2e": {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": 8 * n * n + 8 * B.numel(),
                    "d2h_bytes_per_step": 8 * B.numel()},
            "fp64_path": compare,
            "gpu_launches": n_launches, "gpu_launches_per_step": n_launches / args.steps,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
