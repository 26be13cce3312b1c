#!/usr/bin/env python3
"""Time to a 1e-12 relative residual per frontal solve, HODLR-preconditioned GMRES.

Workload (default): the n = 32768 plane front -- the exact Schur complement onto
the middle plane of a 7-point lognormal (sigma = 0.5) diffusion operator on a
128 x 256 x 9 grid (4 planes on each side, Dirichlet), 32 N(0,1) right-hand
sides; FP16 HODLR storage (a power-of-two scale per node column) with FP32
factor arithmetic, ACA tol 1e-3, leaf 256 (depth 7); FP64-accurate GMRES to
1e-12.  One step = hodlr_build (which also factors) + gmres_solve for the 32
right-hand sides, with A and B resident in HBM (A is 8.6 GB, far beyond L2).
The plain FP64 HODLR + GMRES path on the same GPU is timed beside it.

`--impl reference` times the CPU FP64 oracle on the same workload (one host
core): a bounded sample (its build + factor once, then one Arnoldi iteration of
one right-hand side per step), scaled to the workload as stated in its line.
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
# front (frontgen.make_front arguments), right-hand sides, and the precision and
# tolerance each configuration is quoted with
WORKLOADS = {
    "plane32768": dict(front=dict(nx=128, ny=256, below=4, above=4, field="lognormal", sigma=0.5, leaf=256, seed=0),
                       nrhs=32, precision="fp16", tol=1e-3,
                       desc="plane32768: n=32768 plane front of a 128x256x9 lognormal (sigma 0.5) 7-point operator "
                            "(4 planes per side), 32 rhs, FP16 HODLR (per-column power-of-two scales, FP32 factor), "
                            "ACA tol 1e-3, leaf 256, depth 7"),
    "plane4096": dict(front=dict(nx=64, ny=64, below=32, above=32, field="lognormal", sigma=0.5, leaf=128, seed=0),
                      nrhs=4, precision="fp32", tol=1e-4,
                      desc="plane4096: n=4096 plane front of a 64x64x65 lognormal (sigma 0.5) 7-point operator, "
                           "4 rhs, FP32 HODLR, ACA tol 1e-4, leaf 128"),
    "plane576": dict(front=dict(nx=24, ny=24, below=8, above=8, field="lognormal", sigma=0.5, leaf=64, seed=0),
                     nrhs=1, precision="fp64", tol=1e-6,
                     desc="plane576: n=576 plane front of a 24x24x17 lognormal (sigma 0.5) 7-point operator, 1 rhs, "
                          "plain FP64 HODLR, ACA tol 1e-6, leaf 64"),
    "checker16384": dict(front=dict(nx=128, ny=128, below=16, above=16, field="checkerboard", leaf=256, seed=0),
                         nrhs=1, precision="bf16", tol=1e-3,
                         desc="checker16384: n=16384 plane front of a 128x128x33 checkerboard (1/1e6 in 8^3 cells) "
                              "7-point operator, 1 rhs, BF16 HODLR, ACA tol 1e-3, leaf 256"),
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
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/dram_traffic.txt), or None when it holds no figure for this case."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
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
    w = WORKLOADS[wl]
    F = fg.make_front(**w["front"], device=device, cache=True)
    B = fg.rhs(F.n, w["nrhs"], seed=1)
    return F, B


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


# --------------------------------------------------------------------------- the CPU oracle
def _oracle_child(spec_path):
    """Run in a child process with one BLAS thread and no GPU.  Loads the
    cached front, builds and factors the oracle's FP64 HODLR preconditioner
    (timed), then
      baseline:  GMRES to 1e-12 on right-hand side 0 (timed; x saved) and the
                 preconditioner error on the seeded probe block Omega;
      reference: GMRES on right-hand side 0 for its iteration count, then per
                 step one Arnoldi iteration of one right-hand side (P^-1 v,
                 A z, modified Gram-Schmidt against half the iteration count
                 of basis vectors), timed."""
    with open(spec_path) as f:
        spec = json.load(f)
    import frontgen as fg
    from oracle import hodlr_oracle as O
    w = WORKLOADS[spec["workload"]]
    F = fg.make_front(**w["front"], device="cpu", cache=True)
    A, n = F.A, F.n
    b = fg.rhs(n, 1, seed=1)[:, 0]
    tree = O.make_tree(n, w["front"]["leaf"], F.bounds)
    t0 = time.perf_counter()
    _, _, P = O.hodlr_precond(A, tree, spec["method"], spec["tol"], graph=(F.rowptr, F.colind), symmetric=True)
    out = {"n": n, "t_build_factor": time.perf_counter() - t0}
    t0 = time.perf_counter()
    r = O.gmres(A, b, prec=P, tol=1e-12)
    out.update(t_gmres=time.perf_counter() - t0, iters=r.iters, true_relres=r.true_relres)
    if spec["mode"] == "baseline":
        np.save(spec["x_path"], r.x)
        if spec.get("omega"):
            out["precond_error"] = O.precond_error(A, P, fg.rhs(n, 16, seed=2))
    else:
        j = max(1, r.iters // 2)
        rng = np.random.default_rng(0)
        V = rng.standard_normal((j + 1, n))
        V /= np.linalg.norm(V, axis=1, keepdims=True)
        ts = []
        for _ in range(spec["warmup"] + spec["steps"]):
            t0 = time.perf_counter()
            z = P(V[0])
            wv = A @ z
            for i in range(j):
                wv = wv - (V[i] @ wv) * V[i]
            float(np.linalg.norm(wv))
            ts.append(time.perf_counter() - t0)
        out["t_iteration"] = ts[spec["warmup"]:]
    print(json.dumps(out))


def _run_oracle(spec):
    """The oracle child (one BLAS thread, no GPU); returns its JSON result."""
    fd, path = tempfile.mkstemp(suffix=".json", dir=_scratch_dir())
    with os.fdopen(fd, "w") as f:
        json.dump(spec, f)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = "import sys; sys.path.insert(0, %r); import bench; bench._oracle_child(%r)" % (ROOT, path)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=3000)
    finally:
        os.unlink(path)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the workload, a bounded sample
    (see _oracle_child), value = build + factor + nrhs x iterations x the
    median iteration time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    try:   # the front, generated (or found) in the cache the oracle reads
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        F, _ = make_inputs(args.workload, dev)
        n = F.n
        del F
        if dev == "cuda":
            torch.cuda.empty_cache()
    except Exception:
        F, _ = make_inputs(args.workload, "cpu")
        n = F.n
    r = _run_oracle({"workload": args.workload, "method": args.method, "tol": args.tol, "mode": "reference",
                     "steps": args.steps, "warmup": args.warmup})
    t_it = statistics.median(r["t_iteration"])
    ms = 1e3 * (r["t_build_factor"] + w["nrhs"] * r["iters"] * t_it)
    sample = (f"FP64 oracle (NumPy, one BLAS thread): build + factor once ({r['t_build_factor']:.1f} s), GMRES on "
              f"rhs 0 for its iteration count ({r['iters']}), then per step one Arnoldi iteration of one rhs "
              f"(median {1e3 * t_it:.0f} ms); value = build + factor + {w['nrhs']} rhs x {r['iters']} iterations "
              f"x that time")
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, n),
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_iters": r["iters"], "oracle_true_relres": r["true_relres"],
        "oracle_gmres_rhs0_s": r["t_gmres"],
    }
    print(json.dumps(line))


def _config(args, n):
    w = WORKLOADS[args.workload]
    return {"workload": w["desc"], "n": int(n), "nrhs": w["nrhs"], "leaf": w["front"]["leaf"],
            "method": args.method, "tol": args.tol, "precision": args.precision, "gmres_tol": 1e-12,
            "l2": "inputs larger than L2 (A is 8 n^2 bytes) and a 256 MiB write between steps",
            "parallelism": f"replicas x{args.gpus}"}


def run_batch(args):
    """The 585 octree fronts of a 64^3 lognormal (sigma = 1) grid solved as one
    batch per step (1 right-hand side each): batched build, factor and GMRES,
    with the leaf size and rank cap of each front size chosen by measurement
    (paper_1403_5337_gb300.autotune, once, before the timed steps).
    value = batch time / number of fronts."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    from paper_1403_5337_gb300 import autotune
    import frontgen as fg
    torch.cuda.set_device(0)
    boxes = fg.octree_boxes(64, 8)
    # every front in the recursive-bisection order down to 64-vertex rectangles:
    # a tree with larger leaves (halving the index range) has rectangles as nodes too
    As = []
    for s_, org in boxes:
        F = fg.make_octree_front(s_, org, 64, sigma=1.0, seed=0, device="cuda")
        As.append(F.A if torch.is_tensor(F.A) else torch.as_tensor(F.A, device="cuda"))
    Bs = [torch.as_tensor(np.ascontiguousarray(fg.rhs(A.shape[0], 1, seed=1 + f).T), device="cuda")
          for f, A in enumerate(As)]
    ctx = H.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # tune on the first front of every size
    samples = {}
    for f, A in enumerate(As):
        samples.setdefault(A.shape[0], (A, Bs[f]))
    choice = autotune.tune(ctx, samples, tol=args.tol, precision=args.precision)
    autotune.save(choice, os.path.join(_scratch_dir(), "autotune_octree585.json"))
    # the per-size choices are timed on one front alone; the batch runs the
    # fronts concurrently, one batched build per rank cap, so the batch step
    # itself decides between them, the tuned leaves without caps (one group)
    # and the fixed rule (leaf 128 from n = 1024 on, else 64; no cap)
    candidates = {
        "tuned": [autotune.lookup(choice, A.shape[0]) for A in As],
        "tuned_leaves_uncapped": [(autotune.lookup(choice, A.shape[0])[0], 0) for A in As],
        "fixed": [(128 if A.shape[0] >= 1024 else 64, 0) for A in As],
    }

    def grouped(setting):
        groups = {}   # one batched build per rank cap
        for f, (leaf, cap) in enumerate(setting):
            groups.setdefault(cap, []).append(f)
        return groups

    def step(marks=None):
        hs = [None] * len(As)
        for cap, idx in groups.items():
            hg = H.hodlr_build_batched(ctx, [As[f] for f in idx], [setting[f][0] for f in idx], args.tol, "aca",
                                       precision=args.precision, rank_cap=cap)
            for f, h in zip(idx, hg):
                hs[f] = h
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

    batch_ms = {}
    for name, cand in candidates.items():
        setting, groups = cand, grouped(cand)
        step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        batch_ms[name] = min(ts)
    chosen = min(batch_ms, key=batch_ms.get)
    setting = candidates[chosen]
    groups = grouped(setting)
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
                       "autotuned": {str(k): {"leaf": v["leaf"], "rank_cap": v["rank_cap"], "ms": v["ms"]}
                                     for k, v in choice.items()},
                       "setting": chosen, "batch_ms_by_setting": batch_ms,
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
    leaf = WORKLOADS[args.workload]["front"]["leaf"]
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


def run_matvec_probe(args):
    """The many-rhs product alone: hodlr_matvec of a random n x n FP64 matrix
    with s right-hand sides (A's digit split and the tensor-core product), for
    a profiler capture of a case smaller than the workloads (--probe N S)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    n, s = args.probe
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    Z = torch.randn(s, n, dtype=torch.float64, device="cuda", generator=g)
    ctx = H.Context(0)
    for _ in range(args.warmup):
        H.hodlr_matvec(ctx, A, Z)
    torch.cuda.synchronize()
    H.hodlr_profile_enable(True)
    for _ in range(args.steps):
        H.hodlr_matvec(ctx, A, Z)
    torch.cuda.synchronize()
    out = {"n": n, "s": s}
    for k in ("oz_split_rows_kernel", "oz_split_cols_kernel", "oz_tc_gemm_kernel", "df_matvec_kernel"):
        ms, cnt = H.hodlr_profile_read(k)
        if cnt:
            out[k + "_ms"] = ms / cnt
    H.hodlr_profile_enable(False)
    print(json.dumps(out))


def run_apply_probe(args):
    """The HODLR apply alone on a workload's front: build and factor, release A,
    then time hodlr_solve on the workload's right-hand sides, for a profiler
    capture that holds only the factors on the device (--probe-apply)."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_1403_5337_gb300 as H
    F, Bh = make_inputs(args.workload, "cuda")
    leaf = WORKLOADS[args.workload]["front"]["leaf"]
    ctx = H.Context(0)
    h0 = H.hodlr_build(ctx, F.A, leaf, args.tol, args.method, graph=(F.rowptr, F.colind), precision=args.precision)
    image = H.hodlr_save(h0)
    h0.close()
    del F, h0
    torch.cuda.empty_cache()
    h = H.hodlr_load(ctx, image)        # the same factors, without A
    torch.cuda.reset_peak_memory_stats()
    X = torch.as_tensor(np.ascontiguousarray(Bh.T), device="cuda")
    for _ in range(args.warmup):
        H.hodlr_solve(h, X)
    torch.cuda.synchronize()
    H.hodlr_profile_enable(True)
    for _ in range(args.steps):
        H.hodlr_solve(h, X)
    torch.cuda.synchronize()
    ms, cnt = H.hodlr_profile_read("apply_fused_kernel")
    if not cnt:
        ms, cnt = H.hodlr_profile_read("apply_phase_kernel")
    H.hodlr_profile_enable(False)
    st = h.stats()
    h.close()
    print(json.dumps({"workload": args.workload, "precision": args.precision, "nrhs": int(X.shape[0]),
                      "apply_fused_kernel_ms": ms / max(cnt, 1), "launches": cnt,
                      "rank_pad": st["rank_pad"], "image_bytes": len(image),
                      "device_bytes_after_load": torch.cuda.max_memory_allocated()}))



def run_peaks(args):
    """Measured GEMM rates of the pipes the path uses beside the tensor cores:
    torch.matmul at 8192^3 in FP64 and in FP32 with TF32 off (SIMT), best of
    five with CUDA events (2 n^3 flops each)."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    n = 8192
    for name, dt in (("fp64_tflops", torch.float64), ("fp32_simt_tflops", torch.float32)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b
    out["how"] = "torch.matmul 8192^3, best of 5, CUDA events; FP32 with allow_tf32 = False"
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plane32768", choices=sorted(WORKLOADS) + ["octree585"])
    ap.add_argument("--method", default="aca", choices=["aca", "bdlr"])
    ap.add_argument("--tol", type=float, default=None, help="default: the workload's")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp16", "fp64"],
                    help="default: the workload's")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--nvtx", action="store_true", help="wrap every timed step in an NVTX range 'bench_step'")
    ap.add_argument("--kernels", action="store_true",
                    help="time each component alone (build, factor, apply, matvec, GMRES) with CUDA events; "
                         "the last repetition of each runs inside an NVTX range 'kernels' for ncu")
    ap.add_argument("--probe", type=int, nargs=2, metavar=("N", "S"),
                    help="time hodlr_matvec of a random N x N matrix with S right-hand sides")
    ap.add_argument("--peaks", action="store_true", help="measure the FP64 and FP32 (SIMT) GEMM rates")
    ap.add_argument("--probe-apply", action="store_true",
                    help="time hodlr_solve alone on the workload's factors, with A released")
    args = ap.parse_args()
    if args.peaks:
        return run_peaks(args)
    if args.workload == "octree585":
        args.precision = args.precision or "fp32"
        args.tol = args.tol or 1e-4
    else:
        args.precision = args.precision or WORKLOADS[args.workload]["precision"]
        args.tol = args.tol or WORKLOADS[args.workload]["tol"]
    if args.impl == "reference":
        return run_reference(args)
    if args.probe:
        return run_matvec_probe(args)
    if args.probe_apply:
        return run_apply_probe(args)
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
    import frontgen as fg
    import paper_1403_5337_gb300 as H

    wl = WORKLOADS[args.workload]
    F, Bh = make_inputs(args.workload, "cuda")
    A = F.A
    n = F.n
    nrhs = wl["nrhs"]
    leaf = wl["front"]["leaf"]
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
    x_gpu = X.cpu().numpy()

    # ---- the dominant kernels: their own launches, CUDA events on the
    # launching stream recorded by the library (after the timed region; inputs
    # larger than L2, and a 256 MiB write before each call)
    hbm, _, peak_kind = _peaks()
    comp_ms = statistics.median(s["ms_compress"] for _, s in infos)
    H.hodlr_profile_enable(True)
    hp = H.hodlr_build(ctx, A, leaf, args.tol, args.method, graph=graph, precision=args.precision)
    Z = torch.randn(nrhs, n, dtype=torch.float64, device="cuda")
    Xa = torch.empty_like(Z)
    for _ in range(5):
        flush.zero_()
        H.hodlr_matvec(ctx, A, Z)
        Xa.copy_(Z)
        flush.zero_()
        H.hodlr_solve(hp, Xa)
    torch.cuda.synchronize()
    prof = {}
    for k in ("aca_cluster_kernel", "gj_cluster_kernel", "apply_fused_kernel", "apply_phase_kernel", "df_matvec_kernel",
              "oz_split_rows_kernel", "oz_split_cols_kernel", "oz_tc_gemm_kernel"):
        ms, cnt = H.hodlr_profile_read(k)
        if cnt:
            prof[k] = {"launch_ms": ms / cnt, "launches": cnt}
    H.hodlr_profile_enable(False)
    pst = hp.stats()
    # the O10 preconditioner error on the seeded probe block (n x 16, stream 2)
    Om = torch.as_tensor(np.ascontiguousarray(fg.rhs(n, 16, seed=2).T), device="cuda")
    perr_gpu = H.hodlr_precond_error(hp, Om)
    hp.close()
    del Om
    n_mv = int(np.max(info.iters)) + 1 + info.restarts      # products per solve
    n_ap = int(np.max(info.iters)) + info.restarts          # applies per solve
    kernels = {}
    ranks = st["rank_mean"]
    w_c = 8 if args.precision == "fp64" else 4   # compression precision (FP32 below FP64)
    # ACA reads each pivot row/column of A once (FP64) and writes u_k, v_k once
    aca_bytes = sum((2 ** l) * ranks[l - 1] * 2 * (n / 2 ** l) * (8 + w_c) for l in range(1, st["levels"] + 1))
    kernels["aca_cluster_kernel"] = {"launch_ms": comp_ms, "ms_per_step": comp_ms, "bytes": aca_bytes,
                                     "note": "all levels' launches, concurrent: their wall time"}
    if "oz_tc_gemm_kernel" in prof:
        # the FP64-accurate product: 8 n^2 bytes of A per product (the
        # algorithm's), plus Z read and W written; the kernel itself streams
        # 7 n_p k_p bytes, A's exact digit bytes made once per solve
        t = prof["oz_tc_gemm_kernel"]["launch_ms"]
        kernels["oz_tc_gemm_kernel"] = {"launch_ms": t, "ms_per_step": t * n_mv,
                                        "bytes": 8.0 * n * n + 16.0 * n * nrhs,
                                        "kernel_bytes": 7.0 * (-(-n // 128) * 128) * (-(-n // 32) * 32)}
    elif "df_matvec_kernel" in prof:
        t = prof["df_matvec_kernel"]["launch_ms"] * -(-nrhs // 4)   # one launch per 4 rhs
        kernels["df_matvec_kernel"] = {"launch_ms": t, "ms_per_step": t * n_mv, "bytes": 8.0 * n * n + 16.0 * n * nrhs}
    # the apply: one cooperative launch, or (many tiles) one launch per phase
    # (timed over the phases of one call)
    ap_name = "apply_fused_kernel" if "apply_fused_kernel" in prof else "apply_phase_kernel"
    if ap_name in prof:
        t = prof[ap_name]["launch_ms"]
        ew = 8 if args.precision == "fp64" else (2 if args.precision in ("bf16", "fp16") else 4)
        wtot = sum(pst["rank_pad"])
        # V (n x rp) and E (n x 2 rp) of every level, the leaf inverses' rows, X in and out
        ap_bytes = 3.0 * n * wtot * ew + n * leaf * (8 if args.precision == "fp64" else 4) + 16.0 * n * nrhs
        kernels[ap_name] = {"launch_ms": t, "ms_per_step": t * n_ap, "bytes": ap_bytes}
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    kd = kernels[dom]
    achieved = kd["bytes"] / (kd["launch_ms"] * 1e-3) / 1e9
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": _traffic(dom, args.workload, args.precision),
                "share_of_step": kd["ms_per_step"] / ms_per_step,
                "others": {k: {"launch_ms": v["launch_ms"], "GBs": v["bytes"] / (v["launch_ms"] * 1e-3) / 1e9,
                               "ms_per_step": v["ms_per_step"]} for k, v in kernels.items()},
                "profiled_launch_ms": {k: v["launch_ms"] for k, v in prof.items()}}
    if "kernel_bytes" in kd:
        roofline["kernel_bytes"] = kd["kernel_bytes"]
        roofline["kernel_GBs"] = kd["kernel_bytes"] / (kd["launch_ms"] * 1e-3) / 1e9


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
    del A_host

    # ---- CPU oracle on the host cores (rank 0, N = 1): a bounded sample
    cpu, oracle = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fd, xpath = tempfile.mkstemp(suffix=".npy", dir=_scratch_dir())
        os.close(fd)
        try:
            r = _run_oracle({"workload": args.workload, "method": args.method, "tol": args.tol,
                             "mode": "baseline", "x_path": xpath, "omega": True})
            x_o = np.load(xpath)
            est = 1e3 * (r["t_build_factor"] + nrhs * r["t_gmres"])
            cpu = {"value": est, "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": f"FP64 oracle (NumPy, one BLAS thread) on the same front: build + factor "
                             f"({r['t_build_factor']:.1f} s) and GMRES to 1e-12 on rhs 0 ({r['t_gmres']:.1f} s, "
                             f"{r['iters']} iterations); value = build + factor + {nrhs} x that GMRES",
                   "oracle_iters_rhs0": r["iters"]}
            oracle = {"x_relerr_rhs0": float(np.linalg.norm(x_gpu[0] - x_o) / np.linalg.norm(x_o)),
                      "precond_error_fp64_oracle": r["precond_error"], "true_relres_rhs0": r["true_relres"]}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
        finally:
            os.unlink(xpath)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": _config(args, n),
            "converged": converged, "iters": info.iters.tolist(), "true_relres": info.true_relres.tolist(),
            "ranks_max": st["rank_max"], "ms_compress": comp_ms,
            "core_guard": {"threshold": st["core_cond_threshold"], "kappa1_max": st["core_cond_max"],
                           "cores_promoted": st["cores_promoted"]},
            # compression and factorisation overlap (level l is factored while
            # the levels above it are compressed): each phase is its own span
            "phases_ms": {"compress": comp_ms,
                          "factor": statistics.median(s["ms_factor"] for _, s in infos),
                          "gmres": statistics.median(i.ms_total for i, _ in infos),
                          "build_and_factor": ms_per_step - statistics.median(i.ms_total for i, _ in infos)},
            "precond_error": {"omega": "n x 16 N(0,1), counter stream 2",
                              "gpu": perr_gpu,
                              "fp64_oracle": oracle["precond_error_fp64_oracle"] if oracle else None},
            "x_vs_oracle": oracle,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "e2e": {"value": e2e_ms / world, "unit": "ms", "median_ms": statistics.median(e2e) / world,
                    "h2d_bytes_per_step": 8 * n * n + 8 * B.numel(),
                    "d2h_bytes_per_step": 8 * B.numel()},
            "fp64_path": compare,
            "gpu_launches": n_launches, "gpu_launches_per_step": n_launches / args.steps,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
