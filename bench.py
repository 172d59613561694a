"""Benchmark: NNLS solves/s of LHDM vs one-column LH on one GB300.

Workload (one "step" = one complete solve, every row of the hot path):
dense overdetermined NNLS, A 4096 x 2048 with U[0,1) entries, half of x zero,
b = A x + N(0, 1e-4) noise (seed 0), FP64.  The step is LHDM with k_max = 32
(tau1 = 0.6, tau2 = 0.15, delta = 0.9); the one-column LH solve of the same
instance on the same GPU is timed beside it.  A (64 MiB) fits in L2, so L2 is
flushed (a 512 MiB device write) before every timed solve.

Default arm: the CUDA path through the C ABI.  --impl reference: the CPU
oracle (plain C, the checker of the tests) timed on the host cores.

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy
(replicas; there is no data-path collective), the time is the max over ranks
and value = the solves of all ranks per second.
"""
import argparse
import json
import multiprocessing as mp
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NNLS solves/s: LHDM vs 1-col LH, same GB300, passive set exact, rel err<=1e-10"
WORKLOAD = ("overdetermined dense NNLS, A 4096x2048 U[0,1), 50% zero x, nonzeros U(0,1], "
            "b = A x + N(0,1e-4), seed 0, FP64")
DFMA_PER_CLK_PER_SM = 2.0  # measured on this machine's GB300 (DFMA microbenchmark)
MMA_SYNC_BF16_TFLOPS = 581.0  # mma.sync m16n8k16 bf16 with FP32 accumulation, measured on this machine's GB300


def _oracle_solve(k_max):
    """Runs in a spawned process: one oracle solve of the benchmark instance."""
    import numpy as np
    from oracle import oracle as O
    from paper_2108_05345_gb300 import workloads as WL
    A, b, _ = WL.overdetermined_uniform(0)
    t0 = time.perf_counter()
    r = O.nnls(A, b, k_max=k_max)
    dt = time.perf_counter() - t0
    return dict(seconds=dt, x=r["x"].tolist(), passive=r["passive"].tolist(), n_outer=r["n_outer"],
                status=r["status"])


class ClockSampler:
    """nvidia-smi samples of SM clock, power and throttle reasons."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "lhdm_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return out
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=sm[len(sm) // 2] if sm else None,
                   sm_max_mhz=float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def reference_arm(args):
    """The CPU oracle timed on the host cores: each step is one complete
    oracle solve of the benchmark instance; steps run in parallel on a
    spawned pool (one core each)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = max(1, min(os.cpu_count() or 1, args.steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        if args.warmup > 0:
            pool.map(_oracle_solve, [args.kmax] * min(args.warmup, cores))
        t0 = time.perf_counter()
        res = pool.map(_oracle_solve, [args.kmax] * args.steps)
        wall = time.perf_counter() - t0
    value = args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "k_max": args.kmax, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": "%d complete oracle LHDM solves of the benchmark instance, one per core" % args.steps},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "mean_solve_s": sum(r["seconds"] for r in res) / len(res),
    }
    print(json.dumps(line), flush=True)
    return 0


def once(args):
    """One solve (for ncu captures): the benchmark instance family at m x n."""
    import torch
    from paper_2108_05345_gb300 import lhdm, workloads as WL
    A, b, _ = WL.overdetermined_uniform(0, m=args.m, n=args.n)
    At = lhdm.colmajor(torch.from_numpy(A).cuda())
    bt = torch.from_numpy(b).cuda()
    ctx = lhdm.Context(args.m, args.n)
    x, p, info = ctx.solve(At, bt, lhdm.default_params(k_max=args.kmax))
    torch.cuda.synchronize()
    print(json.dumps({"once": True, "m": args.m, "n": args.n, "k_max": args.kmax, "info": info}))
    return 0



def kernel_sources_sha256():
    """Hash of the sources the solve kernel is built from (CUDA sources and
    the C header): a stored ncu traffic figure only applies to this hash."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_05345_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "lhdm.h"), "rb").read())
    return h.hexdigest()


def stored_profile(workload_tag):
    """The committed ncu summary (profiles/<kernel>_<workload>.json) of the
    solve kernel on this workload, if it was taken on the current sources:
    DRAM bytes per launch and the counters it lists; None otherwise."""
    path = os.path.join(ROOT, "profiles", "lhdm_solve_grid_kernel_%s.json" % workload_tag)
    try:
        prof = json.load(open(path))
        if prof.get("sources_sha256") == kernel_sources_sha256():
            return prof
    except Exception:
        pass
    return None


def _oracle_batched(i):
    """Spawned worker: one oracle solve of instance i of the batched workload
    (k_max 16, the value the tuner picks for the mid-size buckets)."""
    from oracle import oracle as O
    from paper_2108_05345_gb300 import workloads as WL
    m = WL.batched_sizes()[i]
    A, b, _ = WL.batched_instance(i, m)
    t0 = time.perf_counter()
    O.nnls(A, b, k_max=16)
    return time.perf_counter() - t0


def _oracle_layer(i):
    """Spawned worker: forward (oracle LHDM, k_max 32) and the closed-form
    adjoint of instance i of the layer workload."""
    import numpy as np
    from oracle import oracle as O
    from oracle.adjoint import nnls_adjoint
    from paper_2108_05345_gb300 import workloads as WL
    A, b, _, xt = WL.layer_batch(count=1, seed0=i)[0]
    t0 = time.perf_counter()
    r = O.nnls(A, b, k_max=32)
    nnls_adjoint(A, b, r["x"], r["passive"], 2.0 * (r["x"] - xt))
    return time.perf_counter() - t0


def cpu_pool_baseline(fn, items, unit, what):
    """fn over items on a spawned pool of every host core; solves/s of the
    sample and the core count."""
    cores = max(1, os.cpu_count() or 1)
    # one thread per worker: numpy's BLAS would otherwise start a thread per
    # core in every worker
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(fn, items[:cores])  # warm the workers (imports, oracle build)
            t0 = time.perf_counter()
            secs = pool.map(fn, items)
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": len(items) / wall, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": "%s: %d instances on %d spawned workers, %.1f s wall, %.2f s per instance"
                      % (what, len(items), cores, wall, sum(secs) / len(secs))}


def batched_section(lhdm, WL, torch, np):
    """Batched uneven workload (1024 instances, m ~ U{64..512}, n = 2m): k_max
    per size bucket from the autotuner, one persistent launch replayed from a
    captured CUDA graph, against a loop of single solves (a sample)."""
    inst = WL.batched_uneven(batch_seed=0, count=1024)
    As = [lhdm.colmajor(torch.from_numpy(A).cuda()) for A, _, _ in inst]
    bs = [torch.from_numpy(b).cuda() for _, b, _ in inst]
    table = lhdm.batch_autotune(As, bs, lhdm.default_params())
    batch = lhdm.Batch(As, bs, lhdm.default_params(k_max=0))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.run(stream)
    g.replay()
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / reps
    infos = batch.info()
    ok = all(i["status"] == 0 for i in infos)
    # loop of single solves (one whole-GPU launch each) on a sample, same k_max
    sample = list(range(0, 1024, 8))
    ctx = lhdm.Context(max(A.shape[0] for A in As), max(A.shape[1] for A in As))
    worst, same_p = 0.0, True
    ts = []
    for i in sample:
        prm = lhdm.default_params(k_max=batch.kmax(i))
        ctx.solve(As[i], bs[i], prm)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        x, p, _ = ctx.solve(As[i], bs[i], prm, sync=False)
        c.record()
        ts.append((a, c))
        xb = batch.xs[i]
        worst = max(worst, float(torch.linalg.norm(xb - x) / max(float(torch.linalg.norm(x)), 1e-300)))
        same_p = same_p and bool(torch.equal(batch.ps[i], p))
    torch.cuda.synchronize()
    ms_single = float(np.mean([a.elapsed_time(c) for a, c in ts]))
    ctx.close()
    batch.close()
    return {
        "workload": "1024 instances, m ~ U{64..512}, n = 2m, A ~ N(0,1/m), 10% nonzeros U(0.1,1], "
                    "b = A x0 + N(0,1e-3), batch seed 0",
        "kmax_table": table, "ms_per_batch": ms_batch, "solves_per_s": 1024 * 1000.0 / ms_batch,
        "graph": True, "all_status_ok": ok,
        "loop_of_single_solves": {"ms_per_solve": ms_single, "solves_per_s": 1000.0 / ms_single,
                                  "sample": "every 8th instance (128), same k_max, one launch each"},
        "speedup_vs_loop": (1024.0 / ms_batch) / (1.0 / ms_single),
        "parity_vs_single": {"max_rel_err": worst, "passive_identical": same_p},
    }


def layer_section(lhdm, WL, torch, np):
    """NNLS layer workload (256 instances of A 512x1024): batched forward
    (k_max = 32) and the batched adjoint for L = ||x - x_target||^2, against
    per-instance solve + backward on a sample."""
    inst = WL.layer_batch(count=256)
    As = [lhdm.colmajor(torch.from_numpy(A).cuda()) for A, _, _, _ in inst]
    bs = [torch.from_numpy(b).cuda() for _, b, _, _ in inst]
    xt = [torch.from_numpy(t).cuda() for _, _, _, t in inst]
    prm = lhdm.default_params(k_max=32)
    batch = lhdm.Batch(As, bs, prm)
    batch.run()
    torch.cuda.synchronize()
    gs = [2.0 * (x - t) for x, t in zip(batch.xs, xt)]
    batch.backward(gs)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    batch.run()
    e[1].record()
    torch.cuda.synchronize()
    gs = [2.0 * (x - t) for x, t in zip(batch.xs, xt)]
    torch.cuda.synchronize()
    e[1].record()
    dbs, dAs = batch.backward(gs)
    e[2].record()
    torch.cuda.synchronize()
    ms_f, ms_b = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    ok = all(i["status"] == 0 for i in batch.info())
    ctx = lhdm.Context(512, 1024)
    worst_x, worst_db, worst_dA = 0.0, 0.0, 0.0
    tf, tb = [], []
    for i in range(0, 256, 8):
        a, c, d = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        x, p, _ = ctx.solve(As[i], bs[i], prm, sync=False)
        c.record()
        db, dA = ctx.backward(As[i], 2.0 * (x - xt[i]))
        d.record()
        torch.cuda.synchronize()
        tf.append(a.elapsed_time(c))
        tb.append(c.elapsed_time(d))
        rel = lambda u, v: float(torch.linalg.norm(u - v) / max(float(torch.linalg.norm(v)), 1e-300))
        worst_x = max(worst_x, rel(batch.xs[i], x))
        worst_db = max(worst_db, rel(dbs[i], db))
        worst_dA = max(worst_dA, rel(dAs[i], dA))
    ctx.close()
    batch.close()
    return {
        "workload": "256 instances of A 512x1024 ~ N(0,1/512), 40 nonzeros U(0.1,1], b = A x0 + N(0,1e-3), "
                    "L = ||x - x_target||^2, x_target = x0 + 1e-2 xi",
        "k_max": 32, "forward_ms": ms_f, "backward_ms": ms_b,
        "solves_per_s": 256 * 1000.0 / ms_f, "all_status_ok": ok,
        "single": {"forward_ms_per_instance": float(np.mean(tf)), "backward_ms_per_instance": float(np.mean(tb)),
                   "sample": "every 8th instance (32)"},
        "parity_vs_single": {"x": worst_x, "dLdb": worst_db, "dLdA": worst_dA},
    }


def _time_solve(ctx, lhdm, torch, At, bt, prm, reps=3, flush=None, **kw):
    """Median CUDA-event time (ms) of `reps` solves (one warm-up first) and
    the info of the last; kw selects solve_l1 (lam=...)."""
    def run():
        if "lam" in kw:
            return ctx.solve_l1(At, bt, kw["lam"], prm, sync=False)
        return ctx.solve(At, bt, prm, sync=False)
    run()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = run()
        c.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(c))
    ts.sort()
    return ts[len(ts) // 2], out, ctx.info()


def kmax_section(lhdm, WL, torch, np, At, bt, ctx, flush):
    """The 4096 x 2048 benchmark instance at k_max 16 and 64 (the headline
    is k_max 32)."""
    out = {}
    for k in (16, 64):
        ms, _, info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=k), flush=flush)
        out["k%d" % k] = {"ms": ms, "solves_per_s": 1000.0 / ms, "n_outer": int(info["n_outer"]),
                          "n_passive": int(info["n_passive"])}
    return out


def small_section(lhdm, WL, torch, np):
    """The 256 x 512 recovery instance (seed 0): LHDM k_max = 8 vs LH."""
    A, b, x0 = WL.small_recovery(0)
    At = lhdm.colmajor(torch.from_numpy(A).cuda())
    bt = torch.from_numpy(b).cuda()
    ctx = lhdm.Context(*A.shape)
    out = {"workload": "A 256x512 N(0,1/256), x0 25 nonzeros U(0.1,1], b = A x0, seed 0 (L2-resident; no flush)"}
    for name, k in (("lhdm_k8", 8), ("lh", 1)):
        ms, (x, p, _), info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=k), reps=10)
        xr = x.cpu().numpy()
        out[name] = {"ms": ms, "solves_per_s": 1000.0 / ms, "n_outer": int(info["n_outer"]),
                     "recovery_rel_err": float(np.linalg.norm(xr - x0) / np.linalg.norm(x0))}
    out["speedup_vs_lh"] = out["lh"]["ms"] / out["lhdm_k8"]["ms"]
    ctx.close()
    return out


def sparse_section(lhdm, WL, torch, np):
    """Sparse-recovery sweep (A 2048x8192 Gaussian, unit-norm columns,
    s in {64, ..., 1024} nonzeros, noiseless): LHDM k_max = 64 vs LH,
    time-to-solution and recovery per s."""
    out = {"workload": "A 2048x8192 N(0,1) unit-norm columns, x0 s nonzeros U(0.1,1], b = A x0, seed 0"}
    ctx = lhdm.Context(2048, 8192)
    for s in (64, 128, 256, 512, 1024):
        A, b, x0 = WL.sparse_recovery_sweep(0, s)
        At = lhdm.colmajor(torch.from_numpy(A).cuda())
        bt = torch.from_numpy(b).cuda()
        row = {}
        for name, k in (("lhdm_k64", 64), ("lh", 1)):
            ms, (x, p, _), info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=k), reps=1)
            xr = x.cpu().numpy()
            row[name] = {"ms": ms, "n_outer": int(info["n_outer"]), "n_passive": int(info["n_passive"]),
                         "resid": float(info["resid_norm"]),
                         "recovery_rel_err": float(np.linalg.norm(xr - x0) / np.linalg.norm(x0)),
                         "support_exact": np.flatnonzero(xr > 1e-9 * xr.max()).tolist() == np.flatnonzero(x0).tolist()}
        row["speedup_vs_lh"] = row["lh"]["ms"] / row["lhdm_k64"]["ms"]
        out["s%d" % s] = row
        del At, bt
    ctx.close()
    return out


def signed_section(lhdm, WL, torch, np):
    """Positivity trick (NNLS on [A -A] without forming -A), LHDM k_max and
    LH, each with the inner loop and with the sign flip: signed sparse
    recovery (A 2048x8192 unit-norm Gaussian columns, s = 128 signed
    nonzeros, noiseless; no negative y arises) and signed least squares
    (A 2048x1024 Gaussian, x ~ N(0,1), b = A x + N(0,1): the inner loop and
    the sign flip both run)."""
    out = {}
    cases = (("recovery", WL.signed_recovery(0, m=2048, n=8192, s=128, unit_columns=True), 64,
              "[A -A], A 2048x8192 N(0,1) unit-norm columns, x0 128 signed nonzeros, b = A x0, seed 0"),
             ("least_squares", WL.signed_overdetermined(0, m=2048, n=1024, noise_var=1.0), 32,
              "[A -A], A 2048x1024 N(0,1/2048), x ~ N(0,1), b = A x + N(0,1), seed 0"))
    for tag, (A, b, x0), k_dm, desc in cases:
        At = lhdm.colmajor(torch.from_numpy(A).cuda())
        bt = torch.from_numpy(b).cuda()
        ctx = lhdm.Context(*A.shape)
        row = {"workload": desc}
        for name, k, mode in (("lhdm_k%d" % k_dm, k_dm, 1), ("lhdm_k%d_flip" % k_dm, k_dm, 2), ("lh", 1, 1),
                              ("lh_flip", 1, 2)):
            ms, (x, p, _), info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=k, mode=mode), reps=1)
            xr = x.cpu().numpy()
            n = A.shape[1]
            r = {"ms": ms, "n_outer": int(info["n_outer"]), "n_inner": int(info["n_inner"]),
                 "n_flip": int(info["n_flip"]), "resid": float(info["resid_norm"])}
            if tag == "recovery":
                expect = np.concatenate([np.maximum(x0, 0), np.maximum(-x0, 0)])
                r["recovery_rel_err"] = float(np.linalg.norm(xr - expect) / np.linalg.norm(expect))
            row[name] = r
        row["lh_flip_speedup_vs_lh"] = row["lh"]["ms"] / row["lh_flip"]["ms"]
        row["lhdm_speedup_vs_lh"] = row["lh"]["ms"] / row["lhdm_k%d" % k_dm]["ms"]
        out[tag] = row
        ctx.close()
    return out


def l1_section(lhdm, WL, torch, np):
    """l1-NNLS (the stacked [1^T 1^T; lam A -lam A] system) on A 512x1024
    with noisy signed sparse data, a sweep of lam."""
    A, b0, x0 = WL.signed_recovery(0, m=512, n=1024, s=40)
    b = b0 + 1e-3 * np.random.default_rng(5).normal(size=512)
    At = lhdm.colmajor(torch.from_numpy(A).cuda())
    bt = torch.from_numpy(b).cuda()
    ctx = lhdm.Context(513, 2048)
    out = {"workload": "l1-NNLS, A 512x1024 N(0,1/512), x0 40 signed nonzeros, b = A x0 + 1e-3 N(0,1), seed 0",
           "k_max": 32, "sweep": {}}
    total = 0.0
    for lam in (1.0, 10.0, 100.0):
        ms, (x, p, _), info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=32), reps=3, lam=lam)
        xr = x.cpu().numpy()
        xs = xr[:1024] - xr[1024:]
        total += ms
        out["sweep"]["lam=%g" % lam] = {"ms": ms, "n_outer": int(info["n_outer"]), "n_passive": int(info["n_passive"]),
                                        "l1": float(np.abs(xs).sum()),
                                        "dist_to_x0": float(np.linalg.norm(xs - x0) / np.linalg.norm(x0))}
    out["sweep_ms"] = total
    ctx.close()
    return out


def conditioned_section(lhdm, WL, torch, np):
    """Ill-conditioned dense NNLS (condition number ~1e6): A 2048x1024,
    LHDM k_max = 32 vs LH."""
    A, b, _ = WL.conditioned_overdetermined(0, kappa=1e6)
    At = lhdm.colmajor(torch.from_numpy(A).cuda())
    bt = torch.from_numpy(b).cuda()
    ctx = lhdm.Context(*A.shape)
    out = {"workload": "A 2048x1024 = U diag(sigma) V^T, sigma 1..1e-6 log-spaced, unit-norm columns, "
                       "50% zero x, b = A x + N(0,1e-4), seed 0"}
    for name, k in (("lhdm_k32", 32), ("lh", 1)):
        ms, _, info = _time_solve(ctx, lhdm, torch, At, bt, lhdm.default_params(k_max=k), reps=1)
        out[name] = {"ms": ms, "n_outer": int(info["n_outer"]), "n_passive": int(info["n_passive"])}
    out["speedup_vs_lh"] = out["lh"]["ms"] / out["lhdm_k32"]["ms"]
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lhdm", choices=["lhdm", "reference"])
    ap.add_argument("--kmax", type=int, default=32)
    ap.add_argument("--lh-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline and parity leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, layer and sparse-recovery workloads reported beside the headline")
    ap.add_argument("--once", action="store_true",
                    help="profiling mode: exactly one solve of the benchmark instance, no warm-up")
    ap.add_argument("--m", type=int, default=4096, help="rows of the instance (--once only)")
    ap.add_argument("--n", type=int, default=2048, help="columns of the instance (--once only)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.once:
        return once(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU leg starts first, in a spawned process (before any CUDA call)
    cpu_job = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pool = mp.get_context("spawn").Pool(1)
        cpu_job = pool.apply_async(_oracle_solve, (args.kmax,))

    import numpy as np
    import torch
    from paper_2108_05345_gb300 import lhdm, workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    A, b, _ = WL.overdetermined_uniform(0)
    m, n = A.shape
    dev = torch.device("cuda", local)
    At = lhdm.colmajor(torch.from_numpy(A).to(dev))
    bt = torch.from_numpy(b).to(dev)
    ctx = lhdm.Context(m, n)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    prm = lhdm.default_params(k_max=args.kmax)
    prm_lh = lhdm.default_params(k_max=1)

    def timed(params, steps):
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.solve(At, bt, params, sync=False)
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in ts]

    # warm-up, then the timed LHDM steps with clocks sampled meanwhile
    timed(prm, max(3, args.warmup))
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    t_lhdm = timed(prm, args.steps)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    x, p, info = ctx.solve(At, bt, prm)
    ms_ph, fl_ph, n_mma = ctx.profile_full()
    trace = ctx.trace()
    ms = float(np.mean(t_lhdm))
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * 1000.0 / ms

    # one-column LH on the same GPU
    timed(prm_lh, 1)
    t_lh = timed(prm_lh, args.lh_steps)
    x_lh, p_lh, info_lh = ctx.solve(At, bt, prm_lh)
    ms_lh = float(np.mean(t_lh))

    # end to end: host buffers through lhdm_solve_host (copies inside)
    Ah = torch.from_numpy(np.asfortranarray(A).T.copy()).pin_memory()  # column-major bytes
    bh = torch.from_numpy(b.copy()).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    ph = torch.empty(n, dtype=torch.int32).pin_memory()
    ctx.solve_host_ptr(m, n, Ah.data_ptr(), m, bh.data_ptr(), xh.data_ptr(), ph.data_ptr(), prm)
    e2e_ts = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_host_ptr(m, n, Ah.data_ptr(), m, bh.data_ptr(), xh.data_ptr(), ph.data_ptr(), prm)
        e2e_ts.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_ts))

    if rank != 0:
        return 0

    # roofline of the solve kernel (FP64-ALU bound) and of its dual GEMV phase
    sm_mhz_peak = 2070.0
    try:
        mp_json = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(mp_json.get("hbm_gbs", 6791.4))
        sm_mhz_peak = float(mp_json.get("sm_max_mhz", 2070.0))
        hbm_src = "measured"
    except Exception:
        hbm, hbm_src = 6800.0, "fallback"
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = DFMA_PER_CLK_PER_SM * 2.0 * nsm * sm_mhz_peak * 1e6 / 1e12  # TFLOP/s
    flops_total = sum(fl_ph.values())
    kernel_ms = float(np.median(t_lhdm))
    achieved = flops_total / (kernel_ms * 1e-3) / 1e12
    nZ_bytes = fl_ph["dual"] / 2.0 * 8.0 if fl_ph["dual"] else 0.0  # 8 bytes of A per FMA
    dual_gbs = nZ_bytes / (ms_ph["dual"] * 1e-3) / 1e9 if ms_ph["dual"] > 0 else None
    # the units that bind the solve, each against its own peak:
    #  - streaming A: 8 m n per outer step plus 8 m nP for the residual
    #    (the per-solve bytes of the method's BLAS-2 part), over the solve time;
    #  - the FP64 pipe: the algorithmic FP64 flops of every phase but the
    #    tensor-core commit, over the time of those phases;
    #  - the tensor pipe: the commit's bf16 MMAs (m16n8k16, 4096 flops),
    #    over the commit time, against the mma.sync bf16 rate measured on this
    #    pool's GB300 (the cuBLAS figure of MEASURED_PEAKS is tcgen05)
    sum_np = float(trace[:, 3].sum()) if len(trace) else 0.0
    bytes_stream = 8.0 * m * n * info["n_outer"] + 8.0 * m * sum_np
    stream_gbs = bytes_stream / (kernel_ms * 1e-3) / 1e9
    fp64_ms = sum(v for k, v in ms_ph.items() if k != "commit")
    fp64_flops = sum(v for k, v in fl_ph.items() if k != "commit")
    mma_tflops = n_mma * 4096.0 / (ms_ph["commit"] * 1e-3) / 1e12 if ms_ph["commit"] > 0 else 0.0
    prof = stored_profile("4096x2048")

    # parity against the CPU oracle (same instance, same parameters)
    x_np, p_np = x.cpu().numpy(), p.cpu().numpy()
    parity = None
    cpu_baseline = None
    if cpu_job is not None:
        ref = cpu_job.get()
        xr = np.array(ref["x"])
        Pg = p_np[p_np >= 0].tolist()
        rel = float(np.linalg.norm(x_np - xr) / np.linalg.norm(xr))
        xl = x_lh.cpu().numpy()
        pl = p_lh.cpu().numpy()
        parity = {"passive_exact": Pg == ref["passive"], "rel_err": rel,
                  "lh_passive_exact": pl[pl >= 0].tolist() == ref["passive"],
                  "lh_rel_err": float(np.linalg.norm(xl - xr) / np.linalg.norm(xr)),
                  "oracle_outer": ref["n_outer"], "gpu_outer": int(info["n_outer"])}
        cpu_baseline = {"value": 1.0 / ref["seconds"], "unit": "solves/s", "cores": 1, "kind": "oracle",
                        "sample": "one complete oracle LHDM (k_max=%d) solve of the benchmark instance (%.1f s)"
                                  % (args.kmax, ref["seconds"])}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "k_max": args.kmax, "tau1": 0.6, "tau2": 0.15, "delta": 0.9,
                   "l2": "flushed before every timed solve (512 MiB device write)",
                   "parallelism": "replicas" if world > 1 else "single GPU, one persistent launch per solve"},
        "lh": {"value": world * 1000.0 / ms_lh, "unit": "solves/s", "ms_per_step": ms_lh,
               "n_outer": int(info_lh["n_outer"]), "steps": args.lh_steps},
        "speedup_vs_lh": ms_lh / ms,
        "solve": {k: info[k] for k in ("status", "n_outer", "n_inner", "n_drop", "n_passive")},
        "parity": parity,
        "roofline": {"bound": "alu", "kernel": "lhdm_solve_grid_kernel", "achieved": achieved,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "peak_source": "derived: %.0f DFMA/clk/SM (measured) x %d SMs x %.0f MHz"
                                    % (DFMA_PER_CLK_PER_SM, nsm, sm_mhz_peak),
                     "algorithmic_flops": flops_total,
                     "achieved_meaning": "FP64-equivalent: the commit's share runs on the bf16 tensor cores",
                     "traffic": prof["dram_bytes_per_launch"] if prof else None,
                     "traffic_unit": "DRAM bytes per launch (ncu, profiles/*.json; null if the sources changed since)",
                     "units": {
                         "hbm_stream_A": {"achieved": stream_gbs, "peak": hbm, "unit": "GB/s",
                                          "frac": stream_gbs / hbm, "peak_source": hbm_src,
                                          "bytes": bytes_stream,
                                          "bytes_formula": "8 m n N_outer + 8 m sum_steps nP"},
                         "fp64_pipe": {"achieved": fp64_flops / (fp64_ms * 1e-3) / 1e12 if fp64_ms > 0 else None,
                                       "peak": fp64_peak, "unit": "TFLOP/s",
                                       "frac": (fp64_flops / (fp64_ms * 1e-3) / 1e12) / fp64_peak if fp64_ms > 0 else None,
                                       "scope": "all phases but the commit, over their time"},
                         "tensor_pipe": {"achieved": mma_tflops, "peak": MMA_SYNC_BF16_TFLOPS, "unit": "TFLOP/s",
                                         "frac": mma_tflops / MMA_SYNC_BF16_TFLOPS, "mma_instructions": n_mma,
                                         "scope": "the commit's bf16 mma.sync digit products over the commit time",
                                         "peak_source": "measured mma.sync m16n8k16 bf16 rate on this pool's GB300"},
                     },
                     "ncu": {k: prof[k] for k in prof if k not in ("sources_sha256",)} if prof else None},
        "dual_gemv": {"achieved_gbs": dual_gbs, "hbm_peak_gbs": hbm, "hbm_source": hbm_src,
                      "frac_of_hbm": (dual_gbs / hbm) if dual_gbs else None,
                      "fp64_frac": ((fl_ph["dual"] / (ms_ph["dual"] * 1e-3) / 1e12) / fp64_peak) if ms_ph["dual"] else None},
        "phases_ms": {k: round(v, 4) for k, v in ms_ph.items()},
        "cpu_baseline": cpu_baseline,
        "e2e": {"value": 1.0 / e2e_s * world, "unit": "solves/s",
                "h2d_bytes_per_step": 8 * m * n + 8 * m, "d2h_bytes_per_step": 8 * n + 4 * n + 48},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if not args.no_extra and world == 1:
        line["kmax"] = kmax_section(lhdm, WL, torch, np, At, bt, ctx, flush)
        line["small"] = small_section(lhdm, WL, torch, np)
        line["batched"] = batched_section(lhdm, WL, torch, np)
        line["layer"] = layer_section(lhdm, WL, torch, np)
        line["sparse_recovery"] = sparse_section(lhdm, WL, torch, np)
        line["signed"] = signed_section(lhdm, WL, torch, np)
        line["l1"] = l1_section(lhdm, WL, torch, np)
        line["conditioned"] = conditioned_section(lhdm, WL, torch, np)
        if not args.no_cpu:
            sizes = WL.batched_sizes()
            line["batched"]["cpu_baseline"] = cpu_pool_baseline(
                _oracle_batched, list(range(0, 1024, 8)), "solves/s",
                "oracle LHDM (k_max 16) of every 8th batched instance")
            line["layer"]["cpu_baseline"] = cpu_pool_baseline(
                _oracle_layer, list(range(0, 256, 4)), "solves/s",
                "oracle LHDM (k_max 32) forward + closed-form adjoint of every 4th layer instance")
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
