"""Benchmark: batched FastGM sketch throughput on one GB300 (or N, one per rank).

Workload (a step = one gm_sketch call over the whole batch): 4,096 CSR rows,
n+ ~ LogNormal(ln 2000, 1) clipped to [10, 200,000], ids uniform without
replacement in [0, 2^24), weights Exp(1), k = 1024, seed 1 -- the synthetic
stand-in for the paper's sparse-vector workloads.  Inputs (~163 MB of ids and
weights) are larger than the 129 MB L2, so no flush is needed between steps.

Reported: sketches/s (value), elements/s, the O(k n+) plain sketch on the same
batch, the same at k = 4096, an end-to-end number through host buffers, the
roofline of the dominant kernel, and the CPU oracle as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketches/s and elements/s at k=1024/4096 FastGM vs plain O(kn+) on 1 GB300; % roofline"
WORKLOAD = ("lognormal_batch: 4096 CSR rows, n+ ~ LogNormal(ln 2000, 1) clipped to [10, 200000], "
            "ids uniform w/o replacement in [0, 2^24), weights Exp(1), k=1024, seed=1")
N_ROWS, K_MAIN, K_ALT, SEED = 4096, 1024, 4096, 1
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--cpu-rows", type=int, default=0, help="rows of the CPU-oracle sample (0 = auto)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only", default="all", choices=["all", "fastgm"],
                    help="fastgm: time only the FastGM step (the case profiled with ncu)")
    ap.add_argument("--k", type=int, default=K_MAIN, help="k of the --only fastgm step")
    ap.add_argument("--arith", action="store_true",
                    help="time the per-arrival arithmetic: FP64 unit vs integer pipes (diagnostic kernels)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[0]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for i, n in enumerate(names) if any(r[3 + i].lower().startswith("active") for r in rows)]
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": num(rows[0][1]), "reasons": reasons,
                "samples": len(rows), "power_w_max": float(np.nanmax([num(r[2]) for r in rows]))}


def algorithmic_bytes(nnz, n_rows, k):
    """Bytes a sketch launch must move at least: read each (int32 id, f64 weight) once,
    write each register (int32 s, f64 y) once."""
    return 12 * nnz + 12 * n_rows * k


def cpu_baseline(X, k, seed, rows_budget_s=15.0, n_rows=0):
    """The oracle (unpruned full stream, plain C, one row per call on a thread pool) on a
    bounded random sample of the batch's rows; throughput scaled to sketches/s."""
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(12345)
    lens = np.diff(X.row_ptr)
    if n_rows <= 0:
        # size the sample for ~rows_budget_s at ~4e6 arrivals/s per core
        per_row_s = float(lens.mean()) * k / 4.0e6
        n_rows = int(max(threads, min(X.n_rows, rows_budget_s * threads / max(per_row_s, 1e-9))))
    rows = np.sort(rng.choice(X.n_rows, size=min(n_rows, X.n_rows), replace=False))
    oracle.lib()
    t0 = time.perf_counter()
    oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, seed, rows, threads=threads)
    dt = time.perf_counter() - t0
    nnz = int(lens[rows].sum())
    return {"value": rows.size / dt, "unit": "sketches/s", "cores": threads, "kind": "oracle",
            "elements_per_s": nnz / dt, "seconds": dt,
            "sample": "%d random rows of the batch (%d elements), k=%d, unpruned full stream, %d host threads" %
                      (rows.size, nnz, k, threads)}


def run_arith(args):
    """Throughput of the FP64 / FP32 FMA units and of the per-arrival operations on
    the FP64 unit and on the integer pipes (include/gm_diag.h)."""
    import ctypes
    import torch
    from paper_2302_05176_gb300 import build as libbuild
    L = ctypes.CDLL(libbuild.build())
    vp = ctypes.c_void_p
    L.gm_diag_fma.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp]
    L.gm_diag_neglog.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    L.gm_diag_dmul.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    L.gm_diag_drcp.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    st = vp(torch.cuda.current_stream().cuda_stream)
    P = lambda t: vp(t.data_ptr())
    nsm = torch.cuda.get_device_properties(0).multi_processor_count

    def time_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"metric": "arithmetic throughput per GB300", "unit": "ops/s"}
    blocks, iters = nsm * 8, 4096
    buf = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    for fp64, name in ((1, "fp64_fma"), (0, "fp32_fma")):
        it = iters if fp64 else iters * 8
        ms = time_ms(lambda: L.gm_diag_fma(fp64, blocks, it, P(buf), st))
        out[name] = 8.0 * it * blocks * 256 / (ms * 1e-3)
    n = 1 << 24
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.integers(0, 2**62, size=n, dtype=np.int64)).cuda()
    a = torch.from_numpy(1.0 + rng.random(n)).cuda()
    b = torch.from_numpy(1.0 + rng.random(n)).cuda()
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    for fp64, tag in ((1, "fp64_unit"), (0, "integer")):
        out["neg_log_" + tag] = n / (time_ms(lambda: L.gm_diag_neglog(P(x), n, fp64, P(y), st)) * 1e-3)
        out["mul_" + tag] = n / (time_ms(lambda: L.gm_diag_dmul(P(a), P(b), n, fp64, P(y), st)) * 1e-3)
        out["rcp_" + tag] = n / (time_ms(lambda: L.gm_diag_drcp(P(a), n, fp64, P(y), st)) * 1e-3)
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2302_05176_gb300 import workloads as W
    X = W.lognormal_batch(seed=SEED, n_rows=N_ROWS)
    per_step = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(X, K_MAIN, SEED, rows_budget_s=3.0)
        if i >= args.warmup:
            per_step.append(info["seconds"] / info["value"] * N_ROWS)  # seconds for the whole batch
    v = float(np.mean([N_ROWS / s for s in per_step]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sketches/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(per_step)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "sketches/s", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"] + "; each step extrapolated to the 4096-row batch"},
            "e2e": {"value": v, "unit": "sketches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.arith:
        return run_arith(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2302_05176_gb300 import gm
    from paper_2302_05176_gb300 import workloads as W
    gm.lib()

    # weak scaling: every rank sketches its own batch of the same shape
    X = W.lognormal_batch(seed=SEED + rank, n_rows=N_ROWS)
    rp, ids, w = gm.to_device(X)
    n_rows, nnz = X.n_rows, X.nnz
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, k, steps, warmup, flags=0):
        s_out = torch.empty((n_rows, k), dtype=torch.int32, device="cuda")
        y_out = torch.empty((n_rows, k), dtype=torch.float64, device="cuda")
        ws = gm.workspace(n_rows, nnz, k)
        for _ in range(warmup):
            fn(rp, ids, w, k, SEED, flags=flags, s_out=s_out, y_out=y_out, ws=ws)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn(rp, ids, w, k, SEED, flags=flags, s_out=s_out, y_out=y_out, ws=ws)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        code, st = gm.gm_status(ws)
        if code != gm.GM_OK:
            raise RuntimeError("device status %s" % gm.strerror(code))
        return ms, st

    if args.only == "fastgm":
        ms, st = timed(gm.gm_sketch, args.k, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * n_rows / (ms * 1e-3), "unit": "sketches/s",
                              "ms_per_step": ms, "only": "fastgm k=%d" % args.k, "stats": st}), flush=True)
        return
    clocks = ClockSampler(local)
    clocks.start()
    ms_main, st_main = timed(gm.gm_sketch, K_MAIN, args.steps, args.warmup)
    clk = clocks.stop()
    ms_alt, st_alt = timed(gm.gm_sketch, K_ALT, max(2, args.steps // 3), args.warmup)
    ms_plain, st_plain = timed(gm.gm_sketch_plain, K_MAIN, args.plain_steps, 1)

    # end to end through the C-ABI with host buffers: H2D of the inputs and D2H of the
    # registers inside the timed region, every step
    h_rp = torch.from_numpy(X.row_ptr).pin_memory()
    h_ids = torch.from_numpy(X.ids).pin_memory()
    h_w = torch.from_numpy(X.w).pin_memory()
    h_s = torch.empty((n_rows, K_MAIN), dtype=torch.int32).pin_memory()
    h_y = torch.empty((n_rows, K_MAIN), dtype=torch.float64).pin_memory()
    d_rp, d_ids, d_w = torch.empty_like(rp), torch.empty_like(ids), torch.empty_like(w)
    d_s = torch.empty((n_rows, K_MAIN), dtype=torch.int32, device="cuda")
    d_y = torch.empty((n_rows, K_MAIN), dtype=torch.float64, device="cuda")
    ws = gm.workspace(n_rows, nnz, K_MAIN)

    def e2e_step():
        d_rp.copy_(h_rp, non_blocking=True)
        d_ids.copy_(h_ids, non_blocking=True)
        d_w.copy_(h_w, non_blocking=True)
        gm.gm_sketch(d_rp, d_ids, d_w, K_MAIN, SEED, s_out=d_s, y_out=d_y, ws=ws)
        h_s.copy_(d_s, non_blocking=True)
        h_y.copy_(d_y, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = X.row_ptr.nbytes + X.ids.nbytes + X.w.nbytes
    d2h = n_rows * K_MAIN * (4 + 8)

    hbm_gbs, peak_src = peaks()
    abytes = algorithmic_bytes(nnz, n_rows, K_MAIN)
    achieved = abytes / (ms_main * 1e-3) / 1e9
    value = world * n_rows / (ms_main * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "sketches/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_main, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows_per_gpu": n_rows, "nnz_per_gpu": nnz, "k": K_MAIN,
                   "l2": "inputs %.0f MB > 129 MB L2; no flush" % (h2d / 1e6), "parallelism": "rows sharded, dp%d" % world},
        "elements_per_s": world * nnz / (ms_main * 1e-3),
        "arrivals_per_sketch": st_main["arrivals"] / n_rows,
        "k4096": {"sketches_per_s": world * n_rows / (ms_alt * 1e-3), "ms_per_step": ms_alt,
                  "elements_per_s": world * nnz / (ms_alt * 1e-3)},
        "plain_k1024": {"sketches_per_s": world * n_rows / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                        "arrivals_per_s": st_plain["arrivals"] / (args.plain_steps + 1) / (ms_plain * 1e-3)},
        "speedup_vs_plain_k1024": ms_plain / ms_main,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                     "frac": achieved / hbm_gbs, "traffic": None, "peak_source": peak_src,
                     "kernel": "sketch_kernel<false>", "algorithmic_bytes_per_launch": abytes},
        "e2e": {"value": world * n_rows / e2e_s, "unit": "sketches/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(X, K_MAIN, SEED, n_rows=args.cpu_rows)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
