#!/usr/bin/env python3
"""Benchmark of the GP marginal log-likelihood + gradient on GB300.

One step = one evaluation of loglik and d loglik / d(log s2, log rho, log tau2)
through the C ABI (gp_loglik_grad): covariance fill, blocked Cholesky,
solves with refinement, reductions, blocked inverse and the gradient
contraction.  Default workload: the paper-scale problem n = 67,275 (the size
of the Sec. 4 supernova data set), Matern 3/2 with sigma2 = 1, rho = 0.02,
tau2 = 0.1 on 50 Gaussian clusters (sd 0.02) plus 20% uniform background,
y = L z, in the mixed form (BF16-slice tcgen05 contractions, FP64 pivots,
log-determinant and residuals).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun, one rank per GPU) every rank evaluates its own
replica: the single large problem does not shard (replicas only), so the
whole-job value is N x K evaluations over the slowest rank's time.

After the timed region (unless --no-extras) the same JSON line also carries,
measured in the same run: the Cholesky factorisation alone in the mixed and
FP64-grade forms (n^3/3 over its CUDA-event time), the FP64-grade form's
loglik+grad on the same inputs (its time and the mixed form's error against
it), and the batched workload (512 problems, one CUDA-graph replay per step)
in the mixed and FP64 forms.

--impl reference times the FP64 CPU oracle (the plain implementation the
parity tests use) on the host cores, on a bounded sample of the same
workload, and prints the same JSON line with "impl": "reference".
--cpu-plan n1,n2,.. times the oracle at those sizes with all cores and one
thread, and LAPACK's Cholesky, and prints one JSON line per measurement.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_HEADLINE = 67275
METRIC = "GP loglik+grad evaluations/s at n=67,275"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_HEADLINE, help="problem size (exploration only)")
    ap.add_argument("--precision", default="mixed_f16", choices=["mixed_f16", "emu_fp64", "fp64"],
                    help="mixed_f16: three FP16 slices (6 products); emu_fp64: five BF16 "
                         "integer slices (15 products, FP64-grade); fp64: CUDA-core FP64")
    ap.add_argument("--workload", default="single", choices=["single", "batched"],
                    help="single: the n=67,275 problem (default); batched: 512 small problems")
    ap.add_argument("--nprob", type=int, default=512,
                    help="batched workload: number of problems (exploration only; 512 is the workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-error", action="store_true",
                    help="(kept for older command lines; the comparison is part of the extras)")
    ap.add_argument("--accuracy", default=None,
                    help="comma-separated n: print mixed / FP64-grade errors against the "
                         "FP64 path on the config-3 recipe at each n, then exit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline run without the Cholesky-only timing, the FP64-grade "
                         "form and the batched workload")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="evaluations in the end-to-end (host buffers) measurement")
    ap.add_argument("--emu-steps", type=int, default=2,
                    help="timed evaluations of the FP64-grade form")
    ap.add_argument("--batched-steps", type=int, default=10,
                    help="timed graph replays of the batched workload")
    ap.add_argument("--case", default=None,
                    choices=["fill", "loglik", "loglik_grad", "syrk", "predict", "product"],
                    help="run one small invocation of a single step (--n, --precision, --reps) "
                         "for kernel captures, print its CUDA-event times, then exit")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cpu-plan", default=None,
                    help="comma-separated n: time the oracle (all cores and one thread) "
                         "and LAPACK's Cholesky at each n, then exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def lpt_partition(sizes, world, rank):
    """Problems of rank `rank` when independent problems of the given sizes are
    shared over `world` ranks: longest-processing-time first (cost ~ n^3), each
    to the least-loaded rank; returns the problem indices in ascending order."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    loads = [0.0] * world
    mine = []
    for i in order:
        k = min(range(world), key=lambda r: (loads[r], r))
        loads[k] += float(sizes[i]) ** 3
        if k == rank:
            mine.append(i)
    return sorted(mine)


def gather_batched(local, mine, nprob, dist, device):
    """The batched results of every rank on every rank: `local` holds this
    rank's rows (k columns) for its problems `mine` (ascending indices);
    returns the nprob x k array with every problem's row in its place.  One
    all-gather of fixed-size row blocks (the ranks' shares differ in length:
    each is padded to the longest) and of the index lists; without a process
    group, the local rows in place."""
    import torch
    local = torch.as_tensor(local, dtype=torch.float64, device=device)
    k = local.shape[1]
    full = torch.full((nprob, k), float("nan"), dtype=torch.float64, device=device)
    if dist is None:
        full[torch.as_tensor(mine, device=device)] = local
        return full
    world = dist.get_world_size()
    cnt = torch.tensor([len(mine)], dtype=torch.int64, device=device)
    cnts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(cnts, cnt)
    m = int(max(int(c.item()) for c in cnts))
    rows = torch.full((m, k), float("nan"), dtype=torch.float64, device=device)
    rows[: len(mine)] = local
    idx = torch.full((m,), -1, dtype=torch.int64, device=device)
    idx[: len(mine)] = torch.as_tensor(mine, dtype=torch.int64, device=device)
    all_rows = [torch.empty_like(rows) for _ in range(world)]
    all_idx = [torch.empty_like(idx) for _ in range(world)]
    dist.all_gather(all_rows, rows)
    dist.all_gather(all_idx, idx)
    for r in range(world):
        sel = all_idx[r] >= 0
        full[all_idx[r][sel]] = all_rows[r][sel]
    return full


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest rank's time); the value
    itself without a process group."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(n, precision):
    return {
        "workload": f"GP loglik+grad, Matern 3/2, n={n}, 2-D clustered locations "
                    "(50 clusters sd 0.02 + 20% uniform), sigma2=1 rho=0.02 tau2=0.1, y=Lz",
        "n": n,
        "kernel": "matern32",
        "precision": precision,
        "seed": 48863,
        "l2": "inputs larger than L2 (n_p^2 FP64 matrix, no flush needed)",
    }


# ---------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def source_digest(path):
    """sha256 prefix of a source file's code: comments and blank lines are left
    out, so that an edit of the comments keeps a measurement valid."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    code = "\n".join(ln for ln in lines if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "tc_gemm3_kernel_traffic.json")
TRAFFIC_SRC = os.path.join(ROOT, "paper_1305_4886_gb300", "csrc", "tc_gemm.cu")


def contraction_traffic(flops_per_launch, prec, path=TRAFFIC_FILE, src=TRAFFIC_SRC):
    """DRAM bytes per average contraction launch: the committed ncu figure
    (dram bytes read + written per slice-product flop over every contraction
    launch of one loglik+grad step) times this run's slice-product flops per
    launch; None when the kernel's code has changed since the capture or no
    figure exists for this precision."""
    try:
        with open(path) as f:
            rec = json.load(f)
        digest = source_digest(src)
    except (OSError, ValueError):
        return None
    if rec.get("tc_gemm_code_sha256_prefix") != digest:
        return None
    ratio = rec.get("bytes_per_slice_flop", {}).get(prec)
    if not ratio or not flops_per_launch:
        return None
    return {"bytes_per_launch": float(ratio) * flops_per_launch,
            "source": f"{os.path.relpath(path, ROOT)} (n={rec.get('n')}): dram bytes per "
                      "slice-product flop x this run's flops per launch"}


# The oracle sample that both arms time: one loglik+grad on the headline
# recipe at this size, extrapolated to the headline n by the n^3 cost.
CPU_SAMPLE_N = 4096


def oracle_time(n, threads=None):
    """Seconds of one oracle loglik+grad on the config-3 recipe at size n."""
    import oracle
    from paper_1305_4886_gb300 import inputs
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    p = inputs.config3(n)
    t0 = time.perf_counter()
    oracle.loglik_grad(p.x, p.z, p.kernel, p.s2, p.rho, p.tau2)
    return time.perf_counter() - t0


def oracle_sample(n_target, n_s=CPU_SAMPLE_N):
    """The oracle's loglik+grad at n_s (after a small warm-up call),
    extrapolated to n_target by n^3.  Returns (evals/s at n_target,
    description, threads)."""
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    oracle_time(256)  # thread start-up and page faults
    t_s = oracle_time(n_s)
    t_full = t_s * (n_target / n_s) ** 3
    desc = (f"oracle loglik+grad on the same recipe at n={n_s} ({t_s:.2f} s, {threads} threads), "
            f"extrapolated to n={n_target} by n^3")
    return 1.0 / t_full, desc, threads


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    # one step = one oracle loglik+grad on the same bounded sample of the
    # workload that our arm's cpu_baseline times, extrapolated by n^3
    n_s = min(CPU_SAMPLE_N, args.n)
    oracle_time(256)
    for _ in range(args.warmup):
        oracle_time(n_s)
    ts = [oracle_time(n_s) for _ in range(args.steps)]
    t_step = sum(ts) / len(ts)
    t_full = t_step * (args.n / n_s) ** 3
    value = 1.0 / t_full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_full * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.n, "fp64 (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step: oracle loglik+grad at n={n_s} "
                                   f"({t_step:.2f} s mean over {args.steps}), extrapolated "
                                   f"to n={args.n} by n^3"},
        "measured_ms_per_sample": t_step * 1e3,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cpu_plan(args):
    """The CPU baseline table: the oracle's loglik+grad at several n, with all
    host cores and with one thread, and LAPACK's Cholesky (scipy cho_factor)
    on the oracle's covariance, one JSON line per measurement."""
    import numpy as np
    import oracle
    import scipy.linalg
    from paper_1305_4886_gb300 import inputs
    oracle.build()
    cores = oracle.num_threads()
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
    except OSError:
        pass
    host = {"nproc": os.cpu_count(), "model": model}
    oracle_time(256)
    sizes = [int(v) for v in args.cpu_plan.split(",")]
    for n in sizes:
        for thr in (cores, 1):
            if thr == 1 and n > 4096:
                continue  # one thread at n > 4096 takes longer than a bench call allows
            t = oracle_time(n, threads=thr)
            print(json.dumps({"kind": "oracle loglik+grad", "n": n, "threads": thr, "s": t,
                              "extrapolated_to_67275_s": t * (67275 / n) ** 3, "host": host}),
                  flush=True)
        oracle.set_threads(cores)
        p = inputs.config3(n)
        C = oracle.cov_fill(p.x, p.kernel, p.s2, p.rho, p.tau2)
        t0 = time.perf_counter()
        scipy.linalg.cho_factor(C, lower=True, overwrite_a=True, check_finite=False)
        t = time.perf_counter() - t0
        print(json.dumps({"kind": "library CPU: scipy.linalg.cho_factor (LAPACK)", "n": n,
                          "threads": "library default", "s": t,
                          "gflops": n ** 3 / 3 / t / 1e9, "host": host}), flush=True)
        del C
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _mk_graph(fn):
    """Capture fn() (launches on the current stream) into a CUDA graph on a side
    stream and return the graph."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    return graph


def batched_measure(probs, prec, steps, warmup, autotune=True, task_stats=True):
    """Config-5 style batch: one gp_loglik_grad_batched call per step, captured
    once into a CUDA graph and replayed; returns a dict of measurements."""
    import numpy as np
    import torch

    from paper_1305_4886_gb300 import gp

    xs = [torch.as_tensor(p.x, device="cuda") for p in probs]
    zs = [torch.as_tensor(p.z, device="cuda") for p in probs]
    prms = [gp.params(p.kernel, p.s2, p.rho, p.tau2) for p in probs]
    r = gp.loglik_grad_batched(xs, zs, prms, precision=prec)
    torch.cuda.synchronize()
    batch, ws = r["batch"], r["ws"]
    out, grad, info = r["out"], r["grad"], r["info"]
    tile_policy = None
    if prec == "mixed_f16" and autotune:
        # the tile autotuner: FP64 64 x 64 tiles below a size threshold,
        # tensor-core 128 x 128 tiles above it, chosen by timing this batch
        choice, cand_ms = gp.gp_batched_autotune(batch, prec, ws, out, grad, info)
        torch.cuda.synchronize()
        tile_policy = {"fp64_tiles_up_to_n": choice,
                       "candidates_ms": {str(k): round(v, 3) for k, v in cand_ms.items()}}
    for _ in range(max(0, warmup - 1)):
        gp.gp_loglik_grad_batched(batch, prec, ws, out, grad, info)
    torch.cuda.synchronize()
    graph = _mk_graph(lambda: gp.gp_loglik_grad_batched(batch, prec, ws, out, grad, info))
    graph.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    bad = int((info != 0).sum().item())
    rres = out[:, 3].double().cpu().numpy()
    flops = sum(float(p.n) ** 3 for p in probs)
    res = {"precision": prec, "steps": steps, "warmup": warmup, "ms_per_batch": ms / steps,
           "evals_per_s": len(probs) * steps / (ms / 1e3), "failed_problems": bad,
           "loglik_grad_alg_tflops": flops * steps / (ms / 1e3) / 1e12,
           "graph": "one CUDA graph per step", "tiles": tile_policy or "FP64 64 x 64",
           "out": out.cpu().numpy(), "grad": grad.cpu().numpy()}
    if prec == "mixed_f16":
        res["refine_resid"] = {"max": float(np.max(rres)), "median": float(np.median(rres))}
    if task_stats and prec in ("fp64", "mixed_f16"):
        # one more (untimed) batch with the task graph's cycle counters on:
        # where the persistent launch spends its CTA time, per task class
        gp.gp_batched_profile(True)
        gp.gp_loglik_grad_batched(batch, prec, ws, out, grad, info)
        torch.cuda.synchronize()
        gp.gp_batched_profile(False)
        st = gp.gp_batched_task_stats(ws)
        mhz = 2070.0
        ts = {k: {"cta_ms": v["cycles"] / (mhz * 1e3), "wait_ms": v["wait_cycles"] / (mhz * 1e3),
                  "tasks": v["tasks"]}
              for k, v in st.items() if k != "steps" and v["tasks"]}
        if st["steps"]:
            # one step: a 128 x 128 x 128 tile product, six 16-bit slice products
            ts["tensor_steps"] = st["steps"]
            ts["slice_tflops_per_step_time"] = st["steps"] * 6 * 2 * 128.0 ** 3 / (ms / steps / 1e3) / 1e12
        res["task_stats"] = ts
    del ws, r, graph
    torch.cuda.empty_cache()
    return res


def time_cholesky(x, prm, n, prec, ws, info, reps):
    """CUDA-event time of gp_chol alone (the fill is redone, untimed, before
    each repetition) on the matrix region of a loglik workspace, whose tail
    serves as the factorisation's workspace.  Returns the median ms."""
    import torch

    from paper_1305_4886_gb300 import gp
    np_ = gp.gp_padded_order(n)
    A = ws[: np_ * np_ * 8].view(torch.float64)
    tail = ws[np_ * np_ * 8:]
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        gp.gp_cov_fill(x, prm, A, np_, precision=prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gp.gp_chol(A, n, np_, prec, tail, info)
        e1.record(stream)
        torch.cuda.synchronize()
        if int(info.item()) != 0:
            raise RuntimeError(f"gp_chol failed, info={int(info.item())}")
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1305_4886_gb300 import gp, inputs

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gp.lib()

    n = args.n
    prec = args.precision
    p = inputs.config3(n)
    prm = gp.params(p.kernel, p.s2, p.rho, p.tau2)
    np_ = gp.gp_padded_order(n)
    x = torch.as_tensor(p.x, device="cuda")
    z = torch.as_tensor(p.z, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    grad = torch.empty(3, dtype=torch.float64, device="cuda")
    alpha = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    extras = rank == 0 and not args.no_extras and prec == "mixed_f16"

    # y = L z with the FP64-grade factor of C(theta) (untimed set-up; at this
    # size the CUDA-core FP64 factor takes minutes, and the FP64-grade one
    # agrees with it to about 1e-12)
    y_form = "emu_fp64" if prec != "fp64" else "fp64"
    ws_ref = gp.workspace(n, y_form, want_grad=True)
    gp.gp_loglik(x, z, None, n, prm, y_form, ws_ref, out, None, info)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    gp.gp_mult_chol(ws_ref[: np_ * np_ * 8].view(torch.float64), n, np_, z, y)
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"set-up factorisation failed, info={int(info.item())}")
    if not extras:
        del ws_ref
        ws_ref = None
        torch.cuda.empty_cache()
    ws = gp.workspace(n, prec, want_grad=True)

    def step():
        gp.gp_loglik_grad(x, y, None, n, prm, prec, ws, out, alpha, grad, info)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"warm-up failed, info={int(info.item())}")

    # ---- timed region: inputs resident in HBM ----
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    gp.gp_prof_enable(True)
    launches0 = gp.gp_launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = gp.gp_launch_count() - launches0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    # every profiled launch of the timed region is recorded, or this raises
    prof = {c: gp.gp_prof_read(c) for c in gp.PROF_CLASSES}
    roles = {c: gp.gp_prof_read(c) for c in gp.PROF_CONTRACT_ROLES}
    gp.gp_prof_enable(False)
    if int(info.item()) != 0:
        raise RuntimeError(f"timed steps failed, info={int(info.item())}")
    elapsed_ms = max_over_ranks(elapsed_ms, dist if dist else None, "cuda")
    value = world * args.steps / (elapsed_ms / 1e3)
    res = out.cpu().numpy()
    g_res = grad.cpu().numpy()
    a_res = alpha.cpu().numpy()

    # ---- end to end through the public API: host buffers in, scalars out ----
    e2e = None
    if not args.no_e2e:
        ksteps = max(1, min(args.steps, args.e2e_steps))
        x_h = torch.as_tensor(p.x).pin_memory()
        y_h = y.cpu().pin_memory()
        out_h = torch.empty(4, dtype=torch.float64).pin_memory()
        grad_h = torch.empty(3, dtype=torch.float64).pin_memory()
        x_d = torch.empty_like(x)
        y_d = torch.empty_like(y)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(ksteps):
            x_d.copy_(x_h, non_blocking=True)
            y_d.copy_(y_h, non_blocking=True)
            gp.gp_loglik_grad(x_d, y_d, None, n, prm, prec, ws, out, alpha, grad, info)
            out_h.copy_(out, non_blocking=True)
            grad_h.copy_(grad, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        e2e_ms = max_over_ranks(e2e_ms, dist if dist else None, "cuda")
        e2e = {"value": world * ksteps / (e2e_ms / 1e3), "unit": UNIT, "steps": ksteps,
               "h2d_bytes_per_step": int(x_h.numel() * 8 + y_h.numel() * 8),
               "d2h_bytes_per_step": int((out_h.numel() + grad_h.numel()) * 8)}

    peaks, peak_src = measured_peaks()
    ms_c, cnt_c, fl_c, _ = prof["contract"]
    peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    pairs = {"mixed_f16": 6, "emu_fp64": 15}.get(prec, 0)
    slice_tf = fl_c / (ms_c / 1e3) / 1e12 if ms_c > 0 else None
    # algorithmic (FP64-equivalent) flops of the contractions: the useful
    # output entries and K ranges, 2 flops per multiply-add, not the split
    # products that carry them
    alg_c = fl_c / pairs if pairs else fl_c
    alg_tf = alg_c / (ms_c / 1e3) / 1e12 if ms_c > 0 else None
    traffic = contraction_traffic(fl_c / max(cnt_c, 1), prec)
    kname = {"mixed_f16": "tc_gemm3_kernel (tcgen05 contraction, three FP16 slices, one "
                          "accumulator per product group, two MMA issuers",
             "emu_fp64": "tc_gemm_kernel<4> (tcgen05 contraction, five BF16 slices"}.get(
                 prec, "gemm_f64_kernel (FP64 CUDA cores")
    roofline = {
        "kernel": kname + "; Cholesky update, panel solve, TRTRI/LAUUM)",
        "bound": "tensor", "achieved": alg_tf, "peak": peak_tf, "unit": "TFLOP/s",
        "frac": (alg_tf / peak_tf) if alg_tf else None,
        "traffic": traffic["bytes_per_launch"] if traffic else None,
        "traffic_source": traffic["source"] if traffic else None,
        "peak_source": f"bf16 sustained, {peak_src}", "launches": cnt_c,
        "share_of_step": ms_c / elapsed_ms if elapsed_ms > 0 else None,
        "flops_counted": "algorithmic: 2 flops per multiply-add of the FP64 products the "
                         "contractions stand for (useful output entries and K ranges), per launch "
                         "(average)",
        "alg_flops_per_step": alg_c / args.steps,
        "slice_products": {"per_fp64_product": pairs, "achieved": slice_tf,
                           "frac": (slice_tf / peak_tf) if slice_tf else None,
                           "note": "the tensor pipe's own work: every 16-bit slice product "
                                   "counted"},
    }
    ms_f, cnt_f, _, by_f = prof["fill"]
    fill = {"achieved_gbs": (by_f / (ms_f / 1e3) / 1e9) if ms_f > 0 else None,
            "peak_gbs": peaks.get("hbm_gbs"), "ms_per_launch": ms_f / max(cnt_f, 1),
            "bound": "fp32 alu (double-float kernel evaluation)" if prec != "fp64"
                     else "fp64 alu (exp)"}
    fill["frac_of_hbm"] = (fill["achieved_gbs"] / fill["peak_gbs"]) if fill["achieved_gbs"] else None
    chol_alg = n ** 3 / 3.0
    per_step = {c: prof[c][0] / args.steps for c in prof}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed_f16": "f64 + fp16 slices (fp32 accumulate)",
                  "emu_fp64": "f64 + bf16 integer slices (fp32 accumulate)"}.get(prec, "f64"),
        "data": "synthetic", "config": workload_config(n, prec), "clocks": clk,
        "e2e": e2e, "gpu_launches": int(launches), "launches_before_timed": int(launches0),
        "roofline": roofline, "fill": fill,
        "result": {"loglik": float(res[0]), "logdet": float(res[1]), "quad": float(res[2]),
                   "refine_resid": float(res[3]), "grad": [float(v) for v in g_res]},
        "loglik_grad_alg_tflops": n ** 3 / (elapsed_ms / args.steps / 1e3) / 1e12,
        "per_step_ms": per_step,
        "per_step_ms_profiled_sum": sum(per_step.values()),
        "per_step_ms_note": ("diag_chol, diag_inv and the diagonal rows' fold run on a side "
                             "stream under the trailing updates (lookahead): the classes "
                             "overlap, so their sum exceeds ms_per_step"),
        "per_step_launches": {c: prof[c][1] / args.steps for c in prof},
        "contract_by_role": {c: {"ms_per_step": roles[c][0] / args.steps,
                                 "alg_tflops": (roles[c][2] / pairs / (roles[c][0] / 1e3) / 1e12)
                                 if roles[c][0] > 0 and pairs else None}
                             for c in roles},
        "cholesky_alg_flop": chol_alg,
        "y": f"L z with the {y_form} factor",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }

    if extras:
        # ---- the Cholesky alone (the metric's first clause), mixed form ----
        t_chol = time_cholesky(x, prm, n, prec, ws, info, reps=3)
        chol = {prec: {"ms": t_chol, "tflops": chol_alg / (t_chol / 1e3) / 1e12}}
        del ws
        torch.cuda.empty_cache()
        # ---- the FP64-grade form (five BF16 integer slices), same workload ----
        r_ws = ws_ref
        for _ in range(1):
            gp.gp_loglik_grad(x, y, None, n, prm, "emu_fp64", r_ws, out, alpha, grad, info)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.emu_steps):
            gp.gp_loglik_grad(x, y, None, n, prm, "emu_fp64", r_ws, out, alpha, grad, info)
        f1.record(stream)
        torch.cuda.synchronize()
        if int(info.item()) != 0:
            raise RuntimeError(f"FP64-grade evaluation failed, info={int(info.item())}")
        emu_ms = f0.elapsed_time(f1) / args.emu_steps
        ro, rg, ra = out.cpu().numpy(), grad.cpu().numpy(), alpha.cpu().numpy()
        t_chol_e = time_cholesky(x, prm, n, "emu_fp64", r_ws, info, reps=2)
        chol["emu_fp64"] = {"ms": t_chol_e, "tflops": chol_alg / (t_chol_e / 1e3) / 1e12}
        del r_ws, ws_ref
        torch.cuda.empty_cache()
        line["cholesky"] = chol
        line["cholesky_tflops"] = chol[prec]["tflops"]
        line["emu_fp64"] = {
            "evals_per_s": 1e3 / emu_ms, "ms_per_eval": emu_ms, "steps": args.emu_steps,
            "warmup": 1, "speedup_of_mixed": emu_ms / (elapsed_ms / args.steps),
            "result": {"loglik": float(ro[0]), "grad": [float(v) for v in rg]}}
        line["error"] = {
            "against": "emu_fp64 (five BF16 integer slices, FP64-grade), same run and inputs",
            "loglik_rel": float(abs(res[0] - ro[0]) / abs(ro[0])),
            "grad_rel_inf": float(np.max(np.abs(g_res - rg)) / np.max(np.abs(rg))),
            "alpha_rel": float(np.linalg.norm(a_res - ra) / np.linalg.norm(ra))}
        # ---- the batched workload (512 problems, one graph replay per step) ----
        probs = inputs.config5(nprob=args.nprob)
        bm = batched_measure(probs, "mixed_f16", args.batched_steps, 3)
        bf = batched_measure(probs, "fp64", 2, 1, task_stats=False)
        ob, gb = bm.pop("out"), bm.pop("grad")
        of, gf = bf.pop("out"), bf.pop("grad")
        bm["error_vs_fp64"] = {
            "loglik_rel_max": float(np.max(np.abs(ob[:, 0] - of[:, 0]) / np.abs(of[:, 0]))),
            "grad_rel_inf_max": float(np.max(np.max(np.abs(gb - gf), axis=1) /
                                              np.max(np.abs(gf), axis=1)))}
        line["batched"] = {"workload": "512 independent GPs, n log-uniform [256, 4096], 2-D "
                                       "uniform locations, exp / Matern 3/2 alternating, "
                                       "y ~ N(0, I)", "seed": 48865,
                           "mixed_f16": bm, "fp64": bf}

    if rank == 0 and not args.no_cpu_baseline:
        v, desc, thr = oracle_sample(n)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_accuracy(args):
    """Errors of the mixed and FP64-grade forms against the CUDA-core FP64
    path (config-3 recipe, y = L z with the FP64 factor), one JSON line per n
    and form, with each form's evaluation time."""
    import numpy as np
    import torch

    from paper_1305_4886_gb300 import gp, inputs

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    for n in [int(v) for v in args.accuracy.split(",")]:
        p = inputs.config3(n)
        x = torch.as_tensor(p.x, device="cuda")
        z = torch.as_tensor(p.z, device="cuda")
        np_ = gp.gp_padded_order(n)
        ws = gp.workspace(n, "fp64", want_grad=True)
        gp.loglik(x, z, p.kernel, p.s2, p.rho, p.tau2, precision="fp64", ws=ws)
        y = torch.empty_like(z)
        gp.gp_mult_chol(gp.factor_view(ws, n).reshape(-1), n, np_, z, y)
        ref, ms64 = timed(lambda: gp.loglik_grad(x, y, p.kernel, p.s2, p.rho, p.tau2,
                                                 precision="fp64", ws=ws))
        ro, rg, ra = (ref["out"].cpu().numpy(), ref["grad"].cpu().numpy(),
                      ref["alpha"].cpu().numpy())
        print(json.dumps({"n": n, "precision": "fp64", "ms": ms64, "loglik": float(ro[0]),
                          "grad": [float(v) for v in rg]}), flush=True)
        del ws, ref
        torch.cuda.empty_cache()
        for prec in ["mixed_f16", "emu_fp64"]:
            r, ms = timed(lambda: gp.loglik_grad(x, y, p.kernel, p.s2, p.rho, p.tau2,
                                                 precision=prec))
            o, g, a = r["out"].cpu().numpy(), r["grad"].cpu().numpy(), r["alpha"].cpu().numpy()
            del r
            torch.cuda.empty_cache()
            print(json.dumps({"n": n, "precision": prec, "against": "fp64", "ms": ms,
                              "loglik_rel": float(abs(o[0] - ro[0]) / abs(ro[0])),
                              "logdet_rel": float(abs(o[1] - ro[1]) / abs(ro[1])),
                              "grad_rel_inf": float(np.max(np.abs(g - rg)) / np.max(np.abs(rg))),
                              "alpha_rel": float(np.linalg.norm(a - ra) / np.linalg.norm(ra))}),
                  flush=True)
    return 0


def run_batched(args, rank, world, local):
    """The batched workload: 512 independent problems, n log-uniform in
    [256, 4096], exponential / Matern 3/2 alternating, one gp_loglik_grad_batched
    call per step, captured once into a CUDA graph and replayed.  With N ranks
    the problems are partitioned by cost (no collective on the data path)."""
    import torch

    from paper_1305_4886_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    probs = inputs.config5(nprob=args.nprob)
    # longest-processing-time partition of the problems over ranks
    mine = lpt_partition([p.n for p in probs], world, rank)
    sel = [probs[i] for i in mine]
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    res = batched_measure(sel, args.precision, args.steps, args.warmup)
    clk = clocks.stop()
    # every problem's loglik and gradient on rank 0's side too (host gather)
    outs = gather_batched(res.pop("out"), mine, len(probs), dist, "cuda")
    grads = gather_batched(res.pop("grad"), mine, len(probs), dist, "cuda")
    res["gathered_problems"] = int(torch.isfinite(outs[:, 0]).sum().item())
    res["gathered_grad_finite"] = bool(torch.isfinite(grads).all().item())
    ms = max_over_ranks(res["ms_per_batch"] * args.steps, dist, "cuda")
    value = len(probs) * args.steps / (ms / 1e3)
    prec = args.precision
    line = {"metric": f"batched GP loglik+grad evaluations/s ({len(probs)} problems, n in [256, 4096])",
            "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed_f16": "f64 + fp16 slices (fp32 accumulate)",
                      "emu_fp64": "f64 + bf16 integer slices (fp32 accumulate)"}.get(prec, "f64"),
            "data": "synthetic",
            "config": {"workload": "512 independent GPs, n log-uniform [256, 4096], 2-D uniform "
                                   "locations, exp / Matern 3/2 alternating, y ~ N(0, I)",
                       "precision": prec, "seed": 48865, "graph": res["graph"],
                       "tiles": res["tiles"]},
            "clocks": clk, "detail": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_case(args):
    """One step of the path on its own, --reps times, on the config-3 recipe
    at --n: the case a kernel capture (ncu) runs.  Prints one JSON line with
    the CUDA-event time of each repetition."""
    import torch

    from paper_1305_4886_gb300 import gp, inputs
    n, prec = args.n, args.precision
    p = inputs.config3(n)
    prm = gp.params(p.kernel, p.s2, p.rho, p.tau2)
    x = torch.as_tensor(p.x, device="cuda")
    z = torch.as_tensor(p.z, device="cuda")
    np_ = gp.gp_padded_order(n)
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    if args.case == "fill":
        C = torch.empty(np_ * np_, dtype=torch.float64, device="cuda")
        fn = lambda: gp.gp_cov_fill(x, prm, C, np_, precision=prec)  # noqa: E731
        work = {"bytes": 8.0 * np_ * (np_ + 64) / 2}
    elif args.case in ("loglik", "loglik_grad"):
        ws = gp.workspace(n, prec, want_grad=args.case == "loglik_grad")
        if args.case == "loglik":
            fn = lambda: gp.loglik(x, z, p.kernel, p.s2, p.rho, p.tau2, precision=prec, ws=ws)  # noqa: E731
        else:
            fn = lambda: gp.loglik_grad(x, z, p.kernel, p.s2, p.rho, p.tau2, precision=prec, ws=ws)  # noqa: E731
        work = {"flop": n ** 3 / 3.0 if args.case == "loglik" else float(n) ** 3}
    elif args.case == "syrk":
        # one trailing update C -= P P^T with P n x 512 (a Cholesky step)
        P = torch.randn(512 * n, dtype=torch.float64, device="cuda")
        C = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        ws = torch.empty(max(1, gp.gp_syrk_workspace_bytes(n, 512, prec)), dtype=torch.uint8,
                         device="cuda")
        fn = lambda: gp.gp_syrk_lower(C, n, P, n, n, 512, prec, ws, info)  # noqa: E731
        work = {"flop": float(n) * n * 512}
    elif args.case == "product":
        # the paper's example model on its data set's shape: 25 phases x n/25
        # log wavelengths (n = 67,275 is the paper's 25 x 2691)
        q = inputs.product_grid(25, max(1, n // 25))
        xq = torch.as_tensor(q.x, device="cuda")
        yq = torch.as_tensor(q.z, device="cuda") * 0.1
        vq = torch.as_tensor(q.meta["v"], device="cuda")
        wsq = gp.workspace(q.n, prec, want_grad=True)
        fn = lambda: gp.loglik_product(xq, yq, q.s2, q.rho, q.meta["rho_w"], q.tau2, v=vq,  # noqa: E731
                                       precision=prec, ws=wsq)
        work = {"flop": float(q.n) ** 3, "n_product": q.n}
    else:
        m = max(1, n // 2)
        xs = torch.as_tensor(inputs.uniform_points(m, 4242), device="cuda")
        lk = gp.loglik(x, z, p.kernel, p.s2, p.rho, p.tau2, precision=prec)
        mean = torch.empty(m, dtype=torch.float64, device="cuda")
        var = torch.empty(m, dtype=torch.float64, device="cuda")
        pws = torch.empty(gp.gp_predict_workspace_bytes(n, m, True), dtype=torch.uint8,
                          device="cuda")
        L = lk["ws"][: np_ * np_ * 8].view(torch.float64)
        fn = lambda: gp.gp_predict(x, n, xs, m, prm, lk["alpha"], L, np_, 0.0, mean, var, pws,  # noqa: E731
                                   info)
        work = {"flop": float(np_) * np_ * m, "m": m}
    times = []
    for _ in range(max(1, args.reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if int(info.item()) != 0:
        raise RuntimeError(f"case {args.case} failed, info={int(info.item())}")
    print(json.dumps({"case": args.case, "n": n, "precision": prec, "ms": times, **work}),
          flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.cpu_plan:
        return run_cpu_plan(args) if rank == 0 else 0
    if args.accuracy:
        return run_accuracy(args) if rank == 0 else 0
    if args.case:
        return run_case(args) if rank == 0 else 0
    if args.workload == "batched":
        return run_batched(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
