"""Benchmark: H^2 x H^2 products per second at block-relative eps = 1e-6.

Workload (one step = one product C = A*B through h2_mul, inputs resident in
HBM): 128 x 128 grid on the unit square (n = 16384), A = -log|x-y|/(2 pi)
(diagonal 1), B = exp(-|x-y|^2/0.1), leaf size 64, eta 2, tensor Chebyshev
order 4 (k = 16).  `value` is the chosen form: the products run as batches
(h2_batch: merged launches and persistent GEMM chains, one CUDA graph replay
per batch) with the tensor-core contractions (precision 4), timed with CUDA
events around the replays; `plain_fp64` is h2_mul one product per step in
FP64, timed the same way; the served form and a request stream shaped like
the serving workload are reported beside them.

Roofline: the algorithmic work of one product is the one counted by the CPU
oracle's counters (tests/golden/work_counts.json, written from the oracle
alone); the dominant kernel kind's share of it over that kind's measured time
gives `achieved`.  The work the GPU kernels execute (their own counts) is
reported beside it.

Prints one JSON line (rank 0).  Multi-GPU (torchrun): independent replicas,
one per GPU, no collective on the data path ("scaling": "weak").

--impl reference times the CPU oracle (numpy FP64, single thread, spawned
process) on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H²×H² products/s at block-rel eps=1e-6, chosen vs plain FP64 form; p50/p99 ms"
UNIT = "products/s"
GRID = 128
EPS = 1e-6
KIND_NAMES = ["k_gemm", "k_copy", "k_qr", "k_qapply", "k_svd", "k_scan", "k_finalize", "k_norm"]
# profile kind 8: the tensor-core GEMM stages again (a subset of k_gemm), with
# the multiply-adds issued to the tensor cores as their flops
TC_KIND = "k_gemm_tc"


def workload_config(grid=GRID):
    return {
        "workload": f"grid2d_n{grid * grid}: C=A*B, A=-log|x-y|/(2pi) diag 1, B=exp(-|x-y|^2/0.1), "
                    f"leaf 64, eta 2, Chebyshev order 4 (k=16), eps={EPS:g}",
        "n": grid * grid, "k": 16, "leaf_size": 64, "eta": 2.0, "eps": EPS,
        "l2": "flushed between timed steps (256 MiB write)",
    }


def load_json(*parts):
    try:
        return json.load(open(os.path.join(ROOT, *parts)))
    except (OSError, ValueError):
        return None


# oracle work kinds charged to each GPU kernel kind
ORACLE_KIND = {"k_gemm": ("gemm",), "k_qr": ("qr",), "k_qapply": (), "k_svd": ("svd",), "k_norm": ("norm",)}


def kernel_table(kinds, mw, peak, hbm_peak, tc=None, bf16_peak=None):
    """Per kernel of the profiled product: launches, time, executed and
    oracle-counted work, and the fraction of its roofline (FP64 ALU peak for
    the arithmetic kernels, HBM copy bandwidth for k_copy).  k_gemm mixes
    tensor-core and compensated-FP32 stages; its fraction is against the FP64
    peak the plain form would be bound by.  tc: the tensor-core stages of
    k_gemm, their multiply-adds on the tensor cores against the BF16 peak."""
    out = {}
    if tc is not None and tc.launches:
        s = tc.ms / 1e3
        out[TC_KIND + " (tensor-core stages of k_gemm)"] = {
            "launches": tc.launches, "jobs": tc.jobs, "ms": round(tc.ms, 4),
            "tensor_tflops": round(tc.flops / s / 1e12, 3) if s > 0 else None,
            "bf16_peak_tflops": bf16_peak,
            "frac_tensor": round(tc.flops / s / 1e12 / bf16_peak, 4) if (s > 0 and bf16_peak) else None,
            "what": "BF16 slice products issued (mma.sync m16n8k16, padding included) per second, against the "
                    "measured BF16 burst peak"}
    for nm, p_ in kinds:
        if p_.launches == 0:
            continue
        s = p_.ms / 1e3
        row = {"launches": p_.launches, "jobs": p_.jobs, "ms": round(p_.ms, 4),
               "gflop": round(p_.flops / 1e9, 4), "gb": round(p_.bytes / 1e9, 4)}
        if p_.flops > 0 and s > 0:
            row["tflops_executed"] = round(p_.flops / s / 1e12, 4)
            if peak:
                row["frac_executed"] = round(p_.flops / s / 1e12 / peak, 4)
            keys = ORACLE_KIND.get(nm, ())
            if mw and keys:
                mf = sum(mw["flops"][k] for k in keys)
                row["tflops_method"] = round(mf / s / 1e12, 4)
                if peak:
                    row["frac_method"] = round(mf / s / 1e12 / peak, 4)
        elif p_.bytes > 0 and s > 0:
            row["gbs"] = round(p_.bytes / s / 1e9, 1)
            if hbm_peak:
                row["frac_hbm"] = round(p_.bytes / s / 1e9 / hbm_peak, 4)
        out[nm] = row
    return out


def method_work(grid, eps):
    """Oracle-counted work of one product of the workload (None if not recorded)."""
    wc = load_json("tests", "golden", "work_counts.json")
    if not wc:
        return None
    return wc["cases"].get(f"grid2d_n{grid * grid}_eps{eps:g}")


def fp64_peak():
    """FP64 ALU peak of the part: 152 SMs x 2 FP64 FMA/clk/SM x 2 flops x max SM clock."""
    mhz = 2070.0
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz = float(peaks.get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 2 * 2 * mhz * 1e6 / 1e12  # TFLOP/s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_subprocess(grid, eps, nprod):
    """Time `nprod` oracle products (build excluded) in a spawned single-thread process."""
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from oracle import h2oracle as O\n"
        "from paper_2403_01566_gb300 import inputs as I\n"
        f"w = I.grid_2d({grid}, {eps!r})\n"
        "X = O.build_h2(w.points, w.kernel_a.kind, w.kernel_a.kparam(), w.eta, w.leaf_size, w.order)\n"
        "Y = O.build_h2(w.points, w.kernel_b.kind, w.kernel_b.kparam(), w.eta, w.leaf_size, w.order, tree=X.rows)\n"
        "ts = []\n"
        f"for _ in range({nprod}):\n"
        "    t0 = time.perf_counter(); O.multiply(X, Y, w.eps); ts.append(time.perf_counter() - t0)\n"
        "print(json.dumps(ts))\n")
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself for one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, max_total_ms):
    """Products per second of all ranks together: every rank runs `steps`
    independent products (replicas), the job takes the slowest rank's time."""
    return world * steps / (max_total_ms / 1e3)


REFERENCE_BUDGET_S = 180.0  # the reference arm stops taking steps after this much oracle time


def run_reference(args, rank, world):
    if rank != 0:
        return
    # warm-up: W products on a 16 x 16 grid (imports, BLAS start-up); timed
    # steps: one full product of the workload each, at most K, stopping once
    # the oracle time passes REFERENCE_BUDGET_S
    oracle_subprocess(16, EPS, max(1, args.warmup))
    ts = []
    while len(ts) < max(1, args.steps) and sum(ts) < REFERENCE_BUDGET_S:
        ts += oracle_subprocess(GRID, EPS, 1)
    nprod = len(ts)
    value = nprod / sum(ts)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": nprod,
        "warmup": max(1, args.warmup), "ms_per_step": 1e3 * sum(ts) / nprod, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": dict(workload_config(), parallelism=f"replicas x{world}"), "form": "CPU oracle, FP64",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{nprod} full product(s) of the workload on one host thread "
                                   f"(numpy FP64 oracle, input build excluded; at most {args.steps} steps, "
                                   f"stopping after {REFERENCE_BUDGET_S:.0f} s); warm-up on a 16x16 grid"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_size_for(steps, cap=24):
    """Largest divisor of `steps` not above `cap`: products per batch replay
    (every product of a batch holds its own workspace)."""
    for b in range(min(cap, steps), 0, -1):
        if steps % b == 0:
            return b
    return 1


def percentile(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def serving_stream(h2, I, np, torch, nreq=48, rate=200.0, nmax=16384, seed=20240308):
    """Requests shaped like the serving workload, scaled to one GPU: Poisson
    arrivals at `rate` per second of products over a resident pool of 3D
    uniform point sets (n log-uniform in [4096, nmax], k = 64, both kernels
    1/|x-y| and exp(-|x-y|)), eps per request drawn from {1e-4, 1e-6, 1e-8};
    continuous batching on 8 streams with admission by device memory; latency
    from arrival to completion."""
    rng = np.random.default_rng(seed)
    pool = []
    for j in range(4):
        n = int(round(math.exp(rng.uniform(math.log(4096), math.log(nmax)))))
        pts = I.uniform_points(n, 3, 5000 + j)
        pool.append((n, h2.build(pts, I.INV, 2.0, 64, 4), h2.build(pts, I.EXP, 2.0, 64, 4)))
    reqs = []
    t = 0.0
    for _ in range(nreq):
        t += rng.exponential(1.0 / rate)
        n, a, b = pool[int(rng.integers(len(pool)))]
        ka, kb = int(rng.integers(2)), int(rng.integers(2))
        eps = float(rng.choice([1e-4, 1e-6, 1e-8]))
        reqs.append((t, (a, b)[ka], (a, b)[kb], eps, n))
    srv = h2.Server(slots=8)
    for n, a, b in pool:  # plans and graphs of every structure before the stream
        srv.wait(srv.submit(a, b, 1e-6, precision=4))[0].free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for (ta, A, B, eps, n) in reqs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((srv.submit(A, B, eps, precision=4), ta))
    lat = []
    t_last = 0.0
    refused = {}
    for (tk, ta), r in zip(tickets, reqs):
        try:
            C, _, tot = srv.wait(tk)
            C.free()
            lat.append(tot)
        except h2.H2Error as ex:  # e.g. ranks above the cap of 64 at eps = 1e-8
            key = f"{h2._lib().h2_strerror(ex.code).decode()} (eps {r[3]:g})"
            refused[key] = refused.get(key, 0) + 1
        t_last = max(t_last, time.perf_counter() - t0)
    srv.close()
    return {"requests": nreq, "completed": len(lat), "refused": refused, "rate_per_s": rate,
            "n_range": [min(r[4] for r in reqs), max(r[4] for r in reqs)],
            "value": len(lat) / t_last, "unit": UNIT, "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99),
            "form": "served (continuous batching, 8 streams, memory admission), tensor-core contractions",
            "workload": f"3D uniform points, n log-uniform in [4096, {nmax}] (4 resident point sets), k=64, leaf 64, "
                        "eta 2, A/B in {1/|x-y|, exp(-|x-y|)}, eps in {1e-4, 1e-6, 1e-8}, Poisson arrivals",
            "timing": "host wall clock; latency = arrival to completion, throughput = requests / last completion"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the served, stream and end-to-end measurements")
    ap.add_argument("--grid", type=int, default=GRID,
                    help="grid side (default 128 = the benchmark workload; smaller for profiler captures)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")

    from paper_2403_01566_gb300 import h2
    from paper_2403_01566_gb300 import inputs as I

    grid = args.grid
    w = I.grid_2d(grid, EPS)
    A = h2.build(w.points, w.kernel_a, w.eta, w.leaf_size, w.order)
    B = h2.build(w.points, w.kernel_b, w.eta, w.leaf_size, w.order)
    # a dedicated stream: the legacy default stream has handle 0, which the
    # library would read as "use the library stream"
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    assert sptr != 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    warm = max(args.warmup, 3)

    # ---- chosen form: the benchmark products as batches of the tensor-core
    # precision form (7-slice BF16 on the 64 x 64 stages, compensated FP32 on
    # the others; FP64 QR/SVD/norms), each batch one CUDA graph replay
    bs = batch_size_for(args.steps)
    batch = h2.Batch([(A, B, EPS)] * bs, precision=4)
    for _ in range(warm):
        batch.run(sync=False, stream=sptr)
    torch.cuda.synchronize()
    nrep = args.steps // bs
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nrep)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nrep)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t_wall0 = time.perf_counter()
    for i in range(nrep):
        flush.fill_(float(i))
        starts[i].record(stream)
        batch.run(sync=False, stream=sptr)
        ends[i].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    if dist is not None:
        dist.barrier()
    batch.run(sync=True, stream=sptr)  # device error state of the products
    rep_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = max_over_ranks(sum(rep_ms), dist, "cuda")
    value = whole_job_rate(world, args.steps, total_ms)
    binfo = batch.info()
    launches = binfo["kernel_launches"] * nrep
    st_c = batch.result(0).info()
    y_chk = batch.result(0).matvec(I.random_vector(w.n, 3))
    batch.free()

    # ---- plain FP64 form: one product per step through h2_mul
    for _ in range(warm):
        h2.mul(A, B, EPS, stream=sptr)
    torch.cuda.synchronize()
    p_st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    p_en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    outs = []
    for i in range(args.steps):
        flush.fill_(float(i))
        p_st[i].record(stream)
        outs.append(h2.mul(A, B, EPS, sync=False, stream=sptr))
        p_en[i].record(stream)
    torch.cuda.synchronize()
    for C in outs:
        C.check()
    y_ref = outs[0].matvec(I.random_vector(w.n, 3))
    st0 = outs[0].info()
    for C in outs:
        C.free()
    outs.clear()
    plain_ms = [s_.elapsed_time(e_) for s_, e_ in zip(p_st, p_en)]
    plain_total = max_over_ranks(sum(plain_ms), dist, "cuda")
    plain_value = whole_job_rate(world, args.steps, plain_total)
    agree = float(np.linalg.norm(y_chk - y_ref) / np.linalg.norm(y_ref))

    served = stream_run = None
    e2e_value = None
    x = np.ascontiguousarray(I.random_vector(w.n, 1))
    pts_pinned = torch.from_numpy(np.ascontiguousarray(w.points)).pin_memory()
    if not args.no_extras:
        # served form: `steps` products submitted at once (continuous batching)
        slots = 4
        srv = h2.Server(slots=slots)
        for t in [srv.submit(A, B, EPS, precision=4) for _ in range(slots)]:
            srv.wait(t)[0].free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit(A, B, EPS, precision=4) for _ in range(args.steps)]
        lat = []
        for t in tickets:
            Cs, _, tot = srv.wait(t)
            lat.append(tot)
            Cs.free()
        el = time.perf_counter() - t0
        srv.close()
        served = {"form": f"served: continuous batching on {slots} streams, tensor-core contractions",
                  "value": args.steps / el, "unit": UNIT, "p50_ms": percentile(lat, 0.5),
                  "p99_ms": percentile(lat, 0.99),
                  "timing": f"host wall clock over {args.steps} products submitted at once (latency = submit to done)"}
        # end to end through the public API: points from pinned host memory ->
        # h2_build (A, B) -> h2_mul (tensor-core form) -> C x read back, per step
        e2e_steps = max(2, min(5, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p = pts_pinned.numpy()
            Ae = h2.build(p, w.kernel_a, w.eta, w.leaf_size, w.order)
            Be = h2.build(p, w.kernel_b, w.eta, w.leaf_size, w.order)
            Ce = h2.mul(Ae, Be, EPS, stream=sptr, precision=4)
            y = Ce.matvec(x)
            Ce.free()
            Ae.free()
            Be.free()
        torch.cuda.synchronize()
        e2e_value = e2e_steps / (time.perf_counter() - t0)
        assert np.isfinite(y).all()
        # last: the stream's structures take the places of the plan cache
        if rank == 0:
            stream_run = serving_stream(h2, I, np, torch)

    # roofline of the dominant kernel of the chosen form: one profiled product
    # (stages one by one, CUDA events around each)
    prof = (h2.KernelProf * h2.PROFILE_KINDS)()
    Cp = h2.mul_profile(A, B, EPS, prof, stream=sptr, precision=4)
    Cp.free()
    kinds = [(KIND_NAMES[i], prof[i]) for i in range(len(KIND_NAMES))]
    prof_total = sum(p_.ms for _, p_ in kinds)
    dom_name, dom = max(kinds, key=lambda kv: kv[1].ms)
    peak = fp64_peak()
    executed = dom.flops / (dom.ms / 1e3) / 1e12 if dom.ms > 0 else 0.0
    mw = method_work(grid, EPS)
    method_flops = sum(mw["flops"][k] for k in ORACLE_KIND.get(dom_name, ())) if mw else None
    achieved = method_flops / (dom.ms / 1e3) / 1e12 if (method_flops and dom.ms > 0) else executed
    hbm_peak = (load_json("MEASURED_PEAKS.json") or {}).get("hbm_gbs")
    kc = dict(kinds).get("k_copy")
    # DRAM bytes per launch from the committed ncu capture, valid only while the
    # kernel source is the one the counters were taken on
    traffic = None
    try:
        import hashlib
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        src = os.path.join(ROOT, "paper_2403_01566_gb300", "csrc", "h2_kernels.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest() == tr.get("kernels_source_sha256"):
            traffic = tr["per_launch_bytes"].get(dom_name)
    except (OSError, ValueError, KeyError):
        pass

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ts = oracle_subprocess(grid, EPS, 1)
        cpu = {"value": 1.0 / ts[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one full product of the workload on one host thread (numpy FP64 oracle, "
                         "input build excluded)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(grid), parallelism=f"replicas x{world}"),
            "form": "chosen: batched products, tensor-core contractions",
            "chosen_form": {"form": f"batched: {bs} products per CUDA-graph replay (merged launches, persistent GEMM "
                                    "chains), 7-slice BF16 tensor-core GEMMs on 64x64 stages and compensated FP32 "
                                    "on the others, FP64 QR/SVD/rank decisions/norms",
                            "products_per_batch": bs, "replays": nrep,
                            "p50_ms_per_batch": percentile(rep_ms, 0.5), "p99_ms_per_batch": percentile(rep_ms, 0.99),
                            "vs_plain_fp64": value / plain_value, "Cx_rel_diff_vs_plain_fp64": agree,
                            "launches_per_batch": binfo},
            "plain_fp64": {"value": plain_value, "unit": UNIT, "ms_per_step": plain_total / args.steps,
                           "p50_ms": percentile(plain_ms, 0.5), "p99_ms": percentile(plain_ms, 0.99),
                           "form": "h2_mul one product per step, FP64 throughout"},
            "p50_ms": percentile(rep_ms, 0.5) / bs, "p99_ms": percentile(rep_ms, 0.99) / bs, "wall_s": t_wall,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * w.points.nbytes + x.nbytes), "d2h_bytes_per_step": int(x.nbytes),
                    "what": "h2_build(A), h2_build(B) from pinned host points, h2_mul (tensor-core form), "
                            "C x read back"} if e2e_value else None,
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": traffic,
                         "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                         "launches": dom.launches,
                         "flop_per_launch": (method_flops if method_flops else dom.flops) / dom.launches
                         if dom.launches else None,
                         "work_source": "oracle counters, tests/golden/work_counts.json" if method_flops
                         else "kernel counts (no oracle count recorded for this workload)",
                         "peak_source": "FP64 ALU peak derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
                         "profiled_form": "tensor-core form (precision 4), stages one by one",
                         "share": dom.ms / prof_total if prof_total else None,
                         "executed": {"achieved": executed, "frac": executed / peak if peak else None,
                                      "gpu_flops_per_product": dom.flops,
                                      "method_flops_per_product": method_flops,
                                      "gpu_over_method": dom.flops / method_flops if method_flops else None},
                         "product": {"method_gflop": sum(mw["flops"].values()) / 1e9 if mw else None,
                                     "gpu_gflop": sum(p_.flops for _, p_ in kinds) / 1e9,
                                     "method_tflops_over_product_time":
                                         sum(mw["flops"].values()) / (prof_total / 1e3) / 1e12 if mw else None},
                         "hbm_copy": {"kernel": "k_copy", "gb": kc.bytes / 1e9, "ms": kc.ms,
                                      "achieved_gbs": kc.bytes / (kc.ms / 1e3) / 1e9 if kc.ms > 0 else None,
                                      "peak_gbs": hbm_peak,
                                      "frac": (kc.bytes / (kc.ms / 1e3) / 1e9) / hbm_peak
                                      if (kc.ms > 0 and hbm_peak) else None} if kc else None},
            "kernels": kernel_table(kinds, mw, peak, hbm_peak, tc=prof[len(KIND_NAMES)],
                                    bf16_peak=(load_json("MEASURED_PEAKS.json") or {}).get("bf16_tflops")),
            "product": {"nadm": st0.nadm, "ninadm": st0.ninadm, "agglomerated": st0.nagglomerated,
                        "rank_max": max(st0.row_rank_max, st0.col_rank_max), "workspace_gb": st0.workspace_bytes / 1e9,
                        "rank_max_chosen": max(st_c.row_rank_max, st_c.col_rank_max)},
            "clocks": clocks,
            "served_form": served,
            "serving_stream": stream_run,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
