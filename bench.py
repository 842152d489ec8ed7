"""Benchmark of the SIPG hp-multigrid hot path on GB300 (one JSON line on stdout).

Workload: 3D unit cube, 32^3 hexahedra, GLL degree p = 3 (64 DoF per cell,
2,097,152 DoF), kappa = 1, f = 3 pi^2 prod_i sin(pi x_i); FP64 PCG with the
hp V(2,2) cycle as preconditioner, solved from x = 0 to ||b - A x|| <= 1e-10 ||b||.
One bench step is one complete solve: every stage of the path (warm-up
projections, single-touch smoothing steps, residual + p-restriction, Q1
levels, coarsest solve, p-prolongation, FP64 apply and CG vector work) runs
in it. The metric is GDoF/s per smoothing step: DoF x (fine-level
smoothing steps executed in the step) / step time, so everything else the
solve does counts against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the plain CPU oracle on the host cores (the same
metric and unit, on a bounded sample of the workload). Under torchrun (N > 1)
every rank solves its own replica of the workload (weak scaling, no
collective on the data path); rank 0 prints.
"""
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

N_CELLS = (32, 32, 32)
DEGREE = 3
RTOL = 1e-10
WORKLOAD = "sipg_3d_32^3_p3_kappa1_fp64_pcg_vcycle22"
SAMPLE_CELLS = (16, 16, 16)      # bounded CPU sample: same p, 1/8 of the DoFs
FP64_NOMINAL_TFLOPS = 1.25       # nominal GB300 dense FP64, context beside the measured peak
# DRAM bytes (read + write) of one launch of the FP64 smoothing kernel on this
# workload from one ncu capture, valid only for the kernel sources it was taken
# on (SHA-256 of the files below); once they change, `traffic` reads null
SMOOTH_TRAFFIC = {"kernel": "k_smooth_cells<double,4>", "bytes": 116_628_736 + 10_494_464,
                  "sources_sha256": "7b1b09b1125962089f573f3432c4a423ffed4cdec4c1dcacfab6e84818cc62ad",
                  "files": ("smooth_cells.cuh", "dg_kernels.cuh", "dg_fp64.cu")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    # library default tiles instead of timing candidates at set-up: for runs under
    # a profiler, whose per-launch overhead distorts the tuner's timings (for this
    # workload the defaults are the tiles the tuner picks)
    ap.add_argument("--no-autotune", action="store_true")
    # skip the 64^3 p=4 mixed-precision section (the FP32 smoothing step)
    ap.add_argument("--no-mixed", action="store_true")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max_sum(values, world, device):
    """Max of values[0] and sum of values[1] over ranks (identity for one rank)."""
    if world == 1:
        return values[0], values[1]
    import torch
    import torch.distributed as dist
    t = torch.tensor([values[0]], dtype=torch.float64, device=device)
    s = torch.tensor([values[1]], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


def sources_sha256(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2510_00998_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def smooth_traffic(kernel):
    """(bytes, note) of the recorded ncu capture if it was taken on the current
    sources of `kernel`, else (None, why)."""
    t = SMOOTH_TRAFFIC
    if t["bytes"] is None or kernel != t["kernel"]:
        return None, "no ncu capture recorded for this kernel"
    sha = sources_sha256(t["files"])
    if sha != t["sources_sha256"]:
        return None, "kernel sources changed since the recorded ncu capture"
    return t["bytes"], ("dram__bytes_read.sum + dram__bytes_write.sum of one launch, one ncu capture on these "
                        f"kernel sources (sha256 {sha[:12]})")


# ---------------------------------------------------------------- flop model
def smooth_flops(n, q):
    """Floating-point operations of one launch of the FP64 fused smoothing kernel
    as implemented (an FMA counts 2, a multiplication 1): facet mass on the two
    neighbour fields of every interior face side (each 1D mass in its rank-one
    form diag(w) - u u^T: per pencil of q values a dot product, q multiplications
    and q FMAs, 5q operations); lifting (per face node q FMAs for the value
    field, one for the derivative field); S^T and S along every axis; the
    inverse eigenvalue sums (with the damping folded in) as one multiplication
    per node; the update (1 - omega) u + y as one FMA per node; the derivative
    traces of every face."""
    d = len(n)
    ncell = 1
    for v in n:
        ncell *= v
    nf = q ** (d - 1)
    nl = q ** d
    sides = 0                       # interior face sides (each interior facet has two)
    for a in range(d):
        other = ncell // n[a]
        sides += 2 * (n[a] - 1) * other
    facet_mass = sides * 2 * (d - 1) * 5 * nf
    lift = sides * nf * (q * 2 + 2)
    per_cell = 2 * d * nl * q * 2 + nl * 1 + nl * 2 + d * nf * 2 * q * 2
    return facet_mass + lift + ncell * per_cell


def smooth_bytes_per_cell(d, q, s=8):
    """Algorithmic HBM bytes of one cell of the smoothing step: read u, b, write u;
    read the 2d neighbour traces (value + derivative) and write the cell's own;
    read the per-cell fast-diagonalisation factors d (q^2 + q) and kappa of the
    cell and its neighbours."""
    nl = q ** d
    nf = q ** (d - 1)
    return s * (3 * nl + 2 * (2 * d * 2 * nf) + d * (q * q + q) + (2 * d + 1))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle
ORACLE_WORKER = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import sipg
m = sipg.Mesh({cells!r}, {degree})
bj = sipg.BlockJacobi(m)
rng = np.random.default_rng(0)
u, b = rng.normal(size=m.ndof), rng.normal(size=m.ndof)
u, _ = bj.step_alg4(u, b, 0.8, 1)
open({ready!r} + str({wid}), "w").close()
while not os.path.exists({go!r}):
    time.sleep(0.01)
secs = []
for _ in range({chunks}):
    t = time.perf_counter()
    u, _ = bj.step_alg4(u, b, 0.8, {steps})
    secs.append(time.perf_counter() - t)
print(json.dumps({{"ndof": m.ndof, "seconds": secs}}))
"""


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_run(workers, chunks, steps_per_chunk):
    """The oracle's Alg. 4 smoothing steps on the bounded sample in `workers`
    single-threaded processes at once (one per core, each its own replica of
    the sample): every process does its block-inverse set-up and one warm-up
    step, then all start together and time `chunks` chunks of
    `steps_per_chunk` steps. Returns (ndof per replica, [[seconds per chunk]
    per process])."""
    tmp = tempfile.mkdtemp(prefix="oracle_")
    ready, go = os.path.join(tmp, "ready"), os.path.join(tmp, "go")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    procs = []
    for w in range(workers):
        code = ORACLE_WORKER.format(root=ROOT, cells=SAMPLE_CELLS, degree=DEGREE, ready=ready, wid=w, go=go,
                                    chunks=chunks, steps=steps_per_chunk)
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, env=env))
    try:
        while sum(os.path.exists(ready + str(w)) for w in range(workers)) < workers:
            if any(p.poll() not in (None, 0) for p in procs):
                raise RuntimeError("oracle worker failed: " + "".join(p.stderr.read() for p in procs if p.poll()))
            time.sleep(0.02)
        open(go, "w").close()
        res = []
        for p in procs:
            out, err = p.communicate()
            if p.returncode != 0:
                raise RuntimeError("oracle worker failed: " + err)
            res.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
        for f in os.listdir(tmp):
            os.unlink(os.path.join(tmp, f))
        os.rmdir(tmp)
    return res[0]["ndof"], [r["seconds"] for r in res]


def oracle_rate(workers, chunks=6, steps=8):
    """Aggregate GDoF/s of `workers` concurrent oracle processes: per process the
    median of its chunks after the first (a warm-up), summed over processes."""
    ndof, secs = oracle_run(workers, chunks, steps)
    rates = [ndof * steps / statistics.median(s[1:]) / 1e9 for s in secs]
    return sum(rates), secs


def sample_text(steps, workers):
    who = "one thread" if workers == 1 else f"{workers} single-threaded processes at once, one replica each"
    return (f"oracle Alg. 4 smoothing steps on {SAMPLE_CELLS[0]}x{SAMPLE_CELLS[1]}x{SAMPLE_CELLS[2]} cells, "
            f"p={DEGREE} (1/8 of the workload's DoF, same degree), chunks of {steps} steps after the "
            f"block-inverse set-up, median of 5 chunks after one warm-up chunk, {who}, FP64")


def cpu_baseline():
    """The oracle on all host cores (the reported baseline) and on one core."""
    ncores = os.cpu_count() or 1
    v_all, _ = oracle_rate(ncores)
    v_one, _ = oracle_rate(1)
    return {"value": v_all, "unit": "GDoF/s", "cores": ncores, "kind": "oracle", "sample": sample_text(8, ncores),
            "nproc": ncores, "cpu_model": cpu_model(),
            "one_core": {"value": v_one, "unit": "GDoF/s", "cores": 1, "sample": sample_text(8, 1)}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    steps_per = 4
    ndof, secs = oracle_run(ncores, args.warmup + args.steps, steps_per)
    timed = [s[args.warmup:] for s in secs]
    # per bench step: all processes' DoF x steps over the slowest process's chunk time
    per_step = [max(s[k] for s in timed) for k in range(args.steps)]
    value = ncores * ndof * steps_per * args.steps / sum(per_step) / 1e9
    text = (f"oracle Alg. 4 smoothing steps on {SAMPLE_CELLS[0]}x{SAMPLE_CELLS[1]}x{SAMPLE_CELLS[2]} cells, "
            f"p={DEGREE} (1/8 of the workload's DoF, same degree), {steps_per} steps per bench step in each of "
            f"{ncores} single-threaded processes at once (one replica each), after the block-inverse set-up, FP64")
    line = {
        "impl": "reference", "metric": "GDoF/s per smoothing step", "value": value, "unit": "GDoF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(per_step) / len(per_step), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": text},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": ncores, "kind": "oracle", "sample": text,
                         "nproc": ncores, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving
SERVE_RATES = (0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0)   # x the FP64 one-at-a-time capacity
SERVE_MAX_REQUESTS = 128
SERVE_WINDOW_S = 16.0    # arrival window per rate at most: fewer requests at the low rates
SERVE_FP64_SAMPLE = 8    # served results checked against an FP64 solve of the same request


def measured_hbm_gbs():
    """Copy bandwidth measured on this machine (MEASURED_PEAKS.json beside bench.py),
    else the profiling recipe's fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def timed_ms(fn, flush, stream, reps):
    """Mean device time of fn() over reps calls, L2 flushed before each (outside
    the events)."""
    import torch
    total = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / reps


def mixed_section(flush, stream):
    """64^3 cells, p = 4, lognormal kappa: the FP32 V-cycle inside reliable-update
    FP32 CG with FP64 residuals; solve time and the FP32 smoothing step against the
    HBM roofline (algorithmic bytes per launch / mean launch time)."""
    import torch
    from paper_2510_00998_gb300 import dgmg, workloads
    ctx, b = workloads.make("3d64_p4_mixed")
    x = torch.zeros_like(b)

    def solve():
        x.zero_()
        return ctx.solve(b, x)[0]

    st = solve()
    ms = timed_ms(solve, flush, stream, 2)
    ctx.profile(True)
    solve()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    sm_ms = prof["smooth"][0] / max(prof["smooth"][1], 1)
    d, q = 3, 5
    nbytes = smooth_bytes_per_cell(d, q, 4) * ctx.info.ncell
    peak, how = measured_hbm_gbs()
    achieved = nbytes / (sm_ms * 1e-3) / 1e9
    kern = "k_smooth_cells<float,5>" if ctx.info.tiles[4] == 0 else "k_smooth<3,5,float>"
    return {"workload": "sipg_3d_64^3_p4_lognormal_kappa_mixed", "ndof": ctx.ndof, "solve_ms": ms,
            "iterations": st.iterations, "rel_residual": st.rel_residual, "fp64_applies": st.fp64_applies,
            "smoothing_step": {"kernel": kern, "avg_launch_ms": sm_ms, "gdofs": ctx.ndof / (sm_ms * 1e-3) / 1e9,
                               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                                            "unit": "GB/s", "frac": achieved / peak, "peak_source": how,
                                            "bytes_per_launch": nbytes}}}


def serving_run():
    """Solves/s and p50/p99 latency (arrival to completion, rel. residual 1e-10)
    of the mixed-precision solve server against plain FP64 one-at-a-time solving,
    for Poisson arrivals of requests with n in [8,48]^3 cells, p in 2..5 and
    kappa in {1, lognormal, two-phase}, at rising multiples of the FP64
    capacity until the served rate stops tracking the arrival rate (the served
    capacity); the error of a sample of served results against FP64 solves of
    the same requests."""
    import numpy as np
    import torch
    from paper_2510_00998_gb300 import dgmg
    from paper_2510_00998_gb300 import workloads as wl
    reqs = wl.request_stream("serve", SERVE_MAX_REQUESTS, 5)
    wl.build_rhs(reqs)
    service = wl.one_at_a_time(reqs, precision=0)
    capacity = len(service) / sum(service)
    gaps = np.random.default_rng(1005).exponential(size=len(reqs))
    rates, xs_last, sub_last = [], None, None
    for m in SERVE_RATES:
        lam = m * capacity
        n = int(min(SERVE_MAX_REQUESTS, max(32, lam * SERVE_WINDOW_S)))
        sub = reqs[:n]
        arrivals = list(np.cumsum(gaps[:n] / lam))
        fifo = wl.fifo_latencies(arrivals, service[:n])
        lat, makespan, stats, info, xs = wl.serve_trace(sub, arrivals, 96 << 30, 16, return_x=True)
        served = n / makespan
        rates.append({"rate_x_fp64_capacity": m, "rate_per_s": lam, "requests": n,
                      "served_mixed": {"solves_per_s": served, "p50_s": wl.pct(lat, 50), "p99_s": wl.pct(lat, 99),
                                       "max_rel_residual": max(st.rel_residual for st in stats)},
                      "fp64_one_at_a_time": {"solves_per_s": n / max(a + l for a, l in zip(arrivals, fifo)),
                                             "p50_s": wl.pct(fifo, 50), "p99_s": wl.pct(fifo, 99)}})
        xs_last, sub_last = xs, sub
        if served < 0.8 * lam:
            break                       # saturated: the served rate no longer follows the arrivals
    # accuracy: served (mixed-precision) results against FP64 solves of the same requests
    errs = []
    for k in range(min(SERVE_FP64_SAMPLE, len(sub_last))):
        r = sub_last[k]
        ctx = dgmg.Context(r["n"], r["p"], r["kappa"], precision=0, rtol=1e-12)
        x64 = torch.zeros_like(r["b"])
        ctx.solve(r["b"], x64)
        ctx.close()
        errs.append(float(torch.linalg.norm(xs_last[k] - x64) / torch.linalg.norm(x64)))
    served_all = [e["served_mixed"]["solves_per_s"] for e in rates]
    return {"fp64_capacity_solves_per_s": capacity,
            "served_capacity_solves_per_s": max(served_all),
            "saturated": rates[-1]["served_mixed"]["solves_per_s"] < 0.8 * rates[-1]["rate_per_s"],
            "rates": rates,
            "max_rel_err_vs_fp64": max(errs), "fp64_check_sample": len(errs),
            "workload": "Poisson arrivals (seeds 5, 1005), n in [8,48]^3, p in 2..5, kappa in {1, lognormal, "
                        "two-phase 1/100}, 8 random Fourier modes; up to 128 requests per rate, "
                        "16 slots, 96 GB budget; FP64 check: rtol 1e-12 FP64 PCG"}


BATCH_COUNT = 256


def batch_run():
    """256 independent solves (n in [8,24]^3, p in {2,3,4}, lognormal kappa,
    8 Fourier modes, default_rng(4)) as one batch (one persistent launch per
    stage and degree group), FP64 and mixed precision, against FP64 solves one
    at a time; solves/s with and without set-up."""
    from paper_2510_00998_gb300 import workloads as wl
    reqs = wl.request_stream("batch", BATCH_COUNT, 4)
    wl.build_rhs(reqs)
    solve_only = []
    alone = wl.one_at_a_time(reqs, precision=0, solve_times=solve_only)
    out = {"workload": f"{BATCH_COUNT} 3D solves, n in [8,24], p in 2..4, lognormal kappa, Fourier RHS "
                       "(default_rng(4)), every problem to rel. residual 1e-10",
           "fp64_one_at_a_time": {"solves_per_s": BATCH_COUNT / sum(alone),
                                  "solve_only_solves_per_s": BATCH_COUNT / sum(solve_only)}}
    for name, prec in (("batched_fp64", 0), ("batched_mixed", 1)):
        setup, times, stats, info = wl.batched(reqs, solves=3, precision=prec)
        out[name] = {"setup_s": setup, "solve_s": min(times),
                     "solves_per_s": BATCH_COUNT / (setup + min(times)),
                     "solve_only_solves_per_s": BATCH_COUNT / min(times),
                     "iterations_max": max(s.iterations for s in stats),
                     "max_rel_residual": max(s.rel_residual for s in stats),
                     "kernels_per_iteration": info.kernels_per_iteration, "ndof": info.ndof}
    return out


# ---------------------------------------------------------------- GPU arm
def run_gb300(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg

    ctx = dgmg.Context(N_CELLS, DEGREE, rtol=RTOL, autotune=0 if args.no_autotune else 1)
    ndof = ctx.ndof
    d, q = 3, DEGREE + 1
    # right-hand side b_i = (f, phi_i) from f at the library's quadrature points
    mq = DEGREE + 2
    xq = torch.empty(ctx.info.ncell * mq ** 3 * 3, dtype=torch.float64, device=dev)
    ctx.quad_points(xq)
    X = xq.view(-1, 3)
    fq = (3 * np.pi ** 2) * torch.sin(np.pi * X[:, 0]) * torch.sin(np.pi * X[:, 1]) * torch.sin(np.pi * X[:, 2])
    b = torch.empty(ndof, dtype=torch.float64, device=dev)
    ctx.load_vector(fq.contiguous(), b)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def one_solve():
        x.zero_()
        st, _ = ctx.solve(b, x)
        return st

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    launches0 = dgmg.kernel_launches()
    total_ms, iters, relres = 0.0, [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st = one_solve()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters.append(st.iterations)
        relres.append(st.rel_residual)
    launches = dgmg.kernel_launches() - launches0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    # per-stage device times from separate, profiled solves (the profiler brackets
    # every stage launch with events and runs without CUDA graphs, so it stays
    # out of the timed steps above); same iterations, so the same smoothing steps
    prof_solves = min(args.steps, 3)
    ctx.profile(True)
    for _ in range(prof_solves):
        flush.fill_(1.0)
        one_solve()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    smooth_steps_per_solve = prof["smooth"][1] / prof_solves
    smooth_steps_total = smooth_steps_per_solve * args.steps
    units_local = float(ndof) * smooth_steps_total
    t_max, units = reduce_max_sum((total_ms, units_local), world, dev)
    value = units / (t_max * 1e-3) / 1e9
    # roofline of the dominant kernel (the fused smoothing step): FP64-pipe
    # bound, against the FP64 FMA-loop peak measured here, in this run
    sm_ms, sm_n = prof["smooth"]
    avg_ms = sm_ms / max(sm_n, 1)
    flops = smooth_flops(N_CELLS, q)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    peak_clocks = ClockSampler(local)
    fp64_peak = dgmg.fma_peak(0)
    fp32_peak = dgmg.fma_peak(1)
    fp32x2_peak = dgmg.fma_peak(2)
    peak_clk = peak_clocks.stop()
    survey_flops = 10 * d * q * ndof          # sum-factorised minimum, 10 d q flop per DoF
    shares = {k: round(v[0] / max(sum(w[0] for w in prof.values()), 1e-30), 4) for k, v in prof.items()}

    # end to end through the host-buffer entry point
    bh = b.cpu().pin_memory()
    xh = torch.zeros(ndof, dtype=torch.float64).pin_memory()
    e2e_ms = 0.0
    e2e_units = 0.0
    for k in range(args.warmup + args.steps):
        xh.zero_()
        t = time.perf_counter()
        st = ctx.solve_host(bh, xh)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            e2e_ms += 1e3 * dt
            e2e_units += float(ndof) * st.iterations * (ctx.opts.nu_pre + ctx.opts.nu_post)
    e2e_t, e2e_u = reduce_max_sum((e2e_ms, e2e_units), world, dev)

    # GDoF/s of one FP64 apply (warm-up projection + cell equation) and the time
    # of one FP64 V-cycle, on the same context
    y = torch.empty_like(b)
    apply_ms = timed_ms(lambda: ctx.apply(b, y), flush, stream, 10)
    vcycle_ms = timed_ms(lambda: ctx.vcycle(b, y), flush, stream, 10)

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_run()
    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_run()
    mixed = None
    if rank == 0 and not args.no_mixed:
        mixed = mixed_section(flush, stream)

    # the smoothing kernel the tuned context runs (tile 0 = one thread per cell)
    cells_kernel = ctx.info.tiles[1] == 0 and d == 3 and q <= 4
    smooth_kernel = f"k_smooth_cells<double,{q}>" if cells_kernel else f"k_smooth<{d},{q},double>"
    traffic, traffic_note = smooth_traffic(smooth_kernel)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline()
        line = {
            "metric": "GDoF/s per smoothing step", "value": value, "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": list(N_CELLS), "p": DEGREE, "ndof": ndof,
                       "kappa": "1", "rhs": "3 pi^2 prod sin(pi x_i)", "rtol": RTOL, "cycle": "V(2,2)",
                       "outer": "FP64 PCG", "step": "one full solve from x=0",
                       "l2": "flushed (256 MB write) before every timed step, outside the step's events",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak,
                         "traffic": traffic, "traffic_note": traffic_note,
                         "kernel": smooth_kernel, "avg_launch_ms": avg_ms,
                         "flops_per_launch": flops,
                         "frac_at_10dq_flop_per_dof": survey_flops / (avg_ms * 1e-3) / 1e12 / fp64_peak,
                         "hbm_bytes_per_launch": smooth_bytes_per_cell(d, q) * ctx.info.ncell,
                         "peak_note": ("FP64 FMA-loop peak measured in this run (dgmg_fma_peak), of measured; "
                                       f"nominal {FP64_NOMINAL_TFLOPS}"),
                         "measured_peaks_tflops": {"fp64_fma": fp64_peak, "fp32_fma": fp32_peak,
                                                   "fp32x2_fma": fp32x2_peak, "clocks": peak_clk}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_u / (e2e_t * 1e-3) / 1e9, "unit": "GDoF/s",
                    "h2d_bytes_per_step": 2 * 8 * ndof, "d2h_bytes_per_step": 8 * ndof},
            "gpu_launches": launches,
            "clocks": clk,
            "solves_per_s": args.steps / (t_max * 1e-3),
            "iterations": statistics.median(iters), "rel_residual_max": max(relres),
            "smoothing_steps": smooth_steps_total, "stage_share": shares,
            "apply": {"ms": apply_ms, "gdofs": ndof / (apply_ms * 1e-3) / 1e9},
            "vcycle_ms": vcycle_ms,
            "mixed_64cube_p4": mixed,
            "serving": serving,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
