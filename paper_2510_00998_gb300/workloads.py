"""Named synthetic workloads and a small runner (solves, timing, stage profile).

    python -m paper_2510_00998_gb300.workloads NAME [--solves K] [--warmup W]

Workloads (every input seeded and synthetic):
  2d16_p2        2D unit square, 16x16 cells, p = 2, kappa = 1,
                 f = 2 pi^2 sin(pi x) sin(pi y), FP64 V-cycle
  3d32_p3        3D unit cube, 32^3 cells, p = 3, kappa = 1,
                 f = 3 pi^2 prod sin(pi x_i), FP64 V-cycle
  3d64_p4_mixed  3D unit cube, 64^3 cells, p = 4, kappa_K = exp(N(0,1)) from
                 numpy default_rng(3), f as above, FP32 V-cycle in FP64 CG
  3d64_p4_fp64   the same problem with the FP64 V-cycle
  batch          256 independent 3D solves (n in [8,24], p in 2..4, lognormal
                 kappa, 8 random Fourier modes, default_rng(4)) through the
                 solve server vs plain FP64 one-at-a-time
  serve          Poisson arrivals (default_rng(5)) of requests with n in [8,48],
                 p in 2..5, kappa in {1, lognormal, two-phase 1/100}, at
                 multiples of the FP64 one-at-a-time capacity; p50/p99 latency
  *_gradual, *_gl  the 3D problems above with gradual p-coarsening (DG p,
                 p-1, ..., 1, then Q1) or in the Gauss-Legendre basis
  tables34       MGMult cycle counts of Tables 3-4 ("sin-product", GLL), 2D
                 9^2 .. 243^2, p = 2..6, direct and gradual p-coarsening
  table5         the same for the "two-peak" solution in the GLL and the GL basis
  volume_ab      the volume term r = b - kappa E u alone, 64^3 cells, p = 4, FP32:
                 sum-factorised CUDA-core kernel vs tcgen05 tensor-core contraction
  table6         the setting of Table 6: 2D 729^2 cells, FP64, p = 1..6, smoothing
                 step with the block factors precomputed vs recomputed per step
"""
import argparse
import json
import math
import time

import numpy as np

WORKLOADS = {
    "2d16_p2": dict(n=(16, 16), p=2, kappa=None, precision=0),
    "3d32_p3": dict(n=(32, 32, 32), p=3, kappa=None, precision=0),
    "3d64_p4_mixed": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=1),
    "3d64_p4_fp64": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=0),
    # the same problems with gradual p-coarsening (DG p, p-1, ..., 1, then Q1)
    "3d32_p3_gradual": dict(n=(32, 32, 32), p=3, kappa=None, precision=0, p_coarsening=1),
    "3d64_p4_mixed_gradual": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=1, p_coarsening=1),
    "3d64_p4_fp64_gradual": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=0, p_coarsening=1),
    # the same problems in the Gauss-Legendre nodal basis (Sec. 6.4)
    "3d64_p4_mixed_gl": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=1, basis=1),
    "3d64_p4_fp64_gl": dict(n=(64, 64, 64), p=4, kappa="lognormal3", precision=0, basis=1),
}


def kappa_field(spec, n):
    if spec is None:
        return None
    if spec == "lognormal3":
        return np.exp(np.random.default_rng(3).normal(size=int(np.prod(n))))
    raise ValueError(spec)


def sine_rhs(ctx, device):
    """b = (f, phi_i) for f = d pi^2 prod sin(pi x_i), through the library's quadrature."""
    import torch
    d = ctx.info.dim
    mq = ctx.p + 2
    xq = torch.empty(int(ctx.info.ncell) * mq ** d * d, dtype=torch.float64, device=device)
    ctx.quad_points(xq)
    X = xq.view(-1, d)
    f = torch.full((X.shape[0],), d * math.pi ** 2, dtype=torch.float64, device=device)
    for a in range(d):
        f = f * torch.sin(math.pi * X[:, a])
    b = torch.empty(ctx.ndof, dtype=torch.float64, device=device)
    ctx.load_vector(f.contiguous(), b)
    return b


def sin_product_rhs_2d(ctx, device):
    """b = (f, phi_i) for the "sin-product" solution sin(2 pi x) sin(2 pi y) of
    Sec. 6 (f = 8 pi^2 sin(2 pi x) sin(2 pi y)), through the library's quadrature."""
    import torch
    mq = ctx.p + 2
    xq = torch.empty(int(ctx.info.ncell) * mq ** 2 * 2, dtype=torch.float64, device=device)
    ctx.quad_points(xq)
    X = xq.view(-1, 2)
    f = 8 * math.pi ** 2 * torch.sin(2 * math.pi * X[:, 0]) * torch.sin(2 * math.pi * X[:, 1])
    b = torch.empty(ctx.ndof, dtype=torch.float64, device=device)
    ctx.load_vector(f.contiguous(), b)
    return b


# "two-peak" solution of Sec. 6 (Eq. two_peak_exact): u = g h with the bubble
# g = x(1-x)y(1-y) and h = 2 G_1 - G_2, G_k a Gaussian of width sigma_k centred
# at (x_0k, y_0k)
TWO_PEAK = ((0.3, 0.4, 0.2, 2.0), (0.8, 0.6, 0.1, -1.0))   # (x0, y0, sigma, weight)


def two_peak_u(x, y, xp=np):
    """The "two-peak" reference solution at points (x, y); xp = numpy or torch."""
    h = 0.0
    for x0, y0, sg, w in TWO_PEAK:
        h = h + w * xp.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2 * sg * sg))
    return x * (1 - x) * y * (1 - y) * h


def two_peak_f(x, y, xp=np):
    """f = -Lap u for the "two-peak" solution, written out by the product rule:
    Lap(g h) = h Lap g + 2 grad g . grad h + g Lap h with, per Gaussian G of
    width s, grad G = -(x - x0, y - y0) G / s^2 and Lap G = (r^2 / s^4 - 2 / s^2) G."""
    g = x * (1 - x) * y * (1 - y)
    gx, gy = (1 - 2 * x) * y * (1 - y), x * (1 - x) * (1 - 2 * y)
    lap_g = -2 * (y * (1 - y) + x * (1 - x))
    h = hx = hy = lap_h = 0.0
    for x0, y0, sg, w in TWO_PEAK:
        s2 = sg * sg
        dx, dy = x - x0, y - y0
        r2 = dx * dx + dy * dy
        G = w * xp.exp(-r2 / (2 * s2))
        h = h + G
        hx = hx - dx / s2 * G
        hy = hy - dy / s2 * G
        lap_h = lap_h + (r2 / (s2 * s2) - 2 / s2) * G
    return -(h * lap_g + 2 * (gx * hx + gy * hy) + g * lap_h)


def two_peak_rhs_2d(ctx, device):
    """b = (f, phi_i) for the "two-peak" solution, through the library's quadrature."""
    import torch
    mq = ctx.p + 2
    xq = torch.empty(int(ctx.info.ncell) * mq ** 2 * 2, dtype=torch.float64, device=device)
    ctx.quad_points(xq)
    X = xq.view(-1, 2)
    f = two_peak_f(X[:, 0], X[:, 1], torch)
    b = torch.empty(ctx.ndof, dtype=torch.float64, device=device)
    ctx.load_vector(f.contiguous(), b)
    return b


def tables34(meshes=(9, 27, 81, 243), degrees=(2, 3, 4, 5, 6), nu=4, device="cuda", p_coarsening=0,
             rhs="sin_product", basis=0, **opts):
    """MGMult cycles (Alg. 7) to reduce the unpreconditioned and the
    preconditioned residual by 1e-7 on n x n meshes, factor-3 h-coarsening: the
    setting of the paper's Tables 3-4 ("sin-product" or "two-peak" right-hand
    side, GLL basis) and Table 5 ("two-peak", GL basis: basis=1). The paper
    does not state the smoothing steps or the damping of these tables; nu = 4
    pre- and post-smoothing steps with the default omega = 0.8 reproduce them
    best among omega in 0.6..1.0 and nu in 1..4 (exact or interior-only block).
    Further
    keyword arguments are context options (omega_dg, block_inverse, ...).
    Returns {(n, p): (cycles unpreconditioned, cycles preconditioned)}, -1 where
    1000 cycles did not reach the tolerance."""
    import torch
    from . import dgmg
    make_rhs = {"sin_product": sin_product_rhs_2d, "two_peak": two_peak_rhs_2d}[rhs]
    out = {}
    for n in meshes:
        for p in degrees:
            ks = []
            for outer in (dgmg.DGMG_OUTER_MGMULT, dgmg.DGMG_OUTER_MGMULT_PREC):
                ctx = dgmg.Context((n, n), p, outer=outer, coarsening=3, nu_pre=nu, nu_post=nu, rtol=1e-7,
                                   maxit=1000, p_coarsening=p_coarsening, basis=basis, **opts)
                b = make_rhs(ctx, device)
                x = torch.zeros_like(b)
                st, rc = ctx.solve(b, x, allow_notconverged=True)
                ks.append(int(st.iterations) if rc == dgmg.DGMG_OK else -1)
                ctx.close()
            out[(n, p)] = tuple(ks)
    return out


def make(name, device="cuda", **overrides):
    """Create (ctx, b) for a named workload."""
    from . import dgmg
    w = dict(WORKLOADS[name])
    w.update(overrides)
    ctx = dgmg.Context(w["n"], w["p"], kappa_field(w["kappa"], w["n"]), precision=w["precision"], autotune=1,
                       p_coarsening=w.get("p_coarsening", 0), basis=w.get("basis", 0))
    return ctx, sine_rhs(ctx, device)


def run(name, solves=3, warmup=1):
    import torch
    from . import dgmg
    ctx, b = make(name)
    x = torch.zeros_like(b)
    for _ in range(warmup):
        x.zero_()
        ctx.solve(b, x)
    torch.cuda.synchronize()
    ctx.profile(True)
    t = time.perf_counter()
    its, res = [], []
    for _ in range(solves):
        x.zero_()
        st, _ = ctx.solve(b, x)
        its.append(st.iterations)
        res.append(st.rel_residual)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / solves
    prof = ctx.profile_read()
    ctx.profile(False)
    return {"workload": name, "ndof": ctx.ndof, "solve_ms": 1e3 * dt, "iterations": its,
            "rel_residual": max(res), "stages_ms_launches": prof,
            "launches": dgmg.kernel_launches(), "tiles": list(ctx.info.tiles)}


def run_volume_ab(n=(64, 64, 64), reps=20):
    """The volume term r = b - kappa E u (3D, p = 4, FP32 vectors) in both forms
    of dgmg_volume_residual_f32: sum-factorised CUDA-core kernel (method 0) and
    tcgen05 tensor-core contraction (method 1, TF32). Mean CUDA-event time per
    launch over `reps` launches (inputs larger than L2), algorithmic HBM bytes
    (u, b, r in FP32 and kappa in FP64 per cell) against the measured copy rate,
    and the TF32 result's difference from the FP32 one."""
    import torch
    from . import dgmg
    kappa = np.exp(np.random.default_rng(3).normal(size=int(np.prod(n))))
    ctx = dgmg.Context(n, 4, kappa)
    g = torch.Generator(device="cuda").manual_seed(9)
    u = torch.randn(ctx.ndof, dtype=torch.float32, device="cuda", generator=g)
    b = torch.randn(ctx.ndof, dtype=torch.float32, device="cuda", generator=g)
    out = {"workload": f"volume term, {n[0]}x{n[1]}x{n[2]} cells, p = 4, FP32", "ncell": int(ctx.info.ncell)}
    bytes_per_launch = int(ctx.info.ncell) * (3 * 125 * 4 + 8)
    res = {}
    for method, name in ((0, "sum_factorised_fp32"), (1, "tcgen05_tf32")):
        r = torch.empty_like(u)
        for _ in range(3):
            ctx.volume_residual_f32(u, b, r, method)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.volume_residual_f32(u, b, r, method)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[method] = r
        out[name] = {"ms": ms, "gb_per_s": bytes_per_launch / (ms * 1e-3) / 1e9, "bytes_per_launch": bytes_per_launch}
    vol = (b - res[0]).abs().max().item()
    out["tf32_max_diff_rel"] = float((res[1] - res[0]).abs().max().item() / vol)
    out["wait_timeouts"] = dgmg.wait_timeouts()
    return out


def run_table6(n=729, degrees=(1, 2, 3, 4, 5, 6), steps=10):
    """The setting of the paper's Table 6 on the GPU: 2D, n x n cells, FP64, the
    fused single-touch smoothing step (Alg. 4) with the block inverses'
    factors precomputed at set-up and recomputed before every step
    (opts.recompute_block); time per step and per DoF (CUDA events of the
    library's per-stage profile, smoothing stage only)."""
    import torch
    from . import dgmg
    out = {"workload": f"2D {n}x{n} cells, kappa = 1, FP64, {steps} smoothing steps", "rows": []}
    for p in degrees:
        row = {"p": p}
        for rb, key in ((0, "precomputed"), (1, "recompute")):
            ctx = dgmg.Context((n, n), p, None, recompute_block=rb)
            g = torch.Generator(device="cuda").manual_seed(5)
            u = torch.randn(ctx.ndof, dtype=torch.float64, device="cuda", generator=g)
            b = torch.randn(ctx.ndof, dtype=torch.float64, device="cuda", generator=g)
            ctx.smooth(u, b, 2)
            torch.cuda.synchronize()
            ctx.profile(True)
            ctx.smooth(u, b, steps)
            torch.cuda.synchronize()
            ms, k = ctx.profile_read()["smooth"]
            ctx.profile(False)
            row[key] = {"ms_per_step": ms / k, "ns_per_dof": ms / k * 1e6 / ctx.ndof}
            row["ndof"] = ctx.ndof
            ctx.close()
        out["rows"].append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(WORKLOADS) + ["batch", "serve", "tables34", "table5", "volume_ab", "table6"])
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--count", type=int, default=0)
    ap.add_argument("--max-active", type=int, default=0)
    a = ap.parse_args()
    if a.name == "batch":
        kw = {}
        if a.count:
            kw["count"] = a.count
        if a.max_active:
            kw["max_active"] = a.max_active
        print(json.dumps(run_batch(**kw)))
    elif a.name == "serve":
        kw = {}
        if a.count:
            kw["count"] = a.count
        if a.max_active:
            kw["max_active"] = a.max_active
        print(json.dumps(run_serve(**kw)))
    elif a.name == "tables34":
        out = {}
        for pc in (0, 1):
            res = tables34(p_coarsening=pc)
            out["gradual" if pc else "direct"] = {f"{n}x{n} p={p}": {"unprec": v[0], "prec": v[1]}
                                                  for (n, p), v in res.items()}
        print(json.dumps(out))
    elif a.name == "table5":
        out = {}
        for basis, key in ((0, "two_peak_gll"), (1, "two_peak_gl")):
            res = tables34(rhs="two_peak", basis=basis)
            out[key] = {f"{n}x{n} p={p}": {"unprec": v[0], "prec": v[1]} for (n, p), v in res.items()}
        print(json.dumps(out))
    elif a.name == "volume_ab":
        print(json.dumps(run_volume_ab()))
    elif a.name == "table6":
        print(json.dumps(run_table6()))
    else:
        print(json.dumps(run(a.name, a.solves, a.warmup)))



# ------------------------------------------------------------------ many solves
def fourier_rhs_values(X, coeffs, waves):
    """f = sum_m a_m prod_i sin(k_{m,i} pi x_i) at points X (torch, [npts, d])."""
    import torch
    f = torch.zeros(X.shape[0], dtype=torch.float64, device=X.device)
    for a, k in zip(coeffs, waves):
        term = torch.full_like(f, float(a))
        for i in range(X.shape[1]):
            term = term * torch.sin(float(k[i]) * math.pi * X[:, i])
        f += term
    return f


def two_phase_kappa(n, rng):
    """kappa in {1, 100}: 100 on the side of a random plane through the cube."""
    d = len(n)
    normal = rng.normal(size=d)
    normal /= np.linalg.norm(normal)
    centres = [(np.arange(v) + 0.5) / v for v in n]
    grids = np.meshgrid(*centres[::-1], indexing="ij")[::-1]      # x fastest when flattened
    s = sum(normal[a] * (grids[a] - 0.5) for a in range(d)) + rng.uniform(-0.2, 0.2)
    return np.where(s.reshape(-1) > 0, 100.0, 1.0)


def request_stream(kind, count, seed):
    """Seeded problem list. kind 'batch': n in [8,24], p in {2,3,4}, lognormal kappa,
    8 random Fourier modes; kind 'serve': n in [8,48], p in 2..5, kappa one of
    {1, lognormal, two-phase 1/100}, same RHS family."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        if kind == "batch":
            nn = int(rng.integers(8, 25))
            p = int(rng.integers(2, 5))
            kk = "lognormal"
        else:
            nn = int(rng.integers(8, 49))
            p = int(rng.integers(2, 6))
            kk = ["one", "lognormal", "two-phase"][int(rng.integers(0, 3))]
        n = (nn, nn, nn)
        ncell = nn ** 3
        if kk == "one":
            kappa = None
        elif kk == "lognormal":
            kappa = np.exp(rng.normal(size=ncell))
        else:
            kappa = two_phase_kappa(n, rng)
        coeffs = rng.normal(size=8)
        waves = rng.integers(1, 5, size=(8, 3))
        out.append(dict(n=n, p=p, kappa=kappa, kappa_kind=kk, coeffs=coeffs, waves=waves))
    return out


def build_rhs(reqs, device="cuda"):
    """b for every request, through the library's quadrature (one kappa = 1
    context per distinct mesh and degree, freed afterwards)."""
    import torch
    from . import dgmg
    cache = {}
    for r in reqs:
        key = (r["n"], r["p"])
        if key not in cache:
            ctx = dgmg.Context(r["n"], r["p"])
            mq = r["p"] + 2
            xq = torch.empty(int(ctx.info.ncell) * mq ** 3 * 3, dtype=torch.float64, device=device)
            ctx.quad_points(xq)
            cache[key] = (ctx, xq.view(-1, 3))
        ctx, X = cache[key]
        b = torch.empty(ctx.ndof, dtype=torch.float64, device=device)
        ctx.load_vector(fourier_rhs_values(X, r["coeffs"], r["waves"]).contiguous(), b)
        r["b"] = b
    torch.cuda.synchronize()
    for ctx, _ in cache.values():
        ctx.close()


def one_at_a_time(reqs, precision=0, solve_times=None):
    """Solve every request alone in order (create, solve, destroy); returns the
    per-request service times in seconds (set-up included). With a list as
    `solve_times`, the solve-only time of each request is appended to it."""
    import torch
    from . import dgmg
    times = []
    for r in reqs:
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx = dgmg.Context(r["n"], r["p"], r["kappa"], precision=precision)
        x = torch.zeros_like(r["b"])
        ts = time.perf_counter()
        st, _ = ctx.solve(r["b"], x)
        if solve_times is not None:
            solve_times.append(time.perf_counter() - ts)
        ctx.close()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
        assert st.rel_residual <= 1e-10, st.rel_residual
    return times


def batched(reqs, solves=2, precision=0):
    """All requests as one dgmg_batch: set-up time, then `solves` batched
    solves from x = 0 (the second and later replay the captured iteration).
    Returns (setup_s, [solve_s], stats of the last solve, batch info)."""
    import torch
    from . import dgmg
    torch.cuda.synchronize()
    t = time.perf_counter()
    batch = dgmg.Batch([(r["n"], r["p"], r["kappa"]) for r in reqs], autotune=1, precision=precision)
    setup = time.perf_counter() - t
    bs = [r["b"] for r in reqs]
    times, stats = [], None
    for _ in range(solves):
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        t = time.perf_counter()
        stats, _ = batch.solve(bs, xs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    info = batch.info()
    batch.close()
    return setup, times, stats, info


def fifo_latencies(arrivals, service):
    """Latencies of a one-at-a-time FIFO server with the given service times."""
    t, out = 0.0, []
    for a, s in zip(arrivals, service):
        t = max(t, a) + s
        out.append(t - a)
    return out


def serve_trace(reqs, arrivals, budget, max_active, precision=1, return_x=False):
    """Submit each request at its arrival time to a server; returns
    (latencies, makespan, stats list, server info), and the solutions with
    `return_x`."""
    import torch
    from . import dgmg
    srv = dgmg.Server(budget, max_active, precision=precision)
    xs = [torch.zeros_like(r["b"]) for r in reqs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets, sub_t = [None] * len(reqs), [0.0] * len(reqs)
    done = {}
    k = 0
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(reqs) and arrivals[k] <= now:
            r = reqs[k]
            tickets[k] = srv.submit(r["n"], r["p"], r["b"], xs[k], r["kappa"])
            sub_t[k] = arrivals[k]
            k += 1
        for i in range(k):
            if i in done:
                continue
            st, stats = srv.poll(tickets[i])
            if st == dgmg.DGMG_DONE:
                done[i] = (time.perf_counter() - t0, stats)
        time.sleep(0.0002)
    makespan = time.perf_counter() - t0
    lat = [done[i][0] - sub_t[i] for i in range(len(reqs))]
    stats = [done[i][1] for i in range(len(reqs))]
    info = srv.info()
    srv.close()
    if return_x:
        return lat, makespan, stats, info, xs
    return lat, makespan, stats, info


def pct(v, q):
    return float(np.percentile(np.asarray(v), q))


def run_batch(count=256, seed=4, max_active=32, budget_gb=64):
    """All requests submitted at once to a mixed-precision server vs plain FP64
    one-at-a-time. solves/s for both (set-up included in both)."""
    reqs = request_stream("batch", count, seed)
    build_rhs(reqs)
    solve_only = []
    t_alone = one_at_a_time(reqs, precision=0, solve_times=solve_only)
    setup, bt, bstats, binfo = batched(reqs)
    msetup, mbt, mstats, minfo = batched(reqs, precision=1)
    lat, makespan, stats, info = serve_trace(reqs, [0.0] * count, budget_gb << 30, max_active)
    return {"workload": f"batch of {count} 3D solves, n in [8,24], p in 2..4, lognormal kappa, Fourier RHS",
            "fp64_one_at_a_time_solves_per_s": count / sum(t_alone),
            "fp64_one_at_a_time_solve_only_solves_per_s": count / sum(solve_only),
            "batched_fp64": {"setup_s": setup, "solve_s": bt, "solves_per_s": count / (setup + bt[0]),
                             "solve_only_solves_per_s": count / min(bt),
                             "iterations_max": max(s.iterations for s in bstats),
                             "max_rel_residual": max(s.rel_residual for s in bstats),
                             "groups": binfo.groups, "kernels_per_iteration": binfo.kernels_per_iteration,
                             "tiles": {f"q={binfo.group_q[k]}": list(binfo.group_tiles[k])
                                       for k in range(min(binfo.groups, 4))},
                             "ndof": binfo.ndof},
            "batched_mixed": {"setup_s": msetup, "solve_s": mbt, "solves_per_s": count / (msetup + mbt[0]),
                              "solve_only_solves_per_s": count / min(mbt),
                              "iterations_max": max(s.iterations for s in mstats),
                              "max_rel_residual": max(s.rel_residual for s in mstats),
                              "kernels_per_iteration": minfo.kernels_per_iteration,
                              "tiles": {f"q={minfo.group_q[k]}": list(minfo.group_tiles[k])
                                        for k in range(min(minfo.groups, 4))}},
            "served_mixed_solves_per_s": count / makespan,
            "served_p50_s": pct(lat, 50), "served_p99_s": pct(lat, 99),
            "max_rel_residual": max(s.rel_residual for s in stats),
            "cache_misses": info.cache_misses, "max_active": max_active}


def run_serve(count=64, seed=5, rates=(0.25, 0.5, 1.0, 2.0, 4.0), max_active=16, budget_gb=96):
    """Poisson arrivals at multiples of the plain FP64 one-at-a-time capacity."""
    reqs = request_stream("serve", count, seed)
    build_rhs(reqs)
    service = one_at_a_time(reqs, precision=0)
    capacity = len(service) / sum(service)
    rng = np.random.default_rng(seed + 1000)
    gaps = rng.exponential(size=count)
    out = {"workload": f"{count} requests, n in [8,48], p in 2..5, kappa in {{1, lognormal, two-phase}}",
           "fp64_capacity_solves_per_s": capacity, "rates": []}
    for m in rates:
        lam = m * capacity
        arrivals = list(np.cumsum(gaps / lam))
        fifo = fifo_latencies(arrivals, service)
        lat, makespan, stats, info = serve_trace(reqs, arrivals, budget_gb << 30, max_active)
        out["rates"].append({"rate_x_capacity": m, "rate_per_s": lam,
                             "served": {"solves_per_s": count / makespan, "p50_s": pct(lat, 50),
                                        "p99_s": pct(lat, 99)},
                             "fp64_one_at_a_time": {
                                 "solves_per_s": count / max(a + l for a, l in zip(arrivals, fifo)),
                                 "p50_s": pct(fifo, 50), "p99_s": pct(fifo, 99)},
                             "max_rel_residual": max(s.rel_residual for s in stats)})
    return out


if __name__ == "__main__":
    main()
