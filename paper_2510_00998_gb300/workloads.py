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


def make(name, device="cuda", **overrides):
    """Create (ctx, b) for a named workload."""
    from . import dgmg
    w = dict(WORKLOADS[name])
    w.update(overrides)
    ctx = dgmg.Context(w["n"], w["p"], kappa_field(w["kappa"], w["n"]), precision=w["precision"])
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
            "launches": dgmg.kernel_launches()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(WORKLOADS))
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(a.name, a.solves, a.warmup)))


if __name__ == "__main__":
    main()
