"""Fixed workloads for profiling the CUDA path under ncu.

    python profile_cases.py solve-c2    # set-up + 2 solves, 100^3
    python profile_cases.py solve-c2-hostloop  # the same, PCG driven from the host
    python profile_cases.py smooth-c2   # set-up, one packed smoothing call, 3 fine smoothing passes
    python profile_cases.py apply-c2    # the same, then 5 fine operator applies (handle's own vectors)
    python profile_cases.py smooth-l1-c2  # set-up + 3 level-1 smoothing passes (the level's default kernel)
    python profile_cases.py apply-l1-c2   # set-up + 3 level-1 operator applies (matrix-free where exact)
    python profile_cases.py smooth-c2-bf16x3  # fine smoothing, tensor-core contraction
    python profile_cases.py smooth-c2-pair    # fine smoothing, two element columns a thread (8x16 threads, 17 planes)
    python profile_cases.py warmstart-80  # 80^3 set-up, one learned warm start + solve
    python profile_cases.py warmstart-80-tf32  # the same with tensor-core convolutions
    python profile_cases.py train-48      # 48^3 set-up, 3 energy-loss train steps (batch 4)
    python profile_cases.py multi-64      # 64^3 (a batch grid), one 16-load solve, host-driven loop
    python profile_cases.py multi-apply-c2  # 100^3, 16 loads: packing, then 5 multi-load operator applies
    python profile_cases.py multi-apply-c2-tc  # the same with the tensor-core level-0 operator

Each case prints the library's kernel-launch counter after set-up, so that
``ncu -s`` can skip the set-up kernels.  The solve normally runs its PCG
iterations as one CUDA graph with a conditional while node, whose kernels a
per-launch ncu list does not show; the host-loop case launches the same kernels
in the same order one by one.

    python profile_cases.py summarize LAUNCHES.csv [FIRST_ID]

reads the CSV that ``ncu --metrics gpu__time_duration.sum --csv --log-file``
writes and prints, per kernel, its launches, total time and share of the time of
the launches with ID >= FIRST_ID (e.g. the set-up launch count, to keep only the
solves).
"""

from __future__ import annotations

import sys


def summarize(path: str, first_id: int = 0) -> str:
    import collections
    import csv
    import re

    with open(path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    agg = collections.defaultdict(lambda: [0, 0.0])
    n = 0
    for row in csv.DictReader(lines):
        if row.get("Metric Name") != "gpu__time_duration.sum" or int(row["ID"]) < first_id:
            continue
        us = float(row["Metric Value"].replace(",", ""))
        us *= {"nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "second": 1e6, "s": 1e6}[row["Metric Unit"]]
        name = re.sub(r"^void ", "", row["Kernel Name"])
        name = re.sub(r"<unnamed>::|\(anonymous namespace\)::|gmg::", "", name)
        name = re.sub(r"\((FineArgs|BsrArgs|GHat|CoarseFused|const|int|float|double|unsigned|long|std::).*$", "", name)
        agg[name][0] += 1
        agg[name][1] += us
        n += 1
    tot = sum(v[1] for v in agg.values())
    out = [f"launches {n}, total {tot:.1f} us", "", "| kernel | launches | total us | share | us/launch |",
           "|---|---:|---:|---:|---:|"]
    for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"| `{k}` | {c} | {t:.1f} | {100 * t / tot:.2f} % | {t / c:.2f} |")
    return "\n".join(out)


def main(case: str) -> None:
    import torch

    from paper_2604_26441_b300 import gmg, inputs

    if case in ("warmstart-80", "warmstart-80-tf32", "train-48"):
        return net_case(case)
    if case.startswith("multi-"):
        return multi_case(case)
    cfg = inputs.CONFIGS["c2"]
    fine = "bf16x3" if case.endswith("-bf16x3") else "fp32"
    S = gmg.Solver(torch.from_numpy(cfg.rho()).cuda(), p=cfg.p,
                   opts=gmg.config_options(cfg, device_loop=case != "solve-c2-hostloop", fine_smoother=fine))
    torch.cuda.synchronize()
    print("setup launches", gmg.kernel_launches(), flush=True)
    if case in ("solve-c2", "solve-c2-hostloop"):
        f = torch.from_numpy(cfg.load()).cuda()
        for _ in range(2):
            u, info = S.solve(f, tol=cfg.tol, maxit=cfg.maxit)
            print(info, flush=True)
    elif case == "apply-l1-c2":
        n1 = S.level_nodes(1)
        x = torch.ones(3 * n1, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            S.level_apply(1, x, y)
        torch.cuda.synchronize()
    elif case == "smooth-l1-c2":
        n1 = S.level_nodes(1)
        b = torch.ones(3 * n1, device="cuda")
        x = torch.zeros(3 * n1, device="cuda")
        for _ in range(3):
            S.level_smooth(1, b, x)
        torch.cuda.synchronize()
    elif case in ("smooth-c2", "smooth-c2-bf16x3", "smooth-c2-pair", "apply-c2"):
        if case == "smooth-c2-pair":
            S.set_fine_plan("pair-8x16", 17)
        # one level-0 smoothing call packs seeded vectors into the handle's own
        # right-hand side and iterate (and runs 3 smoothing steps); the passes
        # then run the fine kernel on those vectors (no repacking kernels)
        x = torch.from_numpy(inputs.random_free_vector(cfg.fixed(), 1)).cuda()
        y = torch.from_numpy(inputs.random_free_vector(cfg.fixed(), 2)).cuda()
        S.level_smooth(0, x, y)
        torch.cuda.synchronize()
        print("after packing", gmg.kernel_launches(), flush=True)
        for _ in range(3 if case.startswith("smooth-c2") else 5):
            S.fine_pass("smooth" if case.startswith("smooth-c2") else "apply")
        torch.cuda.synchronize()
        S.set_fine_plan(None)
    else:
        raise SystemExit(f"unknown case {case}")
    print("total launches", gmg.kernel_launches(), flush=True)


def multi_case(case: str) -> None:
    """The multi-load path: a batch grid's 16-load solve (the loop launched
    from the host, so that every kernel is its own launch), or the 100^3
    multi-load level-0 operator alone."""
    import torch

    from paper_2604_26441_b300 import gmg, inputs

    n = 64 if case == "multi-64" else 100
    rho = torch.from_numpy(inputs.filtered_random_density(n, n, n, 305)).cuda()
    if case == "multi-64":
        opts = gmg.options(levels=0, smoother="jacobi", degree=2, coarse_smoother=None, coarse_degree=None,
                           omega=0.5, coarse_omega=None, device_loop=False)
    else:
        opts = gmg.options(levels=2, smoother="jacobi", coarse_smoother=None, omega=0.5)
    S = gmg.Solver(rho, p=3.0, opts=opts)
    if case.endswith("-tc"):
        S.set_multi_kernel("tc")
    fs = [torch.from_numpy(inputs.rotated_tip_edge_load(n, n, n, k, 16)).cuda() for k in range(16)]
    fixed = inputs.clamp_xmin_mask(n, n, n)
    xs = [torch.from_numpy(inputs.random_free_vector(fixed, 50 + k)).cuda() for k in range(16)]
    S.apply_multi(xs)  # allocates the workspace and packs the operands
    torch.cuda.synchronize()
    print("setup launches", gmg.kernel_launches(), flush=True)
    if case == "multi-64":
        _, infos = S.solve_multi(fs)
        print([i["iterations"] for i in infos], flush=True)
    else:
        for _ in range(5):
            S.apply_multi(xs)
    torch.cuda.synchronize()
    print("total launches", gmg.kernel_launches(), flush=True)


def net_case(case: str) -> None:
    """The learned warm start with seeded (untrained) parameters: the kernels
    and their costs do not depend on the parameter values."""
    import torch

    from paper_2604_26441_b300 import gmg, inputs, warmstart as ws

    n = 80 if case.startswith("warmstart-80") else 48
    rho = torch.from_numpy(inputs.filtered_random_density(n, n, n, 4242)).cuda()
    fixed = torch.from_numpy(inputs.clamp_xmin_mask(n, n, n)).cuda()
    S = gmg.Solver(rho, p=3.0, opts=ws.solver_options())
    net = gmg.WarmNet(ws.initial_params(0))
    if case.endswith("-tf32"):
        net.set_arith("tf32")
    fs = [torch.from_numpy(inputs.rotated_tip_edge_load(n, n, n, k)).cuda() for k in range(4)]
    if case == "train-48":
        xs = [gmg.net_features((n, n, n), rho, f, fixed) for f in fs]
        ts = [gmg.net_target((n, n, n), S.solve(f)[0]) for f in fs]
    torch.cuda.synchronize()
    print("setup launches", gmg.kernel_launches(), flush=True)
    if case.startswith("warmstart-80"):
        u0, alpha = net.warm_start(S, rho, fs[0])
        net.status()
        _, info = S.solve(fs[0], u0)
        print("alpha", alpha, info, flush=True)
    else:
        for _ in range(3):
            net.train_step((n, n, n), xs, ts, 1e-4, clip=1.0, ops=[S] * 4)
    torch.cuda.synchronize()
    print("total launches", gmg.kernel_launches(), flush=True)


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[1] == "summarize":
        print(summarize(sys.argv[2], int(sys.argv[3]) if len(sys.argv) > 3 else 0))
    else:
        main(sys.argv[1] if len(sys.argv) > 1 else "solve-c2")
