"""Fixed workloads for profiling the CUDA path under ncu.

    python -m paper_2604_26441_b300.profile_cases solve-c2    # set-up + 2 solves, 100^3
    python -m paper_2604_26441_b300.profile_cases smooth-c2   # set-up + 3 fine smoothing passes
    python -m paper_2604_26441_b300.profile_cases apply-c2    # set-up + 5 fine operator applies

Each case prints the library's kernel-launch counter after set-up, so that
``ncu -s`` can skip the set-up kernels.
"""

from __future__ import annotations

import sys


def main(case: str) -> None:
    import torch

    from paper_2604_26441_b300 import gmg, inputs

    cfg = inputs.CONFIGS["c2"]
    S = gmg.Solver(torch.from_numpy(cfg.rho()).cuda(), p=cfg.p, opts=gmg.config_options(cfg))
    torch.cuda.synchronize()
    print("setup launches", gmg.kernel_launches(), flush=True)
    if case == "solve-c2":
        f = torch.from_numpy(cfg.load()).cuda()
        for _ in range(2):
            u, info = S.solve(f, tol=cfg.tol, maxit=cfg.maxit)
            print(info, flush=True)
    elif case in ("smooth-c2", "apply-c2"):
        x = torch.from_numpy(inputs.random_free_vector(cfg.fixed(), 1)).cuda()
        y = torch.from_numpy(inputs.random_free_vector(cfg.fixed(), 2)).cuda()
        for _ in range(3 if case == "smooth-c2" else 5):
            if case == "smooth-c2":
                S.level_smooth(0, x, y)
            else:
                S.apply(x, y)
        torch.cuda.synchronize()
    else:
        raise SystemExit(f"unknown case {case}")
    print("total launches", gmg.kernel_launches(), flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "solve-c2")
