"""Learned warm start for GMG-PCG: training data from the solver, training with
the library's kernels, and evaluation against the cold start.

* ``generate``: seeded heterogeneous cantilevers (the Gaussian-filtered density
  recipe, p = 3) on several cubic grids, each solved by cold-start GMG-PCG for a
  few of the 16 rotated tip-edge loads; the network input is built by
  ``gmg_net_features`` and the target (the solution over its RMS) by
  ``gmg_net_target``, both kept on the device.  Fields the set-up screen refuses
  and loads whose solve misses the tolerance within the cap are left out and
  counted (a target must be a converged solution).
* ``train``: Adam steps (``gmg_net_train_step``) on random batches of one grid
  at a time, the gradient clipped to L2 norm ``clip``, the learning rate
  decayed on a cosine from ``lr`` to ``lr_final``; the loss is the error in the
  energy norm of each sample's own stiffness (the dataset keeps every field's
  solver for its matrix-free operator) or, with ``loss="mse"``, the mean
  squared error.
* ``evaluate``: for each problem, cold-start PCG against network warm start +
  PCG to the same tolerance, both timed with CUDA events on the solver's
  stream (the warm-start side includes the features, the forward pass and the
  energy-optimal rescaling), and the warm start's error in the energy norm
  and in L2 against a tightly converged cold-start solution.

Every numerical step runs in the CUDA library; this module only orchestrates.
"""

from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import gmg, inputs

TRAIN_GRIDS = (32, 40, 48, 56, 64)
N_DIRECTIONS = 16


def solver_options(stream: int | None = None, levels: int = 0):
    """The solver of the training data and of the evaluation: degree-2
    Chebyshev-Jacobi on every level (its band follows each level's
    lambda_max, so no field of the recipe trips the damped-Jacobi stability
    screen), automatic depth."""
    return gmg.options(levels=levels, smoother="chebyshev", degree=2, coarse_smoother=None, coarse_degree=None,
                       stream=stream)


@dataclasses.dataclass
class Dataset:
    """Per grid size n: inputs xs [M, (n+1)^3, 12], targets ts [M, (n+1)^3, 3]
    and ops[n][i], the solver of sample i's density field."""
    xs: dict
    ts: dict
    ops: dict
    iterations: list
    seconds: float
    skipped_fields: int = 0
    skipped_solves: int = 0

    def close(self):
        for lst in self.ops.values():
            for S in {id(S): S for S in lst}.values():
                S.close()
        self.ops = {}

    @property
    def size(self) -> int:
        return sum(int(x.shape[0]) for x in self.xs.values())


def generate(n_solves: int = 2000, grids=TRAIN_GRIDS, loads_per_field: int = 5, seed: int = 1000,
             tol: float = 1e-6, maxit: int = 500, device: str = "cuda") -> Dataset:
    import torch
    t0 = time.perf_counter()
    stream = torch.cuda.current_stream().cuda_stream
    per_grid = [n_solves // len(grids) + (1 if i < n_solves % len(grids) else 0) for i in range(len(grids))]
    rng = np.random.default_rng(seed)
    xs, ts, ops, its = {}, {}, {}, []
    field = skipped = unsolved = 0
    for n, m in zip(grids, per_grid):
        nn = (n + 1) ** 3
        X = torch.empty(m, nn, gmg.NET_IN, dtype=torch.float32, device=device)
        T = torch.empty(m, nn, 3, dtype=torch.float32, device=device)
        fixed = torch.from_numpy(inputs.clamp_xmin_mask(n, n, n)).to(device)
        k = 0
        ops[n] = []
        while k < m:
            rho = torch.from_numpy(inputs.filtered_random_density(n, n, n, seed + field)).to(device)
            field += 1
            try:
                S = gmg.Solver(rho, p=3.0, opts=solver_options(stream))
            except gmg.GMGError:
                skipped += 1  # a field the setup's failure screen refuses
                continue
            for d in rng.choice(N_DIRECTIONS, size=min(loads_per_field, m - k), replace=False):
                f = torch.from_numpy(inputs.rotated_tip_edge_load(n, n, n, int(d), N_DIRECTIONS)).to(device)
                u, info = S.solve(f, None, tol=tol, maxit=maxit)
                if info["status"] != 0:
                    unsolved += 1  # no converged target for this load: leave it out
                    continue
                its.append(info["iterations"])
                gmg.net_features((n, n, n), rho, f, fixed, X[k])
                gmg.net_target((n, n, n), u, T[k])
                ops[n].append(S)
                k += 1
        xs[n], ts[n] = X, T
    torch.cuda.synchronize()
    return Dataset(xs, ts, ops, its, time.perf_counter() - t0, skipped, unsolved)


def initial_params(seed: int = 0):
    import torch
    shapes = [(co, 27, ci) for ci, co, _, _ in gmg.net_layer_shapes()]
    return torch.from_numpy(inputs.he_normal_params(shapes, seed)).cuda()


def train(net: "gmg.WarmNet", data: Dataset, steps: int, batch: int = 4, lr: float = 5e-4, lr_final: float = 5e-5,
          clip: float = 1.0, seed: int = 0, loss: str = "energy"):
    """Runs ``steps`` Adam steps; returns (losses as a numpy array, seconds)."""
    import torch
    rng = np.random.default_rng(seed)
    sizes = sorted(data.xs)
    counts = np.array([data.xs[n].shape[0] for n in sizes], dtype=np.float64)
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        n = sizes[rng.choice(len(sizes), p=counts / counts.sum())]
        m = data.xs[n].shape[0]
        idx = rng.choice(m, size=min(batch, m), replace=False)
        c = 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps - 1)))
        ops = [data.ops[n][i] for i in idx] if loss == "energy" else None
        net.train_step((n, n, n), [data.xs[n][i] for i in idx], [data.ts[n][i] for i in idx],
                       lr_final + (lr - lr_final) * c, losses[s:s + 1], clip=clip, ops=ops)
    torch.cuda.synchronize()
    return losses.cpu().numpy(), time.perf_counter() - t0


def energy_error(S: "gmg.Solver", u0, u_ref) -> float:
    """||u0 - u_ref||_K / ||u_ref||_K with K applied by the FP32 operator."""
    import torch
    e = (u0 - u_ref).float()
    r = u_ref.float()
    ee = float(torch.dot(e.double(), S.apply(e).double()))
    rr = float(torch.dot(r.double(), S.apply(r).double()))
    return math.sqrt(max(ee, 0.0) / rr) if rr > 0 else float("nan")


def evaluate(net: "gmg.WarmNet", problems, tol: float = 1e-6, maxit: int = 500, reps: int = 3) -> list:
    """problems: [(rho (nz, ny, nx) device float, f device double)], cubic
    grids with sides a multiple of 8.  Per problem: iterations and median
    milliseconds of the cold and the warm-started solve, alpha, and the warm
    start's energy-norm and L2 errors."""
    import torch
    stream = torch.cuda.current_stream()
    out = []
    for rho, f in problems:
        S = gmg.Solver(rho, p=3.0, opts=solver_options(stream.cuda_stream))
        u_ref, _ = S.solve(f, None, tol=1e-10, maxit=2000)
        u = torch.zeros_like(f)

        def timed(fn):
            ms = []
            res = None
            for _ in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                res = fn()
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            return res, float(np.median(ms[1:]))

        def cold():
            u.zero_()
            return S.solve(f, u, tol=tol, maxit=maxit)[1]

        def warm():
            net.warm_start(S, rho, f, u, sync=False)
            return S.solve(f, u, tol=tol, maxit=maxit)[1]

        ic, ms_c = timed(cold)
        iw, ms_w = timed(warm)
        u0, alpha = net.warm_start(S, rho, f)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            net.warm_start(S, rho, f, u, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        out.append({"n": tuple(int(v) for v in S.dims), "cold_iterations": ic["iterations"],
                    "warm_iterations": iw["iterations"], "cold_ms": ms_c, "warm_ms": ms_w,
                    "warm_start_ms": a.elapsed_time(b) / reps, "cold_status": ic["status"],
                    "warm_status": iw["status"], "warm_rel_residual": iw["rel_residual"], "alpha": alpha,
                    "energy_error": energy_error(S, u0, u_ref),
                    "l2_error": float(torch.linalg.norm(u0 - u_ref) / torch.linalg.norm(u_ref))})
        S.close()
    return out


def held_out_problems(n: int, count: int, seed: int = 900000, device: str = "cuda"):
    """Cubic cantilevers of side n with densities and loads the training set never used."""
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        rho = torch.from_numpy(inputs.filtered_random_density(n, n, n, seed + i)).to(device)
        d = int(rng.integers(N_DIRECTIONS))
        f = torch.from_numpy(inputs.rotated_tip_edge_load(n, n, n, d, N_DIRECTIONS)).to(device)
        out.append((rho, f))
    return out
