"""Shared helpers of the GPU parity tests: build the CUDA hierarchy and the FP64
oracle hierarchy from the same seeded inputs and options."""

from __future__ import annotations

import numpy as np

from oracle import fem, hierarchy as hy, solver as so
from paper_2604_26441_b300 import inputs


def gpu_solver(rho: np.ndarray, p: float, fixed: np.ndarray | None = None, **opt):
    import torch
    from paper_2604_26441_b300 import gmg
    o = gmg.options(**opt)
    rho_d = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).cuda()
    return gmg.Solver(rho_d, p=p, fixed=fixed, opts=o)


def oracle_spec(**opt) -> so.SmootherSpec:
    kind = opt.get("smoother", "chebyshev")
    ck = opt.get("coarse_smoother", "jacobi")
    return so.SmootherSpec(kind, opt.get("degree", 2), opt.get("omega", 0.5), opt.get("alpha", 1.0 / 30.0),
                           opt.get("lambda_safety", 1.1), coarse_kind=ck,
                           coarse_degree=opt.get("coarse_degree", 2), coarse_omega=opt.get("coarse_omega", 0.5))


def config_opts(cfg) -> dict:
    return dict(levels=cfg.levels, smoother=cfg.smoother, degree=cfg.degree, coarse_smoother=None,
                coarse_degree=None, omega=cfg.omega, coarse_omega=None)


def oracle_hierarchy(rho, p, fixed, levels, matrix_free_fine=False):
    nz, ny, nx = rho.shape
    E = fem.moduli(rho, p)
    return hy.build_hierarchy((nx, ny, nz), E, fixed, levels=levels, matrix_free_fine=matrix_free_fine), E


def oracle_spec_from_opts(opts: dict) -> so.SmootherSpec:
    kind = opts["smoother"]
    ck = opts.get("coarse_smoother") or kind
    cd = opts.get("coarse_degree") or opts["degree"]
    co = opts.get("coarse_omega") or opts["omega"]
    return so.SmootherSpec(kind, opts["degree"], opts["omega"], opts.get("alpha", 1.0 / 30.0),
                           opts.get("lambda_safety", 1.1), coarse_kind=ck, coarse_degree=cd, coarse_omega=co)


def planes_from_csr(lev: hy.Level) -> np.ndarray:
    """The oracle's free x free operator laid out like gmg_get_bsr: [243, n_nodes]."""
    g = fem.Grid(*lev.dims)
    A = lev.K.tocoo()
    rows, cols = lev.free[A.row], lev.free[A.col]
    nr, r = rows // 3, rows % 3
    nc, c = cols // 3, cols % 3
    NX, NY = g.nx + 1, g.ny + 1
    ox = nc % NX - nr % NX
    oy = (nc // NX) % NY - (nr // NX) % NY
    oz = nc // (NX * NY) - nr // (NX * NY)
    assert np.abs(ox).max() <= 1 and np.abs(oy).max() <= 1 and np.abs(oz).max() <= 1
    slot = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)
    out = np.zeros((243, g.n_nodes))
    out[slot * 9 + r * 3 + c, nr] = A.data
    return out


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def structural_patterns(dims, fixed: np.ndarray, levels: int) -> list:
    """Boolean free x free patterns of K^l from boolean products (no cancellation):
    level 0 couples every DOF pair of nodes sharing an element."""
    import scipy.sparse as sp
    g = fem.Grid(*dims)
    dofs = g.element_dofs()
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    S = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(g.n_dof, g.n_dof)).tocsr()
    free = fem.free_dofs(fixed)
    S = S[free][:, free]
    out = [S]
    d, fx = tuple(dims), fixed
    for _ in range(1, levels):
        fc = hy.inject_fixed(d, fx)
        P = hy.prolongation(d)[free][:, fem.free_dofs(fc)]
        P.data[:] = 1.0
        S = (P.T @ S @ P).tocsr()
        d, fx, free = hy.coarse_dims(d), fc, fem.free_dofs(fc)
        out.append(S)
    return out


def pattern_planes(S, dims, free) -> np.ndarray:
    """A boolean free x free pattern laid out as [243, n_nodes]."""
    g = fem.Grid(*dims)
    A = S.tocoo()
    rows, cols = free[A.row], free[A.col]
    nr, r, nc, c = rows // 3, rows % 3, cols // 3, cols % 3
    NX, NY = g.nx + 1, g.ny + 1
    ox = nc % NX - nr % NX
    oy = (nc // NX) % NY - (nr // NX) % NY
    oz = nc // (NX * NY) - nr // (NX * NY)
    slot = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)
    out = np.zeros((243, g.n_nodes), dtype=bool)
    out[slot * 9 + r * 3 + c, nr] = A.data != 0
    return out


def slot_pattern_from_mask(mask: np.ndarray, dims) -> np.ndarray:
    """The CUDA path's implicit index map: slot (s, r, c) of node n is present iff
    the neighbour is inside the grid and DOFs (n, r), (n+o_s, c) are free."""
    nx, ny, nz = dims
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    n = np.arange(NX * NY * NZ)
    i, j, k = n % NX, (n // NX) % NY, n // (NX * NY)
    out = np.zeros((243, n.size), dtype=bool)
    for s in range(27):
        ox, oy, oz = s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1
        inside = (i + ox >= 0) & (i + ox < NX) & (j + oy >= 0) & (j + oy < NY) & (k + oz >= 0) & (k + oz < NZ)
        m = np.where(inside, n + ox + NX * (oy + NY * oz), 0)
        for r in range(3):
            for c in range(3):
                out[s * 9 + r * 3 + c] = inside & (((mask >> r) & 1) == 0) & (((mask[m] >> c) & 1) == 0)
    return out
