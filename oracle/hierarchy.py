"""Oracle: the Galerkin geometric-multigrid hierarchy (TEST INFRASTRUCTURE ONLY; FP64).

Paper passages followed:

* Sec. "Transfer Operators and Boundary Masking", Eq. trilinear_weights and
  Eq. vector_prolongation -- 2:1 coarsening, tensor-product 1D weights
  {1, 1/2, 0}, P = P_s (x) I_3, R = P^T;
* same section, Dirichlet inheritance by injection -- a coarse DOF is free iff
  the fine DOF at (2i, 2j, 2k) is free;
* same section, Eq. galerkin_level1 and "Coarser levels" --
  K^{l+1} = R^l K^l P^l, the level-1 operator also written element by element
  over the eight child prolongation patterns;
* Sec. "Chebyshev-Jacobi Smoother" and "Spectral-radius estimation" -- D =
  diag(K^l), power iteration on D^{-1} K^l (20 fine / 10 coarse iterations,
  floor 1e-6);
* Sec. "Matrix-Free V-Cycle" and the reported safeguards -- coarsest level by
  dense Cholesky of K^L + eps I, eps = max(mean_diag * 1e-8, 1e-14), when it
  has at most the dense-Cholesky cutoff (5000) free DOFs; above the cutoff a
  fixed-count PCG (80 steps, the reproducibility defaults table) instead.

Readings where the paper is silent:

* coarse element counts are floor(N/2) per axis; an odd fine node index equal
  to 2*Nc + 1 (only when N is odd) takes weight 1 from coarse node Nc;
* the power iteration starts from v_i = ((i * 2654435761) mod 2^32) / 2^32 - 0.5
  over the level's full DOF index i, restricted to free DOFs, is normalised in
  the 2-norm every step, and returns the D-Rayleigh quotient v^T K v / v^T D v;
* automatic depth coarsens while the coarsest free-DOF count exceeds the
  Cholesky cutoff and every element count is at least 2;
* the fixed-count coarsest PCG is preconditioned by the level's diagonal
  (Jacobi), starts from 0, takes exactly the configured number of steps, and
  stops early only when r.z becomes exactly 0 (the solution is then exact).
"""

from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np
import scipy.sparse as sp

from .fem import Grid, LOCAL_NODES, assemble, free_dofs, matfree_apply

HASH_MULT = 2654435761


def coarse_dims(dims):
    return tuple(int(d) // 2 for d in dims)


def prolongation_1d(nf: int) -> sp.csr_matrix:
    """(nf+1) x (nc+1) 1D trilinear prolongation, nc = nf // 2 (Eq. trilinear_weights)."""
    nc = nf // 2
    rows, cols, vals = [], [], []
    for f in range(nf + 1):
        if f % 2 == 0:
            rows.append(f), cols.append(f // 2), vals.append(1.0)
        elif f < 2 * nc:
            rows += [f, f]
            cols += [(f - 1) // 2, (f + 1) // 2]
            vals += [0.5, 0.5]
        else:  # f == 2*nc + 1: the clamp reading for odd nf
            rows.append(f), cols.append(nc), vals.append(1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf + 1, nc + 1))


def scalar_prolongation(dims) -> sp.csr_matrix:
    """P_s with entries w_x w_y w_z over node indices (x fastest)."""
    nx, ny, nz = dims
    return sp.kron(prolongation_1d(nz), sp.kron(prolongation_1d(ny), prolongation_1d(nx))).tocsr()


def prolongation(dims) -> sp.csr_matrix:
    """Vector transfer P = P_s (x) I_3 on all DOFs (Eq. vector_prolongation)."""
    return sp.kron(scalar_prolongation(dims), sp.identity(3)).tocsr()


def inject_fixed(dims_f, fixed_f: np.ndarray) -> np.ndarray:
    """Coarse fixed flags: DOF (I,J,K,c) copies fine DOF (2I,2J,2K,c)."""
    gf = Grid(*dims_f)
    gc = Grid(*coarse_dims(dims_f))
    I, J, K = gc.node_ijk()
    nf = gf.node(2 * I, 2 * J, 2 * K)
    return np.asarray(fixed_f).reshape(-1, 3)[nf].reshape(-1).copy()


def galerkin(Kff: sp.csr_matrix, Pff: sp.csr_matrix) -> sp.csr_matrix:
    """K^{l+1} = P_ff^T K^l_ff P_ff by explicit sparse products."""
    return (Pff.T @ Kff @ Pff).tocsr()


def _child_weights_1d(e: np.ndarray, nf: int) -> tuple[np.ndarray, np.ndarray]:
    """Parent coarse element and (len(e), 2, 2) local 1D weights W[fine_local, coarse_local]
    for fine elements e along one axis."""
    nc = nf // 2
    parent = np.minimum(e // 2, nc - 1)
    W = np.zeros((e.size, 2, 2))
    clamp = (nf % 2 == 1) & (e == nf - 1)
    pos = e - 2 * parent
    p0 = (~clamp) & (pos == 0)
    p1 = (~clamp) & (pos == 1)
    W[p0] = [[1.0, 0.0], [0.5, 0.5]]
    W[p1] = [[0.5, 0.5], [0.0, 1.0]]
    W[clamp] = [[0.0, 1.0], [0.0, 1.0]]
    return parent, W


def level1_elementwise(dims_f, E: np.ndarray, Ke: np.ndarray, fixed_f: np.ndarray,
                       fixed_c: np.ndarray, batch: int = 65536) -> sp.csr_matrix:
    """Eq. galerkin_level1: K^1 = sum_e E_e (P_e)^T K_e P_e, where P_e is the 24x24
    restriction of the prolongation to fine element e (its coarse parent's eight
    nodes -> its own eight nodes, rows of fixed fine DOFs removed).  Returned on
    the coarse free DOFs, without any global fine matrix."""
    gf = Grid(*dims_f)
    gc = Grid(*coarse_dims(dims_f))
    nx, ny, nz = dims_f
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    cx, Wx = _child_weights_1d(ex, nx)
    cy, Wy = _child_weights_1d(ey, ny)
    cz, Wz = _child_weights_1d(ez, nz)
    fdofs = gf.element_dofs()
    cen = np.empty((ex.size, 8), dtype=np.int64)
    for b, (bx, by, bz) in enumerate(LOCAL_NODES):
        cen[:, b] = gc.node(cx + bx, cy + by, cz + bz)
    cdofs = (3 * cen[:, :, None] + np.arange(3)).reshape(-1, 24)
    free_f = (np.asarray(fixed_f) == 0).astype(np.float64)
    # Contributions are summed batch by batch into one sparse matrix, so memory
    # stays near the size of K^1 itself rather than of all 576 n_elem terms.
    K1 = sp.csr_matrix((gc.n_dof, gc.n_dof))
    for s in range(0, ex.size, batch):
        sl = slice(s, min(s + batch, ex.size))
        n = sl.stop - sl.start
        # scalar 8x8 weights: w[a, b] = Wx[ax,bx] Wy[ay,by] Wz[az,bz]
        w = np.ones((n, 8, 8))
        for a, (ax, ay, az) in enumerate(LOCAL_NODES):
            for b, (bx, by, bz) in enumerate(LOCAL_NODES):
                w[:, a, b] = Wx[sl, ax, bx] * Wy[sl, ay, by] * Wz[sl, az, bz]
        Pe = np.einsum("nab,cd->nacbd", w, np.eye(3)).reshape(n, 24, 24)
        Pe *= free_f[fdofs[sl]][:, :, None]
        T = np.einsum("nai,ab,nbj->nij", Pe, Ke, Pe, optimize=True) * E[sl, None, None]
        d = cdofs[sl]
        K1 = K1 + sp.coo_matrix((T.reshape(-1), (np.repeat(d, 24, axis=1).reshape(-1),
                                                 np.tile(d, (1, 24)).reshape(-1))),
                                shape=(gc.n_dof, gc.n_dof)).tocsr()
    fc = free_dofs(fixed_c)
    return K1[fc][:, fc].tocsr()


def power_start_vector(n_dof_full: int, free: np.ndarray) -> np.ndarray:
    i = np.arange(n_dof_full, dtype=np.uint64)
    v = ((i * np.uint64(HASH_MULT)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5
    return v[free]


def lambda_max(apply_K: Callable, diag: np.ndarray, v0: np.ndarray, n_iter: int,
               floor: float = 1e-6) -> float:
    """Power iteration on D^{-1} K (Sec. "Spectral-radius estimation")."""
    v = v0 / np.linalg.norm(v0)
    for _ in range(n_iter):
        w = apply_K(v) / diag
        nw = float(np.linalg.norm(w))
        if not (np.isfinite(nw) and nw > 0.0):
            return floor      # a vanishing or non-finite iterate: use the floor
        v = w / nw
    lam = float(v @ apply_K(v)) / float(v @ (diag * v))
    return lam if (np.isfinite(lam) and lam > floor) else floor


class CholeskyFailure(RuntimeError):
    pass


def coarse_factor(Kff_dense: np.ndarray) -> tuple[np.ndarray, float]:
    """Lower Cholesky factor of K^L_ff + eps I, eps = max(mean(diag) 1e-8, 1e-14)."""
    A = np.array(Kff_dense, dtype=np.float64)
    eps = max(float(np.mean(np.diag(A))) * 1e-8, 1e-14) if A.size else 1e-14
    A[np.diag_indices_from(A)] += eps
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError as exc:
        raise CholeskyFailure(str(exc)) from exc
    if not np.all(np.isfinite(L)):
        raise CholeskyFailure("non-finite factor")
    return L, eps


def coarse_solve(L: np.ndarray, r: np.ndarray) -> np.ndarray:
    import scipy.linalg as sla
    y = sla.solve_triangular(L, r, lower=True, check_finite=False)
    return sla.solve_triangular(L.T, y, lower=False, check_finite=False)


def coarse_pcg(apply_K: Callable, diag: np.ndarray, b: np.ndarray, steps: int) -> np.ndarray:
    """Fixed-count Jacobi-preconditioned CG from x = 0 (the coarsest solve above
    the dense-Cholesky cutoff): `steps` updates x += alpha p, r -= alpha q, each
    followed by z = D^{-1} r, beta = r.z / r_old.z_old, p = z + beta p."""
    x = np.zeros_like(b)
    r = np.array(b, dtype=np.float64)
    z = r / diag
    p = z.copy()
    rz = float(r @ z)
    for _ in range(steps):
        if rz == 0.0:
            break
        q = apply_K(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = r / diag
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def coarsest_solve(lev, r: np.ndarray) -> np.ndarray:
    """The coarsest-level solve of Eq. vcycle: Cholesky when the level has a
    factor, else the fixed-count PCG."""
    if lev.L is not None:
        return coarse_solve(lev.L, r)
    return coarse_pcg(lev.apply, lev.diag, r, lev.coarse_steps)


@dataclasses.dataclass
class Level:
    dims: tuple
    fixed: np.ndarray           # uint8 per DOF of the level grid
    free: np.ndarray            # free DOF indices
    K: sp.csr_matrix | None     # free x free (None when the fine level is matrix-free)
    apply: Callable             # free vector -> free vector
    diag: np.ndarray            # diag(K_ff)
    lam: float = 0.0            # lambda_max(D^{-1} K)
    P: sp.csr_matrix | None = None   # free_f x free_c transfer to the next level
    L: np.ndarray | None = None      # Cholesky factor (coarsest only, at most chol_cutoff free DOFs)
    eps: float = 0.0
    coarse_steps: int = 0            # fixed-count PCG steps (coarsest only, above the cutoff)

    @property
    def n_free(self) -> int:
        return int(self.free.size)


def auto_levels(dims, fixed0: np.ndarray, chol_cutoff: int = 5000) -> int:
    dims = tuple(dims)
    fixed = fixed0
    n = 1
    while int((fixed == 0).sum()) > chol_cutoff and min(dims) >= 2:
        fixed = inject_fixed(dims, fixed)
        dims = coarse_dims(dims)
        n += 1
    return n


def build_hierarchy(dims, E: np.ndarray, fixed0: np.ndarray, nu: float = 0.3,
                    levels: int = 0, chol_cutoff: int = 5000, power_fine: int = 20,
                    power_coarse: int = 10, matrix_free_fine: bool = False,
                    Ke: np.ndarray | None = None, coarse_pcg_steps: int = 80) -> list[Level]:
    """All levels: fine K (assembled, or matrix-free), Galerkin coarse operators,
    diagonals, lambda_max estimates and the coarsest solve: the Cholesky factor
    up to chol_cutoff free DOFs, else coarse_pcg_steps of Jacobi-PCG."""
    from .fem import element_stiffness

    if Ke is None:
        Ke = element_stiffness(nu)
    dims = tuple(int(d) for d in dims)
    if levels <= 0:
        levels = auto_levels(dims, fixed0, chol_cutoff)
    g0 = Grid(*dims)
    free0 = free_dofs(fixed0)
    if matrix_free_fine:
        edofs = g0.element_dofs()

        def apply0(v, _free=free0, _n=g0.n_dof):
            full = np.zeros(_n)
            full[_free] = v
            return matfree_apply(g0, E, Ke, full, edofs)[_free]

        diag_full = np.bincount(edofs.reshape(-1),
                                weights=(E[:, None] * np.diag(Ke)[None, :]).reshape(-1),
                                minlength=g0.n_dof)
        K0 = None
        diag0 = diag_full[free0]
    else:
        K0 = assemble(g0, E, Ke)[free0][:, free0].tocsr()
        apply0 = K0.dot
        diag0 = K0.diagonal()
    H = [Level(dims, np.asarray(fixed0), free0, K0, apply0, diag0)]
    for _ in range(1, levels):
        f = H[-1]
        cdims = coarse_dims(f.dims)
        cfixed = inject_fixed(f.dims, f.fixed)
        cfree = free_dofs(cfixed)
        P = prolongation(f.dims)[f.free][:, cfree].tocsr()
        if f.K is not None:
            Kc = galerkin(f.K, P)
        else:
            Kc = level1_elementwise(f.dims, E, Ke, f.fixed, cfixed)
        f.P = P
        H.append(Level(cdims, cfixed, cfree, Kc, Kc.dot, Kc.diagonal()))
    for li, lev in enumerate(H):
        v0 = power_start_vector(3 * Grid(*lev.dims).n_nodes, lev.free)
        lev.lam = lambda_max(lev.apply, lev.diag, v0, power_fine if li == 0 else power_coarse)
    last = H[-1]
    if last.n_free > chol_cutoff:
        last.coarse_steps = int(coarse_pcg_steps)
        return H
    dense = last.K.toarray() if last.K is not None else np.column_stack(
        [last.apply(e) for e in np.eye(last.n_free)])
    last.L, last.eps = coarse_factor(dense)
    return H
