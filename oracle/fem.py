"""Oracle: hex8 finite-element pieces (TEST INFRASTRUCTURE ONLY; FP64 throughout).

Paper passages followed:

* Sec. "Problem Setup", Eq. simp_filter -- E_e = Emin + (E0 - Emin) rho_e^p;
* Sec. "Problem Setup", Eq. state_eq -- K = sum_e E_e K_e with K_e the 24x24
  unit trilinear-hexahedron stiffness, nu = 0.3, free-DOF system K_ff u_f = f_f;
* Sec. "Transfer Operators and Boundary Masking", Eq. mf_matvec -- the fine
  operator is the action of sum_e E_e K_e without assembling it.

Numbering (a reading; the paper is silent): local node a of an element sits at
offset LOCAL_NODES[a] = (dx, dy, dz); local DOF 3a + c; global node
n = i + (nx+1)(j + (ny+1)k); global DOF 3n + c; element e = ex + nx(ey + ny ez).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

LOCAL_NODES = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def lame(E: float, nu: float) -> tuple[float, float]:
    """Lame constants of isotropic linear elasticity."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_matrix(nu: float, E: float = 1.0) -> np.ndarray:
    """6x6 Voigt matrix for strains (exx, eyy, ezz, gyz, gxz, gxy), engineering shears."""
    lam, mu = lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] += 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def shape_gradients(xi: np.ndarray) -> np.ndarray:
    """(8, 3) gradients of the trilinear shape functions on the unit cube at xi."""
    g = np.zeros((8, 3))
    for a, node in enumerate(LOCAL_NODES):
        f = [xi[k] if node[k] else 1.0 - xi[k] for k in range(3)]
        s = [1.0 if node[k] else -1.0 for k in range(3)]
        g[a, 0] = s[0] * f[1] * f[2]
        g[a, 1] = f[0] * s[1] * f[2]
        g[a, 2] = f[0] * f[1] * s[2]
    return g


def b_matrix(xi: np.ndarray) -> np.ndarray:
    """6x24 strain-displacement matrix at xi (Voigt order as elasticity_matrix)."""
    g = shape_gradients(xi)
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = g[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 1] = gz
        B[3, 3 * a + 2] = gy
        B[4, 3 * a + 0] = gz
        B[4, 3 * a + 2] = gx
        B[5, 3 * a + 0] = gy
        B[5, 3 * a + 1] = gx
    return B


def element_stiffness(nu: float = 0.3, npts: int = 2) -> np.ndarray:
    """K_e = integral over [0,1]^3 of B^T C B (E = 1), tensor Gauss-Legendre rule.

    The integrand is at most quadratic in each coordinate, so npts = 2 is exact.
    """
    C = elasticity_matrix(nu)
    pts, wts = np.polynomial.legendre.leggauss(npts)
    x = 0.5 * (pts + 1.0)
    w = 0.5 * wts
    Ke = np.zeros((24, 24))
    for i in range(npts):
        for j in range(npts):
            for k in range(npts):
                B = b_matrix(np.array([x[i], x[j], x[k]]))
                Ke += w[i] * w[j] * w[k] * (B.T @ C @ B)
    return Ke


def moduli(rho: np.ndarray, p: float, E0: float = 1.0, Emin: float = 1e-9) -> np.ndarray:
    """Eq. simp_filter on the float32 densities, evaluated in FP64; flat [n_elem]."""
    r = np.asarray(rho, dtype=np.float32).astype(np.float64).reshape(-1)
    return Emin + (E0 - Emin) * r ** p


class Grid:
    """Structured nx x ny x nz grid of unit hex8 elements."""

    def __init__(self, nx: int, ny: int, nz: int):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)

    @property
    def dims(self) -> tuple[int, int, int]:
        return self.nx, self.ny, self.nz

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node_ijk(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Node coordinates (i, j, k) in node order."""
        k, j, i = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1),
                              np.arange(self.nx + 1), indexing="ij")
        return i.reshape(-1), j.reshape(-1), k.reshape(-1)

    def element_nodes(self) -> np.ndarray:
        """(n_elem, 8) global node ids in LOCAL_NODES order, elements in e order."""
        ez, ey, ex = np.meshgrid(np.arange(self.nz), np.arange(self.ny),
                                 np.arange(self.nx), indexing="ij")
        ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
        out = np.empty((ex.size, 8), dtype=np.int64)
        for a, (dx, dy, dz) in enumerate(LOCAL_NODES):
            out[:, a] = self.node(ex + dx, ey + dy, ez + dz)
        return out

    def element_dofs(self) -> np.ndarray:
        """(n_elem, 24) global DOF ids, local DOF 3a + c."""
        en = self.element_nodes()
        return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(en.shape[0], 24)


def assemble(grid: Grid, E: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """Global K = sum_e E_e K_e on all DOFs (duplicates summed), Eq. state_eq."""
    dofs = grid.element_dofs()
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    vals = (E[:, None, None] * Ke[None, :, :]).reshape(-1)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(grid.n_dof, grid.n_dof)).tocsr()
    K.sum_duplicates()
    return K


def matfree_apply(grid: Grid, E: np.ndarray, Ke: np.ndarray, u: np.ndarray,
                  dofs: np.ndarray | None = None) -> np.ndarray:
    """y = (sum_e E_e K_e) u on all DOFs by gather / element product / scatter-sum
    (Eq. mf_matvec); no masking."""
    if dofs is None:
        dofs = grid.element_dofs()
    U = np.asarray(u, dtype=np.float64)[dofs]
    F = (U @ Ke.T) * E[:, None]
    return np.bincount(dofs.reshape(-1), weights=F.reshape(-1), minlength=grid.n_dof)


def matfree_apply_at_nodes(grid: Grid, E: np.ndarray, Ke: np.ndarray, u: np.ndarray,
                           nodes: np.ndarray) -> np.ndarray:
    """(len(nodes), 3) rows of (sum_e E_e K_e) u at the given nodes only: for each
    node, the sum over its (up to 8) elements of E_e times the node's three rows
    of K_e applied to the element's displacements.  Used for sampled parity at
    sizes where the full operator is too slow for a test."""
    u = np.asarray(u, dtype=np.float64)
    nx, ny, nz = grid.dims
    out = np.zeros((len(nodes), 3))
    i = nodes % (nx + 1)
    j = (nodes // (nx + 1)) % (ny + 1)
    k = nodes // ((nx + 1) * (ny + 1))
    for a, (dx, dy, dz) in enumerate(LOCAL_NODES):
        ex, ey, ez = i - dx, j - dy, k - dz
        ok = (ex >= 0) & (ex < nx) & (ey >= 0) & (ey < ny) & (ez >= 0) & (ez < nz)
        if not ok.any():
            continue
        e = ex[ok] + nx * (ey[ok] + ny * ez[ok])
        Ue = np.zeros((ok.sum(), 24))
        for b, (bx, by, bz) in enumerate(LOCAL_NODES):
            m = grid.node(ex[ok] + bx, ey[ok] + by, ez[ok] + bz)
            Ue[:, 3 * b:3 * b + 3] = u.reshape(-1, 3)[m]
        out[ok] += E[e][:, None] * (Ue @ Ke[3 * a:3 * a + 3, :].T)
    return out


def free_dofs(fixed: np.ndarray) -> np.ndarray:
    """Indices of free DOFs (fixed flag 0), ascending."""
    return np.flatnonzero(np.asarray(fixed) == 0)
