"""CPU check of the formulation the matrix-free level-1 kernels rely on.

For even fine sizes the level-1 Galerkin operator of Eq. galerkin_level1 is,
per coarse element, sum_k E_k P_k^T K_e P_k over its 8 children.  In the
Walsh-Hadamard mode basis of the coarse corners the children are reflections
of child 0, so the element matrix is G0_ij * Ehat[pi_i xor pi_j], with G0 the
child-0 contribution, pi the parity of a mode and Ehat the 8-point Hadamard
transform of the children's moduli.  The tests check that formula against the
oracle's element-wise assembly (clamped cantilevers, where every fixed fine
DOF has fixed prolongation parents), that G0 has the same 279 non-zero
positions for every Poisson ratio, and that a point constraint on an odd fine
node (whose parents stay free) breaks the equality, which is why set-up keeps
the assembled operator there.
"""

import numpy as np
import pytest

from oracle import fem, hierarchy as hy
from paper_2604_26441_b300 import inputs


def _hadamard():
    s = 2 * fem.LOCAL_NODES - 1
    H = np.zeros((8, 8))
    for m in range(8):
        for a in range(8):
            H[m, a] = np.prod([s[a, k] for k in range(3) if (m >> k) & 1])
    return np.kron(H, np.eye(3))


def _child0_modes(nu):
    """G0 = H P_0^T K_e P_0 H^T / 64 (rows and columns 3 m + c)."""
    w0 = np.array([[1.0, 0.0], [0.5, 0.5]])
    P = np.zeros((8, 8))
    for a, (ax, ay, az) in enumerate(fem.LOCAL_NODES):
        for b, (bx, by, bz) in enumerate(fem.LOCAL_NODES):
            P[a, b] = w0[ax, bx] * w0[ay, by] * w0[az, bz]
    P3 = np.kron(P, np.eye(3))
    H3 = _hadamard()
    return H3 @ (P3.T @ fem.element_stiffness(nu) @ P3) @ H3.T / 64


def _parity(i):
    m, c = divmod(i, 3)
    return m ^ (1 << c)


def _structured_apply(dims_f, E, u_c, G0):
    nx, ny, nz = (d // 2 for d in dims_f)
    gc = fem.Grid(nx, ny, nz)
    H3 = _hadamard()
    Ef = E.reshape(dims_f[2], dims_f[1], dims_f[0])
    delta = np.array([[_parity(i) ^ _parity(j) for j in range(24)] for i in range(24)])
    sign = np.array([[(-1) ** bin(k & d).count("1") for k in range(8)] for d in range(8)])
    y = np.zeros(gc.n_dof)
    for K in range(nz):
        for J in range(ny):
            for I in range(nx):
                nodes = [gc.node(I + bx, J + by, K + bz) for (bx, by, bz) in fem.LOCAL_NODES]
                dofs = np.array([3 * n + c for n in nodes for c in range(3)])
                Ek = np.array([Ef[2 * K + (k >> 2 & 1), 2 * J + (k >> 1 & 1), 2 * I + (k & 1)] for k in range(8)])
                Eh = sign @ Ek
                y[dofs] += H3.T @ ((G0 * Eh[delta]) @ (H3 @ u_c[dofs]))
    return y


@pytest.mark.parametrize("dims", [(4, 4, 2), (6, 4, 4), (8, 6, 4)])
def test_structured_level1_equals_elementwise_assembly(dims):
    nx, ny, nz = dims
    rho = inputs.filtered_random_density(nx, ny, nz, 3)
    E = fem.moduli(rho, 3.0).reshape(-1)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    fixed_c = hy.inject_fixed(dims, fixed)
    K1 = hy.level1_elementwise(dims, E, fem.element_stiffness(0.3), fixed, fixed_c)
    fc = fem.free_dofs(fixed_c)
    u = np.zeros(fixed_c.size)
    u[fc] = np.random.default_rng(1).standard_normal(fc.size)
    y = _structured_apply(dims, E, u, _child0_modes(0.3))
    ref = K1 @ u[fc]
    assert np.max(np.abs(y[fc] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_child_terms_are_reflections_of_child0():
    """H P_k^T K_e P_k H^T / 64 = D_k G0 D_k with D_k = (-1)^{k . pi}."""
    H3 = _hadamard()
    Ke = fem.element_stiffness(0.3)
    G0 = _child0_modes(0.3)
    for k in range(8):
        w = {0: np.array([[1.0, 0.0], [0.5, 0.5]]), 1: np.array([[0.5, 0.5], [0.0, 1.0]])}
        pos = (k & 1, k >> 1 & 1, k >> 2 & 1)
        P = np.zeros((8, 8))
        for a, (ax, ay, az) in enumerate(fem.LOCAL_NODES):
            for b, (bx, by, bz) in enumerate(fem.LOCAL_NODES):
                P[a, b] = w[pos[0]][ax, bx] * w[pos[1]][ay, by] * w[pos[2]][az, bz]
        P3 = np.kron(P, np.eye(3))
        Gk = H3 @ (P3.T @ Ke @ P3) @ H3.T / 64
        d = np.array([(-1) ** bin(k & _parity(i)).count("1") for i in range(24)])
        assert np.max(np.abs(Gk - d[:, None] * G0 * d[None, :])) < 1e-14


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.25, 0.3, 0.45, 0.49])
def test_child0_pattern_has_279_fixed_entries(nu):
    G0 = _child0_modes(nu)
    ref = np.abs(_child0_modes(0.37)) > 1e-12 * np.max(np.abs(_child0_modes(0.37)))
    nz = np.abs(G0) > 1e-12 * np.max(np.abs(G0))
    assert ref.sum() == 279
    assert not np.any(nz & ~ref)               # no entry off the pattern
    assert nu == 0.0 or np.array_equal(nz, ref)  # and all of it in use
    assert not np.any(ref[0:3]) and not np.any(ref[:, 0:3])  # constant modes carry nothing


def test_point_constraint_on_an_odd_node_breaks_the_equality():
    dims = (4, 4, 2)
    nx, ny, nz = dims
    rho = inputs.filtered_random_density(nx, ny, nz, 3)
    E = fem.moduli(rho, 3.0).reshape(-1)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz).reshape(nz + 1, ny + 1, nx + 1, 3).copy()
    fixed[1, 1, 3, 2] = 1  # an odd node: its coarse parents stay free
    fixed = fixed.reshape(-1)
    fixed_c = hy.inject_fixed(dims, fixed)
    K1 = hy.level1_elementwise(dims, E, fem.element_stiffness(0.3), fixed, fixed_c)
    fc = fem.free_dofs(fixed_c)
    u = np.zeros(fixed_c.size)
    u[fc] = np.random.default_rng(2).standard_normal(fc.size)
    y = _structured_apply(dims, E, u, _child0_modes(0.3))
    ref = K1 @ u[fc]
    assert np.max(np.abs(y[fc] - ref)) > 1e-3 * np.max(np.abs(ref))
