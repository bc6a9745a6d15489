"""Pins for the oracle's finite-element pieces (CPU only).

Each check ties the oracle to something other than itself: exact symbolic
integration of the continuum strain energy of polynomial fields, rigid-body
modes, the FEM patch test, closed-form energies of linear fields, the SIMP law
at its end points, and the paper's free-DOF counts.
"""

import itertools
from fractions import Fraction

import numpy as np
import pytest
import sympy as sym

from oracle import fem
from paper_2604_26441_b300 import inputs

X, Y, Z = sym.symbols("x y z")
MONOMIALS = [sym.Integer(1), X, Y, Z, X * Y, Y * Z, X * Z, X * Y * Z]


def _poly_integral_unit_cube(expr):
    """Exact integral over [0,1]^3 of a polynomial: sum c x^a y^b z^c -> c/((a+1)(b+1)(c+1))."""
    poly = sym.Poly(sym.expand(expr), X, Y, Z)
    tot = sym.Rational(0)
    for (a, b, c), coef in poly.terms():
        tot += coef / ((a + 1) * (b + 1) * (c + 1))
    return tot


def _exact_ke(nu):
    """K_e from the continuum bilinear form a(u, v) = int lam tr(eps u) tr(eps v) + 2 mu eps u : eps v,
    evaluated exactly on the 24 fields monomial * e_d, then mapped to nodal DOFs."""
    E = sym.Integer(1)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    fields = []
    for m in MONOMIALS:
        for d in range(3):
            u = [sym.Integer(0)] * 3
            u[d] = m
            grad = sym.Matrix(3, 3, lambda i, j: sym.diff(u[i], (X, Y, Z)[j]))
            fields.append((grad + grad.T) / 2)
    n = len(fields)
    A = sym.zeros(n, n)
    for p in range(n):
        for q in range(p, n):
            ep, eq = fields[p], fields[q]
            dens = lam * ep.trace() * eq.trace() + 2 * mu * sum(
                ep[i, j] * eq[i, j] for i in range(3) for j in range(3))
            A[p, q] = A[q, p] = _poly_integral_unit_cube(dens)
    V = sym.zeros(24, n)
    for a, (dx, dy, dz) in enumerate(fem.LOCAL_NODES.tolist()):
        for mi, m in enumerate(MONOMIALS):
            val = m.subs({X: dx, Y: dy, Z: dz})
            for d in range(3):
                V[3 * a + d, 3 * mi + d] = val
    Vinv = V.inv()
    return Vinv.T * A * Vinv


@pytest.fixture(scope="module")
def ke_exact():
    return np.array(_exact_ke(sym.Rational(3, 10)).evalf(30), dtype=np.float64)


def test_ke_matches_exact_continuum_energy(ke_exact):
    Ke = fem.element_stiffness(0.3)
    assert np.max(np.abs(Ke - ke_exact)) < 1e-14


def test_ke_other_poisson_ratio():
    ex = np.array(_exact_ke(sym.Rational(1, 4)).evalf(30), dtype=np.float64)
    assert np.max(np.abs(fem.element_stiffness(0.25) - ex)) < 1e-14


def test_ke_quadrature_exact():
    assert np.max(np.abs(fem.element_stiffness(0.3, 2) - fem.element_stiffness(0.3, 3))) < 1e-15


def test_ke_symmetric_psd_rank18():
    Ke = fem.element_stiffness(0.3)
    assert np.array_equal(Ke, Ke.T) or np.max(np.abs(Ke - Ke.T)) < 1e-16
    ev = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(ev) < 1e-12) == 6
    assert ev.min() > -1e-12


def _rigid_modes(coords):
    """(3*n, 6) translations and linearised rotations evaluated at node coordinates."""
    n = coords.shape[0]
    R = np.zeros((3 * n, 6))
    for d in range(3):
        R[d::3, d] = 1.0
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    R[0::3, 3], R[1::3, 3] = -y, x
    R[1::3, 4], R[2::3, 4] = -z, y
    R[0::3, 5], R[2::3, 5] = z, -x
    return R


def test_ke_null_space_is_rigid_body_modes():
    Ke = fem.element_stiffness(0.3)
    R = _rigid_modes(fem.LOCAL_NODES.astype(float))
    assert np.max(np.abs(Ke @ R)) < 1e-14
    # the null space is exactly their span
    _, s, vt = np.linalg.svd(Ke)
    null = vt[s < 1e-12].T
    proj = R @ np.linalg.lstsq(R, null, rcond=None)[0]
    assert np.max(np.abs(proj - null)) < 1e-12


def test_ke_integer_structure_nu03():
    """For nu = 0.3 the unit-cube K_e is (5/1872) times an integer matrix."""
    Ke = fem.element_stiffness(0.3)
    S = Ke * 1872 / 5
    assert np.max(np.abs(S - np.round(S))) < 1e-12
    assert np.max(np.abs(np.round(S))) == 88


@pytest.mark.parametrize("strain", list(itertools.product([0, 1], repeat=6))[1:12])
def test_patch_energy_constant_strain(strain):
    """u = eps x (symmetric eps): u^T K_e u = eps : C : eps on the unit cube."""
    nu = 0.3
    lam, mu = fem.lame(1.0, nu)
    e = np.zeros((3, 3))
    e[0, 0], e[1, 1], e[2, 2] = strain[0], strain[1], strain[2]
    e[1, 2] = e[2, 1] = 0.5 * strain[3]
    e[0, 2] = e[2, 0] = 0.25 * strain[4]
    e[0, 1] = e[1, 0] = 0.75 * strain[5]
    u = (fem.LOCAL_NODES.astype(float) @ e.T).reshape(-1)
    exact = lam * np.trace(e) ** 2 + 2 * mu * np.sum(e * e)
    assert abs(u @ fem.element_stiffness(nu) @ u - exact) < 1e-13


def test_moduli_endpoints():
    rho = np.array([0.0, 1.0, 0.5], dtype=np.float32)
    E = fem.moduli(rho, 3.0, E0=2.0, Emin=1e-9)
    assert E[0] == 1e-9 and E[1] == 2.0
    assert abs(E[2] - (1e-9 + (2.0 - 1e-9) * 0.125)) < 1e-16
    assert np.allclose(fem.moduli(rho, 1.0, 1.0, 0.0), rho.astype(np.float64), rtol=0, atol=0)


def test_global_patch_test_interior_equilibrium():
    """Uniform E, linear displacement field: K u = 0 at every interior node."""
    g = fem.Grid(4, 3, 3)
    Ke = fem.element_stiffness(0.3)
    K = fem.assemble(g, np.full(g.n_elem, 1.7), Ke)
    i, j, k = g.node_ijk()
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 3))
    u = (np.stack([i, j, k], 1) @ A.T + rng.normal(size=3)).reshape(-1)
    y = (K @ u).reshape(-1, 3)
    interior = (i > 0) & (i < 4) & (j > 0) & (j < 3) & (k > 0) & (k < 3)
    assert np.max(np.abs(y[interior])) < 1e-12
    # and the total energy is volume * E * eps:C:eps
    lam, mu = fem.lame(1.7, 0.3)
    e = 0.5 * (A + A.T)
    assert abs(u @ K @ u - g.n_elem * (lam * np.trace(e) ** 2 + 2 * mu * np.sum(e * e))) < 1e-9


def test_global_rigid_modes_and_translation_sum():
    g = fem.Grid(3, 2, 2)
    rng = np.random.default_rng(1)
    E = rng.uniform(0.1, 2.0, g.n_elem)
    K = fem.assemble(g, E, fem.element_stiffness(0.3))
    i, j, k = g.node_ijk()
    R = _rigid_modes(np.stack([i, j, k], 1).astype(float))
    assert np.max(np.abs(K @ R)) < 1e-13
    assert np.max(np.abs(K - K.T)) < 1e-15


def test_matfree_equals_assembled_and_sampled_rows():
    g = fem.Grid(5, 3, 4)
    rng = np.random.default_rng(2)
    E = rng.uniform(0.01, 1.0, g.n_elem)
    Ke = fem.element_stiffness(0.3)
    u = rng.normal(size=g.n_dof)
    y_a = fem.assemble(g, E, Ke) @ u
    y_m = fem.matfree_apply(g, E, Ke, u)
    assert np.max(np.abs(y_a - y_m)) < 1e-13
    nodes = np.array([0, 7, 23, g.n_nodes - 1, 40])
    y_s = fem.matfree_apply_at_nodes(g, E, Ke, u, nodes)
    assert np.max(np.abs(y_s - y_m.reshape(-1, 3)[nodes])) < 1e-13


def test_kff_spd_config0():
    c = inputs.CONFIGS["c0"]
    g = fem.Grid(c.nx, c.ny, c.nz)
    E = fem.moduli(c.rho(), c.p)
    free = fem.free_dofs(c.fixed())
    K = fem.assemble(g, E, fem.element_stiffness(0.3))[free][:, free].toarray()
    assert free.size == 3888
    np.linalg.cholesky(K)
    assert np.linalg.eigvalsh(K)[0] > 0


def test_free_dof_counts_match_paper(golden):
    for case in golden["free_dof_counts"]["cases"]:
        nx, ny, nz = case["dims"]
        fixed = inputs.clamp_xmin_mask(nx, ny, nz)
        assert int((fixed == 0).sum()) == case["n_free"]
