"""Pins for the oracle's multigrid hierarchy (CPU only).

Transfer operators are pinned against hand-written matrices from the paper's
weight rule and against brute-force dense construction; Galerkin operators
against brute-force dense P^T K P on tiny grids and against the element-wise
level-1 formula; the spectral estimate against a dense eigensolver; the
hierarchy sizes against the counts the paper prints.
"""

import numpy as np
import pytest

from oracle import fem, hierarchy as hy
from paper_2604_26441_b300 import inputs


def test_prolongation_1d_hand_written():
    # even fine index injects, odd splits 1/2-1/2 (Eq. trilinear_weights)
    P4 = hy.prolongation_1d(4).toarray()
    assert np.array_equal(P4, np.array([[1, 0, 0], [.5, .5, 0], [0, 1, 0], [0, .5, .5], [0, 0, 1]]))
    # odd count: floor coarsening, the last odd node clamps to the last coarse node
    P5 = hy.prolongation_1d(5).toarray()
    assert np.array_equal(P5, np.array([[1, 0, 0], [.5, .5, 0], [0, 1, 0], [0, .5, .5],
                                        [0, 0, 1], [0, 0, 1]]))
    P3 = hy.prolongation_1d(3).toarray()
    assert np.array_equal(P3, np.array([[1, 0], [.5, .5], [0, 1], [0, 1]]))


def _brute_force_P(dims):
    """Dense vector prolongation built node pair by node pair from the 1D rule."""
    def w1(f, c, nf):
        nc = nf // 2
        if f % 2 == 0:
            return 1.0 if c == f // 2 else 0.0
        if f < 2 * nc:
            return 0.5 if c in ((f - 1) // 2, (f + 1) // 2) else 0.0
        return 1.0 if c == nc else 0.0
    gf, gc = fem.Grid(*dims), fem.Grid(*hy.coarse_dims(dims))
    P = np.zeros((gf.n_dof, gc.n_dof))
    for k in range(gf.nz + 1):
        for j in range(gf.ny + 1):
            for i in range(gf.nx + 1):
                for K in range(gc.nz + 1):
                    for J in range(gc.ny + 1):
                        for I in range(gc.nx + 1):
                            w = w1(i, I, gf.nx) * w1(j, J, gf.ny) * w1(k, K, gf.nz)
                            if w:
                                for c in range(3):
                                    P[3 * gf.node(i, j, k) + c, 3 * gc.node(I, J, K) + c] = w
    return P


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 2, 2), (5, 3, 3), (4, 5, 3)])
def test_prolongation_matches_brute_force(dims):
    assert np.array_equal(hy.prolongation(dims).toarray(), _brute_force_P(dims))


@pytest.mark.parametrize("dims", [(4, 4, 2), (5, 3, 7)])
def test_prolongation_partition_of_unity_and_linear_fields(dims):
    Ps = hy.scalar_prolongation(dims)
    assert np.allclose(np.asarray(Ps.sum(axis=1)).ravel(), 1.0, atol=0)
    gf, gc = fem.Grid(*dims), fem.Grid(*hy.coarse_dims(dims))
    I, J, K = gc.node_ijk()
    i, j, k = gf.node_ijk()
    # a coarse linear field (coarse spacing 2) interpolates to the fine linear field
    # wherever the odd-end clamp is not involved
    lin_c = 2.0 * I + 3.0 * J - 1.0 * K
    lin_f = i + 1.5 * j - 0.5 * k
    ok = np.ones_like(i, dtype=bool)
    for idx, n in zip((i, j, k), dims):
        if n % 2 == 1:
            ok &= idx < n
    assert np.max(np.abs((Ps @ lin_c - lin_f)[ok])) < 1e-14
    # injection: even fine nodes copy their coarse node
    even = (i % 2 == 0) & (j % 2 == 0) & (k % 2 == 0)
    assert np.array_equal((Ps @ lin_c)[even], lin_c[gc.node(i[even] // 2, j[even] // 2, k[even] // 2)])


def test_injection_keeps_clamped_face():
    dims = (6, 4, 4)
    fixed = inputs.clamp_xmin_mask(*dims)
    fc = hy.inject_fixed(dims, fixed)
    assert np.array_equal(fc, inputs.clamp_xmin_mask(3, 2, 2))


def test_injection_point_constraint_on_odd_node_does_not_propagate():
    dims = (4, 4, 4)
    g = fem.Grid(*dims)
    fixed = np.zeros(g.n_dof, dtype=np.uint8)
    fixed[3 * g.node(1, 2, 2) + 1] = 1     # odd x index: no coarse node injects there
    fixed[3 * g.node(2, 2, 2) + 2] = 1     # even node: inherited by coarse node (1,1,1)
    fc = hy.inject_fixed(dims, fixed)
    gc = fem.Grid(2, 2, 2)
    expect = np.zeros(gc.n_dof, dtype=np.uint8)
    expect[3 * gc.node(1, 1, 1) + 2] = 1
    assert np.array_equal(fc, expect)


def test_level_sizes_match_paper(golden):
    g1 = golden["level1_free_216k"]
    dims = tuple(g1["dims"])
    f1 = hy.inject_fixed(dims, inputs.clamp_xmin_mask(*dims))
    n1 = int((f1 == 0).sum())
    assert abs(n1 - g1["approx"]) / g1["approx"] < g1["rel_tol"]
    gL = golden["coarsest_free_216k_4level"]
    f, d = inputs.clamp_xmin_mask(*dims), dims
    for _ in range(gL["levels"] - 1):
        f = hy.inject_fixed(d, f)
        d = hy.coarse_dims(d)
    nL = int((f == 0).sum())
    assert abs(nL - gL["approx"]) / gL["approx"] < gL["rel_tol"]


def _random_mask(g, rng, p=0.1):
    fixed = inputs.clamp_xmin_mask(*g.dims)
    extra = rng.random(g.n_dof) < p
    fixed = fixed | extra.astype(np.uint8)
    return fixed


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 2, 2), (4, 4, 4), (5, 3, 3), (6, 5, 3)])
@pytest.mark.parametrize("mask", ["clamp", "random"])
def test_galerkin_brute_force_and_elementwise(dims, mask):
    rng = np.random.default_rng(sum(dims))
    g = fem.Grid(*dims)
    E = rng.uniform(0.05, 1.0, g.n_elem)
    Ke = fem.element_stiffness(0.3)
    fixed = inputs.clamp_xmin_mask(*dims) if mask == "clamp" else _random_mask(g, rng)
    fixed_c = hy.inject_fixed(dims, fixed)
    ff, fc = fem.free_dofs(fixed), fem.free_dofs(fixed_c)
    Kd = fem.assemble(g, E, Ke).toarray()
    Pd = _brute_force_P(dims)
    brute = Pd[ff][:, fc].T @ Kd[ff][:, ff] @ Pd[ff][:, fc]
    Kff = fem.assemble(g, E, Ke)[ff][:, ff].tocsr()
    Pff = hy.prolongation(dims)[ff][:, fc].tocsr()
    K1 = hy.galerkin(Kff, Pff).toarray()
    K1e = hy.level1_elementwise(dims, E, Ke, fixed, fixed_c).toarray()
    scale = np.abs(brute).max()
    assert np.max(np.abs(K1 - brute)) < 1e-14 * scale
    assert np.max(np.abs(K1e - brute)) < 1e-14 * scale
    # energy identity v^T K1 v = (P v)^T K (P v), symmetric, SPD
    v = rng.normal(size=fc.size)
    assert abs(v @ K1 @ v - (Pff @ v) @ (Kff @ (Pff @ v))) < 1e-12 * abs(v @ K1 @ v)
    assert np.max(np.abs(K1 - K1.T)) < 1e-15 * scale
    if fc.size:
        assert np.linalg.eigvalsh(K1)[0] > 0


def test_galerkin_pattern_is_27_point_block_stencil():
    dims = (6, 4, 4)
    g = fem.Grid(*dims)
    E = np.random.default_rng(3).uniform(0.1, 1, g.n_elem)
    fixed = inputs.clamp_xmin_mask(*dims)
    H = hy.build_hierarchy(dims, E, fixed, levels=3)
    for lev in H[1:]:
        gc = fem.Grid(*lev.dims)
        A = lev.K.tocoo()
        nr, nc_ = lev.free[A.row] // 3, lev.free[A.col] // 3
        i1, j1, k1 = nr % (gc.nx + 1), (nr // (gc.nx + 1)) % (gc.ny + 1), nr // ((gc.nx + 1) * (gc.ny + 1))
        i2, j2, k2 = nc_ % (gc.nx + 1), (nc_ // (gc.nx + 1)) % (gc.ny + 1), nc_ // ((gc.nx + 1) * (gc.ny + 1))
        assert max(np.abs(i1 - i2).max(), np.abs(j1 - j2).max(), np.abs(k1 - k2).max()) <= 1


def test_lambda_max_power_iteration_config0():
    """The estimate is a lower bound of the dense lambda_max(D^-1 K); 20 fine
    iterations land within 1 %, and the estimator converges to the dense value
    when run long enough on every level."""
    c = inputs.CONFIGS["c0"]
    E = fem.moduli(c.rho(), c.p)
    H = hy.build_hierarchy((c.nx, c.ny, c.nz), E, c.fixed(), levels=3)
    for li, lev in enumerate(H):
        K = lev.K.toarray()
        d = np.sqrt(lev.diag)
        lam_true = np.linalg.eigvalsh(K / np.outer(d, d))[-1]
        assert lev.lam <= lam_true * (1 + 1e-12)
        if li == 0:
            assert lev.lam > 0.99 * lam_true
        v0 = hy.power_start_vector(3 * fem.Grid(*lev.dims).n_nodes, lev.free)
        lam_long = hy.lambda_max(lev.apply, lev.diag, v0, 3000)
        assert abs(lam_long - lam_true) < 2e-3 * lam_true
        # damped Jacobi with omega = 0.6 is stable on every level of config 0
        assert 0.6 * lam_true < 2.0


def test_lambda_floor():
    lam = hy.lambda_max(lambda v: 0 * v, np.ones(4), np.ones(4), 3)
    assert lam == 1e-6


def test_coarse_regularisation_and_failure():
    A = np.diag([2.0, 4.0, 6.0])
    L, eps = hy.coarse_factor(A)
    assert eps == 4.0 * 1e-8
    assert np.allclose(L @ L.T, A + eps * np.eye(3), atol=1e-15)
    _, eps2 = hy.coarse_factor(np.diag([1e-9, 1e-9]))
    assert eps2 == 1e-14
    with pytest.raises(hy.CholeskyFailure):
        hy.coarse_factor(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_auto_levels():
    # coarsen while the coarsest free count exceeds the cutoff
    dims = (40, 40, 40)
    n = hy.auto_levels(dims, inputs.clamp_xmin_mask(*dims), 5000)
    f, d = inputs.clamp_xmin_mask(*dims), dims
    counts = [int((f == 0).sum())]
    for _ in range(n - 1):
        f = hy.inject_fixed(d, f)
        d = hy.coarse_dims(d)
        counts.append(int((f == 0).sum()))
    assert counts[-1] <= 5000 and counts[-2] > 5000


# ---------------------------------------------------------------------------
# coarsest solve above the dense-Cholesky cutoff: fixed-count Jacobi-PCG
# (Sec. "Matrix-Free V-Cycle"; the reproducibility defaults: 80 PCG steps)
# ---------------------------------------------------------------------------
def _small_level_operator():
    dims = (6, 3, 3)
    fixed = inputs.clamp_xmin_mask(*dims)
    rho = inputs.filtered_random_density(*dims, 5)
    g = fem.Grid(*dims)
    K = fem.assemble(g, fem.moduli(rho, 3.0), fem.element_stiffness(0.3))
    free = fem.free_dofs(fixed)
    return K[free][:, free].tocsr()


def test_coarse_pcg_matches_scipy_cg_iterates():
    """k steps of the oracle's fixed-count PCG equal scipy's preconditioned CG
    after k iterations (an independent implementation of the same Krylov
    iterate), for k below the system size; a wrong preconditioner (D instead of
    D^-1) or a wrong beta would break this."""
    import scipy.sparse.linalg as spla
    A = _small_level_operator()
    d = A.diagonal()
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    M = spla.LinearOperator(A.shape, matvec=lambda v: v / d)
    for k in (1, 3, 10, 25):
        x = hy.coarse_pcg(A.dot, d, b, k)
        xs, _ = spla.cg(A, b, x0=np.zeros_like(b), rtol=0.0, atol=0.0, maxiter=k, M=M)
        assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs), k


def test_coarse_pcg_with_enough_steps_is_the_exact_solve():
    """CG terminates in at most n steps: with steps >= n the fixed-count PCG
    reproduces the dense solution (rounding aside); its residual also falls
    monotonically in the energy norm as steps grow."""
    A = _small_level_operator()
    n = A.shape[0]
    d = A.diagonal()
    b = np.random.default_rng(4).standard_normal(n)
    x_exact = np.linalg.solve(A.toarray(), b)
    x = hy.coarse_pcg(A.dot, d, b, 3 * n)
    assert np.linalg.norm(x - x_exact) <= 1e-8 * np.linalg.norm(x_exact)
    errs = [float((xe := hy.coarse_pcg(A.dot, d, b, k) - x_exact) @ (A @ xe)) for k in (2, 8, 32)]
    assert errs[0] > errs[1] > errs[2]


def test_hierarchy_above_cutoff_uses_fixed_count_pcg():
    """A coarsest level with more free DOFs than the cutoff gets no Cholesky
    factor but the fixed-count PCG (80 steps by default); with a step count at
    least its size, the V-cycle equals the one with an exact coarsest solve (a
    Cholesky factor of K^L without the eps regularisation)."""
    from oracle import solver as so
    dims = (8, 4, 4)
    fixed = inputs.clamp_xmin_mask(*dims)
    E = fem.moduli(inputs.uniform_density(*dims), 3.0)
    H_chol = hy.build_hierarchy(dims, E, fixed, levels=2)
    H_chol[-1].L = np.linalg.cholesky(H_chol[-1].K.toarray())
    n_c = H_chol[-1].n_free
    H_pcg = hy.build_hierarchy(dims, E, fixed, levels=2, chol_cutoff=n_c - 1)
    assert H_pcg[-1].L is None and H_pcg[-1].coarse_steps == 80
    H_big = hy.build_hierarchy(dims, E, fixed, levels=2, chol_cutoff=n_c - 1, coarse_pcg_steps=3 * n_c)
    spec = so.SmootherSpec("jacobi", 2, 0.5)
    r = inputs.random_free_vector(fixed, seed=9)[H_chol[0].free]
    z_chol = so.vcycle(H_chol, r, spec)
    z_big = so.vcycle(H_big, r, spec)
    assert np.linalg.norm(z_big - z_chol) <= 1e-9 * np.linalg.norm(z_chol)
    z_80 = so.vcycle(H_pcg, r, spec)
    assert np.all(np.isfinite(z_80)) and np.linalg.norm(z_80 - z_chol) > 0.0
