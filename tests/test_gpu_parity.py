"""GPU parity of every step of the hot path against the FP64 CPU oracle.

Tolerances: the FP32 operator apply (fine and assembled levels), transfers and
smoother passes within 1e-6 relative L2 (FP32 arithmetic on O(1) data, ~600
terms per output); Galerkin operators bit-exact in pattern and within 1e-12
relative in value (both FP64); masks bit-exact; converged displacements within
1e-5 relative L2 of the oracle's exact solution with an FP64 true residual
below 1e-6; pass/fail under the cap identical and iteration counts within
max(2, 10 %) of the oracle's.
"""

import numpy as np
import pytest

from oracle import fem, hierarchy as hy, solver as so
from paper_2604_26441_b300 import inputs

from gpu_helpers import (config_opts, gpu_solver, oracle_hierarchy, oracle_spec_from_opts, pattern_planes,
                         planes_from_csr, rel_l2, slot_pattern_from_mask, structural_patterns)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_26441_b300 import build
    build.build_library()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


# ---------------------------------------------------------------------------
# fine operator
# ---------------------------------------------------------------------------
APPLY_CASES = [
    ("c0", 16, 8, 8, "uniform", 3.0),
    ("ragged", 37, 13, 9, "filtered", 3.0),
    ("thin", 33, 2, 5, "filtered", 1.0),
    ("c1", 40, 40, 40, "filtered", 2.0),
]


@pytest.mark.parametrize("name,nx,ny,nz,dens,p", APPLY_CASES)
def test_fine_apply_matches_oracle(name, nx, ny, nz, dens, p):
    rho = inputs.uniform_density(nx, ny, nz) if dens == "uniform" else inputs.filtered_random_density(nx, ny, nz, 7)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    S = gpu_solver(rho, p, levels=0, smoother="jacobi", coarse_smoother=None, omega=0.5)
    u = inputs.random_free_vector(fixed, seed=11)
    u_in = u.copy()
    u_in[fixed == 1] = 1e3  # values on fixed DOFs must be ignored
    y = S.apply(_t(u_in)).cpu().numpy()
    g = fem.Grid(nx, ny, nz)
    yref = fem.matfree_apply(g, fem.moduli(rho, p), fem.element_stiffness(0.3), u.astype(np.float64))
    yref[fixed == 1] = 0.0
    assert np.all(y[fixed == 1] == 0.0)
    assert rel_l2(y, yref) < 1e-6
    # bitwise reproducible (no atomics)
    y2 = S.apply(_t(u_in)).cpu().numpy()
    assert np.array_equal(y, y2)


def test_fine_apply_random_mask():
    nx, ny, nz = 12, 7, 5
    rng = np.random.default_rng(3)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz) | (rng.random(3 * (nx + 1) * (ny + 1) * (nz + 1)) < 0.1).astype(np.uint8)
    rho = inputs.filtered_random_density(nx, ny, nz, 5)
    S = gpu_solver(rho, 3.0, fixed=fixed, levels=2, smoother="jacobi", coarse_smoother=None, omega=0.4)
    u = inputs.random_free_vector(fixed, seed=2)
    y = S.apply(_t(u)).cpu().numpy()
    yref = fem.matfree_apply(fem.Grid(nx, ny, nz), fem.moduli(rho, 3.0), fem.element_stiffness(0.3),
                             u.astype(np.float64))
    yref[fixed == 1] = 0
    assert rel_l2(y, yref) < 1e-6


def test_fine_apply_full_size_sampled():
    """100^3 (the throughput configuration): sampled rows against the oracle."""
    c = inputs.CONFIGS["c2"]
    rho = inputs.filtered_random_density(c.nx, c.ny, c.nz, 3)
    S = gpu_solver(rho, 3.0, levels=0, smoother="jacobi", coarse_smoother=None, omega=0.5)
    fixed = c.fixed()
    u = inputs.random_free_vector(fixed, seed=4)
    y = S.apply(_t(u)).cpu().numpy().reshape(-1, 3)
    g = fem.Grid(c.nx, c.ny, c.nz)
    rng = np.random.default_rng(0)
    nodes = np.concatenate([rng.integers(0, g.n_nodes, 3000), [0, g.n_nodes - 1, c.nx, g.n_nodes // 2]])
    ref = fem.matfree_apply_at_nodes(g, fem.moduli(rho, 3.0), fem.element_stiffness(0.3), u, nodes)
    ref[fixed.reshape(-1, 3)[nodes] == 1] = 0
    assert rel_l2(y[nodes], ref) < 1e-6


# ---------------------------------------------------------------------------
# hierarchy: masks, Galerkin operators, spectral estimates
# ---------------------------------------------------------------------------
HIER_CASES = [
    ("c0", 16, 8, 8, 3, "clamp"),
    ("odd", 13, 7, 11, 3, "clamp"),
    ("random_mask", 10, 6, 6, 3, "random"),
    ("c1", 40, 40, 40, 4, "clamp"),
]


def _case_inputs(nx, ny, nz, mask):
    rho = inputs.filtered_random_density(nx, ny, nz, 9)
    if mask == "clamp":
        return rho, inputs.clamp_xmin_mask(nx, ny, nz), None
    rng = np.random.default_rng(1)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz) | (rng.random(3 * (nx + 1) * (ny + 1) * (nz + 1)) < 0.08).astype(np.uint8)
    return rho, fixed, fixed


@pytest.mark.parametrize("name,nx,ny,nz,levels,mask", HIER_CASES)
def test_masks_and_galerkin_operators(name, nx, ny, nz, levels, mask):
    rho, fixed, fixed_arg = _case_inputs(nx, ny, nz, mask)
    S = gpu_solver(rho, 3.0, fixed=fixed_arg, levels=levels, smoother="jacobi", coarse_smoother=None, omega=0.4)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, levels)
    patterns = structural_patterns((nx, ny, nz), fixed, levels)
    assert S.num_levels == levels
    for li, lev in enumerate(H):
        assert S.level_dims(li) == lev.dims
        m = S.get_mask(li)
        bits = lev.fixed.reshape(-1, 3)
        assert np.array_equal(m, (bits[:, 0] | bits[:, 1] << 1 | bits[:, 2] << 2).astype(np.uint8))
        if li == 0:
            continue
        A = S.get_bsr(li)
        R = planes_from_csr(lev)
        # pattern: the GPU's implicit index map (27 slots, free DOF pairs) equals
        # the oracle's structural pattern of P^T K P, bit for bit
        gpu_pat = slot_pattern_from_mask(m, lev.dims)
        ora_pat = pattern_planes(patterns[li], lev.dims, lev.free)
        if mask == "clamp":
            assert np.array_equal(gpu_pat, ora_pat)
        else:  # point constraints may remove structural couplings inside a slot
            assert not np.any(ora_pat & ~gpu_pat)
        assert not np.any(A[~gpu_pat])
        assert np.max(np.abs(A - R)) <= 1e-12 * np.max(np.abs(R))


# Kernels of the assembled levels: the default at these sizes (K-split with 32 or
# 16 slices by the size rule), bsr_tma_nodes=1 forces the TMA-staged kernel onto
# every assembled level, bsr_kernel=0 the streaming one-thread-per-node kernel,
# and bsr_kernel=1 / 2 the K-split kernel with 8 / 2 slices.
KERNEL_MODES = [pytest.param({}, id="ksplit"), pytest.param({"bsr_tma_nodes": 1}, id="tma"),
                pytest.param({"bsr_kernel": 0}, id="stream"), pytest.param({"bsr_kernel": 1}, id="ks8"),
                pytest.param({"bsr_kernel": 2}, id="ks2")]


@pytest.mark.parametrize("kmode", KERNEL_MODES)
@pytest.mark.parametrize("name,nx,ny,nz,levels,mask", HIER_CASES[:3])
def test_lambda_estimates(name, nx, ny, nz, levels, mask, kmode):
    rho, fixed, fixed_arg = _case_inputs(nx, ny, nz, mask)
    S = gpu_solver(rho, 3.0, fixed=fixed_arg, levels=levels, smoother="jacobi", coarse_smoother=None, omega=0.4,
                   **kmode)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, levels)
    for li, lev in enumerate(H):
        assert abs(S.get_lambda(li) - lev.lam) < 1e-4 * lev.lam


@pytest.mark.parametrize("kmode", KERNEL_MODES)
@pytest.mark.parametrize("name,nx,ny,nz,levels,mask", HIER_CASES)
def test_level_ops_restrict_prolong_coarse(name, nx, ny, nz, levels, mask, kmode):
    rho, fixed, fixed_arg = _case_inputs(nx, ny, nz, mask)
    S = gpu_solver(rho, 3.0, fixed=fixed_arg, levels=levels, smoother="jacobi", coarse_smoother=None, omega=0.4,
                   **kmode)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, levels)
    rng = np.random.default_rng(5)
    for li, lev in enumerate(H):
        n = 3 * fem.Grid(*lev.dims).n_nodes
        x = np.zeros(n, dtype=np.float32)
        x[lev.free] = rng.uniform(-1, 1, lev.n_free)
        if li > 0:
            y = S.level_apply(li, _t(x)).cpu().numpy()
            yref = np.zeros(n)
            yref[lev.free] = lev.K @ x[lev.free].astype(np.float64)
            assert rel_l2(y, yref) < 1e-6
        if li + 1 < len(H):
            c = H[li + 1]
            P = hy.prolongation(lev.dims)[lev.free][:, c.free]
            xc = S.restrict(li, _t(x)).cpu().numpy()
            ref = np.zeros(3 * fem.Grid(*c.dims).n_nodes)
            ref[c.free] = P.T @ x[lev.free].astype(np.float64)
            assert rel_l2(xc, ref) < 1e-6
            e = np.zeros_like(ref, dtype=np.float32)
            e[c.free] = rng.uniform(-1, 1, c.n_free)
            base = np.zeros(n, dtype=np.float32)
            base[lev.free] = rng.uniform(-1, 1, lev.n_free)
            out = S.prolong_add(li, _t(e), _t(base)).cpu().numpy()
            ref_f = base.astype(np.float64)
            ref_f[lev.free] += P @ e[c.free].astype(np.float64)
            assert rel_l2(out, ref_f) < 1e-6
    last = H[-1]
    nL = 3 * fem.Grid(*last.dims).n_nodes
    b = np.zeros(nL, dtype=np.float32)
    b[last.free] = rng.uniform(-1, 1, last.n_free)
    x = S.coarse_solve(_t(b)).cpu().numpy()
    ref = np.zeros(nL)
    ref[last.free] = hy.coarse_solve(last.L, b[last.free].astype(np.float64))
    assert rel_l2(x, ref) < 1e-5


@pytest.mark.parametrize("name,nx,ny,nz,levels,mask", HIER_CASES[:3])
def test_coarse_solve_overwrites_every_dof(name, nx, ny, nz, levels, mask):
    """The coarsest dense solve writes every entry of its output: the fixed DOFs
    of the coarsest level exactly 0 and the free ones the oracle's solve, also
    when the output buffer starts out holding NaN (twice in a row, so nothing is
    left over from the first call)."""
    rho, fixed, fixed_arg = _case_inputs(nx, ny, nz, mask)
    S = gpu_solver(rho, 3.0, fixed=fixed_arg, levels=levels, smoother="jacobi", coarse_smoother=None, omega=0.4)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, levels)
    last = H[-1]
    nL = 3 * fem.Grid(*last.dims).n_nodes
    rng = np.random.default_rng(17)
    for _ in range(2):
        b = np.zeros(nL, dtype=np.float32)
        b[last.free] = rng.uniform(-1, 1, last.n_free)
        x = torch.full((nL,), float("nan"), dtype=torch.float32, device="cuda")
        out = S.coarse_solve(_t(b), x).cpu().numpy()
        fixed_dofs = np.setdiff1d(np.arange(nL), last.free)
        assert fixed_dofs.size > 0 and np.all(out[fixed_dofs] == 0.0)
        ref = hy.coarse_solve(last.L, b[last.free].astype(np.float64))
        assert np.all(np.isfinite(out)) and rel_l2(out[last.free], ref) < 1e-5


# ---------------------------------------------------------------------------
# smoothers and the V-cycle (oracle lambda injected so both use one band)
# ---------------------------------------------------------------------------
SMOOTH_OPTS = [
    dict(levels=3, smoother="jacobi", degree=2, coarse_smoother=None, coarse_degree=None, omega=0.5, coarse_omega=None),
    dict(levels=3, smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
         coarse_omega=None),
    dict(levels=3, smoother="chebyshev", degree=2, coarse_smoother="jacobi", coarse_degree=2, omega=0.5,
         coarse_omega=0.5),
]


@pytest.mark.parametrize("kmode", KERNEL_MODES)
@pytest.mark.parametrize("opts", SMOOTH_OPTS, ids=["jacobi", "cheb3", "cheb2+jacobi"])
def test_smoothers_and_vcycle(opts, kmode):
    c = inputs.CONFIGS["c0"]
    rho = inputs.filtered_random_density(c.nx, c.ny, c.nz, 2)
    fixed = c.fixed()
    S = gpu_solver(rho, 3.0, **opts, **kmode)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, opts["levels"])
    for li, lev in enumerate(H):
        S.set_lambda(li, lev.lam)
    spec = oracle_spec_from_opts(opts)
    rng = np.random.default_rng(8)
    for li, lev in enumerate(H[:-1]):
        n = 3 * fem.Grid(*lev.dims).n_nodes
        b = np.zeros(n, dtype=np.float32)
        b[lev.free] = rng.uniform(-1, 1, lev.n_free)
        x0 = np.zeros(n, dtype=np.float32)
        x0[lev.free] = rng.uniform(-1, 1, lev.n_free)
        xs = S.level_smooth(li, _t(b)).cpu().numpy()
        ref = np.zeros(n)
        ref[lev.free] = so.smooth(lev, b[lev.free].astype(np.float64), np.zeros(lev.n_free), spec, li)
        assert rel_l2(xs, ref) < 1e-6
        xs = S.level_smooth(li, _t(b), _t(x0)).cpu().numpy()
        ref[lev.free] = so.smooth(lev, b[lev.free].astype(np.float64), x0[lev.free].astype(np.float64), spec, li)
        assert rel_l2(xs, ref) < 1e-6
    r = np.zeros(3 * c.n_nodes, dtype=np.float32)
    r[H[0].free] = rng.uniform(-1, 1, H[0].n_free)
    z = S.vcycle(_t(r)).cpu().numpy()
    zref = np.zeros(3 * c.n_nodes)
    zref[H[0].free] = so.vcycle(H, r[H[0].free].astype(np.float64), spec)
    assert rel_l2(z, zref) < 1e-5


# ---------------------------------------------------------------------------
# end-to-end solves
# ---------------------------------------------------------------------------
def _solve_and_compare(rho, p, fixed, f, opts, cap=200, exact=True):
    S = gpu_solver(rho, p, **opts)
    H, E = oracle_hierarchy(rho, p, fixed, opts["levels"])
    spec = oracle_spec_from_opts(opts)
    u_or, res = so.gmg_pcg(H, f, spec, tol=1e-6, maxit=cap)
    u_gpu, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=cap)
    u_gpu = u_gpu.cpu().numpy()
    assert (info["status"] == 0) == (res.status == so.OK)
    if res.status == so.OK:
        assert abs(info["iterations"] - res.iterations) <= max(2, 0.1 * res.iterations)
        # the oracle recomputes the residual of the GPU solution independently
        nz, ny, nx = rho.shape
        g = fem.Grid(nx, ny, nz)
        r = f - fem.matfree_apply(g, E, fem.element_stiffness(0.3), u_gpu)
        free = fem.free_dofs(fixed)
        assert np.linalg.norm(r[free]) / np.linalg.norm(f[free]) <= 1e-6
        assert abs(info["rel_residual"] - np.linalg.norm(r[free]) / np.linalg.norm(f[free])) < 1e-9
        assert np.all(u_gpu[fixed == 1] == 0)
        if exact:
            ue = so.exact_solve(H, f, spec)
            assert rel_l2(u_gpu, ue) < 1e-5
    return info, res


def test_solve_config0():
    c = inputs.CONFIGS["c0"]
    info, res = _solve_and_compare(c.rho(), c.p, c.fixed(), c.load(), config_opts(c))
    assert info["status"] == 0


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0])
def test_solve_config1(p):
    c = inputs.CONFIGS["c1"]
    info, res = _solve_and_compare(c.rho(), p, c.fixed(), c.load(), config_opts(c))
    assert info["status"] == 0


@pytest.mark.parametrize("kmode", KERNEL_MODES)
def test_solve_ragged_chebyshev(kmode):
    nx, ny, nz = 23, 11, 9
    rho = inputs.filtered_random_density(nx, ny, nz, 4)
    opts = dict(levels=3, smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None, **kmode)
    info, res = _solve_and_compare(rho, 3.0, inputs.clamp_xmin_mask(nx, ny, nz), inputs.tip_edge_load(nx, ny, nz), opts)
    assert info["status"] == 0


@pytest.mark.parametrize("kmode", [pytest.param({}, id="stream"), pytest.param({"bsr_tma_nodes": 65536}, id="tma"),
                                   pytest.param({"bsr_kernel": 1}, id="ksplit")])
def test_solve_full_size_config2(kmode):
    """100^3, 5 levels, Chebyshev degree 3: the oracle judges the GPU solution by
    its own FP64 residual and the energy identity.  The tma variant runs level 1
    (132,651 nodes) through the TMA-staged operator kernel, the ksplit one every
    assembled level (level 1 included) through the K-split kernel."""
    c = inputs.CONFIGS["c2"]
    S = gpu_solver(c.rho(), c.p, **config_opts(c), **kmode)
    f = c.load()
    u, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=200)
    assert info["status"] == 0
    u = u.cpu().numpy()
    g = fem.Grid(c.nx, c.ny, c.nz)
    E = fem.moduli(c.rho(), c.p)
    Ku = fem.matfree_apply(g, E, fem.element_stiffness(0.3), u)
    free = fem.free_dofs(c.fixed())
    rel = np.linalg.norm((f - Ku)[free]) / np.linalg.norm(f[free])
    assert rel <= 1e-6
    assert abs(u @ Ku - f @ u) <= 1e-5 * abs(f @ u)


# ---------------------------------------------------------------------------
# edge cases and failure reporting
# ---------------------------------------------------------------------------
def test_edge_cases():
    from paper_2604_26441_b300 import gmg
    c = inputs.CONFIGS["c0"]
    S = gpu_solver(c.rho(), c.p, **config_opts(c))
    f = _t(c.load(), torch.float64)
    # zero load: zero solution, no iterations
    u, info = S.solve(torch.zeros_like(f))
    assert info["status"] == 0 and info["iterations"] == 0 and float(u.abs().max()) == 0.0
    # cap reached
    u, info = S.solve(f, tol=1e-6, maxit=1)
    assert info["status"] == gmg.GMG_NOT_CONVERGED and info["iterations"] == 1
    # warm start from the converged solution: accepted at once
    u, info = S.solve(f)
    u2, info2 = S.solve(f, u=u.clone())
    assert info2["status"] == 0 and info2["iterations"] == 0
    # non-finite load
    fb = f.clone()
    fb[3 * 40 + 1] = float("nan")
    _, info = S.solve(fb)
    assert info["status"] == gmg.GMG_NONFINITE
    # unstable damping is refused at set-up
    with pytest.raises(gmg.GMGError) as ei:
        gpu_solver(c.rho(), c.p, levels=3, smoother="jacobi", coarse_smoother=None, omega=1.0, coarse_omega=None)
    assert ei.value.code == -4
    # too many levels for the grid
    with pytest.raises(gmg.GMGError):
        gpu_solver(c.rho(), c.p, levels=6, smoother="jacobi", coarse_smoother=None, omega=0.5)


def test_grid_barrier_timeout_is_reported_and_recovered():
    """The fused lower V-cycle's grid barrier is a bounded poll of a generation
    word.  With a bound of 0 polls every block that is not the last to arrive
    gives up at once (the wait runs out; nothing faults or hangs), so the solve
    must report GMG_TIMEOUT, not a solution.  After the default bound is
    restored, the same handle solves normally and matches the per-level path."""
    from paper_2604_26441_b300 import gmg
    c = inputs.CONFIGS["c0"]
    S = gpu_solver(c.rho(), c.p, **config_opts(c), fused_coarse_nodes=65536, spin_limit=0)
    f = _t(c.load(), torch.float64)
    with pytest.raises(gmg.GMGError) as ei:
        S.solve(f)
    assert ei.value.code == gmg.GMG_TIMEOUT
    assert b"grid barrier" in gmg.load_library().gmg_last_error()
    with pytest.raises(gmg.GMGError) as ei:  # still bounded at 0: reported again, not accepted
        S.solve(f)
    assert ei.value.code == gmg.GMG_TIMEOUT
    S.set_spin_limit(1 << 24)
    u, info = S.solve(f)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-6
    S_ref = gpu_solver(c.rho(), c.p, **config_opts(c), fused_coarse_nodes=0)
    u_ref, info_ref = S_ref.solve(f)
    assert abs(info["iterations"] - info_ref["iterations"]) <= 1
    assert rel_l2(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-5
    assert info["setup_ms"] > 0.0


COARSE_PCG_OPTS = dict(levels=2, smoother="jacobi", degree=2, coarse_smoother=None, coarse_degree=None, omega=0.6,
                       coarse_omega=None, chol_cutoff=500)


@pytest.mark.parametrize("steps,tol", [(5, 1e-4), (20, 1e-3)])
def test_coarsest_pcg_fallback_matches_oracle(steps, tol):
    """The coarsest level above the dense-Cholesky cutoff (16x8x8 in two levels
    with cutoff 500: level 1 has 600 free DOFs) is solved by a fixed count of
    Jacobi-PCG steps from 0 (Sec. "Matrix-Free V-Cycle"); FP32 against the
    oracle's FP64 iterate after the same steps."""
    c = inputs.CONFIGS["c0"]
    rho, fixed = c.rho(), c.fixed()
    S = gpu_solver(rho, c.p, **COARSE_PCG_OPTS, coarse_pcg_steps=steps)
    H = hy.build_hierarchy((c.nx, c.ny, c.nz), fem.moduli(rho, c.p), fixed, levels=2, chol_cutoff=500,
                           coarse_pcg_steps=steps)
    last = H[-1]
    assert last.L is None and last.n_free > 500
    b = inputs.random_free_vector(last.fixed, seed=21)
    x = S.coarse_solve(_t(b)).cpu().numpy()
    ref = np.zeros_like(b, dtype=np.float64)
    ref[last.free] = hy.coarse_pcg(last.apply, last.diag, b[last.free].astype(np.float64), steps)
    assert np.all(x[last.fixed == 1] == 0)
    assert rel_l2(x, ref) < tol, rel_l2(x, ref)


def test_coarsest_pcg_fallback_solve():
    """A full GMG-PCG solve with the 80-step coarsest PCG: the same outcome as
    the oracle's, the oracle's own FP64 residual of the GPU solution below 1e-6,
    and the displacement within 1e-5 of the oracle's exact solution."""
    c = inputs.CONFIGS["c0"]
    rho, fixed, f = c.rho(), c.fixed(), c.load()
    S = gpu_solver(rho, c.p, **COARSE_PCG_OPTS)
    H = hy.build_hierarchy((c.nx, c.ny, c.nz), fem.moduli(rho, c.p), fixed, levels=2, chol_cutoff=500)
    spec = so.SmootherSpec("jacobi", 2, 0.6)
    u_or, res = so.gmg_pcg(H, f, spec, tol=1e-6, maxit=200)
    u, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=200)
    assert (info["status"] == 0) == (res.status == so.OK)
    assert info["status"] == 0
    assert abs(info["iterations"] - res.iterations) <= max(2, 0.1 * res.iterations), (info, res.iterations)
    u = u.cpu().numpy()
    g = fem.Grid(c.nx, c.ny, c.nz)
    r = f - fem.matfree_apply(g, fem.moduli(rho, c.p), fem.element_stiffness(0.3), u)
    free = fem.free_dofs(fixed)
    assert np.linalg.norm(r[free]) / np.linalg.norm(f[free]) <= 1e-6
    H_exact = hy.build_hierarchy((c.nx, c.ny, c.nz), fem.moduli(rho, c.p), fixed, levels=c.levels)
    assert rel_l2(u, so.exact_solve(H_exact, f)) < 1e-5


def test_smallest_grid():
    rho = inputs.uniform_density(2, 2, 2)
    opts = dict(levels=2, smoother="jacobi", degree=2, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    info, res = _solve_and_compare(rho, 3.0, inputs.clamp_xmin_mask(2, 2, 2), inputs.tip_edge_load(2, 2, 2), opts)
    assert info["status"] == 0


@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
def test_fused_lower_vcycle_matches_per_level_kernels(cfg_name):
    """The persistent kernel that runs the assembled levels below the node
    threshold (and the coarsest solve) gives the same V-cycle and the same
    solve as one kernel launch per step."""
    c = inputs.CONFIGS[cfg_name]
    rho = c.rho()
    opts = config_opts(c)
    S_f = gpu_solver(rho, c.p, **opts, fused_coarse_nodes=65536)
    S_u = gpu_solver(rho, c.p, **opts, fused_coarse_nodes=0)
    rng = np.random.default_rng(12)
    r = inputs.random_free_vector(c.fixed(), seed=13)
    zf = S_f.vcycle(_t(r)).cpu().numpy()
    zu = S_u.vcycle(_t(r)).cpu().numpy()
    assert rel_l2(zf, zu) < 1e-5
    f = _t(c.load(), torch.float64)
    _, inf_f = S_f.solve(f)
    _, inf_u = S_u.solve(f)
    assert inf_f["status"] == 0 and inf_u["status"] == 0
    assert abs(inf_f["iterations"] - inf_u["iterations"]) <= 1


# ---------------------------------------------------------------------------
# device-resident PCG loop (CUDA graph with a conditional while node)
# ---------------------------------------------------------------------------
LOOP_CASES = [
    ("c0", 1e-6, 200),
    ("c1", 1e-6, 200),
    ("c0", 1e-9, 60),   # tight: residual replacements relaunch the graph
    ("c1", 1e-6, 5),    # the cap ends the loop
]


@pytest.mark.parametrize("cfg_name,tol,maxit", LOOP_CASES)
def test_device_loop_matches_host_loop(cfg_name, tol, maxit):
    """The graph runs the host loop's kernels in the same order: the iterates,
    counts and residuals agree bit for bit, also across replacements and the cap."""
    c = inputs.CONFIGS[cfg_name]
    f = _t(c.load(), torch.float64)
    res = {}
    for dev in (True, False):
        S = gpu_solver(c.rho(), c.p, **config_opts(c), device_loop=dev)
        u = torch.zeros_like(f)
        _, info = S.solve(f, u, tol=tol, maxit=maxit)
        first = u.clone()
        u.zero_()
        _, info2 = S.solve(f, u, tol=tol, maxit=maxit)  # same iterate buffer: the captured graph is reused
        assert torch.equal(u, first) and info["iterations"] == info2["iterations"]
        res[dev] = (u.cpu().numpy(), info)
    (ud, idv), (uh, ih) = res[True], res[False]
    assert np.array_equal(ud, uh)
    for key in ("status", "iterations", "replacements", "rel_residual", "rel_residual_recursive"):
        assert idv[key] == ih[key], key
    if maxit == 5:
        assert idv["iterations"] == 5 and idv["status"] != 0


# ---------------------------------------------------------------------------
# outer FP64 iterative refinement around the FP32 inner PCG
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
def test_iterative_refinement_reaches_fp64_tolerance(cfg_name):
    """tol 1e-10 is below what the FP32 recursion alone can certify; with outer
    FP64 refinement the oracle's own FP64 residual of the returned u meets it."""
    c = inputs.CONFIGS[cfg_name]
    f = c.load()
    S = gpu_solver(c.rho(), c.p, **config_opts(c), ir_factor=1e-3)
    u, info = S.solve(_t(f, torch.float64), tol=1e-10, maxit=400)
    assert info["status"] == 0 and info["rel_residual"] < 1e-10
    assert info["replacements"] >= 1  # at least one outer refinement step
    u = u.cpu().numpy()
    g = fem.Grid(c.nx, c.ny, c.nz)
    E = fem.moduli(c.rho(), c.p)
    r = f - fem.matfree_apply(g, E, fem.element_stiffness(0.3), u)
    free = fem.free_dofs(c.fixed())
    rel = np.linalg.norm(r[free]) / np.linalg.norm(f[free])
    assert rel < 1e-10
    assert abs(rel - info["rel_residual"]) < 1e-12
    if cfg_name == "c0":  # dense FP64 Cholesky of K_ff
        H, _ = oracle_hierarchy(c.rho(), c.p, c.fixed(), c.levels)
        ue = so.exact_solve(H, f, oracle_spec_from_opts(config_opts(c)))
        assert rel_l2(u, ue) < 1e-8
    # the device-resident and host-driven loops agree bit for bit in this mode too
    S2 = gpu_solver(c.rho(), c.p, **config_opts(c), ir_factor=1e-3, device_loop=False)
    u2, info2 = S2.solve(_t(f, torch.float64), tol=1e-10, maxit=400)
    assert np.array_equal(u, u2.cpu().numpy()) and info2["iterations"] == info["iterations"]


# ---------------------------------------------------------------------------
# tensor-core fine smoother (BF16 / split-BF16 element contraction on tcgen05)
# ---------------------------------------------------------------------------
TC_MODES = [pytest.param("bf16x3", 3e-5, id="bf16x3"), pytest.param("bf16", 2e-2, id="bf16")]


@pytest.mark.parametrize("mode,tol", TC_MODES)
@pytest.mark.parametrize("name,nx,ny,nz,levels", [("c0", 16, 8, 8, 3), ("ragged", 23, 11, 9, 3), ("c1", 40, 40, 40, 4)])
def test_tensor_core_smoother_matches_oracle(mode, tol, name, nx, ny, nz, levels):
    """One fine smoothing pass through the tensor-core kernel against the oracle's
    FP64 smoother on the same FP32 inputs (Chebyshev degree 3 exercises the
    increment recurrence and the zero / nonzero initial iterate)."""
    rho = inputs.filtered_random_density(nx, ny, nz, 3)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    opts = dict(levels=levels, smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    S = gpu_solver(rho, 3.0, **opts, fine_smoother=mode)
    H, _ = oracle_hierarchy(rho, 3.0, fixed, levels)
    S.set_lambda(0, H[0].lam)
    spec = oracle_spec_from_opts(opts)
    lev = H[0]
    rng = np.random.default_rng(21)
    n = 3 * fem.Grid(nx, ny, nz).n_nodes
    b = np.zeros(n, dtype=np.float32)
    b[lev.free] = rng.uniform(-1, 1, lev.n_free)
    x0 = np.zeros(n, dtype=np.float32)
    x0[lev.free] = rng.uniform(-1, 1, lev.n_free)
    xs = S.level_smooth(0, _t(b), _t(x0)).cpu().numpy()
    ref = np.zeros(n)
    ref[lev.free] = so.smooth(lev, b[lev.free].astype(np.float64), x0[lev.free].astype(np.float64), spec, 0)
    assert rel_l2(xs, ref) < tol
    assert np.all(xs[fixed == 1] == 0)


@pytest.mark.parametrize("mode,extra,outer", [("bf16x3", 1, "pcg"), ("bf16", 6, "fgmres")])
@pytest.mark.parametrize("cfg_name", ["c0", "c1", "c2"])
def test_tensor_core_smoother_solves(mode, extra, outer, cfg_name):
    """The tensor-core fine smoother converges to the FP64-checked tolerance:
    split BF16 under PCG with at most one more iteration than the FP32
    smoother; plain BF16 under FGMRES, the outer solver the paper pairs it
    with (its rounding makes the V-cycle too far from a symmetric operator for
    CG: with PCG it stagnated at 6e-5 on 100^3 with the per-level coarse path)."""
    c = inputs.CONFIGS[cfg_name]
    f = c.load()
    iters = {}
    for sm in ("fp32", mode):
        S = gpu_solver(c.rho(), c.p, **config_opts(c), fine_smoother=sm, outer=outer)
        u, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=200)
        assert info["status"] == 0 and info["rel_residual"] < 1e-6
        iters[sm] = info["iterations"]
    assert iters[mode] <= iters["fp32"] + extra
    u = u.cpu().numpy()
    g = fem.Grid(c.nx, c.ny, c.nz)
    r = f - fem.matfree_apply(g, fem.moduli(c.rho(), c.p), fem.element_stiffness(0.3), u)
    free = fem.free_dofs(c.fixed())
    assert np.linalg.norm(r[free]) / np.linalg.norm(f[free]) < 1e-6


# ---------------------------------------------------------------------------
# solver variants and diagnostics: W-cycle, FGMRES, kappa_eff, symmetry defect,
# deterministic stress states
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["jacobi", "chebyshev"])
def test_wcycle_matches_oracle(kind):
    c = inputs.CONFIGS["c1"]
    rho = c.rho()
    opts = dict(levels=4, smoother=kind, degree=2 if kind == "jacobi" else 3, coarse_smoother=None,
                coarse_degree=None, omega=0.5, coarse_omega=None)
    S = gpu_solver(rho, c.p, **opts, cycle="W")
    H, _ = oracle_hierarchy(rho, c.p, c.fixed(), 4)
    for li, lev in enumerate(H):
        S.set_lambda(li, lev.lam)
    spec = oracle_spec_from_opts(opts)
    r = np.zeros(3 * c.n_nodes, dtype=np.float32)
    r[H[0].free] = np.random.default_rng(31).uniform(-1, 1, H[0].n_free)
    z = S.vcycle(_t(r)).cpu().numpy()
    zref = np.zeros(3 * c.n_nodes)
    zref[H[0].free] = so.mgcycle(H, r[H[0].free].astype(np.float64), spec, gamma=2)
    assert rel_l2(z, zref) < 1e-5


@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
def test_wcycle_and_fgmres_solves(cfg_name):
    c = inputs.CONFIGS[cfg_name]
    f = c.load()
    H, E = oracle_hierarchy(c.rho(), c.p, c.fixed(), c.levels)
    spec = oracle_spec_from_opts(config_opts(c))
    lev = H[0]
    res = {}
    for name, extra in (("V", {}), ("W", dict(cycle="W")), ("fgmres", dict(outer="fgmres", restart=32))):
        S = gpu_solver(c.rho(), c.p, **config_opts(c), **extra)
        u, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=200)
        assert info["status"] == 0, name
        u = u.cpu().numpy()
        r = f - fem.matfree_apply(fem.Grid(c.nx, c.ny, c.nz), E, fem.element_stiffness(0.3), u)
        free = fem.free_dofs(c.fixed())
        assert np.linalg.norm(r[free]) / np.linalg.norm(f[free]) < 1e-6
        res[name] = info["iterations"]
    assert res["W"] <= res["V"]
    ores = so.fgmres(lev.apply, lambda v: so.vcycle(H, v, spec), f[lev.free], tol=1e-6, restart=32)
    assert ores.status == so.OK and abs(res["fgmres"] - ores.iterations) <= 2


def test_kappa_eff_matches_oracle():
    c = inputs.CONFIGS["c1"]
    S = gpu_solver(c.rho(), c.p, **config_opts(c))
    H, _ = oracle_hierarchy(c.rho(), c.p, c.fixed(), c.levels)
    for li, lev in enumerate(H):
        S.set_lambda(li, lev.lam)
    b = np.zeros(3 * c.n_nodes)
    b[H[0].free] = np.random.default_rng(41).normal(size=H[0].n_free)
    lmin, lmax, kap = S.kappa_eff(_t(b, torch.float64), steps=15)
    olmin, olmax, okap = so.kappa_eff(H, b[H[0].free], oracle_spec_from_opts(config_opts(c)), 15)
    assert abs(lmax - olmax) < 1e-3 * olmax and abs(lmin - olmin) < 1e-3 * olmin
    assert abs(kap - okap) < 2e-3 * okap and kap > 1.0


@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
def test_vcycle_symmetry_defect_is_rounding_level(cfg_name):
    c = inputs.CONFIGS[cfg_name]
    S = gpu_solver(c.rho(), c.p, **config_opts(c))
    fixed = c.fixed()
    x = inputs.random_free_vector(fixed, 51)
    y = inputs.random_free_vector(fixed, 52)
    assert S.vcycle_symmetry(_t(x), _t(y)) < 1e-5


@pytest.mark.parametrize("state", ["checkerboard", "layered"])
def test_stress_states_agree_with_oracle(state):
    nx, ny, nz = 24, 12, 12
    rho = (inputs.checkerboard_density if state == "checkerboard" else inputs.layered_band_density)(nx, ny, nz)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    f = inputs.tip_edge_load(nx, ny, nz)
    opts = dict(levels=3, smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    S = gpu_solver(rho, 3.0, **opts, outer="fgmres", restart=50)
    u, info = S.solve(_t(f, torch.float64), tol=1e-6, maxit=300)
    H, E = oracle_hierarchy(rho, 3.0, fixed, 3)
    lev = H[0]
    ores = so.fgmres(lev.apply, lambda v: so.vcycle(H, v, oracle_spec_from_opts(opts)), f[lev.free], tol=1e-6,
                     maxit=300, restart=50)
    assert (info["status"] == 0) == (ores.status == so.OK)
    if info["status"] == 0:
        u = u.cpu().numpy()
        r = f - fem.matfree_apply(fem.Grid(nx, ny, nz), E, fem.element_stiffness(0.3), u)
        free = fem.free_dofs(fixed)
        assert np.linalg.norm(r[free]) / np.linalg.norm(f[free]) < 1e-6


# ---------------------------------------------------------------------------
# batched solves: uneven instances x several loads in one CUDA graph
# ---------------------------------------------------------------------------
def _batch_problems():
    grids = [(16, 8, 8, 3), (23, 11, 9, 3), (24, 24, 24, 3)]
    out = []
    for gi, (nx, ny, nz, levels) in enumerate(grids):
        rho = inputs.filtered_random_density(nx, ny, nz, 100 + gi)
        loads = [inputs.rotated_tip_edge_load(nx, ny, nz, k, nrhs=16) for k in (0, 5, 11)]
        out.append((rho, levels, loads))
    return out


def test_batch_matches_single_solves():
    """Clones of one hierarchy run as one multi-load chunk: per item bitwise the
    answers and iteration counts of gmg_solve_multi on the same loads, and the
    status of a single solve with its count within one (the multi-load path
    sums its reductions in another grouping, so its iterates agree with the
    single solve's only to rounding) and its solution within 1e-5."""
    from paper_2604_26441_b300 import gmg
    opts = dict(smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    solvers, fs, ref, multi = [], [], [], []
    for rho, levels, loads in _batch_problems():
        base = gpu_solver(rho, 3.0, levels=levels, **opts)
        for k, load in enumerate(loads):
            solvers.append(base if k == 0 else base.clone())
            fs.append(_t(load, torch.float64))
        single = gpu_solver(rho, 3.0, levels=levels, **opts, fused_coarse_nodes=0)
        for load in loads:
            u, info = single.solve(_t(load, torch.float64))
            ref.append((u.cpu().numpy(), info))
        um, im = single.solve_multi([_t(load, torch.float64) for load in loads])
        multi += [(u.cpu().numpy(), i) for u, i in zip(um, im)]
    us, infos = gmg.solve_batch(solvers, fs)
    for (u_ref, info_ref), (u_m, info_m), u, info in zip(ref, multi, us, infos):
        assert info["status"] == 0 and info["rel_residual"] < 1e-6
        assert info["iterations"] == info_m["iterations"]
        assert abs(info["iterations"] - info_ref["iterations"]) <= 1
        assert rel_l2(u.cpu().numpy(), u_ref) < 1e-5
        assert np.array_equal(u.cpu().numpy(), u_m)
    # the captured graph is replayed for the same handles and iterates
    first = [u.clone() for u in us]
    for u in us:
        u.zero_()
    us2, infos2 = gmg.solve_batch(solvers, fs, us)
    assert all(torch.equal(a, b) for a, b in zip(first, us2))
    # the oracle's own FP64 residual of one batched answer
    rho, levels, loads = _batch_problems()[2]
    nz, ny, nx = rho.shape
    u = us[-1].cpu().numpy()
    r = loads[-1] - fem.matfree_apply(fem.Grid(nx, ny, nz), fem.moduli(rho, 3.0), fem.element_stiffness(0.3), u)
    free = fem.free_dofs(inputs.clamp_xmin_mask(nx, ny, nz))
    assert np.linalg.norm(r[free]) / np.linalg.norm(loads[-1][free]) < 1e-6


def test_batch_of_distinct_grids_equals_single_solves():
    """Handles that share no hierarchy keep their own single-load loops as
    graph branches: bitwise the iterates of gmg_solve."""
    from paper_2604_26441_b300 import gmg
    opts = dict(smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    solvers, fs, ref = [], [], []
    for rho, levels, loads in _batch_problems():
        solvers.append(gpu_solver(rho, 3.0, levels=levels, **opts))
        fs.append(_t(loads[1], torch.float64))
        single = gpu_solver(rho, 3.0, levels=levels, **opts, fused_coarse_nodes=0)
        u, info = single.solve(_t(loads[1], torch.float64))
        ref.append((u.cpu().numpy(), info))
    us, infos = gmg.solve_batch(solvers, fs)
    for (u_ref, info_ref), u, info in zip(ref, us, infos):
        assert info["status"] == 0 and info["iterations"] == info_ref["iterations"]
        assert np.array_equal(u.cpu().numpy(), u_ref)


@pytest.mark.parametrize("cfg_name", ["c1", "c2"])
def test_autotune_keeps_operator_results(cfg_name):
    """gmg_autotune picks launch shapes only: the fine operator's output is
    bitwise the same under the tuned plan, solves still converge to the same
    solution, and the kept choice is the fastest measured."""
    cfg = inputs.CONFIGS[cfg_name]
    opts = config_opts(cfg)
    S = gpu_solver(cfg.rho(), cfg.p, **opts)
    u = _t(inputs.random_free_vector(cfg.fixed(), seed=31))
    y0 = S.apply(u).cpu().numpy()
    f = _t(cfg.load(), torch.float64)
    ub, ib = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
    try:
        t = S.autotune(reps=3)
        assert t["fine_candidates"] >= 2 and t["fine_us"] <= t["model_us"]
        assert all(b["us"] <= b["other_us"] for b in t["bsr"])
        y1 = S.apply(u).cpu().numpy()
        assert np.array_equal(y0, y1)
        ua, ia = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
        assert ia["status"] == 0 and ia["rel_residual"] <= cfg.tol
        assert abs(ia["iterations"] - ib["iterations"]) <= 1
        assert rel_l2(ua.cpu().numpy(), ub.cpu().numpy()) < 1e-5
    finally:
        S.autotune(reps=0)


def test_alternating_iterate_buffers_reuse_their_loop_graphs():
    """Solves into several u buffers in turn (more than the handle keeps
    captured loops for) give bitwise the same iterates and solutions as
    solves into one buffer."""
    cfg = inputs.CONFIGS["c1"]
    S = gpu_solver(cfg.rho(), cfg.p, **config_opts(cfg))
    f = _t(cfg.load(), torch.float64)
    ref, iref = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
    us = [torch.zeros_like(f) for _ in range(5)]
    for rnd in range(2):
        for u in us:
            u.zero_()
            _, info = S.solve(f, u, tol=cfg.tol, maxit=cfg.maxit)
            assert info["iterations"] == iref["iterations"] and info["status"] == 0
            assert torch.equal(u, ref)
