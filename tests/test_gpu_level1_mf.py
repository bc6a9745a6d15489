"""Level 1 applied matrix-free (Eq. galerkin_level1 summed per coarse element
from the fine moduli) against the assembled level-1 operator and the oracle.

Where the fine sizes are even and every fixed fine DOF has only fixed
prolongation parents (the clamped cantilever), the size rule applies level 1
matrix-free; the two forms are the same operator and differ by FP32 rounding,
so applies and smoothing steps agree within 1e-6 and solves take the same
iteration counts within one.  Other grids keep the assembled operator.
"""

import numpy as np
import pytest

from oracle import fem, hierarchy as hy
from paper_2604_26441_b300 import inputs

from gpu_helpers import config_opts, gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_26441_b300 import build
    build.build_library()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _level1_kind(S):
    kinds = {b["level"]: b["kind"] for b in S.autotune(reps=0)["bsr"]}
    return kinds.get(1)


GRIDS = [(16, 8, 8, 3), (20, 12, 6, 3), (24, 24, 24, 3), (40, 40, 40, 4)]


@pytest.mark.parametrize("nx,ny,nz,levels", GRIDS)
@pytest.mark.parametrize("smoother", ["chebyshev", "jacobi"])
def test_level1_matrix_free_equals_assembled(nx, ny, nz, levels, smoother):
    rho = inputs.filtered_random_density(nx, ny, nz, 9)
    opts = dict(levels=levels, smoother=smoother, degree=3 if smoother == "chebyshev" else 2, omega=0.5,
                coarse_smoother=None, coarse_degree=None, coarse_omega=None)
    S = gpu_solver(rho, 3.0, **opts)
    A = gpu_solver(rho, 3.0, bsr_kernel=0, **opts)
    assert _level1_kind(S) == "matrix-free" and _level1_kind(A) == "streaming"
    fixed1 = S.get_mask(1)
    free1 = ((fixed1[:, None] >> np.arange(3)) & 1 == 0).reshape(-1)
    rng = np.random.default_rng(nx + ny + nz)
    x = np.where(free1, rng.uniform(-1, 1, free1.size), 0.0).astype(np.float32)
    b = np.where(free1, rng.uniform(-1, 1, free1.size), 0.0).astype(np.float32)
    ys, ya = S.level_apply(1, _t(x)).cpu().numpy(), A.level_apply(1, _t(x)).cpu().numpy()
    assert rel_l2(ys, ya) < 1e-6
    # values on fixed DOFs of the input are ignored, as by the assembled operator
    xd = x.copy()
    xd[~free1] = 1e3
    assert rel_l2(S.level_apply(1, _t(xd)).cpu().numpy(), ya) < 1e-6
    for zero in (True, False):
        xs = S.level_smooth(1, _t(b), None if zero else _t(x)).cpu().numpy()
        xa = A.level_smooth(1, _t(b), None if zero else _t(x)).cpu().numpy()
        assert rel_l2(xs, xa) < 1e-6


def test_level1_matrix_free_matches_oracle():
    nx, ny, nz = 20, 12, 6
    rho = inputs.filtered_random_density(nx, ny, nz, 4)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    S = gpu_solver(rho, 3.0, levels=3, smoother="jacobi", omega=0.5, coarse_smoother=None)
    assert _level1_kind(S) == "matrix-free"
    E = fem.moduli(rho, 3.0).reshape(-1)
    fixed_c = hy.inject_fixed((nx, ny, nz), fixed)
    K1 = hy.level1_elementwise((nx, ny, nz), E, fem.element_stiffness(0.3), fixed, fixed_c)
    fc = fem.free_dofs(fixed_c)
    x = np.zeros(fixed_c.size)
    x[fc] = np.random.default_rng(5).uniform(-1, 1, fc.size)
    y = S.level_apply(1, _t(x)).cpu().numpy().astype(np.float64)
    assert rel_l2(y[fc], K1 @ x[fc]) < 1e-6
    assert np.all(y[fixed_c == 1] == 0.0)


@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
def test_level1_matrix_free_solves(cfg_name):
    cfg = inputs.CONFIGS[cfg_name]
    f = _t(cfg.load(), torch.float64)
    S = gpu_solver(cfg.rho(), cfg.p, **config_opts(cfg))
    A = gpu_solver(cfg.rho(), cfg.p, bsr_kernel=0, **config_opts(cfg))
    assert _level1_kind(S) == "matrix-free"
    us, is_ = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
    ua, ia = A.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
    assert is_["status"] == ia["status"] == 0
    assert abs(is_["iterations"] - ia["iterations"]) <= 1
    assert rel_l2(us.cpu().numpy(), ua.cpu().numpy()) < 1e-5


def test_level1_stays_assembled_where_not_exact():
    # odd fine sizes, and a point constraint on an odd fine node (its coarse
    # parents are free)
    S = gpu_solver(inputs.filtered_random_density(37, 13, 9, 2), 3.0, levels=3, smoother="jacobi", omega=0.5,
                   coarse_smoother=None)
    assert _level1_kind(S) != "matrix-free"
    nx, ny, nz = 16, 8, 8
    fixed = inputs.clamp_xmin_mask(nx, ny, nz).reshape(nz + 1, ny + 1, nx + 1, 3).copy()
    fixed[3, 3, 5, 1] = 1
    S = gpu_solver(inputs.uniform_density(nx, ny, nz), 3.0, fixed=fixed.reshape(-1), levels=3, smoother="jacobi",
                   omega=0.5, coarse_smoother=None)
    assert _level1_kind(S) != "matrix-free"
