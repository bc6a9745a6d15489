"""The fine kernel's two-column tiles against its one-column tiles.

A two-column thread runs each element's arithmetic with the same operations in
the same order as the one-column kernel (packed pairs whose lanes are two
elements), so the operator, the smoothing steps and the V-cycle must come out
bitwise equal under every plan: tile shape and node planes per block only move
work between threads.  Solves group their reduction partial sums by block, so
they are compared by convergence and solution, not bit for bit.  The
one-column kernel itself is checked against the oracle in test_gpu_parity.py;
one case here checks a two-column plan against the oracle directly.
"""

import numpy as np
import pytest

from oracle import fem
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


PAIR_TILES = ["pair-8x16", "pair-16x8", "pair-16x16"]

# grids with ragged tiles in x and y, chunks of 1 .. all planes in z, single
# elements, thin slabs, and a random fixed-DOF mask
CASES = [
    ("c0", 16, 8, 8, "uniform", 3.0, "clamp"),
    ("ragged", 37, 13, 9, "filtered", 3.0, "clamp"),
    ("thin", 33, 2, 5, "filtered", 1.0, "clamp"),
    ("wide", 70, 9, 6, "filtered", 3.0, "random"),
    ("one", 1, 1, 1, "uniform", 3.0, "clamp"),
    ("two", 2, 3, 2, "filtered", 2.0, "random"),
    ("c1", 40, 40, 40, "filtered", 2.0, "clamp"),
]


def _case(nx, ny, nz, dens, mask):
    rho = inputs.uniform_density(nx, ny, nz) if dens == "uniform" else inputs.filtered_random_density(nx, ny, nz, 5)
    if mask == "clamp":
        fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    else:
        rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
        fixed = (rng.uniform(size=3 * inputs.n_nodes(nx, ny, nz)) < 0.15).astype(np.uint8)
        fixed[:3] = 1  # at least one fixed DOF
    return rho, fixed


def _outputs(S, fixed, seed):
    """Operator, two smoothing passes (from zero and from a nonzero iterate) and
    one V-cycle on seeded vectors."""
    u = _t(inputs.random_free_vector(fixed, seed=seed))
    b = _t(inputs.random_free_vector(fixed, seed=seed + 1))
    x = _t(inputs.random_free_vector(fixed, seed=seed + 2))
    out = [S.apply(u).cpu().numpy()]
    if S.num_levels > 1:  # (a one-level hierarchy has no fine smoother)
        out.append(S.level_smooth(0, b).cpu().numpy())
        out.append(S.level_smooth(0, b, x.clone()).cpu().numpy())
        out.append(S.vcycle(b).cpu().numpy())
    return out


@pytest.mark.parametrize("name,nx,ny,nz,dens,p,mask", CASES)
@pytest.mark.parametrize("smoother", ["chebyshev", "jacobi"])
def test_pair_tiles_are_bitwise_equal_to_single_column(name, nx, ny, nz, dens, p, mask, smoother):
    rho, fixed = _case(nx, ny, nz, dens, mask)
    levels = 2 if min(nx, ny, nz) >= 2 else 1
    S = gpu_solver(rho, p, fixed=fixed, levels=levels, smoother=smoother, degree=3, omega=0.5,
                   coarse_smoother=None)
    assert S.num_levels == levels
    NZ = nz + 1
    try:
        refs = {}
        for tile in ["32x8", "16x16"]:
            S.set_fine_plan(tile, NZ)
            refs[tile] = _outputs(S, fixed, 17)
        for a, b in zip(refs["32x8"], refs["16x16"]):
            assert np.array_equal(a, b)
        ref = refs["16x16"]
        for tile in PAIR_TILES:
            for zc in sorted({1, 4, 5, NZ}):
                S.set_fine_plan(tile, zc)
                got = _outputs(S, fixed, 17)
                for k, (g, r) in enumerate(zip(got, ref)):
                    assert np.array_equal(g, r), f"{tile} zchunk {zc} output {k}"
    finally:
        S.set_fine_plan(None)


def test_pair_apply_matches_oracle():
    nx, ny, nz = 37, 13, 9
    rho = inputs.filtered_random_density(nx, ny, nz, 7)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    S = gpu_solver(rho, 3.0, levels=0, smoother="jacobi", coarse_smoother=None, omega=0.5)
    u = inputs.random_free_vector(fixed, seed=11)
    u_in = u.copy()
    u_in[fixed == 1] = 1e3  # values on fixed DOFs must be ignored
    try:
        S.set_fine_plan("pair-8x16", 4)
        y = S.apply(_t(u_in)).cpu().numpy()
    finally:
        S.set_fine_plan(None)
    yref = fem.matfree_apply(fem.Grid(nx, ny, nz), fem.moduli(rho, 3.0), fem.element_stiffness(0.3),
                             u.astype(np.float64))
    yref[fixed == 1] = 0.0
    assert np.all(y[fixed == 1] == 0.0)
    assert rel_l2(y, yref) < 1e-6


@pytest.mark.parametrize("cfg_name", ["c0", "c1"])
@pytest.mark.parametrize("tile", PAIR_TILES)
def test_pair_tiles_solve_like_single_column(cfg_name, tile):
    cfg = inputs.CONFIGS[cfg_name]
    S = gpu_solver(cfg.rho(), cfg.p, **config_opts(cfg))
    f = _t(cfg.load(), torch.float64)
    try:
        S.set_fine_plan("16x16", cfg.nz + 1)
        u1, i1 = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
        S.set_fine_plan(tile, 4)
        u2, i2 = S.solve(f, None, tol=cfg.tol, maxit=cfg.maxit)
    finally:
        S.set_fine_plan(None)
    assert i1["status"] == 0 and i2["status"] == 0
    assert i2["rel_residual"] <= cfg.tol and abs(i2["iterations"] - i1["iterations"]) <= 1
    assert rel_l2(u2.cpu().numpy(), u1.cpu().numpy()) < 1e-5


def test_set_fine_plan_rejects_bad_plans():
    from paper_2604_26441_b300 import gmg
    cfg = inputs.CONFIGS["c0"]
    S = gpu_solver(cfg.rho(), cfg.p, **config_opts(cfg))
    for tile, zc in [(5, 4), (2, 0), (0, -1)]:
        with pytest.raises(gmg.GMGError):
            S.set_fine_plan(tile, zc)
    S.set_fine_plan(None)
