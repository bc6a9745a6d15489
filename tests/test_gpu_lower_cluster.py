"""The bottom of the V-cycle as one thread-block cluster launch (`lower_cluster`)
against the per-level kernels it replaces.

With the option on (opt-in) and a hierarchy of at least four levels whose
last assembled level fits the cluster's shared memory, the smoothing passes,
residual and transfers of that level and the coarsest solve run as one launch
(the inverse applied in double-float).  The steps' arithmetic is the per-level
kernels' up to the summation order of the operator rows and of the
restriction, so V-cycle outputs agree to FP32 rounding, solves take the same
iteration counts within one and return the same solution to 1e-5, and the
oracle's FP64 residual of the answer meets the tolerance.
"""

import numpy as np
import pytest

from oracle import fem
from paper_2604_26441_b300 import gmg, inputs

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


def _vcycle_launches(S, r):
    n0 = gmg.kernel_launches()
    S.vcycle(r)
    torch.cuda.synchronize()
    return gmg.kernel_launches() - n0


# (name, nx, ny, nz, levels, density): the 40^3 and 100^3 configurations and a
# ragged grid whose coarse sizes are odd in every direction
CASES = [("c1", 40, 40, 40, 4, "filtered"), ("ragged", 37, 13, 9, 4, "filtered"), ("c2", 100, 100, 100, 5, "uniform")]


@pytest.mark.parametrize("name,nx,ny,nz,levels,dens", CASES)
def test_cluster_vcycle_and_solve_match_per_level(name, nx, ny, nz, levels, dens):
    rho = (inputs.filtered_random_density(nx, ny, nz, 7) if dens == "filtered"
           else inputs.CONFIGS[name].rho())
    opts = dict(levels=levels, smoother="chebyshev", degree=3, coarse_smoother=None, coarse_degree=None, omega=0.5,
                coarse_omega=None)
    S_on = gpu_solver(rho, 3.0, **opts, lower_cluster=True)
    S_off = gpu_solver(rho, 3.0, **opts)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    r = _t(inputs.random_free_vector(fixed, seed=3))
    # one launch replaces the ~10 of the per-level bottom
    assert _vcycle_launches(S_on, r) < _vcycle_launches(S_off, r) - 5
    z_on = S_on.vcycle(r).cpu().numpy()
    z_off = S_off.vcycle(r).cpu().numpy()
    assert rel_l2(z_on, z_off) < 1e-5
    # bitwise repeatable
    assert np.array_equal(z_on, S_on.vcycle(r).cpu().numpy())
    f = inputs.rotated_tip_edge_load(nx, ny, nz, 0)
    u_on, i_on = S_on.solve(_t(f, torch.float64))
    u_off, i_off = S_off.solve(_t(f, torch.float64))
    assert i_on["status"] == 0 and i_off["status"] == 0
    assert abs(i_on["iterations"] - i_off["iterations"]) <= 1
    assert rel_l2(u_on.cpu().numpy(), u_off.cpu().numpy()) < 1e-5
    if nx * ny * nz <= 64000:
        u = u_on.cpu().numpy()
        res = f - fem.matfree_apply(fem.Grid(nx, ny, nz), fem.moduli(rho, 3.0), fem.element_stiffness(0.3), u)
        free = fem.free_dofs(fixed)
        assert np.linalg.norm(res[free]) / np.linalg.norm(f[free]) < 1e-6


def test_cluster_path_with_w_cycle_and_graph_loop():
    """The W-cycle's second visit of the level starts from the first visit's
    result and runs the per-level kernels; the device-resident loop and the
    host-driven loop stay bitwise equal with the cluster launch in the graph."""
    c = inputs.CONFIGS["c1"]
    rho = c.rho()
    f = _t(c.load(), torch.float64)
    S_w = gpu_solver(rho, c.p, **config_opts(c), cycle="W", lower_cluster=True)
    S_w_off = gpu_solver(rho, c.p, **config_opts(c), cycle="W")
    u_w, i_w = S_w.solve(f)
    u_w2, i_w2 = S_w_off.solve(f)
    assert i_w["status"] == 0 and abs(i_w["iterations"] - i_w2["iterations"]) <= 1
    assert rel_l2(u_w.cpu().numpy(), u_w2.cpu().numpy()) < 1e-5
    S_g = gpu_solver(rho, c.p, **config_opts(c), lower_cluster=True)
    S_h = gpu_solver(rho, c.p, **config_opts(c), device_loop=False, lower_cluster=True)
    u_g, i_g = S_g.solve(f)
    u_h, i_h = S_h.solve(f)
    assert i_g["iterations"] == i_h["iterations"]
    assert np.array_equal(u_g.cpu().numpy(), u_h.cpu().numpy())


def test_cluster_path_in_clones():
    """Clones share the split inverse and keep their own level vectors: a clone's
    solves equal the source's bit for bit."""
    c = inputs.CONFIGS["c1"]
    rho = c.rho()
    base = gpu_solver(rho, c.p, **config_opts(c), lower_cluster=True)
    loads = [inputs.rotated_tip_edge_load(c.nx, c.ny, c.nz, k, nrhs=16) for k in (1, 6)]
    ref = [base.solve(_t(l, torch.float64)) for l in loads]
    clone = base.clone()
    for l, (u_ref, i_ref) in zip(loads, ref):
        u, i = clone.solve(_t(l, torch.float64))
        assert i["iterations"] == i_ref["iterations"]
        assert np.array_equal(u.cpu().numpy(), u_ref.cpu().numpy())
