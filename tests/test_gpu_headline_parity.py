"""The 100^3 cantilever (1,000,000 elements, 3,060,300 free DOF) solved on the
GPU with exactly the options the throughput benchmark times, against the FP64
CPU oracle's own GMG-PCG on the same hierarchy recipe.

Checked, with the tolerances of the other solve tests (Sec. "Outer Krylov
Solver and Convergence Statement"; Table phase1, check M1):
  - pass/fail under the 200-iteration cap is the same on both sides;
  - the GPU's iteration count is within max(2, 10 %) of the oracle's;
  - the oracle recomputes the GPU solution's FP64 true residual (<= 1e-6);
  - the GPU displacement is within 1e-5 relative L2 of the oracle's reference
    solution u*, which is the oracle's PCG continued to a 1e-12 true residual.

The oracle runs matrix-free on the fine level (its level-1 operator comes from
the element-wise formula, Eq. galerkin_level1, summed batch by batch), which
keeps its memory near 3 GB; it takes a few minutes of host time.
"""

import numpy as np
import pytest

from oracle import fem, solver as so
from paper_2604_26441_b300 import inputs

from gpu_helpers import config_opts, gpu_solver, oracle_hierarchy, oracle_spec_from_opts, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_26441_b300 import build
    build.build_library()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_headline_100cube_matches_oracle():
    c = inputs.CONFIGS["c2"]
    rho, fixed, f = c.rho(), c.fixed(), c.load()
    opts = config_opts(c)
    # GPU: the benchmark's configuration (5 levels, Chebyshev degree 3 everywhere)
    S = gpu_solver(rho, c.p, **opts)
    u_gpu, info = S.solve(torch.from_numpy(f).cuda(), tol=c.tol, maxit=c.maxit)
    u_gpu = u_gpu.cpu().numpy()
    S.close()
    # oracle: same hierarchy recipe and smoother, FP64 throughout
    H, E = oracle_hierarchy(rho, c.p, fixed, c.levels, matrix_free_fine=True)
    spec = oracle_spec_from_opts(opts)
    u_or, res = so.gmg_pcg(H, f, spec, tol=c.tol, maxit=c.maxit)
    assert (info["status"] == 0) == (res.status == so.OK), (info, res.status, res.iterations)
    assert res.status == so.OK
    assert abs(info["iterations"] - res.iterations) <= max(2, 0.1 * res.iterations), \
        (info["iterations"], res.iterations)
    # the oracle's own residual of the GPU solution
    free = fem.free_dofs(fixed)
    r = f - fem.matfree_apply(fem.Grid(c.nx, c.ny, c.nz), E, fem.element_stiffness(0.3), u_gpu)
    rel = np.linalg.norm(r[free]) / np.linalg.norm(f[free])
    assert rel <= c.tol, rel
    assert abs(info["rel_residual"] - rel) < 1e-9
    assert np.all(u_gpu[fixed == 1] == 0)
    # reference solution: the oracle's PCG continued from its own iterate to 1e-12
    lev = H[0]
    ref = so.pcg(lev.apply, lambda v: so.vcycle(H, v, spec), f[lev.free], u_or[lev.free], 1e-12, 2000)
    assert ref.status == so.OK, ref.rel_residual
    u_ref = np.zeros_like(u_or)
    u_ref[lev.free] = ref.x
    err = rel_l2(u_gpu, u_ref)
    print(f"100^3: GPU {info['iterations']} iterations, oracle {res.iterations}; "
          f"GPU residual {rel:.3e}; displacement error vs the 1e-12 solution {err:.3e}")
    assert err < 1e-5, err
