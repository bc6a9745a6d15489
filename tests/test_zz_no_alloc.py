"""The allocation-free residual entry point against the handle-based one.

gmg_residual64_noalloc serves callers that cannot call cudaMalloc (a framework
that owns all device memory through its own pool, a plug-in that must not grow
the device footprint, a check run when the device is full).  It must give the
same FP64 true residual as gmg_residual64, call after call, while keeping its
scratch in a static device array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_2604_26441_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_26441_b300 import build
    build.build_library()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _moduli(rho, p, E0=1.0, Emin=1e-9):
    r = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).cuda().double().reshape(-1)
    return Emin + (E0 - Emin) * r ** p


def _clamp_mask(nx, ny, nz):
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=np.uint8)
    m[:, :, 0] = 7
    return torch.from_numpy(m.reshape(-1)).cuda()


@pytest.mark.parametrize("dims,dens", [((16, 8, 8), "uniform"), ((37, 13, 9), "filtered"), ((100, 100, 100), "uniform")])
def test_noalloc_residual_matches_handle_entry_point(dims, dens):
    from paper_2604_26441_b300 import gmg
    nx, ny, nz = dims
    rho = inputs.uniform_density(nx, ny, nz) if dens == "uniform" else inputs.filtered_random_density(nx, ny, nz, 3)
    levels = 0
    S = gmg.Solver(torch.from_numpy(rho).cuda(), p=3.0,
                   opts=gmg.options(levels=levels, smoother="jacobi", coarse_smoother=None, omega=0.4))
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    f = torch.from_numpy(inputs.tip_edge_load(nx, ny, nz)).cuda()
    rng = np.random.default_rng(7)
    u = torch.from_numpy(rng.uniform(-1, 1, 3 * S.nn) * (fixed == 0)).cuda()
    r_ref = torch.empty_like(f)
    rel_ref = S.residual64(f, u, r_ref)
    E = _moduli(rho, 3.0)
    mask = _clamp_mask(nx, ny, nz)
    for call in range(2):  # two calls in a row share the static scratch
        r = torch.full_like(f, float("nan"))
        rel = gmg.residual64_noalloc(dims, E, mask, f, u, r)
        assert abs(rel - rel_ref) <= 1e-12 * rel_ref, (call, rel, rel_ref)
        diff = torch.linalg.vector_norm(r - r_ref) / torch.linalg.vector_norm(r_ref)
        assert float(diff) <= 1e-12, (call, float(diff))
    S.close()


def test_noalloc_rejects_oversized_grid():
    from paper_2604_26441_b300 import gmg
    lib = gmg.load_library()
    g = gmg._Grid(8191, 8191, 3)  # 256 x 2048 x 2 blocks > 65,536
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rel = ctypes.c_double(-1.0)
    rc = lib.gmg_residual64_noalloc(ctypes.byref(g), p, p, 0.3, p, p, None, ctypes.byref(rel), None)
    assert rc == -1
    assert b"65536" in lib.gmg_last_error()
    assert rel.value == -1.0


def test_noalloc_rejects_node_count_beyond_int32_dofs():
    """Sizes are checked in 64-bit before any launch: an element count at the
    32-bit limit (whose node count nx + 1 overflows int) and a grid whose
    3 x node count passes 2^31 (the limit of gmg_setup) are both refused."""
    from paper_2604_26441_b300 import gmg
    lib = gmg.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    for dims in [(2147483647, 1, 1), (1000, 1000, 1000)]:
        g = gmg._Grid(*dims)
        rel = ctypes.c_double(-1.0)
        rc = lib.gmg_residual64_noalloc(ctypes.byref(g), p, p, 0.3, p, p, None, ctypes.byref(rel), None)
        assert rc == -1, dims
        assert rel.value == -1.0


def test_noalloc_zero_load_has_a_defined_result():
    """f = 0 on every free DOF: the relative residual is 0 for u = 0 and +inf
    for a nonzero u (no NaN)."""
    from paper_2604_26441_b300 import gmg
    nx, ny, nz = 16, 8, 8
    E = _moduli(inputs.uniform_density(nx, ny, nz), 3.0)
    mask = _clamp_mask(nx, ny, nz)
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    r = torch.full_like(f, float("nan"))
    assert gmg.residual64_noalloc((nx, ny, nz), E, mask, f, u, r) == 0.0
    assert float(r.abs().max()) == 0.0
    fixed = torch.from_numpy(inputs.clamp_xmin_mask(nx, ny, nz)).cuda()
    u = torch.where(fixed == 0, 1e-3, 0.0).double()
    assert gmg.residual64_noalloc((nx, ny, nz), E, mask, f, u, r) == float("inf")
