"""Parity cases run against the bounds-checked build of the library.

Run as a script in a fresh process with GMG_LIBRARY naming the checked build
(tests/test_gpu_checked.py does this).  Each case compares the CUDA path with
the FP64 oracle as the main parity tests do; after every case the device-side
bounds words must be clear.  Prints one JSON line per case.
"""

import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from gpu_helpers import config_opts, gpu_solver, oracle_hierarchy, oracle_spec_from_opts, rel_l2  # noqa: E402
from oracle import fem, solver as so  # noqa: E402
from paper_2604_26441_b300 import gmg, inputs  # noqa: E402


def main() -> None:
    lib = gmg.load_library()
    assert lib.gmg_bounds_checked() == 1, "not the bounds-checked build"
    assert os.path.abspath(gmg.LIB_PATH).endswith("libgmg_b300_checked.so")
    for name, p in (("c0", 3.0), ("c1", 3.0)):
        c = inputs.CONFIGS[name]
        rho, fixed, f = c.rho(), c.fixed(), c.load()
        opts = config_opts(c)
        S = gpu_solver(rho, p, **opts)
        # operator apply
        u = inputs.random_free_vector(fixed, seed=11)
        y = S.apply(torch.from_numpy(u).float().cuda()).cpu().numpy()
        g = fem.Grid(c.nx, c.ny, c.nz)
        E = fem.moduli(rho, p)
        yref = fem.matfree_apply(g, E, fem.element_stiffness(0.3), u.astype(np.float32).astype(np.float64))
        yref[fixed == 1] = 0.0
        err_apply = rel_l2(y, yref)
        site = lib.gmg_bounds_site()
        # a V-cycle and a restriction / prolongation round trip
        r = torch.from_numpy(inputs.random_free_vector(fixed, seed=13)).float().cuda()
        S.vcycle(r)
        coarse = S.restrict(0, r)
        fine = torch.zeros_like(r)
        S.prolong_add(0, coarse, fine)
        site = site or lib.gmg_bounds_site()
        # a full solve against the oracle's GMG-PCG
        H, _ = oracle_hierarchy(rho, p, fixed, opts["levels"])
        u_or, res = so.gmg_pcg(H, f, oracle_spec_from_opts(opts), tol=1e-6, maxit=200)
        u_gpu, info = S.solve(torch.from_numpy(f).cuda(), tol=1e-6, maxit=200)
        site = site or lib.gmg_bounds_site()
        ue = so.exact_solve(H, f, oracle_spec_from_opts(opts))
        S.close()
        print(json.dumps({"case": name, "site": int(site), "apply_err": err_apply, "status": info["status"],
                          "iterations": info["iterations"], "oracle_iterations": res.iterations,
                          "oracle_ok": res.status == so.OK,
                          "u_err": rel_l2(u_gpu.cpu().numpy(), ue)}), flush=True)


if __name__ == "__main__":
    main()
