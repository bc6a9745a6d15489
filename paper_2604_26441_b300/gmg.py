"""Python binding of the C ABI in include/gmg.h (ctypes; argument marshalling only).

Every numerical step runs in the CUDA library ``libgmg_b300.so`` built in-tree by
``paper_2604_26441_b300.build``.  PyTorch supplies device memory and the stream;
if the library is missing this module raises instead of computing anything
another way.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# GMG_LIBRARY may name another build of the same library (e.g. the
# bounds-checked libgmg_b300_checked.so built with -DGMG_CHECKED)
LIB_PATH = os.environ.get("GMG_LIBRARY") or os.path.join(HERE, "libgmg_b300.so")

GMG_OK, GMG_NOT_CONVERGED, GMG_NONFINITE = 0, 1, 2
GMG_TIMEOUT = -7
BC_CLAMP_XMIN, BC_MASK = 0, 1
JACOBI, CHEBYSHEV = 0, 1
_KINDS = {"jacobi": JACOBI, "chebyshev": CHEBYSHEV}


class GMGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gmg error {code}: {msg}")
        self.code = code


# arithmetic of the fine-level smoother's element contraction (gmg_options.fine_smoother)
FINE_SMOOTHERS = {"fp32": 0, "bf16x3": 1, "bf16": 2}
# assembled-level kernels (gmg_options.bsr_kernel, gmg_tuning.bsr_kind); kind 6 is level 1
# applied matrix-free from the fine moduli (chosen where it equals the assembled operator)
BSR_KINDS = ["streaming", "k-split-8", "k-split-2", "k-split-4", "k-split-16", "k-split-32", "matrix-free"]
# fine kernel tiles (GMG_FINE_TILE_*): threads per block, "pair" = two element columns a thread
FINE_TILES = ["32x8", "16x16", "pair-8x16", "pair-16x8", "pair-16x16"]


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class _BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("fixed", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("smoother", ctypes.c_int), ("degree", ctypes.c_int),
                ("coarse_smoother", ctypes.c_int), ("coarse_degree", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_omega", ctypes.c_double),
                ("cheb_alpha", ctypes.c_double), ("lambda_safety", ctypes.c_double),
                ("power_iters_fine", ctypes.c_int), ("power_iters_coarse", ctypes.c_int),
                ("chol_cutoff", ctypes.c_int), ("fused_coarse_nodes", ctypes.c_int),
                ("bsr_tma_nodes", ctypes.c_int), ("device_loop", ctypes.c_int),
                ("ir_factor", ctypes.c_double),
                ("fine_smoother", ctypes.c_int),
                ("cycle_index", ctypes.c_int), ("outer", ctypes.c_int), ("restart", ctypes.c_int),
                ("bsr_kernel", ctypes.c_int), ("stream", ctypes.c_void_p), ("spin_limit", ctypes.c_longlong),
                ("coarse_pcg_steps", ctypes.c_int), ("lower_cluster", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("replacements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("rel_residual_recursive", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("setup_ms", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [("fine_tile", ctypes.c_int), ("fine_zchunk", ctypes.c_int), ("model_tile", ctypes.c_int),
                ("model_zchunk", ctypes.c_int), ("fine_candidates", ctypes.c_int),
                ("fine_us", ctypes.c_double), ("model_us", ctypes.c_double),
                ("bsr_kind", ctypes.c_int * 16), ("bsr_us", ctypes.c_double * 16),
                ("bsr_alt_us", ctypes.c_double * 16)]


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "gmg_default_options": (None, [ctypes.POINTER(_Options)]),
    "gmg_setup": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_Grid), _P, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_BC),
                                 ctypes.POINTER(_Options)]),
    "gmg_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Info)]),
    "gmg_apply": (ctypes.c_int, [_P, _P, _P]),
    "gmg_destroy": (None, [_P]),
    "gmg_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "gmg_set_spin_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "gmg_bounds_checked": (ctypes.c_int, []),
    "gmg_bounds_site": (ctypes.c_uint, []),
    "gmg_last_error": (ctypes.c_char_p, []),
    "gmg_kernel_launches": (ctypes.c_ulonglong, []),
    "gmg_num_levels": (ctypes.c_int, [_P]),
    "gmg_level_dims": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gmg_get_mask": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "gmg_get_bsr": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "gmg_get_lambda": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gmg_set_lambda": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "gmg_level_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_level_smooth": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "gmg_restrict": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_fine_pass": (ctypes.c_int, [_P, ctypes.c_int]),
    "gmg_prolong_add": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_coarse_solve": (ctypes.c_int, [_P, _P, _P]),
    "gmg_vcycle": (ctypes.c_int, [_P, _P, _P]),
    "gmg_kappa_eff": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gmg_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_Tuning)]),
    "gmg_set_fine_plan": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gmg_clone": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "gmg_solve_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                       ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Info)]),
    "gmg_solve_multi": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_double,
                                       ctypes.c_int, ctypes.POINTER(_Info)]),
    "gmg_apply_multi": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "gmg_set_multi_kernel": (ctypes.c_int, [_P, ctypes.c_int]),
    "gmg_multi_fine_pass": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gmg_vcycle_symmetry": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "gmg_residual64": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "gmg_residual64_noalloc": (ctypes.c_int, [ctypes.POINTER(_Grid), _P, _P, ctypes.c_double, _P, _P, _P,
                                              ctypes.POINTER(ctypes.c_double), _P]),
    # learned warm start (include/gmg_warmnet.h)
    "gmg_net_num_params": (ctypes.c_longlong, []),
    "gmg_net_layer_shape": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gmg_net_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P]),
    "gmg_net_set_params": (ctypes.c_int, [_P, _P]),
    "gmg_net_get_params": (ctypes.c_int, [_P, _P]),
    "gmg_net_get_grads": (ctypes.c_int, [_P, _P]),
    "gmg_net_forward": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "gmg_net_train_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_float,
                                          ctypes.c_float, _P]),
    "gmg_net_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "gmg_net_target": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "gmg_warm_start": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "gmg_net_destroy": (None, [_P]),
    "gmg_net_set_arith": (ctypes.c_int, [_P, ctypes.c_int]),
    "gmg_net_status": (ctypes.c_int, [_P]),
}


def exported_symbols() -> list[str]:
    return list(_SIGS)


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with "
                           "`python -m paper_2604_26441_b300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().gmg_kernel_launches())


def _check(rc: int, allow=(GMG_OK,)) -> int:
    if rc in allow:
        return rc
    lib = load_library()
    raise GMGError(rc, f"{lib.gmg_status_str(rc).decode()}: {lib.gmg_last_error().decode()}")


def _ptr(t, dtype, numel: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def options(levels: int = 4, smoother: str = "chebyshev", degree: int = 2, coarse_smoother: str | None = "jacobi",
            coarse_degree: int | None = 2, omega: float = 0.5, coarse_omega: float | None = 0.5,
            alpha: float = 1.0 / 30.0, lambda_safety: float = 1.1, power_iters_fine: int = 20,
            power_iters_coarse: int = 10, chol_cutoff: int = 5000, fused_coarse_nodes: int = 0,
            bsr_tma_nodes: int = 0, device_loop: bool = True, ir_factor: float = 0.0,
            fine_smoother: str = "fp32", cycle: str = "V", outer: str = "pcg", restart: int = 32,
            bsr_kernel: int = -1, stream: int | None = None, spin_limit: int = 1 << 24,
            coarse_pcg_steps: int = 80, lower_cluster: bool = False) -> _Options:
    o = _Options()
    load_library().gmg_default_options(ctypes.byref(o))
    o.levels = levels
    o.smoother = _KINDS[smoother]
    o.degree = degree
    o.coarse_smoother = -1 if coarse_smoother is None else _KINDS[coarse_smoother]
    o.coarse_degree = -1 if coarse_degree is None else coarse_degree
    o.omega = omega
    o.coarse_omega = -1.0 if coarse_omega is None else coarse_omega
    o.cheb_alpha = alpha
    o.lambda_safety = lambda_safety
    o.power_iters_fine = power_iters_fine
    o.power_iters_coarse = power_iters_coarse
    o.chol_cutoff = chol_cutoff
    o.fused_coarse_nodes = fused_coarse_nodes
    o.bsr_tma_nodes = bsr_tma_nodes
    o.device_loop = 1 if device_loop else 0
    o.ir_factor = ir_factor
    o.fine_smoother = FINE_SMOOTHERS[fine_smoother]
    o.cycle_index = {"V": 1, "W": 2}[cycle]
    o.outer = {"pcg": 0, "fgmres": 1}[outer]
    o.restart = restart
    o.bsr_kernel = bsr_kernel
    o.stream = stream
    o.spin_limit = spin_limit
    o.coarse_pcg_steps = coarse_pcg_steps
    o.lower_cluster = 1 if lower_cluster else 0
    return o


def config_options(cfg, stream: int | None = None, fused_coarse_nodes: int = 0,
                   bsr_tma_nodes: int = 0, device_loop: bool = True, ir_factor: float = 0.0,
                   fine_smoother: str = "fp32", cycle: str = "V", outer: str = "pcg",
                   restart: int = 32, bsr_kernel: int = -1, lower_cluster: bool = False) -> _Options:
    """Options for one of the synthetic configurations in ``inputs.CONFIGS``."""
    return options(levels=cfg.levels, smoother=cfg.smoother, degree=cfg.degree, coarse_smoother=None,
                   coarse_degree=None, omega=cfg.omega, coarse_omega=None, fused_coarse_nodes=fused_coarse_nodes,
                   bsr_tma_nodes=bsr_tma_nodes, device_loop=device_loop, ir_factor=ir_factor,
                   fine_smoother=fine_smoother, cycle=cycle, outer=outer, restart=restart, bsr_kernel=bsr_kernel,
                   stream=stream, lower_cluster=lower_cluster)


def residual64_noalloc(dims, E, mask, f, u, r=None, nu: float = 0.3, stream: int | None = None) -> float:
    """FP64 relative true residual through the allocation-free entry point: no
    handle, no device allocation inside the library (the caller's tensors are
    the only device memory it touches besides its static scratch)."""
    import torch
    lib = load_library()
    nx, ny, nz = dims
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    g = _Grid(nx, ny, nz)
    rel = ctypes.c_double()
    rp = None if r is None else _ptr(r, torch.float64, 3 * nn, "r")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.gmg_residual64_noalloc(ctypes.byref(g), _ptr(E, torch.float64, nx * ny * nz, "E"),
                                      _ptr(mask, torch.uint8, nn, "mask"), nu, _ptr(f, torch.float64, 3 * nn, "f"),
                                      _ptr(u, torch.float64, 3 * nn, "u"), rp, ctypes.byref(rel), stream))
    return rel.value


class Solver:
    """A GMG-PCG hierarchy for one frozen density field on one structured grid."""

    def __init__(self, rho, p: float = 3.0, E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3,
                 fixed: np.ndarray | None = None, opts: _Options | None = None):
        import torch
        lib = load_library()
        if rho.dim() != 3:
            raise ValueError("rho must have shape (nz, ny, nx)")
        nz, ny, nx = (int(s) for s in rho.shape)
        self.dims = (nx, ny, nz)
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        g = _Grid(nx, ny, nz)
        if fixed is None:
            bc = _BC(BC_CLAMP_XMIN, None)
            self._fixed_host = None
        else:
            self._fixed_host = np.ascontiguousarray(fixed, dtype=np.uint8)
            if self._fixed_host.size != 3 * self.nn:
                raise ValueError("fixed must have 3*n_nodes entries")
            bc = _BC(BC_MASK, self._fixed_host.ctypes.data)
        if opts is None:
            opts = options()
        if opts.stream is None:
            opts.stream = torch.cuda.current_stream().cuda_stream
        self.stream = opts.stream
        h = ctypes.c_void_p()
        rp = _ptr(rho, torch.float32, nx * ny * nz, "rho")
        _check(lib.gmg_setup(ctypes.byref(h), ctypes.byref(g), rp, p, E0, Emin, nu, ctypes.byref(bc),
                             ctypes.byref(opts)))
        self._h = h
        self._lib = lib

    # -- lifetime
    def clone(self) -> "Solver":
        """A solver sharing this hierarchy with a workspace of its own (for
        further right-hand sides, e.g. in solve_batch).  Keeps this solver
        alive while the clone exists."""
        c = object.__new__(Solver)
        c.dims, c.nn, c.stream, c._fixed_host, c._lib = self.dims, self.nn, self.stream, self._fixed_host, self._lib
        c._source = self
        h = ctypes.c_void_p()
        _check(self._lib.gmg_clone(self._h, ctypes.byref(h)))
        c._h = h
        return c

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- geometry
    @property
    def num_levels(self) -> int:
        return self._lib.gmg_num_levels(self._h)

    def level_dims(self, level: int) -> tuple[int, int, int]:
        d = (ctypes.c_int * 3)()
        _check(self._lib.gmg_level_dims(self._h, level, d))
        return int(d[0]), int(d[1]), int(d[2])

    def level_nodes(self, level: int) -> int:
        nx, ny, nz = self.level_dims(level)
        return (nx + 1) * (ny + 1) * (nz + 1)

    # -- main entry points
    def apply(self, u, y=None):
        import torch
        if y is None:
            y = torch.empty_like(u)
        _check(self._lib.gmg_apply(self._h, _ptr(u, torch.float32, 3 * self.nn, "u"),
                                   _ptr(y, torch.float32, 3 * self.nn, "y")))
        return y

    def solve(self, f, u=None, tol: float = 1e-6, maxit: int = 200):
        import torch
        if u is None:
            u = torch.zeros_like(f)
        info = _Info()
        rc = self._lib.gmg_solve(self._h, _ptr(f, torch.float64, 3 * self.nn, "f"),
                                 _ptr(u, torch.float64, 3 * self.nn, "u"), tol, maxit, ctypes.byref(info))
        _check(rc, allow=(GMG_OK, GMG_NOT_CONVERGED, GMG_NONFINITE))
        return u, {"status": info.status, "iterations": info.iterations, "replacements": info.replacements,
                   "rel_residual": info.rel_residual, "rel_residual_recursive": info.rel_residual_recursive,
                   "solve_ms": info.solve_ms, "setup_ms": info.setup_ms}

    def solve_multi(self, fs, us=None, tol: float = 1e-6, maxit: int = 200):
        """Solves up to 16 loads fs[l] (device FP64) on this hierarchy together
        (gmg_solve_multi): one PCG loop with per-load step lengths and stopping
        decisions; us[l] initial guesses (zeros when None).  Returns (us, infos)."""
        import torch
        n = len(fs)
        if us is None:
            us = [torch.zeros_like(f) for f in fs]
        if len(us) != n or not 1 <= n <= 16:
            raise ValueError("1..16 loads, one iterate per load")
        fp = (_P * n)(*[_ptr(f, torch.float64, 3 * self.nn, "f") for f in fs])
        up = (_P * n)(*[_ptr(u, torch.float64, 3 * self.nn, "u") for u in us])
        infos = (_Info * n)()
        rc = self._lib.gmg_solve_multi(self._h, n, fp, up, tol, maxit, infos)
        _check(rc, allow=(GMG_OK, GMG_NOT_CONVERGED, GMG_NONFINITE))
        return us, [_info_dict(i) for i in infos]

    def apply_multi(self, us, ys=None):
        """ys[l] = K us[l] for up to 16 loads (device FP32) in one launch of the
        multi-load level-0 operator (gmg_apply_multi)."""
        import torch
        n = len(us)
        if ys is None:
            ys = [torch.empty_like(u) for u in us]
        if len(ys) != n or not 1 <= n <= 16:
            raise ValueError("1..16 loads, one output per load")
        up = (_P * n)(*[_ptr(u, torch.float32, 3 * self.nn, "u") for u in us])
        yp = (_P * n)(*[_ptr(y, torch.float32, 3 * self.nn, "y") for y in ys])
        _check(self._lib.gmg_apply_multi(self._h, n, up, yp))
        return ys

    def multi_fine_pass(self, what: str = "apply", nl: int = 16) -> None:
        """One multi-load level-0 operator pass on this handle's own multi-load
        vectors ("apply" or "smooth"), for timing (gmg_multi_fine_pass)."""
        _check(self._lib.gmg_multi_fine_pass(self._h, nl, {"apply": 0, "smooth": 1}[what]))

    def set_multi_kernel(self, kind: str) -> None:
        """Level-0 operator of the multi-load path: "simt" (CUDA cores) or
        "tc" (tensor cores)."""
        _check(self._lib.gmg_set_multi_kernel(self._h, {"simt": 0, "tc": 1}[kind]))

    def set_spin_limit(self, polls: int) -> None:
        """Polls a block of the fused lower V-cycle makes at a grid barrier
        before it gives up (gmg_set_spin_limit); drops captured solve graphs."""
        _check(self._lib.gmg_set_spin_limit(self._h, int(polls)))

    def autotune(self, reps: int = 5) -> dict:
        """Times the fine kernel's launch shapes and each assembled level's
        SpMV kernel on this handle and keeps the fastest (gmg_autotune);
        reps = 0 returns to the untuned choices."""
        t = _Tuning()
        _check(self._lib.gmg_autotune(self._h, reps, ctypes.byref(t)))
        L = self.num_levels
        return {"fine_tile": FINE_TILES[t.fine_tile], "fine_zchunk": t.fine_zchunk,
                "model_tile": FINE_TILES[t.model_tile], "model_zchunk": t.model_zchunk,
                "fine_candidates": t.fine_candidates, "fine_us": t.fine_us, "model_us": t.model_us,
                "bsr": [{"level": l, "kind": BSR_KINDS[t.bsr_kind[l]],
                         "us": t.bsr_us[l],
                         "other_us": t.bsr_alt_us[l]} for l in range(1, min(L, 16)) if t.bsr_kind[l] >= 0]}

    def set_fine_plan(self, tile, zchunk: int = 0) -> None:
        """Pins the fine kernel's tile (a FINE_TILES name or index) and node
        planes per block for this fine grid (gmg_set_fine_plan); tile None or
        < 0 returns to the cost model's plan."""
        if tile is None:
            tile = -1
        elif isinstance(tile, str):
            tile = FINE_TILES.index(tile)
        _check(self._lib.gmg_set_fine_plan(self._h, int(tile), int(zchunk)))

    # -- per-step entry points
    def get_mask(self, level: int) -> np.ndarray:
        out = np.empty(self.level_nodes(level), dtype=np.uint8)
        _check(self._lib.gmg_get_mask(self._h, level, out.ctypes.data))
        return out

    def get_bsr(self, level: int) -> np.ndarray:
        out = np.empty(243 * self.level_nodes(level), dtype=np.float64)
        _check(self._lib.gmg_get_bsr(self._h, level, out.ctypes.data))
        return out.reshape(243, -1)

    def get_lambda(self, level: int) -> float:
        v = ctypes.c_double()
        _check(self._lib.gmg_get_lambda(self._h, level, ctypes.byref(v)))
        return v.value

    def set_lambda(self, level: int, lam: float):
        _check(self._lib.gmg_set_lambda(self._h, level, lam))

    def level_apply(self, level: int, x, y=None):
        import torch
        n = 3 * self.level_nodes(level)
        if y is None:
            y = torch.empty_like(x)
        _check(self._lib.gmg_level_apply(self._h, level, _ptr(x, torch.float32, n, "x"),
                                         _ptr(y, torch.float32, n, "y")))
        return y

    def level_smooth(self, level: int, b, x=None):
        import torch
        n = 3 * self.level_nodes(level)
        zero = x is None
        if zero:
            x = torch.zeros_like(b)
        _check(self._lib.gmg_level_smooth(self._h, level, _ptr(b, torch.float32, n, "b"),
                                          _ptr(x, torch.float32, n, "x"), int(zero)))
        return x

    def fine_pass(self, what: str = "smooth") -> None:
        """The fine-level operator on the handle's own vectors ("apply": one
        y = K x; "smooth": one smoothing pass), for timing the fused fine kernel
        without repacking caller vectors (gmg_fine_pass)."""
        _check(self._lib.gmg_fine_pass(self._h, {"apply": 0, "smooth": 1}[what]))

    def restrict(self, level: int, fine, coarse=None):
        import torch
        nc = 3 * self.level_nodes(level + 1)
        if coarse is None:
            coarse = torch.empty(nc, dtype=torch.float32, device=fine.device)
        _check(self._lib.gmg_restrict(self._h, level, _ptr(fine, torch.float32, 3 * self.level_nodes(level), "fine"),
                                      _ptr(coarse, torch.float32, nc, "coarse")))
        return coarse

    def prolong_add(self, level: int, coarse, fine):
        import torch
        _check(self._lib.gmg_prolong_add(self._h, level,
                                         _ptr(coarse, torch.float32, 3 * self.level_nodes(level + 1), "coarse"),
                                         _ptr(fine, torch.float32, 3 * self.level_nodes(level), "fine")))
        return fine

    def coarse_solve(self, b, x=None):
        import torch
        L = self.num_levels - 1
        n = 3 * self.level_nodes(L)
        if x is None:
            x = torch.empty_like(b)
        _check(self._lib.gmg_coarse_solve(self._h, _ptr(b, torch.float32, n, "b"), _ptr(x, torch.float32, n, "x")))
        return x

    def vcycle(self, r, z=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(self._lib.gmg_vcycle(self._h, _ptr(r, torch.float32, 3 * self.nn, "r"),
                                    _ptr(z, torch.float32, 3 * self.nn, "z")))
        return z


    def kappa_eff(self, b, steps: int = 20) -> tuple[float, float, float]:
        """(lambda_min, lambda_max, kappa_eff) of M K from a CG-Lanczos probe
        started at the FP64 device vector b."""
        import torch
        out = (ctypes.c_double * 3)()
        _check(self._lib.gmg_kappa_eff(self._h, _ptr(b, torch.float64, 3 * self.nn, "b"), steps, out))
        return out[0], out[1], out[2]

    def vcycle_symmetry(self, x, y) -> float:
        """|x.M(y) - y.M(x)| / max(|x.M(y)|, |y.M(x)|) for one multigrid cycle M."""
        import torch
        v = ctypes.c_double()
        _check(self._lib.gmg_vcycle_symmetry(self._h, _ptr(x, torch.float32, 3 * self.nn, "x"),
                                             _ptr(y, torch.float32, 3 * self.nn, "y"), ctypes.byref(v)))
        return v.value
    def residual64(self, f, u, r=None) -> float:
        import torch
        rel = ctypes.c_double()
        rp = None if r is None else _ptr(r, torch.float64, 3 * self.nn, "r")
        _check(self._lib.gmg_residual64(self._h, _ptr(f, torch.float64, 3 * self.nn, "f"),
                                        _ptr(u, torch.float64, 3 * self.nn, "u"), rp, ctypes.byref(rel)))
        return rel.value


def _info_dict(i) -> dict:
    return {"status": i.status, "iterations": i.iterations, "replacements": i.replacements,
            "rel_residual": i.rel_residual, "rel_residual_recursive": i.rel_residual_recursive,
            "solve_ms": i.solve_ms, "setup_ms": i.setup_ms}


def solve_batch(solvers, fs, us=None, tol: float = 1e-6, maxit: int = 200):
    """Solves solvers[i] with load fs[i] (device FP64) into us[i] (initial guess;
    zeros when None) through one CUDA graph; returns (us, infos)."""
    import torch
    n = len(solvers)
    if len(fs) != n or (us is not None and len(us) != n):
        raise ValueError("one load and one iterate per solver")
    if us is None:
        us = [torch.zeros_like(f) for f in fs]
    hs = (_P * n)(*[s._h for s in solvers])
    fp = (_P * n)(*[_ptr(f, torch.float64, 3 * s.nn, "f") for s, f in zip(solvers, fs)])
    up = (_P * n)(*[_ptr(u, torch.float64, 3 * s.nn, "u") for s, u in zip(solvers, us)])
    infos = (_Info * n)()
    rc = load_library().gmg_solve_batch(hs, n, fp, up, tol, maxit, infos)
    _check(rc, allow=(GMG_OK, GMG_NOT_CONVERGED, GMG_NONFINITE))
    return us, [{"status": i.status, "iterations": i.iterations, "replacements": i.replacements,
                 "rel_residual": i.rel_residual, "rel_residual_recursive": i.rel_residual_recursive,
                 "solve_ms": i.solve_ms, "setup_ms": i.setup_ms} for i in infos]


# ---------------------------------------------------------------- learned warm start

NET_IN, NET_OUT, NET_LAYERS = 12, 3, 12
NET_ARITH = {"fp32": 0, "tf32": 1}


def net_num_params() -> int:
    return int(load_library().gmg_net_num_params())


def net_layer_shapes() -> list[tuple[int, int, int, int]]:
    """(cin, cout, stride, has_activation) per layer, in parameter order."""
    lib = load_library()
    out = []
    for l in range(NET_LAYERS):
        sh = (ctypes.c_int * 4)()
        _check(lib.gmg_net_layer_shape(l, sh))
        out.append(tuple(int(v) for v in sh))
    return out


def net_features(dims, rho, f, fixed, x=None, stream: int | None = None):
    """Input features [n_nodes, 12] (device float) of one problem."""
    import torch
    nx, ny, nz = dims
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    if x is None:
        x = torch.empty(nn, NET_IN, dtype=torch.float32, device=f.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load_library().gmg_net_features(nx, ny, nz, _ptr(rho, torch.float32, nx * ny * nz, "rho"),
                                           _ptr(f, torch.float64, 3 * nn, "f"),
                                           _ptr(fixed, torch.uint8, 3 * nn, "fixed"),
                                           _ptr(x, torch.float32, NET_IN * nn, "x"), stream))
    return x


def net_target(dims, u, t=None, stream: int | None = None):
    """Training target u / RMS(u) (device float [n_nodes, 3])."""
    import torch
    nx, ny, nz = dims
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    if t is None:
        t = torch.empty(nn, 3, dtype=torch.float32, device=u.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load_library().gmg_net_target(nx, ny, nz, _ptr(u, torch.float64, 3 * nn, "u"),
                                         _ptr(t, torch.float32, 3 * nn, "t"), stream))
    return t


class WarmNet:
    """The warm-start encoder-decoder: parameters, Adam state and per-shape
    workspaces live in the CUDA library."""

    def __init__(self, params, stream: int | None = None):
        import torch
        lib = load_library()
        self._lib = lib
        self.n_params = int(lib.gmg_net_num_params())
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.gmg_net_create(ctypes.byref(h), _ptr(params, torch.float32, self.n_params, "params"), stream))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gmg_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_arith(self, arith: str):
        """'fp32' (CUDA-core convolutions) or 'tf32' (tensor-core stride-1 convolutions)."""
        _check(self._lib.gmg_net_set_arith(self._h, NET_ARITH[arith]))

    def status(self):
        """Raises if a tensor-core kernel gave up waiting for its operands."""
        _check(self._lib.gmg_net_status(self._h))

    def set_params(self, params):
        import torch
        _check(self._lib.gmg_net_set_params(self._h, _ptr(params, torch.float32, self.n_params, "params")))

    def params(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(self._lib.gmg_net_get_params(self._h, _ptr(out, torch.float32, self.n_params, "params")))
        return out

    def grads(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(self._lib.gmg_net_get_grads(self._h, _ptr(out, torch.float32, self.n_params, "grads")))
        return out

    def forward(self, dims, x, g=None):
        """x: [B, n_nodes, 12] (or [n_nodes, 12]) device float -> g of shape [..., n_nodes, 3]."""
        import torch
        nx, ny, nz = dims
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        B = x.numel() // (NET_IN * nn)
        if g is None:
            g = torch.empty(*x.shape[:-1], 3, dtype=torch.float32, device=x.device)
        _check(self._lib.gmg_net_forward(self._h, nx, ny, nz, B, _ptr(x, torch.float32, B * NET_IN * nn, "x"),
                                         _ptr(g, torch.float32, B * 3 * nn, "g")))
        return g

    def train_step(self, dims, xs, ts, lr: float, loss_out=None, clip: float = 0.0, ops=None):
        """One Adam step on the batch (lists of [n_nodes, 12] / [n_nodes, 3]
        device tensors of one grid), the gradient clipped to L2 norm clip
        (0 = no clipping); ops: None (mean squared error) or one Solver per
        sample (energy-norm loss with that problem's stiffness); loss_out:
        optional one-element device float tensor (a view) receiving the batch
        loss."""
        import torch
        nx, ny, nz = dims
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        B = len(xs)
        if len(ts) != B or B == 0:
            raise ValueError("xs and ts must be non-empty lists of equal length")
        xp = (ctypes.c_void_p * B)(*[_ptr(x, torch.float32, NET_IN * nn, "x").value for x in xs])
        tp = (ctypes.c_void_p * B)(*[_ptr(t, torch.float32, 3 * nn, "t").value for t in ts])
        lp = None
        if loss_out is not None:
            if not (loss_out.is_cuda and loss_out.dtype == torch.float32 and loss_out.numel() >= 1):
                raise TypeError("loss_out must be a CUDA float32 tensor")
            lp = ctypes.c_void_p(loss_out.data_ptr())
        op = None
        if ops is not None:
            if len(ops) != B:
                raise ValueError("ops must hold one solver per sample")
            op = (ctypes.c_void_p * B)(*[o._h.value for o in ops])
        _check(self._lib.gmg_net_train_step(self._h, nx, ny, nz, B, xp, tp, op, float(lr), float(clip), lp))

    def warm_start(self, solver: "Solver", rho, f, u0=None, sync: bool = True):
        """u0 = alpha g for solver (energy-optimal alpha; 0 keeps the cold start).
        Returns (u0, alpha or None when sync is False)."""
        import torch
        if u0 is None:
            u0 = torch.empty_like(f)
        nx, ny, nz = solver.dims
        a = ctypes.c_double()
        _check(self._lib.gmg_warm_start(solver._h, self._h, _ptr(rho, torch.float32, nx * ny * nz, "rho"),
                                        _ptr(f, torch.float64, 3 * solver.nn, "f"),
                                        _ptr(u0, torch.float64, 3 * solver.nn, "u0"),
                                        ctypes.byref(a) if sync else None))
        return u0, (a.value if sync else None)
