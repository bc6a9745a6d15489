"""Oracle: smoothers, V-cycle and PCG (TEST INFRASTRUCTURE ONLY; FP64).

Paper passages followed:

* Sec. "Chebyshev-Jacobi Smoother", Algorithm cheb -- degree-nu Chebyshev on
  [alpha lambda_max, lambda_max] of D^{-1} K, alpha = 1/30.  The printed
  recurrence does not reproduce the Chebyshev residual polynomial at its first
  momentum step; the reading used is the standard semi-iteration it cites
  (Saad, Iterative Methods, Ch. 12, Chebyshev acceleration) with M = D, whose
  residual polynomial is T_nu((theta - lambda)/delta) / T_nu(theta/delta);
* the reproducibility defaults -- damped Jacobi x <- x + omega D^{-1}(b - K x),
  fine smoother degree 2, two coarse-level smoothing steps, omega capped at 0.5
  on coarse levels;
* Sec. "Matrix-Free V-Cycle", Eq. vcycle -- pre-smooth from zero, residual,
  restrict, recurse, prolong-add, post-smooth; coarsest level solved by dense
  Cholesky, or by a fixed-count PCG above the dense-Cholesky cutoff;
* Sec. "Outer Krylov Solver and Convergence Statement" -- left-preconditioned
  CG with the frozen V-cycle, ||r_k|| / ||b|| < tol accepted only by the true
  residual; iteration caps and non-finite iterates are failures; restarted
  right-preconditioned flexible GMRES with modified Gram-Schmidt Arnoldi,
  Givens rotations for the incremental QR update and a happy-breakdown test on
  the new Hessenberg entry (1e-14), default restart 32;
* Sec. "Ablations", item (c) -- the W-cycle (cycle index 2);
* Sec. "Outer Krylov Solver and Convergence Statement" (Remark on the frozen
  hierarchy) and the appendix on the effective condition number --
  kappa_eff = lambda_max(M K) / lambda_min(M K), estimated by a Lanczos probe;
  here the Lanczos tridiagonal is the one CG builds from its coefficients
  (alpha_k, beta_k), the standard CG-Lanczos correspondence;
* the same section's symmetry-defect diagnostic of the applied preconditioner.

Readings: the smoother may differ between the fine level and the coarse levels
(same count before and after the coarse correction); the Chebyshev band uses
the power-iteration estimate times a safety factor (default 1.1; 1.0 is the
literal reading, under which the 20-step estimate sits ~8 % below lambda_max on
a 40^3 cantilever and degree-2 Chebyshev-PCG fails the 200 cap there, whereas
the paper reports it converging); an iteration is one
completed x/r update; when the recursive residual passes the test but the
recomputed true residual does not, the recursive residual is replaced by the
true one and the search direction restarts from its preconditioned value (a
replacement that keeps the old direction stalls near the attainable accuracy).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .hierarchy import Level, coarsest_solve

OK, NOT_CONVERGED, NONFINITE = 0, 1, 2


def jacobi(lev: Level, b: np.ndarray, x: np.ndarray, omega: float, steps: int) -> np.ndarray:
    dinv = 1.0 / lev.diag
    for _ in range(steps):
        x = x + omega * dinv * (b - lev.apply(x))
    return x


def chebyshev(lev: Level, b: np.ndarray, x: np.ndarray, degree: int,
              alpha: float = 1.0 / 30.0, lam: float | None = None) -> np.ndarray:
    """Chebyshev acceleration of D^{-1} K x = D^{-1} b on [alpha lam, lam]."""
    lam = lev.lam if lam is None else lam
    dinv = 1.0 / lev.diag
    theta = 0.5 * (1.0 + alpha) * lam
    delta = 0.5 * (1.0 - alpha) * lam
    sigma1 = theta / delta
    rho = 1.0 / sigma1
    r = b - lev.apply(x)
    d = dinv * r / theta
    for k in range(degree):
        x = x + d
        if k == degree - 1:
            break
        r = b - lev.apply(x)
        rho_next = 1.0 / (2.0 * sigma1 - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * (dinv * r)
        rho = rho_next
    return x


@dataclasses.dataclass
class SmootherSpec:
    """Smoother of the non-coarsest levels.  ``kind``/``degree``/``omega`` act on
    the fine level; the ``coarse_*`` fields (default: same as the fine level) on
    levels 1..L-1.  Chebyshev uses the band [alpha s lam, s lam] with
    s = ``lambda_safety`` applied to the power-iteration estimate lam."""

    kind: str = "jacobi"   # "jacobi" | "chebyshev"
    degree: int = 2
    omega: float = 0.6
    alpha: float = 1.0 / 30.0
    lambda_safety: float = 1.1
    coarse_kind: str | None = None
    coarse_degree: int | None = None
    coarse_omega: float | None = None

    def at(self, level: int) -> tuple[str, int, float]:
        if level == 0:
            return self.kind, self.degree, self.omega
        return (self.coarse_kind or self.kind,
                self.coarse_degree if self.coarse_degree is not None else self.degree,
                self.coarse_omega if self.coarse_omega is not None else self.omega)


def smooth(lev: Level, b, x, spec: SmootherSpec, level: int = 0):
    kind, degree, omega = spec.at(level)
    if kind == "jacobi":
        return jacobi(lev, b, x, omega, degree)
    return chebyshev(lev, b, x, degree, spec.alpha, lam=lev.lam * spec.lambda_safety)


def vcycle(H: list[Level], r: np.ndarray, spec: SmootherSpec, l: int = 0) -> np.ndarray:
    """Eq. vcycle on the free-DOF vector r of level l."""
    lev = H[l]
    if l == len(H) - 1:
        return coarsest_solve(lev, r)
    x = smooth(lev, r, np.zeros_like(r), spec, l)
    t = r - lev.apply(x)
    e = vcycle(H, lev.P.T @ t, spec, l + 1)
    x = x + lev.P @ e
    return smooth(lev, r, x, spec, l)


def mgcycle(H: list[Level], b: np.ndarray, spec: SmootherSpec, l: int = 0, gamma: int = 1,
            x0: np.ndarray | None = None) -> np.ndarray:
    """Multigrid cycle with cycle index gamma (1: V, 2: W) on level l, from the
    initial guess x0 (zero if None): pre-smooth, residual, gamma coarse visits
    (the second one starting from the first one's result), prolong-add,
    post-smooth; the coarsest level is solved exactly."""
    lev = H[l]
    if l == len(H) - 1:
        return coarsest_solve(lev, b)
    x = smooth(lev, b, np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64), spec, l)
    t = b - lev.apply(x)
    bc = lev.P.T @ t
    e = None
    for _ in range(gamma):
        e = mgcycle(H, bc, spec, l + 1, gamma, e)
    x = x + lev.P @ e
    return smooth(lev, b, x, spec, l)


def cg_lanczos_tridiagonal(alphas, betas) -> tuple[np.ndarray, np.ndarray]:
    """Diagonal and off-diagonal of the Lanczos matrix of the preconditioned
    operator from k CG steps: T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_j)/alpha_j (beta_j = r_{j+1}.z_{j+1} / r_j.z_j)."""
    a = np.asarray(alphas, dtype=np.float64)
    bt = np.asarray(betas, dtype=np.float64)
    k = len(a)
    diag = 1.0 / a
    diag[1:] += bt[:k - 1] / a[:k - 1]
    off = np.sqrt(bt[:k - 1]) / a[:k - 1]
    return diag, off


def kappa_eff(H: list[Level], b_free: np.ndarray, spec: SmootherSpec, steps: int,
              precond=None) -> tuple[float, float, float]:
    """Lanczos estimate of lambda_min, lambda_max and kappa_eff of M K from
    `steps` CG steps on K x = b (start vector b), M one V-cycle by default."""
    lev = H[0]
    M = precond or (lambda r: vcycle(H, r, spec))
    r = np.array(b_free, dtype=np.float64)
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for _ in range(steps):
        q = lev.apply(p)
        alpha = rz / float(p @ q)
        r = r - alpha * q
        z = M(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    d, o = cg_lanczos_tridiagonal(alphas, betas)
    T = np.diag(d) + np.diag(o, 1) + np.diag(o, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1]), float(ev[-1] / ev[0])


def symmetry_defect(precond, x: np.ndarray, y: np.ndarray) -> float:
    """|x.M(y) - y.M(x)| / max(|x.M(y)|, |y.M(x)|) for the operator M."""
    a = float(x @ precond(y))
    b = float(y @ precond(x))
    return abs(a - b) / max(abs(a), abs(b))


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    status: int
    iterations: int
    rel_residual: float
    history: list


def pcg(apply_K, precond, f: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6,
        maxit: int = 200) -> PCGResult:
    """Left-preconditioned CG with true-residual acceptance (free-DOF vectors)."""
    nf = float(np.linalg.norm(f))
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    if nf == 0.0:
        return PCGResult(np.zeros_like(f), OK, 0, 0.0, [0.0])
    r = f - apply_K(x)
    rel = float(np.linalg.norm(r)) / nf
    hist = [rel]
    if not np.isfinite(rel):
        return PCGResult(x, NONFINITE, 0, rel, hist)
    if rel < tol:
        return PCGResult(x, OK, 0, rel, hist)
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    k = 0
    while k < maxit:
        q = apply_K(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        rel = float(np.linalg.norm(r)) / nf
        hist.append(rel)
        if not (np.isfinite(rel) and np.isfinite(alpha)):
            return PCGResult(x, NONFINITE, k, rel, hist)
        if rel < tol:
            rt = f - apply_K(x)
            rel_t = float(np.linalg.norm(rt)) / nf
            if rel_t < tol:
                return PCGResult(x, OK, k, rel_t, hist)
            r = rt  # residual replacement, and the search direction restarts
            z = precond(r)
            p = z.copy()
            rz = float(r @ z)
            continue
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    rt = f - apply_K(x)
    return PCGResult(x, NOT_CONVERGED, k, float(np.linalg.norm(rt)) / nf, hist)


def fgmres(apply_K, precond, f: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6,
           maxit: int = 200, restart: int = 32, breakdown: float = 1e-14) -> PCGResult:
    """Restarted right-preconditioned flexible GMRES (free-DOF vectors).

    Each cycle starts from the true residual r = f - K x, beta = ||r||,
    v_1 = r / beta; step j stores z_j = M v_j, forms w = K z_j, orthogonalises
    it against v_1..v_j by modified Gram-Schmidt (h_ij), h_{j+1,j} = ||w||,
    applies the previous Givens rotations to column j of H and a new one that
    annihilates h_{j+1,j}; |g_{j+1}| is the residual norm of the minimiser.
    The cycle ends at restart, at |g_{j+1}| / ||f|| < tol, or when h_{j+1,j} <
    breakdown; then x += Z y with H y = g (upper triangular).  A solve is
    accepted only by the true residual.  `iterations` counts Arnoldi steps."""
    nf = float(np.linalg.norm(f))
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    if nf == 0.0:
        return PCGResult(np.zeros_like(f), OK, 0, 0.0, [0.0])
    k = 0
    hist = []
    while True:
        r = f - apply_K(x)
        beta = float(np.linalg.norm(r))
        rel = beta / nf
        hist.append(rel)
        if not np.isfinite(rel):
            return PCGResult(x, NONFINITE, k, rel, hist)
        if rel < tol:
            return PCGResult(x, OK, k, rel, hist)
        if k >= maxit:
            return PCGResult(x, NOT_CONVERGED, k, rel, hist)
        V = [r / beta]
        Z = []
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        while j < restart and k < maxit:
            z = precond(V[j])
            Z.append(z)
            w = apply_K(z)
            for i in range(j + 1):
                Hm[i, j] = float(w @ V[i])
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):  # previous rotations on column j
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            happy = Hm[j + 1, j] < breakdown
            if not happy:
                V.append(w / Hm[j + 1, j])
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            k += 1
            if happy or abs(g[j]) / nf < tol:
                break
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:j] @ y[i + 1:j]) / Hm[i, i]
        for i in range(j):
            x = x + y[i] * Z[i]


def gmg_pcg(H: list[Level], f_full: np.ndarray, spec: SmootherSpec, tol: float = 1e-6,
            maxit: int = 200, u0_full: np.ndarray | None = None) -> tuple[np.ndarray, PCGResult]:
    """GMG-preconditioned CG on the fine free-DOF system; returns the full-DOF
    solution (0 on fixed DOFs) and the PCG record."""
    lev = H[0]
    f = np.asarray(f_full, dtype=np.float64)[lev.free]
    x0 = None if u0_full is None else np.asarray(u0_full, dtype=np.float64)[lev.free]
    res = pcg(lev.apply, lambda r: vcycle(H, r, spec), f, x0, tol, maxit)
    u = np.zeros(lev.fixed.shape[0])
    u[lev.free] = res.x
    return u, res


def exact_solve(H: list[Level], f_full: np.ndarray, spec: SmootherSpec | None = None,
                dense_limit: int = 6000) -> np.ndarray:
    """u* of K_ff u_f = f_f: dense Cholesky when small, else this oracle's own
    GMG-PCG run to a 1e-12 true residual."""
    lev = H[0]
    f = np.asarray(f_full, dtype=np.float64)[lev.free]
    u = np.zeros(lev.fixed.shape[0])
    if lev.n_free <= dense_limit and lev.K is not None:
        import scipy.linalg as sla
        c = sla.cho_factor(lev.K.toarray(), lower=True)
        u[lev.free] = sla.cho_solve(c, f)
        return u
    res = pcg(lev.apply, lambda r: vcycle(H, r, spec or SmootherSpec()), f, None, 1e-12, 2000)
    if res.status != OK:
        raise RuntimeError(f"oracle exact solve did not reach 1e-12: {res.rel_residual}")
    u[lev.free] = res.x
    return u
