/*
 * gmg.h -- C ABI of the B300 (sm_103a) matrix-free Galerkin geometric-multigrid
 * preconditioned-CG solver for the frozen-density 3D SIMP elasticity system
 * K(rho) u = f on a structured grid of unit hex8 elements.
 *
 * The method is the one of "A Matrix-Free Galerkin Multigrid Solver and
 * Failure-Mode Screen for Single-GPU 3D SIMP Linear Systems" (arXiv 2604.26441):
 *   - Sec. "Problem Setup", Eq. simp_filter / Eq. state_eq: E_e = Emin +
 *     (E0 - Emin) rho_e^p, K = sum_e E_e K_e, free-DOF system K_ff u_f = f_f;
 *   - Sec. "Transfer Operators and Boundary Masking": 2:1 trilinear transfers
 *     (Eq. trilinear_weights, Eq. vector_prolongation), Dirichlet inheritance by
 *     injection, matrix-free fine operator (Eq. mf_matvec), element-wise level-1
 *     Galerkin operator (Eq. galerkin_level1), Galerkin triple products below;
 *   - Sec. "Chebyshev-Jacobi Smoother" (Algorithm cheb) and damped Jacobi;
 *   - Sec. "Matrix-Free V-Cycle" (Eq. vcycle) with a dense Cholesky coarsest solve;
 *   - Sec. "Outer Krylov Solver and Convergence Statement": left-preconditioned
 *     CG, acceptance only by the true residual ||f - K u|| / ||f|| < tol.
 *
 * Conventions shared by every entry point:
 *   - grid: nx, ny, nz unit elements; node n = i + (nx+1)*(j + (ny+1)*k);
 *     DOF 3n + c (c = x, y, z); element e = ex + nx*(ey + ny*ez);
 *   - all vectors are node-major with 3 values per node (length 3*n_nodes of
 *     the level they live on); fixed DOFs are ignored on input and written as 0;
 *   - pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees them and keeps no reference past the call; the
 *     handle owns the hierarchy and all workspaces;
 *   - every call returns an int status: 0 = success, > 0 = a solve outcome that
 *     is not success (GMG_NOT_CONVERGED, GMG_NONFINITE), < 0 = an error; no C++
 *     exception crosses the ABI; gmg_last_error() gives a text for the last error
 *     of the calling thread;
 *   - all device work is issued on the stream given in gmg_options.stream
 *     (NULL = the legacy default stream).  gmg_setup and gmg_solve return after
 *     their work is complete; the other compute calls are asynchronous.
 */
#ifndef GMG_B300_H
#define GMG_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GMG_OK 0
#define GMG_NOT_CONVERGED 1      /* iteration cap reached; u holds the last iterate */
#define GMG_NONFINITE 2          /* a non-finite residual or step length appeared */
#define GMG_ERR_ARG (-1)         /* bad argument (null pointer, size, level index...) */
#define GMG_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define GMG_ERR_CHOLESKY (-3)    /* coarsest matrix not positive definite */
#define GMG_ERR_SMOOTHER (-4)    /* damped Jacobi with omega * lambda_max >= 2 */
#define GMG_ERR_NOMEM (-5)       /* device allocation failed */
#define GMG_ERR_NO_DEVICE (-6)   /* no CUDA device usable by this build (sm_103a) */
#define GMG_TIMEOUT (-7)         /* a bounded device-side wait gave up (the grid barrier of the
                                    fused lower V-cycle after gmg_options.spin_limit polls, or an
                                    mbarrier wait of a TMA-staged / tensor-core kernel); the
                                    failure is recorded, never accepted (Sec. "Outer Krylov Solver
                                    and Convergence Statement"), u is not a solution, and the
                                    handle's wait state is reset so the next call can run */

/* ---- boundary conditions ----------------------------------------------- */
#define GMG_BC_CLAMP_XMIN 0      /* every DOF of the face i = 0 fixed */
#define GMG_BC_MASK 1            /* per-DOF flags supplied by the caller */

/* ---- smoothers ---------------------------------------------------------- */
#define GMG_SMOOTHER_JACOBI 0
#define GMG_SMOOTHER_CHEBYSHEV 1

/* Fine-level smoother arithmetic (gmg_options.fine_smoother).  Plain BF16
 * makes the V-cycle an inexact, non-symmetric preconditioner: pair it with
 * GMG_OUTER_FGMRES (under PCG it can stagnate); split BF16 (BF16X3) is close
 * enough to FP32 for PCG. */
#define GMG_FINE_FP32 0
#define GMG_FINE_BF16X3 1
#define GMG_FINE_BF16 2

/* Outer Krylov solver (gmg_options.outer). */
#define GMG_OUTER_PCG 0
#define GMG_OUTER_FGMRES 1

typedef struct gmg_handle gmg_handle;

typedef struct {
    int nx, ny, nz;              /* element counts, each >= 1 */
} gmg_grid;

typedef struct {
    int kind;                    /* GMG_BC_CLAMP_XMIN or GMG_BC_MASK */
    const uint8_t* fixed;        /* HOST pointer, 3*n_nodes bytes, 1 = fixed (kind == MASK) */
} gmg_bc;

typedef struct {
    int levels;                  /* number of grids including the fine one; 0 = automatic
                                    (coarsen while the coarsest free-DOF count exceeds
                                    chol_cutoff and every element count is >= 2) */
    int smoother, degree;        /* fine-level smoother kind and steps per pass */
    int coarse_smoother;         /* levels 1..L-1; -1 = same as the fine level */
    int coarse_degree;           /* -1 = same as the fine level */
    double omega;                /* Jacobi damping, fine level */
    double coarse_omega;         /* Jacobi damping, coarse levels; <= 0: same as omega */
    double cheb_alpha;           /* Chebyshev band [alpha*lam, lam], paper default 1/30 */
    double lambda_safety;        /* Chebyshev uses lam = safety * power-iteration estimate */
    int power_iters_fine;        /* power iterations for lambda_max(D^-1 K), fine (20) */
    int power_iters_coarse;      /* ... on assembled levels (10) */
    int chol_cutoff;             /* dense-Cholesky size limit for the coarsest level (5000) */
    int fused_coarse_nodes;      /* assembled levels with fewer nodes than this run, together with
                                    the coarsest solve, as one persistent cooperative kernel; 0 = off
                                    (default: the per-level kernels, which inside the device-resident
                                    PCG graph were faster at every size measured) */
    int bsr_tma_nodes;           /* assembled levels with at least this many nodes load their
                                    operator planes as TMA-staged shared-memory tiles;
                                    <= 0 (default) = never: levels of >= 65536 nodes stream one
                                    thread per node, smaller ones use the K-split kernel */
    int device_loop;             /* 1 (default): PCG iterations run as one CUDA graph with a
                                    conditional while node, returning to the host only for the
                                    FP64 acceptance test; 0: one host round trip per iteration.
                                    Both run the same kernels in the same order. */
    double ir_factor;            /* 0 (default): plain PCG to tol.  In (0, 1): outer FP64 iterative
                                    refinement -- each inner FP32 PCG phase starts from the FP64
                                    residual of the current u and stops when its recursive residual
                                    is ir_factor times smaller (not below tol); the FP64 residual
                                    is then recomputed (gmg_info.replacements counts the outer
                                    steps after the first).  Reaches tolerances below FP32 reach. */
    int fine_smoother;           /* arithmetic of the fine-level smoother's element contraction:
                                    GMG_FINE_FP32 (default, CUDA cores), GMG_FINE_BF16X3 (tensor
                                    cores, split BF16: 3 MMA passes, ~16 significant bits) or
                                    GMG_FINE_BF16 (tensor cores, one BF16 pass).  FP32
                                    accumulation; the PCG operator, residuals and coarser levels
                                    are unaffected. */
    int cycle_index;             /* multigrid cycle: 1 = V-cycle (default), 2 = W-cycle (each coarse
                                    level visited twice, the second visit from the first's result;
                                    Sec. Ablations (c)) */
    int outer;                   /* GMG_OUTER_PCG (default): left-preconditioned CG;
                                    GMG_OUTER_FGMRES: restarted right-preconditioned flexible GMRES
                                    (MGS Arnoldi, Givens rotations, happy breakdown at 1e-14);
                                    gmg_info.iterations counts Arnoldi steps, .replacements restarts */
    int restart;                 /* FGMRES restart length (32) */
    int bsr_kernel;              /* kernel of the assembled levels outside the TMA-staged and fused
                                    paths: -1 (default) = by size (streaming from 65,536 nodes;
                                    below, K-split with the most of 32 / 16 / 8 slices that
                                    keeps the grid within ~4 blocks per SM), and level 1 applied
                                    matrix-free from the fine moduli where that equals the
                                    assembled operator (even fine sizes, every fixed fine DOF with
                                    fixed prolongation parents; Eq. galerkin_level1 summed per
                                    coarse element); 0 = streaming, one thread per
                                    node; 1 / 2 / 3 / 4 / 5 = K-split with 8 / 2 / 4 / 16 / 32
                                    slices per node (these pin the assembled operator).
                                    The assembled kernels give the same results (each node's
                                    arithmetic is the same); the matrix-free level 1 agrees with
                                    them to FP32 rounding.  gmg_autotune overrides it per level. */
    void* stream;                /* cudaStream_t for all device work; NULL = default stream */
    long long spin_limit;        /* polls (each followed by a ~64 ns sleep) that a block of the fused
                                    lower V-cycle makes at a grid barrier before it gives up and the
                                    call returns GMG_TIMEOUT; default 2^24 (about a second); >= 0 */
    int coarse_pcg_steps;        /* when the coarsest level has more free DOFs than chol_cutoff (the
                                    hierarchy was not coarsened enough, e.g. a fixed `levels`), it is
                                    solved by this many Jacobi-preconditioned CG steps from 0 instead
                                    of dense Cholesky (Sec. "Matrix-Free V-Cycle"; 80 in the paper's
                                    defaults).  The V-cycle is then a fixed nonlinear operator: pair
                                    it with GMG_OUTER_FGMRES when PCG stalls.  A single-level
                                    hierarchy above the cutoff is refused (GMG_ERR_ARG). */
    int lower_cluster;           /* 0 (default): one launch per step of the V-cycle's bottom.  1: when
                                    the last assembled level m >= 2 is small enough that its operator
                                    fits the shared memory of one 16-CTA thread-block cluster (~3,000
                                    nodes) and the coarsest level is solved densely, level m's
                                    smoothing passes, residual and transfers and the coarsest solve
                                    (the inverse applied in double-float, ~44 bits) run as one
                                    cluster launch whose steps are separated by the cluster barrier;
                                    results agree with the per-level kernels to FP32 rounding.  At
                                    100^3 the one launch (59 us) is slower than the ten per-level
                                    launches it replaces (5.49 against 5.17 ms per solve), so it is
                                    off by default.  Not used with fused_coarse_nodes > 0 or a
                                    pinned bsr_kernel. */
} gmg_options;

typedef struct {
    int status;                  /* same value the solve call returned */
    int iterations;              /* completed PCG updates */
    int replacements;            /* residual replacements after a failed true-residual check */
    double rel_residual;         /* FP64 true ||f - K u|| / ||f|| over free DOFs at return */
    double rel_residual_recursive; /* last recursive (FP32-updated) residual ratio */
    double solve_ms;             /* wall time of the call on the host clock */
    double setup_ms;             /* wall time of the gmg_setup call that built this handle's
                                    hierarchy (host clock, synchronous; a clone reports its source's) */
} gmg_info;

/* Fills *opt with the paper's defaults: 4 levels, Chebyshev degree 2 on the
 * fine level, 2 Jacobi steps with omega 0.5 on the coarse levels, alpha = 1/30,
 * lambda_safety 1.1, 20/10 power iterations, Cholesky cutoff 5000, NULL stream,
 * spin_limit 2^24, 80 coarsest PCG steps. */
void gmg_default_options(gmg_options* opt);

/* Builds the hierarchy for one frozen density field (Eq. simp_filter, Eq.
 * state_eq, Eq. galerkin_level1, "Coarser levels", "Spectral-radius estimation",
 * coarsest dense Cholesky of K^L_ff + eps I with eps = max(mean_diag 1e-8, 1e-14)).
 *   rho_dev : device float[nx*ny*nz] densities, element order as above;
 *   p, E0, Emin : SIMP law; nu : Poisson ratio of the unit element stiffness;
 *   bc : Dirichlet set (the mask, if any, is copied; the pointer is not kept);
 *   opt : options, or NULL for gmg_default_options().
 * On success *h receives a new handle (free it with gmg_destroy).  Errors:
 * GMG_ERR_ARG, GMG_ERR_CUDA, GMG_ERR_NOMEM, GMG_ERR_CHOLESKY, GMG_ERR_SMOOTHER,
 * GMG_ERR_NO_DEVICE; *h is left NULL. */
int gmg_setup(gmg_handle** h, const gmg_grid* g, const float* rho_dev, double p, double E0,
              double Emin, double nu, const gmg_bc* bc, const gmg_options* opt);

/* Solves K_ff u_f = f_f by GMG-preconditioned CG (Sec. "Outer Krylov Solver and
 * Convergence Statement").  f_dev: device double[3*n_nodes]; u_dev: device
 * double[3*n_nodes], on entry the initial guess (zeros = cold start), on exit the
 * solution with fixed DOFs set to 0.  The inner iteration runs in FP32 with FP64
 * dot products; u is accumulated in FP64 and a solve is accepted only when the
 * FP64 true residual is below tol.  Returns GMG_OK, GMG_NOT_CONVERGED (maxit
 * reached), GMG_NONFINITE, or an error.  info may be NULL. */
int gmg_solve(gmg_handle* h, const double* f_dev, double* u_dev, double tol, int maxit,
              gmg_info* info);

/* y = K_ff u on the fine level in FP32 (Eq. mf_matvec): u_dev, y_dev device
 * float[3*n_nodes]; fixed DOFs of u are ignored and written as 0 in y.
 * Asynchronous on the handle's stream.  u_dev and y_dev must not overlap. */
int gmg_apply(gmg_handle* h, const float* u_dev, float* y_dev);

/* Frees every device resource of the handle.  NULL is accepted. */
void gmg_destroy(gmg_handle* h);

/* Replaces the handle's spin_limit (see gmg_options): later calls use the new
 * bound.  Drops the handle's captured solve graphs (they hold the old value).
 * polls >= 0, else GMG_ERR_ARG.  A test sets it to 0 to make the fused lower
 * V-cycle's barrier give up and checks that the solve reports GMG_TIMEOUT and
 * that the next solve with the default bound succeeds. */
int gmg_set_spin_limit(gmg_handle* h, long long polls);

/* Bounds-checked build.  Compiled with -DGMG_CHECKED, the kernels of the solve
 * path check the indices they compute (neighbour, transfer, mask,
 * coarsest-solve and layout-conversion accesses) against the size of the
 * buffer addressed; an index out of range records the number of its check
 * site in a sticky device word and the access is redirected to element 0 (no
 * trap, nothing read or written outside the buffer), and every solve then
 * returns GMG_ERR_CUDA naming the site.  gmg_bounds_checked() is 1 in that
 * build and 0 otherwise; gmg_bounds_site() synchronises the device and returns
 * the first recorded site (0 = none), clearing the words (always 0 in the
 * normal build).  This is the device-side stand-in for a memory checker. */
int gmg_bounds_checked(void);
unsigned gmg_bounds_site(void);

/* Static text for a status code. */
const char* gmg_status_str(int status);

/* Text of the last error recorded on the calling thread ("" if none). */
const char* gmg_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far (all
 * handles); the difference across a region counts the kernels it ran. */
unsigned long long gmg_kernel_launches(void);

/* ---- introspection and per-step entry points ----------------------------
 * These expose the individual steps of the hot path so that each can be checked
 * on its own.  Vectors are device float[3*n_nodes(level)] unless stated; all
 * are asynchronous on the handle's stream except the host-output getters, which
 * synchronise that stream before returning.  Internally the fine level's
 * vectors pad every node row to a multiple of 4 nodes (16-byte aligned rows for
 * the TMA-fed operator); the level-0 calls copy the caller's dense vectors in
 * and out of that layout, using the handle's own work vectors. */

int gmg_num_levels(const gmg_handle* h);

/* dims[0..2] = element counts of the level. */
int gmg_level_dims(const gmg_handle* h, int level, int dims[3]);

/* HOST uint8[n_nodes(level)] of fixed-component bits (bit c set = DOF c fixed),
 * inherited level to level by injection (Sec. "Transfer Operators and Boundary
 * Masking"). */
int gmg_get_mask(gmg_handle* h, int level, uint8_t* host_out);

/* HOST double[243*n_nodes(level)] (level >= 1): the 3x3-block 27-point Galerkin
 * operator K^level in FP64 (Eq. galerkin_level1 for level 1, R K P below),
 * plane-major: entry (slot s, row r, col c) of node n at [(s*9 + r*3 + c)*n_nodes
 * + n], slot s = (dx+1) + 3(dy+1) + 9(dz+1) for the neighbour n + (dx, dy, dz).
 * Rows and columns of fixed DOFs and neighbours outside the grid are 0. */
int gmg_get_bsr(gmg_handle* h, int level, double* host_out);

/* lambda_max(D^-1 K) estimate of a level before lambda_safety (Sec.
 * "Spectral-radius estimation"), and an override that also refreshes the
 * level's smoother coefficients. */
int gmg_get_lambda(gmg_handle* h, int level, double* out);
int gmg_set_lambda(gmg_handle* h, int level, double lam);

/* y = K^level x (masked), FP32 (level 0 matrix-free, levels >= 1 from the BSR). */
int gmg_level_apply(gmg_handle* h, int level, const float* x_dev, float* y_dev);

/* One smoothing pass (degree steps of the level's smoother, Algorithm cheb or
 * damped Jacobi) on K^level x = b; x_is_zero != 0 means x enters as 0 (and is
 * not read). */
int gmg_level_smooth(gmg_handle* h, int level, const float* b_dev, float* x_dev, int x_is_zero);

/* The fine-level operator on the handle's own level-0 vectors, whatever values
 * they hold, for timing the fused fine-level kernel in isolation (without the
 * repacking of caller vectors that the level-0 calls above perform):
 * what = 0: one application y = K x (Eq. mf_matvec); what = 1: one smoothing
 * pass, degree fused operator + smoother steps from a nonzero iterate
 * (Algorithm cheb / damped Jacobi; GMG_ERR_ARG on a single-level hierarchy).
 * Asynchronous on the handle's stream. */
int gmg_fine_pass(gmg_handle* h, int what);

/* coarse = R^level fine (R = P^T, Eq. vector_prolongation; coarse fixed DOFs 0):
 * fine on `level`, coarse on level+1. */
int gmg_restrict(gmg_handle* h, int level, const float* fine_dev, float* coarse_dev);

/* fine += P^level coarse (fine fixed DOFs untouched). */
int gmg_prolong_add(gmg_handle* h, int level, const float* coarse_dev, float* fine_dev);

/* x = (K^L_ff + eps I)^-1 b on the coarsest level (FP64 Cholesky factor), or,
 * above the dense-Cholesky cutoff, coarse_pcg_steps Jacobi-PCG steps from 0. */
int gmg_coarse_solve(gmg_handle* h, const float* b_dev, float* x_dev);

/* Lanczos probe of the effective condition number of the preconditioned
 * operator M K (M = one multigrid cycle): `steps` CG iterations on K x = b from
 * x = 0 (b: device FP64, fixed DOFs ignored), the Lanczos tridiagonal built
 * from the CG coefficients (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
 * T_{j,j+1} = sqrt(beta_j)/alpha_j), its extreme eigenvalues by Sturm-sequence
 * bisection.  out = {lambda_min, lambda_max, kappa_eff}.  Stops early at a
 * breakdown (beta = 0).  Synchronous. */
int gmg_kappa_eff(gmg_handle* h, const double* b_dev, int steps, double out[3]);

/* Symmetry defect of the applied preconditioner: |x.M(y) - y.M(x)| /
 * max(|x.M(y)|, |y.M(x)|) for one multigrid cycle M (x, y device FP32, zero on
 * fixed DOFs).  0 in exact arithmetic for matched pre/post smoothers. */
int gmg_vcycle_symmetry(gmg_handle* h, const float* x_dev, const float* y_dev, double* defect);

/* A handle that shares src's hierarchy (operators, masks, smoother
 * coefficients, coarsest factor, moduli) and owns a workspace of its own, for
 * solving further right-hand sides on the same density field (e.g. in one
 * gmg_solve_batch).  src must outlive the clone; gmg_set_lambda on either
 * changes the shared smoother coefficients.  Release with gmg_destroy. */
int gmg_clone(const gmg_handle* src, gmg_handle** out);

/* Solves count independent problems -- handles of different grids, clones for
 * further loads -- f[i] -> u[i] (device FP64, u[i] the initial guess), sharing
 * tol and maxit.  Items whose handles share one hierarchy (a handle and its
 * clones, on the multi-load path's options) are solved together as multi-load
 * chunks of up to 16 loads (the loop of gmg_solve_multi, owned by the chunk's
 * first handle, whose multi-load workspace it allocates on first use); every
 * other item runs its own device-resident PCG loop.  The loops run as
 * independent branches of one CUDA graph (captured on the first call for a
 * given list of handles and iterates, then replayed), so small instances run
 * concurrently; the FP64 acceptance test is taken for all items after one
 * synchronisation.  A single item's iterates equal those of gmg_solve on a
 * handle with fused_coarse_nodes = 0 (the per-level lower V-cycle); a chunk's
 * equal those of gmg_solve_multi on the same loads.  Items whose options need
 * the host loop (outer FGMRES, ir_factor, device_loop = 0) make the batch run
 * one gmg_solve after the other.  Each handle appears at most once.  Runs on
 * the first handle's stream.  Returns GMG_OK when every item converged, else
 * the last failing status; infos[i] per item. */
int gmg_solve_batch(gmg_handle* const* handles, int count, const double* const* f_dev, double* const* u_dev,
                    double tol, int maxit, gmg_info* infos);

/* Multi-load solve (the batching line; Sec. "Outer Krylov Solver and
 * Convergence Statement" per load): nl <= 16 right-hand sides f[l] -> u[l]
 * (host arrays of device FP64 pointers, dense numbering; u[l] the initial
 * guess) on one hierarchy, advanced together by one device-resident PCG loop
 * with per-load step lengths, directions and stopping decisions: every kernel
 * of the V-cycle serves all loads in one launch (levels >= 1 read each operator
 * block once for all loads).  A load stops where gmg_solve would stop it;
 * the FP64 acceptance test follows per load, and a load whose recursive
 * residual passed but whose FP64 residual did not continues alone (residual
 * replacement, as gmg_solve).  Options outside this path (outer FGMRES,
 * ir_factor, a tensor-core fine smoother, the host loop, a W-cycle, a single
 * level, a coarsest level above the Cholesky cutoff) make the call run one
 * gmg_solve after the other.  Allocates the handle's multi-load workspace on
 * first use (7 level-0 vectors of 256 bytes per node, 5 per coarser level,
 * the coarsest inverse as FP32 hi + lo).  Synchronous on the handle's stream.
 * infos[l] per load; returns GMG_OK when every load converged, else the last
 * failing status. */
int gmg_solve_multi(gmg_handle* h, int nl, const double* const* f_dev, double* const* u_dev, double tol, int maxit,
                    gmg_info* infos);

/* y[l] = K_ff u[l] (Eq. mf_matvec; fixed DOFs of u[l] ignored, of y[l] set
 * to 0) for nl <= 16 loads in one launch of the multi-load level-0 operator
 * (host arrays of device FP32 pointers, dense numbering).  Asynchronous. */
int gmg_apply_multi(gmg_handle* h, int nl, const float* const* u_dev, float* const* y_dev);

/* One pass of the multi-load level-0 operator on the handle's own multi-load
 * vectors, for timing: what = 0: q = K p; what = 1: a smoothing pass (degree
 * fused operator + smoother steps from the iterate z, right-hand side r).
 * nl loads (1..16).  Allocates the multi-load workspace on first use.
 * Asynchronous. */
int gmg_multi_fine_pass(gmg_handle* h, int nl, int what);

/* Level-0 operator of the multi-load path: 0 = CUDA cores (Hadamard form, one
 * block per tile and load), 1 = tensor cores (element contraction on tcgen05).
 * GMG_ERR_ARG for an unknown kind or one this build lacks. */
int gmg_set_multi_kernel(gmg_handle* h, int kind);

/* Tiles of the fine-level kernel.  One element column per thread: 32 x 8
 * threads owning 31 x 7 nodes, or 16 x 16 threads owning 15 x 15.  Two
 * x-adjacent columns per thread (every value a packed pair over the two
 * columns): 8 x 16 threads owning 15 x 15 nodes, 16 x 8 owning 31 x 7, or
 * 16 x 16 owning 31 x 15.  The two-column tiles apply to the solver's own
 * level-0 vectors (the TMA-fed path). */
#define GMG_FINE_TILE_32X8 0
#define GMG_FINE_TILE_16X16 1
#define GMG_FINE_TILE_PAIR_8X16 2
#define GMG_FINE_TILE_PAIR_16X8 3
#define GMG_FINE_TILE_PAIR_16X16 4

/* Result of gmg_autotune. */
typedef struct {
    int fine_tile;               /* fine kernel tile (GMG_FINE_TILE_*) */
    int fine_zchunk;             /* node planes per block of the z-marching fine kernel */
    int model_tile, model_zchunk;  /* the cost model's choice (used without tuning) */
    int fine_candidates;         /* plans timed */
    double fine_us, model_us;    /* one fine smoothing step: tuned plan, model plan (median of reps) */
    int bsr_kind[16];            /* per level: 0 streaming (a thread per node), 1 / 2 / 3 / 4 / 5 K-split
                                    with 8 / 2 / 4 / 16 / 32 slices per node, 6 level 1 applied
                                    matrix-free from the fine moduli (only where that equals the
                                    assembled operator: even fine sizes, every fixed fine DOF with
                                    fixed prolongation parents), -1 not tuned (fine level, TMA-staged
                                    levels, levels inside the fused lower V-cycle) */
    double bsr_us[16];           /* chosen kernel, one smoothing step */
    double bsr_alt_us[16];       /* the fastest other kernel */
} gmg_tuning;

/* Measures the launch shapes of the handle's hot kernels on its own operands
 * and keeps the fastest: the fine kernel's tile shape and z-chunk length
 * (candidates of both tile shapes and z-chunks from the whole depth down to 4
 * planes, timed as fused Chebyshev/Jacobi smoothing steps; the choice holds
 * for every handle of that fine grid in this process), and per assembled
 * level outside the TMA-staged and fused paths the streaming SpMV kernel or
 * the K-split one with 8, 2, 4, 16 or 32 slices per node (kept in this handle).  The operator's results do not depend on
 * these shapes (each node's arithmetic is the same); reduction partial sums
 * are grouped differently.  reps: timed launches per candidate (>= 1); 0
 * returns to the cost model's plan and to the options' bsr_kernel choice.  Drops the handle's
 * captured solve graphs.  Synchronous.  out may be NULL. */
int gmg_autotune(gmg_handle* h, int reps, gmg_tuning* out);

/* Pins the fine kernel's plan for the handle's fine grid: tile (GMG_FINE_TILE_*)
 * and zchunk node planes per block (>= 1; clamped to the grid's depth); the
 * choice holds for every handle of that fine grid in this process, like
 * gmg_autotune's.  tile < 0 returns to the cost model's plan.  The operator's
 * results do not depend on the plan (each element's arithmetic is the same);
 * reduction partial sums are grouped differently.  GMG_ERR_ARG for an unknown
 * tile, zchunk < 1, or a plan with more blocks than the handle's partial-sum
 * buffer holds.  Drops the handle's captured solve graphs.  Synchronous. */
int gmg_set_fine_plan(gmg_handle* h, int tile, int zchunk);

/* z = V(r): one V-cycle of Eq. vcycle on the fine level. */
int gmg_vcycle(gmg_handle* h, const float* r_dev, float* z_dev);

/* FP64 true residual r = f - K u on the fine level (r_dev may be NULL) and
 * *rel_out = ||r_free|| / ||f_free|| (HOST double; synchronises). */
int gmg_residual64(gmg_handle* h, const double* f_dev, const double* u_dev, double* r_dev,
                   double* rel_out);

/* ---- allocation-free residual check -------------------------------------
 * The paper has no counterpart of this entry point.  It computes the same FP64
 * true residual as gmg_residual64 (r = f - K u on the fine level, *rel_out =
 * ||r_free|| / ||f_free||) for callers that cannot call cudaMalloc: code that
 * runs inside a framework owning every device allocation through its own pool,
 * a plug-in that must not grow the process's device footprint behind its host,
 * or a check run when the device has no free memory left.  It needs no handle
 * and allocates nothing; the caller passes every input and output:
 *   g       : element counts; the grid must need at most 65,536 blocks of 32x4x2
 *             nodes (e.g. 100^3 needs 5,304), otherwise GMG_ERR_ARG with a message
 *             in gmg_last_error() and nothing is launched;
 *   E_dev   : device double[nx*ny*nz] element moduli E_e;
 *   mask_dev: device uint8[n_nodes] fixed-component bits (bit c set = DOF c fixed);
 *   nu      : Poisson ratio of the unit element stiffness;
 *   f_dev, u_dev : device double[3*n_nodes]; r_dev : device double[3*n_nodes] or NULL;
 *   rel_out : HOST double; stream : cudaStream_t or NULL (the call synchronises it).
 *             When f has no nonzero free entry, *rel_out is 0 if r_free is zero
 *             too and +inf otherwise.
 * Grids whose 3 x node count reaches 2^31 are rejected like oversized ones.
 * A failed copy or synchronisation (where faults of the kernels surface)
 * returns GMG_ERR_CUDA with the CUDA error text in gmg_last_error().
 * Its scratch (the element stiffness, two sums and the per-block partial sums:
 * (576 + 2 + 65,536) doubles = 528,912 bytes, 516.5 KiB) is a static device
 * array that every GPU loading this library holds until the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  All calls share the array: calls whose kernels
 * overlap on the GPU (for example on two streams) race and must be serialised
 * by the caller.  Each call rewrites every scratch word it reads, so nothing
 * carries over from the previous call. */
int gmg_residual64_noalloc(const gmg_grid* g, const double* E_dev, const uint8_t* mask_dev, double nu,
                           const double* f_dev, const double* u_dev, double* r_dev, double* rel_out,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GMG_B300_H */
