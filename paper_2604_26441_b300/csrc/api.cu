// C ABI of the GMG-preconditioned CG solver: set-up of the hierarchy, the
// V-cycle of Eq. vcycle, and the outer PCG with true-residual acceptance
// (Sec. "Outer Krylov Solver and Convergence Statement").  Host code here only
// sequences kernels and moves scalars; every arithmetic step runs on the GPU.
#include <algorithm>
#include <vector>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

#include "internal.cuh"

using namespace gmg;

namespace {

thread_local std::string g_err;

}  // namespace

namespace gmg {
std::atomic<unsigned long long> g_kernel_launches{0};
void set_error_text(const std::string& msg) { g_err = msg; }

namespace {
std::vector<BoundsReader>& bounds_readers() {
    static std::vector<BoundsReader> v;  // filled during static initialisation
    return v;
}
}  // namespace
void register_bounds_reader(BoundsReader r) { bounds_readers().push_back(r); }
// The first recorded out-of-range site of any translation unit (0: none); all
// words are cleared.  Synchronises the device first.
unsigned bounds_site_collect() {
    if (bounds_readers().empty()) return 0;
    cudaDeviceSynchronize();
    unsigned first = 0;
    for (BoundsReader r : bounds_readers()) {
        const unsigned v = r();
        if (!first) first = v;
    }
    return first;
}
}  // namespace gmg

namespace {

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CU(expr)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) return fail(GMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                 \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != GMG_OK) return rc_; \
    } while (0)

template <class T>
int dalloc(gmg_handle* h, T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GMG_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return GMG_OK;
}

void dfree(gmg_handle* h, void* p) {
    if (!p) return;
    for (auto& a : h->allocs)
        if (a == p) { a = nullptr; break; }
    cudaFree(p);
}

long long nodes_of(int nx, int ny, int nz) { return (long long)(nx + 1) * (ny + 1) * (nz + 1); }

// ---- level operations -----------------------------------------------------
FineArgs fine_args(gmg_handle* h) {
    const Level& l = h->lev[0];
    FineArgs a{};
    a.nx = l.nx; a.ny = l.ny; a.nz = l.nz;
    a.pitch = l.px; a.epitch = h->ex; a.Ep = h->E32p;
    a.E = h->E32; a.mask = l.maskp; a.kd = h->kd; a.inv0 = h->inv0; a.coef = l.coef;
    a.tcB = h->tcB; a.err = h->kerr;
    return a;
}

BsrArgs bsr_args(gmg_handle* h, int li) {
    const Level& l = h->lev[li];
    BsrArgs a{};
    a.nx = l.nx; a.ny = l.ny; a.nz = l.nz; a.nn = l.nn;
    a.A = l.A32; a.ps = l.ps; a.invdiag = l.invdiag; a.mask = l.mask; a.coef = l.coef;
    a.err = h->kerr;
    a.kind = l.bsr_kind;
    if (l.tma) { a.tm_own = &l.tm_own; a.tm_back = &l.tm_back; }
    if (l.eh) { a.eh = l.eh; a.l1g = &h->l1g; a.cf = l.cf; }
    return a;
}

// The level kernel a level uses without tuning: the options' choice, or for
// level 1 under the size rule the matrix-free form where it is exact.
int default_bsr_kind(const gmg_handle* h, int li) {
    const Level& l = h->lev[li];
    if (li == 1 && l.eh && h->opt.bsr_kernel < 0 && !l.tma) return kBsrMatrixFree;
    return h->opt.bsr_kernel;
}

// The device view of assembled level li used by the cooperative and
// single-block kernels (coarse_fused.cu).
CoarseLevel coarse_view(const gmg_handle* h, int li) {
    const Level& l = h->lev[li];
    CoarseLevel c{};
    c.nx = l.nx; c.ny = l.ny; c.nz = l.nz; c.nn = (int)l.nn;
    c.mask = l.mask; c.A = l.A32; c.ps = (int)l.ps; c.invdiag = l.invdiag;
    c.x = l.x; c.x2 = l.x2; c.b = l.b; c.t = l.t; c.d = l.d;
    c.coef = l.coef; c.kind = l.kind; c.degree = l.degree;
    return c;
}

int partial_count(gmg_handle* h, int li, int kind) {
    // kind 0: operator-kernel partials, 1: vector-kernel partials
    if (kind == 1) return vec_grid_blocks();
    if (li == 0) return fine_grid_blocks(h->lev[0].nx, h->lev[0].ny, h->lev[0].nz);
    const Level& l = h->lev[li];
    if (l.bsr_kind == kBsrMatrixFree && l.eh && !l.tma) return l1mf_grid_blocks(l.nx, l.ny, l.nz);
    return bsr_grid_blocks(l.nn, l.tma, l.bsr_kind);
}

// y = K^l x (masked); with dot: partial += x . y and finalised into `slot`.
// Level-0 operands are level-0 vectors (padded rows, 0 on fixed DOFs); entry
// points that take a caller's dense vector pack it first (launch_pack0).
void level_apply(gmg_handle* h, int li, const float* x, float* y, int dot_slot = -1, int op = FIN_NONE) {
    cudaStream_t s = h->stream;
    const bool dot = dot_slot >= 0;
    if (li == 0) {
        FineArgs a = fine_args(h);
        a.xin = x; a.out = y; a.partial = dot ? h->partials : nullptr;
        launch_fine(FM_APPLY, dot, 0, a, h->gs, s);
    } else {
        BsrArgs a = bsr_args(h, li);
        a.xin = x; a.out = y; a.partial = dot ? h->partials : nullptr;
        launch_bsr(FM_APPLY, dot, a, s);
    }
    if (dot) launch_finalize(h->partials, partial_count(h, li, 0), h->sc, dot_slot, op, s);
}

void level_resid(gmg_handle* h, int li, const float* b, const float* x, float* t) {
    if (li == 0) {
        FineArgs a = fine_args(h);
        a.xin = x; a.b = b; a.out = t;
        launch_fine(FM_RESID, 0, 0, a, h->gs, h->stream);
    } else {
        BsrArgs a = bsr_args(h, li);
        a.xin = x; a.b = b; a.out = t;
        launch_bsr(FM_RESID, 0, a, h->stream);
    }
}

// One smoother step k on level li: reads x_cur (ignored when zero_init), writes x_next.
// rfrom (levels >= 1, zero_init only): the finer level's residual; the step then
// first restricts it into the level's own b (l.b, which b must be).
// dold_from (level 0): read the previous increment from there instead of the
// level's d vector (after a first step from zero, whose increment is its output).
void smooth_step(gmg_handle* h, int li, int k, bool zero_init, const float* b, const float* xcur, float* xnext,
                 bool write_d, bool dot, const float* rfrom = nullptr, const float* dold_from = nullptr) {
    Level& l = h->lev[li];
    float* d = li == 0 ? h->d0 : l.d;
    cudaStream_t s = h->stream;
    if (li == 0) {
        FineArgs a = fine_args(h);
        a.b = b; a.out = xnext; a.step = k; a.dold = dold_from ? dold_from : d; a.dnew = write_d ? d : nullptr;
        a.partial = dot ? h->partials : nullptr;
        if (zero_init) launch_fine_smooth0(a, s);
        else if (h->opt.fine_smoother != GMG_FINE_FP32) {
            a.xin = xcur;
            launch_fine_tc(h->opt.fine_smoother == GMG_FINE_BF16X3 ? 3 : 1, dot, a, s);
        } else { a.xin = xcur; launch_fine(FM_SMOOTH, dot, 0, a, h->gs, s); }
    } else {
        BsrArgs a = bsr_args(h, li);
        a.b = b; a.out = xnext; a.step = k; a.dold = d; a.dnew = write_d ? d : nullptr;
        a.partial = dot ? h->partials : nullptr;
        if (zero_init && rfrom) launch_restrict_smooth0(h->lev[li - 1], rfrom, a, l.b, s);
        else if (zero_init) launch_bsr_smooth0(a, s);
        else { a.xin = xcur; launch_bsr(FM_SMOOTH, dot, a, s); }
    }
}

// A smoothing pass of `degree` steps.  Writes alternate S, X, S, ...; returns the
// buffer holding the result.  With dot_slot >= 0 the last step also forms b . x.
float* smooth_pass(gmg_handle* h, int li, const float* b, float* cur, float* X, float* S, bool zero_init,
                   int& writes, int dot_slot = -1, int op = FIN_NONE, const float* rfrom = nullptr) {
    Level& l = h->lev[li];
    const bool cheb = l.kind == GMG_SMOOTHER_CHEBYSHEV;
    // fine level: a first step from zero leaves d = x, so the next step reads its
    // increment from that step's output and no copy of it is written
    const float* d_alias = nullptr;
    for (int k = 0; k < l.degree; ++k) {
        float* next = (writes % 2 == 0) ? S : X;
        const bool last = k == l.degree - 1;
        const bool dot = last && dot_slot >= 0;
        const bool alias = li == 0 && zero_init && k == 0;
        smooth_step(h, li, k, zero_init && k == 0, b, cur, next, cheb && !last && !alias, dot, k == 0 ? rfrom : nullptr,
                    k == 1 ? d_alias : nullptr);
        if (alias && cheb && !last) d_alias = next;
        if (dot) launch_finalize(h->partials, partial_count(h, li, 0), h->sc, dot_slot, op, h->stream);
        cur = next;
        ++writes;
    }
    return cur;
}

// Eq. vcycle on level li: X = V(b), using S as the ping-pong partner.  With
// cycle index 2 (W-cycle) the coarse level is visited twice, the second visit
// starting from the first one's result (warm: pre-smoothing from the current X).
// rfrom: b is this level's own b, still to be restricted from the finer level's
// residual rfrom; the first pre-smoothing step does that (one launch instead of
// a restriction and a first step).
void vcycle_level(gmg_handle* h, int li, const float* b, float* X, float* S, int dot_slot, int op,
                  bool warm = false, const float* rfrom = nullptr) {
    Level& l = h->lev[li];
    cudaStream_t s = h->stream;
    if (h->use_fused && li == h->cf.start && !warm) {
        // levels li..L-1 and the coarsest solve in one persistent kernel; b and X
        // are this level's own b and x buffers on this path
        launch_coarse_fused(h->cf, h->fused_blocks, s);
        return;
    }
    if (h->use_lc && li == h->L - 2 && !warm && rfrom && b == l.b && X == l.x) {
        // this level and the coarsest solve in one cluster launch; the result in l.x
        const Level& f = h->lev[li - 1];
        const Level& c = h->lev[li + 1];
        LowerClusterArgs a{};
        a.fnx = f.nx; a.fny = f.ny; a.fnz = f.nz; a.ft = rfrom;
        a.m = coarse_view(h, li);
        a.cnx = c.nx; a.cny = c.ny; a.cnz = c.nz; a.cnn = (int)c.nn;
        a.cmask = c.mask; a.cb = c.b; a.cx = c.x;
        a.nL = h->nL; a.free_idx = h->free_idx; a.Ahi = h->Ahi; a.Alo = h->Alo;
        launch_lower_cluster(a, h->lc_smem, s);
        return;
    }
    if (li == h->L - 1) {
        if (h->coarse_pcg) launch_coarse_pcg(coarse_view(h, li), b, X, l.t, l.d, l.x2, h->opt.coarse_pcg_steps, s);
        else launch_coarse_solve(h->nL, h->free_idx_p, h->Ainv, b, X, l.maskp, l.nnp, s);
        return;
    }
    int writes = 0;
    float* cur = smooth_pass(h, li, b, warm ? X : nullptr, X, S, !warm, writes, -1, FIN_NONE, warm ? nullptr : rfrom);
    float* t = li == 0 ? h->t0 : l.t;
    level_resid(h, li, b, cur, t);
    Level& c = h->lev[li + 1];
    // the restriction rides on the coarse level's first smoothing step, except
    // into the coarsest level (dense solve) or the fused lower V-cycle
    const bool fuse = li + 1 < h->L - 1 && !(h->use_fused && li + 1 == h->cf.start);
    if (!fuse) launch_restrict(l, c, t, c.b, s);
    const int gamma = li + 1 == h->L - 1 ? 1 : std::max(1, h->opt.cycle_index);  // exact coarsest: one visit
    for (int g = 0; g < gamma; ++g)
        vcycle_level(h, li + 1, c.b, c.x, c.x2, -1, FIN_NONE, g > 0, fuse && g == 0 ? t : nullptr);
    launch_prolong_add(l, c, c.x, cur, s);
    smooth_pass(h, li, b, cur, X, S, false, writes, dot_slot, op);
}

// lambda_max(D^{-1} K) of level li by power iteration (Sec. "Spectral-radius estimation").
void power_iteration(gmg_handle* h, int li, int iters) {
    Level& l = h->lev[li];
    cudaStream_t s = h->stream;
    const long long n = 3 * l.nnp;
    float* v = li == 0 ? h->t0 : l.t;
    float* w = li == 0 ? h->x2_0 : l.x2;
    float* y = li == 0 ? h->d0 : l.d;
    cudaMemsetAsync(h->sc + SC_TMP, 0, sizeof(double), s);
    launch_power_start(v, l, s);
    launch_dot_f32(v, v, n, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_NRM, FIN_NRMCHK, s);
    launch_scale_by_inv_sqrt(v, n, h->sc, SC_NRM, s);
    for (int it = 0; it < iters; ++it) {
        level_apply(h, li, v, y);
        if (li == 0) launch_scale_invdiag_fine(y, w, h->E32, l, h->kd, s);
        else launch_scale_invdiag_bsr(y, w, l.invdiag, n, s);
        launch_dot_f32(w, w, n, h->partials, s);
        launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_NRM, FIN_NRMCHK, s);
        launch_scale_by_inv_sqrt(w, n, h->sc, SC_NRM, s);
        std::swap(v, w);
    }
    level_apply(h, li, v, y);
    launch_dot_f32(v, y, n, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_VKV, FIN_NONE, s);
    if (li == 0) launch_diag_dot_fine(v, h->E32, l, h->kd, h->partials, s);
    else launch_diag_dot_bsr(v, l.invdiag, n, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_VDV, FIN_NONE, s);
    launch_lambda_finish(h->sc, h->lam + li, s);
}

void refresh_coef(gmg_handle* h, int li) {
    Level& l = h->lev[li];
    launch_smoother_coef(l.coef, h->lam + li, l.kind, l.degree, l.omega, h->opt.cheb_alpha, h->opt.lambda_safety,
                         h->stream);
}

int check_level(const gmg_handle* h, int li) {
    if (!h) return fail(GMG_ERR_ARG, "null handle");
    if (li < 0 || li >= h->L) return fail(GMG_ERR_ARG, "level index out of range");
    return GMG_OK;
}

// Device scalars -> sc_host (and the sticky error words -> err_host): the device
// writes the pinned host-mapped block itself, so the read-back uses no copy
// engine and cannot wait behind a caller's large copies on other streams.
int sync_scalars(gmg_handle* h) {
    launch_publish(h->sc, SC_COUNT, h->sc_map, h->kerr, h->use_fused ? h->cf.err : nullptr, h->err_map, h->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    return GMG_OK;
}

// The pinned host-mapped block of sc_host and err_host.
int alloc_mirror(gmg_handle* h) {
    const size_t bytes = sizeof(double) * SC_COUNT + 4 * sizeof(int) + sizeof(double) * (kMaxRestart + 2);
    if (cudaHostAlloc(&h->pinned, bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        h->pinned = nullptr;
        return fail(GMG_ERR_NOMEM, "pinned host-mapped scalar block");
    }
    void* dev = nullptr;
    if (cudaHostGetDevicePointer(&dev, h->pinned, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(GMG_ERR_CUDA, "no device address for the host-mapped scalar block");
    }
    memset(h->pinned, 0, bytes);
    h->sc_host = static_cast<double*>(h->pinned);
    h->err_host = reinterpret_cast<int*>(h->sc_host + SC_COUNT);
    h->sc_map = static_cast<double*>(dev);
    h->err_map = reinterpret_cast<int*>(h->sc_map + SC_COUNT);
    h->hcol_host = reinterpret_cast<double*>(h->err_host + 4);
    h->hcol_map = reinterpret_cast<double*>(h->err_map + 4);
    return GMG_OK;
}

int build(gmg_handle* h, const gmg_grid* g, const float* rho, double p, double E0, double Emin, double nu,
          const gmg_bc* bc) {
    cudaStream_t s = h->stream;
    const gmg_options& o = h->opt;
    // ---- fine level and masks
    Level& l0 = h->lev[0];
    l0.nx = g->nx; l0.ny = g->ny; l0.nz = g->nz;
    l0.nn = nodes_of(g->nx, g->ny, g->nz);
    l0.px = (g->nx + 1 + 3) / 4 * 4;
    l0.nnp = (long long)l0.px * (g->ny + 1) * (g->nz + 1);
    TRY(dalloc(h, &l0.mask, l0.nn));
    if (bc->kind == GMG_BC_CLAMP_XMIN) {
        launch_mask_clamp(l0.mask, l0.nx, l0.ny, l0.nz, s);
    } else {
        uint8_t* tmp = nullptr;
        TRY(dalloc(h, &tmp, 3 * l0.nn));
        CU(cudaMemcpyAsync(tmp, bc->fixed, 3 * l0.nn, cudaMemcpyHostToDevice, s));
        launch_mask_from_dofs(tmp, l0.mask, l0.nn, s);
        CU(cudaStreamSynchronize(s));
        dfree(h, tmp);
    }
    int* cnt = nullptr;
    TRY(dalloc(h, &cnt, 1));
    auto count_free = [&](const Level& l, int* out) -> int {
        launch_count_free(l.mask, l.nn, cnt, s);
        CU(cudaMemcpyAsync(out, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        return GMG_OK;
    };
    TRY(count_free(l0, &l0.n_free));
    TRY(dalloc(h, &l0.maskp, l0.nnp));
    launch_mask_pad(l0, s);
    int L = 1;
    const int want = o.levels;
    while (true) {
        const Level& f = h->lev[L - 1];
        const bool can = f.nx >= 2 && f.ny >= 2 && f.nz >= 2 && L < kMaxLevels;
        const bool more = want > 0 ? (L < want) : (f.n_free > o.chol_cutoff);
        if (!more) break;
        if (!can) {
            if (want > 0) return fail(GMG_ERR_ARG, "grid too small for the requested number of levels");
            break;
        }
        Level& c = h->lev[L];
        c.nx = f.nx / 2; c.ny = f.ny / 2; c.nz = f.nz / 2;
        c.nn = nodes_of(c.nx, c.ny, c.nz);
        c.px = c.nx + 1;
        c.nnp = c.nn;
        TRY(dalloc(h, &c.mask, c.nn));
        c.maskp = c.mask;
        launch_mask_inject(f, c, s);
        TRY(count_free(c, &c.n_free));
        ++L;
    }
    h->L = L;
    // ---- smoother settings and buffers
    for (int li = 0; li < L; ++li) {
        Level& l = h->lev[li];
        if (li == 0) { l.kind = o.smoother; l.degree = o.degree; l.omega = o.omega; }
        else {
            l.kind = o.coarse_smoother >= 0 ? o.coarse_smoother : o.smoother;
            l.degree = o.coarse_degree > 0 ? o.coarse_degree : o.degree;
            l.omega = o.coarse_omega > 0 ? o.coarse_omega : o.omega;
        }
        TRY(dalloc(h, &l.coef, 2 * kMaxDegree));
        if (li > 0) {
            TRY(dalloc(h, &l.A64, (size_t)kPlanes * l.nn));
            l.ps = (l.nn + 3) / 4 * 4;
            TRY(dalloc(h, &l.A32, (size_t)kSymPlanes * l.ps));
            CU(cudaMemsetAsync(l.A32, 0, sizeof(float) * kSymPlanes * l.ps, s));
            TRY(dalloc(h, &l.invdiag, 3 * l.nn));
            TRY(dalloc(h, &l.x, 3 * l.nn));
            TRY(dalloc(h, &l.x2, 3 * l.nn));
            TRY(dalloc(h, &l.b, 3 * l.nn));
            TRY(dalloc(h, &l.t, 3 * l.nn));
            TRY(dalloc(h, &l.d, 3 * l.nn));
        }
    }
    const long long n0 = 3 * l0.nnp;
    for (float** v : {&h->r, &h->z, &h->p, &h->q, &h->x2_0, &h->t0, &h->d0, &h->wh, &h->wl}) {
        TRY(dalloc(h, v, n0));
        CU(cudaMemsetAsync(*v, 0, sizeof(float) * n0, s));  // the pads stay 0
    }
    const long long ne = (long long)l0.nx * l0.ny * l0.nz;
    TRY(dalloc(h, &h->E32, ne));
    h->ex = (l0.nx + 3) / 4 * 4;
    TRY(dalloc(h, &h->E32p, (long long)h->ex * l0.ny * l0.nz));
    CU(cudaMemsetAsync(h->E32p, 0, sizeof(float) * h->ex * l0.ny * l0.nz, s));
    TRY(dalloc(h, &h->E64, ne));
    TRY(dalloc(h, &h->lam, kMaxLevels));
    TRY(dalloc(h, &h->sc, SC_COUNT));
    CU(cudaMemsetAsync(h->sc, 0, sizeof(double) * SC_COUNT, s));
    TRY(dalloc(h, &h->kerr, 1));
    CU(cudaMemsetAsync(h->kerr, 0, sizeof(int), s));
    int maxp = vec_grid_blocks();
    maxp = std::max(maxp, fine_grid_blocks(l0.nx, l0.ny, l0.nz));
    maxp = std::max(maxp, resid64_grid_blocks(l0.nx, l0.ny, l0.nz));
    // (the kernel of a level is chosen later or by gmg_autotune: size for
    // every kernel, and leave room for the fine kernel's tuning candidates)
    for (int li = 1; li < L; ++li)
        for (int kind = 0; kind < kBsrKinds; ++kind)
            maxp = std::max({maxp, bsr_grid_blocks(h->lev[li].nn, true), bsr_grid_blocks(h->lev[li].nn, false, kind)});
    if (L >= 2) maxp = std::max(maxp, l1mf_grid_blocks(h->lev[1].nx, h->lev[1].ny, h->lev[1].nz));
    maxp = std::max(maxp, 4096);
    h->max_partials = maxp;
    TRY(dalloc(h, &h->partials, maxp));
    TRY(alloc_mirror(h));

    // ---- moduli (Eq. simp_filter) and K_e
    launch_moduli(rho, ne, p, E0, Emin, h->E64, h->E32, s);
    CU(cudaMemcpy2DAsync(h->E32p, sizeof(float) * h->ex, h->E32, sizeof(float) * l0.nx, sizeof(float) * l0.nx,
                         (size_t)l0.ny * l0.nz, cudaMemcpyDeviceToDevice, s));
    double* Ke = nullptr;
    TRY(dalloc(h, &Ke, 576));
    launch_element_stiffness(nu, Ke, s);
    CU(cudaMemcpyAsync(h->keD.v, Ke, sizeof(double) * 576, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int i = 0; i < 576; ++i) h->keF.v[i] = (float)h->keD.v[i];
    h->kd = h->keF.v[0];
    TRY(dalloc(h, &h->inv0, l0.nnp));
    CU(cudaMemsetAsync(h->inv0, 0, sizeof(float) * l0.nnp, s));
    launch_fine_inv0(l0.nx, l0.ny, l0.nz, l0.px, h->E32, h->kd, h->inv0, s);
    {
        double* g72 = nullptr;
        double gh[72];
        TRY(dalloc(h, &g72, 72));
        launch_hadamard_blocks(Ke, g72, s);
        CU(cudaMemcpyAsync(gh, g72, sizeof gh, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (!gsym_from_blocks(gh, &h->gs, h->gs64) || !l1_coef_from_blocks(gh, &h->l1g))
            return fail(GMG_ERR_CUDA, "element stiffness lacks the cube-symmetric block structure");
        if (o.fine_smoother != GMG_FINE_FP32) {
            uint16_t op[2048];
            build_tc_operand(gh, op);
            uint16_t* dev = nullptr;
            TRY(dalloc(h, &dev, 2048));
            CU(cudaMemcpyAsync(dev, op, sizeof op, cudaMemcpyHostToDevice, s));
            CU(cudaStreamSynchronize(s));
            h->tcB = dev;
        }
        dfree(h, g72);
    }

    // ---- Galerkin hierarchy
    if (L >= 2) {
        Level& c = h->lev[1];
        double *Mpat = nullptr, *Kc = nullptr;
        const long long nce = (long long)c.nx * c.ny * c.nz;
        TRY(dalloc(h, &Mpat, 27 * 576));
        TRY(dalloc(h, &Kc, (size_t)nce * 576));
        launch_child_patterns(Ke, Mpat, s);
        launch_coarse_element_matrices(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, Ke, Mpat, Kc, s);
        launch_gather_level1(c, Kc, c.A64, s);
        launch_finish_bsr(c, s);
        CU(cudaStreamSynchronize(s));
        dfree(h, Kc);
        dfree(h, Mpat);
        for (int li = 2; li < L; ++li) {
            launch_galerkin_rap(h->lev[li - 1], h->lev[li], s);
            launch_finish_bsr(h->lev[li], s);
        }
    }
    // ---- level 1 matrix-free where that equals the assembled operator (a
    // smoothed level, even fine sizes, fixed fine DOFs with fixed parents)
    if (L >= 3 && !(o.bsr_tma_nodes > 0 && h->lev[1].nn >= o.bsr_tma_nodes)) {
        std::vector<uint8_t> m0((size_t)l0.nn);
        CU(cudaMemcpyAsync(m0.data(), l0.mask, m0.size(), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (l1mf_eligible(l0.nx, l0.ny, l0.nz, m0.data())) {
            Level& c = h->lev[1];
            TRY(dalloc(h, &c.eh, 8 * (size_t)c.nx * c.ny * c.nz));
            TRY(dalloc(h, &c.cf, 32 * (size_t)c.nx * c.ny * c.nz));
            launch_l1_ehat(h->E64, l0.nx, l0.ny, l0.nz, c.eh, s);
        }
    }
    for (int li = 1; li < L; ++li) h->lev[li].bsr_kind = default_bsr_kind(h, li);
    CU(cudaGetLastError());

    // ---- spectral estimates and smoother coefficients
    for (int li = 0; li < L; ++li) {
        power_iteration(h, li, li == 0 ? o.power_iters_fine : o.power_iters_coarse);
        refresh_coef(h, li);
    }
    double lam_host[kMaxLevels];
    CU(cudaMemcpyAsync(lam_host, h->lam, sizeof(double) * L, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int li = 0; li + 1 < L; ++li) {
        const Level& l = h->lev[li];
        if (l.kind == GMG_SMOOTHER_JACOBI && l.omega * lam_host[li] >= 2.0) {
            char buf[160];
            snprintf(buf, sizeof buf, "damped Jacobi unstable on level %d: omega %.3g * lambda_max %.4g >= 2", li,
                     l.omega, lam_host[li]);
            return fail(GMG_ERR_SMOOTHER, buf);
        }
    }

    // ---- coarsest level: dense K^L_ff + eps I, Cholesky, inverse
    Level& cl = h->lev[L - 1];
    TRY(dalloc(h, &h->free_idx, 3 * cl.nn));
    launch_free_index(cl.mask, cl.nn, h->free_idx, cnt, s);
    CU(cudaMemcpyAsync(&h->nL, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h->nL > o.chol_cutoff) {
        // above the cutoff the coarsest level is solved by a fixed-count PCG on
        // its assembled operator (the fine level has none: one level is refused)
        if (L == 1)
            return fail(GMG_ERR_ARG, "a single-level hierarchy with " + std::to_string(h->nL) +
                                         " free DOFs exceeds the dense-Cholesky cutoff; use more levels");
        h->coarse_pcg = true;
    }
    if (h->nL > 0 && !h->coarse_pcg) {
        const int n = h->nL;
        double *dense = nullptr, *work = nullptr, *eps_dev = nullptr;
        int* info = nullptr;
        TRY(dalloc(h, &dense, (size_t)n * n));
        TRY(dalloc(h, &work, (size_t)n * n));
        TRY(dalloc(h, &h->Ainv, (size_t)n * n));
        TRY(dalloc(h, &eps_dev, 1));
        TRY(dalloc(h, &info, 1));
        if (L == 1) {
            // one-level hierarchy: assemble the fine operator into the 27-slot
            // planes (element matrices E_e K_e scattered by owner nodes) so that the
            // dense coarsest gather below can read it
            double* Kc = nullptr;
            const long long ne0 = (long long)l0.nx * l0.ny * l0.nz;
            TRY(dalloc(h, &l0.A64, (size_t)kPlanes * l0.nn));
            l0.ps = (l0.nn + 3) / 4 * 4;
            TRY(dalloc(h, &l0.A32, (size_t)kSymPlanes * l0.ps));
            CU(cudaMemsetAsync(l0.A32, 0, sizeof(float) * kSymPlanes * l0.ps, s));
            TRY(dalloc(h, &l0.invdiag, 3 * l0.nn));
            TRY(dalloc(h, &Kc, (size_t)ne0 * 576));
            launch_fine_element_matrices(h->E64, ne0, Ke, Kc, s);
            launch_gather_level1(l0, Kc, l0.A64, s);
            launch_finish_bsr(l0, s);
            CU(cudaStreamSynchronize(s));
            dfree(h, Kc);
        }
        launch_dense_gather(cl, h->free_idx, n, dense, s);
        if (L == 1) {  // the coarsest level is level 0: its vectors have padded rows
            TRY(dalloc(h, &h->free_idx_p, n));
            launch_pad_index(h->free_idx, n, l0, h->free_idx_p, s);
        }
        launch_regularise(dense, n, eps_dev, s);
        CU(cudaMemcpyAsync(&h->eps, eps_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        const int rc = cholesky_and_inverse(dense, n, work, info, h->Ainv, s);
        if (rc == GMG_ERR_CHOLESKY) return fail(rc, "coarsest matrix is not positive definite");
        if (rc != GMG_OK) return fail(rc, "coarsest factorisation failed");
        CU(cudaStreamSynchronize(s));
        dfree(h, dense);
        dfree(h, work);
    }
    if (!h->free_idx_p) h->free_idx_p = h->free_idx;
    // ---- TMA-staged operator for the large assembled levels
    for (int li = 1; li < L; ++li) {
        Level& l = h->lev[li];
        if (o.bsr_tma_nodes > 0 && l.nn >= o.bsr_tma_nodes) {
            const int rc = encode_bsr_maps(l);
            if (rc != GMG_OK) return fail(rc, "could not encode the tensor maps of an assembled level");
        }
    }
    // ---- fused lower V-cycle: every assembled level below the node threshold
    if (o.fused_coarse_nodes > 0 && L >= 2 && o.cycle_index <= 1 && !h->coarse_pcg) {
        int start = L - 1;
        while (start - 1 >= 1 && h->lev[start - 1].nn < o.fused_coarse_nodes) --start;
        if (h->lev[start].nn < o.fused_coarse_nodes || start == L - 1) {
            CoarseFused& cf = h->cf;
            cf.start = start;
            cf.L = L;
            cf.nL = h->nL;
            cf.free_idx = h->free_idx;
            cf.Ainv = h->Ainv;
            for (int li = 1; li < L; ++li) {
                const Level& l = h->lev[li];
                CoarseLevel& c = cf.lev[li];
                c.nx = l.nx; c.ny = l.ny; c.nz = l.nz; c.nn = (int)l.nn;
                c.mask = l.mask; c.A = l.A32; c.ps = (int)l.ps; c.invdiag = l.invdiag;
                c.x = l.x; c.x2 = l.x2; c.b = l.b; c.t = l.t; c.d = l.d;
                c.coef = l.coef; c.kind = l.kind; c.degree = l.degree;
            }
            unsigned* words = nullptr;
            TRY(dalloc(h, &words, 4));
            CU(cudaMemsetAsync(words, 0, 4 * sizeof(unsigned), s));
            cf.bar_count = words;
            cf.bar_gen = words + 1;
            cf.err = reinterpret_cast<int*>(words + 2);
            cf.spin_limit = o.spin_limit;
            if (coarse_fused_blocks(&h->fused_blocks, sizeof(double) * (size_t)std::max(h->nL, 1)) == GMG_OK &&
                h->fused_blocks > 0)
                h->use_fused = true;
        }
    }
    // ---- the bottom of the V-cycle (level L-2 >= 2 and the dense coarsest solve)
    // as one thread-block cluster launch, when its operator fits the cluster
    if (o.lower_cluster && !h->use_fused && o.bsr_kernel < 0 && !h->coarse_pcg && h->nL > 0 && L >= 4) {
        const size_t smem = lower_cluster_smem((int)h->lev[L - 2].nn, h->nL);
        if (lower_cluster_available(smem)) {
            const size_t n2 = (size_t)h->nL * h->nL;
            TRY(dalloc(h, &h->Ahi, n2));
            TRY(dalloc(h, &h->Alo, n2));
            launch_split_inverse(h->Ainv, (long long)n2, h->Ahi, h->Alo, s);
            h->use_lc = true;
            h->lc_smem = smem;
        }
    }
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
    return GMG_OK;
}

// ---- PCG steps (Sec. "Outer Krylov Solver and Convergence Statement"), shared
// by the host-driven loop and the captured graph ---------------------------------
// z = V(r), rz = r . z, p = z
void pcg_restart(gmg_handle* h) {
    const long long n = 3 * h->lev[0].nnp;
    vcycle_level(h, 0, h->r, h->z, h->x2_0, SC_RZ, FIN_NONE);
    launch_copy_f32(h->p, h->z, n, h->stream);
}
// q = K p, alpha = rz / p.q, w += alpha p (the iterate's pending change, added
// to u by flush_w), r -= alpha q, ||r||^2; with cond (inside the captured loop)
// the ||r||^2 reduction also takes the loop's convergence test.
void pcg_step(gmg_handle* h, const cudaGraphConditionalHandle* cond = nullptr) {
    level_apply(h, 0, h->p, h->q, SC_PQ, FIN_ALPHA);
    launch_pcg_update(h->wh, h->wl, h->r, h->p, h->q, h->lev[0], h->sc, h->partials, h->stream);
    if (cond) launch_finalize_check(h->partials, vec_grid_blocks(), h->sc, *cond, h->stream);
    else launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_RR, FIN_NONE, h->stream);
    h->w_dirty = true;
}
// u += w, w = 0 (before u is read: the FP64 residual, the end of a solve)
void flush_w(gmg_handle* h, double* u) {
    if (!h->w_dirty) return;
    launch_flush_w(u, h->wh, h->wl, h->lev[0], h->stream);
    h->w_dirty = false;
}
// w = 0 without touching an iterate (steps of an abandoned call)
int reset_w(gmg_handle* h) {
    if (!h->w_dirty) return GMG_OK;
    const long long n = 3 * h->lev[0].nnp;
    CU(cudaMemsetAsync(h->wh, 0, sizeof(float) * n, h->stream));
    CU(cudaMemsetAsync(h->wl, 0, sizeof(float) * n, h->stream));
    h->w_dirty = false;
    return GMG_OK;
}
// z = V(r), beta = r.z / rz, p = z + beta p
void pcg_direction(gmg_handle* h) {
    const long long n = 3 * h->lev[0].nnp;
    vcycle_level(h, 0, h->r, h->z, h->x2_0, SC_RZNEW, FIN_BETA);
    launch_p_update(h->p, h->z, n, h->sc, h->stream);
}

// After a solve that ended non-finite, a non-finite step length may have been
// spread over the pad entries of the level-0 vectors by the full-length vector
// kernels; the next call on the handle starts from zeroed vectors.
int clear_pads(gmg_handle* h) {
    if (!h->pads_dirty) return GMG_OK;
    const long long n = 3 * h->lev[0].nnp;
    for (float* v : {h->r, h->z, h->p, h->q, h->x2_0, h->t0, h->d0, h->wh, h->wl})
        CU(cudaMemsetAsync(v, 0, sizeof(float) * n, h->stream));
    if (h->fg_V) CU(cudaMemsetAsync(h->fg_V, 0, sizeof(float) * (size_t)(h->fg_m + 1) * n, h->stream));
    if (h->fg_Z) CU(cudaMemsetAsync(h->fg_Z, 0, sizeof(float) * (size_t)h->fg_m * n, h->stream));
    h->w_dirty = false;
    h->pads_dirty = false;
    return GMG_OK;
}

void loop_free(gmg_handle* h) {
    if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
    if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    h->loop_u = nullptr;
    for (auto& e : h->loop_cache) {
        cudaGraphExecDestroy(e.ex);
        cudaGraphDestroy(e.g);
    }
    h->loop_cache.clear();
}

// Captures the device-resident PCG loop for iterate u:
//   restart; step; check; while (condition) { direction; step; check }
// so that one graph launch runs PCG until the recursive residual passes the
// tolerance (or the cap, or a non-finite scalar) with no host round trip; the
// host then takes the FP64 acceptance decision.  The kernel sequence is that of
// the host-driven loop, so both give bitwise-identical iterates.
// Captures [restart, step, check, while (condition) {direction, step, check}]
// for handle h and iterate u into graph g as an independent branch (no
// dependencies on nodes already in g), using stream cap for the capture.
// Returns false on any capture error; prefix / body receive the kernel counts.
bool capture_loop(gmg_handle* h, double* u, cudaGraph_t g, cudaStream_t cap, unsigned long long& prefix,
                  unsigned long long& body_k) {
    const unsigned long long l0 = g_kernel_launches.load();
    cudaStream_t user = h->stream;
    h->stream = cap;
    cudaGraph_t body = nullptr, out = nullptr;
    cudaGraphConditionalHandle cond{};
    unsigned long long l1 = l0, l2 = l0;
    bool ok = cudaGraphConditionalHandleCreate(&cond, g, 0, 0) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        pcg_restart(h);
        pcg_step(h, &cond);
        l1 = g_kernel_launches.load();
        cudaStreamCaptureStatus st{};
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode = nullptr;
        ok = cudaStreamGetCaptureInfo(cap, &st, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess &&
             st == cudaStreamCaptureStatusActive;
        if (ok) ok = cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp) == cudaSuccess;
        if (ok) ok = cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                     cudaSuccess;
        if (ok) body = cp.conditional.phGraph_out[0];
        ok = (cudaStreamEndCapture(cap, &out) == cudaSuccess) && ok;
    }
    if (ok) {
        ok = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            pcg_direction(h);
            pcg_step(h, &cond);
            l2 = g_kernel_launches.load();
            ok = cudaStreamEndCapture(cap, &body) == cudaSuccess;
        }
    }
    h->stream = user;
    g_kernel_launches.fetch_sub(g_kernel_launches.load() - l0);  // capturing launches nothing
    cudaGetLastError();
    prefix = l1 - l0;
    body_k = l2 - l1;
    return ok;
}

int ensure_cap_stream(gmg_handle* h) {
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return GMG_ERR_CUDA;
    }
    return GMG_OK;
}

// Captures the loop for u into the handle's current slot (which must be empty).
int loop_capture(gmg_handle* h, double* u) {
    TRY(ensure_cap_stream(h));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    unsigned long long pre = 0, bod = 0;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess && capture_loop(h, u, g, h->cap_stream, pre, bod);
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    cudaGetLastError();
    if (!ok) {
        if (g) cudaGraphDestroy(g);
        return GMG_ERR_CUDA;
    }
    h->loop_graph = g;
    h->loop_exec = ex;
    h->loop_u = u;
    h->loop_prefix_kernels = pre;
    h->loop_body_kernels = bod;
    return GMG_OK;
}

constexpr size_t kLoopCache = 3;  // loops kept besides the current one

// Makes the loop of iterate u the current one: taken from the cache when it
// was captured before, else captured now; the previous current loop is kept
// in the cache (the least recently used one is dropped beyond kLoopCache).
int loop_select(gmg_handle* h, double* u) {
    if (h->loop_exec && h->loop_u == u) return GMG_OK;
    auto park = [&] {
        if (!h->loop_exec) return;
        h->loop_cache.push_back({h->loop_u, h->loop_graph, h->loop_exec, h->loop_prefix_kernels, h->loop_body_kernels});
        h->loop_exec = nullptr;
        h->loop_graph = nullptr;
        h->loop_u = nullptr;
        if (h->loop_cache.size() > kLoopCache) {
            cudaGraphExecDestroy(h->loop_cache.front().ex);
            cudaGraphDestroy(h->loop_cache.front().g);
            h->loop_cache.erase(h->loop_cache.begin());
        }
    };
    for (size_t i = 0; i < h->loop_cache.size(); ++i)
        if (h->loop_cache[i].u == u) {
            const gmg_handle::LoopGraph e = h->loop_cache[i];
            h->loop_cache.erase(h->loop_cache.begin() + (long)i);
            park();
            h->loop_u = e.u;
            h->loop_graph = e.g;
            h->loop_exec = e.ex;
            h->loop_prefix_kernels = e.pre;
            h->loop_body_kernels = e.body;
            return GMG_OK;
        }
    park();
    return loop_capture(h, u);
}

// ---- diagnostics: extreme eigenvalues of a symmetric tridiagonal matrix by
// Sturm-sequence bisection (number of eigenvalues below x from the LDL^T pivots)
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int c = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        const double e2 = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i > 0 ? e2 / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++c;
    }
    return c;
}

double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, int k) {
    // k-th smallest eigenvalue (k = 1..n) within the Gershgorin interval
    double lo = d[0], hi = d[0];
    for (size_t i = 0; i < d.size(); ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) >= k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Restarted right-preconditioned flexible GMRES (Sec. "Outer Krylov Solver and
// Convergence Statement"): modified Gram-Schmidt Arnoldi on FP32 vectors with
// FP64-accumulated inner products, Givens rotations on the host, a happy
// breakdown when the new Hessenberg entry drops below 1e-14, the update
// u += Z y accumulated in FP64, and every cycle started from (and every
// solve accepted by) the FP64 true residual.
int fgmres_solve(gmg_handle* h, const double* f, double* u, double tol, int maxit, double nf, gmg_info& inf) {
    cudaStream_t s = h->stream;
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.nnp;
    const int m = h->opt.restart;
    if (h->fg_m != m) {
        dfree(h, h->fg_V);
        dfree(h, h->fg_Z);
        dfree(h, h->fg_h);
        h->fg_V = h->fg_Z = nullptr;
        h->fg_h = nullptr;
        TRY(dalloc(h, &h->fg_V, (size_t)(m + 1) * n));
        TRY(dalloc(h, &h->fg_Z, (size_t)m * n));
        CU(cudaMemsetAsync(h->fg_V, 0, sizeof(float) * (size_t)(m + 1) * n, s));  // the pads stay 0
        CU(cudaMemsetAsync(h->fg_Z, 0, sizeof(float) * (size_t)m * n, s));
        TRY(dalloc(h, &h->fg_h, (size_t)m + 2));
        h->fg_m = m;
    }
    double* sch = h->sc_host;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hcol(m + 2), y(m);
    int k = 0;
    while (true) {
        double rel = 0.0;
        launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f, u, nullptr, h->r, l0.px, h->sc, h->partials,
                            h->gs64, s);
        launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), h->sc, SC_TRR, FIN_NONE, s);
        TRY(sync_scalars(h));
        const double beta = std::sqrt(sch[SC_TRR]);
        rel = beta / nf;
        inf.rel_residual = rel;
        inf.iterations = k;
        if (!std::isfinite(rel)) return GMG_NONFINITE;
        if (rel < tol) return GMG_OK;
        if (k >= maxit) return GMG_NOT_CONVERGED;
        if (k > 0) ++inf.replacements;  // restarts
        float* V0 = h->fg_V;
        CU(cudaMemcpyAsync(V0, h->r, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        launch_scale_by_inv_sqrt(V0, n, h->sc, SC_TRR, s);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        bool stop = false;
        while (j < m && k < maxit && !stop) {
            float* Vj = h->fg_V + (size_t)j * n;
            float* Zj = h->fg_Z + (size_t)j * n;
            float* W = h->fg_V + (size_t)(j + 1) * n;
            vcycle_level(h, 0, Vj, Zj, h->x2_0, -1, FIN_NONE);   // z_j = M v_j
            level_apply(h, 0, Zj, W);                             // w = K z_j
            for (int i = 0; i <= j; ++i) {                        // modified Gram-Schmidt
                const float* Vi = h->fg_V + (size_t)i * n;
                launch_dot_f32(W, Vi, n, h->partials, s);
                launch_finalize(h->partials, vec_grid_blocks(), h->fg_h, i, FIN_NONE, s);
                launch_axpy_dev(W, Vi, n, h->fg_h + i, -1.f, s);
            }
            launch_dot_f32(W, W, n, h->partials, s);
            launch_finalize(h->partials, vec_grid_blocks(), h->fg_h, j + 1, FIN_NONE, s);
            launch_scale_by_inv_sqrt(W, n, h->fg_h, j + 1, s);    // v_{j+1} = w / ||w||
            launch_publish(h->fg_h, j + 2, h->hcol_map, nullptr, nullptr, nullptr, s);
            CU(cudaGetLastError());
            CU(cudaStreamSynchronize(s));
            std::copy(h->hcol_host, h->hcol_host + j + 2, hcol.begin());
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
            double hn = std::sqrt(std::max(hcol[j + 1], 0.0));
            if (!std::isfinite(hn)) return GMG_NONFINITE;
            for (int i = 0; i < j; ++i) {  // previous rotations on column j
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double hjj = H[(size_t)j * m + j];
            const double den = std::hypot(hjj, hn);
            const bool happy = hn < 1e-14;
            cs[j] = hjj / den;
            sn[j] = hn / den;
            H[(size_t)j * m + j] = den;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++j;
            ++k;
            inf.rel_residual_recursive = std::fabs(g[j]) / nf;
            stop = happy || std::fabs(g[j]) / nf < tol;
        }
        for (int i = j - 1; i >= 0; --i) {  // H y = g
            double acc = g[i];
            for (int q = i + 1; q < j; ++q) acc -= H[(size_t)i * m + q] * y[q];
            y[i] = acc / H[(size_t)i * m + i];
        }
        for (int i = 0; i < j; ++i) launch_axpy_u64(u, h->fg_Z + (size_t)i * n, l0, y[i], s);
    }
}

// Reports a timed-out wait of a TMA-staged / tensor-core kernel or of the fused
// lower V-cycle.  Both error words are sticky on the device; once reported they
// are cleared, together with the grid barrier's arrival counter (blocks that
// gave up may have left it non-zero), so the handle's next call starts clean.
int check_fused(gmg_handle* h) {
    TRY(sync_scalars(h));
#ifdef GMG_CHECKED
    if (const unsigned site = bounds_site_collect(); site != 0)
        return fail(GMG_ERR_CUDA, "bounds-checked build: out-of-range index at check site " + std::to_string(site));
#endif
    const int err[2] = {h->err_host[0], h->err_host[1]};
    if (!err[0] && !err[1]) return GMG_OK;
    CU(cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream));
    if (h->use_fused) {
        CU(cudaMemsetAsync(h->cf.bar_count, 0, sizeof(unsigned), h->stream));
        CU(cudaMemsetAsync(h->cf.err, 0, sizeof(int), h->stream));
    }
    CU(cudaStreamSynchronize(h->stream));
    h->err_host[0] = h->err_host[1] = 0;
    if (err[0]) return fail(GMG_TIMEOUT, "a TMA-staged or tensor-core kernel gave up waiting for its shared-memory tiles");
    return fail(GMG_TIMEOUT, "the fused coarse-level V-cycle gave up waiting at a grid barrier after " +
                                 std::to_string(h->cf.spin_limit) + " polls");
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

void gmg_default_options(gmg_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->levels = 4;
    o->smoother = GMG_SMOOTHER_CHEBYSHEV;
    o->degree = 2;
    o->coarse_smoother = GMG_SMOOTHER_JACOBI;
    o->coarse_degree = 2;
    o->omega = 0.5;
    o->coarse_omega = 0.5;
    o->cheb_alpha = 1.0 / 30.0;
    o->lambda_safety = 1.1;
    o->power_iters_fine = 20;
    o->power_iters_coarse = 10;
    o->chol_cutoff = 5000;
    o->fused_coarse_nodes = 0;
    o->bsr_tma_nodes = 0;
    o->device_loop = 1;
    o->ir_factor = 0.0;
    o->fine_smoother = GMG_FINE_FP32;
    o->cycle_index = 1;
    o->outer = GMG_OUTER_PCG;
    o->restart = 32;
    o->bsr_kernel = -1;
    o->stream = nullptr;
    o->spin_limit = 1LL << 24;
    o->coarse_pcg_steps = 80;
    o->lower_cluster = 0;
}

const char* gmg_status_str(int st) {
    switch (st) {
        case GMG_OK: return "ok";
        case GMG_NOT_CONVERGED: return "not converged (iteration cap)";
        case GMG_NONFINITE: return "non-finite residual or step";
        case GMG_ERR_ARG: return "invalid argument";
        case GMG_ERR_CUDA: return "CUDA error";
        case GMG_ERR_CHOLESKY: return "coarsest Cholesky failed";
        case GMG_ERR_SMOOTHER: return "unstable Jacobi damping";
        case GMG_ERR_NOMEM: return "device out of memory";
        case GMG_ERR_NO_DEVICE: return "no usable CUDA device";
        case GMG_TIMEOUT: return "a bounded device-side wait gave up";
        default: return "unknown status";
    }
}

const char* gmg_last_error(void) { return g_err.c_str(); }

unsigned long long gmg_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

void gmg_destroy(gmg_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    loop_free(h);
    multi_free(h);
    if (h->batch_exec) cudaGraphExecDestroy(h->batch_exec);
    if (h->batch_graph) cudaGraphDestroy(h->batch_graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
}

int gmg_setup(gmg_handle** out, const gmg_grid* g, const float* rho_dev, double p, double E0, double Emin,
              double nu, const gmg_bc* bc, const gmg_options* opt) {
    if (!out) return fail(GMG_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    if (!g || !rho_dev || !bc) return fail(GMG_ERR_ARG, "null grid, density or boundary-condition pointer");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(GMG_ERR_ARG, "element counts must be >= 1");
    if (nodes_of(g->nx, g->ny, g->nz) > (1LL << 31) / 3) return fail(GMG_ERR_ARG, "grid too large");
    if (bc->kind != GMG_BC_CLAMP_XMIN && bc->kind != GMG_BC_MASK) return fail(GMG_ERR_ARG, "unknown bc kind");
    if (bc->kind == GMG_BC_MASK && !bc->fixed) return fail(GMG_ERR_ARG, "bc kind MASK needs a fixed-flag array");
    if (!(nu > -1.0 && nu < 0.5)) return fail(GMG_ERR_ARG, "Poisson ratio outside (-1, 0.5)");
    if (!(E0 > 0.0) || !(Emin >= 0.0) || !std::isfinite(p)) return fail(GMG_ERR_ARG, "bad SIMP parameters");
    gmg_options o;
    if (opt) o = *opt; else gmg_default_options(&o);
    auto bad_kind = [](int k) { return k != GMG_SMOOTHER_JACOBI && k != GMG_SMOOTHER_CHEBYSHEV; };
    if (bad_kind(o.smoother) || (o.coarse_smoother >= 0 && bad_kind(o.coarse_smoother)))
        return fail(GMG_ERR_ARG, "unknown smoother kind");
    if (o.degree < 1 || o.degree > kMaxDegree || o.coarse_degree > kMaxDegree)
        return fail(GMG_ERR_ARG, "smoother degree outside [1, 16]");
    if (o.levels < 0 || o.levels > kMaxLevels) return fail(GMG_ERR_ARG, "levels outside [0, 16]");
    if (!(o.omega > 0.0) || !(o.cheb_alpha > 0.0 && o.cheb_alpha < 1.0) || !(o.lambda_safety > 0.0))
        return fail(GMG_ERR_ARG, "bad smoother parameters");
    if (!(o.ir_factor >= 0.0 && o.ir_factor < 1.0)) return fail(GMG_ERR_ARG, "ir_factor must be in [0, 1)");
    if (o.fine_smoother != GMG_FINE_FP32 && o.fine_smoother != GMG_FINE_BF16 && o.fine_smoother != GMG_FINE_BF16X3)
        return fail(GMG_ERR_ARG, "unknown fine_smoother");
    if (o.cycle_index < 1 || o.cycle_index > 2) return fail(GMG_ERR_ARG, "cycle_index must be 1 (V) or 2 (W)");
    if (o.bsr_kernel < -1 || o.bsr_kernel >= kBsrKinds) return fail(GMG_ERR_ARG, "bsr_kernel outside [-1, 5]");
    if (o.outer != GMG_OUTER_PCG && o.outer != GMG_OUTER_FGMRES) return fail(GMG_ERR_ARG, "unknown outer solver");
    if (o.restart < 1 || o.restart > kMaxRestart) return fail(GMG_ERR_ARG, "restart must be in [1, 256]");
    if (o.power_iters_fine < 1 || o.power_iters_coarse < 1 || o.chol_cutoff < 1)
        return fail(GMG_ERR_ARG, "bad iteration counts or cutoff");
    if (o.spin_limit < 0) return fail(GMG_ERR_ARG, "spin_limit must be >= 0");
    if (o.coarse_pcg_steps < 1 || o.coarse_pcg_steps > 100000)
        return fail(GMG_ERR_ARG, "coarse_pcg_steps must be in [1, 100000]");
    if (o.lower_cluster != 0 && o.lower_cluster != 1) return fail(GMG_ERR_ARG, "lower_cluster must be 0 or 1");

    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(GMG_ERR_NO_DEVICE, "no CUDA device");
    }
    if (prop.major != 10 || prop.minor != 3)
        return fail(GMG_ERR_NO_DEVICE, "this library is built for sm_103a (compute capability 10.3) only");

    gmg_handle* h = new gmg_handle();
    h->opt = o;
    h->device = dev;
    h->stream = static_cast<cudaStream_t>(o.stream);
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = build(h, g, rho_dev, p, E0, Emin, nu, bc);
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != GMG_OK) {
        std::string keep = g_err;
        gmg_destroy(h);
        g_err = keep;
        return rc;
    }
    *out = h;
    return GMG_OK;
}

// The per-step entry points take level-0 vectors in the dense numbering of the
// ABI; they pack them into the handle's own (padded) level-0 vectors and unpack
// the results.  They run between solves, so those vectors are free.
int gmg_apply(gmg_handle* h, const float* u, float* y) {
    if (!h || !u || !y) return fail(GMG_ERR_ARG, "null argument");
    TRY(clear_pads(h));
    const Level& l0 = h->lev[0];
    launch_pack0(u, l0, h->p, h->stream);
    level_apply(h, 0, h->p, h->q);
    launch_unpack0(h->q, l0, y, h->stream);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_solve(gmg_handle* h, const double* f, double* u, double tol, int maxit, gmg_info* info) {
    if (!h || !f || !u) return fail(GMG_ERR_ARG, "null argument");
    if (!(tol > 0.0) || maxit < 0) return fail(GMG_ERR_ARG, "tol must be > 0 and maxit >= 0");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = h->stream;
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.nn;
    double* sch = h->sc_host;
    gmg_info inf{};
    TRY(clear_pads(h));
    TRY(reset_w(h));
    auto finish = [&](int st) -> int {
        flush_w(h, u);  // the steps since the last FP64 residual
        if (st == GMG_NONFINITE) h->pads_dirty = true;
        const int fe = check_fused(h);
        if (fe != GMG_OK) { h->pads_dirty = true; return fe; }
        inf.status = st;
        inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        inf.setup_ms = h->setup_ms;
        if (info) *info = inf;
        return st;
    };
    auto true_residual = [&](double& rel) -> int {
        flush_w(h, u);
        launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f, u, nullptr, h->r, l0.px, h->sc, h->partials,
                            h->gs64, s);
        launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), h->sc, SC_TRR, FIN_NONE, s);
        TRY(sync_scalars(h));
        rel = std::sqrt(sch[SC_TRR]) / std::sqrt(sch[SC_FF]);
        return GMG_OK;
    };

    // fixed DOFs of u -> 0, nonzero count of u, ||f_free||^2
    launch_mask_u64(u, l0.mask, l0.nn, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_UNZ, FIN_NONE, s);
    launch_dot_f64_masked(f, f, l0.mask, l0.nn, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_FF, FIN_NONE, s);
    TRY(sync_scalars(h));
    if (!(sch[SC_FF] > 0.0)) {
        if (!std::isfinite(sch[SC_FF])) { inf.rel_residual = NAN; return finish(GMG_NONFINITE); }
        CU(cudaMemsetAsync(u, 0, sizeof(double) * n, s));
        CU(cudaStreamSynchronize(s));
        return finish(GMG_OK);
    }
    double rel = 0.0;
    if (sch[SC_UNZ] == 0.0) {
        // zero iterate (a cold start): K u = 0 exactly, so r = f and ||r|| / ||f|| = 1
        launch_cast_masked(f, l0, h->r, s);
        rel = 1.0;
    } else {
        TRY(true_residual(rel));  // r (FP32) = f - K u, FP64 norm
    }
    // every later operator application sees u != 0 through the PCG updates
    inf.rel_residual = rel;
    inf.rel_residual_recursive = rel;
    if (!std::isfinite(rel)) return finish(GMG_NONFINITE);
    if (rel < tol) return finish(GMG_OK);
    sch[SC_UNZ] = 1.0;
    launch_set_scalars(h->sc + SC_UNZ, 1, 1.0, 0.0, 0.0, 0.0, s);

    const double nf = std::sqrt(sch[SC_FF]);
    // Stopping target of an inner PCG phase.  Plain solve: tol.  Outer FP64
    // iterative refinement (ir_factor in (0, 1)): each phase, started from the
    // FP64 residual of the current u, stops once its recursive residual is
    // ir_factor times smaller (but not below tol); the FP64 residual
    // replacement and restart that follow are the outer refinement step.
    if (h->opt.outer == GMG_OUTER_FGMRES) {
        const int st = fgmres_solve(h, f, u, tol, maxit, nf, inf);
        if (st < 0) return st;
        CU(cudaGetLastError());
        return finish(st);
    }
    const double irf = h->opt.ir_factor;
    auto inner_target = [&](double rel_start) { return irf > 0.0 ? std::max(tol, irf * rel_start) : tol; };
    double target = inner_target(rel);
    if (maxit > 0 && h->opt.device_loop && !h->loop_unavailable && h->loop_u != u) {
        if (loop_select(h, u) != GMG_OK) h->loop_unavailable = true;  // e.g. no graph support: host loop
    }
    if (maxit > 0 && h->opt.device_loop && h->loop_exec && h->loop_u == u) {
        // device-resident loop: one graph launch per convergence candidate
        sch[SC_IT] = 0.0;
        sch[SC_TOL] = target;
        sch[SC_MAXIT] = (double)maxit;
        sch[SC_NF] = nf;
        launch_set_scalars(h->sc + SC_IT, 4, sch[SC_IT], sch[SC_TOL], sch[SC_MAXIT], sch[SC_NF], s);
        int k = 0;
        while (true) {
            if (sch[SC_TOL] != target) {
                sch[SC_TOL] = target;
                launch_set_scalars(h->sc + SC_TOL, 1, target, 0.0, 0.0, 0.0, s);
            }
            CU(cudaGraphLaunch(h->loop_exec, s));
            h->w_dirty = true;
            TRY(sync_scalars(h));
            const int k_new = (int)sch[SC_IT];
            note_launch(h->loop_prefix_kernels + h->loop_body_kernels * (unsigned long long)(k_new - k - 1));
            k = k_new;
            const double relr = std::sqrt(sch[SC_RR]) / nf;
            inf.iterations = k;
            inf.rel_residual_recursive = relr;
            if (!std::isfinite(relr) || !std::isfinite(sch[SC_ALPHA])) {
                inf.rel_residual = relr;
                return finish(GMG_NONFINITE);
            }
            if (!(relr < target)) break;  // the cap
            TRY(true_residual(rel));
            inf.rel_residual = rel;
            if (rel < tol) return finish(GMG_OK);
            if (!std::isfinite(rel)) return finish(GMG_NONFINITE);
            ++inf.replacements;  // residual replacement (r now holds f - K u); restart the direction
            target = inner_target(rel);
            if (k >= maxit) break;
        }
        TRY(true_residual(rel));
        inf.rel_residual = rel;
        CU(cudaGetLastError());
        return finish(GMG_NOT_CONVERGED);
    }

    // host-driven loop (same kernels, one scalar read-back per iteration)
    pcg_restart(h);
    int k = 0;
    while (k < maxit) {
        pcg_step(h);
        ++k;
        TRY(sync_scalars(h));
        const double relr = std::sqrt(sch[SC_RR]) / nf;
        inf.iterations = k;
        inf.rel_residual_recursive = relr;
        if (!std::isfinite(relr) || !std::isfinite(sch[SC_ALPHA])) {
            inf.rel_residual = relr;
            return finish(GMG_NONFINITE);
        }
        if (relr < target) {
            TRY(true_residual(rel));
            inf.rel_residual = rel;
            if (rel < tol) return finish(GMG_OK);
            if (!std::isfinite(rel)) return finish(GMG_NONFINITE);
            ++inf.replacements;  // residual replacement (r now holds f - K u); restart the direction
            target = inner_target(rel);
            pcg_restart(h);
            continue;
        }
        pcg_direction(h);
    }
    TRY(true_residual(rel));
    inf.rel_residual = rel;
    CU(cudaGetLastError());
    return finish(GMG_NOT_CONVERGED);
}

// Drops every graph the handle captured (solve loops and the batch graph):
// they would keep the launch shapes they were captured with.
static void drop_captured(gmg_handle* h) {
    loop_free(h);
    if (h->batch_exec) cudaGraphExecDestroy(h->batch_exec);
    if (h->batch_graph) cudaGraphDestroy(h->batch_graph);
    h->batch_exec = nullptr;
    h->batch_graph = nullptr;
    h->batch_key.clear();
}

int gmg_set_fine_plan(gmg_handle* h, int tile, int zchunk) {
    if (!h) return fail(GMG_ERR_ARG, "null handle");
    const Level& l0 = h->lev[0];
    if (tile >= 0) {
        if (tile >= kFineTiles || zchunk < 1) return fail(GMG_ERR_ARG, "unknown fine tile or zchunk < 1");
        if (fine_plan_blocks(l0.nx, l0.ny, l0.nz, tile, zchunk) > h->max_partials)
            return fail(GMG_ERR_ARG, "fine plan needs more blocks than the handle's partial sums hold");
    }
    CU(cudaStreamSynchronize(h->stream));
    fine_set_plan(l0.nx, l0.ny, l0.nz, tile, zchunk);
    drop_captured(h);
    return GMG_OK;
}

int gmg_autotune(gmg_handle* h, int reps, gmg_tuning* out) {
    if (!h || reps < 0) return fail(GMG_ERR_ARG, "null handle or reps < 0");
    if (h->is_clone) return fail(GMG_ERR_ARG, "tune the source handle, not a clone");
    cudaStream_t s = h->stream;
    CU(cudaStreamSynchronize(s));
    if (reps == 0) {  // back to the cost model and the size rule
        fine_set_plan(h->lev[0].nx, h->lev[0].ny, h->lev[0].nz, -1, 0);
        for (int li = 1; li < h->L; ++li) h->lev[li].bsr_kind = default_bsr_kind(h, li);
        loop_free(h);
        if (out) {
            *out = gmg_tuning{};
            fine_model_plan(h->lev[0].nx, h->lev[0].ny, h->lev[0].nz, &out->fine_tile, &out->fine_zchunk);
            out->model_tile = out->fine_tile;
            out->model_zchunk = out->fine_zchunk;
            for (int li = 0; li < 16; ++li) out->bsr_kind[li] = li >= 1 && li < h->L ? default_bsr_kind(h, li) : -1;
        }
        return GMG_OK;
    }
    gmg_tuning t{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(GMG_ERR_CUDA, "cudaEventCreate failed");
    }
    // median of three timed batches of `reps` launches, after one warm-up
    auto timed = [&](auto&& launch, double& us) -> int {
        launch();
        double m[3];
        for (int r = 0; r < 3; ++r) {
            CU(cudaEventRecord(e0, s));
            for (int i = 0; i < reps; ++i) launch();
            CU(cudaEventRecord(e1, s));
            CU(cudaEventSynchronize(e1));
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, e0, e1));
            m[r] = 1000.0 * ms / reps;
        }
        std::sort(m, m + 3);
        us = m[1];
        return GMG_OK;
    };
    int rc = GMG_OK;
    {
        // fine level: fused smoothing step (the dominant launch of a V-cycle)
        const Level& l0 = h->lev[0];
        FineArgs a = fine_args(h);
        a.xin = h->z;
        a.b = h->r;
        a.out = h->q;
        a.dold = nullptr;
        a.dnew = nullptr;
        a.step = 0;
        auto fine = [&] { launch_fine(FM_SMOOTH, 0, 0, a, h->gs, s); };
        int tiles[64], zcs[64];
        const int nc = fine_candidates(l0.nx, l0.ny, l0.nz, h->max_partials, tiles, zcs, 64);
        fine_model_plan(l0.nx, l0.ny, l0.nz, &t.model_tile, &t.model_zchunk);
        fine_set_plan(l0.nx, l0.ny, l0.nz, t.model_tile, t.model_zchunk);
        if (rc == GMG_OK) rc = timed(fine, t.model_us);
        t.fine_tile = t.model_tile;
        t.fine_zchunk = t.model_zchunk;
        t.fine_us = t.model_us;
        for (int c = 0; c < nc && rc == GMG_OK; ++c) {
            fine_set_plan(l0.nx, l0.ny, l0.nz, tiles[c], zcs[c]);
            double us = 0.0;
            rc = timed(fine, us);
            if (rc == GMG_OK && us < t.fine_us) {
                t.fine_us = us;
                t.fine_tile = tiles[c];
                t.fine_zchunk = zcs[c];
            }
        }
        t.fine_candidates = nc;
        fine_set_plan(l0.nx, l0.ny, l0.nz, t.fine_tile, t.fine_zchunk);
    }
    for (int li = 0; li < 16; ++li) t.bsr_kind[li] = -1;
    const int fused_start = h->use_fused ? h->cf.start : h->L;
    for (int li = 1; li < h->L - 1 && li < 16 && rc == GMG_OK; ++li) {
        Level& l = h->lev[li];
        if (l.tma || li >= fused_start) continue;
        // the assembled kernels, and on level 1 the matrix-free form where exact
        const int nkinds = l.eh ? kBsrMatrixFree + 1 : kBsrKinds;
        double us[kBsrMatrixFree + 1] = {};
        for (int kind = 0; kind < nkinds && rc == GMG_OK; ++kind) {
            l.bsr_kind = kind;
            BsrArgs a = bsr_args(h, li);
            a.xin = l.x;
            a.b = l.b;
            a.out = l.x2;
            a.dold = nullptr;
            a.dnew = nullptr;
            a.step = 0;
            rc = timed([&] { launch_bsr(FM_SMOOTH, 0, a, s); }, us[kind]);
        }
        int best = 0;
        for (int kind = 1; kind < nkinds; ++kind)
            if (us[kind] < us[best]) best = kind;
        int second = best == 0 ? 1 : 0;
        for (int kind = 0; kind < nkinds; ++kind)
            if (kind != best && us[kind] < us[second]) second = kind;
        l.bsr_kind = best;
        t.bsr_kind[li] = best;
        t.bsr_us[li] = us[best];
        t.bsr_alt_us[li] = us[second];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GMG_OK) return rc;
    // graphs captured with the former shapes are dropped (they stay correct,
    // but would keep the old shapes)
    drop_captured(h);
    CU(cudaGetLastError());
    if (out) *out = t;
    return GMG_OK;
}

int gmg_kappa_eff(gmg_handle* h, const double* b, int steps, double out[3]) {
    if (!h || !b || !out) return fail(GMG_ERR_ARG, "null argument");
    if (steps < 1 || steps > 1000) return fail(GMG_ERR_ARG, "steps must be in [1, 1000]");
    if (h->L == 1) return fail(GMG_ERR_ARG, "single-level hierarchy");
    TRY(clear_pads(h));
    TRY(reset_w(h));
    h->pads_dirty = true;  // the probe may stop at a breakdown with non-finite scalars
    cudaStream_t s = h->stream;
    Level& l0 = h->lev[0];
    const long long n = 3 * l0.nn;
    if (!h->kap_u) TRY(dalloc(h, &h->kap_u, (size_t)n));
    CU(cudaMemsetAsync(h->kap_u, 0, sizeof(double) * n, s));
    launch_cast_masked(b, l0, h->r, s);
    pcg_restart(h);
    std::vector<double> al, be;
    for (int k = 0; k < steps; ++k) {
        pcg_step(h);
        pcg_direction(h);
        TRY(sync_scalars(h));
        const double a = h->sc_host[SC_ALPHA], bt = h->sc_host[SC_BETA];
        if (!(std::isfinite(a) && a > 0.0 && std::isfinite(bt) && bt >= 0.0)) break;
        al.push_back(a);
        be.push_back(bt);
        if (bt == 0.0) break;
    }
    TRY(reset_w(h));  // the probe's iterate is not kept
    if (al.empty()) return fail(GMG_NONFINITE, "the Lanczos probe broke down at its first step");
    // Lanczos matrix from the CG coefficients
    const size_t kk = al.size();
    std::vector<double> d(kk), e(kk > 1 ? kk - 1 : 1, 0.0);
    for (size_t j = 0; j < kk; ++j) d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    for (size_t j = 0; j + 1 < kk; ++j) e[j] = std::sqrt(be[j]) / al[j];
    out[0] = tridiag_eig(d, e, 1);
    out[1] = tridiag_eig(d, e, (int)kk);
    out[2] = out[1] / out[0];
    return GMG_OK;
}

int gmg_vcycle_symmetry(gmg_handle* h, const float* x, const float* y, double* defect) {
    if (!h || !x || !y || !defect) return fail(GMG_ERR_ARG, "null argument");
    if (h->L == 1) return fail(GMG_ERR_ARG, "single-level hierarchy");
    TRY(clear_pads(h));
    cudaStream_t s = h->stream;
    const Level& l0 = h->lev[0];
    const long long n = 3 * l0.nnp;
    launch_pack0(x, l0, h->r, s);
    launch_pack0(y, l0, h->q, s);
    vcycle_level(h, 0, h->q, h->z, h->x2_0, -1, FIN_NONE);   // M y
    vcycle_level(h, 0, h->r, h->p, h->x2_0, -1, FIN_NONE);   // M x
    launch_dot_f32(h->r, h->z, n, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_TMP, FIN_NONE, s);
    launch_dot_f32(h->q, h->p, n, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_TMP + 1, FIN_NONE, s);
    TRY(sync_scalars(h));
    const double a = h->sc_host[SC_TMP], b = h->sc_host[SC_TMP + 1];
    *defect = std::fabs(a - b) / std::max(std::fabs(a), std::fabs(b));
    return GMG_OK;
}

int gmg_clone(const gmg_handle* src, gmg_handle** out) {
    if (!src || !out) return fail(GMG_ERR_ARG, "null argument");
    *out = nullptr;
    gmg_handle* h = new gmg_handle(*src);
    // nothing of src is owned by the clone
    h->allocs.clear();
    h->pinned = nullptr;
    h->sc_host = nullptr;
    h->sc_map = nullptr;
    h->err_host = nullptr;
    h->err_map = nullptr;
    h->hcol_host = nullptr;
    h->hcol_map = nullptr;
    h->cap_stream = nullptr;
    h->loop_graph = nullptr;
    h->loop_exec = nullptr;
    h->loop_u = nullptr;
    h->loop_cache.clear();  // the source's graphs stay the source's
    h->loop_unavailable = false;
    h->fg_V = h->fg_Z = nullptr;
    h->fg_h = nullptr;
    h->fg_m = 0;
    h->kap_u = nullptr;
    h->batch_graph = nullptr;
    h->batch_exec = nullptr;
    h->batch_key.clear();
    h->batch_counts.clear();
    h->mw = nullptr;  // the multi-load workspace stays the source's
    h->is_clone = true;
    auto bad = [&](int rc) {
        std::string keep = g_err;
        gmg_destroy(h);
        g_err = keep;
        return rc;
    };
    cudaStream_t s = h->stream;
    const long long n0 = 3 * h->lev[0].nnp;
    int rc = GMG_OK;
    for (int li = 1; li < h->L && rc == GMG_OK; ++li) {
        Level& l = h->lev[li];
        rc = dalloc(h, &l.x, 3 * l.nn);
        if (rc == GMG_OK) rc = dalloc(h, &l.x2, 3 * l.nn);
        if (rc == GMG_OK) rc = dalloc(h, &l.b, 3 * l.nn);
        if (rc == GMG_OK) rc = dalloc(h, &l.t, 3 * l.nn);
        if (rc == GMG_OK) rc = dalloc(h, &l.d, 3 * l.nn);
        // the matrix-free level 1's corner forces are workspace of each handle
        if (rc == GMG_OK && l.cf) rc = dalloc(h, &l.cf, 32 * (size_t)l.nx * l.ny * l.nz);
    }
    float** fv[] = {&h->r, &h->z, &h->p, &h->q, &h->x2_0, &h->t0, &h->d0, &h->wh, &h->wl};
    for (float** v : fv) {
        if (rc == GMG_OK) rc = dalloc(h, v, n0);
        if (rc == GMG_OK && cudaMemsetAsync(*v, 0, sizeof(float) * n0, s) != cudaSuccess) rc = GMG_ERR_CUDA;
    }
    h->pads_dirty = false;
    if (rc == GMG_OK) rc = dalloc(h, &h->sc, SC_COUNT);
    if (rc == GMG_OK) rc = dalloc(h, &h->kerr, 1);
    if (rc == GMG_OK) rc = dalloc(h, &h->partials, h->max_partials);
    if (rc != GMG_OK) return bad(rc);
    if (cudaMemsetAsync(h->sc, 0, sizeof(double) * SC_COUNT, s) != cudaSuccess ||
        cudaMemsetAsync(h->kerr, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return bad(fail(GMG_ERR_CUDA, "clone workspace"));
    }
    if (int rc2 = alloc_mirror(h); rc2 != GMG_OK) return bad(rc2);
    if (h->use_fused) {
        CoarseFused& cf = h->cf;
        for (int li = 1; li < h->L; ++li) {
            const Level& l = h->lev[li];
            CoarseLevel& c = cf.lev[li];
            c.x = l.x; c.x2 = l.x2; c.b = l.b; c.t = l.t; c.d = l.d;
        }
        unsigned* words = nullptr;
        if (dalloc(h, &words, 4) != GMG_OK || cudaMemsetAsync(words, 0, 4 * sizeof(unsigned), s) != cudaSuccess)
            return bad(fail(GMG_ERR_CUDA, "clone barrier words"));
        cf.bar_count = words;
        cf.bar_gen = words + 1;
        cf.err = reinterpret_cast<int*>(words + 2);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return bad(fail(GMG_ERR_CUDA, "clone synchronisation"));
    }
    *out = h;
    return GMG_OK;
}

int gmg_solve_batch(gmg_handle* const* hs, int count, const double* const* f, double* const* u, double tol,
                    int maxit, gmg_info* infos) {
    if (!hs || !f || !u || !infos || count < 1) return fail(GMG_ERR_ARG, "null argument or empty batch");
    if (!(tol > 0.0) || maxit < 0) return fail(GMG_ERR_ARG, "tol must be > 0 and maxit >= 0");
    for (int i = 0; i < count; ++i)
        if (!hs[i] || !f[i] || !u[i]) return fail(GMG_ERR_ARG, "null handle or vector in the batch");
    bool plain = true;  // the batch graph covers the plain device-resident PCG
    for (int i = 0; i < count; ++i) {
        const gmg_options& o = hs[i]->opt;
        plain = plain && o.outer == GMG_OUTER_PCG && o.device_loop && o.ir_factor == 0.0 && maxit > 0;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(GMG_ERR_ARG, "a handle appears twice in the batch");
    }
    if (!plain) {  // one solve after the other
        int worst = GMG_OK;
        for (int i = 0; i < count; ++i) {
            const int rc = gmg_solve(hs[i], f[i], u[i], tol, maxit, &infos[i]);
            if (rc < 0) return rc;
            if (rc != GMG_OK) worst = rc;
        }
        return worst;
    }
    // ---- items that share a hierarchy (a handle and its clones) are solved
    // together as multi-load chunks of up to 16 loads, owned by the chunk's
    // first handle; the other items keep their own single-load loops
    struct Chunk {
        gmg_handle* owner;
        std::vector<int> items;
    };
    std::vector<Chunk> chunks;
    std::vector<int> chunk_of(count, -1), slot_of(count, -1);
    {
        std::vector<bool> seen(count, false);
        for (int i = 0; i < count; ++i) {
            if (seen[i]) continue;
            std::vector<int> grp;
            for (int j = i; j < count; ++j)
                if (!seen[j] && hs[j]->E32 == hs[i]->E32 && hs[j]->L == hs[i]->L &&
                    hs[j]->lev[0].maskp == hs[i]->lev[0].maskp) {
                    grp.push_back(j);
                    seen[j] = true;
                }
            bool ok = grp.size() >= 2;
            for (int j : grp) ok = ok && multi_ok(hs[j], nullptr);
            if (!ok) continue;
            for (size_t a = 0; a < grp.size(); a += kLoads) {
                Chunk c{hs[grp[a]], {}};
                for (size_t b = a; b < std::min(grp.size(), a + kLoads); ++b) {
                    chunk_of[grp[b]] = (int)chunks.size();
                    slot_of[grp[b]] = (int)c.items.size();
                    c.items.push_back(grp[b]);
                }
                if (c.items.size() < 2) {  // a lone remainder stays a single-load item
                    chunk_of[c.items[0]] = slot_of[c.items[0]] = -1;
                    continue;
                }
                chunks.push_back(c);
            }
        }
    }
    for (Chunk& c : chunks)
        if (int rc = multi_workspace(c.owner); rc != GMG_OK) return rc;
    gmg_handle* h0 = hs[0];
    cudaStream_t s = h0->stream;
    std::vector<cudaStream_t> saved(count);
    for (int i = 0; i < count; ++i) {
        saved[i] = hs[i]->stream;
        hs[i]->stream = s;
    }
    auto restore = [&]() {
        for (int i = 0; i < count; ++i) hs[i]->stream = saved[i];
    };
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&]() { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); };
    // each item's FP64 scalars (host mirror): its own block, or its load slot in the chunk owner's
    auto sch = [&](int i) -> double* {
        return chunk_of[i] < 0 ? hs[i]->sc_host : chunks[chunk_of[i]].owner->mw->sc_host + slot_of[i] * SC_COUNT;
    };
    auto sync_all = [&]() -> int {
        PublishBatch pb{};
        pb.n = SC_COUNT;
        for (int i = 0; i < count; ++i) {
            if (chunk_of[i] >= 0) continue;
            const int k = pb.count++;
            pb.sc[k] = hs[i]->sc;
            pb.out[k] = hs[i]->sc_map;
            pb.e0[k] = hs[i]->kerr;
            pb.e1[k] = hs[i]->use_fused ? hs[i]->cf.err : nullptr;
            pb.eout[k] = hs[i]->err_map;
            if (pb.count == kPublishItems) {
                launch_publish_batch(pb, s);
                pb.count = 0;
            }
        }
        launch_publish_batch(pb, s);
        for (Chunk& c : chunks) multi_publish(c.owner);
        CU(cudaGetLastError());
        CU(cudaStreamSynchronize(s));
        for (Chunk& c : chunks)
            if (c.owner->mw->err_host[0] != 0) {
                cudaMemsetAsync(c.owner->kerr, 0, sizeof(int), s);
                cudaStreamSynchronize(s);
                return fail(GMG_TIMEOUT, "batch: a TMA wait of the multi-load level-0 operator gave up");
            }
        return GMG_OK;
    };
    std::vector<int> state(count, 0);  // 0: active, 1: done
    std::vector<double> nf(count, 0.0);
    std::vector<bool> cold(count, false);
    for (int i = 0; i < count; ++i) infos[i] = gmg_info{};
    for (int i = 0; i < count; ++i) {
        if (int rc = clear_pads(hs[i]); rc != GMG_OK) { restore(); return rc; }
        if (int rc = reset_w(hs[i]); rc != GMG_OK) { restore(); return rc; }
    }
    // the loads and iterates of a chunk, in slot order
    auto chunk_vecs = [&](const Chunk& c, const double** fc, double** uc) {
        for (size_t l = 0; l < c.items.size(); ++l) {
            fc[l] = f[c.items[l]];
            uc[l] = u[c.items[l]];
        }
    };
    // ---- norms, nonzero count of u, fixed DOFs of u to 0
    for (int i = 0; i < count; ++i) {
        if (chunk_of[i] >= 0) continue;
        gmg_handle* h = hs[i];
        const Level& l0 = h->lev[0];
        launch_mask_u64(u[i], l0.mask, l0.nn, h->partials, s);
        launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_UNZ, FIN_NONE, s);
        launch_dot_f64_masked(f[i], f[i], l0.mask, l0.nn, h->partials, s);
        launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_FF, FIN_NONE, s);
    }
    for (Chunk& c : chunks) {
        const double* fc[kLoads] = {};
        double* uc[kLoads] = {};
        chunk_vecs(c, fc, uc);
        multi_norms(c.owner, (int)c.items.size(), fc, uc);
    }
    if (int rc = sync_all(); rc != GMG_OK) { restore(); return rc; }
    bool need_rel = false;
    for (int i = 0; i < count; ++i) {
        const Level& l0 = hs[i]->lev[0];
        const double ff = sch(i)[SC_FF];
        if (!(ff > 0.0)) {
            state[i] = 1;
            if (!std::isfinite(ff)) { infos[i].status = GMG_NONFINITE; infos[i].rel_residual = NAN; }
            else cudaMemsetAsync(u[i], 0, sizeof(double) * 3 * l0.nn, s);
            continue;
        }
        nf[i] = std::sqrt(ff);
        cold[i] = sch(i)[SC_UNZ] == 0.0;
        if (cold[i]) infos[i].rel_residual = 1.0;
        else need_rel = true;
    }
    // initial residuals: single items into their own r, chunks into their load slots
    for (int i = 0; i < count; ++i) {
        if (chunk_of[i] >= 0 || state[i] != 0) continue;
        gmg_handle* h = hs[i];
        const Level& l0 = h->lev[0];
        if (cold[i]) {
            launch_cast_masked(f[i], l0, h->r, s);
        } else {
            launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f[i], u[i], nullptr, h->r, l0.px, h->sc,
                                h->partials, h->gs64, s);
            launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), h->sc, SC_TRR, FIN_NONE, s);
        }
    }
    for (Chunk& c : chunks) {
        const int nl = (int)c.items.size();
        const double* fc[kLoads] = {};
        bool cc[kLoads] = {};
        for (int l = 0; l < nl; ++l) {
            fc[l] = f[c.items[l]];
            cc[l] = state[c.items[l]] == 0 && cold[c.items[l]];
        }
        multi_cast(c.owner, nl, fc, cc);
        for (int l = 0; l < nl; ++l) {
            const int i = c.items[l];
            if (state[i] == 0 && !cold[i]) multi_true_residual(c.owner, l, f[i], u[i], true);
        }
    }
    if (need_rel) {
        if (int rc = sync_all(); rc != GMG_OK) { restore(); return rc; }
        for (int i = 0; i < count; ++i)
            if (state[i] == 0 && !cold[i]) infos[i].rel_residual = std::sqrt(sch(i)[SC_TRR]) / nf[i];
    }
    for (int i = 0; i < count; ++i)
        if (state[i] == 0) {
            const double rel = infos[i].rel_residual;
            infos[i].rel_residual_recursive = rel;
            if (!std::isfinite(rel)) { infos[i].status = GMG_NONFINITE; state[i] = 1; }
            else if (rel < tol) { infos[i].status = GMG_OK; state[i] = 1; }
        }
    // ---- one graph: independent branches, each the device-resident PCG loop of
    // a single item or of a chunk (the per-level lower V-cycle: concurrent
    // cooperative kernels could not all be co-resident)
    std::vector<bool> chunk_live(chunks.size(), false);
    for (size_t c = 0; c < chunks.size(); ++c)
        for (int i : chunks[c].items) chunk_live[c] = chunk_live[c] || state[i] == 0;
    std::vector<std::pair<const gmg_handle*, const double*>> key;
    for (int i = 0; i < count; ++i)
        if ((chunk_of[i] < 0 && state[i] == 0) || (chunk_of[i] >= 0 && chunk_live[chunk_of[i]]))
            key.emplace_back(hs[i], u[i]);
    if (!key.empty()) {
        if (key != h0->batch_key || !h0->batch_exec || h0->batch_gen != multi_generation()) {
            if (h0->batch_exec) cudaGraphExecDestroy(h0->batch_exec);
            if (h0->batch_graph) cudaGraphDestroy(h0->batch_graph);
            h0->batch_exec = nullptr;
            h0->batch_graph = nullptr;
            h0->batch_key.clear();
            h0->batch_counts.clear();
            if (int rc = ensure_cap_stream(h0); rc != GMG_OK) { restore(); return rc; }
            cudaGraph_t g = nullptr;
            bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
            for (int i = 0; i < count && ok; ++i) {
                if (chunk_of[i] >= 0 || state[i] != 0) continue;
                unsigned long long pre = 0, bod = 0;
                const bool fused = hs[i]->use_fused;
                hs[i]->use_fused = false;
                ok = capture_loop(hs[i], u[i], g, h0->cap_stream, pre, bod);
                hs[i]->use_fused = fused;
                h0->batch_counts.emplace_back(pre, bod);
            }
            for (size_t c = 0; c < chunks.size() && ok; ++c) {
                if (!chunk_live[c]) continue;
                double* uc[kLoads] = {};
                const int nl = (int)chunks[c].items.size();
                for (int l = 0; l < nl; ++l) uc[l] = u[chunks[c].items[l]];
                unsigned long long pre = 0, bod = 0;
                ok = multi_capture_loop(chunks[c].owner, uc, nl, g, h0->cap_stream, pre, bod);
                h0->batch_counts.emplace_back(pre, bod);
            }
            cudaGraphExec_t ex = nullptr;
            if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
            cudaGetLastError();
            if (!ok) {
                if (g) cudaGraphDestroy(g);
                h0->batch_counts.clear();
                restore();
                return fail(GMG_ERR_CUDA, "could not capture the batch graph");
            }
            h0->batch_graph = g;
            h0->batch_exec = ex;
            h0->batch_key = key;
            h0->batch_gen = multi_generation();
        }
        for (int i = 0; i < count; ++i) {
            if (chunk_of[i] >= 0 || state[i] != 0) continue;
            double* sh = hs[i]->sc_host;
            sh[SC_IT] = 0.0;
            sh[SC_TOL] = tol;
            sh[SC_MAXIT] = (double)maxit;
            sh[SC_NF] = nf[i];
            launch_set_scalars(hs[i]->sc + SC_IT, 4, sh[SC_IT], sh[SC_TOL], sh[SC_MAXIT], sh[SC_NF], s);
        }
        for (size_t c = 0; c < chunks.size(); ++c) {
            const int nl = (int)chunks[c].items.size();
            double nfc[kLoads] = {};
            bool act[kLoads] = {};
            for (int l = 0; l < nl; ++l) {
                nfc[l] = nf[chunks[c].items[l]];
                act[l] = state[chunks[c].items[l]] == 0;
            }
            multi_set_loop_scalars(chunks[c].owner, nl, tol, maxit, nfc, act);
        }
        CU(cudaGraphLaunch(h0->batch_exec, s));
        for (int i = 0; i < count; ++i)
            if (chunk_of[i] < 0 && state[i] == 0) hs[i]->w_dirty = true;  // their loops took PCG steps
        for (size_t c = 0; c < chunks.size(); ++c)
            if (chunk_live[c]) chunks[c].owner->mw->w_dirty = true;
        if (int rc = sync_all(); rc != GMG_OK) { restore(); return rc; }
        // launches: per single item and per chunk (its longest-running load)
        {
            size_t q = 0;
            for (int i = 0; i < count; ++i) {
                if (chunk_of[i] >= 0 || state[i] != 0) continue;
                const int k = (int)hs[i]->sc_host[SC_IT];
                note_launch(h0->batch_counts[q].first + h0->batch_counts[q].second * (unsigned long long)std::max(0, k - 1));
                ++q;
            }
            for (size_t c = 0; c < chunks.size(); ++c) {
                if (!chunk_live[c]) continue;
                int k = 0;
                for (int i : chunks[c].items) k = std::max(k, (int)sch(i)[SC_IT]);
                note_launch(h0->batch_counts[q].first + h0->batch_counts[q].second * (unsigned long long)std::max(0, k - 1));
                ++q;
            }
        }
        // FP64 true residual of every item that left its loop
        for (int i = 0; i < count; ++i) {
            if (state[i] != 0) continue;
            const double* sh = sch(i);
            infos[i].iterations = (int)sh[SC_IT];
            infos[i].rel_residual_recursive = std::sqrt(sh[SC_RR]) / nf[i];
            if (!std::isfinite(infos[i].rel_residual_recursive) || !std::isfinite(sh[SC_ALPHA])) {
                infos[i].status = GMG_NONFINITE;
                infos[i].rel_residual = infos[i].rel_residual_recursive;
                state[i] = 1;
                continue;
            }
            if (chunk_of[i] >= 0) {
                continue;  // one launch per chunk below
            } else {
                gmg_handle* h = hs[i];
                const Level& l0 = h->lev[0];
                flush_w(h, u[i]);
                launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f[i], u[i], nullptr, h->r, l0.px, h->sc,
                                    h->partials, h->gs64, s);
                launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), h->sc, SC_TRR, FIN_NONE, s);
            }
        }
        for (size_t c = 0; c < chunks.size(); ++c) {
            if (!chunk_live[c]) continue;
            const double* fc[kLoads] = {};
            double* uc[kLoads] = {};
            chunk_vecs(chunks[c], fc, uc);
            multi_true_residuals(chunks[c].owner, (int)chunks[c].items.size(), fc, uc);
        }
        if (int rc = sync_all(); rc != GMG_OK) { restore(); return rc; }
        for (int i = 0; i < count; ++i) {
            if (state[i] != 0) continue;
            gmg_handle* h = hs[i];
            const double rel = std::sqrt(sch(i)[SC_TRR]) / nf[i];
            infos[i].rel_residual = rel;
            state[i] = 1;
            if (!std::isfinite(rel)) infos[i].status = GMG_NONFINITE;
            else if (rel < tol) infos[i].status = GMG_OK;
            else if (!(infos[i].rel_residual_recursive < tol) || infos[i].iterations >= maxit)
                infos[i].status = GMG_NOT_CONVERGED;
            else {
                // residual replacement: continue this item alone from its current
                // iterate, with the same (per-level) lower V-cycle as the batch; the
                // loop graph captured for it is dropped again afterwards
                gmg_info more{};
                const bool fused = h->use_fused;
                h->use_fused = false;
                loop_free(h);
                const int rc = gmg_solve(h, f[i], u[i], tol, maxit - infos[i].iterations, &more);
                loop_free(h);
                h->use_fused = fused;
                if (rc < 0) { restore(); return rc; }
                infos[i].status = more.status;
                infos[i].iterations += more.iterations;
                infos[i].replacements += 1 + more.replacements;
                infos[i].rel_residual = more.rel_residual;
                infos[i].rel_residual_recursive = more.rel_residual_recursive;
            }
        }
    }
    int worst = GMG_OK;
    for (int i = 0; i < count; ++i)
        if (chunk_of[i] < 0) flush_w(hs[i], u[i]);  // items that stopped without an FP64 residual
    for (int i = 0; i < count; ++i)
        if (infos[i].status == GMG_NONFINITE) hs[i]->pads_dirty = true;
    for (int i = 0; i < count; ++i) {
        if (int fe = check_fused(hs[i]); fe != GMG_OK) { hs[i]->pads_dirty = true; restore(); return fe; }
        infos[i].solve_ms = elapsed();
        infos[i].setup_ms = hs[i]->setup_ms;
        if (infos[i].status != GMG_OK) worst = infos[i].status;
    }
    restore();
    CU(cudaGetLastError());
    return worst;
}

int gmg_bounds_checked(void) {
#ifdef GMG_CHECKED
    return 1;
#else
    return 0;
#endif
}

unsigned gmg_bounds_site(void) { return bounds_site_collect(); }

int gmg_set_spin_limit(gmg_handle* h, long long polls) {
    if (!h) return fail(GMG_ERR_ARG, "null handle");
    if (polls < 0) return fail(GMG_ERR_ARG, "spin_limit must be >= 0");
    CU(cudaStreamSynchronize(h->stream));
    h->opt.spin_limit = polls;
    h->cf.spin_limit = polls;
    // captured graphs hold the former bound in their kernel arguments
    drop_captured(h);
    return GMG_OK;
}

int gmg_num_levels(const gmg_handle* h) { return h ? h->L : 0; }

int gmg_level_dims(const gmg_handle* h, int level, int dims[3]) {
    TRY(check_level(h, level));
    if (!dims) return fail(GMG_ERR_ARG, "null dims");
    dims[0] = h->lev[level].nx; dims[1] = h->lev[level].ny; dims[2] = h->lev[level].nz;
    return GMG_OK;
}

int gmg_get_mask(gmg_handle* h, int level, uint8_t* out) {
    TRY(check_level(h, level));
    if (!out) return fail(GMG_ERR_ARG, "null output");
    CU(cudaMemcpyAsync(out, h->lev[level].mask, h->lev[level].nn, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return GMG_OK;
}

int gmg_get_bsr(gmg_handle* h, int level, double* out) {
    TRY(check_level(h, level));
    if (level == 0) return fail(GMG_ERR_ARG, "the fine level is matrix-free");
    if (!out) return fail(GMG_ERR_ARG, "null output");
    const Level& l = h->lev[level];
    CU(cudaMemcpyAsync(out, l.A64, sizeof(double) * kPlanes * l.nn, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return GMG_OK;
}

int gmg_get_lambda(gmg_handle* h, int level, double* out) {
    TRY(check_level(h, level));
    if (!out) return fail(GMG_ERR_ARG, "null output");
    CU(cudaMemcpyAsync(out, h->lam + level, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return GMG_OK;
}

int gmg_set_lambda(gmg_handle* h, int level, double lam) {
    TRY(check_level(h, level));
    if (!(lam > 0.0) || !std::isfinite(lam)) return fail(GMG_ERR_ARG, "lambda must be positive");
    h->sc_host[SC_TMP + 1] = lam;
    CU(cudaMemcpyAsync(h->lam + level, h->sc_host + SC_TMP + 1, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    refresh_coef(h, level);
    CU(cudaStreamSynchronize(h->stream));
    return GMG_OK;
}

int gmg_level_apply(gmg_handle* h, int level, const float* x, float* y) {
    TRY(check_level(h, level));
    if (!x || !y) return fail(GMG_ERR_ARG, "null vector");
    if (level == 0) return gmg_apply(h, x, y);
    level_apply(h, level, x, y);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_level_smooth(gmg_handle* h, int level, const float* b, float* x, int x_is_zero) {
    TRY(check_level(h, level));
    if (level == h->L - 1) return fail(GMG_ERR_ARG, "the coarsest level has no smoother");
    if (!b || !x) return fail(GMG_ERR_ARG, "null vector");
    Level& l = h->lev[level];
    int writes = 0;
    if (level == 0) {
        TRY(clear_pads(h));
        launch_pack0(b, l, h->r, h->stream);
        if (!x_is_zero) launch_pack0(x, l, h->z, h->stream);
        float* res = smooth_pass(h, 0, h->r, h->z, h->z, h->x2_0, x_is_zero != 0, writes);
        launch_unpack0(res, l, x, h->stream);
        CU(cudaGetLastError());
        return GMG_OK;
    }
    float* res = smooth_pass(h, level, b, x, x, l.x2, x_is_zero != 0, writes);
    if (res != x) CU(cudaMemcpyAsync(x, res, sizeof(float) * 3 * l.nn, cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_fine_pass(gmg_handle* h, int what) {
    if (!h) return fail(GMG_ERR_ARG, "null handle");
    if (what != 0 && what != 1) return fail(GMG_ERR_ARG, "what must be 0 (apply) or 1 (smoothing pass)");
    if (what == 1 && h->L == 1) return fail(GMG_ERR_ARG, "single-level hierarchy");
    TRY(clear_pads(h));
    if (what == 0) {
        level_apply(h, 0, h->p, h->q);
    } else {
        int writes = 0;
        smooth_pass(h, 0, h->r, h->z, h->z, h->x2_0, false, writes);
    }
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_restrict(gmg_handle* h, int level, const float* fine, float* coarse) {
    TRY(check_level(h, level));
    if (level + 1 >= h->L) return fail(GMG_ERR_ARG, "no coarser level");
    if (!fine || !coarse) return fail(GMG_ERR_ARG, "null vector");
    if (level == 0) {
        TRY(clear_pads(h));
        launch_pack0(fine, h->lev[0], h->t0, h->stream);
        fine = h->t0;
    }
    launch_restrict(h->lev[level], h->lev[level + 1], fine, coarse, h->stream);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_prolong_add(gmg_handle* h, int level, const float* coarse, float* fine) {
    TRY(check_level(h, level));
    if (level + 1 >= h->L) return fail(GMG_ERR_ARG, "no coarser level");
    if (!fine || !coarse) return fail(GMG_ERR_ARG, "null vector");
    if (level == 0) {
        TRY(clear_pads(h));
        const Level& l0 = h->lev[0];
        launch_pack0(fine, l0, h->z, h->stream);
        launch_prolong_add(l0, h->lev[1], coarse, h->z, h->stream);
        launch_unpack0(h->z, l0, fine, h->stream);
        CU(cudaGetLastError());
        return GMG_OK;
    }
    launch_prolong_add(h->lev[level], h->lev[level + 1], coarse, fine, h->stream);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_coarse_solve(gmg_handle* h, const float* b, float* x) {
    if (!h || !b || !x) return fail(GMG_ERR_ARG, "null argument");
    const Level& l = h->lev[h->L - 1];
    if (h->L == 1) {  // the coarsest level is level 0
        TRY(clear_pads(h));
        launch_pack0(b, l, h->r, h->stream);
        launch_coarse_solve(h->nL, h->free_idx_p, h->Ainv, h->r, h->z, l.maskp, l.nnp, h->stream);
        launch_unpack0(h->z, l, x, h->stream);
        CU(cudaGetLastError());
        return GMG_OK;
    }
    if (h->coarse_pcg) launch_coarse_pcg(coarse_view(h, h->L - 1), b, x, l.t, l.d, l.x2, h->opt.coarse_pcg_steps,
                                         h->stream);
    else launch_coarse_solve(h->nL, h->free_idx, h->Ainv, b, x, l.mask, l.nn, h->stream);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_vcycle(gmg_handle* h, const float* r, float* z) {
    if (!h || !r || !z) return fail(GMG_ERR_ARG, "null argument");
    if (h->L == 1) return fail(GMG_ERR_ARG, "single-level hierarchy");
    TRY(clear_pads(h));
    const Level& l0 = h->lev[0];
    launch_pack0(r, l0, h->r, h->stream);
    vcycle_level(h, 0, h->r, h->z, h->x2_0, -1, FIN_NONE);
    launch_unpack0(h->z, l0, z, h->stream);
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_residual64(gmg_handle* h, const double* f, const double* u, double* r, double* rel_out) {
    if (!h || !f || !u) return fail(GMG_ERR_ARG, "null argument");
    Level& l0 = h->lev[0];
    cudaStream_t s = h->stream;
    h->sc_host[SC_UNZ] = 1.0;
    launch_set_scalars(h->sc + SC_UNZ, 1, 1.0, 0.0, 0.0, 0.0, s);
    launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f, u, r, nullptr, l0.px, h->sc, h->partials, h->gs64,
                        s);
    launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), h->sc, SC_TRR, FIN_NONE, s);
    launch_dot_f64_masked(f, f, l0.mask, l0.nn, h->partials, s);
    launch_finalize(h->partials, vec_grid_blocks(), h->sc, SC_FF, FIN_NONE, s);
    TRY(sync_scalars(h));
    if (rel_out) *rel_out = std::sqrt(h->sc_host[SC_TRR]) / std::sqrt(h->sc_host[SC_FF]);
    return GMG_OK;
}

}  // extern "C"
