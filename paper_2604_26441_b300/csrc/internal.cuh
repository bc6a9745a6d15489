// Internal declarations shared by the CUDA translation units of the GMG library.
// Layout conventions are those of include/gmg.h.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <atomic>
#include <string>
#include <vector>

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched through the runtime)

#include "gmg.h"

namespace gmg {

// Process-wide count of kernels this library has launched (read by
// gmg_kernel_launches; every launcher adds the number of kernels it starts).
extern std::atomic<unsigned long long> g_kernel_launches;
inline void note_launch(unsigned long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Records the text gmg_last_error() returns on the calling thread.
void set_error_text(const std::string& msg);

// ---- bounds-checked build (compiled with -DGMG_CHECKED) ----------------------
// GMG_B(i, n, site) is the index i of a global access into a buffer of n
// elements.  In the checked build an index outside [0, n) records `site` in
// the translation unit's sticky word (the first site wins) and is replaced by
// 0, so the access stays inside the buffer: nothing traps and nothing is read
// or written out of range.  The host collects the words with
// bounds_site_collect() (gmg_bounds_site, and every solve's final check).  In
// the normal build GMG_B(i, n, site) is just i.
using BoundsReader = unsigned (*)();
void register_bounds_reader(BoundsReader r);
unsigned bounds_site_collect();
#ifdef GMG_CHECKED
static __device__ unsigned g_bounds_site = 0u;
__device__ __forceinline__ long long bounds_index(long long i, long long n, unsigned site) {
    if (i < 0 || i >= n) {
        atomicCAS(&g_bounds_site, 0u, site);
        return 0;
    }
    return i;
}
#define GMG_B(i, n, site) ::gmg::bounds_index((long long)(i), (long long)(n), (site))
namespace {
struct BoundsReg {
    static unsigned read_and_clear() {
        unsigned v = 0, z = 0;
        if (cudaMemcpyFromSymbol(&v, g_bounds_site, sizeof v) != cudaSuccess) { cudaGetLastError(); return 0; }
        if (v) cudaMemcpyToSymbol(g_bounds_site, &z, sizeof z);
        return v;
    }
    BoundsReg() { register_bounds_reader(&read_and_clear); }
};
static BoundsReg g_bounds_reg;
}  // namespace
#else
#define GMG_B(i, n, site) (i)
#endif

constexpr int kMaxLevels = 16;
constexpr int kMaxDegree = 16;
constexpr int kSlots = 27;     // 27-point neighbourhood of a node
constexpr int kPlanes = 243;   // 27 slots x 3 x 3 block entries
constexpr int kSelfSlot = 13;  // slot of offset (0, 0, 0)
constexpr int kSymPlanes = 126;  // stored FP32 planes: diagonal + 13 forward blocks

// Local node a of a hex8 element sits at offset (ldx(a), ldy(a), ldz(a)) from the
// element's lowest corner; local DOF 3a + c.
__host__ __device__ constexpr int ldx(int a) { return (a == 1 || a == 2 || a == 5 || a == 6) ? 1 : 0; }
__host__ __device__ constexpr int ldy(int a) { return (a == 2 || a == 3 || a == 6 || a == 7) ? 1 : 0; }
__host__ __device__ constexpr int ldz(int a) { return a >= 4 ? 1 : 0; }
__host__ __device__ constexpr int slot_of(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }

// Unit-element stiffness passed by value (lands in the kernel-parameter constant
// bank, which broadcasts a warp-uniform read like __constant__ memory but is
// private to each launch, so handles with different nu never collide).
struct KeF { float v[576]; };
struct KeD { double v[576]; };

// The same blocks reduced by the symmetry of the cube (any Poisson ratio): with
// the classes numbered as in fine.cu, the 72 entries take eight distinct values
// and 27 of them vanish --
//   class 0 (modes X, Y, Z of components x, y, z) and class 7 (YZ, XZ, XY of x,
//     y, z): a on the diagonal and b off it, so w_i = (a - b) u_i + b (u_x + u_y + u_z);
//   classes 1, 2 and 4 (two modes each): the block [[p, q], [q, p]];
//   classes 3, 5 and 6: a 2x2 block of equal entries c (both outputs are
//     c (u_i + u_j)) and one entry d for the XYZ mode.
// GSym holds (a - b, b) of class 0, the same of class 7, (p, q) and (c, d).
struct GSym { float2 ab0, ab7, pq, cd; };
// The level-1 operator in the coarse element's mode basis: G0 = T0^T G T0 on
// the structural pattern of level1_mf.cu (279 entries, which take 21 values up
// to sign for every Poisson ratio; L1Coef holds those 21).
constexpr int kL1Coefs = 279, kL1Classes = 21;
struct L1Coef { float g[kL1Classes]; };
// Host: GSym from the 72 FP64 block entries (each value the mean of its equal
// entries); false when an entry departs from the pattern by more than 1e-12 of
// the largest one.  v64, when given, receives the eight values in FP64 in the
// order of GSym (a - b, b, a' - b', b', p, q, c, d).
bool gsym_from_blocks(const double g[72], GSym* out, double* v64 = nullptr);

// Rounded lane arithmetic for one element (float) or two (float2).
__device__ __forceinline__ float g_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 g_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float g_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 g_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float g_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 g_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// One element's coefficients: E_e times the eight values of GSym.
template <class L>
struct GElem {
    L a0, b0, a7, b7, p, q, c, d;
};
__device__ __forceinline__ GElem<float> gsym_scale(const GSym& G, float E) {
    const float2 e2 = make_float2(E, E);
    const float2 ab0 = __fmul2_rn(G.ab0, e2), ab7 = __fmul2_rn(G.ab7, e2);
    const float2 pq = __fmul2_rn(G.pq, e2), cd = __fmul2_rn(G.cd, e2);
    return {ab0.x, ab0.y, ab7.x, ab7.y, pq.x, pq.y, cd.x, cd.y};
}
// two elements with moduli E.x and E.y
__device__ __forceinline__ GElem<float2> gsym_scale2(const GSym& G, float2 E) {
    auto b = [](float v) { return make_float2(v, v); };
    return {__fmul2_rn(b(G.ab0.x), E), __fmul2_rn(b(G.ab0.y), E), __fmul2_rn(b(G.ab7.x), E),
            __fmul2_rn(b(G.ab7.y), E), __fmul2_rn(b(G.pq.x), E),  __fmul2_rn(b(G.pq.y), E),
            __fmul2_rn(b(G.cd.x), E),  __fmul2_rn(b(G.cd.y), E)};
}

// w[m][c] = (E_e G u)[m][c] for the 21 non-constant modes (m = 1..7; monomial
// bits X = 1, Y = 2, Z = 4; c the displacement component), every operation
// rounded on its own and in this order in every kernel.
template <class L>
__device__ __forceinline__ void gsym_contract(const GElem<L>& k, const L (&u)[8][3], L (&w)[8][3]) {
    {  // class 0: (X, x), (Y, y), (Z, z)
        const L t = g_mul(k.b0, g_add(g_add(u[1][0], u[2][1]), u[4][2]));
        w[1][0] = g_fma(k.a0, u[1][0], t);
        w[2][1] = g_fma(k.a0, u[2][1], t);
        w[4][2] = g_fma(k.a0, u[4][2], t);
    }
    {  // class 7: (YZ, x), (XZ, y), (XY, z)
        const L t = g_mul(k.b7, g_add(g_add(u[6][0], u[5][1]), u[3][2]));
        w[6][0] = g_fma(k.a7, u[6][0], t);
        w[5][1] = g_fma(k.a7, u[5][1], t);
        w[3][2] = g_fma(k.a7, u[3][2], t);
    }
    // class 1: (XY, y), (XZ, z); class 2: (XY, x), (YZ, z); class 4: (XZ, x), (YZ, y)
    w[3][1] = g_fma(k.p, u[3][1], g_mul(k.q, u[5][2]));
    w[5][2] = g_fma(k.q, u[3][1], g_mul(k.p, u[5][2]));
    w[3][0] = g_fma(k.p, u[3][0], g_mul(k.q, u[6][2]));
    w[6][2] = g_fma(k.q, u[3][0], g_mul(k.p, u[6][2]));
    w[5][0] = g_fma(k.p, u[5][0], g_mul(k.q, u[6][1]));
    w[6][1] = g_fma(k.q, u[5][0], g_mul(k.p, u[6][1]));
    {  // class 3: (Y, x), (X, y) and (XYZ, z)
        const L h = g_mul(k.c, g_add(u[2][0], u[1][1]));
        w[2][0] = h;
        w[1][1] = h;
        w[7][2] = g_mul(k.d, u[7][2]);
    }
    {  // class 5: (Z, x), (X, z) and (XYZ, y)
        const L h = g_mul(k.c, g_add(u[4][0], u[1][2]));
        w[4][0] = h;
        w[1][2] = h;
        w[7][1] = g_mul(k.d, u[7][1]);
    }
    {  // class 6: (Z, y), (Y, z) and (XYZ, x)
        const L h = g_mul(k.c, g_add(u[4][1], u[2][2]));
        w[4][1] = h;
        w[2][2] = h;
        w[7][0] = g_mul(k.d, u[7][0]);
    }
}

// Scalar slots of the per-handle FP64 scalar array.
enum Scalar {
    SC_FF = 0,      // ||f_free||^2
    SC_RR = 1,      // ||r||^2 (recursive residual)
    SC_RZ = 2,      // r . z
    SC_PQ = 3,      // p . q
    SC_ALPHA = 4,
    SC_BETA = 5,
    SC_RZNEW = 6,
    SC_TRR = 7,     // ||f - K u||^2 in FP64 (true residual)
    SC_NRM = 8,     // power iteration: ||w||^2
    SC_VKV = 9,
    SC_VDV = 10,
    SC_UNZ = 11,    // nonzero count of u (> 0: u is not the zero vector)
    SC_TMP = 12,    // 12, 13: scratch
    SC_IT = 16,     // PCG iterations completed (device-resident loop)
    SC_TOL = 17,    // relative tolerance
    SC_MAXIT = 18,  // iteration cap
    SC_NF = 19,     // ||f_free||
    SC_ACT = 20,    // multi-load solve: this load still iterates (1) or has stopped (0)
    SC_COUNT = 24
};

// Operations the reduction finaliser applies after storing its sum.
enum FinOp { FIN_NONE = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_NRMCHK = 3 };

struct Level {
    int nx = 0, ny = 0, nz = 0;     // element counts
    long long nn = 0;               // node count (nx+1)(ny+1)(nz+1)
    // Vectors of a level are node-major, 3 floats per node, node (i, j, k) at
    // i + px (j + (ny+1) k).  Levels >= 1: px = nx + 1 (dense).  Level 0 pads
    // every node row to px = nx + 1 rounded up to a multiple of 4, so that each
    // row starts on a 16-byte boundary (TMA-fed fine operator); pad nodes hold 0.
    int px = 0;                     // nodes per row of the level's vectors
    long long nnp = 0;              // nodes allocated per vector: px (ny+1)(nz+1)
    uint8_t* mask = nullptr;        // [nn] fixed-component bits (dense numbering)
    uint8_t* maskp = nullptr;       // [nnp] the same bits in the vectors' numbering (pads: 7)
    float* invdiag = nullptr;       // [3nn] D^{-1} (levels >= 1), 0 on fixed DOFs
    double* A64 = nullptr;          // [243 nn] Galerkin operator planes, FP64 (levels >= 1)
    float* A32 = nullptr;           // [126 ps] FP32 diagonal + forward blocks (levels >= 1)
    long long ps = 0;               // plane stride of A32: nn rounded up to 4 (16-byte aligned planes)
    bool tma = false;               // operator streamed by the TMA-staged kernel (tm_own / tm_back valid)
    int bsr_kind = -1;              // kernel of the non-TMA operator (bsr_grid_blocks), set by gmg_autotune
    float* eh = nullptr;            // level 1: Ehat per coarse element when the matrix-free form is exact
    float* cf = nullptr;            // level 1: corner forces of the matrix-free form [8][ne] float4 (per handle)
    CUtensorMap tm_own{};           // A32 as a [126][ps] FP32 tensor, box 126 planes x 64 nodes
    CUtensorMap tm_back{};          // same tensor, box 9 planes x 68 nodes
    float* x = nullptr;             // [3nn] smoother iterate / V-cycle output (levels >= 1)
    float* x2 = nullptr;            // [3nn] ping-pong partner of x
    float* b = nullptr;             // [3nn] right-hand side (levels >= 1)
    float* t = nullptr;             // [3nn] residual before restriction
    float* d = nullptr;             // [3nn] Chebyshev increment
    double* coef = nullptr;         // [2 kMaxDegree] (c_d, c_a) per smoother step
    int kind = GMG_SMOOTHER_JACOBI;
    int degree = 2;
    double omega = 0.5;
    int n_free = 0;
};

// Device view of one assembled level for the fused lower V-cycle (coarse_fused.cu).
struct CoarseLevel {
    int nx, ny, nz, nn;
    const uint8_t* mask;
    const float* A;          // symmetric half storage, [126][ps]
    int ps;
    const float* invdiag;
    float *x, *x2, *b, *t, *d;
    const double* coef;
    int kind, degree;
};

// ---- the bottom of the V-cycle as one cluster launch (lower_cluster.cu) -------
struct LowerClusterArgs {
    // finer level m - 1 (dense vectors): its residual, restricted into level m
    int fnx, fny, fnz;
    const float* ft;
    // level m, the last assembled level (dense vectors); its x holds the result
    CoarseLevel m;
    // coarsest level (dense vectors), its free DOFs and the inverse's FP32 parts
    int cnx, cny, cnz, cnn;
    const uint8_t* cmask;
    float *cb, *cx;
    int nL;
    const int* free_idx;
    const float *Ahi, *Alo;
};
// shared memory per CTA for a level m of nn nodes and nL coarsest free DOFs
size_t lower_cluster_smem(int nn, int nL);
// whether a cluster with that shared memory can run (sets the kernel attributes)
bool lower_cluster_available(size_t smem);
void launch_lower_cluster(const LowerClusterArgs& a, size_t smem, cudaStream_t s);
// hi[i] = (float)A[i], lo[i] = (float)(A[i] - hi[i])
void launch_split_inverse(const double* A, long long n, float* hi, float* lo, cudaStream_t s);

// ---- multi-load vectors (multi.cu) ------------------------------------------
// Up to kLoads right-hand sides on one hierarchy advance together.  A level's
// multi-load vector holds, for node n (the level's vector numbering; level 0:
// rows padded to px nodes) and load l, the record (u_x, u_y, u_z, 0) at float
// offset (n * kLoads + l) * 4: 16-byte records, 256 bytes per node.
constexpr int kLoads = 16;
constexpr int kNodeF = 4 * kLoads;  // floats per node of a multi-load vector

struct MultiLevel {
    float *x = nullptr, *x2 = nullptr, *b = nullptr, *t = nullptr, *d = nullptr;
};

// Workspace of the multi-load solve, owned by one handle (allocated on its
// first multi-load call; its device buffers are in the handle's allocation list).
struct MultiWork {
    float *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x2 = nullptr, *t = nullptr, *d = nullptr;
    MultiLevel lev[kMaxLevels];
    double* sc = nullptr;        // [kLoads][SC_COUNT] device scalars, one block per load
    double* partials = nullptr;  // [kLoads][pstride]
    int pstride = 0;
    float* Ahi = nullptr;        // coarsest inverse split into FP32 hi + lo (double-float apply)
    float* Alo = nullptr;
    float* bc = nullptr;         // [nL][kLoads] gathered coarsest right-hand sides
    float2* wcor = nullptr;      // [kLoads][3 nn] the PCG steps since the iterates were last updated
                                 // (double-float hi, lo per DOF); added to them before the FP64 residual
    bool w_dirty = false;        // steps were launched since the last flush
    void* pinned = nullptr;      // host-mapped mirror of sc and the sticky error words
    double* sc_host = nullptr;
    double* sc_map = nullptr;
    int* err_host = nullptr;
    int* err_map = nullptr;
    int fine_kernel = 0;         // level-0 operator: 0 CUDA-core (Hadamard), 1 tensor cores
    float* tcB = nullptr;        // tensor-core operator: K_e operand, [hi, lo][4 corner pairs][2][32][4] FP32
    float tc_scale = 1.f;        // K_e = tc_scale * (hi + lo)
    int tc_passes = 0;           // MMA passes per corner pair: 3 (K_e exact in TF32) or 5 (K_e split)
    int launch_err = 0;          // a level-0 launch could not be prepared (tensor map encoding)
    // captured loops, keyed by the iterate pointers
    struct Loop {
        std::vector<const double*> u;
        cudaGraph_t g;
        cudaGraphExec_t ex;
        unsigned long long pre, body;
    };
    std::vector<Loop> loops;
};

// Arguments of the fused lower V-cycle: levels start..L-1, coarsest solve data,
// and the grid-barrier words (arrival count, generation, error flag).
struct CoarseFused {
    CoarseLevel lev[kMaxLevels];
    int start, L, nL;
    const int* free_idx;
    const double* Ainv;
    unsigned* bar_count;
    unsigned* bar_gen;
    int* err;
    long long spin_limit;
};

// float -> double, equal to (double)f for every input, with the conversion of
// zeros and normal values done by integer operations (IEEE 754: the binary64
// exponent is the binary32 exponent + 896, the 23 mantissa bits move up by 29).
// The FP64 pipe of this part issues a small fraction of the FP32 rate, and a
// conversion costs it as much as a DFMA; subnormal, inf and NaN inputs (which do
// not occur in the solve's vectors) take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu, e = a >> 23;
    if ((e == 0u && a != 0u) || e == 0xffu) return (double)f;
    const unsigned hi = (b & 0x80000000u) | (a == 0u ? 0u : (a >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
}

// 1 / (k_d sum E), the fine level's Jacobi scale: the hardware reciprocal
// approximation (rcp.approx, within about one ulp), one instruction where the
// IEEE reciprocal takes a refinement sequence.  Every kernel that forms the
// scale uses it, so the fine kernels stay bitwise equal to each other.
__device__ __forceinline__ float jacobi_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-thread dot-product accumulator in double-single arithmetic: products are
// split exactly with an FMA and summed with TwoSum, so a thread's partial is
// accurate to ~2^-48 of the sum of |terms| while staying on the FP32 pipes (FP64
// issue is a small fraction of FP32 on this part).  Partials are combined across
// threads and blocks in FP64.
struct DSAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        // every operation rounded on its own (no contraction into an FMA)
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---- programmatic dependent launch: kernels of the solve path start with
// pdl_entry() -- wait until the grids they depend on have completed and their
// writes are visible, then let the next kernel in the stream begin launching --
// and are launched with pdl_launch, so that consecutive kernels overlap their
// launch latency instead of serialising it.  A kernel launched without the
// attribute passes pdl_entry() at once.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- TMA and mbarrier primitives (inline PTX, sm_90+ forms; this build targets sm_103a)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes initialised mbarriers visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Arrives once on `bar` and adds `bytes` to the transaction count of its phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One bounded probe of phase `parity` of `bar` (true once that phase has completed).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Tiled TMA loads into shared memory completing on `bar`.  The innermost
// coordinate must be a multiple of 4 FP32 elements (16-byte aligned start);
// coordinates outside the tensor read as zero.
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, int x, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
          "r"(smem_u32(bar))
        : "memory");
}

// Host: tiled tensor map of an FP32 array, rank 1 (dims[0] elements, box[0]) or
// rank 2 (dims[0] x dims[1], row pitch dims[0] elements, box[0] x box[1]).
// Returns false when the driver entry point is unavailable or the encoder
// rejects the geometry (e.g. an address that is not 16-byte aligned).
bool encode_f32_map(CUtensorMap* map, const float* base, int rank, const unsigned long long* dims,
                    const unsigned* box);
// Host: tiled tensor map of an FP32 array of rank 1..5 with explicit byte
// strides of dimensions 1..rank-1 (multiples of 16); out-of-range boxes read 0.
bool encode_f32_map_strided(CUtensorMap* map, const float* base, int rank, const unsigned long long* dims,
                            const unsigned long long* strides, const unsigned* box);

}  // namespace gmg

struct gmg_handle {
    int L = 0;                                  // number of levels
    gmg::Level lev[gmg::kMaxLevels];
    cudaStream_t stream = nullptr;
    gmg_options opt{};
    int device = 0;
    float* E32 = nullptr;                       // fine moduli, FP32, [nz][ny][nx]
    float* E32p = nullptr;                      // the same, rows padded: [nz][ny][ex]
    int ex = 0;                                 // nx rounded up to a multiple of 4
    int* free_idx_p = nullptr;                  // coarsest free DOFs in the vectors' numbering
    bool pads_dirty = false;                    // a solve ended non-finite: re-zero level-0 vectors
    bool coarse_pcg = false;                    // coarsest above the Cholesky cutoff: fixed-count PCG
    double* E64 = nullptr;                      // fine moduli, FP64
    gmg::KeF keF{};
    gmg::KeD keD{};
    gmg::GSym gs{};                             // fine operator coefficients (symmetric form of G)
    gmg::L1Coef l1g{};                          // level-1 matrix-free coefficients (G0 on its pattern)
    double gs64[8] = {};                        // the same eight values in FP64 (FP64 true residual)
    float kd = 0.f;                             // diagonal entry of K_e (all equal)
    double setup_ms = 0.0;                      // host wall time of gmg_setup (clones: the source's)
    float* inv0 = nullptr;                      // [n_nodes] fine Jacobi scale 1 / (kd * sum of adjacent E_e)
    double* lam = nullptr;                      // [kMaxLevels] lambda estimates (device)
    // fine-level PCG vectors
    float *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x2_0 = nullptr, *t0 = nullptr, *d0 = nullptr;
    // the PCG steps since the FP64 iterate was last updated, in double-float
    // (level-0 layout); added to u by launch_flush_w before u is read
    float *wh = nullptr, *wl = nullptr;
    bool w_dirty = false;                       // steps were launched since the last flush
    // reductions
    double* partials = nullptr;
    int max_partials = 0;
    double* sc = nullptr;                       // [SC_COUNT] device scalars
    double* sc_host = nullptr;                  // pinned, host-mapped mirror (written by k_publish)
    double* sc_map = nullptr;                   // device address of sc_host
    int* err_host = nullptr;                    // [2] sticky error words, same pinned block
    int* err_map = nullptr;                     // device address of err_host
    double* hcol_host = nullptr;                // [kMaxRestart + 2] FGMRES Hessenberg column, same block
    double* hcol_map = nullptr;                 // device address of hcol_host
    // coarsest dense solve
    int nL = 0;
    int* free_idx = nullptr;                    // [nL] DOF indices of the coarsest free DOFs
    double* Ainv = nullptr;                     // [nL nL]
    float *Ahi = nullptr, *Alo = nullptr;       // [nL nL] FP32 parts of Ainv (cluster path)
    bool use_lc = false;                        // bottom of the V-cycle as one cluster launch
    size_t lc_smem = 0;                         // its shared memory per CTA
    double eps = 0.0;
    gmg::CoarseFused cf{};                      // fused lower V-cycle (levels cf.start..L-1)
    bool use_fused = false;
    int* kerr = nullptr;                        // sticky error word of the TMA / tensor-core kernels
    void* tcB = nullptr;                        // tensor-core smoother operand (device, 4 KB)
    // device-resident PCG loop: a CUDA graph [restart, step, check, while{direction, step, check}]
    cudaStream_t cap_stream = nullptr;          // private stream used only to capture the graph
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    const double* loop_u = nullptr;             // iterate the captured graph updates
    unsigned long long loop_prefix_kernels = 0, loop_body_kernels = 0;
    bool loop_unavailable = false;              // capture failed once: use the host loop
    // loops captured for other iterate buffers (least recently used first), so
    // that a caller alternating between a few u buffers does not recapture
    struct LoopGraph {
        const double* u;
        cudaGraph_t g;
        cudaGraphExec_t ex;
        unsigned long long pre, body;
    };
    std::vector<LoopGraph> loop_cache;
    // restarted FGMRES (outer = 1): Arnoldi basis V (restart + 1 vectors),
    // preconditioned directions Z (restart vectors), Hessenberg column (device)
    float* fg_V = nullptr;
    float* fg_Z = nullptr;
    double* fg_h = nullptr;
    int fg_m = 0;
    double* kap_u = nullptr;                    // FP64 scratch iterate of the kappa_eff probe
    bool is_clone = false;                      // shares the hierarchy of another handle
    // gmg_solve_batch: the last batch graph captured with this handle first
    cudaGraph_t batch_graph = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<std::pair<const gmg_handle*, const double*>> batch_key;
    std::vector<std::pair<unsigned long long, unsigned long long>> batch_counts;
    unsigned batch_gen = 0;                     // multi_generation() when batch_graph was captured
    int fused_blocks = 0;
    gmg::MultiWork* mw = nullptr;               // multi-load solve workspace (multi.cu), lazily allocated
    std::vector<void*> allocs;                  // every device allocation, freed by gmg_destroy
    void* pinned = nullptr;                     // pinned host-mapped block (sc_host, err_host)
};

namespace gmg {

// ---- launchers implemented in hot.cu ------------------------------------------
enum FineMode { FM_APPLY = 0, FM_SMOOTH = 1, FM_RESID = 2 };

struct FineArgs {
    int nx, ny, nz;
    int pitch;             // nodes per row of the vectors and the mask (nx + 1, or the padded
                           // level-0 pitch, a multiple of 4)
    int epitch;            // moduli per row of Ep (a multiple of 4)
    const float* Ep;       // moduli in the padded layout [nz][ny][epitch] (TMA-fed kernel)
    const float* E;
    const uint8_t* mask;
    const float* xin;      // operand of K
    const float* b;        // right-hand side (smooth / resid)
    const float* dold;     // previous increment (smooth, c_d != 0)
    float* dnew;           // new increment (smooth, may alias dold; nullptr = not written)
    float* out;            // y, x_new or t
    const double* coef;    // smoother coefficient table
    int step;
    double* partial;       // per-block partial dots (nullptr = none)
    float kd;
    const float* inv0;     // [n_nodes] 1 / (kd * sum of the adjacent moduli), from set-up
    float* scratch;        // fine-level vector used to mask a caller's operand (apply only)
    const void* tcB;       // tensor-core smoother: BF16 mode-to-corner operand (hi, lo), 4 KB
    int* err;              // sticky error word (a tensor-core wait that gave up)
};

// Tiles of the fine kernel: one element column per thread (0: 32x8 threads,
// 1: 16x16), or two x-adjacent columns per thread (fine_pair.cu; 2: 8x16
// threads = 16x16 columns, 3: 16x8 threads = 32x8 columns, 4: 16x16 threads =
// 32x16 columns).  The two-column tiles run only on the TMA-fed path.
constexpr int kFineTiles = 5;
constexpr int kFinePair8x16 = 2, kFinePair16x8 = 3, kFinePair16x16 = 4;
int fine_grid_blocks(int nx, int ny, int nz);
// Candidate (tile, z-chunk) plans of the fine kernel for a grid with at most
// max_blocks blocks; the cost model's plan; and the process-wide override that
// gmg_autotune sets (tile < 0 clears it).
int fine_candidates(int nx, int ny, int nz, int max_blocks, int* tiles, int* zcs, int cap);
void fine_model_plan(int nx, int ny, int nz, int* tile, int* zc);
int fine_plan_blocks(int nx, int ny, int nz, int tile, int zc);
void fine_set_plan(int nx, int ny, int nz, int tile, int zc);
// mask_in: treat fixed DOFs of the operand as 0 (for operands that may hold
// values there, e.g. user input); internal vectors are already 0 on them.
void launch_fine(int mode, int dot, int mask_in, const FineArgs& a, const GSym& G, cudaStream_t s);
// The TMA-fed fine operator on padded level-0 vectors (a.pitch and a.epitch
// multiples of 4, a.Ep the padded moduli); GMG_OK, or an error when a tensor map
// cannot be encoded (nothing is launched then).
int launch_fine_tma(int mode, int dot, const FineArgs& a, const GSym& G, cudaStream_t s);
// The two-column operator (tiles 2..4) on a grid of `grid` blocks, zc node
// planes per block; GMG_ERR_ARG for another tile or unpadded vectors.
int launch_fine_pair(int tile, int mode, int dot, dim3 grid, int zc, const FineArgs& a, const GSym& G,
                     cudaStream_t s);
void launch_hadamard_blocks(const double* Ke, double* g72, cudaStream_t s);
// Tensor-core fine smoother step (SMOOTH mode): passes = 1 (BF16) or 3 (split BF16).
void launch_fine_tc(int passes, int dot, const FineArgs& a, cudaStream_t s);
// Host: the BF16 hi/lo mode-to-corner operand of the tensor-core smoother from G.
void build_tc_operand(const double g[72], uint16_t out[2048]);
int resid64_grid_blocks(int nx, int ny, int nz);
// The FP64 residual of nl <= kLoads loads in one launch (no vector output):
// ||f_l - K u_l||^2 partials of load l at partial[l * pstride ...], its grid
// (blocks per load) from resid64_grid_blocks_multi; sc: the loads' scalar
// blocks (SC_COUNT apart, SC_UNZ read).
int resid64_grid_blocks_multi(int nx, int ny, int nz, int nl);
void launch_fine_resid64_multi(int nx, int ny, int nz, const double* E, const uint8_t* mask, int nl,
                               const double* const* f, const double* const* u, const double* sc, double* partial,
                               int pstride, const double* g8, cudaStream_t s);
void launch_fine_smooth0(const FineArgs& a, cudaStream_t s);
// inv0[n] = 1 / (kd * sum of the moduli of the elements around node n), once at set-up.
void launch_fine_inv0(int nx, int ny, int nz, int px, const float* E, float kd, float* inv0, cudaStream_t s);
// r64 (optional) in the dense numbering; r32 (optional) in the level-0 vector
// numbering of pitch px.
void launch_fine_resid64(int nx, int ny, int nz, const double* E, const uint8_t* mask,
                         const double* f, const double* u, double* r64, float* r32, int px,
                         const double* sc, double* partial, const double* g8, cudaStream_t s);

struct BsrArgs {
    int nx, ny, nz;
    long long nn;
    long long ps;                // plane stride of A
    const float* A;
    const float* invdiag;
    const uint8_t* mask;
    const float* xin;
    const float* b;
    const float* dold;
    float* dnew;
    float* out;
    const double* coef;
    int step;
    double* partial;
    int* err;                    // sticky error word (a TMA wait that gave up)
    int kind;                    // kernel choice, as bsr_grid_blocks
    const CUtensorMap* tm_own;   // non-null: stream through the TMA-staged kernel
    const CUtensorMap* tm_back;
    const float* eh;             // level 1 applied matrix-free (kind kBsrMatrixFree): Ehat per coarse element
    const L1Coef* l1g;           // and its coefficients (host copy, passed by value to the kernel)
    float* cf;                   // and its corner-force workspace [8][ne] float4
};
// Blocks (= dot partials) of the operator launch for a level of nn nodes: 64
// nodes per block for the TMA-staged and K-split kernels, 256 for streaming.
// kind: -1 = by size (streaming kernel from 65,536 nodes, K-split below),
// 0 = streaming k_bsr, 1 / 2 / 3 / 4 / 5 = K-split k_bsr_ks with 8 / 2 / 4 /
// 16 / 32 slices (ignored when tma)
constexpr int kBsrKinds = 6;
// Level 1 applied matrix-free from the fine moduli (level1_mf.cu), where exact.
constexpr int kBsrMatrixFree = 6;
int l1mf_grid_blocks(int nx, int ny, int nz);
void launch_l1mf(int mode, int dot, const BsrArgs& a, const L1Coef& G, float* cf, cudaStream_t s);
// Ehat (8 floats per coarse element, [ne1][8]) from the FP64 fine moduli; fine sizes even.
void launch_l1_ehat(const double* E_fine, int nx, int ny, int nz, float* eh, cudaStream_t s);
// Host: the 21 class values from the FP64 blocks of G; false if G0 has entries off
// the pattern or a class whose entries differ.
bool l1_coef_from_blocks(const double g[72], L1Coef* out);
// Host: whether the matrix-free form equals the assembled level-1 operator for a
// fine grid of nx x ny x nz elements with fixed-component bits fine_mask_host
// (dense numbering): even sizes, and every fixed fine DOF with only fixed
// prolongation parents.
bool l1mf_eligible(int nx, int ny, int nz, const uint8_t* fine_mask_host);
int bsr_grid_blocks(long long nn, bool tma, int kind = -1);
// Encodes the two tensor maps of a level's FP32 planes; GMG_OK or an error code.
int encode_bsr_maps(Level& l);
void launch_bsr(int mode, int dot, const BsrArgs& a, cudaStream_t s);
// b = P^T t (restriction from fine level f) fused with the first smoothing
// step from zero on the coarse level of a (a.b unused; b is written to bout).
void launch_restrict_smooth0(const Level& f, const float* t, const BsrArgs& a, float* bout, cudaStream_t s);
void launch_bsr_smooth0(const BsrArgs& a, cudaStream_t s);

void launch_restrict(const Level& f, const Level& c, const float* fine, float* coarse, cudaStream_t s);
void launch_prolong_add(const Level& f, const Level& c, const float* coarse, float* fine, cudaStream_t s);
constexpr int kMaxRestart = 256;  // FGMRES restart length limit (gmg_options.restart)
// Scalars between host and device without a copy engine (so they never queue
// behind a caller's large copies on other streams): k_publish writes the device
// scalars and the two sticky error words (e1 may be null) into the pinned
// host-mapped block (err_map null: values only); k_set_scalars writes up to four
// values passed as kernel arguments.
void launch_publish(const double* sc, int n, double* out_map, const int* e0, const int* e1, int* err_map,
                    cudaStream_t s);
void launch_set_scalars(double* sc, int n, double v0, double v1, double v2, double v3, cudaStream_t s);
// k_publish for the items of a batch, up to kPublishItems per launch.
constexpr int kPublishItems = 128;
struct PublishBatch {
    const double* sc[kPublishItems];
    double* out[kPublishItems];
    const int* e0[kPublishItems];
    const int* e1[kPublishItems];
    int* eout[kPublishItems];
    int count, n;
};
void launch_publish_batch(const PublishBatch& b, cudaStream_t s);
// y[0..n) = x[0..n) by a kernel (a device-to-device cudaMemcpyAsync may take a
// copy engine that a caller's host copies keep busy)
void launch_copy_f32(float* y, const float* x, long long n, cudaStream_t s);
// x = Ainv b on the coarsest level's free DOFs, 0 on its fixed DOFs (mask).
void launch_coarse_solve(int nL, const int* free_idx, const double* Ainv, const float* b, float* x,
                         const uint8_t* mask, long long n_nodes, cudaStream_t s);

int vec_grid_blocks();
void launch_dot_f32(const float* a, const float* b, long long n, double* partial, cudaStream_t s);
void launch_dot_f64_masked(const double* a, const double* b, const uint8_t* mask, long long nn,
                           double* partial, cudaStream_t s);
void launch_finalize(const double* partial, int n, double* sc, int slot, int op, cudaStream_t s);
// w = wh + wl (double-float) += alpha p; r -= alpha q; ||r||^2 partials
// (level-0 vectors of pitch px)
void launch_pcg_update(float* wh, float* wl, float* r, const float* p, const float* q, const Level& l0,
                       const double* sc, double* partial, cudaStream_t s);
// u (dense numbering, FP64) += wh + wl, then wh = wl = 0
void launch_flush_w(double* u, float* wh, float* wl, const Level& l0, cudaStream_t s);
void launch_p_update(float* p, const float* z, long long n, const double* sc, cudaStream_t s);
void launch_mask_u64(double* u, const uint8_t* mask, long long nn, double* partial, cudaStream_t s);
// r = f on free DOFs, 0 elsewhere (pads included): f dense, r a level-0 vector
void launch_cast_masked(const double* f, const Level& l0, float* r, cudaStream_t s);
// Level-0 vectors to and from the dense numbering a caller uses: pack writes
// every entry of out (fixed DOFs and pads 0); unpack writes every dense entry.
void launch_pack0(const float* in, const Level& l0, float* out, cudaStream_t s);
void launch_unpack0(const float* in, const Level& l0, float* out, cudaStream_t s);
// ||r||^2 into SC_RR (as launch_finalize) and the convergence test of the
// device-resident loop: counts the iteration and sets the while-node condition
// to 1 while ||r|| / ||f|| >= tol, the scalars are finite and the cap is not
// reached.
void launch_finalize_check(const double* partial, int n, double* sc, cudaGraphConditionalHandle cond,
                           cudaStream_t s);
void launch_axpy_dev(float* y, const float* x, long long n, const double* coef, float sign, cudaStream_t s);
// u (dense, FP64) += a z (a level-0 vector)
void launch_axpy_u64(double* u, const float* z, const Level& l0, double a, cudaStream_t s);
void launch_scale_by_inv_sqrt(float* v, long long n, const double* sc, int slot, cudaStream_t s);
void launch_scale_invdiag_fine(const float* y, float* w, const float* E, const Level& l0, float kd, cudaStream_t s);
void launch_scale_invdiag_bsr(const float* y, float* w, const float* invdiag, long long n, cudaStream_t s);
void launch_diag_dot_fine(const float* v, const float* E, const Level& l0, float kd, double* partial, cudaStream_t s);
void launch_diag_dot_bsr(const float* v, const float* invdiag, long long n, double* partial, cudaStream_t s);
// start vector over the level's dense DOF index, written in its vector numbering
void launch_power_start(float* v, const Level& l, cudaStream_t s);

// ---- launchers implemented in setup.cu ----------------------------------------
void launch_moduli(const float* rho, long long ne, double p, double E0, double Emin, double* E64,
                   float* E32, cudaStream_t s);
void launch_element_stiffness(double nu, double* Ke, cudaStream_t s);
void launch_mask_clamp(uint8_t* mask, int nx, int ny, int nz, cudaStream_t s);
void launch_mask_from_dofs(const uint8_t* fixed_dofs, uint8_t* mask, long long nn, cudaStream_t s);
void launch_mask_inject(const Level& f, Level& c, cudaStream_t s);
void launch_count_free(const uint8_t* mask, long long nn, int* out, cudaStream_t s);
// l0.maskp from l0.mask (pad nodes fixed); dense DOF indices -> level-0 vector numbering
void launch_mask_pad(const Level& l0, cudaStream_t s);
void launch_pad_index(const int* idx, int n, const Level& l0, int* out, cudaStream_t s);
void launch_child_patterns(const double* Ke, double* Mpat, cudaStream_t s);
void launch_coarse_element_matrices(int nx, int ny, int nz, const double* E, const uint8_t* fine_mask,
                                    const double* Ke, const double* Mpat, double* Kc, cudaStream_t s);
void launch_fine_element_matrices(const double* E, long long ne, const double* Ke, double* Kc, cudaStream_t s);
void launch_gather_level1(const Level& c, const double* Kc, double* A64, cudaStream_t s);
void launch_galerkin_rap(const Level& f, const Level& c, cudaStream_t s);
void launch_finish_bsr(Level& l, cudaStream_t s);
void launch_smoother_coef(double* coef, const double* lam, int kind, int degree, double omega,
                          double alpha, double safety, cudaStream_t s);
void launch_free_index(const uint8_t* mask, long long nn, int* free_idx, int* count, cudaStream_t s);
void launch_dense_gather(const Level& l, const int* free_idx, int n, double* dense, cudaStream_t s);
void launch_regularise(double* dense, int n, double* eps_out, cudaStream_t s);
int cholesky_and_inverse(double* A, int n, double* work, int* info_dev, double* Ainv, cudaStream_t s);

// ---- coarse_fused.cu ------------------------------------------------------------
int coarse_fused_blocks(int* blocks_out, size_t shm);
int launch_coarse_fused(const CoarseFused& a, int blocks, cudaStream_t s);
// x = `steps` Jacobi-PCG steps on K^L x = b from 0 (the coarsest solve above the
// dense-Cholesky cutoff); r, p, q: level-sized scratch vectors.
void launch_coarse_pcg(const CoarseLevel& l, const float* b, float* x, float* r, float* p, float* q, int steps,
                       cudaStream_t s);
void launch_lambda_finish(double* sc, double* lam_slot, cudaStream_t s);

// ---- the level-0 operator of the multi-load path (multi.cu, multi_tc.cu) ------------
struct MFineArgs {
    int nx, ny, nz;
    int px;                // nodes per row of the level-0 vectors (multiple of 4)
    int epitch;            // moduli per row of Ep
    int nl;                // loads processed
    const float* Ep;       // moduli [nz][ny][epitch]
    const uint8_t* maskp;  // level-0 mask, vector numbering
    const float* inv0;     // [nnp] fine Jacobi scale (tensor-core smoother)
    const float* xin;
    const float* b;
    const float* dold;
    float* dnew;
    float* out;
    const double* coef;
    int step;
    double* partial;       // [kLoads][pstride] (nullptr = no dot)
    int pstride;
    float kd;
    int* err;
};
// CUDA-core operator: one block per (tile, load); GMG_OK or an error (tensor maps).
int launch_mfine(int mode, int dot, const MFineArgs& a, const GSym& G, cudaStream_t s);
int mfine_blocks(int nx, int ny, int nz, int nl);
// Tensor-core operator (multi_tc.cu): blocks per load group, and the launch.
int mfine_tc_blocks(int nx, int ny, int nz);
int launch_mfine_tc(int mode, int dot, const MFineArgs& a, const float* Bop, float scale, int passes,
                    cudaStream_t s);
// Host: the K_e operand of the tensor-core operator from K_e (FP64, 24 x 24):
// returns the MMA passes (3 when K_e is a multiple of an integer matrix exact in
// TF32, else 5) and the scale; out receives 2 x 1024 floats.
int build_mfine_tc_operand(const double* Ke, float* out, float* scale);

// ---- multi.cu: multi-load solve pieces used by gmg_solve_batch ---------------------
// Allocates h's multi-load workspace once (GMG_OK or an error code).
int multi_workspace(gmg_handle* h);
void multi_free(gmg_handle* h);
void multi_drop_loops(gmg_handle* h);
// True when h's options and hierarchy suit the multi-load path (else *why says why).
bool multi_ok(const gmg_handle* h, std::string* why);
// Asynchronous per-load pieces, writing load l's scalar block h->mw->sc + l * SC_COUNT.
void multi_norms(gmg_handle* h, int nl, const double* const* f, double* const* u);
// (adds the pending PCG steps to the iterates first)
void multi_true_residuals(gmg_handle* h, int nl, const double* const* f, double* const* u);
void multi_cast(gmg_handle* h, int nl, const double* const* f, const bool* cold);
void multi_true_residual(gmg_handle* h, int l, const double* f, const double* u, bool into_r);
// Per-load loop scalars (iteration count 0, tolerance, cap, ||f||, active flag) of all 16 slots.
void multi_set_loop_scalars(gmg_handle* h, int nl, double tol, int maxit, const double* nf, const bool* active);
void multi_publish(gmg_handle* h);
// Changes whenever some handle's multi-load level-0 operator is switched (a
// captured batch graph records the value it was built under).
unsigned multi_generation();
bool multi_capture_loop(gmg_handle* h, double* const* u, int nl, cudaGraph_t g, cudaStream_t cap,
                        unsigned long long& prefix, unsigned long long& body_k);

}  // namespace gmg
