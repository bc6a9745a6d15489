// Multi-load solve: up to 16 right-hand sides on one hierarchy (the batching
// line: many loads on one density field share every operator byte, mask and
// modulus, and one launch of each kernel serves all of them).
//
// Every level's vectors hold the loads side by side, 16-byte records
// (u_x, u_y, u_z, 0) per (node, load), 256 bytes per node (internal.cuh).  The
// V-cycle (Eq. vcycle), the smoothers (Algorithm cheb, damped Jacobi), the
// transfers (Eq. vector_prolongation) and the outer PCG (Sec. "Outer Krylov
// Solver and Convergence Statement") are those of the single-load path, with
// per-load step lengths alpha_l, directions beta_l and stopping decisions: a
// load whose recursive residual passes the tolerance (or that reaches the cap,
// or turns non-finite) stops updating its iterate, residual and direction,
// exactly where the single-load loop would have left; the loop runs while any
// load iterates.  Kernels read the per-load scalars from a [16][SC_COUNT]
// block; the loads are independent in every kernel (no arithmetic mixes them).
//
// Levels >= 1 apply the stored Galerkin operator once per node for all loads
// (the 126 operator planes are read once, not once per load); the coarsest
// level applies its FP64 Cholesky-derived inverse split into FP32 hi + lo parts
// with double-float accumulation (FP64-class accuracy on the FP32 pipes, which
// issue many times faster than FP64 on this part).  Level 0 runs the TMA-fed
// z-marching operator of fine.cu, one block per (tile, load), or the tensor-core
// element contraction (multi_tc.cu).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int kMT = 256;              // threads of the multi-load vector kernels
constexpr int kMBlocks = 148 * 4;     // their fixed grid (grid-stride loops)

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

// Per-load block sums.  In the grid-stride record kernels every stride is a
// multiple of 16, so a thread always sees the load threadIdx.x % 16; the sum
// of load l over the block is written by thread l (fixed order: lanes l and
// l + 16, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum_load(double v, int tid) {
    __shared__ double red[NT / 32][kLoads];
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    if ((tid & 31) < kLoads) red[tid >> 5][tid & 31] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < kLoads) {
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += red[w][tid];
    }
    return s;
}

template <int NTH>
__device__ __forceinline__ double block_sum_all(double v, int tid) {
    __shared__ double warp_part[NTH / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) warp_part[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int w = 0; w < NTH / 32; ++w) s += warp_part[w];
    }
    return s;
}

struct F64In { const double* p[kLoads]; };
struct F64Out { double* p[kLoads]; };
struct F32In { const float* p[kLoads]; };
struct F32Out { float* p[kLoads]; };

// ---- level-0 packing ----------------------------------------------------------
// r(l) = f_l on free DOFs (FP32), 0 on fixed DOFs, pads and loads without f.
__global__ void __launch_bounds__(kMT) k_mcast(const __grid_constant__ F64In f, int nl, const uint8_t* maskp, int NX, int px, long long nnp,
                                               float* r) {
    pdl_entry();
    const long long nrec = nnp * kLoads;
    for (long long q = blockIdx.x * (long long)kMT + threadIdx.x; q < nrec; q += (long long)gridDim.x * kMT) {
        const long long n = q >> 4;
        const int l = (int)(q & 15);
        const long long row = n / px;
        const int i = (int)(n - row * px);
        float v[3] = {0.f, 0.f, 0.f};
        if (l < nl && i < NX && f.p[l]) {
            const uint8_t m = maskp[n];
            const double* src = f.p[l] + 3 * (row * NX + i);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = fixed_bit(m, c) ? 0.f : (float)src[c];
        }
        reinterpret_cast<float4*>(r)[q] = make_float4(v[0], v[1], v[2], 0.f);
    }
}

// Per load: fixed DOFs of u_l to 0, the nonzero count of u_l (partial) and
// ||f_l||^2 over the free DOFs (partial2), in the dense numbering.  A block of
// 16 warps takes 32 consecutive nodes, warp l load l.
__global__ void __launch_bounds__(32 * kLoads) k_mnorms(const __grid_constant__ F64Out u,
                                                       const __grid_constant__ F64In f, int nl, const uint8_t* mask,
                                                       long long nn, double* partial, double* partial2, int pstride) {
    pdl_entry();
    const int l = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double cnt = 0.0, ff = 0.0;
    if (l < nl) {
        double* ul = u.p[l];
        const double* fl = f.p[l];
        for (long long n = blockIdx.x * 32LL + lane; n < nn; n += (long long)gridDim.x * 32) {
            const uint8_t m = mask[n];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (fixed_bit(m, c)) {
                    ul[3 * n + c] = 0.0;
                } else {
                    if (ul[3 * n + c] != 0.0) cnt += 1.0;
                    const double fv = fl[3 * n + c];
                    ff += fv * fv;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        ff += __shfl_down_sync(0xffffffffu, ff, o);
    }
    if (lane == 0) {
        partial[(long long)l * pstride + blockIdx.x] = cnt;
        partial2[(long long)l * pstride + blockIdx.x] = ff;
    }
}

// Slot l of a multi-load vector from a single-load level-0 vector (padded rows).
__global__ void k_mpack_slot(const float* v, long long nnp, int l, float* mv) {
    pdl_entry();
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nnp; n += (long long)gridDim.x * blockDim.x)
        reinterpret_cast<float4*>(mv)[n * kLoads + l] = make_float4(v[3 * n], v[3 * n + 1], v[3 * n + 2], 0.f);
}

// Multi-load level-0 vector from per-load dense FP32 vectors (fixed DOFs and
// pads 0; loads >= nl 0), and back.
__global__ void k_mpack_dense(const __grid_constant__ F32In in, int nl, const uint8_t* maskp, int NX, int px, long long nnp, float* mv) {
    pdl_entry();
    const long long nrec = nnp * kLoads;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nrec; q += (long long)gridDim.x * blockDim.x) {
        const long long n = q >> 4;
        const int l = (int)(q & 15);
        const long long row = n / px;
        const int i = (int)(n - row * px);
        float v[3] = {0.f, 0.f, 0.f};
        if (l < nl && i < NX) {
            const uint8_t m = maskp[n];
            const float* src = in.p[l] + 3 * (row * NX + i);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = fixed_bit(m, c) ? 0.f : src[c];
        }
        reinterpret_cast<float4*>(mv)[q] = make_float4(v[0], v[1], v[2], 0.f);
    }
}

__global__ void k_munpack_dense(const float* mv, int nl, int NX, int px, long long nn, const __grid_constant__ F32Out out) {
    pdl_entry();
    const long long nrec = nn * nl;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nrec; q += (long long)gridDim.x * blockDim.x) {
        const long long dn = q / nl;
        const int l = (int)(q - dn * nl);
        const long long row = dn / NX;
        const long long n = dn + row * (px - NX);
        const float4 v = reinterpret_cast<const float4*>(mv)[n * kLoads + l];
        float* o = out.p[l] + 3 * dn;
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
    }
}

// ---- PCG scalars --------------------------------------------------------------
// sc(l)[slot] = sum of partial[l * pstride + 0 .. n), then the operation of
// k_finalize (hot.cu) on load l's scalars.  One block per load.
__global__ void __launch_bounds__(kMT) k_mfinalize(const double* partial, int n, int pstride, double* sc, int slot,
                                                   int op) {
    pdl_entry();
    const int l = blockIdx.x;
    const double* pp = partial + (long long)l * pstride;
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += kMT) s += pp[q];
    s = block_sum_all<kMT>(s, threadIdx.x);
    if (threadIdx.x == 0) {
        double* c = sc + l * SC_COUNT;
        c[slot] = s;
        if (op == FIN_ALPHA) {
            c[SC_ALPHA] = c[SC_RZ] / s;
        } else if (op == FIN_BETA) {
            c[SC_BETA] = s / c[SC_RZ];
            c[SC_RZ] = s;
        }
    }
}

// ||r_l||^2 and the per-load convergence test of the device-resident loop
// (k_finalize_check for each load still iterating); the while condition
// (set_cond; the host-driven loop reads the active flags instead) is set while
// any load iterates.  One block, warp l takes load l.
__global__ void __launch_bounds__(32 * kLoads) k_mfinalize_check(const double* partial, int n, int pstride, double* sc,
                                                                 cudaGraphConditionalHandle cond, int set_cond) {
    pdl_entry();
    __shared__ int go_any[kLoads];
    const int l = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* pp = partial + (long long)l * pstride;
    double s = 0.0;
    for (int q = lane; q < n; q += 32) s += pp[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double* c = sc + l * SC_COUNT;
        int go = 0;
        if (c[SC_ACT] != 0.0) {
            c[SC_RR] = s;
            const double k = c[SC_IT] + 1.0;
            c[SC_IT] = k;
            const double relr = sqrt(s) / c[SC_NF];
            go = isfinite(relr) && isfinite(c[SC_ALPHA]) && !(relr < c[SC_TOL]) && k < c[SC_MAXIT];
            if (!go) c[SC_ACT] = 0.0;
        }
        go_any[l] = go;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
#pragma unroll
        for (int q = 0; q < kLoads; ++q) any |= go_any[q];
        if (set_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
}

// w_l += alpha_l p (the double-float correction of load l's FP64 iterate,
// dense numbering), r -= alpha_l q, partial ||r_l||^2, for the loads still
// iterating (the others keep their values).  The product by the FP64 alpha is
// formed exactly as ah p + (al p + e) and added with a TwoSum, on the FP32
// pipes (the FP64 pipe, a small fraction of the FP32 rate on this part, bound
// the FP64 update).  A block of 16 warps takes 32 consecutive nodes, warp l
// load l: a load's correction is read and written in 768-byte runs, and the
// records of a node's 16 loads are read by the 16 warps of the same block.
constexpr int kPcgThreads = 32 * kLoads;
__device__ __forceinline__ float2 df_add_prod(float2 w, float ah, float al, float p) {
    const float ph = __fmul_rn(ah, p);
    const float pl = __fmaf_rn(al, p, __fmaf_rn(ah, p, -ph));
    const float s = __fadd_rn(w.x, ph);
    const float bb = __fsub_rn(s, w.x);
    const float e = __fadd_rn(__fsub_rn(w.x, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
    const float lo = __fadd_rn(w.y, __fadd_rn(pl, e));
    const float hi = __fadd_rn(s, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}
__global__ void __launch_bounds__(kPcgThreads) k_mpcg_update(float2* wcor, long long n3, int nl, float* r,
                                                             const float* p, const float* q, int NX, int px,
                                                             long long nnp, const double* sc, double* partial,
                                                             int pstride) {
    pdl_entry();
    const int l = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* c = sc + l * SC_COUNT;
    const bool act = l < nl && c[SC_ACT] != 0.0;
    DSAcc acc;
    if (act) {
        const double alpha = c[SC_ALPHA];
        const float af = (float)alpha;
        const float ah = af, al = (float)(alpha - (double)ah);
        float2* wl = wcor + (long long)l * n3;
        for (long long n = blockIdx.x * 32LL + lane; n < nnp; n += (long long)gridDim.x * 32) {
            const long long row = n / px;
            const int i = (int)(n - row * px);
            if (i >= NX) continue;  // pad node: stays 0
            const long long qi = n * kLoads + l;
            const float4 pv = reinterpret_cast<const float4*>(p)[qi];
            const float4 qv = reinterpret_cast<const float4*>(q)[qi];
            float4 rv = reinterpret_cast<float4*>(r)[qi];
            float2* wd = wl + GMG_B(3 * (row * NX + i), n3 - 2, 501);
            wd[0] = df_add_prod(wd[0], ah, al, pv.x);
            wd[1] = df_add_prod(wd[1], ah, al, pv.y);
            wd[2] = df_add_prod(wd[2], ah, al, pv.z);
            rv.x = fmaf(-af, qv.x, rv.x);
            rv.y = fmaf(-af, qv.y, rv.y);
            rv.z = fmaf(-af, qv.z, rv.z);
            acc.add_prod(rv.x, rv.x);
            acc.add_prod(rv.y, rv.y);
            acc.add_prod(rv.z, rv.z);
            reinterpret_cast<float4*>(r)[qi] = rv;
        }
    }
    double v = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partial[(long long)l * pstride + blockIdx.x] = v;
}

// u_l += w_l (FP64), then w_l = 0, for loads 0..nl-1.
__global__ void k_mflush(const __grid_constant__ F64Out u, int nl, float2* wcor, long long n3) {
    pdl_entry();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nl * n3;
         q += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(q / n3);
        const long long i = q - l * n3;
        const float2 w = wcor[q];
        u.p[l][i] = u.p[l][i] + (f2d_exact(w.x) + f2d_exact(w.y));
        wcor[q] = make_float2(0.f, 0.f);
    }
}

// p = z + beta_l p for the loads still iterating.
__global__ void __launch_bounds__(kMT) k_mp_update(float* p, const float* z, long long nrec, const double* sc) {
    pdl_entry();
    const int l = threadIdx.x & 15;
    const double* c = sc + l * SC_COUNT;
    if (c[SC_ACT] == 0.0) return;
    const float beta = (float)c[SC_BETA];
    for (long long q = blockIdx.x * (long long)kMT + threadIdx.x; q < nrec; q += (long long)gridDim.x * kMT) {
        float4 v = reinterpret_cast<float4*>(p)[q];
        const float4 w = reinterpret_cast<const float4*>(z)[q];
        v.x = fmaf(beta, v.x, w.x);
        v.y = fmaf(beta, v.y, w.y);
        v.z = fmaf(beta, v.z, w.z);
        reinterpret_cast<float4*>(p)[q] = v;
    }
}

// Loop scalars of the 16 load slots: iteration count 0, tolerance, cap, ||f||
// and the active flag.
struct LoopScalars {
    double nf[kLoads];
    double act[kLoads];
    double tol, maxit;
};
__global__ void k_mset_loop(double* sc, LoopScalars v) {
    const int l = threadIdx.x;
    if (l >= kLoads) return;
    double* c = sc + l * SC_COUNT;
    c[SC_IT] = 0.0;
    c[SC_TOL] = v.tol;
    c[SC_MAXIT] = v.maxit;
    c[SC_NF] = v.nf[l];
    c[SC_ACT] = v.act[l];
    // every later residual of an iterating load sees u != 0 (the PCG updates)
    if (v.act[l] != 0.0) c[SC_UNZ] = 1.0;
}

// ---- level 0: first smoother step from zero: x = c_a D^-1 b (d = x) -----------
__global__ void __launch_bounds__(kMT) k_mfine_smooth0(const float* b, const float* inv0, const uint8_t* maskp,
                                                       long long nnp, const double* coef, float* out, float* dnew) {
    pdl_entry();
    const float ca = (float)coef[1];
    const long long nrec = nnp * kLoads;
    for (long long q = blockIdx.x * (long long)kMT + threadIdx.x; q < nrec; q += (long long)gridDim.x * kMT) {
        const long long n = q >> 4;
        const float inv = inv0[n];
        const uint8_t m = maskp[n];
        const float4 bv = reinterpret_cast<const float4*>(b)[q];
        const float4 v = make_float4(fixed_bit(m, 0) ? 0.f : ca * inv * bv.x, fixed_bit(m, 1) ? 0.f : ca * inv * bv.y,
                                     fixed_bit(m, 2) ? 0.f : ca * inv * bv.z, 0.f);
        reinterpret_cast<float4*>(out)[q] = v;
        if (dnew) reinterpret_cast<float4*>(dnew)[q] = v;
    }
}

// ---- assembled levels ----------------------------------------------------------
struct MBsrArgs {
    int nx, ny, nz;
    int nn;
    long long ps;
    const float* A;          // symmetric half storage (hot.cu): diagonal + 13 forward blocks, plane-major
    const float* invdiag;
    const uint8_t* mask;
    const float* xin;
    const float* b;
    const float* dold;
    float* dnew;
    float* out;
    const double* coef;
    int step;
};

// y = K^l x on multi-load vectors.  16 / LQ threads share a node, each taking
// LQ of its loads: the node's operator blocks are read once per thread (the
// reads of a node's threads hit the same L1 line) and applied to the thread's
// LQ records of each neighbour (same branch-free neighbour handling as k_bsr:
// clamped indices, zero-stored forward blocks outside the grid, backward terms
// scaled by 0 outside it).
template <int MODE, int kBsrLq>
__global__ void __launch_bounds__(128) k_mbsr(MBsrArgs a) {
    pdl_entry();
    constexpr int TPN = kLoads / kBsrLq;  // threads per node
    const long long t = blockIdx.x * 128LL + threadIdx.x;
    const int n = (int)(t / TPN), g = (int)(t % TPN);
    if (n >= a.nn) return;
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
    const long long N = a.ps;
    const float4* X = reinterpret_cast<const float4*>(a.xin) + kBsrLq * g;
    float y[kBsrLq][3];
#pragma unroll
    for (int l = 0; l < kBsrLq; ++l) y[l][0] = y[l][1] = y[l][2] = 0.f;
#pragma unroll
    for (int u = 0; u < 14; ++u) {
        const int sl = 13 + u;
        const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
        const int off = dx + NX * (dy + NY * dz);
        const bool okf = i + dx >= 0 && i + dx < NX && j + dy >= 0 && j + dy < NY && k + dz < NZ;
        const int mf = (int)GMG_B(okf ? n + off : n, a.nn, 511);
        const float* Ap = a.A + (long long)(u * 9) * N + n;
        float A[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) A[e] = __ldg(Ap + e * N);
        const float4* xf = X + (long long)mf * kLoads;
#pragma unroll
        for (int l = 0; l < kBsrLq; ++l) {
            const float4 v = __ldg(xf + l);
            y[l][0] = fmaf(A[0], v.x, fmaf(A[1], v.y, fmaf(A[2], v.z, y[l][0])));
            y[l][1] = fmaf(A[3], v.x, fmaf(A[4], v.y, fmaf(A[5], v.z, y[l][1])));
            y[l][2] = fmaf(A[6], v.x, fmaf(A[7], v.y, fmaf(A[8], v.z, y[l][2])));
        }
        if (u > 0) {
            const bool okb = i - dx >= 0 && i - dx < NX && j - dy >= 0 && j - dy < NY && k - dz >= 0;
            const int mb = (int)GMG_B(okb ? n - off : n, a.nn, 512);
            const float wgt = okb ? 1.f : 0.f;
            const float* Bp = a.A + (long long)(u * 9) * N + mb;
            float B[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) B[e] = wgt * __ldg(Bp + e * N);
            const float4* xb = X + (long long)mb * kLoads;
#pragma unroll
            for (int l = 0; l < kBsrLq; ++l) {
                const float4 w = __ldg(xb + l);
                y[l][0] = fmaf(B[0], w.x, fmaf(B[3], w.y, fmaf(B[6], w.z, y[l][0])));
                y[l][1] = fmaf(B[1], w.x, fmaf(B[4], w.y, fmaf(B[7], w.z, y[l][1])));
                y[l][2] = fmaf(B[2], w.x, fmaf(B[5], w.y, fmaf(B[8], w.z, y[l][2])));
            }
        }
    }
    const uint8_t msk = a.mask[n];
    const bool f0 = !fixed_bit(msk, 0), f1 = !fixed_bit(msk, 1), f2 = !fixed_bit(msk, 2);
    const long long base = (long long)n * kLoads + kBsrLq * g;
    if (MODE == FM_APPLY) {
#pragma unroll
        for (int l = 0; l < kBsrLq; ++l)
            reinterpret_cast<float4*>(a.out)[base + l] =
                make_float4(f0 ? y[l][0] : 0.f, f1 ? y[l][1] : 0.f, f2 ? y[l][2] : 0.f, 0.f);
    } else if (MODE == FM_RESID) {
#pragma unroll
        for (int l = 0; l < kBsrLq; ++l) {
            const float4 bv = reinterpret_cast<const float4*>(a.b)[base + l];
            reinterpret_cast<float4*>(a.out)[base + l] = make_float4(
                f0 ? bv.x - y[l][0] : 0.f, f1 ? bv.y - y[l][1] : 0.f, f2 ? bv.z - y[l][2] : 0.f, 0.f);
        }
    } else {
        const float cd = (float)a.coef[2 * a.step], ca = (float)a.coef[2 * a.step + 1];
        const float i0 = a.invdiag[3 * n], i1 = a.invdiag[3 * n + 1], i2 = a.invdiag[3 * n + 2];
#pragma unroll
        for (int l = 0; l < kBsrLq; ++l) {
            const float4 bv = reinterpret_cast<const float4*>(a.b)[base + l];
            const float4 xv = reinterpret_cast<const float4*>(a.xin)[base + l];
            float d0 = ca * i0 * (bv.x - y[l][0]), d1 = ca * i1 * (bv.y - y[l][1]), d2 = ca * i2 * (bv.z - y[l][2]);
            if (cd != 0.f) {
                const float4 dv = reinterpret_cast<const float4*>(a.dold)[base + l];
                d0 = fmaf(cd, dv.x, d0);
                d1 = fmaf(cd, dv.y, d1);
                d2 = fmaf(cd, dv.z, d2);
            }
            d0 = f0 ? d0 : 0.f;
            d1 = f1 ? d1 : 0.f;
            d2 = f2 ? d2 : 0.f;
            reinterpret_cast<float4*>(a.out)[base + l] =
                make_float4(f0 ? xv.x + d0 : 0.f, f1 ? xv.y + d1 : 0.f, f2 ? xv.z + d2 : 0.f, 0.f);
            if (a.dnew) reinterpret_cast<float4*>(a.dnew)[base + l] = make_float4(d0, d1, d2, 0.f);
        }
    }
}

__global__ void __launch_bounds__(kMT) k_mbsr_smooth0(MBsrArgs a) {
    pdl_entry();
    const float ca = (float)a.coef[1];
    const long long nrec = (long long)a.nn * kLoads;
    for (long long q = blockIdx.x * (long long)kMT + threadIdx.x; q < nrec; q += (long long)gridDim.x * kMT) {
        const long long n = q >> 4;
        const float4 bv = reinterpret_cast<const float4*>(a.b)[q];
        // invdiag is 0 on fixed DOFs
        const float4 v = make_float4(ca * a.invdiag[3 * n] * bv.x, ca * a.invdiag[3 * n + 1] * bv.y,
                                     ca * a.invdiag[3 * n + 2] * bv.z, 0.f);
        reinterpret_cast<float4*>(a.out)[q] = v;
        if (a.dnew) reinterpret_cast<float4*>(a.dnew)[q] = v;
    }
}

// ---- transfers (Eq. vector_prolongation; weights as hot.cu) ----------------------
__device__ __forceinline__ void msupport3(int I, int nf, int idx[3], float w[3]) {
    const int nc = nf >> 1, f = 2 * I + 1;
    idx[0] = I >= 1 ? 2 * I - 1 : 2 * I; w[0] = I >= 1 ? 0.5f : 0.f;
    idx[1] = 2 * I; w[1] = 1.f;
    idx[2] = f <= nf ? f : 2 * I; w[2] = f <= nf ? (f < 2 * nc ? 0.5f : 1.f) : 0.f;
}

__device__ __forceinline__ void mparents2(int f, int nf, int idx[2], float w[2]) {
    const int nc = nf >> 1;
    if ((f & 1) == 0) { idx[0] = idx[1] = f >> 1; w[0] = 1.f; w[1] = 0.f; }
    else if (f < 2 * nc) { idx[0] = (f - 1) >> 1; idx[1] = (f + 1) >> 1; w[0] = w[1] = 0.5f; }
    else { idx[0] = idx[1] = nc; w[0] = 1.f; w[1] = 0.f; }
}

// coarse(n, l) = P^T fine at coarse node n, load l (masked): one thread per record.
__global__ void __launch_bounds__(kMT) k_mrestrict(int fnx, int fny, int fnz, int fpx, int cnx, int cny, int cnz,
                                                   const uint8_t* cmask, const float* fine, float* coarse) {
    pdl_entry();
    const int CX = cnx + 1, CY = cny + 1;
    const long long nrec = (long long)CX * CY * (cnz + 1) * kLoads;
    const long long q = blockIdx.x * (long long)kMT + threadIdx.x;
    if (q >= nrec) return;
    const int n = (int)(q >> 4), l = (int)(q & 15);
    const int FX = fpx, FY = fny + 1;
    const int I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    msupport3(I, fnx, ix, wx);
    msupport3(J, fny, iy, wy);
    msupport3(K, fnz, iz, wz);
    const float4* F = reinterpret_cast<const float4*>(fine);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float w = wx[a] * wy[b] * wz[c];
                const long long f = GMG_B(ix[a] + (long long)FX * (iy[b] + FY * iz[c]), (long long)FX * FY * (fnz + 1), 521);
                const float4 v = F[f * kLoads + l];
                s0 = fmaf(w, v.x, s0);
                s1 = fmaf(w, v.y, s1);
                s2 = fmaf(w, v.z, s2);
            }
    const uint8_t m = cmask[n];
    reinterpret_cast<float4*>(coarse)[q] =
        make_float4(fixed_bit(m, 0) ? 0.f : s0, fixed_bit(m, 1) ? 0.f : s1, fixed_bit(m, 2) ? 0.f : s2, 0.f);
}

// fine(n, l) += P coarse on the free DOFs of fine node n: one thread per record.
__global__ void __launch_bounds__(kMT) k_mprolong_add(int fnx, int fny, int fnz, int fpx, int cnx, int cny,
                                                      const uint8_t* fmask, const float* coarse, float* fine) {
    pdl_entry();
    const int FX = fnx + 1, FY = fny + 1;
    const long long nrec = (long long)FX * FY * (fnz + 1) * kLoads;
    const long long q = blockIdx.x * (long long)kMT + threadIdx.x;
    if (q >= nrec) return;
    const int n = (int)(q >> 4), l = (int)(q & 15);
    const int CX = cnx + 1, CY = cny + 1;
    const int i = n % FX, j = (n / FX) % FY, k = n / (FX * FY);
    int ix[2], iy[2], iz[2];
    float wx[2], wy[2], wz[2];
    mparents2(i, fnx, ix, wx);
    mparents2(j, fny, iy, wy);
    mparents2(k, fnz, iz, wz);
    const float4* C = reinterpret_cast<const float4*>(coarse);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float w = wx[a] * wy[b] * wz[c];
                const long long m = GMG_B(ix[a] + (long long)CX * (iy[b] + CY * iz[c]), (long long)CX * CY * (fnz / 2 + 1), 522);
                const float4 v = C[m * kLoads + l];
                s0 = fmaf(w, v.x, s0);
                s1 = fmaf(w, v.y, s1);
                s2 = fmaf(w, v.z, s2);
            }
    const uint8_t msk = fmask[n];
    const long long np = GMG_B(i + (long long)fpx * (j + FY * k), (long long)fpx * FY * (fnz + 1), 523);
    float4* o = reinterpret_cast<float4*>(fine) + np * kLoads + l;
    float4 v = *o;
    if (!fixed_bit(msk, 0)) v.x += s0;
    if (!fixed_bit(msk, 1)) v.y += s1;
    if (!fixed_bit(msk, 2)) v.z += s2;
    *o = v;
}

// ---- coarsest level: x(l) = Ainv b(l) on the free DOFs, 0 on fixed ones ---------
// k_mcoarse_gather packs the free entries of b as bc[j][l] (and zeroes the
// fixed DOFs of x); k_mcoarse then forms x = Ainv bc with Ainv = Ahi + Alo
// (FP32 parts of the FP64 inverse): each product is split exactly with an FMA
// and summed in double-float, so a row's sum carries ~44 significant bits.  A
// block takes 4 rows x 16 loads, each row's sum split over 4 interleaved
// column slices that are added in a fixed order at the end.
__global__ void __launch_bounds__(256) k_mcoarse_gather(int nL, const int* free_idx, const float* b, float* bc,
                                                        float* x, const uint8_t* mask, int n_nodes) {
    pdl_entry();
    const long long stride = (long long)gridDim.x * 256;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < 3LL * n_nodes * kLoads; q += stride) {
        const long long rec = q / 3;
        const int c = (int)(q - rec * 3);
        if (fixed_bit(mask[rec >> 4], c)) x[rec * 4 + c] = 0.f;
    }
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < (long long)nL * kLoads; q += stride) {
        const int jj = (int)(q >> 4), ll = (int)(q & 15);
        const int dof = free_idx[jj];
        const int node = dof / 3, c = dof - 3 * (dof / 3);
        bc[q] = b[GMG_B(((long long)node * kLoads + ll) * 4 + c, (long long)n_nodes * kNodeF, 531)];
    }
}

constexpr int kCoarseRows = 4, kCoarseSlices = 4;
static_assert(kCoarseRows * kCoarseSlices * kLoads == 256, "one block of 256 threads");
__global__ void __launch_bounds__(256) k_mcoarse(int nL, const int* free_idx, const float* Ahi, const float* Alo,
                                                 const float* bc, float* x, int n_nodes) {
    pdl_entry();
    __shared__ double part[kCoarseRows][kCoarseSlices][kLoads];
    const int tid = threadIdx.x, l = tid & 15, sl = (tid >> 4) % kCoarseSlices, rr = (tid >> 4) / kCoarseSlices;
    const int row = blockIdx.x * kCoarseRows + rr;
    float hi = 0.f, lo = 0.f;
    if (row < nL) {
        const float* ah = Ahi + (long long)row * nL;
        const float* al = Alo + (long long)row * nL;
        for (int j = sl; j < nL; j += kCoarseSlices) {
            const float a = __ldg(ah + j), a2 = __ldg(al + j), bv = __ldg(bc + (long long)j * kLoads + l);
            const float p = a * bv;
            const float e = fmaf(a, bv, -p);
            const float s = hi + p;
            const float bb = s - hi;
            const float t = (hi - (s - bb)) + (p - bb);
            hi = s;
            lo += t + fmaf(a2, bv, e);
        }
    }
    part[rr][sl][l] = (double)hi + (double)lo;
    __syncthreads();
    if (sl == 0 && row < nL) {
        double v = part[rr][0][l];
#pragma unroll
        for (int k = 1; k < kCoarseSlices; ++k) v += part[rr][k][l];
        const int dof = free_idx[row];
        const int node = dof / 3, c = dof - 3 * (dof / 3);
        x[GMG_B(((long long)node * kLoads + l) * 4 + c, (long long)n_nodes * kNodeF, 532)] = (float)v;
    }
}

__global__ void k_split_inverse(const double* A, long long n, float* hi, float* lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = A[i];
        const float h = (float)v;
        hi[i] = h;
        lo[i] = (float)(v - (double)h);
    }
}

// ---- level 0: TMA-fed z-marching operator, one block per (tile, load) ------------
// The element arithmetic, schedule and epilogues are those of k_fine_tma
// (fine.cu): the Hadamard form of K_e (G in its symmetric form), a (BX-1) x
// (BY-1) node patch per block marching along z, the stages of a 4-slot ring
// filled by TMA on mbarriers.  Here a node plane of one load is a box of
// 16-byte records (x, y, z, 0) strided 256 bytes apart in the multi-load
// vector (4-D tensor map: 64 floats of a node, x, y, z), so the staged plane
// holds 4 floats per node and a corner is one 16-byte shared-memory load.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
          "r"(smem_u32(bar))
        : "memory");
}

__host__ __device__ constexpr int mround4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int mround128(int v) { return (v + 127) / 128 * 128; }

template <int BX, int BY>
struct MTile {
    static constexpr int XN = BX + 1;                    // staged nodes per row
    static constexpr int XR = BY + 1;                    // staged node rows
    static constexpr int EW = mround4(BX + 3);           // moduli per staged row
    static constexpr int ER = BY;
    static constexpr int ON = BX - 1, OR = BY - 1;       // owned nodes
    static constexpr int XB = XN * XR * 16, EB = EW * ER * 4, OB = ON * OR * 16;
    static constexpr int XOFF = 0;
    static constexpr int EOFF = mround128(XB);
    static constexpr int BOFF = EOFF + mround128(EB);
    static constexpr int DOFF = BOFF + mround128(OB);
    static constexpr int STAGE = DOFF + mround128(OB);
    static constexpr int SXOFF = 4 * STAGE;              // y-exchange [2][BY + 1][BX] float4
    static constexpr int BAROFF = SXOFF + 2 * (BY + 1) * BX * 16;
    static constexpr int SMEM = BAROFF + 4 * 8;
};

constexpr unsigned kMTmaSpin = 1u << 22;

struct MV3 {
    float2 xy;
    float z;
};
__device__ __forceinline__ MV3 madd(const MV3& a, const MV3& b) { return {__fadd2_rn(a.xy, b.xy), __fadd_rn(a.z, b.z)}; }
__device__ __forceinline__ MV3 msub(const MV3& a, const MV3& b) {
    return {__ffma2_rn(b.xy, make_float2(-1.f, -1.f), a.xy), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ MV3 mld4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), v.z};
}
__device__ __forceinline__ float mcomp(const MV3& v, int c) { return c == 0 ? v.xy.x : (c == 1 ? v.xy.y : v.z); }
__device__ __forceinline__ void mface_diffs(const MV3 c[4], MV3 q[4]) {
    const MV3 dx0 = msub(c[1], c[0]), dx1 = msub(c[3], c[2]);
    q[1] = madd(dx0, dx1);
    q[2] = madd(msub(c[2], c[0]), msub(c[3], c[1]));
    q[3] = msub(dx1, dx0);
}
struct MLayer {
    MV3 C[4];
    MV3 Q[4];
    MV3 T[4];
    float E;
};

}  // namespace

namespace {

template <int BX, int BY, int MODE, bool DOT>
__global__ void __launch_bounds__(BX * BY, 2)
k_mfine(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tme,
        const __grid_constant__ CUtensorMap tmb, const __grid_constant__ CUtensorMap tmd, MFineArgs a, GSym G,
        int zchunk, int gx, int gy) {
    using T = MTile<BX, BY>;
    constexpr int NT = BX * BY;
    constexpr bool EPI_B = MODE != FM_APPLY;
    constexpr bool EPI_D = MODE == FM_SMOOTH;
    extern __shared__ __align__(128) unsigned char smem[];
    float4(*sx)[BY + 1][BX] = reinterpret_cast<float4(*)[BY + 1][BX]>(smem + T::SXOFF);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + T::BAROFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int px = a.px, NXYp = px * NY;
    const int l = (int)(blockIdx.x % (unsigned)a.nl);
    const int tile = (int)(blockIdx.x / (unsigned)a.nl);
    const int bxi = tile % gx, byi = (tile / gx) % gy, bzi = tile / (gx * gy);
    const int x0 = bxi * (BX - 1), y0 = byi * (BY - 1);
    const int k0 = bzi * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;
    const int es = (x0 - 1) & ~3;                    // moduli box origin, rounded down to 4
    const int rx = (ty * T::XN + tx) * 4;            // this column's low corner in a node plane
    const int re = ty * T::EW + tx + (x0 - 1 - es);  // this column's modulus in a layer
    const int rb = (ty * T::ON + tx) * 4;            // this owner's record in an epilogue plane
    const int ox = x0 + tx, oy = y0 + ty;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const int onode = oy * px + ox;
    const float cd = EPI_D ? (float)a.coef[2 * a.step] : 0.f;
    const float ca = EPI_D ? (float)a.coef[2 * a.step + 1] : 0.f;
    const bool need_d = EPI_D && cd != 0.f;
    const unsigned epi_bytes = EPI_B ? (unsigned)T::OB * (need_d ? 2u : 1u) : 0u;

    if ((smem_u32(smem) & 127) != 0) {
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) mbar_init(&full[q], 1);
        mbar_fence_init();
    }
    __syncthreads();
    pdl_entry();

    int issued[4] = {0, 0, 0, 0};
    auto issue = [&](int s) {
        const int q = (s - kb) & 3;
        unsigned char* st = smem + q * T::STAGE;
        const bool xe = s < k1;
        const bool ep = EPI_B && s > k0;
        const unsigned bytes = (xe ? (unsigned)(T::XB + T::EB) : 0u) + (ep ? epi_bytes : 0u);
        if (bytes == 0) return;
        ++issued[q];
        mbar_expect_tx(&full[q], bytes);
        if (xe) {
            tma_load_4d(st + T::XOFF, &tmx, 4 * l, x0 - 1, y0 - 1, s + 1, &full[q]);
            tma_load_3d(st + T::EOFF, &tme, es, y0 - 1, s, &full[q]);
        }
        if (ep) {
            tma_load_4d(st + T::BOFF, &tmb, 4 * l, x0, y0, s - 1, &full[q]);
            if (need_d) tma_load_4d(st + T::DOFF, &tmd, 4 * l, x0, y0, s - 1, &full[q]);
        }
    };
    auto wait_full = [&](int q, unsigned parity) -> bool {
        for (unsigned it = 0; it < kMTmaSpin; ++it)
            if (mbar_try_wait(&full[q], parity)) return true;
        return false;
    };
    auto load_mask = [&](int kp) -> int {
        return (owner && kp >= k0 && kp < k1) ? (int)a.maskp[GMG_B(onode + kp * NXYp, (long long)NXYp * NZ, 541)] : 7;
    };

    if (tid == 0) {
        issued[3] = 1;
        mbar_expect_tx(&full[3], (unsigned)T::XB);
        tma_load_4d(smem + 3 * T::STAGE + T::XOFF, &tmx, 4 * l, x0 - 1, y0 - 1, kb, &full[3]);
        issue(kb);
        if (kb + 1 <= k1) issue(kb + 1);
        if (kb + 2 <= k1) issue(kb + 2);
    }
    bool failed = !wait_full(3, 0);
    MLayer s0, s1;
    {
        const float* pl = reinterpret_cast<const float*>(smem + 3 * T::STAGE + T::XOFF) + rx;
        s0.C[0] = mld4(pl);
        s0.C[1] = mld4(pl + 4);
        s0.C[2] = mld4(pl + 4 * T::XN);
        s0.C[3] = mld4(pl + 4 * T::XN + 4);
        mface_diffs(s0.C, s0.Q);
#pragma unroll
        for (int q = 0; q < 4; ++q) s0.T[q] = MV3{make_float2(0.f, 0.f), 0.f};
        s0.E = 0.f;
    }
    // masks four planes ahead, one register per ring slot (the slot of step s
    // holds plane s's mask), so a load's result is not touched before its use
    int mq[4] = {7, load_mask(k0), load_mask(k0 + 1), load_mask(k0 + 2)};
    bool pending = false;
    MV3 R1{make_float2(0.f, 0.f), 0.f}, un_pend{make_float2(0.f, 0.f), 0.f};
    float eR1 = 0.f;
    int m_pend = 7;
    DSAcc dotv;

    auto finish = [&](int kp, int q) {
        const float4 up = sx[kp & 1][ty + 1][tx];
        const float y[3] = {__fadd_rn(R1.xy.x, up.x), __fadd_rn(R1.xy.y, up.y), __fadd_rn(R1.z, up.z)};
        const long long rec =
            owner ? GMG_B(((long long)(onode + kp * NXYp)) * kLoads + l, (long long)NXYp * NZ * kLoads, 542) : 0;
        float4* out = reinterpret_cast<float4*>(a.out) + rec;
        bool fr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) fr[c] = !((m_pend >> c) & 1);
        if (MODE == FM_APPLY) {
            float v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = fr[c] ? y[c] : 0.f;
                if (DOT) dotv.add_prod(fr[c] ? mcomp(un_pend, c) : 0.f, v[c]);
            }
            if (owner) *out = make_float4(v[0], v[1], v[2], 0.f);
        } else {
            const float* bb = reinterpret_cast<const float*>(smem + q * T::STAGE + T::BOFF) + rb;
            if (MODE == FM_RESID) {
                if (owner)
                    *out = make_float4(fr[0] ? __fsub_rn(bb[0], y[0]) : 0.f, fr[1] ? __fsub_rn(bb[1], y[1]) : 0.f,
                                       fr[2] ? __fsub_rn(bb[2], y[2]) : 0.f, 0.f);
            } else {
                const float* dd = reinterpret_cast<const float*>(smem + q * T::STAGE + T::DOFF) + rb;
                const float inv = jacobi_rcp(__fmul_rn(a.kd, __fadd_rn(eR1, up.w)));
                float xn[3], dn[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float d = __fmul_rn(__fmul_rn(ca, inv), __fsub_rn(bb[c], y[c]));
                    if (need_d) d = fmaf(cd, dd[c], d);
                    dn[c] = fr[c] ? d : 0.f;
                    xn[c] = fr[c] ? __fadd_rn(mcomp(un_pend, c), dn[c]) : 0.f;
                    if (DOT) dotv.add_prod(fr[c] ? bb[c] : 0.f, xn[c]);
                }
                if (owner) {
                    *out = make_float4(xn[0], xn[1], xn[2], 0.f);
                    if (a.dnew) reinterpret_cast<float4*>(a.dnew)[rec] = make_float4(dn[0], dn[1], dn[2], 0.f);
                }
            }
        }
    };

    auto step = [&](auto Qc, const int s, const unsigned par, const MLayer& in, MLayer& out) -> bool {
        constexpr int Q = decltype(Qc)::value;
        if (!wait_full(Q, par ^ (Q == 3 ? 1u : 0u))) failed = true;
        if (__syncthreads_or(failed)) return false;
        if (tid == 0 && s + 3 <= k1) issue(s + 3);
        if (pending) finish(s - 1, Q);
        pending = false;
        const int mcur = mq[Q];
        mq[Q] = load_mask(s + 4);
        {
            const float* pl = reinterpret_cast<const float*>(smem + Q * T::STAGE + T::XOFF) + rx;
            out.C[0] = mld4(pl);
            out.C[1] = mld4(pl + 4);
            out.C[2] = mld4(pl + 4 * T::XN);
            out.C[3] = mld4(pl + 4 * T::XN + 4);
            mface_diffs(out.C, out.Q);
        }
        out.E = reinterpret_cast<const float*>(smem + Q * T::STAGE + T::EOFF)[re];
        MV3 v[8];
        {
            const MV3 z00 = msub(out.C[0], in.C[0]), z10 = msub(out.C[1], in.C[1]);
            const MV3 z01 = msub(out.C[2], in.C[2]), z11 = msub(out.C[3], in.C[3]);
            v[4] = madd(madd(z00, z10), madd(z01, z11));
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                v[q] = madd(out.Q[q], in.Q[q]);
                v[q + 4] = msub(out.Q[q], in.Q[q]);
            }
        }
        MV3 w[8];
        w[0] = MV3{make_float2(0.f, 0.f), 0.f};
        {
            float u[8][3], o[8][3];
#pragma unroll
            for (int m = 1; m < 8; ++m) {
                u[m][0] = v[m].xy.x;
                u[m][1] = v[m].xy.y;
                u[m][2] = v[m].z;
            }
            gsym_contract(gsym_scale(G, out.E), u, o);
#pragma unroll
            for (int m = 1; m < 8; ++m) w[m] = MV3{make_float2(o[m][0], o[m][1]), o[m][2]};
        }
        MV3 Bf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out.T[q] = madd(w[q], w[q + 4]);
            Bf[q] = msub(w[q], w[q + 4]);
        }
        if (s >= k0) {
            const MV3 S0 = madd(in.T[0], Bf[0]), S1 = madd(in.T[1], Bf[1]);
            const MV3 S2 = madd(in.T[2], Bf[2]), S3 = madd(in.T[3], Bf[3]);
            const MV3 p = msub(S0, S2), qd = msub(S1, S3), r = madd(S0, S2), sd = madd(S1, S3);
            const MV3 c00 = msub(p, qd), c10 = madd(p, qd), c01 = msub(r, sd), c11 = madd(r, sd);
            MV3 n01, n00;
            n01.xy.x = __shfl_down_sync(0xffffffffu, c01.xy.x, 1, BX);
            n01.xy.y = __shfl_down_sync(0xffffffffu, c01.xy.y, 1, BX);
            n01.z = __shfl_down_sync(0xffffffffu, c01.z, 1, BX);
            n00.xy.x = __shfl_down_sync(0xffffffffu, c00.xy.x, 1, BX);
            n00.xy.y = __shfl_down_sync(0xffffffffu, c00.xy.y, 1, BX);
            n00.z = __shfl_down_sync(0xffffffffu, c00.z, 1, BX);
            R1 = madd(c11, n01);
            const MV3 r0 = madd(c10, n00);
            const float esum = __fadd_rn(in.E, out.E);
            const float er = __fadd_rn(esum, __shfl_down_sync(0xffffffffu, esum, 1, BX));
            sx[s & 1][ty][tx] = make_float4(r0.xy.x, r0.xy.y, r0.z, er);
            pending = true;
            eR1 = er;
            un_pend = in.C[3];
            m_pend = mcur;
        }
        return true;
    };

    unsigned par = 0;
    bool ok = !failed;
    for (int s = kb; ok && s < k1; s += 4, par ^= 1u) {
        ok = step(std::integral_constant<int, 0>{}, s, par, s0, s1);
        if (ok && s + 1 < k1) ok = step(std::integral_constant<int, 1>{}, s + 1, par, s1, s0);
        if (ok && s + 2 < k1) ok = step(std::integral_constant<int, 2>{}, s + 2, par, s0, s1);
        if (ok && s + 3 < k1) ok = step(std::integral_constant<int, 3>{}, s + 3, par, s1, s0);
    }
    if (ok) {
        const int q = (k1 - kb) & 3;
        const unsigned pq = (unsigned)(((k1 - kb) >> 2) & 1) ^ (q == 3 ? 1u : 0u);
        if (EPI_B && !wait_full(q, pq)) failed = true;
        ok = !__syncthreads_or(failed);
        if (ok && pending) finish(k1 - 1, q);
    }
    if (!ok) {
        if (tid == 0) {
            for (int q = 0; q < 4; ++q)
                if (issued[q] > 0) wait_full(q, (unsigned)(issued[q] - 1) & 1u);
            atomicExch(a.err, 1);
        }
        return;
    }
    if (DOT) {
        const double sum = block_sum_all<NT>(dotv.value(), tid);
        if (tid == 0) a.partial[(long long)l * a.pstride + tile] = sum;
    }
}

// ---- launch plans of the level-0 multi-load operator ------------------------------
struct MPlan {
    int tile;  // 0: 32 x 8 threads, 1: 16 x 16
    int zc;
    int gx, gy, gz;
    long long tiles() const { return (long long)gx * gy * gz; }
};

int msm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

// The tile shape and z-chunk that minimise (waves x steps per block) for nl
// blocks per tile and two resident blocks per SM (the cost model of the
// single-load kernel with the load count folded into the block count).
MPlan mplan(int nx, int ny, int nz, int nl) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int slots = 2 * msm_count();
    MPlan best{0, NZ, 1, 1, 1};
    long long best_cost = -1;
    const int shapes[2][2] = {{32, 8}, {16, 16}};
    for (int t = 0; t < 2; ++t) {
        const int bx = shapes[t][0], by = shapes[t][1];
        const int gx = (NX + bx - 2) / (bx - 1), gy = (NY + by - 2) / (by - 1);
        for (int nch = 1; nch <= NZ; ++nch) {
            const int zc = (NZ + nch - 1) / nch;
            if (zc < 4 && nch > 1) break;
            const int gz = (NZ + zc - 1) / zc;
            const long long blocks = (long long)gx * gy * gz * nl;
            const long long waves = (blocks + slots - 1) / slots;
            const long long cost = waves * (zc + 1) * 64 + (blocks % slots == 0 ? 0 : 1);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best = MPlan{t, zc, gx, gy, gz};
            }
        }
    }
    return best;
}

template <int BX, int BY, int MODE, bool DOT>
int mfine_tile(const MPlan& pl, const MFineArgs& a, const GSym& G, cudaStream_t s) {
    using T = MTile<BX, BY>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_mfine<BX, BY, MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM) !=
            cudaSuccess)
            return GMG_ERR_CUDA;
        attr = true;
    }
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    // multi-load vectors: [NZ][NY][px][16 loads][4] FP32; a tensor row is a node's 64 floats
    const unsigned long long vd[4] = {(unsigned long long)kNodeF, (unsigned long long)NX, (unsigned long long)NY,
                                      (unsigned long long)NZ};
    const unsigned long long vs[3] = {4ull * kNodeF, 4ull * kNodeF * a.px, 4ull * kNodeF * a.px * NY};
    const unsigned long long ed[3] = {(unsigned long long)a.nx, (unsigned long long)a.ny, (unsigned long long)a.nz};
    const unsigned long long es[2] = {4ull * a.epitch, 4ull * a.epitch * a.ny};
    const unsigned bx_x[4] = {4u, (unsigned)T::XN, (unsigned)T::XR, 1u};
    const unsigned bx_o[4] = {4u, (unsigned)T::ON, (unsigned)T::OR, 1u};
    const unsigned bx_e[3] = {(unsigned)T::EW, (unsigned)T::ER, 1u};
    CUtensorMap mx, me, mb, md;
    const float* b = a.b ? a.b : a.xin;
    const float* d = a.dold ? a.dold : b;
    if (!encode_f32_map_strided(&mx, a.xin, 4, vd, vs, bx_x) || !encode_f32_map_strided(&me, a.Ep, 3, ed, es, bx_e) ||
        !encode_f32_map_strided(&mb, b, 4, vd, vs, bx_o) || !encode_f32_map_strided(&md, d, 4, vd, vs, bx_o))
        return GMG_ERR_CUDA;
    note_launch();
    pdl_launch(k_mfine<BX, BY, MODE, DOT>, dim3((unsigned)(pl.tiles() * a.nl)), dim3(BX, BY), (size_t)T::SMEM, s, mx,
               me, mb, md, a, G, pl.zc, pl.gx, pl.gy);
    return GMG_OK;
}

template <int MODE, bool DOT>
int mfine_shape(const MPlan& pl, const MFineArgs& a, const GSym& G, cudaStream_t s) {
    return pl.tile == 0 ? mfine_tile<32, 8, MODE, DOT>(pl, a, G, s) : mfine_tile<16, 16, MODE, DOT>(pl, a, G, s);
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------
int mfine_blocks(int nx, int ny, int nz, int nl) { return (int)mplan(nx, ny, nz, nl).tiles(); }

int launch_mfine(int mode, int dot, const MFineArgs& a, const GSym& G, cudaStream_t s) {
    const MPlan pl = mplan(a.nx, a.ny, a.nz, a.nl);
    if (mode == FM_APPLY) return dot ? mfine_shape<FM_APPLY, true>(pl, a, G, s) : mfine_shape<FM_APPLY, false>(pl, a, G, s);
    if (mode == FM_SMOOTH)
        return dot ? mfine_shape<FM_SMOOTH, true>(pl, a, G, s) : mfine_shape<FM_SMOOTH, false>(pl, a, G, s);
    return mfine_shape<FM_RESID, false>(pl, a, G, s);
}

namespace {

int rec_grid(long long nrec) {
    return (int)std::max<long long>(1, std::min<long long>((nrec + kMT - 1) / kMT, kMBlocks));
}

MBsrArgs mbsr_args(const Level& l) {
    MBsrArgs a{};
    a.nx = l.nx; a.ny = l.ny; a.nz = l.nz; a.nn = (int)l.nn;
    a.ps = l.ps; a.A = l.A32; a.invdiag = l.invdiag; a.mask = l.mask; a.coef = l.coef;
    return a;
}

template <int LQ>
void launch_mbsr_lq(int mode, const MBsrArgs& a, cudaStream_t s) {
    const dim3 g((unsigned)(((long long)a.nn * (kLoads / LQ) + 127) / 128));
    if (mode == FM_APPLY) pdl_launch(k_mbsr<FM_APPLY, LQ>, g, dim3(128), 0, s, a);
    else if (mode == FM_RESID) pdl_launch(k_mbsr<FM_RESID, LQ>, g, dim3(128), 0, s, a);
    else pdl_launch(k_mbsr<FM_SMOOTH, LQ>, g, dim3(128), 0, s, a);
}

// Four loads per thread on every level: inside a batch the chunks' kernels run
// concurrently and the GPU is full, so instructions count more than warps in
// flight (8 x 16 loads on 32^3-80^3, one bench run each: 1,560 solves/s with
// four loads per thread everywhere, 1,483 with one per thread below 32,768
// nodes, 1,400 with one everywhere, 1,418 with eight).
void launch_mbsr(int mode, const MBsrArgs& a, cudaStream_t s) {
    note_launch();
    launch_mbsr_lq<4>(mode, a, s);
}

// ---- host side ----------------------------------------------------------------------
int mfail(int code, const std::string& msg) {
    set_error_text(msg);
    return code;
}

template <typename T>
int malloc_dev(gmg_handle* h, T** p, size_t count) {
    *p = nullptr;
    void* q = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return mfail(GMG_ERR_NOMEM, "multi-load workspace: device allocation failed");
    }
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return GMG_OK;
}

#define MTRY(x)                            \
    do {                                   \
        const int rc_ = (x);               \
        if (rc_ != GMG_OK) return rc_;     \
    } while (0)

bool multi_eligible(const gmg_handle* h, std::string* why) {
    const gmg_options& o = h->opt;
    const char* r = nullptr;
    if (h->L < 2) r = "a single-level hierarchy";
    else if (h->coarse_pcg) r = "a coarsest level above the dense-Cholesky cutoff";
    else if (o.outer != GMG_OUTER_PCG) r = "outer FGMRES";
    else if (o.ir_factor != 0.0) r = "iterative refinement";
    else if (o.fine_smoother != GMG_FINE_FP32) r = "a tensor-core fine smoother";
    else if (o.cycle_index != 1) r = "a W-cycle";
    if (r && why) *why = r;
    return r == nullptr;
}

}  // namespace

// Allocates h's multi-load workspace (once).
int multi_workspace(gmg_handle* h) {
    if (h->mw) return GMG_OK;
    MultiWork* w = new MultiWork();
    auto bad = [&](int rc) {
        if (w->pinned) cudaFreeHost(w->pinned);
        delete w;
        return rc;
    };
    cudaStream_t s = h->stream;
    const Level& l0 = h->lev[0];
    const size_t n0 = (size_t)l0.nnp * kNodeF;
    float** v0[] = {&w->r, &w->z, &w->p, &w->q, &w->x2, &w->t, &w->d};
    for (float** v : v0) {
        if (int rc = malloc_dev(h, v, n0); rc != GMG_OK) return bad(rc);
        if (cudaMemsetAsync(*v, 0, n0 * sizeof(float), s) != cudaSuccess) return bad(mfail(GMG_ERR_CUDA, "multi memset"));
    }
    for (int li = 1; li < h->L; ++li) {
        const size_t n = (size_t)h->lev[li].nn * kNodeF;
        MultiLevel& m = w->lev[li];
        float** vl[] = {&m.x, &m.x2, &m.b, &m.t, &m.d};
        for (float** v : vl) {
            if (int rc = malloc_dev(h, v, n); rc != GMG_OK) return bad(rc);
            if (cudaMemsetAsync(*v, 0, n * sizeof(float), s) != cudaSuccess)
                return bad(mfail(GMG_ERR_CUDA, "multi memset"));
        }
    }
    w->pstride = kMBlocks;
    for (int nl = 1; nl <= kLoads; ++nl) w->pstride = std::max(w->pstride, mfine_blocks(l0.nx, l0.ny, l0.nz, nl));
    for (int nl = 1; nl <= kLoads; ++nl)
        w->pstride = std::max(w->pstride, resid64_grid_blocks_multi(l0.nx, l0.ny, l0.nz, nl));
    w->pstride = std::max(w->pstride, mfine_tc_blocks(l0.nx, l0.ny, l0.nz));
    {
        std::vector<float> op(2048);
        w->tc_passes = build_mfine_tc_operand(h->keD.v, op.data(), &w->tc_scale);
        if (int rc = malloc_dev(h, &w->tcB, op.size()); rc != GMG_OK) return bad(rc);
        if (cudaMemcpy(w->tcB, op.data(), sizeof(float) * op.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bad(mfail(GMG_ERR_CUDA, "multi-load tensor-core operand"));
    }
    // two partial arrays of kLoads rows (the norms kernel fills both)
    if (int rc = malloc_dev(h, &w->partials, (size_t)2 * kLoads * w->pstride); rc != GMG_OK) return bad(rc);
    if (int rc = malloc_dev(h, &w->sc, (size_t)kLoads * SC_COUNT); rc != GMG_OK) return bad(rc);
    if (int rc = malloc_dev(h, &w->wcor, (size_t)kLoads * 3 * l0.nn); rc != GMG_OK) return bad(rc);
    if (cudaMemsetAsync(w->wcor, 0, sizeof(float2) * kLoads * 3 * (size_t)l0.nn, s) != cudaSuccess)
        return bad(mfail(GMG_ERR_CUDA, "multi memset"));
    if (cudaMemsetAsync(w->sc, 0, sizeof(double) * kLoads * SC_COUNT, s) != cudaSuccess)
        return bad(mfail(GMG_ERR_CUDA, "multi memset"));
    if (h->nL > 0 && h->Ainv && !h->coarse_pcg) {
        const size_t nn2 = (size_t)h->nL * h->nL;
        if (int rc = malloc_dev(h, &w->Ahi, nn2); rc != GMG_OK) return bad(rc);
        if (int rc = malloc_dev(h, &w->Alo, nn2); rc != GMG_OK) return bad(rc);
        if (int rc = malloc_dev(h, &w->bc, (size_t)h->nL * kLoads); rc != GMG_OK) return bad(rc);
        note_launch();
        k_split_inverse<<<kMBlocks, kMT, 0, s>>>(h->Ainv, (long long)nn2, w->Ahi, w->Alo);
    }
    const size_t bytes = sizeof(double) * kLoads * SC_COUNT + 4 * sizeof(int);
    if (cudaHostAlloc(&w->pinned, bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        w->pinned = nullptr;
        return bad(mfail(GMG_ERR_NOMEM, "multi-load pinned scalars"));
    }
    std::memset(w->pinned, 0, bytes);
    w->sc_host = static_cast<double*>(w->pinned);
    w->err_host = reinterpret_cast<int*>(w->sc_host + kLoads * SC_COUNT);
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&w->sc_map), w->pinned, 0) != cudaSuccess) {
        cudaGetLastError();
        return bad(mfail(GMG_ERR_CUDA, "multi-load pinned scalars"));
    }
    w->err_map = reinterpret_cast<int*>(w->sc_map + kLoads * SC_COUNT);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return bad(mfail(GMG_ERR_CUDA, "multi-load workspace"));
    }
    h->mw = w;
    return GMG_OK;
}

void multi_free(gmg_handle* h) {
    MultiWork* w = h->mw;
    if (!w) return;
    for (auto& e : w->loops) {
        cudaGraphExecDestroy(e.ex);
        cudaGraphDestroy(e.g);
    }
    if (w->pinned) cudaFreeHost(w->pinned);
    delete w;
    h->mw = nullptr;
}

void multi_drop_loops(gmg_handle* h) {
    if (!h->mw) return;
    for (auto& e : h->mw->loops) {
        cudaGraphExecDestroy(e.ex);
        cudaGraphDestroy(e.g);
    }
    h->mw->loops.clear();
}

namespace {
std::atomic<unsigned> g_multi_gen{0};  // bumped whenever a handle's level-0 multi-load operator changes
}  // namespace

unsigned multi_generation() { return g_multi_gen.load(std::memory_order_relaxed); }

namespace {

MFineArgs mfine_args(gmg_handle* h, int nl) {
    const Level& l = h->lev[0];
    MFineArgs a{};
    a.nx = l.nx; a.ny = l.ny; a.nz = l.nz; a.px = l.px; a.epitch = h->ex; a.nl = nl;
    a.Ep = h->E32p; a.maskp = l.maskp; a.inv0 = h->inv0; a.coef = l.coef; a.kd = h->kd; a.err = h->kerr;
    a.pstride = h->mw->pstride;
    return a;
}

// The level-0 operator of the multi-load path on the handle's chosen unit.
int mfine_launch(gmg_handle* h, int mode, int dot, const MFineArgs& a) {
    MultiWork& w = *h->mw;
    if (w.fine_kernel == 1) return launch_mfine_tc(mode, dot, a, w.tcB, w.tc_scale, w.tc_passes, h->stream);
    return launch_mfine(mode, dot, a, h->gs, h->stream);
}
int mfine_partials(gmg_handle* h, int nl) {
    const Level& l0 = h->lev[0];
    return h->mw->fine_kernel == 1 ? mfine_tc_blocks(l0.nx, l0.ny, l0.nz) : mfine_blocks(l0.nx, l0.ny, l0.nz, nl);
}

// y = K^l x on multi-load vectors (dot: partial x . y per load, finalised into slot).
void mlevel_apply(gmg_handle* h, int li, const float* x, float* y, int dot_slot, int op, int nl) {
    MultiWork& w = *h->mw;
    cudaStream_t s = h->stream;
    if (li == 0) {
        MFineArgs a = mfine_args(h, nl);
        a.xin = x; a.out = y; a.partial = dot_slot >= 0 ? w.partials : nullptr;
        if (mfine_launch(h, FM_APPLY, dot_slot >= 0, a) != GMG_OK) w.launch_err = 1;
        if (dot_slot >= 0) {
            note_launch();
            pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, s, (const double*)w.partials, mfine_partials(h, nl),
                       w.pstride, w.sc, dot_slot, op);
        }
    } else {
        MBsrArgs a = mbsr_args(h->lev[li]);
        a.xin = x; a.out = y;
        launch_mbsr(FM_APPLY, a, s);
    }
}

void mlevel_resid(gmg_handle* h, int li, const float* b, const float* x, float* t, int nl) {
    cudaStream_t s = h->stream;
    if (li == 0) {
        MFineArgs a = mfine_args(h, nl);
        a.xin = x; a.b = b; a.out = t;
        if (mfine_launch(h, FM_RESID, 0, a) != GMG_OK) h->mw->launch_err = 1;
    } else {
        MBsrArgs a = mbsr_args(h->lev[li]);
        a.xin = x; a.b = b; a.out = t;
        launch_mbsr(FM_RESID, a, s);
    }
}

// dold_from (level 0): read the previous increment from there instead of the
// level's d vector (after a first step from zero, whose increment is its output).
void msmooth_step(gmg_handle* h, int li, int k, bool zero_init, const float* b, const float* xcur, float* xnext,
                  bool write_d, bool dot, int nl, const float* dold_from = nullptr) {
    MultiWork& w = *h->mw;
    Level& l = h->lev[li];
    cudaStream_t s = h->stream;
    float* d = li == 0 ? w.d : w.lev[li].d;
    if (li == 0) {
        if (zero_init) {
            note_launch();
            pdl_launch(k_mfine_smooth0, dim3(rec_grid(l.nnp * kLoads)), dim3(kMT), 0, s, b, (const float*)h->inv0,
                       (const uint8_t*)l.maskp, l.nnp, (const double*)l.coef, xnext, write_d ? d : (float*)nullptr);
        } else {
            MFineArgs a = mfine_args(h, nl);
            a.xin = xcur; a.b = b; a.out = xnext; a.step = k; a.dold = dold_from ? dold_from : d;
            a.dnew = write_d ? d : nullptr;
            a.partial = dot ? w.partials : nullptr;
            if (mfine_launch(h, FM_SMOOTH, dot, a) != GMG_OK) w.launch_err = 1;
        }
    } else {
        MBsrArgs a = mbsr_args(l);
        a.b = b; a.out = xnext; a.step = k; a.dold = d; a.dnew = write_d ? d : nullptr;
        if (zero_init) {
            note_launch();
            pdl_launch(k_mbsr_smooth0, dim3(rec_grid(l.nn * kLoads)), dim3(kMT), 0, s, a);
        } else {
            a.xin = xcur;
            launch_mbsr(FM_SMOOTH, a, s);
        }
    }
}

float* msmooth_pass(gmg_handle* h, int li, const float* b, float* cur, float* X, float* S, bool zero_init, int& writes,
                    int nl, int dot_slot = -1, int op = FIN_NONE) {
    MultiWork& w = *h->mw;
    Level& l = h->lev[li];
    const bool cheb = l.kind == GMG_SMOOTHER_CHEBYSHEV;
    // level 0: a first step from zero leaves d = x, so the next step reads its
    // increment from that step's output and no copy of it is written
    const float* d_alias = nullptr;
    for (int k = 0; k < l.degree; ++k) {
        float* next = (writes % 2 == 0) ? S : X;
        const bool last = k == l.degree - 1;
        const bool dot = last && dot_slot >= 0;
        const bool alias = li == 0 && zero_init && k == 0;
        msmooth_step(h, li, k, zero_init && k == 0, b, cur, next, cheb && !last && !alias, dot, nl,
                     k == 1 ? d_alias : nullptr);
        if (alias && cheb && !last) d_alias = next;
        if (dot) {
            note_launch();
            pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, h->stream, (const double*)w.partials,
                       mfine_partials(h, nl), w.pstride, w.sc, dot_slot, op);
        }
        cur = next;
        ++writes;
    }
    return cur;
}

void launch_mcoarse(gmg_handle* h, const float* b, float* x) {
    const Level& l = h->lev[h->L - 1];
    note_launch(2);
    pdl_launch(k_mcoarse_gather, dim3(kMBlocks), dim3(256), 0, h->stream, h->nL, (const int*)h->free_idx, b,
               h->mw->bc, x, (const uint8_t*)l.mask, (int)l.nn);
    const int g = std::max(1, (h->nL + kCoarseRows - 1) / kCoarseRows);
    pdl_launch(k_mcoarse, dim3(g), dim3(256), 0, h->stream, h->nL, (const int*)h->free_idx, (const float*)h->mw->Ahi,
               (const float*)h->mw->Alo, (const float*)h->mw->bc, x, (int)l.nn);
}

void launch_mrestrict(const Level& f, const Level& c, const float* fine, float* coarse, cudaStream_t s) {
    note_launch();
    const long long nrec = c.nn * kLoads;
    pdl_launch(k_mrestrict, dim3((unsigned)((nrec + kMT - 1) / kMT)), dim3(kMT), 0, s, f.nx, f.ny, f.nz, f.px, c.nx,
               c.ny, c.nz, (const uint8_t*)c.mask, fine, coarse);
}

void launch_mprolong_add(const Level& f, const Level& c, const float* coarse, float* fine, cudaStream_t s) {
    note_launch();
    const long long nrec = f.nn * kLoads;
    pdl_launch(k_mprolong_add, dim3((unsigned)((nrec + kMT - 1) / kMT)), dim3(kMT), 0, s, f.nx, f.ny, f.nz, f.px, c.nx,
               c.ny, (const uint8_t*)f.mask, coarse, fine);
}

// Eq. vcycle on level li for all loads: X = V(b), S the ping-pong partner.
void mvcycle(gmg_handle* h, int li, const float* b, float* X, float* S, int dot_slot, int op, int nl) {
    MultiWork& w = *h->mw;
    if (li == h->L - 1) {
        launch_mcoarse(h, b, X);
        return;
    }
    int writes = 0;
    float* cur = msmooth_pass(h, li, b, nullptr, X, S, true, writes, nl);
    float* t = li == 0 ? w.t : w.lev[li].t;
    mlevel_resid(h, li, b, cur, t, nl);
    const Level& l = h->lev[li];
    const Level& c = h->lev[li + 1];
    MultiLevel& mc = w.lev[li + 1];
    launch_mrestrict(l, c, t, mc.b, h->stream);
    mvcycle(h, li + 1, mc.b, mc.x, mc.x2, -1, FIN_NONE, nl);
    launch_mprolong_add(l, c, mc.x, cur, h->stream);
    msmooth_pass(h, li, b, cur, X, S, false, writes, nl, dot_slot, op);
}

// ---- PCG steps of the multi-load loop (as pcg_restart / pcg_step / pcg_direction)
void mpcg_restart(gmg_handle* h, int nl) {
    MultiWork& w = *h->mw;
    mvcycle(h, 0, w.r, w.z, w.x2, SC_RZ, FIN_NONE, nl);
    launch_copy_f32(w.p, w.z, h->lev[0].nnp * kNodeF, h->stream);
}

// cond: inside the captured loop (sets the while condition); host_check: the
// host-driven loop (the same per-load test, read back by the host).
void mpcg_step(gmg_handle* h, int nl, const cudaGraphConditionalHandle* cond, bool host_check = false) {
    MultiWork& w = *h->mw;
    const Level& l0 = h->lev[0];
    cudaStream_t s = h->stream;
    mlevel_apply(h, 0, w.p, w.q, SC_PQ, FIN_ALPHA, nl);
    note_launch();
    pdl_launch(k_mpcg_update, dim3(kMBlocks), dim3(kPcgThreads), 0, s, w.wcor, 3 * l0.nn, nl, w.r, (const float*)w.p,
               (const float*)w.q, l0.nx + 1, l0.px, l0.nnp, (const double*)w.sc, w.partials, w.pstride);
    w.w_dirty = true;
    note_launch();
    if (cond || host_check)
        pdl_launch(k_mfinalize_check, dim3(1), dim3(32 * kLoads), 0, s, (const double*)w.partials, kMBlocks, w.pstride,
                   w.sc, cond ? *cond : cudaGraphConditionalHandle{}, cond ? 1 : 0);
    else
        pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, s, (const double*)w.partials, kMBlocks, w.pstride, w.sc,
                   (int)SC_RR, (int)FIN_NONE);
}

void mpcg_direction(gmg_handle* h, int nl) {
    MultiWork& w = *h->mw;
    mvcycle(h, 0, w.r, w.z, w.x2, SC_RZNEW, FIN_BETA, nl);
    note_launch();
    pdl_launch(k_mp_update, dim3(kMBlocks), dim3(kMT), 0, h->stream, w.p, (const float*)w.z, h->lev[0].nnp * kLoads,
               (const double*)w.sc);
}

}  // namespace

// Captures the multi-load PCG loop [restart, step, check, while (any load
// iterates) {direction, step, check}] of handle h for the iterates u[0..nl)
// into graph g as an independent branch, on stream cap.
bool multi_capture_loop(gmg_handle* h, double* const* u, int nl, cudaGraph_t g, cudaStream_t cap,
                        unsigned long long& prefix, unsigned long long& body_k) {
    (void)u;  // the loop updates the handle's correction; u keys the captured graph
    const unsigned long long l0 = g_kernel_launches.load();
    cudaStream_t user = h->stream;
    h->stream = cap;
    cudaGraph_t body = nullptr, out = nullptr;
    cudaGraphConditionalHandle cond{};
    unsigned long long l1 = l0, l2 = l0;
    bool ok = cudaGraphConditionalHandleCreate(&cond, g, 0, 0) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        mpcg_restart(h, nl);
        mpcg_step(h, nl, &cond);
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
            mpcg_direction(h, nl);
            mpcg_step(h, nl, &cond);
            l2 = g_kernel_launches.load();
            ok = cudaStreamEndCapture(cap, &body) == cudaSuccess;
        }
    }
    h->stream = user;
    g_kernel_launches.fetch_sub(g_kernel_launches.load() - l0);
    cudaGetLastError();
    if (h->mw->launch_err) ok = false;
    h->mw->launch_err = 0;
    prefix = l1 - l0;
    body_k = l2 - l1;
    return ok;
}

// ---- the pieces of a multi-load solve shared with gmg_solve_batch --------------------
// Fixed DOFs of u_l to 0, nonzero counts of u_l and ||f_l||^2 of nl loads
// into their scalar blocks (SC_UNZ, SC_FF), three launches (asynchronous).
void multi_norms(gmg_handle* h, int nl, const double* const* f, double* const* u) {
    MultiWork& w = *h->mw;
    const Level& l0 = h->lev[0];
    if (w.w_dirty) {  // steps of an abandoned call: not part of any iterate
        cudaMemsetAsync(w.wcor, 0, sizeof(float2) * kLoads * 3 * (size_t)l0.nn, h->stream);
        w.w_dirty = false;
    }
    F64Out uo{};
    F64In fi{};
    for (int l = 0; l < nl; ++l) {
        uo.p[l] = u[l];
        fi.p[l] = f[l];
    }
    double* p2 = w.partials + (size_t)kLoads * w.pstride;
    note_launch(3);
    pdl_launch(k_mnorms, dim3(kMBlocks), dim3(32 * kLoads), 0, h->stream, uo, fi, nl, (const uint8_t*)l0.mask, l0.nn,
               w.partials, p2, w.pstride);
    pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, h->stream, (const double*)w.partials, kMBlocks, w.pstride,
               w.sc, (int)SC_UNZ, (int)FIN_NONE);
    pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, h->stream, (const double*)p2, kMBlocks, w.pstride, w.sc,
               (int)SC_FF, (int)FIN_NONE);
}

// The FP64 true residual of loads 0..nl-1 into their SC_TRR, one launch.
void multi_true_residuals(gmg_handle* h, int nl, const double* const* f, double* const* u) {
    MultiWork& w = *h->mw;
    const Level& l0 = h->lev[0];
    if (w.w_dirty) {  // the PCG steps since the last flush into the FP64 iterates
        F64Out uo{};
        for (int l = 0; l < nl; ++l) uo.p[l] = u[l];
        const long long n3 = 3 * l0.nn;
        note_launch();
        pdl_launch(k_mflush, dim3(kMBlocks), dim3(256), 0, h->stream, uo, nl, w.wcor, n3);
        w.w_dirty = false;
    }
    launch_fine_resid64_multi(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, nl, f, u, w.sc, w.partials, w.pstride, h->gs64,
                              h->stream);
    note_launch();
    pdl_launch(k_mfinalize, dim3(kLoads), dim3(kMT), 0, h->stream, (const double*)w.partials,
               resid64_grid_blocks_multi(l0.nx, l0.ny, l0.nz, nl), w.pstride, w.sc, (int)SC_TRR, (int)FIN_NONE);
}

// r(l) = f_l for the loads with cold[l] (0 for the others and loads >= nl).
void multi_cast(gmg_handle* h, int nl, const double* const* f, const bool* cold) {
    const Level& l0 = h->lev[0];
    F64In fi{};
    for (int l = 0; l < nl; ++l) fi.p[l] = cold[l] ? f[l] : nullptr;
    note_launch();
    pdl_launch(k_mcast, dim3(kMBlocks), dim3(kMT), 0, h->stream, fi, nl, (const uint8_t*)l0.maskp, l0.nx + 1, l0.px,
               l0.nnp, h->mw->r);
}

// FP64 true residual of load l into its SC_TRR (and, with into_r, its FP32
// residual into slot l of the multi-load r).
void multi_true_residual(gmg_handle* h, int l, const double* f, const double* u, bool into_r) {
    const Level& l0 = h->lev[0];
    double* sc = h->mw->sc + l * SC_COUNT;
    launch_fine_resid64(l0.nx, l0.ny, l0.nz, h->E64, l0.mask, f, u, nullptr, h->r, l0.px, sc, h->partials, h->gs64,
                        h->stream);
    launch_finalize(h->partials, resid64_grid_blocks(l0.nx, l0.ny, l0.nz), sc, SC_TRR, FIN_NONE, h->stream);
    if (into_r) {
        note_launch();
        pdl_launch(k_mpack_slot, dim3(rec_grid(l0.nnp)), dim3(kMT), 0, h->stream, (const float*)h->r, l0.nnp, l,
                   h->mw->r);
    }
}

// The device scalars of every load -> the pinned mirror (no copy engine).
void multi_publish(gmg_handle* h) {
    launch_publish(h->mw->sc, kLoads * SC_COUNT, h->mw->sc_map, h->kerr, nullptr, h->mw->err_map, h->stream);
}

bool multi_ok(const gmg_handle* h, std::string* why) { return multi_eligible(h, why); }

void multi_set_loop_scalars(gmg_handle* h, int nl, double tol, int maxit, const double* nf, const bool* active) {
    LoopScalars v{};
    for (int l = 0; l < kLoads; ++l) {
        const bool a = l < nl && active[l];
        v.nf[l] = a ? nf[l] : 1.0;
        v.act[l] = a ? 1.0 : 0.0;
    }
    v.tol = tol;
    v.maxit = (double)maxit;
    note_launch();
    k_mset_loop<<<1, 32, 0, h->stream>>>(h->mw->sc, v);
}

}  // namespace gmg

using namespace gmg;

extern "C" {

int gmg_apply_multi(gmg_handle* h, int nl, const float* const* u, float* const* y) {
    if (!h || !u || !y || nl < 1 || nl > kLoads) return mfail(GMG_ERR_ARG, "null argument or load count outside 1..16");
    for (int l = 0; l < nl; ++l)
        if (!u[l] || !y[l]) return mfail(GMG_ERR_ARG, "null load vector");
    MTRY(multi_workspace(h));
    MultiWork& w = *h->mw;
    const Level& l0 = h->lev[0];
    cudaStream_t s = h->stream;
    F32In in{};
    F32Out out{};
    for (int l = 0; l < nl; ++l) {
        in.p[l] = u[l];
        out.p[l] = y[l];
    }
    note_launch();
    pdl_launch(k_mpack_dense, dim3(rec_grid(l0.nnp * kLoads)), dim3(kMT), 0, s, in, nl, (const uint8_t*)l0.maskp,
               l0.nx + 1, l0.px, l0.nnp, w.p);
    w.launch_err = 0;
    mlevel_apply(h, 0, w.p, w.q, -1, FIN_NONE, nl);
    if (w.launch_err) {
        w.launch_err = 0;
        return mfail(GMG_ERR_CUDA, "multi-load apply: tensor map encoding failed");
    }
    note_launch();
    pdl_launch(k_munpack_dense, dim3(rec_grid(l0.nn * nl)), dim3(kMT), 0, s, (const float*)w.q, nl, l0.nx + 1, l0.px,
               l0.nn, out);
    if (cudaGetLastError() != cudaSuccess) return mfail(GMG_ERR_CUDA, "multi-load apply launch");
    return GMG_OK;
}

int gmg_multi_fine_pass(gmg_handle* h, int nl, int what) {
    if (!h || nl < 1 || nl > kLoads || what < 0 || what > 1) return mfail(GMG_ERR_ARG, "bad handle, load count or pass");
    if (what == 1 && h->L < 2) return mfail(GMG_ERR_ARG, "smoothing pass needs an assembled level below");
    MTRY(multi_workspace(h));
    MultiWork& w = *h->mw;
    w.launch_err = 0;
    if (what == 0) {
        mlevel_apply(h, 0, w.p, w.q, -1, FIN_NONE, nl);
    } else {
        int writes = 0;  // steps alternate x2, z, ... starting from the iterate in z
        msmooth_pass(h, 0, w.r, w.z, w.z, w.x2, false, writes, nl);
    }
    if (w.launch_err) {
        w.launch_err = 0;
        return mfail(GMG_ERR_CUDA, "multi-load pass: tensor map encoding failed");
    }
    if (cudaGetLastError() != cudaSuccess) return mfail(GMG_ERR_CUDA, "multi-load pass launch");
    return GMG_OK;
}

int gmg_set_multi_kernel(gmg_handle* h, int kind) {
    if (!h || kind < 0 || kind > 1) return mfail(GMG_ERR_ARG, "kind must be 0 (CUDA cores) or 1 (tensor cores)");
    MTRY(multi_workspace(h));
    if (h->mw->fine_kernel != kind) {
        multi_drop_loops(h);
        g_multi_gen.fetch_add(1);  // captured batch graphs that contain this handle's loop are stale
    }
    h->mw->fine_kernel = kind;
    return GMG_OK;
}

int gmg_solve_multi(gmg_handle* h, int nl, const double* const* f, double* const* u, double tol, int maxit,
                    gmg_info* infos) {
    if (!h || !f || !u || !infos || nl < 1 || nl > kLoads)
        return mfail(GMG_ERR_ARG, "null argument or load count outside 1..16");
    if (!(tol > 0.0) || maxit < 0) return mfail(GMG_ERR_ARG, "tol must be > 0 and maxit >= 0");
    for (int l = 0; l < nl; ++l) {
        if (!f[l] || !u[l]) return mfail(GMG_ERR_ARG, "null load vector");
        for (int k = 0; k < l; ++k)
            if (u[k] == u[l]) return mfail(GMG_ERR_ARG, "an iterate appears twice");
    }
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    for (int l = 0; l < nl; ++l) infos[l] = gmg_info{};
    if (!multi_eligible(h, nullptr) || maxit == 0) {
        // options outside the multi-load path: one solve after the other
        int worst = GMG_OK;
        for (int l = 0; l < nl; ++l) {
            const int rc = gmg_solve(h, f[l], u[l], tol, maxit, &infos[l]);
            if (rc < 0) return rc;
            if (rc != GMG_OK) worst = rc;
        }
        return worst;
    }
    MTRY(multi_workspace(h));
    MultiWork& w = *h->mw;
    cudaStream_t s = h->stream;
    const Level& l0 = h->lev[0];
    auto sync = [&]() -> int {
        multi_publish(h);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return mfail(GMG_ERR_CUDA, std::string("multi-load solve: ") + cudaGetErrorString(cudaGetLastError()));
        }
        if (w.err_host[0] != 0) {
            cudaMemsetAsync(h->kerr, 0, sizeof(int), s);
            cudaStreamSynchronize(s);
            return mfail(GMG_TIMEOUT, "multi-load solve: a TMA wait of the level-0 operator gave up");
        }
        return GMG_OK;
    };
    double* sch = w.sc_host;
    auto S = [&](int l, int slot) -> double& { return sch[l * SC_COUNT + slot]; };
    multi_norms(h, nl, f, u);
    MTRY(sync());
    std::vector<int> state(nl, 0);  // 0 active, 1 done
    std::vector<double> nf(nl, 0.0);
    bool cold[kLoads] = {};
    bool warm_any = false;
    for (int l = 0; l < nl; ++l) {
        const double ff = S(l, SC_FF);
        if (!(ff > 0.0)) {
            state[l] = 1;
            if (!std::isfinite(ff)) { infos[l].status = GMG_NONFINITE; infos[l].rel_residual = NAN; }
            else cudaMemsetAsync(u[l], 0, sizeof(double) * 3 * l0.nn, s);
            continue;
        }
        nf[l] = std::sqrt(ff);
        if (S(l, SC_UNZ) == 0.0) { cold[l] = true; infos[l].rel_residual = 1.0; }
        else warm_any = true;
    }
    multi_cast(h, nl, f, cold);
    for (int l = 0; l < nl; ++l)
        if (state[l] == 0 && !cold[l]) multi_true_residual(h, l, f[l], u[l], true);
    if (warm_any) {
        MTRY(sync());
        for (int l = 0; l < nl; ++l)
            if (state[l] == 0 && !cold[l]) infos[l].rel_residual = std::sqrt(S(l, SC_TRR)) / nf[l];
    }
    bool any = false;
    for (int l = 0; l < nl; ++l) {
        if (state[l] != 0) continue;
        const double rel = infos[l].rel_residual;
        infos[l].rel_residual_recursive = rel;
        if (!std::isfinite(rel)) { infos[l].status = GMG_NONFINITE; state[l] = 1; }
        else if (rel < tol) { infos[l].status = GMG_OK; state[l] = 1; }
        else any = true;
    }
    {
        bool act[kLoads] = {};
        for (int l = 0; l < nl; ++l) act[l] = state[l] == 0;
        multi_set_loop_scalars(h, nl, tol, maxit, nf.data(), act);
    }
    if (any && !h->opt.device_loop) {
        // host-driven loop: the kernels of the captured loop, launched one by
        // one, with the per-load test read back after every step
        mpcg_restart(h, nl);
        mpcg_step(h, nl, nullptr, true);
        while (true) {
            MTRY(sync());
            bool go = false;
            for (int l = 0; l < nl; ++l) go = go || (state[l] == 0 && S(l, SC_ACT) != 0.0);
            if (!go) break;
            mpcg_direction(h, nl);
            mpcg_step(h, nl, nullptr, true);
        }
    } else if (any) {
        // the captured loop for these iterates (cached per iterate list)
        std::vector<const double*> key(u, u + nl);
        MultiWork::Loop* lp = nullptr;
        for (auto& e : w.loops)
            if (e.u == key) lp = &e;
        if (!lp) {
            if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return mfail(GMG_ERR_CUDA, "multi-load capture stream");
            }
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            unsigned long long pre = 0, bod = 0;
            bool ok = cudaGraphCreate(&g, 0) == cudaSuccess && multi_capture_loop(h, u, nl, g, h->cap_stream, pre, bod);
            if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
            cudaGetLastError();
            if (!ok) {
                if (g) cudaGraphDestroy(g);
                return mfail(GMG_ERR_CUDA, "could not capture the multi-load loop");
            }
            if (w.loops.size() >= 4) {
                cudaGraphExecDestroy(w.loops.front().ex);
                cudaGraphDestroy(w.loops.front().g);
                w.loops.erase(w.loops.begin());
            }
            w.loops.push_back({key, g, ex, pre, bod});
            lp = &w.loops.back();
        }
        if (cudaGraphLaunch(lp->ex, s) != cudaSuccess) {
            cudaGetLastError();
            return mfail(GMG_ERR_CUDA, "multi-load loop launch");
        }
        w.w_dirty = true;  // the loop's steps went to the correction
        MTRY(sync());
        unsigned long long kmax = 0;
        for (int l = 0; l < nl; ++l) kmax = std::max<unsigned long long>(kmax, (unsigned long long)S(l, SC_IT));
        note_launch(lp->pre + lp->body * (kmax > 0 ? kmax - 1 : 0));
    }
    if (any) {
        for (int l = 0; l < nl; ++l) {
            if (state[l] != 0) continue;
            infos[l].iterations = (int)S(l, SC_IT);
            infos[l].rel_residual_recursive = std::sqrt(S(l, SC_RR)) / nf[l];
            if (!std::isfinite(infos[l].rel_residual_recursive) || !std::isfinite(S(l, SC_ALPHA))) {
                infos[l].status = GMG_NONFINITE;
                infos[l].rel_residual = infos[l].rel_residual_recursive;
                state[l] = 1;
            }
        }
        multi_true_residuals(h, nl, f, u);
        MTRY(sync());
        for (int l = 0; l < nl; ++l) {
            if (state[l] != 0) continue;
            const double rel = std::sqrt(S(l, SC_TRR)) / nf[l];
            infos[l].rel_residual = rel;
            state[l] = 1;
            if (!std::isfinite(rel)) infos[l].status = GMG_NONFINITE;
            else if (rel < tol) infos[l].status = GMG_OK;
            else if (!(infos[l].rel_residual_recursive < tol) || infos[l].iterations >= maxit)
                infos[l].status = GMG_NOT_CONVERGED;
            else {
                // residual replacement: this load continues alone on the handle's own loop
                gmg_info more{};
                const int rc = gmg_solve(h, f[l], u[l], tol, maxit - infos[l].iterations, &more);
                if (rc < 0) return rc;
                infos[l].status = more.status;
                infos[l].iterations += more.iterations;
                infos[l].replacements += 1 + more.replacements;
                infos[l].rel_residual = more.rel_residual;
                infos[l].rel_residual_recursive = more.rel_residual_recursive;
            }
        }
    }
    int worst = GMG_OK;
    for (int l = 0; l < nl; ++l) {
        infos[l].solve_ms = elapsed();
        infos[l].setup_ms = h->setup_ms;
        if (infos[l].status != GMG_OK) worst = infos[l].status;
        if (infos[l].status == GMG_NONFINITE) h->pads_dirty = true;
    }
    if (cudaGetLastError() != cudaSuccess) return mfail(GMG_ERR_CUDA, "multi-load solve");
    return worst;
}

}  // extern "C"
