// Hot-path kernels of the GMG-preconditioned CG solver (sm_103a).
//
//  * k_fine_smooth0  -- first fine-level smoother step from zero (the fused
//                       fine operator lives in fine.cu, its FP64 residual form
//                       in resid64.cu);
//  * k_bsr / k_bsr_ks / k_bsr_pipe -- the same three modes on an assembled
//                       Galerkin level (27-point 3x3-block operator, implicit
//                       structured columns): one streaming thread per node for
//                       large levels, a K-split form for small ones, and a
//                       persistent TMA-pipelined form;
//  * k_restrict / k_prolong_add -- R = P^T and P of Eq. trilinear_weights /
//                       Eq. vector_prolongation with the odd-size clamp;
//  * k_coarse_solve  -- dense FP64 solve with the Cholesky-derived inverse;
//  * vector kernels  -- fused PCG updates and FP64-accumulated dot products
//                       (Sec. "Outer Krylov Solver and Convergence Statement").
//
// Reductions are deterministic: every block writes one partial sum, and a
// single-block finaliser adds the partials in a fixed order.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 148 * 8;

// Sum of v over the block (blockDim.x*y*z == nthreads, multiple of 32); the
// result is valid in thread 0.  Fixed combination order.
template <int NT>
__device__ __forceinline__ double block_sum(double v, int tid) {
    __shared__ double warp_part[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) warp_part[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += warp_part[w];
    }
    return s;
}

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

// The fine level's Jacobi scale per node, 1 / (kd * sum of the moduli of the
// elements around it) (the diagonal of K is kd E_e summed over those elements).
__global__ void k_fine_inv0(int nx, int ny, int nz, int px, const float* E, float kd, float* inv0) {
    const long long NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const long long nn = NX * NY * NZ;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        float esum = 0.f;
#pragma unroll
        for (int ea = 0; ea < 8; ++ea) {
            const int ex = i - ldx(ea), ey = j - ldy(ea), ez = k - ldz(ea);
            if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz)
                esum += E[ex + (long long)nx * (ey + (long long)ny * ez)];
        }
        inv0[i + (long long)px * (j + NY * k)] = jacobi_rcp(__fmul_rn(kd, esum));
    }
}

// First smoother step from x = 0: x_1 = c_a D^{-1} b (no operator application),
// with the Jacobi scale from set-up.
// Four nodes per thread and iteration: the padded level-0 vectors hold a
// multiple of 4 nodes, so the Jacobi scales and masks of 4 nodes are one 16-byte
// and one 4-byte load and their 12 vector entries three float4 (the same
// arithmetic per entry as one node at a time).
__global__ void k_fine_smooth0(FineArgs a) {
    pdl_entry();
    const long long nn = (long long)a.pitch * (a.ny + 1) * (a.nz + 1);  // pads: mask 7, output 0
    const float ca = (float)a.coef[1];
    const long long n4 = nn / 4;
    const float4* inv4 = reinterpret_cast<const float4*>(a.inv0);
    const unsigned* m4 = reinterpret_cast<const unsigned*>(a.mask);
    const float4* b4 = reinterpret_cast<const float4*>(a.b);
    float4* o4 = reinterpret_cast<float4*>(a.out);
    float4* d4 = reinterpret_cast<float4*>(a.dnew);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n4;
         g += (long long)gridDim.x * blockDim.x) {
        const float4 iv = inv4[g];
        const unsigned mw = m4[g];
        const float inv[4] = {iv.x, iv.y, iv.z, iv.w};
        float v[12];
        {
            const float4 x0 = b4[3 * g], x1 = b4[3 * g + 1], x2 = b4[3 * g + 2];
            const float bb[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
#pragma unroll
            for (int e = 0; e < 12; ++e) {
                const unsigned m = (mw >> (8 * (e / 3))) & 0xffu;
                v[e] = fixed_bit((uint8_t)m, e % 3) ? 0.f : __fmul_rn(__fmul_rn(ca, inv[e / 3]), bb[e]);
            }
        }
        o4[3 * g] = make_float4(v[0], v[1], v[2], v[3]);
        o4[3 * g + 1] = make_float4(v[4], v[5], v[6], v[7]);
        o4[3 * g + 2] = make_float4(v[8], v[9], v[10], v[11]);
        if (a.dnew) {
            d4[3 * g] = make_float4(v[0], v[1], v[2], v[3]);
            d4[3 * g + 1] = make_float4(v[4], v[5], v[6], v[7]);
            d4[3 * g + 2] = make_float4(v[8], v[9], v[10], v[11]);
        }
    }
}

// ---------------------------------------------------------------------------
// Assembled levels: K^l is symmetric, so only the diagonal block and the 13
// "forward" neighbour blocks (slots 13..26, offsets after the node in memory
// order) are stored, plane-major: A[(u*9 + r*3 + c)*ps + n] is entry (r, c) of
// block (n, n + o_u), u = slot - 13.  Row n of K^l is then
//   sum_u A_u(n) x(n + o_u)  +  sum_{u>0} A_u(n - o_u)^T x(n - o_u).
// The plane stride ps is nn rounded up to a multiple of 4 (16-byte aligned
// planes, zero padding), which the TMA-staged kernel needs.
// ---------------------------------------------------------------------------

// Node offset of forward block u (slot 13 + u) on a grid of NX x NY nodes per plane.
__device__ __forceinline__ int fwd_offset(int u, int NX, int NY, int& dx, int& dy, int& dz) {
    const int sl = 13 + u;
    dx = sl % 3 - 1; dy = (sl / 3) % 3 - 1; dz = sl / 9 - 1;
    return dx + NX * (dy + NY * dz);
}

// Epilogue of one node's row y = (K x)_n: apply (masked, optional x.y), residual
// b - y, or one smoother step (Jacobi / Chebyshev, optional b.x_new).
template <int MODE, bool DOT>
__device__ __forceinline__ void bsr_epilogue(const BsrArgs& a, int n, const float y[3], DSAcc& dotv) {
    const uint8_t msk = a.mask[n];
    if (MODE == FM_APPLY) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fixed_bit(msk, c) ? 0.f : y[c];
            a.out[3 * n + c] = v;
            if (DOT) dotv.add_prod(a.xin[3 * n + c], v);
        }
    } else if (MODE == FM_RESID) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.out[3 * n + c] = fixed_bit(msk, c) ? 0.f : a.b[3 * n + c] - y[c];
    } else {
        const float cd = (float)a.coef[2 * a.step], ca = (float)a.coef[2 * a.step + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float xn = 0.f, dn = 0.f;
            if (!fixed_bit(msk, c)) {
                const float bc = a.b[3 * n + c];
                dn = ca * a.invdiag[3 * n + c] * (bc - y[c]);
                if (cd != 0.f) dn = fmaf(cd, a.dold[3 * n + c], dn);
                xn = a.xin[3 * n + c] + dn;
                if (DOT) dotv.add_prod(bc, xn);
            }
            a.out[3 * n + c] = xn;
            if (a.dnew) a.dnew[3 * n + c] = dn;
        }
    }
}

// Large levels (bandwidth-bound): one thread per node streaming the planes,
// branch-free so that all of a node's loads can be in flight together: every
// load is unconditional (indices clamped to the node itself for neighbours
// outside the grid); out-of-grid forward blocks are stored as zero and
// out-of-grid backward terms are scaled by 0.
template <int MODE, bool DOT, int NTB>
__global__ void __launch_bounds__(NTB) k_bsr(BsrArgs a) {
    pdl_entry();
    const int nn = (int)a.nn;
    const int n = blockIdx.x * NTB + threadIdx.x;
    DSAcc dotv;
    if (n < nn) {
        const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
        const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
        const long long N = a.ps;
        float y0 = 0.f, y1 = 0.f, y2 = 0.f;
        // branch-free: every load is unconditional (indices clamped to this node
        // when the neighbour is outside the grid), so all of them can be in
        // flight together; out-of-grid forward blocks are stored as zero, and
        // out-of-grid backward terms are scaled by 0
#pragma unroll
        for (int u = 0; u < 14; ++u) {
            const int sl = 13 + u;
            const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
            const int off = dx + NX * (dy + NY * dz);
            const bool okf = i + dx >= 0 && i + dx < NX && j + dy >= 0 && j + dy < NY && k + dz < NZ;
            const int mf = (int)GMG_B(okf ? n + off : n, nn, 201);
            // operator and iterate through the read-only data path
            const float* A = a.A + (long long)(u * 9) * N + n;
            const float v0 = __ldg(a.xin + 3 * mf), v1 = __ldg(a.xin + 3 * mf + 1), v2 = __ldg(a.xin + 3 * mf + 2);
            y0 = fmaf(__ldg(A + 0 * N), v0, fmaf(__ldg(A + 1 * N), v1, fmaf(__ldg(A + 2 * N), v2, y0)));
            y1 = fmaf(__ldg(A + 3 * N), v0, fmaf(__ldg(A + 4 * N), v1, fmaf(__ldg(A + 5 * N), v2, y1)));
            y2 = fmaf(__ldg(A + 6 * N), v0, fmaf(__ldg(A + 7 * N), v1, fmaf(__ldg(A + 8 * N), v2, y2)));
            if (u > 0) {
                const bool okb = i - dx >= 0 && i - dx < NX && j - dy >= 0 && j - dy < NY && k - dz >= 0;
                const int mb = (int)GMG_B(okb ? n - off : n, nn, 202);
                const float wgt = okb ? 1.f : 0.f;
                const float* B = a.A + (long long)(u * 9) * N + mb;
                const float w0 = wgt * __ldg(a.xin + 3 * mb), w1 = wgt * __ldg(a.xin + 3 * mb + 1),
                            w2 = wgt * __ldg(a.xin + 3 * mb + 2);
                y0 = fmaf(__ldg(B + 0 * N), w0, fmaf(__ldg(B + 3 * N), w1, fmaf(__ldg(B + 6 * N), w2, y0)));
                y1 = fmaf(__ldg(B + 1 * N), w0, fmaf(__ldg(B + 4 * N), w1, fmaf(__ldg(B + 7 * N), w2, y1)));
                y2 = fmaf(__ldg(B + 2 * N), w0, fmaf(__ldg(B + 5 * N), w1, fmaf(__ldg(B + 8 * N), w2, y2)));
            }
        }
        const float y[3] = {y0, y1, y2};
        bsr_epilogue<MODE, DOT>(a, n, y, dotv);
    }
    if (DOT) {
        const double s = block_sum<NTB>(dotv.value(), threadIdx.x);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Large levels, TMA-pipelined: a persistent kernel, one block of 256 threads
// per SM, walking tiles of 64 consecutive nodes (tile i of block b is
// b + i * gridDim.x) through a two-stage shared-memory ring.  For each tile,
// thread 0 issues 14 tensor loads on the stage's mbarrier:
//   - the tile's own 126 planes (box 126 x 64: diagonal + forward blocks);
//   - for each backward block u = 1..13, the 9 planes of block u at the nodes
//     n - o_u (box 9 x 68 from (n0 - o_u) rounded down to 4 nodes; the
//     remainder (-o_u) mod 4 is the same for every tile);
// and all threads stage, with 4-byte cp.async, the 9 rows of x that the tile's
// 27 neighbour offsets touch (66 nodes each), the epilogue operands and the
// masks.  The loads of tile i+1 are in flight while tile i is computed.
//
// No neighbour test is needed: a block towards a node outside the grid (or a
// row wrap-around) is stored as zero, and nodes outside [0, nn) read as zero.
// Four 64-thread slices each take a quarter of the 27 blocks of every node;
// the partial rows are added in shared memory in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kTmaNodes = 64;
constexpr int kTmaBackW = kTmaNodes + 4;
constexpr int kTmaOwnFloats = kSymPlanes * kTmaNodes;            // 8064 floats = 252 x 128 B
constexpr int kTmaBackStride = 640;                              // 9 x 68 = 612 floats, padded to 128 B
constexpr unsigned kTmaTxBytes = 4u * (kTmaOwnFloats + 13 * 9 * kTmaBackW);
constexpr int kXRow = 3 * (kTmaNodes + 2);                       // 198 floats of x per neighbour row
constexpr int kXRowS = 200;
constexpr int kPipeThreads = 256;
// stage layout (floats): own | 13 backward boxes | 9 x rows | b, d, D^-1 (3 x 192) | masks (16 words)
constexpr int kStOwn = 0;
constexpr int kStBack = kStOwn + kTmaOwnFloats;
constexpr int kStX = kStBack + 13 * kTmaBackStride;
constexpr int kStEpi = kStX + 9 * kXRowS;
constexpr int kStMask = kStEpi + 3 * 3 * kTmaNodes;
constexpr int kStage = (kStMask + 16 + 31) / 32 * 32;            // 128-byte multiple
constexpr int kPipeSmemBytes = 4 * (2 * kStage + 3 * 3 * kTmaNodes) + 16;
constexpr int kXCopies = (9 * kXRow + kPipeThreads - 1) / kPipeThreads;
constexpr long long kTmaSpin = 1LL << 22;

template <int MODE, bool DOT>
__global__ void __launch_bounds__(kPipeThreads, 1) k_bsr_pipe(const __grid_constant__ CUtensorMap tm_own,
                                                              const __grid_constant__ CUtensorMap tm_back,
                                                              BsrArgs a) {
    extern __shared__ __align__(128) float sm[];
    float* const part = sm + 2 * kStage;  // [3][64][3] partial rows of slices 1..3
    uint64_t* const bars = reinterpret_cast<uint64_t*>(part + 3 * 3 * kTmaNodes);
    const int tid = threadIdx.x, t = tid & (kTmaNodes - 1), slice = tid >> 6;
    const int nn = (int)a.nn;
    const int NX = a.nx + 1, NXY = NX * (a.ny + 1);
    const int ntiles = (nn + kTmaNodes - 1) / kTmaNodes;
    constexpr bool EPI_B = MODE != FM_APPLY;
    constexpr bool EPI_D = MODE == FM_SMOOTH;
    const float cd = EPI_D ? (float)a.coef[2 * a.step] : 0.f;
    const float ca = EPI_D ? (float)a.coef[2 * a.step + 1] : 0.f;
    const bool need_d = EPI_D && cd != 0.f;

    // x staging slots of this thread (the same for every tile): float w of
    // neighbour row c, (dy, dz) = (c % 3 - 1, c / 3 - 1), which starts at node
    // n0 + o_c - 1; its source is x[3 n0 + xs_off]
    int xs_off[kXCopies], xs_dst[kXCopies];
#pragma unroll
    for (int q = 0; q < kXCopies; ++q) {
        const int idx = tid + q * kPipeThreads;
        const int c = idx / kXRow, w = idx % kXRow;
        const int dy = c % 3 - 1, dz = c / 3 - 1;
        const bool used = idx < 9 * kXRow;
        xs_off[q] = used ? 3 * (NX * dy + NXY * dz - 1) + w : 0;
        xs_dst[q] = used ? kStX + c * kXRowS + w : -1;
    }
    if ((smem_u32(sm) & 127) != 0) {  // TMA destinations must be 128-byte aligned
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int st) {
        float* S = sm + st * kStage;
        const int n0 = tile * kTmaNodes;
        if (tid == 0) {
            mbar_expect_tx(&bars[st], kTmaTxBytes);
            tma_load_2d(S + kStOwn, &tm_own, n0, 0, &bars[st]);
#pragma unroll 1
            for (int u = 1; u < 14; ++u) {
                int dx, dy, dz;
                const int off = fwd_offset(u, NX, a.ny + 1, dx, dy, dz);
                tma_load_2d(S + kStBack + (u - 1) * kTmaBackStride, &tm_back, (n0 - off) & ~3, 9 * u, &bars[st]);
            }
        }
        const unsigned sbase = smem_u32(S);
#pragma unroll
        for (int q = 0; q < kXCopies; ++q) {
            if (xs_dst[q] < 0) continue;
            const long long fo = 3LL * n0 + xs_off[q];  // float offset in x
            const bool ok = fo >= 0 && fo < 3LL * nn;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + 4u * xs_dst[q]),
                         "l"(a.xin + (ok ? fo : 0)), "r"(ok ? 4 : 0)
                         : "memory");
        }
        if (tid < 3 * kTmaNodes) {
            const long long fo = 3LL * n0 + tid;
            const bool ok = fo < 3LL * nn;
            const float* srcs[3] = {a.b, a.dold, a.invdiag};
            const bool want[3] = {EPI_B, EPI_D, EPI_D};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (!want[e] || (e == 1 && !need_d)) continue;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + 4u * (kStEpi + e * 3 * kTmaNodes + tid)),
                             "l"(srcs[e] + (ok ? fo : 0)), "r"(ok ? 4 : 0)
                             : "memory");
            }
        }
        if (tid < kTmaNodes / 4) {
            const int b0 = n0 + 4 * tid;
            const int nb = min(4, max(0, nn - b0));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + 4u * (kStMask + tid)),
                         "l"(a.mask + (nb > 0 ? b0 : 0)), "r"(nb)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    DSAcc dotv;
    bool failed = false;
    int it = 0;
    int tile = blockIdx.x;
    if (tile < ntiles) issue(tile, 0);
#pragma unroll 1
    for (; tile < ntiles; tile += gridDim.x, ++it) {
        const int st = it & 1;
        const int next = tile + gridDim.x;
        if (next < ntiles) issue(next, st ^ 1);
        // the tile's TMA boxes (bounded wait) and this thread's cp.async copies
        bool ok = false;
        for (long long k = 0; k < kTmaSpin; ++k)
            if (mbar_try_wait(&bars[st], (it >> 1) & 1)) { ok = true; break; }
        if (next < ntiles) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const float* S = sm + st * kStage;
        const int n0 = tile * kTmaNodes, n = n0 + t;
        float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const int blk = slice + 4 * q;  // 0..13 forward (u = blk), 14..26 backward (u = blk - 13)
            if (blk < 27) {
                const bool fwd = blk < 14;
                const int u = fwd ? blk : blk - 13;
                int dx, dy, dz;
                const int off = fwd_offset(u, NX, a.ny + 1, dx, dy, dz);
                const int sx = fwd ? dx : -dx, sy = fwd ? dy : -dy, sz = fwd ? dz : -dz;
                const float* xr = S + kStX + ((sy + 1) + 3 * (sz + 1)) * kXRowS + 3 * (t + sx + 1);
                const float v0 = xr[0], v1 = xr[1], v2 = xr[2];
                if (fwd) {
                    const float* A = S + kStOwn + 9 * u * kTmaNodes + t;
                    y0 = fmaf(A[0 * kTmaNodes], v0, fmaf(A[1 * kTmaNodes], v1, fmaf(A[2 * kTmaNodes], v2, y0)));
                    y1 = fmaf(A[3 * kTmaNodes], v0, fmaf(A[4 * kTmaNodes], v1, fmaf(A[5 * kTmaNodes], v2, y1)));
                    y2 = fmaf(A[6 * kTmaNodes], v0, fmaf(A[7 * kTmaNodes], v1, fmaf(A[8 * kTmaNodes], v2, y2)));
                } else {
                    const float* B = S + kStBack + (u - 1) * kTmaBackStride + ((-off) & 3) + t;
                    y0 = fmaf(B[0 * kTmaBackW], v0, fmaf(B[3 * kTmaBackW], v1, fmaf(B[6 * kTmaBackW], v2, y0)));
                    y1 = fmaf(B[1 * kTmaBackW], v0, fmaf(B[4 * kTmaBackW], v1, fmaf(B[7 * kTmaBackW], v2, y1)));
                    y2 = fmaf(B[2 * kTmaBackW], v0, fmaf(B[5 * kTmaBackW], v1, fmaf(B[8 * kTmaBackW], v2, y2)));
                }
            }
        }
        if (slice > 0) {
            float* pp = part + ((slice - 1) * kTmaNodes + t) * 3;
            pp[0] = y0; pp[1] = y1; pp[2] = y2;
        }
        __syncthreads();
        if (slice == 0 && n < nn) {
            float y[3] = {y0, y1, y2};
#pragma unroll
            for (int c = 0; c < 3; ++c)
                y[c] = ((y[c] + part[t * 3 + c]) + part[(kTmaNodes + t) * 3 + c]) + part[(2 * kTmaNodes + t) * 3 + c];
            const uint8_t msk = reinterpret_cast<const uint8_t*>(S + kStMask)[t];
            const float* bb = S + kStEpi + 3 * t;
            const float* dd = S + kStEpi + 3 * kTmaNodes + 3 * t;
            const float* iv = S + kStEpi + 6 * kTmaNodes + 3 * t;
            const float* xo = S + kStX + 4 * kXRowS + 3 * (t + 1);  // this node's own x (row dy = dz = 0)
            if (MODE == FM_APPLY) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = fixed_bit(msk, c) ? 0.f : y[c];
                    a.out[3 * n + c] = v;
                    if (DOT) dotv.add_prod(xo[c], v);
                }
            } else if (MODE == FM_RESID) {
#pragma unroll
                for (int c = 0; c < 3; ++c) a.out[3 * n + c] = fixed_bit(msk, c) ? 0.f : bb[c] - y[c];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float xn = 0.f, dn = 0.f;
                    if (!fixed_bit(msk, c)) {
                        dn = ca * iv[c] * (bb[c] - y[c]);
                        if (need_d) dn = fmaf(cd, dd[c], dn);
                        xn = xo[c] + dn;
                        if (DOT) dotv.add_prod(bb[c], xn);
                    }
                    a.out[3 * n + c] = xn;
                    if (a.dnew) a.dnew[3 * n + c] = dn;
                }
            }
        }
        __syncthreads();  // stage st is free for tile + 2 * gridDim.x
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    if (DOT) {
        const double s2 = block_sum<kPipeThreads>(dotv.value(), tid);
        if (tid == 0) a.partial[blockIdx.x] = s2;
    }
}

// Assembled levels, "K-split" form: a block of 256 threads takes 256/NS
// consecutive nodes; its NS slices each apply every NS-th of a node's 27 blocks
// (diagonal, 13 forward, 13 transposed backward), so each thread issues ~324/NS
// loads instead of ~324, all independent, and every plane read is coalesced
// across the block's nodes.  The partial rows are added in shared memory in a
// fixed order.
template <int MODE, bool DOT, int NS>
__global__ void __launch_bounds__(256) k_bsr_ks(BsrArgs a) {
    pdl_entry();
    constexpr int NPB = 256 / NS;
    constexpr int NQ = (27 + NS - 1) / NS;
    __shared__ float part[NS][NPB][3];
    const int nn = (int)a.nn;
    const int t = threadIdx.x % NPB, slice = threadIdx.x / NPB;
    const int n = blockIdx.x * NPB + t;
    const bool live = n < nn;
    const int nsafe = live ? n : 0;
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int i = nsafe % NX, j = (nsafe / NX) % NY, k = nsafe / (NX * NY);
    const long long N = a.ps;
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int blk = slice + NS * q;  // 0..13 forward (u = blk), 14..26 backward (u = blk - 13)
        if (blk < 27) {
            const bool fwd = blk < 14;
            const int u = fwd ? blk : blk - 13;
            const int sl = 13 + u;
            const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
            const int off = dx + NX * (dy + NY * dz);
            const int sx = fwd ? dx : -dx, sy = fwd ? dy : -dy, sz = fwd ? dz : -dz;
            const bool ok = live && i + sx >= 0 && i + sx < NX && j + sy >= 0 && j + sy < NY && k + sz >= 0 && k + sz < NZ;
            const int m = (int)GMG_B(ok ? (fwd ? nsafe + off : nsafe - off) : nsafe, nn, 203);
            const float wgt = ok ? 1.f : 0.f;
            // operator and iterate through the read-only data path
            const float v0 = wgt * __ldg(a.xin + 3 * m), v1 = wgt * __ldg(a.xin + 3 * m + 1),
                        v2 = wgt * __ldg(a.xin + 3 * m + 2);
            const float* A = a.A + (long long)(u * 9) * N + (fwd ? nsafe : m);
            if (fwd) {
                y0 = fmaf(__ldg(A + 0 * N), v0, fmaf(__ldg(A + 1 * N), v1, fmaf(__ldg(A + 2 * N), v2, y0)));
                y1 = fmaf(__ldg(A + 3 * N), v0, fmaf(__ldg(A + 4 * N), v1, fmaf(__ldg(A + 5 * N), v2, y1)));
                y2 = fmaf(__ldg(A + 6 * N), v0, fmaf(__ldg(A + 7 * N), v1, fmaf(__ldg(A + 8 * N), v2, y2)));
            } else {
                y0 = fmaf(__ldg(A + 0 * N), v0, fmaf(__ldg(A + 3 * N), v1, fmaf(__ldg(A + 6 * N), v2, y0)));
                y1 = fmaf(__ldg(A + 1 * N), v0, fmaf(__ldg(A + 4 * N), v1, fmaf(__ldg(A + 7 * N), v2, y1)));
                y2 = fmaf(__ldg(A + 2 * N), v0, fmaf(__ldg(A + 5 * N), v1, fmaf(__ldg(A + 8 * N), v2, y2)));
            }
        }
    }
    part[slice][t][0] = y0;
    part[slice][t][1] = y1;
    part[slice][t][2] = y2;
    __syncthreads();
    DSAcc dotv;
    if (slice == 0 && live) {
        float y[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = part[0][t][c];
#pragma unroll
            for (int q = 1; q < NS; ++q) acc += part[q][t][c];
            y[c] = acc;
        }
        bsr_epilogue<MODE, DOT>(a, n, y, dotv);
    }
    if (DOT) {
        const double s2 = block_sum<256>(dotv.value(), threadIdx.x);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s2;
    }
}

__global__ void k_bsr_smooth0(BsrArgs a) {
    pdl_entry();
    const float ca = (float)a.coef[1];
    const long long n3 = 3 * a.nn;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
         q += (long long)gridDim.x * blockDim.x) {
        const float v = ca * a.invdiag[q] * a.b[q];  // invdiag is 0 on fixed DOFs
        a.out[q] = v;
        if (a.dnew) a.dnew[q] = v;
    }
}

// ---------------------------------------------------------------------------
// Transfers (Eq. trilinear_weights): per axis a coarse node I receives fine
// node 2I with weight 1 and 2I-1, 2I+1 with weight 1/2; when the fine count is
// odd, the last fine node 2*nc+1 hangs on coarse node nc with weight 1.
// ---------------------------------------------------------------------------
// Branch-free 1D stencils: every candidate entry is present, with weight 0 and
// a clamped index when it does not exist, so all loads of a node are
// independent and issue together.
__device__ __forceinline__ void fine_support3(int I, int nf, int idx[3], float w[3]) {
    const int nc = nf >> 1, f = 2 * I + 1;
    idx[0] = I >= 1 ? 2 * I - 1 : 2 * I; w[0] = I >= 1 ? 0.5f : 0.f;
    idx[1] = 2 * I; w[1] = 1.f;
    idx[2] = f <= nf ? f : 2 * I; w[2] = f <= nf ? (f < 2 * nc ? 0.5f : 1.f) : 0.f;
}

__device__ __forceinline__ void coarse_parents2(int f, int nf, int idx[2], float w[2]) {
    const int nc = nf >> 1;
    if ((f & 1) == 0) { idx[0] = idx[1] = f >> 1; w[0] = 1.f; w[1] = 0.f; }
    else if (f < 2 * nc) { idx[0] = (f - 1) >> 1; idx[1] = (f + 1) >> 1; w[0] = w[1] = 0.5f; }
    else { idx[0] = idx[1] = nc; w[0] = 1.f; w[1] = 0.f; }
}

// b_c = P^T t at coarse node n (masked), the restriction of Eq. vcycle.
__device__ __forceinline__ void restrict_node(int n, int fnx, int fny, int fnz, int fpx, int cnx, int cny,
                                              const uint8_t* cmask, const float* fine, float out[3]) {
    const int CX = cnx + 1, CY = cny + 1;
    const int FX = fpx, FY = fny + 1;  // fine vectors: fpx nodes per row
    const int I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    fine_support3(I, fnx, ix, wx);
    fine_support3(J, fny, iy, wy);
    fine_support3(K, fnz, iz, wz);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float w = wx[a] * wy[b] * wz[c];
                const int f = (int)GMG_B(ix[a] + FX * (iy[b] + FY * iz[c]), (long long)FX * FY * (fnz + 1), 211);
                s0 = fmaf(w, fine[3 * f], s0);
                s1 = fmaf(w, fine[3 * f + 1], s1);
                s2 = fmaf(w, fine[3 * f + 2], s2);
            }
    const uint8_t m = cmask[n];
    out[0] = fixed_bit(m, 0) ? 0.f : s0;
    out[1] = fixed_bit(m, 1) ? 0.f : s1;
    out[2] = fixed_bit(m, 2) ? 0.f : s2;
}

// The same restriction for small coarse levels, one coarse node per warp: lane
// a + 3 b + 9 c (< 27) takes the weighted fine node (a, b, c) of the node's
// 3 x 3 x 3 support, and the warp adds the 27 terms in a fixed butterfly order
// (every lane ends with the sums).  With a thread per node these levels leave
// the GPU nearly idle while each thread walks 27 dependent loads.
__device__ __forceinline__ void fine_support1(int I, int nf, int a, int& idx, float& w) {
    const int nc = nf >> 1, f = 2 * I + 1;
    if (a == 0) {
        idx = I >= 1 ? 2 * I - 1 : 2 * I;
        w = I >= 1 ? 0.5f : 0.f;
    } else if (a == 1) {
        idx = 2 * I;
        w = 1.f;
    } else {
        idx = f <= nf ? f : 2 * I;
        w = f <= nf ? (f < 2 * nc ? 0.5f : 1.f) : 0.f;
    }
}
__device__ __forceinline__ void restrict_node_warp(int n, int lane, int fnx, int fny, int fnz, int fpx, int cnx,
                                                   int cny, const uint8_t* cmask, const float* fine, float out[3]) {
    const int CX = cnx + 1, CY = cny + 1;
    const int FX = fpx, FY = fny + 1;  // fine vectors: fpx nodes per row
    const int I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    if (lane < 27) {
        int ix, iy, iz;
        float wx, wy, wz;
        fine_support1(I, fnx, lane % 3, ix, wx);
        fine_support1(J, fny, (lane / 3) % 3, iy, wy);
        fine_support1(K, fnz, lane / 9, iz, wz);
        const float w = wx * wy * wz;
        const int f = (int)GMG_B(ix + FX * (iy + FY * iz), (long long)FX * FY * (fnz + 1), 217);
        s0 = __fmul_rn(w, __ldg(fine + 3 * f));
        s1 = __fmul_rn(w, __ldg(fine + 3 * f + 1));
        s2 = __fmul_rn(w, __ldg(fine + 3 * f + 2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 = __fadd_rn(s0, __shfl_xor_sync(0xffffffffu, s0, o));
        s1 = __fadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
        s2 = __fadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, o));
    }
    const uint8_t m = cmask[n];
    out[0] = fixed_bit(m, 0) ? 0.f : s0;
    out[1] = fixed_bit(m, 1) ? 0.f : s1;
    out[2] = fixed_bit(m, 2) ? 0.f : s2;
}

// The restriction fused with the first smoothing step of the coarse level from
// a zero iterate: b_c = P^T t (stored, later steps and the residual read it),
// then x = c_a D^-1 b_c (and the Chebyshev increment d = x), with the same
// arithmetic as k_restrict followed by k_bsr_smooth0.
__global__ void k_restrict_smooth0(int fnx, int fny, int fnz, int fpx, const float* fine, BsrArgs a, float* bout) {
    pdl_entry();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int)a.nn) return;
    float bc[3];
    restrict_node(n, fnx, fny, fnz, fpx, a.nx, a.ny, a.mask, fine, bc);
    const float ca = (float)a.coef[1];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = 3LL * n + c;
        bout[q] = bc[c];
        const float v = ca * a.invdiag[q] * bc[c];  // invdiag is 0 on fixed DOFs
        a.out[q] = v;
        if (a.dnew) a.dnew[q] = v;
    }
}

__global__ void k_restrict(int fnx, int fny, int fnz, int fpx, int cnx, int cny, int cnz, const uint8_t* cmask,
                           const float* fine, float* coarse) {
    pdl_entry();
    const int nn = (cnx + 1) * (cny + 1) * (cnz + 1);
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    float bc[3];
    restrict_node(n, fnx, fny, fnz, fpx, cnx, cny, cmask, fine, bc);
    coarse[3 * n] = bc[0];
    coarse[3 * n + 1] = bc[1];
    coarse[3 * n + 2] = bc[2];
}

constexpr int kRwWarps = 8;  // coarse nodes per block of the warp-per-node restrictions

__global__ void __launch_bounds__(32 * kRwWarps) k_restrict_smooth0_w(int fnx, int fny, int fnz, int fpx,
                                                                     const float* fine, BsrArgs a, float* bout) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int n = blockIdx.x * kRwWarps + (threadIdx.x >> 5);
    if (n >= (int)a.nn) return;  // whole warps leave together
    float bc[3];
    restrict_node_warp(n, lane, fnx, fny, fnz, fpx, a.nx, a.ny, a.mask, fine, bc);
    if (lane < 3) {
        const int c = lane;
        const long long q = 3LL * n + c;
        const float v0 = c == 0 ? bc[0] : (c == 1 ? bc[1] : bc[2]);
        bout[q] = v0;
        const float v = __fmul_rn(__fmul_rn((float)a.coef[1], a.invdiag[q]), v0);  // invdiag is 0 on fixed DOFs
        a.out[q] = v;
        if (a.dnew) a.dnew[q] = v;
    }
}

__global__ void __launch_bounds__(32 * kRwWarps) k_restrict_w(int fnx, int fny, int fnz, int fpx, int cnx, int cny,
                                                              int cnz, const uint8_t* cmask, const float* fine,
                                                              float* coarse) {
    pdl_entry();
    const int nn = (cnx + 1) * (cny + 1) * (cnz + 1);
    const int lane = threadIdx.x & 31;
    const int n = blockIdx.x * kRwWarps + (threadIdx.x >> 5);
    if (n >= nn) return;
    float bc[3];
    restrict_node_warp(n, lane, fnx, fny, fnz, fpx, cnx, cny, cmask, fine, bc);
    if (lane < 3) coarse[3 * n + lane] = lane == 0 ? bc[0] : (lane == 1 ? bc[1] : bc[2]);
}

__global__ void k_prolong_add(int fnx, int fny, int fnz, int fpx, int cnx, int cny, const uint8_t* fmask,
                              const float* coarse, float* fine) {
    pdl_entry();
    const int FX = fnx + 1, FY = fny + 1, nn = FX * FY * (fnz + 1);
    const int CX = cnx + 1, CY = cny + 1;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const int i = n % FX, j = (n / FX) % FY, k = n / (FX * FY);
    int ix[2], iy[2], iz[2];
    float wx[2], wy[2], wz[2];
    coarse_parents2(i, fnx, ix, wx);
    coarse_parents2(j, fny, iy, wy);
    coarse_parents2(k, fnz, iz, wz);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float w = wx[a] * wy[b] * wz[c];
                const int m = (int)GMG_B(ix[a] + CX * (iy[b] + CY * iz[c]), (long long)CX * CY * (fnz / 2 + 1), 212);
                s0 = fmaf(w, coarse[3 * m], s0);
                s1 = fmaf(w, coarse[3 * m + 1], s1);
                s2 = fmaf(w, coarse[3 * m + 2], s2);
            }
    const uint8_t msk = fmask[n];
    const int np = (int)GMG_B(i + fpx * (j + FY * k), (long long)fpx * FY * (fnz + 1), 213);  // fine vector numbering
    if (!fixed_bit(msk, 0)) fine[3 * np] += s0;
    if (!fixed_bit(msk, 1)) fine[3 * np + 1] += s1;
    if (!fixed_bit(msk, 2)) fine[3 * np + 2] += s2;
}

// The same for a fine level whose rows are padded to a multiple of 4 nodes
// (level 0): a thread takes 4 x-consecutive fine nodes of a row, whose x-parents
// are among 3 coarse nodes, so that each coarse value is loaded once per group
// instead of once per fine node and weight; the fine row segment (12 floats,
// 16-byte aligned) moves as 3 float4.  Per node the weights, parents and the
// order of the sum are those of k_prolong_add, so the results are bitwise equal.
__global__ void k_prolong_add4(int fnx, int fny, int fnz, int fpx, int cnx, int cny, const uint8_t* fmask,
                               const float* coarse, float* fine) {
    pdl_entry();
    const int FX = fnx + 1, FY = fny + 1, NZ = fnz + 1;
    const int CX = cnx + 1, CY = cny + 1;
    const int G = (FX + 3) / 4;  // groups per row
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * FY * NZ) return;
    const int q = t % G, r = t / G, j = r % FY, k = r / FY;
    const int i0 = 4 * q, xb = 2 * q;  // x-parents of the group lie in xb .. xb + 2
    int iy[2], iz[2];
    float wy[2], wz[2];
    coarse_parents2(j, fny, iy, wy);
    coarse_parents2(k, fnz, iz, wz);
    [[maybe_unused]] const long long cn = (long long)CX * CY * (fnz / 2 + 1);  // bounds of the checked build
    // coarse values cv[c][b][x - xb][comp] of the group's parents
    float cv[2][2][3][3];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const bool zdup = c == 1 && iz[1] == iz[0], ydup = b == 1 && iy[1] == iy[0];
            if (zdup || ydup) {  // the same parent row as one already loaded
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int m = 0; m < 3; ++m) cv[c][b][x][m] = zdup ? cv[0][b][x][m] : cv[c][0][x][m];
                continue;
            }
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const int cx = min(xb + x, CX - 1);
                const int mi = (int)GMG_B(cx + CX * (iy[b] + CY * iz[c]), cn, 214);
#pragma unroll
                for (int m = 0; m < 3; ++m) cv[c][b][x][m] = __ldg(coarse + 3 * mi + m);
            }
        }
    const long long row = (long long)fpx * (j + (long long)FY * k);
    float4* seg = reinterpret_cast<float4*>(fine + 3 * GMG_B(row + i0, (long long)fpx * FY * NZ, 215));
    float f[12];
    {
        const float4 a = seg[0], b = seg[1], c = seg[2];
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y;
        f[6] = b.z; f[7] = b.w; f[8] = c.x; f[9] = c.y; f[10] = c.z; f[11] = c.w;
    }
    const long long nrow = (long long)FX * (j + (long long)FY * k);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= FX) break;  // pad nodes stay 0
        int ix[2];
        float wx[2];
        coarse_parents2(i, fnx, ix, wx);  // (parents xb + x below; only the weights are used)
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float w = wx[a] * wy[b] * wz[c];
                    // the parent's slot among the group's three: u / 2 for an even
                    // node (both weights on it), u's two neighbours for an odd one
                    // (at the clamped end of an odd row the second weight is 0)
                    const int x = (a == 0 || !(u & 1)) ? (u >> 1) : ((u + 1) >> 1);
                    s0 = fmaf(w, cv[c][b][x][0], s0);
                    s1 = fmaf(w, cv[c][b][x][1], s1);
                    s2 = fmaf(w, cv[c][b][x][2], s2);
                }
        const uint8_t msk = fmask[GMG_B(nrow + i, (long long)FX * FY * NZ, 216)];
        if (!fixed_bit(msk, 0)) f[3 * u] += s0;
        if (!fixed_bit(msk, 1)) f[3 * u + 1] += s1;
        if (!fixed_bit(msk, 2)) f[3 * u + 2] += s2;
    }
    seg[0] = make_float4(f[0], f[1], f[2], f[3]);
    seg[1] = make_float4(f[4], f[5], f[6], f[7]);
    seg[2] = make_float4(f[8], f[9], f[10], f[11]);
}

// x[free_idx[i]] = sum_j Ainv[i][j] b[free_idx[j]]  (FP64 accumulation), and
// x = 0 on the fixed DOFs (mask; no separate memset): the gathered right-hand
// side is staged in shared memory once per block, then each warp reduces a few
// rows of the inverse.  (Giving each row 128 threads measured
// the same for one 100^3 solve and 5 % slower for a batch of 128 small solves
// running concurrently, whose blocks then repeat the staging four times as often.)
constexpr int kCoarseRowsPerBlock = 8;
__global__ void __launch_bounds__(256) k_coarse_solve(int nL, const int* free_idx, const double* Ainv, const float* b,
                                                      float* x, const uint8_t* mask, int n_nodes) {
    pdl_entry();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 3 * n_nodes; j += gridDim.x * blockDim.x)
        if (fixed_bit(mask[j / 3], j % 3)) x[j] = 0.f;
    extern __shared__ double bs[];
    for (int j = threadIdx.x; j < nL; j += blockDim.x) bs[j] = (double)b[GMG_B(free_idx[j], 3LL * n_nodes, 231)];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kCoarseRowsPerBlock + warp;
    if (row >= nL) return;
    const double* rp = Ainv + (long long)row * nL;
    double s0 = 0.0, s1 = 0.0;
    int jx = lane;
    for (; jx + 32 < nL; jx += 64) {
        s0 = fma(rp[jx], bs[jx], s0);
        s1 = fma(rp[jx + 32], bs[jx + 32], s1);
    }
    if (jx < nL) s0 = fma(rp[jx], bs[jx], s0);
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[GMG_B(free_idx[row], 3LL * n_nodes, 232)] = (float)s;
}

// ---------------------------------------------------------------------------
// Vector kernels (grid-stride over a fixed grid, so the partial layout and the
// summation order are independent of timing).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads) k_dot_f32(const float* a, const float* b, long long n, double* partial) {
    pdl_entry();
    DSAcc acc;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < n; q += (long long)gridDim.x * kVecThreads)
        acc.add_prod(a[q], b[q]);
    const double s = block_sum<kVecThreads>(acc.value(), threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_dot_f64_masked(const double* a, const double* b, const uint8_t* mask,
                                                                long long nn, double* partial) {
    pdl_entry();
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * kVecThreads)
        if (!fixed_bit(mask[q / 3], (int)(q % 3))) s += a[q] * b[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_finalize(const double* partial, int n, double* sc, int slot, int op) {
    pdl_entry();
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += kVecThreads) s += partial[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) {
        sc[slot] = s;
        if (op == FIN_ALPHA) {
            sc[SC_ALPHA] = sc[SC_RZ] / s;
        } else if (op == FIN_BETA) {
            sc[SC_BETA] = s / sc[SC_RZ];
            sc[SC_RZ] = s;
        } else if (op == FIN_NRMCHK) {
            if (!(s > 0.0) || !isfinite(s)) sc[SC_TMP] = 1.0;  // sticky: power iterate vanished
        }
    }
}

// alpha = r.z / p.q (already in sc), r -= alpha q with ||r||^2 partials, and
// the step alpha p added to the double-float correction (wh + wl, level-0
// layout) that stands for the FP64 iterate's change since its last flush
// (k_flush_w): the product by the FP64 alpha is formed exactly as
// ah p + (al p + e) (alpha = ah + al in FP32 parts, e the FMA error of ah p)
// and added with a TwoSum, so the FP64 pipe, a small fraction of the FP32 rate
// on this part, takes no work per entry.  16-byte accesses over whole padded
// rows (pad entries of r, p, q and w are zero, and zero terms leave the ||r||^2
// accumulator unchanged).
__global__ void __launch_bounds__(kVecThreads) k_pcg_update(float* __restrict__ wh, float* __restrict__ wl,
                                                            float* __restrict__ r, const float* __restrict__ p,
                                                            const float* __restrict__ q, long long n4,
                                                            const double* sc, double* partial) {
    pdl_entry();
    const double alpha = sc[SC_ALPHA];
    const float af = (float)alpha;
    const float ah = af, al = (float)(alpha - (double)ah);
    DSAcc acc;
    const long long stride = (long long)gridDim.x * kVecThreads;
    for (long long i = blockIdx.x * (long long)kVecThreads + threadIdx.x; i < n4; i += stride) {
        const float4 pv = reinterpret_cast<const float4*>(p)[i];
        const float4 qv = reinterpret_cast<const float4*>(q)[i];
        const float4 rv = reinterpret_cast<const float4*>(r)[i];
        const float4 hv = reinterpret_cast<const float4*>(wh)[i];
        const float4 lv = reinterpret_cast<const float4*>(wl)[i];
        const float pa[4] = {pv.x, pv.y, pv.z, pv.w}, qa[4] = {qv.x, qv.y, qv.z, qv.w};
        float ra[4] = {rv.x, rv.y, rv.z, rv.w}, ha[4] = {hv.x, hv.y, hv.z, hv.w}, la[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            // w += alpha p in double-float
            const float ph = __fmul_rn(ah, pa[t]);
            const float pl = __fmaf_rn(al, pa[t], __fmaf_rn(ah, pa[t], -ph));
            const float s = __fadd_rn(ha[t], ph);
            const float bb = __fsub_rn(s, ha[t]);
            const float e = __fadd_rn(__fsub_rn(ha[t], __fsub_rn(s, bb)), __fsub_rn(ph, bb));
            const float lo = __fadd_rn(la[t], __fadd_rn(pl, e));
            ha[t] = __fadd_rn(s, lo);
            la[t] = __fsub_rn(lo, __fsub_rn(ha[t], s));
            ra[t] = fmaf(-af, qa[t], ra[t]);
            acc.add_prod(ra[t], ra[t]);
        }
        reinterpret_cast<float4*>(r)[i] = make_float4(ra[0], ra[1], ra[2], ra[3]);
        reinterpret_cast<float4*>(wh)[i] = make_float4(ha[0], ha[1], ha[2], ha[3]);
        reinterpret_cast<float4*>(wl)[i] = make_float4(la[0], la[1], la[2], la[3]);
    }
    const double sum = block_sum<kVecThreads>(acc.value(), threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = sum;
}

// u (dense numbering, FP64) += wh + wl (level-0 layout), then w = 0: the PCG
// steps since the last flush, added to the FP64 iterate once.
__global__ void k_flush_w(double* u, float* wh, float* wl, int NX, int px, long long n) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long row = i / rowd;
        const long long j = GMG_B(i + row * (rowp - rowd), n / rowd * rowp, 226);
        u[i] = u[i] + (f2d_exact(wh[j]) + f2d_exact(wl[j]));
        wh[j] = 0.f;
        wl[j] = 0.f;
    }
}

// p = z + beta p; four consecutive entries per thread and iteration with 16-byte
// accesses when both pointers are 16-byte aligned (vec4), the tail one by one.
__global__ void k_p_update(float* p, const float* z, long long n, const double* sc, int vec4) {
    pdl_entry();
    const float beta = (float)sc[SC_BETA];
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec4) {
        const long long n4 = n / 4;
        float4* p4 = reinterpret_cast<float4*>(p);
        const float4* z4 = reinterpret_cast<const float4*>(z);
        for (long long i = t0; i < n4; i += step) {
            float4 v = p4[i];
            const float4 w = z4[i];
            v.x = fmaf(beta, v.x, w.x);
            v.y = fmaf(beta, v.y, w.y);
            v.z = fmaf(beta, v.z, w.z);
            v.w = fmaf(beta, v.w, w.w);
            p4[i] = v;
        }
        done = 4 * n4;
    }
    for (long long i = done + t0; i < n; i += step) p[i] = fmaf(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(kVecThreads) k_mask_u64(double* u, const uint8_t* mask, long long nn, double* partial) {
    pdl_entry();
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * kVecThreads) {
        if (fixed_bit(mask[q / 3], (int)(q % 3))) u[q] = 0.0;
        else if (u[q] != 0.0) s += 1.0;
    }
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// y += sign * (*coef) * x (FP32 vectors, coefficient from device memory).
__global__ void k_axpy_dev(float* y, const float* x, long long n, const double* coef, float sign) {
    pdl_entry();
    const float c = sign * (float)coef[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(c, x[i], y[i]);
}

// u (dense numbering) += a * z (a level-0 vector of pitch px), accumulated in FP64.
__global__ void k_axpy_u64(double* u, const float* z, int NX, int px, long long n, double a) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long row = i / rowd;
        u[i] = fma(a, f2d_exact(z[GMG_B(i + row * (rowp - rowd), n / rowd * rowp, 225)]), u[i]);
    }
}

// ||r||^2 from the partial sums (the same sum as k_finalize into SC_RR), then
// the convergence test of the device-resident loop in the same launch.
__global__ void __launch_bounds__(kVecThreads) k_finalize_check(const double* partial, int n, double* sc,
                                                                cudaGraphConditionalHandle cond) {
    pdl_entry();
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += kVecThreads) s += partial[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x != 0) return;
    sc[SC_RR] = s;
    const double k = sc[SC_IT] + 1.0;
    sc[SC_IT] = k;
    const double relr = sqrt(s) / sc[SC_NF];
    const bool go = isfinite(relr) && isfinite(sc[SC_ALPHA]) && !(relr < sc[SC_TOL]) && k < sc[SC_MAXIT];
    cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// r = f on free DOFs (as FP32), 0 on fixed ones and on the pads: the residual of
// the zero iterate.  f dense; r and maskp in the level-0 vector numbering.
__global__ void __launch_bounds__(kVecThreads) k_cast_masked(const double* f, const uint8_t* maskp, int NX, int px,
                                                             long long nnp, float* r) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < 3 * nnp; q += (long long)gridDim.x * kVecThreads) {
        const long long row = q / rowp;
        const int c = (int)(q - row * rowp);
        r[q] = (c >= rowd || fixed_bit(maskp[q / 3], c % 3)) ? 0.f
                                                             : (float)f[GMG_B(row * rowd + c, nnp / px * rowd, 222)];
    }
}

// out = in with fixed DOFs and pads 0: in dense, out a level-0 vector.
__global__ void k_pack0(const float* in, const uint8_t* maskp, int NX, int px, long long nnp, float* out) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * nnp; q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / rowp;
        const int c = (int)(q - row * rowp);
        out[q] = (c >= rowd || fixed_bit(maskp[q / 3], c % 3)) ? 0.f : in[GMG_B(row * rowd + c, nnp / px * rowd, 223)];
    }
}

// out (dense) = in (a level-0 vector).
__global__ void k_unpack0(const float* in, int NX, int px, long long n, float* out) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / rowd;
        out[q] = in[GMG_B(q + row * (rowp - rowd), n / rowd * rowp, 224)];
    }
}

__global__ void k_scale_inv_sqrt(float* v, long long n, const double* sc, int slot) {
    pdl_entry();
    const double s = sc[slot];
    if (!(s > 0.0) || !isfinite(s)) return;
    const float f = (float)(1.0 / sqrt(s));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] *= f;
}

__device__ __forceinline__ float fine_diag(const float* E, int nx, int ny, int nz, int i, int j, int k, float kd) {
    float esum = 0.f;
#pragma unroll
    for (int ea = 0; ea < 8; ++ea) {
        const int ex = i - ldx(ea), ey = j - ldy(ea), ez = k - ldz(ea);
        if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz)
            esum += E[ex + (long long)nx * (ey + (long long)ny * ez)];
    }
    return kd * esum;
}

__global__ void k_scale_invdiag_fine(const float* y, float* w, const float* E, const uint8_t* mask, int nx, int ny,
                                     int nz, int px, float kd) {
    pdl_entry();
    const long long NX = nx + 1, NY = ny + 1, nn = NX * NY * (nz + 1);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        const float inv = jacobi_rcp(fine_diag(E, nx, ny, nz, i, j, k, kd));
        const uint8_t m = mask[n];
        const long long v = 3 * (i + px * (j + NY * k));
#pragma unroll
        for (int c = 0; c < 3; ++c) w[v + c] = fixed_bit(m, c) ? 0.f : inv * y[v + c];
    }
}

__global__ void k_scale_invdiag_bsr(const float* y, float* w, const float* invdiag, long long n) {
    pdl_entry();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        w[q] = invdiag[q] * y[q];
}

__global__ void __launch_bounds__(kVecThreads) k_diag_dot_fine(const float* v, const float* E, const uint8_t* mask, int nx,
                                                               int ny, int nz, int px, float kd, double* partial) {
    pdl_entry();
    const long long NX = nx + 1, NY = ny + 1, nn = NX * NY * (nz + 1);
    double s = 0.0;
    for (long long n = blockIdx.x * (long long)kVecThreads + threadIdx.x; n < nn; n += (long long)gridDim.x * kVecThreads) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        const double dg = fine_diag(E, nx, ny, nz, i, j, k, kd);
        const uint8_t m = mask[n];
        const long long q = 3 * (i + px * (j + NY * k));
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (!fixed_bit(m, c)) s += dg * (double)v[q + c] * (double)v[q + c];
    }
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_diag_dot_bsr(const float* v, const float* invdiag, long long n, double* partial) {
    pdl_entry();
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < n; q += (long long)gridDim.x * kVecThreads)
        if (invdiag[q] != 0.f) s += (double)v[q] * (double)v[q] / (double)invdiag[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Power-iteration start vector: v_i = ((i * 2654435761) mod 2^32) / 2^32 - 0.5 over
// the level's DOF index i, 0 on fixed DOFs.
__global__ void k_power_start(float* v, const uint8_t* mask, long long nn, int NX, int px) {
    pdl_entry();
    const int rowd = 3 * NX, rowp = 3 * px;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h = ((unsigned long long)q * 2654435761ull) & 0xffffffffull;
        const double val = (double)h / 4294967296.0 - 0.5;
        v[q + (q / rowd) * (rowp - rowd)] = fixed_bit(mask[q / 3], (int)(q % 3)) ? 0.f : (float)val;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_fine_inv0(int nx, int ny, int nz, int px, const float* E, float kd, float* inv0, cudaStream_t s) {
    note_launch();
    k_fine_inv0<<<kVecBlocks * 2, kVecThreads, 0, s>>>(nx, ny, nz, px, E, kd, inv0);
}

void launch_fine_smooth0(const FineArgs& a, cudaStream_t s) {
    note_launch();
    pdl_launch(k_fine_smooth0, dim3(kVecBlocks * 2), dim3(kVecThreads), 0, s, a);
}

// Standalone launches of the assembled-level operator.  Levels with tensor maps
// (bsr_tma_nodes option) use the TMA-staged kernel; otherwise levels of at
// least kBsrStreamLevel nodes stream with one thread per node and smaller ones,
// which are latency-bound, use the K-split form.
// (K-split slices measured at 100^3: 4 -> 7.78 ms per solve, 8 -> 7.63, 16 -> 7.68;
// the K-split form at level 1 instead of streaming: 8.20 ms.)
constexpr long long kBsrStreamLevel = 65536;
constexpr int kKsSlices = 8;

// Slices of the K-split kernel by level size: the most of 32 / 16 / 8 that keep
// the grid within kKsBlockBudget blocks of 256 threads (about four per SM).
// These levels are latency-bound, and spreading each node's 27 blocks over more
// threads puts more independent loads in flight; past the budget the extra
// blocks only queue.  Measured per level (autotuner, all five slice counts):
// 17,576 nodes -> 8 slices, 9,261 -> 16, 2,197 / 1,331 / 225 -> 32.
constexpr long long kKsBlockBudget = 4 * 148;
int ks_slices_for(long long nn) {
    for (int ns : {32, 16})
        if ((nn * ns + 255) / 256 <= kKsBlockBudget) return ns;
    return kKsSlices;
}

int pipe_blocks(long long nn) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
    }
    const long long tiles = (nn + kTmaNodes - 1) / kTmaNodes;
    return (int)std::min<long long>(tiles, sms);
}

// Slices per node of the level's kernel: 0 = the streaming kernel (one
// thread per node), else the K-split kernel with that many slices.  kind: -1
// by size (streaming from 65,536 nodes, below that ks_slices_for), 0 streaming,
// 1 / 2 / 3 / 4 / 5 K-split with 8 / 2 / 4 / 16 / 32 slices.
int bsr_slices(long long nn, int kind) {
    if (kind < 0) return nn >= kBsrStreamLevel ? 0 : ks_slices_for(nn);
    static const int kSlicesOfKind[kBsrKinds] = {0, 8, 2, 4, 16, 32};
    return (kind >= 0 && kind < kBsrKinds) ? kSlicesOfKind[kind] : kKsSlices;
}

int bsr_grid_blocks(long long nn, bool tma, int kind) {
    if (tma) return pipe_blocks(nn);
    const int ns = bsr_slices(nn, kind);
    const int npb = ns ? 256 / ns : 256;
    return (int)((nn + npb - 1) / npb);
}

template <int NS>
void launch_bsr_ks(int mode, int dot, int g, const BsrArgs& a, cudaStream_t s) {
    if (mode == FM_APPLY) {
        if (dot) pdl_launch(k_bsr_ks<FM_APPLY, true, NS>, dim3(g), dim3(256), 0, s, a);
        else pdl_launch(k_bsr_ks<FM_APPLY, false, NS>, dim3(g), dim3(256), 0, s, a);
    } else if (mode == FM_SMOOTH) {
        if (dot) pdl_launch(k_bsr_ks<FM_SMOOTH, true, NS>, dim3(g), dim3(256), 0, s, a);
        else pdl_launch(k_bsr_ks<FM_SMOOTH, false, NS>, dim3(g), dim3(256), 0, s, a);
    } else {
        pdl_launch(k_bsr_ks<FM_RESID, false, NS>, dim3(g), dim3(256), 0, s, a);
    }
}

template <int MODE, bool DOT>
void launch_bsr_tma(int g, const BsrArgs& a, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_bsr_pipe<MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemBytes);
        attr = true;
    }
    k_bsr_pipe<MODE, DOT><<<g, kPipeThreads, kPipeSmemBytes, s>>>(*a.tm_own, *a.tm_back, a);
}

void launch_bsr(int mode, int dot, const BsrArgs& a, cudaStream_t s) {
    if (a.kind == kBsrMatrixFree && a.eh && a.l1g && a.cf && !a.tm_own) {
        launch_l1mf(mode, dot, a, *a.l1g, a.cf, s);
        return;
    }
    note_launch();
    if (a.tm_own) {
        const int g = bsr_grid_blocks(a.nn, true);
        if (mode == FM_APPLY) {
            if (dot) launch_bsr_tma<FM_APPLY, true>(g, a, s);
            else launch_bsr_tma<FM_APPLY, false>(g, a, s);
        } else if (mode == FM_SMOOTH) {
            if (dot) launch_bsr_tma<FM_SMOOTH, true>(g, a, s);
            else launch_bsr_tma<FM_SMOOTH, false>(g, a, s);
        } else {
            launch_bsr_tma<FM_RESID, false>(g, a, s);
        }
        return;
    }
    const int g = bsr_grid_blocks(a.nn, false, a.kind);
    const int ns = bsr_slices(a.nn, a.kind);
    if (ns == 0) {
        if (mode == FM_APPLY) {
            if (dot) pdl_launch(k_bsr<FM_APPLY, true, 256>, dim3(g), dim3(256), 0, s, a);
            else pdl_launch(k_bsr<FM_APPLY, false, 256>, dim3(g), dim3(256), 0, s, a);
        } else if (mode == FM_SMOOTH) {
            if (dot) pdl_launch(k_bsr<FM_SMOOTH, true, 256>, dim3(g), dim3(256), 0, s, a);
            else pdl_launch(k_bsr<FM_SMOOTH, false, 256>, dim3(g), dim3(256), 0, s, a);
        } else {
            pdl_launch(k_bsr<FM_RESID, false, 256>, dim3(g), dim3(256), 0, s, a);
        }
        return;
    }
    if (ns == 8) launch_bsr_ks<8>(mode, dot, g, a, s);
    else if (ns == 2) launch_bsr_ks<2>(mode, dot, g, a, s);
    else if (ns == 16) launch_bsr_ks<16>(mode, dot, g, a, s);
    else if (ns == 32) launch_bsr_ks<32>(mode, dot, g, a, s);
    else launch_bsr_ks<4>(mode, dot, g, a, s);
}

bool encode_f32_map(CUtensorMap* map, const float* base, int rank, const unsigned long long* dims,
                    const unsigned* box) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode enc = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<Encode>(fn);
    });
    if (!enc || rank < 1 || rank > 2 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t gd[2] = {dims[0], rank > 1 ? dims[1] : 1};
    const cuuint64_t gs[1] = {dims[0] * sizeof(float)};
    const cuuint32_t bx[2] = {box[0], rank > 1 ? box[1] : 1};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), gd, gs, bx, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_f32_map_strided(CUtensorMap* map, const float* base, int rank, const unsigned long long* dims,
                            const unsigned long long* strides, const unsigned* box) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode enc = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<Encode>(fn);
    });
    if (!enc || rank < 1 || rank > 5 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    cuuint64_t gd[5], gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) {
            if (strides[i] % 16 != 0) return false;
            gs[i] = strides[i];
        }
    }
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), gd, gs, bx, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of a level's FP32 planes, [126][ps] row-major (x = node, y = plane):
// the own-block box (64 nodes x 126 planes) and the backward box (68 x 9).
int encode_bsr_maps(Level& l) {
    if (l.ps % 4 != 0) return GMG_ERR_ARG;
    const unsigned long long dims[2] = {(unsigned long long)l.ps, (unsigned long long)kSymPlanes};
    const unsigned box_own[2] = {(unsigned)kTmaNodes, (unsigned)kSymPlanes};
    const unsigned box_back[2] = {(unsigned)kTmaBackW, 9u};
    if (!encode_f32_map(&l.tm_own, l.A32, 2, dims, box_own)) return GMG_ERR_CUDA;
    if (!encode_f32_map(&l.tm_back, l.A32, 2, dims, box_back)) return GMG_ERR_CUDA;
    l.tma = true;
    return GMG_OK;
}

// Coarse levels below this many nodes restrict with a warp per coarse node.
constexpr long long kRestrictWarpNodes = 32768;

void launch_restrict_smooth0(const Level& f, const float* t, const BsrArgs& a, float* bout, cudaStream_t s) {
    note_launch();
    if (a.nn < kRestrictWarpNodes) {
        pdl_launch(k_restrict_smooth0_w, dim3((int)((a.nn + kRwWarps - 1) / kRwWarps)), dim3(32 * kRwWarps), 0, s, f.nx,
                   f.ny, f.nz, f.px, t, a, bout);
        return;
    }
    pdl_launch(k_restrict_smooth0, dim3((int)((a.nn + 127) / 128)), dim3(128), 0, s, f.nx, f.ny, f.nz, f.px, t, a, bout);
}

void launch_bsr_smooth0(const BsrArgs& a, cudaStream_t s) {
    const long long n3 = 3 * a.nn;
    const int g = (int)std::min<long long>((n3 + kVecThreads - 1) / kVecThreads, kVecBlocks * 2);
    note_launch();
    pdl_launch(k_bsr_smooth0, dim3(g), dim3(kVecThreads), 0, s, a);
}

static int grid_for(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, kVecBlocks * 2));
}

void launch_restrict(const Level& f, const Level& c, const float* fine, float* coarse, cudaStream_t s) {
    note_launch();
    if (c.nn < kRestrictWarpNodes) {
        pdl_launch(k_restrict_w, dim3((int)((c.nn + kRwWarps - 1) / kRwWarps)), dim3(32 * kRwWarps), 0, s, f.nx, f.ny,
                   f.nz, f.px, c.nx, c.ny, c.nz, c.mask, fine, coarse);
        return;
    }
    pdl_launch(k_restrict, dim3((int)((c.nn + 127) / 128)), dim3(128), 0, s, f.nx, f.ny, f.nz, f.px, c.nx, c.ny, c.nz, c.mask, fine,
               coarse);
}

void launch_prolong_add(const Level& f, const Level& c, const float* coarse, float* fine, cudaStream_t s) {
    note_launch();
    if (f.px % 4 == 0 && (reinterpret_cast<uintptr_t>(fine) & 15) == 0) {  // padded rows: 4-node groups
        const long long groups = (long long)((f.nx + 1 + 3) / 4) * (f.ny + 1) * (f.nz + 1);
        pdl_launch(k_prolong_add4, dim3((int)((groups + 255) / 256)), dim3(256), 0, s, f.nx, f.ny, f.nz, f.px, c.nx,
                   c.ny, f.mask, coarse, fine);
        return;
    }
    pdl_launch(k_prolong_add, dim3((int)((f.nn + 255) / 256)), dim3(256), 0, s, f.nx, f.ny, f.nz, f.px, c.nx, c.ny, f.mask, coarse,
               fine);
}

namespace {
__global__ void k_publish(const double* sc, int n, double* out, const int* e0, const int* e1, int* eout) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = sc[i];
    if (threadIdx.x == 0 && eout) {
        eout[0] = e0 ? *e0 : 0;
        eout[1] = e1 ? *e1 : 0;
    }
}

__global__ void k_publish_batch(const __grid_constant__ PublishBatch b) {
    const int item = blockIdx.x;
    if (item >= b.count) return;
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) b.out[item][i] = b.sc[item][i];
    if (threadIdx.x == 0) {
        b.eout[item][0] = b.e0[item] ? *b.e0[item] : 0;
        b.eout[item][1] = b.e1[item] ? *b.e1[item] : 0;
    }
}

__global__ void k_copy_f32(float* __restrict__ y, const float* __restrict__ x, long long n) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i];
}

__global__ void k_set_scalars(double* sc, int n, double v0, double v1, double v2, double v3) {
    const int i = threadIdx.x;
    if (i < n) sc[i] = i == 0 ? v0 : (i == 1 ? v1 : (i == 2 ? v2 : v3));
}
}  // namespace

void launch_publish(const double* sc, int n, double* out_map, const int* e0, const int* e1, int* err_map,
                    cudaStream_t s) {
    note_launch();
    k_publish<<<1, 32, 0, s>>>(sc, n, out_map, e0, e1, err_map);
}

void launch_copy_f32(float* y, const float* x, long long n, cudaStream_t s) {
    note_launch();
    const int g = (int)std::max<long long>(1, std::min<long long>((n + kVecThreads - 1) / kVecThreads, kVecBlocks));
    pdl_launch(k_copy_f32, dim3(g), dim3(kVecThreads), 0, s, y, x, n);
}

void launch_publish_batch(const PublishBatch& b, cudaStream_t s) {
    if (b.count <= 0) return;
    note_launch();
    k_publish_batch<<<b.count, 32, 0, s>>>(b);
}

void launch_set_scalars(double* sc, int n, double v0, double v1, double v2, double v3, cudaStream_t s) {
    note_launch();
    k_set_scalars<<<1, 32, 0, s>>>(sc, n, v0, v1, v2, v3);
}

void launch_coarse_solve(int nL, const int* free_idx, const double* Ainv, const float* b, float* x,
                         const uint8_t* mask, long long n_nodes, cudaStream_t s) {
    {
        const size_t smem = sizeof(double) * nL;
        if (smem > 48 * 1024) {  // coarsest levels above ~6,000 free DOFs (a raised chol_cutoff)
            static std::mutex mu;
            static size_t granted = 48 * 1024;
            std::lock_guard<std::mutex> lk(mu);
            if (smem > granted &&
                cudaFuncSetAttribute(k_coarse_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                    cudaSuccess)
                granted = smem;
        }
        note_launch();
        const int g = std::max(1, (nL + kCoarseRowsPerBlock - 1) / kCoarseRowsPerBlock);  // nL = 0: zeroes only
        pdl_launch(k_coarse_solve, dim3(g), dim3(32 * kCoarseRowsPerBlock), smem, s, nL, free_idx, Ainv, b, x, mask,
                   (int)n_nodes);
    }
}

int vec_grid_blocks() { return kVecBlocks; }

void launch_dot_f32(const float* a, const float* b, long long n, double* partial, cudaStream_t s) {
    note_launch();
    pdl_launch(k_dot_f32, dim3(kVecBlocks), dim3(kVecThreads), 0, s, a, b, n, partial);
}

void launch_dot_f64_masked(const double* a, const double* b, const uint8_t* mask, long long nn, double* partial,
                           cudaStream_t s) {
    note_launch();
    pdl_launch(k_dot_f64_masked, dim3(kVecBlocks), dim3(kVecThreads), 0, s, a, b, mask, nn, partial);
}

void launch_finalize(const double* partial, int n, double* sc, int slot, int op, cudaStream_t s) {
    note_launch();
    pdl_launch(k_finalize, dim3(1), dim3(kVecThreads), 0, s, partial, n, sc, slot, op);
}

void launch_pcg_update(float* wh, float* wl, float* r, const float* p, const float* q, const Level& l0,
                       const double* sc, double* partial, cudaStream_t s) {
    note_launch();
    pdl_launch(k_pcg_update, dim3(kVecBlocks), dim3(kVecThreads), 0, s, wh, wl, r, p, q, 3 * l0.nnp / 4, sc, partial);
}

void launch_flush_w(double* u, float* wh, float* wl, const Level& l0, cudaStream_t s) {
    note_launch();
    const long long n = 3 * l0.nn;
    pdl_launch(k_flush_w, dim3(grid_for(n)), dim3(256), 0, s, u, wh, wl, l0.nx + 1, l0.px, n);
}

void launch_p_update(float* p, const float* z, long long n, const double* sc, cudaStream_t s) {
    note_launch();
    const bool vec4 = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(z)) & 15) == 0;
    pdl_launch(k_p_update, dim3(grid_for(vec4 ? (n + 3) / 4 : n)), dim3(256), 0, s, p, z, n, sc, vec4 ? 1 : 0);
}

void launch_mask_u64(double* u, const uint8_t* mask, long long nn, double* partial, cudaStream_t s) {
    note_launch();
    pdl_launch(k_mask_u64, dim3(kVecBlocks), dim3(kVecThreads), 0, s, u, mask, nn, partial);
}

void launch_axpy_dev(float* y, const float* x, long long n, const double* coef, float sign, cudaStream_t s) {
    note_launch();
    pdl_launch(k_axpy_dev, dim3(grid_for(n)), dim3(256), 0, s, y, x, n, coef, sign);
}

void launch_axpy_u64(double* u, const float* z, const Level& l0, double a, cudaStream_t s) {
    note_launch();
    const long long n = 3 * l0.nn;
    pdl_launch(k_axpy_u64, dim3(grid_for(n)), dim3(256), 0, s, u, z, l0.nx + 1, l0.px, n, a);
}

void launch_finalize_check(const double* partial, int n, double* sc, cudaGraphConditionalHandle cond,
                           cudaStream_t s) {
    note_launch();
    pdl_launch(k_finalize_check, dim3(1), dim3(kVecThreads), 0, s, partial, n, sc, cond);
}

void launch_cast_masked(const double* f, const Level& l0, float* r, cudaStream_t s) {
    note_launch();
    pdl_launch(k_cast_masked, dim3(kVecBlocks), dim3(kVecThreads), 0, s, f, l0.maskp, l0.nx + 1, l0.px, l0.nnp, r);
}

void launch_pack0(const float* in, const Level& l0, float* out, cudaStream_t s) {
    note_launch();
    pdl_launch(k_pack0, dim3(grid_for(3 * l0.nnp)), dim3(256), 0, s, in, l0.maskp, l0.nx + 1, l0.px, l0.nnp, out);
}

void launch_unpack0(const float* in, const Level& l0, float* out, cudaStream_t s) {
    note_launch();
    pdl_launch(k_unpack0, dim3(grid_for(3 * l0.nn)), dim3(256), 0, s, in, l0.nx + 1, l0.px, 3 * l0.nn, out);
}

void launch_scale_by_inv_sqrt(float* v, long long n, const double* sc, int slot, cudaStream_t s) {
    note_launch();
    pdl_launch(k_scale_inv_sqrt, dim3(grid_for(n)), dim3(256), 0, s, v, n, sc, slot);
}

void launch_scale_invdiag_fine(const float* y, float* w, const float* E, const Level& l0, float kd, cudaStream_t s) {
    note_launch();
    k_scale_invdiag_fine<<<grid_for(l0.nn), 256, 0, s>>>(y, w, E, l0.mask, l0.nx, l0.ny, l0.nz, l0.px, kd);
}

void launch_scale_invdiag_bsr(const float* y, float* w, const float* invdiag, long long n, cudaStream_t s) {
    note_launch();
    k_scale_invdiag_bsr<<<grid_for(n), 256, 0, s>>>(y, w, invdiag, n);
}

void launch_diag_dot_fine(const float* v, const float* E, const Level& l0, float kd, double* partial, cudaStream_t s) {
    note_launch();
    k_diag_dot_fine<<<kVecBlocks, kVecThreads, 0, s>>>(v, E, l0.mask, l0.nx, l0.ny, l0.nz, l0.px, kd, partial);
}

void launch_diag_dot_bsr(const float* v, const float* invdiag, long long n, double* partial, cudaStream_t s) {
    note_launch();
    k_diag_dot_bsr<<<kVecBlocks, kVecThreads, 0, s>>>(v, invdiag, n, partial);
}

void launch_power_start(float* v, const Level& l, cudaStream_t s) {
    note_launch();
    k_power_start<<<grid_for(3 * l.nn), 256, 0, s>>>(v, l.mask, l.nn, l.nx + 1, l.px);
}

}  // namespace gmg
