// The lower part of the V-cycle (Eq. vcycle) -- every level from `start` down to
// the coarsest solve -- as one persistent cooperative kernel.
//
// These levels hold a few thousand nodes each, so as separate launches every
// step costs a kernel launch plus a few dependent memory round trips while the
// GPU is mostly idle.  Here all blocks stay resident and walk the same sequence
// of phases (smoothing steps, residual, restriction, coarsest solve,
// prolongation), separated by a grid-wide barrier.  The arithmetic of each
// phase is the same as the per-level kernels: one warp per node for the
// 27-point block operator (symmetric half storage), damped Jacobi / Chebyshev
// steps with the same coefficient tables, the branch-free trilinear transfers,
// and the FP64 coarsest solve.
//
// Vectors produced inside the kernel are read with ld.global.cg (L2 only), so
// no block can see a stale L1 copy from an earlier phase.
//
// The barrier is this file's own: an arrival counter and a generation word in
// global memory.  Waiting is bounded: after `spin_limit` polls a block records
// an error flag and leaves, so a fault can never turn into a hang (the host
// reports GMG_TIMEOUT when the flag is set, then clears the flag and the
// arrival counter).  The kernel is launched with
// cudaLaunchCooperativeKernel, which guarantees that all blocks are resident.
#include <algorithm>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

// Grid barrier with bounded waiting.  Returns false when the wait gave up.
__device__ __forceinline__ bool grid_barrier(const CoarseFused& a, unsigned& gen) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned target = gen + 1;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar_count, 1u) + 1;
        if (arrived == gridDim.x) {
            atomicExch(a.bar_count, 0u);
            __threadfence();
            atomicExch(a.bar_gen, target);
        } else {
            long long spins = 0;
            while (true) {
                const unsigned g = *((volatile unsigned*)a.bar_gen);
                if (g == target) break;
                if (++spins > a.spin_limit || *((volatile int*)a.err) != 0) {
                    atomicExch(a.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
    }
    __syncthreads();
    return ok != 0;
}

// Row n of a level's symmetric 27-point block operator applied to x, one warp
// per node: lanes 0..13 diagonal + forward blocks, lanes 14..26 backward blocks.
__device__ __forceinline__ void warp_row(const CoarseLevel& L, int n, const float* x, int lane, float y[3]) {
    const int NX = L.nx + 1, NY = L.ny + 1, NZ = L.nz + 1;
    const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
    const long long N = L.ps;
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
    if (lane < 27) {
        const bool fwd = lane < 14;
        const int u = fwd ? lane : lane - 13;
        const int sl = 13 + u;
        const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
        const int off = dx + NX * (dy + NY * dz);
        const int sx = fwd ? dx : -dx, sy = fwd ? dy : -dy, sz = fwd ? dz : -dz;
        const bool ok = i + sx >= 0 && i + sx < NX && j + sy >= 0 && j + sy < NY && k + sz >= 0 && k + sz < NZ;
        const int m = (int)GMG_B(ok ? (fwd ? n + off : n - off) : n, L.nn, 401);
        const float wgt = ok ? 1.f : 0.f;
        const float v0 = wgt * __ldcg(x + 3 * m), v1 = wgt * __ldcg(x + 3 * m + 1), v2 = wgt * __ldcg(x + 3 * m + 2);
        const float* A = L.A + (long long)(u * 9) * N + (fwd ? n : m);
        if (fwd) {
            y0 = fmaf(A[0 * N], v0, fmaf(A[1 * N], v1, A[2 * N] * v2));
            y1 = fmaf(A[3 * N], v0, fmaf(A[4 * N], v1, A[5 * N] * v2));
            y2 = fmaf(A[6 * N], v0, fmaf(A[7 * N], v1, A[8 * N] * v2));
        } else {
            y0 = fmaf(A[0 * N], v0, fmaf(A[3 * N], v1, A[6 * N] * v2));
            y1 = fmaf(A[1 * N], v0, fmaf(A[4 * N], v1, A[7 * N] * v2));
            y2 = fmaf(A[2 * N], v0, fmaf(A[5 * N], v1, A[8 * N] * v2));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
        y2 += __shfl_xor_sync(0xffffffffu, y2, o);
    }
    y[0] = y0; y[1] = y1; y[2] = y2;
}

// One smoother step on level L: out = x + d_new, d_new = c_d d + c_a D^-1 (b - K x);
// zero_init: x = 0 (no operator application).
__device__ void phase_smooth(const CoarseLevel& L, int step, bool zero_init, const float* b, const float* x,
                             float* out, bool write_d) {
    const float cd = (float)L.coef[2 * step], ca = (float)L.coef[2 * step + 1];
    if (zero_init) {
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * L.nn;
             q += (long long)gridDim.x * blockDim.x) {
            const float v = ca * L.invdiag[q] * __ldcg(b + q);
            out[q] = v;
            if (write_d) L.d[q] = v;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int n = gw; n < L.nn; n += nw) {
        float y[3];
        warp_row(L, n, x, lane, y);
        if (lane < 3) {
            const int c = lane;
            float xn = 0.f, dn = 0.f;
            if (!fixed_bit(L.mask[n], c)) {
                dn = ca * L.invdiag[3 * n + c] * (__ldcg(b + 3 * n + c) - y[c]);
                if (cd != 0.f) dn = fmaf(cd, __ldcg(L.d + 3 * n + c), dn);
                xn = __ldcg(x + 3 * n + c) + dn;
            }
            out[3 * n + c] = xn;
            if (write_d) L.d[3 * n + c] = dn;
        }
    }
}

__device__ void phase_resid(const CoarseLevel& L, const float* b, const float* x, float* t) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int n = gw; n < L.nn; n += nw) {
        float y[3];
        warp_row(L, n, x, lane, y);
        if (lane < 3) t[3 * n + lane] = fixed_bit(L.mask[n], lane) ? 0.f : __ldcg(b + 3 * n + lane) - y[lane];
    }
}

__device__ __forceinline__ void support3(int I, int nf, int idx[3], float w[3]) {
    const int nc = nf >> 1, f = 2 * I + 1;
    idx[0] = I >= 1 ? 2 * I - 1 : 2 * I; w[0] = I >= 1 ? 0.5f : 0.f;
    idx[1] = 2 * I; w[1] = 1.f;
    idx[2] = f <= nf ? f : 2 * I; w[2] = f <= nf ? (f < 2 * nc ? 0.5f : 1.f) : 0.f;
}

__device__ __forceinline__ void parents2(int f, int nf, int idx[2], float w[2]) {
    const int nc = nf >> 1;
    if ((f & 1) == 0) { idx[0] = idx[1] = f >> 1; w[0] = 1.f; w[1] = 0.f; }
    else if (f < 2 * nc) { idx[0] = (f - 1) >> 1; idx[1] = (f + 1) >> 1; w[0] = w[1] = 0.5f; }
    else { idx[0] = idx[1] = nc; w[0] = 1.f; w[1] = 0.f; }
}

__device__ void phase_restrict(const CoarseLevel& F, const CoarseLevel& C, const float* fine, float* coarse) {
    const int CX = C.nx + 1, CY = C.ny + 1, FX = F.nx + 1, FY = F.ny + 1;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < C.nn; n += gridDim.x * blockDim.x) {
        const int I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
        int ix[3], iy[3], iz[3];
        float wx[3], wy[3], wz[3];
        support3(I, F.nx, ix, wx);
        support3(J, F.ny, iy, wy);
        support3(K, F.nz, iz, wz);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const int f = ix[a] + FX * (iy[b] + FY * iz[c]);
                    s0 = fmaf(w, __ldcg(fine + 3 * f), s0);
                    s1 = fmaf(w, __ldcg(fine + 3 * f + 1), s1);
                    s2 = fmaf(w, __ldcg(fine + 3 * f + 2), s2);
                }
        const uint8_t m = C.mask[n];
        coarse[3 * n] = fixed_bit(m, 0) ? 0.f : s0;
        coarse[3 * n + 1] = fixed_bit(m, 1) ? 0.f : s1;
        coarse[3 * n + 2] = fixed_bit(m, 2) ? 0.f : s2;
    }
}

__device__ void phase_prolong_add(const CoarseLevel& F, const CoarseLevel& C, const float* coarse, float* fine) {
    const int FX = F.nx + 1, FY = F.ny + 1, CX = C.nx + 1, CY = C.ny + 1;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < F.nn; n += gridDim.x * blockDim.x) {
        const int i = n % FX, j = (n / FX) % FY, k = n / (FX * FY);
        int ix[2], iy[2], iz[2];
        float wx[2], wy[2], wz[2];
        parents2(i, F.nx, ix, wx);
        parents2(j, F.ny, iy, wy);
        parents2(k, F.nz, iz, wz);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const int m = ix[a] + CX * (iy[b] + CY * iz[c]);
                    s0 = fmaf(w, __ldcg(coarse + 3 * m), s0);
                    s1 = fmaf(w, __ldcg(coarse + 3 * m + 1), s1);
                    s2 = fmaf(w, __ldcg(coarse + 3 * m + 2), s2);
                }
        const uint8_t msk = F.mask[n];
        if (!fixed_bit(msk, 0)) fine[3 * n] = __ldcg(fine + 3 * n) + s0;
        if (!fixed_bit(msk, 1)) fine[3 * n + 1] = __ldcg(fine + 3 * n + 1) + s1;
        if (!fixed_bit(msk, 2)) fine[3 * n + 2] = __ldcg(fine + 3 * n + 2) + s2;
    }
}

// x = Ainv b on the free DOFs of the coarsest level (FP64), fixed DOFs 0.
__device__ void phase_coarse(const CoarseFused& a, const float* b, float* x, double* bs) {
    const CoarseLevel& L = a.lev[a.L - 1];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * L.nn;
         q += (long long)gridDim.x * blockDim.x)
        if (fixed_bit(L.mask[q / 3], (int)(q % 3))) x[q] = 0.f;
    const int nL = a.nL;
    for (int j = threadIdx.x; j < nL; j += blockDim.x) bs[j] = (double)__ldcg(b + a.free_idx[j]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = gw; row < nL; row += nw) {
        const double* rp = a.Ainv + (long long)row * nL;
        double s = 0.0;
        for (int jx = lane; jx < nL; jx += 32) s = fma(rp[jx], bs[jx], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[a.free_idx[row]] = (float)s;
    }
}

__global__ void __launch_bounds__(kThreads) k_coarse_vcycle(CoarseFused a) {
    extern __shared__ double bs[];
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = *((volatile unsigned*)a.bar_gen);
#define BARRIER() \
    do { if (!grid_barrier(a, gen)) return; } while (0)
    // descend: pre-smooth from zero, residual, restrict
    int writes[kMaxLevels];
    float* cur[kMaxLevels];
    for (int l = a.start; l < a.L - 1; ++l) {
        const CoarseLevel& L = a.lev[l];
        const bool cheb = L.kind == GMG_SMOOTHER_CHEBYSHEV;
        writes[l] = 0;
        cur[l] = nullptr;
        for (int k = 0; k < L.degree; ++k) {
            float* next = (writes[l] % 2 == 0) ? L.x2 : L.x;
            phase_smooth(L, k, k == 0, L.b, cur[l], next, cheb && k != L.degree - 1);
            cur[l] = next;
            ++writes[l];
            BARRIER();
        }
        phase_resid(L, L.b, cur[l], L.t);
        BARRIER();
        phase_restrict(L, a.lev[l + 1], L.t, a.lev[l + 1].b);
        BARRIER();
    }
    phase_coarse(a, a.lev[a.L - 1].b, a.lev[a.L - 1].x, bs);
    BARRIER();
    // ascend: prolong-add, post-smooth
    for (int l = a.L - 2; l >= a.start; --l) {
        const CoarseLevel& L = a.lev[l];
        const bool cheb = L.kind == GMG_SMOOTHER_CHEBYSHEV;
        phase_prolong_add(L, a.lev[l + 1], a.lev[l + 1].x, cur[l]);
        BARRIER();
        for (int k = 0; k < L.degree; ++k) {
            float* next = (writes[l] % 2 == 0) ? L.x2 : L.x;
            phase_smooth(L, k, false, L.b, cur[l], next, cheb && k != L.degree - 1);
            cur[l] = next;
            ++writes[l];
            if (!(l == a.start && k == L.degree - 1)) BARRIER();
        }
    }
#undef BARRIER
}

// ---------------------------------------------------------------------------
// Coarsest level above the dense-Cholesky cutoff: a fixed-count PCG
// (Sec. "Matrix-Free V-Cycle": Cholesky if n_L <= cutoff, else PCG; 80 steps in
// the reproducibility defaults) preconditioned by the level's diagonal, from
// x = 0.  Each step: q = K p (one warp per node, warp_row), alpha = rz / p.q,
// x += alpha p, r -= alpha q, z = D^-1 r, beta = r.z / rz, p = z + beta p; it
// stops early only when r.z is exactly 0.  One block of 1024 threads does all
// steps, so the phases are separated by __syncthreads alone (no grid-wide
// wait); vectors FP32, dot products accumulated in FP64.
// ---------------------------------------------------------------------------
constexpr int kCpThreads = 1024;

// Sum over the block of one FP64 value per thread; every thread gets the sum.
__device__ double cp_block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // sh may still be read from the previous sum
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < kCpThreads / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

__global__ void __launch_bounds__(kCpThreads, 1) k_coarse_pcg(CoarseLevel L, const float* b, float* x, float* r,
                                                               float* p, float* q, int steps) {
    __shared__ double sh[33];
    pdl_entry();
    const long long n3 = 3LL * L.nn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double rz_part = 0.0;
    for (long long i = threadIdx.x; i < n3; i += kCpThreads) {
        const float ri = b[i];
        const float zi = L.invdiag[i] * ri;  // 0 on fixed DOFs
        x[i] = 0.f;
        r[i] = ri;
        p[i] = zi;
        rz_part += (double)ri * (double)zi;
    }
    double rz = cp_block_sum(rz_part, sh);
    for (int k = 0; k < steps && rz != 0.0; ++k) {
        // q = K p and p.q
        double pq_part = 0.0;
        for (int n = warp; n < L.nn; n += kCpThreads / 32) {
            float y[3];
            warp_row(L, n, p, lane, y);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    q[3 * n + c] = y[c];
                    pq_part += (double)__ldcg(p + 3 * n + c) * (double)y[c];
                }
            }
        }
        const double pq = cp_block_sum(pq_part, sh);
        const float alpha = (float)(rz / pq);
        double rzn_part = 0.0;
        for (long long i = threadIdx.x; i < n3; i += kCpThreads) {
            x[i] = fmaf(alpha, p[i], x[i]);
            const float ri = fmaf(-alpha, q[i], r[i]);
            r[i] = ri;
            rzn_part += (double)ri * (double)(L.invdiag[i] * ri);
        }
        const double rzn = cp_block_sum(rzn_part, sh);
        const float beta = (float)(rzn / rz);
        rz = rzn;
        for (long long i = threadIdx.x; i < n3; i += kCpThreads) p[i] = fmaf(beta, p[i], L.invdiag[i] * r[i]);
        __syncthreads();
    }
}

}  // namespace

int coarse_fused_blocks(int* blocks_out, size_t shm) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GMG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GMG_ERR_CUDA;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return GMG_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_vcycle, kThreads, shm) != cudaSuccess)
        return GMG_ERR_CUDA;
    *blocks_out = sms * std::max(1, std::min(per_sm, 2));
    return GMG_OK;
}

void launch_coarse_pcg(const CoarseLevel& l, const float* b, float* x, float* r, float* p, float* q, int steps,
                       cudaStream_t s) {
    note_launch();
    pdl_launch(k_coarse_pcg, dim3(1), dim3(kCpThreads), 0, s, l, b, x, r, p, q, steps);
}

int launch_coarse_fused(const CoarseFused& a, int blocks, cudaStream_t s) {
    CoarseFused arg = a;
    void* params[] = {&arg};
    const size_t shm = sizeof(double) * (size_t)std::max(a.nL, 1);
    note_launch();
    return cudaLaunchCooperativeKernel((const void*)k_coarse_vcycle, dim3(blocks), dim3(kThreads), params, shm, s) ==
                   cudaSuccess
               ? GMG_OK
               : GMG_ERR_CUDA;
}

}  // namespace gmg
