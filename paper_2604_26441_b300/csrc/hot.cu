// Hot-path kernels of the GMG-preconditioned CG solver (sm_103a).
//
//  * k_fine_smooth0  -- first fine-level smoother step from zero (the fused
//                       fine operator lives in fine.cu, its FP64 residual form
//                       in resid64.cu);
//  * k_bsr           -- the same three modes on an assembled Galerkin level
//                       (27-point 3x3-block operator, implicit structured columns);
//  * k_restrict / k_prolong_add -- R = P^T and P of Eq. trilinear_weights /
//                       Eq. vector_prolongation with the odd-size clamp;
//  * k_coarse_solve  -- dense FP64 solve with the Cholesky-derived inverse;
//  * vector kernels  -- fused PCG updates and FP64-accumulated dot products
//                       (Sec. "Outer Krylov Solver and Convergence Statement").
//
// Reductions are deterministic: every block writes one partial sum, and a
// single-block finaliser adds the partials in a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 148 * 4;

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

// First smoother step from x = 0: x_1 = c_a D^{-1} b (no operator application).
__global__ void k_fine_smooth0(FineArgs a) {
    const long long NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const long long nn = NX * NY * NZ;
    const float ca = (float)a.coef[1];
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        float esum = 0.f;
#pragma unroll
        for (int ea = 0; ea < 8; ++ea) {
            const int ex = i - ldx(ea), ey = j - ldy(ea), ez = k - ldz(ea);
            if (ex >= 0 && ex < a.nx && ey >= 0 && ey < a.ny && ez >= 0 && ez < a.nz)
                esum += a.E[ex + (long long)a.nx * (ey + (long long)a.ny * ez)];
        }
        const float inv = 1.f / (a.kd * esum);
        const uint8_t m = a.mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fixed_bit(m, c) ? 0.f : ca * inv * a.b[3 * n + c];
            a.out[3 * n + c] = v;
            if (a.dnew) a.dnew[3 * n + c] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Assembled levels: K^l is symmetric, so only the diagonal block and the 13
// "forward" neighbour blocks (slots 13..26, offsets after the node in memory
// order) are stored, plane-major: A[(u*9 + r*3 + c)*nn + n] is entry (r, c) of
// block (n, n + o_u), u = slot - 13.  Row n of K^l is then
//   sum_u A_u(n) x(n + o_u)  +  sum_{u>0} A_u(n - o_u)^T x(n - o_u),
// one thread per node; every plane read is coalesced across consecutive nodes,
// and the transposed reads at n - o_u re-touch planes read a few blocks earlier
// (mostly L2 hits), so each stored value crosses HBM about once.
// ---------------------------------------------------------------------------
template <int MODE, bool DOT>
__global__ void __launch_bounds__(kVecThreads) k_bsr(BsrArgs a) {
    const int n = blockIdx.x * kVecThreads + threadIdx.x;
    const int nn = (int)a.nn;
    double dotv = 0.0;
    if (n < nn) {
        const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
        const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
        float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
        for (int u = 0; u < 14; ++u) {
            const int s = 13 + u;
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
            const int off = dx + NX * (dy + NY * dz);
            // forward block (n, n + o)
            if (i + dx >= 0 && i + dx < NX && j + dy >= 0 && j + dy < NY && k + dz < NZ) {
                const int m = n + off;
                const float v0 = a.xin[3 * m], v1 = a.xin[3 * m + 1], v2 = a.xin[3 * m + 2];
                const float* A = a.A + (long long)(u * 9) * nn + n;
                y0 = fmaf(A[0 * (long long)nn], v0, fmaf(A[1 * (long long)nn], v1, fmaf(A[2 * (long long)nn], v2, y0)));
                y1 = fmaf(A[3 * (long long)nn], v0, fmaf(A[4 * (long long)nn], v1, fmaf(A[5 * (long long)nn], v2, y1)));
                y2 = fmaf(A[6 * (long long)nn], v0, fmaf(A[7 * (long long)nn], v1, fmaf(A[8 * (long long)nn], v2, y2)));
            }
            // backward block (n, n - o) = block (n - o, n)^T
            if (u > 0 && i - dx >= 0 && i - dx < NX && j - dy >= 0 && j - dy < NY && k - dz >= 0) {
                const int m = n - off;
                const float v0 = a.xin[3 * m], v1 = a.xin[3 * m + 1], v2 = a.xin[3 * m + 2];
                const float* A = a.A + (long long)(u * 9) * nn + m;
                y0 = fmaf(A[0 * (long long)nn], v0, fmaf(A[3 * (long long)nn], v1, fmaf(A[6 * (long long)nn], v2, y0)));
                y1 = fmaf(A[1 * (long long)nn], v0, fmaf(A[4 * (long long)nn], v1, fmaf(A[7 * (long long)nn], v2, y1)));
                y2 = fmaf(A[2 * (long long)nn], v0, fmaf(A[5 * (long long)nn], v1, fmaf(A[8 * (long long)nn], v2, y2)));
            }
        }
        const uint8_t msk = a.mask[n];
        const float y[3] = {y0, y1, y2};
        if (MODE == FM_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = fixed_bit(msk, c) ? 0.f : y[c];
                a.out[3 * n + c] = v;
                if (DOT) dotv += (double)a.xin[3 * n + c] * (double)v;
            }
        } else if (MODE == FM_RESID) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                a.out[3 * n + c] = fixed_bit(msk, c) ? 0.f : a.b[3 * n + c] - y[c];
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
                    if (DOT) dotv += (double)bc * (double)xn;
                }
                a.out[3 * n + c] = xn;
                if (a.dnew) a.dnew[3 * n + c] = dn;
            }
        }
    }
    if (DOT) {
        const double s = block_sum<kVecThreads>(dotv, threadIdx.x);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
    }
}

__global__ void k_bsr_smooth0(BsrArgs a) {
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
__device__ __forceinline__ int fine_support(int I, int nf, int* idx, float* w) {
    const int nc = nf >> 1;
    int n = 0;
    idx[n] = 2 * I; w[n++] = 1.f;
    if (I >= 1) { idx[n] = 2 * I - 1; w[n++] = 0.5f; }
    const int f = 2 * I + 1;
    if (f <= nf) { idx[n] = f; w[n++] = (f < 2 * nc) ? 0.5f : 1.f; }
    return n;
}

__device__ __forceinline__ int coarse_parents(int f, int nf, int* idx, float* w) {
    const int nc = nf >> 1;
    if ((f & 1) == 0) { idx[0] = f >> 1; w[0] = 1.f; return 1; }
    if (f < 2 * nc) { idx[0] = (f - 1) >> 1; w[0] = 0.5f; idx[1] = (f + 1) >> 1; w[1] = 0.5f; return 2; }
    idx[0] = nc; w[0] = 1.f; return 1;
}

__global__ void k_restrict(int fnx, int fny, int fnz, int cnx, int cny, int cnz, const uint8_t* cmask,
                           const float* fine, float* coarse) {
    const long long CX = cnx + 1, CY = cny + 1, CZ = cnz + 1, nn = CX * CY * CZ;
    const long long FX = fnx + 1, FY = fny + 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
         n += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(n % CX), J = (int)((n / CX) % CY), K = (int)(n / (CX * CY));
        int ix[3], iy[3], iz[3];
        float wx[3], wy[3], wz[3];
        const int sx = fine_support(I, fnx, ix, wx), sy = fine_support(J, fny, iy, wy),
                  sz = fine_support(K, fnz, iz, wz);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int c = 0; c < sz; ++c)
            for (int b = 0; b < sy; ++b)
                for (int a = 0; a < sx; ++a) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const long long f = ix[a] + FX * (iy[b] + FY * iz[c]);
                    s0 = fmaf(w, fine[3 * f], s0);
                    s1 = fmaf(w, fine[3 * f + 1], s1);
                    s2 = fmaf(w, fine[3 * f + 2], s2);
                }
        const uint8_t m = cmask[n];
        coarse[3 * n] = fixed_bit(m, 0) ? 0.f : s0;
        coarse[3 * n + 1] = fixed_bit(m, 1) ? 0.f : s1;
        coarse[3 * n + 2] = fixed_bit(m, 2) ? 0.f : s2;
    }
}

__global__ void k_prolong_add(int fnx, int fny, int fnz, int cnx, int cny, const uint8_t* fmask,
                              const float* coarse, float* fine) {
    const long long FX = fnx + 1, FY = fny + 1, FZ = fnz + 1, nn = FX * FY * FZ;
    const long long CX = cnx + 1, CY = cny + 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % FX), j = (int)((n / FX) % FY), k = (int)(n / (FX * FY));
        int ix[2], iy[2], iz[2];
        float wx[2], wy[2], wz[2];
        const int sx = coarse_parents(i, fnx, ix, wx), sy = coarse_parents(j, fny, iy, wy),
                  sz = coarse_parents(k, fnz, iz, wz);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int c = 0; c < sz; ++c)
            for (int b = 0; b < sy; ++b)
                for (int a = 0; a < sx; ++a) {
                    const float w = wx[a] * wy[b] * wz[c];
                    const long long m = ix[a] + CX * (iy[b] + CY * iz[c]);
                    s0 = fmaf(w, coarse[3 * m], s0);
                    s1 = fmaf(w, coarse[3 * m + 1], s1);
                    s2 = fmaf(w, coarse[3 * m + 2], s2);
                }
        const uint8_t msk = fmask[n];
        if (!fixed_bit(msk, 0)) fine[3 * n] += s0;
        if (!fixed_bit(msk, 1)) fine[3 * n + 1] += s1;
        if (!fixed_bit(msk, 2)) fine[3 * n + 2] += s2;
    }
}

// x[free_idx[i]] = sum_j Ainv[i][j] b[free_idx[j]]  (FP64 accumulation, one warp per row)
__global__ void k_coarse_solve(int nL, const int* free_idx, const double* Ainv, const float* b, float* x) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nL) return;
    const double* row = Ainv + (long long)warp * nL;
    double s = 0.0;
    for (int jx = lane; jx < nL; jx += 32) s = fma(row[jx], (double)b[free_idx[jx]], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[free_idx[warp]] = (float)s;
}

// ---------------------------------------------------------------------------
// Vector kernels (grid-stride over a fixed grid, so the partial layout and the
// summation order are independent of timing).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads) k_dot_f32(const float* a, const float* b, long long n, double* partial) {
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < n; q += (long long)gridDim.x * kVecThreads)
        s += (double)a[q] * (double)b[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_dot_f64_masked(const double* a, const double* b, const uint8_t* mask,
                                                                long long nn, double* partial) {
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * kVecThreads)
        if (!fixed_bit(mask[q / 3], (int)(q % 3))) s += a[q] * b[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_finalize(const double* partial, int n, double* sc, int slot, int op) {
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

__global__ void __launch_bounds__(kVecThreads) k_pcg_update(double* u, float* r, const float* p, const float* q, long long n,
                                                            const double* sc, double* partial) {
    const double alpha = sc[SC_ALPHA];
    const float af = (float)alpha;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)kVecThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kVecThreads) {
        u[i] = fma(alpha, (double)p[i], u[i]);
        const float rn = fmaf(-af, q[i], r[i]);
        r[i] = rn;
        s += (double)rn * (double)rn;
    }
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_p_update(float* p, const float* z, long long n, const double* sc) {
    const float beta = (float)sc[SC_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(kVecThreads) k_mask_u64(double* u, const uint8_t* mask, long long nn, double* partial) {
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * kVecThreads) {
        if (fixed_bit(mask[q / 3], (int)(q % 3))) u[q] = 0.0;
        else if (u[q] != 0.0) s += 1.0;
    }
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_scale_inv_sqrt(float* v, long long n, const double* sc, int slot) {
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
                                     int nz, float kd) {
    const long long NX = nx + 1, NY = ny + 1, nn = NX * NY * (nz + 1);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        const float inv = 1.f / fine_diag(E, nx, ny, nz, i, j, k, kd);
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) w[3 * n + c] = fixed_bit(m, c) ? 0.f : inv * y[3 * n + c];
    }
}

__global__ void k_scale_invdiag_bsr(const float* y, float* w, const float* invdiag, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        w[q] = invdiag[q] * y[q];
}

__global__ void __launch_bounds__(kVecThreads) k_diag_dot_fine(const float* v, const float* E, const uint8_t* mask, int nx,
                                                               int ny, int nz, float kd, double* partial) {
    const long long NX = nx + 1, NY = ny + 1, nn = NX * NY * (nz + 1);
    double s = 0.0;
    for (long long n = blockIdx.x * (long long)kVecThreads + threadIdx.x; n < nn; n += (long long)gridDim.x * kVecThreads) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        const double dg = fine_diag(E, nx, ny, nz, i, j, k, kd);
        const uint8_t m = mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (!fixed_bit(m, c)) s += dg * (double)v[3 * n + c] * (double)v[3 * n + c];
    }
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_diag_dot_bsr(const float* v, const float* invdiag, long long n, double* partial) {
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)kVecThreads + threadIdx.x; q < n; q += (long long)gridDim.x * kVecThreads)
        if (invdiag[q] != 0.f) s += (double)v[q] * (double)v[q] / (double)invdiag[q];
    s = block_sum<kVecThreads>(s, threadIdx.x);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Power-iteration start vector: v_i = ((i * 2654435761) mod 2^32) / 2^32 - 0.5 over
// the level's DOF index i, 0 on fixed DOFs.
__global__ void k_power_start(float* v, const uint8_t* mask, long long nn) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h = ((unsigned long long)q * 2654435761ull) & 0xffffffffull;
        const double val = (double)h / 4294967296.0 - 0.5;
        v[q] = fixed_bit(mask[q / 3], (int)(q % 3)) ? 0.f : (float)val;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_fine_smooth0(const FineArgs& a, cudaStream_t s) {
    note_launch();
    k_fine_smooth0<<<kVecBlocks * 2, kVecThreads, 0, s>>>(a);
}

int bsr_grid_blocks(long long nn) { return (int)((nn + kVecThreads - 1) / kVecThreads); }

void launch_bsr(int mode, int dot, const BsrArgs& a, cudaStream_t s) {
    const int g = bsr_grid_blocks(a.nn);
    if (mode == FM_APPLY) {
        if (dot) { note_launch(); k_bsr<FM_APPLY, true><<<g, kVecThreads, 0, s>>>(a); }
        else { note_launch(); k_bsr<FM_APPLY, false><<<g, kVecThreads, 0, s>>>(a); }
    } else if (mode == FM_SMOOTH) {
        if (dot) { note_launch(); k_bsr<FM_SMOOTH, true><<<g, kVecThreads, 0, s>>>(a); }
        else { note_launch(); k_bsr<FM_SMOOTH, false><<<g, kVecThreads, 0, s>>>(a); }
    } else {
        note_launch();
        k_bsr<FM_RESID, false><<<g, kVecThreads, 0, s>>>(a);
    }
}

void launch_bsr_smooth0(const BsrArgs& a, cudaStream_t s) {
    const long long n3 = 3 * a.nn;
    const int g = (int)std::min<long long>((n3 + kVecThreads - 1) / kVecThreads, kVecBlocks * 2);
    note_launch();
    k_bsr_smooth0<<<g, kVecThreads, 0, s>>>(a);
}

static int grid_for(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, kVecBlocks * 2));
}

void launch_restrict(const Level& f, const Level& c, const float* fine, float* coarse, cudaStream_t s) {
    note_launch();
    k_restrict<<<grid_for(c.nn), 256, 0, s>>>(f.nx, f.ny, f.nz, c.nx, c.ny, c.nz, c.mask, fine, coarse);
}

void launch_prolong_add(const Level& f, const Level& c, const float* coarse, float* fine, cudaStream_t s) {
    note_launch();
    k_prolong_add<<<grid_for(f.nn), 256, 0, s>>>(f.nx, f.ny, f.nz, c.nx, c.ny, f.mask, coarse, fine);
}

void launch_coarse_solve(int nL, const int* free_idx, const double* Ainv, const float* b, float* x,
                         long long n_dof, cudaStream_t s) {
    cudaMemsetAsync(x, 0, sizeof(float) * n_dof, s);
    if (nL > 0) { note_launch(); k_coarse_solve<<<(nL * 32 + 255) / 256, 256, 0, s>>>(nL, free_idx, Ainv, b, x); }
}

int vec_grid_blocks() { return kVecBlocks; }

void launch_dot_f32(const float* a, const float* b, long long n, double* partial, cudaStream_t s) {
    note_launch();
    k_dot_f32<<<kVecBlocks, kVecThreads, 0, s>>>(a, b, n, partial);
}

void launch_dot_f64_masked(const double* a, const double* b, const uint8_t* mask, long long nn, double* partial,
                           cudaStream_t s) {
    note_launch();
    k_dot_f64_masked<<<kVecBlocks, kVecThreads, 0, s>>>(a, b, mask, nn, partial);
}

void launch_finalize(const double* partial, int n, double* sc, int slot, int op, cudaStream_t s) {
    note_launch();
    k_finalize<<<1, kVecThreads, 0, s>>>(partial, n, sc, slot, op);
}

void launch_pcg_update(double* u, float* r, const float* p, const float* q, long long n, const double* sc,
                       double* partial, cudaStream_t s) {
    note_launch();
    k_pcg_update<<<kVecBlocks, kVecThreads, 0, s>>>(u, r, p, q, n, sc, partial);
}

void launch_p_update(float* p, const float* z, long long n, const double* sc, cudaStream_t s) {
    note_launch();
    k_p_update<<<grid_for(n), 256, 0, s>>>(p, z, n, sc);
}

void launch_mask_u64(double* u, const uint8_t* mask, long long nn, double* partial, cudaStream_t s) {
    note_launch();
    k_mask_u64<<<kVecBlocks, kVecThreads, 0, s>>>(u, mask, nn, partial);
}

void launch_scale_by_inv_sqrt(float* v, long long n, const double* sc, int slot, cudaStream_t s) {
    note_launch();
    k_scale_inv_sqrt<<<grid_for(n), 256, 0, s>>>(v, n, sc, slot);
}

void launch_scale_invdiag_fine(const float* y, float* w, const float* E, const uint8_t* mask, int nx, int ny,
                               int nz, float kd, cudaStream_t s) {
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    note_launch();
    k_scale_invdiag_fine<<<grid_for(nn), 256, 0, s>>>(y, w, E, mask, nx, ny, nz, kd);
}

void launch_scale_invdiag_bsr(const float* y, float* w, const float* invdiag, long long n, cudaStream_t s) {
    note_launch();
    k_scale_invdiag_bsr<<<grid_for(n), 256, 0, s>>>(y, w, invdiag, n);
}

void launch_diag_dot_fine(const float* v, const float* E, const uint8_t* mask, int nx, int ny, int nz, float kd,
                          double* partial, cudaStream_t s) {
    note_launch();
    k_diag_dot_fine<<<kVecBlocks, kVecThreads, 0, s>>>(v, E, mask, nx, ny, nz, kd, partial);
}

void launch_diag_dot_bsr(const float* v, const float* invdiag, long long n, double* partial, cudaStream_t s) {
    note_launch();
    k_diag_dot_bsr<<<kVecBlocks, kVecThreads, 0, s>>>(v, invdiag, n, partial);
}

void launch_power_start(float* v, const uint8_t* mask, long long nn, cudaStream_t s) {
    note_launch();
    k_power_start<<<grid_for(3 * nn), 256, 0, s>>>(v, mask, nn);
}

}  // namespace gmg
